// rng.cuh -- counter-based random numbers and the exponential shared by the
// push (photon kicks) and the Metropolis-Hastings initialisation, FP64.
//
// Translation units that include this are compiled with -fmad=false: every
// expression is the literal sequence of IEEE double operations written, so
// that the draws and the accept/kick decisions fed by them are
// bit-reproducible definitions.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// exp: Cody-Waite reduction with ln2 split into a 40-bit head and a tail,
// degree-13 Taylor polynomial by Horner, scaling by 2^k through the exponent
// bits (two steps below the normal range).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pt {

constexpr int kMaxPhotons = 64;
constexpr int kMaxTries = 64;

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

__device__ __forceinline__ double u01(uint32_t a, uint32_t b) {
    uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return (double)k * 0x1.0p-53;
}

__device__ __forceinline__ void stream_block(uint64_t seed, int64_t step, int64_t ion, int beam,
                                             uint32_t slot, uint32_t out[4]) {
    uint64_t st = (uint64_t)step;
    philox4x32_10((uint32_t)ion, (uint32_t)beam | (slot << 8), (uint32_t)st, (uint32_t)(st >> 32),
                  (uint32_t)seed, (uint32_t)(seed >> 32), out);
}

__device__ __forceinline__ double pt_exp(double x) {
    const double LN2_HI = 0x1.62e42fefa2000p-1;
    const double LN2_LO = 0x1.9ef35793c7673p-41;
    const double INV_LN2 = 0x1.71547652b82fep+0;
    if (x != x) return x;
    if (x > 709.8) return INFINITY;
    if (x < -745.2) return 0.0;
    double kf = floor(x * INV_LN2 + 0.5);
    double r = (x - kf * LN2_HI) - kf * LN2_LO;
    // Taylor coefficients 1/j! (every j! <= 13! is exact in double, so each
    // constant is the correctly rounded quotient)
    const double c[14] = {1.0, 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0,
                          1.0 / 5040.0, 1.0 / 40320.0, 1.0 / 362880.0, 1.0 / 3628800.0,
                          1.0 / 39916800.0, 1.0 / 479001600.0, 1.0 / 6227020800.0};
    double p = c[13];
#pragma unroll
    for (int j = 12; j >= 0; --j) p = p * r + c[j];
    int k = (int)kf;
    if (k >= -1022) return p * __longlong_as_double((long long)(k + 1023) << 52);
    return (p * __longlong_as_double((long long)(k + 600 + 1023) << 52)) *
           __longlong_as_double((long long)(-600 + 1023) << 52);
}

}  // namespace pt
