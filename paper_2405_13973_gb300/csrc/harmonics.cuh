// harmonics.cuh -- Morton codes and normalised regular solid harmonics,
// usable on host and device.
//
// Solid harmonics (Sec. 2.3.1, Eq. FMM_coul): with P_n^m the associated
// Legendre functions without the Condon-Shortley phase,
//   Y_n^m(r)  = r^n P_n^m(cos t) e^{i m f} / (n+m)!        (regular)
//   Th_n^m(r) = (n-m)! P_n^m(cos t) e^{i m f} / r^{n+1}    (irregular)
//   X_n^{-m}  = (-1)^m conj(X_n^m),
// which satisfy 1/|x-y| = sum conj(Y_n^m(y)) Th_n^m(x) for |y| < |x|.
// Multipole: M_n^m = sum_i q_i conj(Y_n^m(x_i - c)) so phi = sum M Th(x - c);
// local: phi(x) = sum L_n^m conj(Y_n^m(x - c)).
//
// Every coefficient is stored normalised by s_nm = sqrt((n+m)!(n-m)!):
// M^ = s M, L^ = L / s, Y^ = s Y.  |Y^_n^m(u)| <= |u|^n, so FP32 and TF32
// keep every coefficient within a few orders of magnitude.  Real storage of
// the (p+1)^2 coefficients of one cell: index n^2 holds Re X_n^0, n^2+2m-1
// holds Re X_n^m and n^2+2m holds Im X_n^m (m = 1..n); X_n^{-m} follows from
// the symmetry.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define PT_HD __host__ __device__ __forceinline__
#else
#define PT_HD inline
#endif

namespace pt {

PT_HD uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
PT_HD uint32_t compact3(uint32_t v) {
    v &= 0x09249249u;
    v = (v ^ (v >> 2)) & 0x030C30C3u;
    v = (v ^ (v >> 4)) & 0x0300F00Fu;
    v = (v ^ (v >> 8)) & 0x030000FFu;
    v = (v ^ (v >> 16)) & 0x000003FFu;
    return v;
}
// Morton code with ix the most significant bit of each triple.
PT_HD uint32_t morton3(uint32_t ix, uint32_t iy, uint32_t iz) {
    return (spread3(ix) << 2) | (spread3(iy) << 1) | spread3(iz);
}
PT_HD void demorton3(uint32_t c, int& ix, int& iy, int& iz) {
    ix = (int)compact3(c >> 2);
    iy = (int)compact3(c >> 1);
    iz = (int)compact3(c);
}

PT_HD int re_idx(int n, int m) { return n * n + (m == 0 ? 0 : 2 * m - 1); }

// Recurrence and gradient coefficient tables for n, m <= kTab - 1.
constexpr int kTab = 18;
template <typename T>
struct HarmTables {
    T a[kTab][kTab];   // (2n-1)/sqrt((n+m)(n-m))
    T b[kTab][kTab];   // sqrt((n+m-1)(n-m-1)/((n+m)(n-m)))
    T c[kTab];         // sqrt((2m-1)/(2m))      diagonal step
    T d[kTab];         // sqrt(2m+1)             first off-diagonal
    T e[kTab][kTab];   // sqrt((n+m+1)(n-m+1))   d/dz factor
    T f[kTab][kTab];   // sqrt((n+m+2)(n+m+1))   (d/dx + i d/dy), m -> m+1 term
    T g[kTab][kTab];   // sqrt((n-m+2)(n-m+1))   (d/dx + i d/dy), m -> m-1 term
};

template <typename T>
inline void fill_harm_tables(HarmTables<T>& t);

}  // namespace pt

#ifndef __CUDACC__
#include <cmath>
#endif
#include <math.h>
namespace pt {
template <typename T>
inline void fill_harm_tables(HarmTables<T>& t) {
    for (int n = 0; n < kTab; ++n)
        for (int m = 0; m < kTab; ++m) {
            double a = 0, b = 0;
            if (n >= m + 2) {
                double nm = (double)(n + m) * (double)(n - m);
                a = (2.0 * n - 1.0) / sqrt(nm);
                b = sqrt((double)(n + m - 1) * (double)(n - m - 1) / nm);
            }
            t.a[n][m] = (T)a;
            t.b[n][m] = (T)b;
            t.e[n][m] = (T)(m <= n ? sqrt((double)(n + m + 1) * (double)(n - m + 1)) : 0.0);
            t.f[n][m] = (T)(m <= n ? sqrt((double)(n + m + 2) * (double)(n + m + 1)) : 0.0);
            t.g[n][m] = (T)(m <= n ? sqrt((double)(n - m + 2) * (double)(n - m + 1)) : 0.0);
        }
    for (int m = 0; m < kTab; ++m) {
        t.c[m] = (T)(m == 0 ? 1.0 : sqrt((2.0 * m - 1.0) / (2.0 * m)));
        t.d[m] = (T)sqrt(2.0 * m + 1.0);
    }
}
}  // namespace pt
