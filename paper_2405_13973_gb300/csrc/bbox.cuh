// bbox.cuh -- reduction of the ions' bounding box and last-block
// finalisation of the octree root cube (Sec. 2.3.2: the smallest cube that
// contains all ions).  Shared by the tree build and the fused drift kernel.
//
// The extremes are reduced as integers: a double maps to a 64-bit key whose
// unsigned order is the numeric order (sign bit set for x >= 0, all bits
// flipped for x < 0), so a warp reduces with shuffles and integer compares,
// and each warp folds its result into an 8-word accumulator in global memory
// by atomicMax (the minimum is kept as the maximum of the complemented key,
// so the identity of every word is 0).  The last block to finish reads and
// clears the accumulator in one atomicExch per word and writes the cube.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace pt {

constexpr int kBboxWords = 8;  // [0..2] ~key of the minimum, [3..5] key of the maximum, [6] bad
constexpr int kBboxThreads = 128;

// blocks of a bounding-box pass over n points: equal shares over the SMs
// (ion_split), at most bbox_blocks (each block folds into the accumulator
// with a few atomics)
inline IonSplit bbox_split(int64_t n, const Workspace& ws) {
    return ion_split(n, kBboxThreads, ws.sms, ws.bbox_blocks);
}

__device__ __forceinline__ unsigned long long ord_key(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_val(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// per-thread extremes of the points it saw
struct BboxAcc {
    unsigned long long k[6] = {0, 0, 0, 0, 0, 0};
    int bad = 0;
    __device__ __forceinline__ void add(double x, double y, double z) {
        const double p[3] = {x, y, z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bad |= !isfinite(p[a]);
            const unsigned long long key = ord_key(p[a]);
            k[a] = umax64(k[a], ~key);
            k[3 + a] = umax64(k[3 + a], key);
        }
    }
};

// Folds every thread's extremes into acc[] (all threads of the block call
// it); the last block writes the root cube exactly as
//   side = max_a (max_a - min_a) (1 if zero); lo_a = (min_a+max_a)/2 - side/2
// and clears acc[] and the ticket.  Returns true in the one thread that
// finalised the cube.
__device__ __forceinline__ bool bbox_commit(BboxAcc& t, unsigned long long* acc, unsigned* ticket,
                                            RootCube* root, int* err) {
    __shared__ bool last;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 0; w < 6; ++w)
        for (int o = 16; o > 0; o >>= 1) t.k[w] = umax64(t.k[w], __shfl_xor_sync(0xffffffffu, t.k[w], o));
    const int wb = __any_sync(0xffffffffu, t.bad);
    if (lane == 0) {
#pragma unroll
        for (int w = 0; w < 6; ++w)
            if (t.k[w] != 0ull) atomicMax(&acc[w], t.k[w]);
        if (wb) atomicOr(&acc[6], 1ull);
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned tk = atomicAdd(ticket, 1u);
        last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return false;
    __threadfence();
    unsigned long long v[7];
#pragma unroll
    for (int w = 0; w < 7; ++w) v[w] = atomicExch(&acc[w], 0ull);
    double u[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        u[a] = ord_val(~v[a]);
        hi[a] = ord_val(v[3 + a]);
    }
    const bool b = v[6] != 0ull;
    if (v[0] == 0ull)  // no point at all: the unit cube at the origin
        for (int a = 0; a < 3; ++a) u[a] = hi[a] = 0.0;
    double side = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = __dsub_rn(hi[a], u[a]);
        if (e > side) side = e;
    }
    if (!(side > 0.0)) side = 1.0;
    if (b || !isfinite(side)) {
        atomicOr(err, ERR_NONFINITE);
        side = 1.0;
        for (int a = 0; a < 3; ++a) u[a] = hi[a] = 0.0;
    }
    for (int a = 0; a < 3; ++a)
        root->lo[a] = __dsub_rn(__dmul_rn(0.5, __dadd_rn(u[a], hi[a])), __dmul_rn(0.5, side));
    root->side = side;
    *ticket = 0u;
    return true;
}

}  // namespace pt
