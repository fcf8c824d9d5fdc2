// bbox.cuh -- block reduction of the ions' bounding box and last-block
// finalisation of the octree root cube (Sec. 2.3.2: the smallest cube that
// contains all ions).  Shared by the tree build and the fused drift kernel.
// Returns true in the one thread that finalised the cube.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace pt {

__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Reduces the block's min/max into partial[blockIdx.x]; the last block to
// finish combines all partials and writes the root cube exactly as
//   side = max_a (max_a - min_a) (1 if zero); lo_a = (min_a+max_a)/2 - side/2.
__device__ __forceinline__ bool bbox_block_and_finalise(double mn[3], double mx[3], int bad, double* partial,
                                        unsigned* ticket, RootCube* root, int* err) {
    __shared__ double smn[3][32], smx[3][32];
    __shared__ int sbad[32];
    __shared__ bool last;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int a = 0; a < 3; ++a) {
        double a0 = warp_min(mn[a]), a1 = warp_max(mx[a]);
        if (lane == 0) { smn[a][wid] = a0; smx[a][wid] = a1; }
    }
    int wb = __any_sync(0xffffffffu, bad);
    if (lane == 0) sbad[wid] = wb;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[7];
        for (int a = 0; a < 3; ++a) {
            double u = smn[a][0], v = smx[a][0];
            for (int w = 1; w < nw; ++w) { u = fmin(u, smn[a][w]); v = fmax(v, smx[a][w]); }
            r[a] = u;
            r[3 + a] = v;
        }
        int b = 0;
        for (int w = 0; w < nw; ++w) b |= sbad[w];
        for (int k = 0; k < 6; ++k) partial[blockIdx.x * 8 + k] = r[k];
        partial[blockIdx.x * 8 + 6] = (double)b;
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // the last block combines every block's partial, all threads in parallel
    double u[3], v[3];
    int b = 0;
    for (int a = 0; a < 3; ++a) { u[a] = INFINITY; v[a] = -INFINITY; }
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
        const volatile double* pp = partial + k * 8;
        for (int a = 0; a < 3; ++a) { u[a] = fmin(u[a], pp[a]); v[a] = fmax(v[a], pp[3 + a]); }
        b |= (pp[6] != 0.0);
    }
    for (int a = 0; a < 3; ++a) {
        double a0 = warp_min(u[a]), a1 = warp_max(v[a]);
        if (lane == 0) { smn[a][wid] = a0; smx[a][wid] = a1; }
    }
    int wb2 = __any_sync(0xffffffffu, b);
    __syncthreads();
    if (lane == 0) sbad[wid] = wb2;
    __syncthreads();
    if (threadIdx.x != 0) return false;
    for (int a = 0; a < 3; ++a) {
        u[a] = smn[a][0];
        v[a] = smx[a][0];
        for (int w = 1; w < nw; ++w) { u[a] = fmin(u[a], smn[a][w]); v[a] = fmax(v[a], smx[a][w]); }
    }
    b = 0;
    for (int w = 0; w < nw; ++w) b |= sbad[w];
    double side = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = __dsub_rn(v[a], u[a]);
        if (e > side) side = e;
    }
    if (!(side > 0.0)) side = 1.0;
    if (b || !isfinite(side)) {
        atomicOr(err, ERR_NONFINITE);
        side = 1.0;
        for (int a = 0; a < 3; ++a) { u[a] = 0.0; v[a] = 0.0; }
    }
    for (int a = 0; a < 3; ++a)
        root->lo[a] = __dsub_rn(__dmul_rn(0.5, __dadd_rn(u[a], v[a])), __dmul_rn(0.5, side));
    root->side = side;
    *ticket = 0u;
    return true;
}

}  // namespace pt
