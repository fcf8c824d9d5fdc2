// bf16split.cuh -- the split of an FP32 value into three bf16 pieces used by
// the BF16x3 tensor-core products (device code).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace pt {

// x = hi + mid + lo, each round-to-nearest bf16 of the remainder so far (an
// FP32 value exactly: 3 x 8 significant bits cover its 24)
__device__ __forceinline__ void split_bf16x3(float x, uint32_t& h, uint32_t& m, uint32_t& l) {
    const __nv_bfloat16 bh = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(bh);
    const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(bm);
    const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(bl);
}

// Rows of bf16 pieces per cell: hi, mid, lo of M, then hi, mid, lo of the
// mirrored multipole (-1)^n M_n^m, n the degree of coefficient k.  The
// mirrored rows serve the pairs of offset -o in a product with the operator
// of +o: the irregular harmonics are odd or even in their argument with
// their degree, Th_n^m(-o) = (-1)^n Th_n^m(o), so the M2L operator of Eq.
// FMM_local obeys T_{-o}[l][j] = (-1)^(j + l) T_o[l][j], and the partial
// local expansion of a mirrored pair is T_o applied to the mirrored M with
// the odd-degree outputs negated.  Negation is exact and the split below is
// odd in x, so the mirrored rows are the pieces of -M where n is odd.
constexpr int kPieceRows = 6;

// degree n of real storage index k (k in [n^2, (n+1)^2))
__device__ __forceinline__ int coef_degree(int k) {
    int n = (int)sqrtf((float)k);
    if ((n + 1) * (n + 1) <= k) ++n;
    if (n * n > k) --n;
    return n;
}

// the pieces of M[cell][k] into Mp[(cell * kPieceRows + q) * ld + k], q =
// hi, mid, lo, and their mirrored copies at q + 3
__device__ __forceinline__ void store_pieces(uint16_t* Mp, int64_t cell, int ld, int k, float v) {
    uint32_t h, m, l;
    split_bf16x3(v, h, m, l);
    uint16_t* row = Mp + cell * kPieceRows * ld + k;
    const uint32_t flip = (coef_degree(k) & 1) ? 0x8000u : 0u;
    row[0] = (uint16_t)h;
    row[ld] = (uint16_t)m;
    row[2 * ld] = (uint16_t)l;
    row[3 * ld] = (uint16_t)(h ^ flip);
    row[4 * ld] = (uint16_t)(m ^ flip);
    row[5 * ld] = (uint16_t)(l ^ flip);
}

}  // namespace pt
