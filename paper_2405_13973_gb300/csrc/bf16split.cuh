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

// the pieces of M[cell][k] into Mp[(cell * 3 + q) * ld + k], q = hi, mid, lo
__device__ __forceinline__ void store_pieces(uint16_t* Mp, int64_t cell, int ld, int k, float v) {
    uint32_t h, m, l;
    split_bf16x3(v, h, m, l);
    uint16_t* row = Mp + cell * 3 * ld + k;
    row[0] = (uint16_t)h;
    row[ld] = (uint16_t)m;
    row[2 * ld] = (uint16_t)l;
}

}  // namespace pt
