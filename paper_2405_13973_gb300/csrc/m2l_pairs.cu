// m2l_pairs.cu -- the pair-packed M2L schedule (see m2l_pairs.h): its work
// list, the per-target reduction of the partial rows, the CUDA-core M2L
// product of every work item (FP64 and FP32 paths) and the CUDA-core L2L
// shifts that follow it.
//
// Work list, per step (reads the tree only):
//   k_pp_count  one warp per target: presence of its 216 candidate offsets
//               (the 189 of its octant plus the 27 neighbours, always
//               absent), its pair count and the per-offset counts;
//   k_pp_scan   one block: target slot bases, offset pair bases, the items
//               (each offset's pairs in runs of kPairRows, offsets in
//               increasing order) and the pool check;
//   k_pp_fill   one warp per target: its pairs, each at the next position of
//               its offset's list, with their sources and slots.
// With mirroring (BF16x3), offsets o and -o count, and fill, as one: the
// pairs of -o (operator index above 171) go to the list of o, marked.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "bf16split.cuh"
#include "harmonics.cuh"
#include "m2l_pairs.h"

namespace pt {

namespace {

struct PpArgs {
    int D;
    int mirror;  // pairs of -o in the runs of o (kPairMirror)
    const LevelInfo* linfo;
    const uint32_t* code;
    const int32_t* cid;
    int64_t off[kMaxDepth + 2];
};

__device__ __forceinline__ void stage_linfo(const LevelInfo* g, LevelInfo* s) {
    const int* src = reinterpret_cast<const int*>(g);
    int* dst = reinterpret_cast<int*>(s);
    for (int i = threadIdx.x; i < (int)(sizeof(LevelInfo) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
}

// Targets are the cells of levels 2..D (global ids gbase[2] .. gbase[D+1]),
// t = g - gbase[2].  Candidate offsets of a target in child octant b are the
// 216 offsets o with o_a in [b_a - 3, b_a + 2] (index c = 36 (o_x - b_x + 3)
// + 6 (o_y - b_y + 3) + (o_z - b_z + 3), increasing with the operator index
// (o_x+3)*49 + (o_y+3)*7 + (o_z+3)); the 27 with |o_a| <= 1 are neighbours.
// A candidate is present when its source cell t - o holds ions.
constexpr int kPpCand = 216;
constexpr int kPpWords = 7;   // 32-bit presence words per target

__device__ __forceinline__ int pp_level(const LevelInfo& li, int D, int g) {
    int l = 2;
    while (l < D && g >= li.gbase[l + 1]) ++l;
    return l;
}

// source of candidate c of the target at (x, y, z) of level l, or -1
__device__ __forceinline__ int pp_source(const PpArgs& a, int l, int x, int y, int z, int c,
                                         int* op) {
    const int ox = (x & 1) - 3 + c / 36, oy = (y & 1) - 3 + (c / 6) % 6, oz = (z & 1) - 3 + c % 6;
    *op = (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3);
    if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) return -1;
    const int sx = x - ox, sy = y - oy, sz = z - oz, lim = 1 << l;
    if (sx < 0 || sy < 0 || sz < 0 || sx >= lim || sy >= lim || sz >= lim) return -1;
    return a.cid[a.off[l] + morton3(sx, sy, sz)];
}

// One warp per target: presence words of its 216 candidates, its pair count,
// and the per-offset pair counts (block histogram, then global).
constexpr int kPpThreads = 256;
__global__ void __launch_bounds__(kPpThreads) k_pp_count(PpArgs a, uint32_t* tmask, int* tcount,
                                                         int* ocnt) {
    __shared__ int hist[343];
    __shared__ LevelInfo li;
    stage_linfo(a.linfo, &li);
    for (int i = threadIdx.x; i < 343; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int g0 = li.gbase[2], g1 = li.gbase[a.D + 1];
    const int wpb = blockDim.x >> 5;
    for (int g = g0 + blockIdx.x * wpb + (threadIdx.x >> 5); g < g1; g += gridDim.x * wpb) {
        const int l = pp_level(li, a.D, g);
        int x, y, z;
        demorton3(a.code[g], x, y, z);
        int cnt = 0;
#pragma unroll
        for (int w = 0; w < kPpWords; ++w) {
            const int c = 32 * w + lane;
            int op = 0, src = -1;
            if (c < kPpCand) src = pp_source(a, l, x, y, z, c, &op);
            const unsigned bal = __ballot_sync(0xffffffffu, src >= 0);
            if (src >= 0) atomicAdd(&hist[a.mirror && op > 171 ? 342 - op : op], 1);
            if (lane == 0) tmask[(int64_t)(g - g0) * kPpWords + w] = bal;
            cnt += __popc(bal);
        }
        if (lane == 0) tcount[g - g0] = cnt;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 343; i += blockDim.x)
        if (hist[i]) atomicAdd(&ocnt[i], hist[i]);
}

// One block: slot bases of the targets (exclusive scan of their counts; tbase
// has n_targets + 1 entries), pair bases of the offsets, and the work items
// (each offset's pairs in runs of 128, offsets in increasing order).
constexpr int kPpScanThreads = 1024;
__global__ void __launch_bounds__(kPpScanThreads) k_pp_scan(int D, const LevelInfo* linfo,
                                                             int64_t slot_cap, int64_t rows_cap,
                                                             int item_cap,
                                                             const int* tcount, int* tbase,
                                                             int* ocnt, int* ofill, int* obase,
                                                             M2lPairHdr* hdr, M2lPairHdr* host_hdr,
                                                             M2lPairItem* items, int* err) {
    pdl_wait();
    __shared__ int wsum[32];
    __shared__ int s_carry;
    __shared__ int s_ibase[344];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nt = linfo->gbase[D + 1] - linfo->gbase[2];
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nt; c0 += kPpScanThreads) {
        const int i = c0 + tid;
        const int v = i < nt ? tcount[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        if (i < nt) tbase[i] = s_carry + (wid > 0 ? wsum[wid - 1] : 0) + x - v;
        __syncthreads();
        if (tid == 0) s_carry += wsum[31];
        __syncthreads();
    }
    const int total = s_carry;
    // offsets: pair bases (scan of the counts) and item bases (scan of the
    // 128-pair runs), 343 entries by the first 11 warps
    __shared__ int s_pb[344], s_nof;
    if (wid < 11) {
        const int o = tid;  // 0 .. 351
        const int c = o < 343 ? ocnt[o] : 0;
        const int runs = (c + kPairRows - 1) / kPairRows;
        // each offset's pairs start on a multiple of 128 rows, so that every
        // work item covers whole 128-row blocks of the partial array
        int x = runs * kPairRows, y = runs, f = c > 0 ? 1 : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const int xa = __shfl_up_sync(0xffffffffu, x, d);
            const int ya = __shfl_up_sync(0xffffffffu, y, d);
            const int fa = __shfl_up_sync(0xffffffffu, f, d);
            if (lane >= d) {
                x += xa;
                y += ya;
                f += fa;
            }
        }
        if (o < 343) {
            s_pb[o + 1] = x;         // inclusive, per warp for now
            s_ibase[o + 1] = y;
        }
        if (lane == 31) wsum[wid] = f;
    }
    __syncthreads();
    __shared__ int s_cx[11], s_cy[11];
    if (tid == 0) {
        // carries of the 11 per-warp inclusive scans
        int cx = 0, cy = 0, nof = 0;
        for (int w = 0; w < 11; ++w) {
            const int last = min(32 * w + 31, 342);
            s_cx[w] = cx;
            s_cy[w] = cy;
            cx += s_pb[last + 1];
            cy += s_ibase[last + 1];
            nof += wsum[w];
        }
        s_nof = nof;
    }
    __syncthreads();
    if (tid < 343) {
        s_pb[tid + 1] += s_cx[tid >> 5];
        s_ibase[tid + 1] += s_cy[tid >> 5];
    }
    if (tid == 0) {
        s_pb[0] = 0;
        s_ibase[0] = 0;
    }
    __syncthreads();
    for (int o = tid; o <= 343; o += kPpScanThreads) obase[o] = s_pb[o];
    if (tid == 0) {
        tbase[nt] = total;
        const int pb = s_pb[343], ib = s_ibase[343];
        const bool over = (int64_t)total > slot_cap || (int64_t)pb > rows_cap || ib > item_cap;
        hdr->overflow = over ? 1 : 0;
        if (over) atomicOr(err, ERR_CAPACITY);
        hdr->n_items = over ? 0 : ib;
        hdr->n_pairs = total;
        hdr->n_targets = nt;
        hdr->n_offsets = s_nof;
        // the header also to pinned host memory, for the host's pool check
        // at the next call (no copy node)
        if (host_hdr) {
            volatile int* h = reinterpret_cast<volatile int*>(host_hdr);
            h[0] = hdr->n_items;
            h[1] = hdr->n_pairs;
            h[2] = hdr->n_targets;
            h[3] = hdr->overflow;
            h[4] = hdr->n_offsets;
        }
    }
    __syncthreads();
    const bool over =
        (int64_t)total > slot_cap || (int64_t)s_pb[343] > rows_cap || s_ibase[343] > item_cap;
    for (int o = tid; o < 344; o += kPpScanThreads) {
        const int c = o < 343 ? ocnt[o] : 0;
        for (int k = 0; !over && k * kPairRows < c; ++k) {
            M2lPairItem it;
            it.op = o;
            it.begin = s_pb[o] + k * kPairRows;
            it.rows = min(kPairRows, c - k * kPairRows);
            it.pad = 0;
            items[s_ibase[o] + k] = it;
        }
        // counts read: zero them and the fill counters for the next work
        // list (zeroed once at allocation)
        ocnt[o] = 0;
        ofill[o] = 0;
    }
}

// One warp per target: each present offset takes the next position of that
// offset's list (an atomic counter: the order of the pairs inside an
// offset's list does not change any result, every product row being
// computed alone), with its source and its slot (the target's slot base plus
// the rank of the offset among the target's present ones).
__global__ void __launch_bounds__(kPpThreads) k_pp_fill(PpArgs a, const uint32_t* tmask,
                                                         const int* tbase, const int* obase,
                                                         int* ofill, const M2lPairHdr* hdr,
                                                         M2lPair* pairs, int* tpair) {
    pdl_wait();
    __shared__ LevelInfo li;
    stage_linfo(a.linfo, &li);
    __syncthreads();
    if (hdr->overflow) return;
    const int lane = threadIdx.x & 31;
    const int g0 = li.gbase[2], g1 = li.gbase[a.D + 1];
    const int wpb = blockDim.x >> 5;
    for (int g = g0 + blockIdx.x * wpb + (threadIdx.x >> 5); g < g1; g += gridDim.x * wpb) {
        const int t = g - g0;
        const int l = pp_level(li, a.D, g);
        int x, y, z;
        demorton3(a.code[g], x, y, z);
        int rank = tbase[t];
#pragma unroll
        for (int w = 0; w < kPpWords; ++w) {
            const uint32_t bits = tmask[(int64_t)t * kPpWords + w];
            if ((bits >> lane) & 1u) {
                const int c = 32 * w + lane;
                int op;
                M2lPair pr;
                pr.src = pp_source(a, l, x, y, z, c, &op);
                pr.slot = rank + __popc(bits & ((1u << lane) - 1u));
                const bool mir = a.mirror && op > 171;
                if (mir) {
                    op = 342 - op;
                    pr.src |= kPairMirror;
                }
                const int pidx = obase[op] + atomicAdd(&ofill[op], 1);
                pairs[pidx] = pr;
                tpair[pr.slot] = mir ? ~pidx : pidx;
            }
            rank += __popc(bits);
        }
    }
}

// L of every target = the sum of its partial rows over its slots (increasing
// offset); `width` columns are written.  Targets without pairs get zeros.  On
// a pool overflow nothing is summed (the call reports it).  FP32 rows with
// width a multiple of 4 (k_pp_reduce_f4): a block per target, the slots in
// four ordered parts; otherwise (k_pp_reduce) a warp per target in slot
// order, lanes over columns.
constexpr int kRedParts = 4;  // slot-range parts per (target, column group)
__global__ void __launch_bounds__(256) k_pp_reduce_f4(int D, int ld, int stride, int width,
                                                       const LevelInfo* linfo,
                                                       const M2lPairHdr* hdr, const int* tbase,
                                                       const int* __restrict__ tpair,
                                                       const float4* __restrict__ part, float* L) {
    pdl_wait();
    // one block per target, kRedParts x (width / 4) threads: thread (j, u)
    // sums column group u of the j-th quarter of the target's slots in slot
    // order (consecutive threads read consecutive columns of a row, the next
    // 8 slot indices loading while 8 rows are in flight); the quarters are
    // then added in order j = 0, 1, 2, 3 (a fixed association: deterministic)
    __shared__ float4 s_part[kRedParts][64];
    const int g0 = linfo->gbase[2], nt = linfo->gbase[D + 1] - g0;
    const int s4 = stride / 4, w4 = width / 4;
    const bool over = hdr->overflow != 0;
    const int j = threadIdx.x / w4, u = threadIdx.x - j * w4;
    // sign bits of this thread's four columns that a mirrored row carries
    // negated (odd degree; tpair entry ~pair)
    uint4 odd;
    odd.x = (coef_degree(4 * u) & 1) ? 0x80000000u : 0u;
    odd.y = (coef_degree(4 * u + 1) & 1) ? 0x80000000u : 0u;
    odd.z = (coef_degree(4 * u + 2) & 1) ? 0x80000000u : 0u;
    odd.w = (coef_degree(4 * u + 3) & 1) ? 0x80000000u : 0u;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int b0 = tbase[t], b1 = over ? b0 : tbase[t + 1];
        const int cs = (b1 - b0 + kRedParts - 1) / kRedParts;
        const int s0 = min(b0 + j * cs, b1), s1 = min(s0 + cs, b1);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < kRedParts) {
            int rw[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) rw[k] = s0 + k < s1 ? tpair[s0 + k] : 0;
            for (int s = s0; s < s1; s += 8) {
                float4 q[8];
                uint32_t fm[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    fm[k] = rw[k] < 0 ? 0xffffffffu : 0u;
                    if (s + k < s1) q[k] = __ldcs(part + (int64_t)(rw[k] ^ (int)fm[k]) * s4 + u);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) rw[k] = s + 8 + k < s1 ? tpair[s + 8 + k] : 0;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (s + k < s1) {
                        v.x += __uint_as_float(__float_as_uint(q[k].x) ^ (odd.x & fm[k]));
                        v.y += __uint_as_float(__float_as_uint(q[k].y) ^ (odd.y & fm[k]));
                        v.z += __uint_as_float(__float_as_uint(q[k].z) ^ (odd.z & fm[k]));
                        v.w += __uint_as_float(__float_as_uint(q[k].w) ^ (odd.w & fm[k]));
                    }
            }
            s_part[j][u] = v;
        }
        __syncthreads();
        if (j == 0) {
#pragma unroll
            for (int k = 1; k < kRedParts; ++k) {
                const float4 w = s_part[k][u];
                v.x += w.x; v.y += w.y; v.z += w.z; v.w += w.w;
            }
            *reinterpret_cast<float4*>(L + (int64_t)(g0 + t) * ld + 4 * u) = v;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_pp_reduce(int D, int ld, int stride, int width,
                                                    const LevelInfo* linfo, const M2lPairHdr* hdr,
                                                    const int* tbase, const int* __restrict__ tpair,
                                                    const T* __restrict__ part, T* L) {
    const int lane = threadIdx.x & 31;
    const int g0 = linfo->gbase[2], nt = linfo->gbase[D + 1] - g0;
    const bool over = hdr->overflow != 0;
    for (int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nt;
         t += gridDim.x * (blockDim.x >> 5)) {
        const int s0 = tbase[t], s1 = over ? s0 : tbase[t + 1];
        for (int u = lane; u < width; u += 32) {
            T v = T(0);
            const bool odd = coef_degree(u) & 1;
            for (int s = s0; s < s1; ++s) {
                const int r = tpair[s];
                const T x = part[(int64_t)(r < 0 ? ~r : r) * stride + u];
                v += r < 0 && odd ? -x : x;  // mirrored row: odd degrees negated
            }
            L[(int64_t)(g0 + t) * ld + u] = v;
        }
    }
}

// CUDA-core M2L of the work items: per item (offset o, up to 128 pairs) the
// product D[pairs x P] = A[pairs x P] B[P x P], A row r = M of pair r's
// source, B[k][n] = T_o[n][k], written to the pairs' slot rows (columns < P).
// Block tile 64 pairs x 64 outputs, K in chunks of 16 through shared
// memory, 4 x 4 outputs per thread; blocks walk (item, row half, column
// block) units.
constexpr int kSimtRows = 64, kSimtCols = 64, kSimtK = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_m2l_pairs_simt(int P, int ld, int stride,
                                                         const M2lPairHdr* hdr,
                                                         const M2lPairItem* items,
                                                         const M2lPair* pairs,
                                                         const T* __restrict__ M,
                                                         const T* __restrict__ Tm2l, T* part) {
    __shared__ __align__(16) T As[kSimtK][kSimtRows];
    __shared__ __align__(16) T Bs[kSimtK][kSimtCols];
    __shared__ int s_src[kSimtRows], s_slot[kSimtRows];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int cb_n = (P + kSimtCols - 1) / kSimtCols;
    const int units = hdr->n_items * 2 * cb_n;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int item = u / (2 * cb_n), rh = (u / cb_n) & 1, cb = u % cb_n;
        const M2lPairItem it = items[item];
        const int r0 = rh * kSimtRows, rows = min(kSimtRows, it.rows - r0);
        if (rows <= 0) continue;  // uniform over the block
        __syncthreads();
        if (tid < kSimtRows) {
            const bool live = tid < rows;
            s_src[tid] = live ? pairs[it.begin + r0 + tid].src : -1;
            s_slot[tid] = live ? it.begin + r0 + tid : -1;  // partial rows in pair order
        }
        __syncthreads();
        const T* To = Tm2l + (int64_t)it.op * P * P;
        const int c0 = cb * kSimtCols;
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        for (int k0 = 0; k0 < P; k0 += kSimtK) {
#pragma unroll
            for (int e = 0; e < (kSimtRows * kSimtK) / 256; ++e) {
                const int idx = tid + 256 * e;
                const int r = idx / kSimtK, kk = idx % kSimtK;
                const int src = s_src[r];
                As[kk][r] = (src >= 0 && k0 + kk < P) ? M[(int64_t)src * ld + k0 + kk] : T(0);
                const int c = c0 + r;
                Bs[kk][r] = (c < P && k0 + kk < P) ? To[(int64_t)c * P + k0 + kk] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kSimtK; ++kk) {
                T a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = ty * 4 + i;
            if (r >= rows) continue;
            T* out = part + (int64_t)s_slot[r] * stride;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = c0 + tx * 4 + j;
                if (c < P) out[c] = acc[i][j];
            }
        }
    }
}

// CUDA-core L2L of level l (after the reduction, which wrote every cell's
// own M2L sum into L): L_child += T_l2l[octant] L_parent, one warp per
// child, lanes over output coefficients, the parent's L staged per warp.
template <typename T>
__global__ void __launch_bounds__(128) k_l2l_simt(int l, int P, int ld, const LevelInfo* linfo,
                                                  const uint32_t* __restrict__ code,
                                                  const int32_t* __restrict__ cid,
                                                  int64_t off_parent, const T* __restrict__ Tl2l,
                                                  T* L) {
    extern __shared__ unsigned char smem_raw[];
    T* sL = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * P;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int g0 = linfo->gbase[l], g1 = linfo->gbase[l + 1];
    for (int g = g0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); g < g1; g += warps) {
        const uint32_t c = code[g];
        const int gp = cid[off_parent + (c >> 3)];
        __syncwarp();
        for (int k = lane; k < P; k += 32) sL[k] = gp >= 0 ? L[(int64_t)gp * ld + k] : T(0);
        __syncwarp();
        const T* To = Tl2l + (int64_t)(c & 7u) * P * P;
        for (int row = lane; row < P; row += 32) {
            T acc = L[(int64_t)g * ld + row];
            const T* tr = To + (int64_t)row * P;
            for (int k = 0; k < P; ++k) acc += tr[k] * sL[k];
            L[(int64_t)g * ld + row] = acc;
        }
    }
}

// Rotation-based M2L of the work items (CUDA cores): per pair, the source's
// multipole rotated so that the offset points along +z (R^M, degree blocks),
// translated along z (one coupling per order m, Re and Im apart), rotated
// back (R^L(Q^T)), in three passes through shared memory over a tile of np
// pairs; the offset's packed operator [R^M | R^L | Z_re | Z_im] is staged
// once per item.  sum_n (2n+1)^2 x 2 + sum_m (p+1-m)^2 (x 2 for m > 0)
// multiply-adds per pair instead of (p+1)^4.
__device__ __forceinline__ int deg_of(int i) {
    int n = (int)sqrtf((float)i + 0.5f);
    while (n * n > i) --n;
    while ((n + 1) * (n + 1) <= i) ++n;
    return n;
}

template <typename T>
__global__ void __launch_bounds__(256) k_m2l_rot(int p, int P, int ld, int stride, int np,
                                                  const M2lPairHdr* hdr,
                                                  const M2lPairItem* items, const M2lPair* pairs,
                                                  const T* __restrict__ M,
                                                  const T* __restrict__ ops, int op_vals,
                                                  T* part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = (p + 1) * (4 * (p + 1) * (p + 1) - 1) / 3;
    const int nz = op_vals / 2 - nb;
    const int lp = P | 1;  // odd row stride of the pair tiles
    T* sOp = reinterpret_cast<T*>(smem_raw);
    T* sA = sOp + op_vals;
    T* sB = sA + np * lp;
    __shared__ int s_src[64], s_slot[64];
    const T* RM = sOp;
    const T* RL = sOp + nb;
    const T* ZR = sOp + 2 * nb;
    const T* ZI = ZR + nz;
    const int tid = threadIdx.x;
    const int S1 = (p + 1) * (p + 2) * (2 * p + 3) / 6;  // sum_{q<=p+1} q^2
    for (int itx = blockIdx.x; itx < hdr->n_items; itx += gridDim.x) {
        const M2lPairItem it = items[itx];
        __syncthreads();
        const T* op = ops + (int64_t)it.op * op_vals;
        for (int e = tid; e < op_vals; e += blockDim.x) sOp[e] = op[e];
        for (int r0 = 0; r0 < it.rows; r0 += np) {
            const int rows = min(np, it.rows - r0);
            __syncthreads();
            if (tid < np) {
                const bool live = tid < rows;
                s_src[tid] = live ? pairs[it.begin + r0 + tid].src : -1;
                s_slot[tid] = live ? it.begin + r0 + tid : -1;  // partial rows in pair order
            }
            __syncthreads();
            for (int e = tid; e < np * P; e += blockDim.x) {
                const int r = e / P, k = e - r * P;
                const int src = s_src[r];
                sA[r * lp + k] = src >= 0 ? M[(int64_t)src * ld + k] : T(0);
            }
            __syncthreads();
            // rotate the multipoles: sB = R^M sA (degree blocks)
            for (int e = tid; e < np * P; e += blockDim.x) {
                const int i = e / np, r = e - i * np;
                const int n = deg_of(i), w = i - n * n, k = 2 * n + 1;
                const T* row = RM + n * (4 * n * n - 1) / 3 + w * k;
                const T* a = sA + r * lp + n * n;
                T acc = T(0);
                for (int u = 0; u < k; ++u) acc += row[u] * a[u];
                sB[r * lp + i] = acc;
            }
            __syncthreads();
            // translate along z: sA = Z sB (order m couples degrees l, j >= m)
            for (int e = tid; e < np * P; e += blockDim.x) {
                const int i = e / np, r = e - i * np;
                const int l = deg_of(i), w = i - l * l;
                const int m = (w + 1) >> 1;
                const int im = (w > 0 && !(w & 1)) ? 1 : 0;
                const int width = p + 1 - m;
                const int q = p + 1 - m;  // zoff(m) = S(p+1) - S(p+1-m)
                const int zo = S1 - q * (q + 1) * (2 * q + 1) / 6;
                const T* row = (im ? ZI : ZR) + zo + (l - m) * width;
                const T* b = sB + r * lp + (m == 0 ? 0 : 2 * m - 1) + im;
                T acc = T(0);
                for (int j = m; j <= p; ++j) acc += row[j - m] * b[j * j];
                sA[r * lp + i] = acc;
            }
            __syncthreads();
            // rotate back: sB = R^L(Q^T) sA
            for (int e = tid; e < np * P; e += blockDim.x) {
                const int i = e / np, r = e - i * np;
                const int n = deg_of(i), w = i - n * n, k = 2 * n + 1;
                const T* row = RL + n * (4 * n * n - 1) / 3 + w * k;
                const T* a = sA + r * lp + n * n;
                T acc = T(0);
                for (int u = 0; u < k; ++u) acc += row[u] * a[u];
                sB[r * lp + i] = acc;
            }
            __syncthreads();
            for (int e = tid; e < rows * P; e += blockDim.x) {
                const int r = e / P, k = e - r * P;
                part[(int64_t)s_slot[r] * stride + k] = sB[r * lp + k];
            }
        }
    }
}

}  // namespace

PairList pair_list(const Workspace& ws, size_t* bytes) {
    PairList L;
    unsigned char* b = static_cast<unsigned char*>(ws.pp_work);
    size_t o = 0;
    auto take = [&](size_t sz) {
        unsigned char* r = b ? b + o : nullptr;
        o += (sz + 255) & ~(size_t)255;
        return r;
    };
    L.hdr = (M2lPairHdr*)take(sizeof(M2lPairHdr));
    L.ocnt = (int*)take(sizeof(int) * 2 * 344);
    L.ofill = L.ocnt + 344;
    L.obase = (int*)take(sizeof(int) * 344);
    L.tbase = (int*)take(sizeof(int) * (ws.cells_max + 1));
    L.tcount = (int*)take(sizeof(int) * ws.cells_max);
    L.tmask = (uint32_t*)take(sizeof(uint32_t) * kPpWords * ws.cells_max);
    L.items = (M2lPairItem*)take(sizeof(M2lPairItem) * ws.pp_item_cap);
    L.pairs = (M2lPair*)take(sizeof(M2lPair) * ws.pp_rows_cap);
    L.tpair = (int*)take(sizeof(int) * ws.pp_slot_cap);
    if (bytes) *bytes = o;
    return L;
}

size_t m2l_pp_work_bytes(const Workspace& ws) {
    Workspace w = ws;
    w.pp_work = nullptr;
    size_t b = 0;
    pair_list(w, &b);
    return b;
}

size_t m2l_pp_part_bytes(const Workspace& ws) {
    return (size_t)ws.pp_rows_cap * ws.pp_stride * (ws.fp64 ? sizeof(double) : sizeof(float));
}

static int64_t target_cells_bound(int64_t n, int D) {
    int64_t t = 0;
    for (int l = 2; l <= D; ++l) {
        const int64_t cl = (int64_t)1 << (3 * l);
        t += n < cl ? n : cl;
    }
    return t > 0 ? t : 1;
}

cudaError_t launch_m2l_pairs_worklist(int64_t n, int D, Workspace& ws, cudaStream_t s) {
    if (D < 2) return cudaSuccess;
    PpArgs a;
    a.D = D;
    // only the BF16x3 tensor-core product reads mirrored pairs (its A rows
    // from the mirrored multipole pieces)
    a.mirror = ws.tc_bf16 && ws.pp_mirror ? 1 : 0;
    a.linfo = ws.linfo;
    a.code = ws.code;
    a.cid = ws.cid;
    const DenseLayout dl = dense_layout(D);
    for (int l = 0; l < kMaxDepth + 2; ++l) a.off[l] = dl.off[l];
    PairList L = pair_list(ws);
    cudaError_t e;
    // the offset counts and fill counters are zero here: zeroed at allocation
    // and by k_pp_scan after use
    const int64_t tb = target_cells_bound(n, D);
    const int64_t warps = kPpThreads / 32;
    const unsigned gc = (unsigned)std::min<int64_t>((tb + warps - 1) / warps, 152 * 8);
    k_pp_count<<<gc, kPpThreads, 0, s>>>(a, L.tmask, L.tcount, L.ocnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_pdl(k_pp_scan, dim3(1), dim3(kPpScanThreads), 0, s, D,
                        (const LevelInfo*)ws.linfo, (int64_t)ws.pp_slot_cap,
                        (int64_t)ws.pp_rows_cap, (int)ws.pp_item_cap, (const int*)L.tcount,
                        L.tbase, L.ocnt, L.ofill, L.obase, L.hdr, (M2lPairHdr*)ws.h_pp_hdr,
                        L.items, ws.err)) != cudaSuccess)
        return e;
    return launch_pdl(k_pp_fill, dim3(gc), dim3(kPpThreads), 0, s, a, (const uint32_t*)L.tmask,
                      (const int*)L.tbase, (const int*)L.obase, L.ofill, (const M2lPairHdr*)L.hdr,
                      L.pairs, L.tpair);
}



cudaError_t launch_m2l_pairs_reduce(int64_t n, int D, Workspace& ws, int width, cudaStream_t s) {
    if (D < 2) return cudaSuccess;
    PairList L = pair_list(ws);
    const int64_t tb = target_cells_bound(n, D);
    const unsigned gr = (unsigned)std::min<int64_t>((tb + 7) / 8, 152 * 16);
    if (ws.fp64) {
        k_pp_reduce<double><<<gr, 256, 0, s>>>(D, ws.ld, ws.pp_stride, width, ws.linfo, L.hdr,
                                               L.tbase, L.tpair, (const double*)ws.pp_part,
                                               (double*)ws.L);
    } else if (width % 4 == 0 && width <= 256 && ws.pp_stride % 4 == 0 && ws.ld % 4 == 0) {
        const unsigned g4 = (unsigned)std::min<int64_t>(tb, 152 * 32);
        return launch_pdl(k_pp_reduce_f4, dim3(g4), dim3(kRedParts * (width / 4)), 0, s, D,
                          ws.ld, ws.pp_stride, width, (const LevelInfo*)ws.linfo,
                          (const M2lPairHdr*)L.hdr, (const int*)L.tbase, (const int*)L.tpair,
                          (const float4*)ws.pp_part, (float*)ws.L);
    } else {
        k_pp_reduce<float><<<gr, 256, 0, s>>>(D, ws.ld, ws.pp_stride, width, ws.linfo, L.hdr,
                                              L.tbase, L.tpair, (const float*)ws.pp_part,
                                              (float*)ws.L);
    }
    return cudaGetLastError();
}

// shared-memory bytes of k_m2l_rot for np pairs per tile
static size_t rot_smem(const Workspace& ws, int np) {
    const size_t tsz = ws.fp64 ? sizeof(double) : sizeof(float);
    return tsz * ((size_t)ws.rot_op_vals + 2 * (size_t)np * (ws.P | 1));
}

int m2l_rot_tile(const Workspace& ws) {
    for (int np = 64; np >= 8; np /= 2)
        if (rot_smem(ws, np) <= 200 * 1024) return np;
    return 0;
}

cudaError_t m2l_rot_init() {
    cudaError_t e = cudaFuncSetAttribute(k_m2l_rot<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_m2l_rot<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
    return e;
}

template <typename T>
static cudaError_t rot_pairs(int64_t n, int D, Workspace& ws, cudaStream_t s) {
    PairList L = pair_list(ws);
    const int np = m2l_rot_tile(ws);
    if (np == 0) return cudaErrorNotSupported;
    const unsigned grid = (unsigned)std::min<int64_t>(ws.pp_item_cap, 152 * 4);
    k_m2l_rot<T><<<grid, 256, rot_smem(ws, np), s>>>(ws.p, ws.P, ws.ld, ws.pp_stride, np, L.hdr,
                                                     L.items, L.pairs, (const T*)ws.M,
                                                     (const T*)ws.T_rot, ws.rot_op_vals,
                                                     (T*)ws.pp_part);
    (void)n;
    (void)D;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t simt_pairs(int64_t n, int D, Workspace& ws, int l2l_last, cudaStream_t s) {
    const int P = ws.P;
    PairList L = pair_list(ws);
    cudaError_t e;
    if (ws.kev[0] && (e = record_timing(ws.kev[0], s)) !=
                         cudaSuccess)
        return e;
    if (ws.m2l_rot) {
        if ((e = rot_pairs<T>(n, D, ws, s)) != cudaSuccess) return e;
    } else {
        const int64_t units = ws.pp_item_cap * 2 * ((P + kSimtCols - 1) / kSimtCols);
        const unsigned grid = (unsigned)std::min<int64_t>(units, 152 * 8);
        k_m2l_pairs_simt<T><<<grid, 256, 0, s>>>(P, ws.ld, ws.pp_stride, L.hdr, L.items, L.pairs,
                                                 (const T*)ws.M, (const T*)ws.T_m2l,
                                                 (T*)ws.pp_part);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (ws.kev[1] && (e = record_timing(ws.kev[1], s)) !=
                         cudaSuccess)
        return e;
    if ((e = launch_m2l_pairs_reduce(n, D, ws, P, s)) != cudaSuccess) return e;
    const DenseLayout dl = dense_layout(D);
    for (int l = 3; l <= l2l_last && l <= D; ++l) {
        const int64_t cl = (int64_t)1 << (3 * l);
        const int64_t cells = n < cl ? n : cl;
        const unsigned g = (unsigned)std::min<int64_t>((cells + 3) / 4, 152 * 16);
        k_l2l_simt<T><<<g, 128, 4 * P * sizeof(T), s>>>(l, P, ws.ld, ws.linfo, ws.code, ws.cid,
                                                        dl.off[l - 1], (const T*)ws.T_l2l,
                                                        (T*)ws.L);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_m2l_pairs_simt(int64_t n, int D, Workspace& ws, int l2l_last, cudaStream_t s) {
    if (D < 2) return cudaSuccess;
    return ws.fp64 ? simt_pairs<double>(n, D, ws, l2l_last, s)
                   : simt_pairs<float>(n, D, ws, l2l_last, s);
}

cudaError_t m2l_pairs_stats(const Workspace& ws, int64_t* out, cudaStream_t s) {
    for (int k = 0; k < 4; ++k) out[k] = 0;
    if (!ws.pp_work) return cudaSuccess;
    M2lPairHdr h;
    cudaError_t e = cudaMemcpyAsync(&h, pair_list(ws).hdr, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    out[0] = h.n_offsets;
    out[1] = h.n_items;
    out[2] = h.n_items;
    out[3] = h.n_pairs;
    return cudaSuccess;
}

}  // namespace pt
