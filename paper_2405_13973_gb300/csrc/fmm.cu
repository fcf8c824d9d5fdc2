// fmm.cu -- the FMM stages on the CUDA cores (Sec. 2.3.2) and the order of
// one evaluation's launches (run_fmm: main chain and side stream).
//
// Upward pass: P2M at the leaves (Eq. FMM_coul2; on the tensor-core path
// also at the leaves' parents, straight from their ions), M2M to the parents.
// Downward pass: at every level l >= 2 the local expansion of a cell is the
// L2L shift of its parent's plus the M2L conversion (Eq. FMM_local) of the
// multipole expansions of the 189 cells that are children of the parent's
// neighbours but not neighbours themselves.  At the leaves the far field is
// the gradient of the local expansion (L2P) and the near field the direct sum
// over the 27 adjacent leaves (P2P).
//
// Cells of one level are stored octant-major, so a tile of target cells
// shares its octant and therefore the same 189 source offsets: M2L becomes,
// per offset o, a dense product L[:, tile] += T_o * M[:, src(tile, o)], the
// L2L shift being one more such product with the parent's L.
//
// Everything is templated on the arithmetic type (double: PT_FP64, float:
// PT_FP32 and the CUDA-core stages of PT_MIXED_TF32X3).  Coefficients are in
// the normalised real storage of harmonics.cuh, scaled by the cell size.
#include <cuda_runtime.h>

#include "bf16split.cuh"
#include "fmm_math.cuh"
#include "harmonics.cuh"
#include "internal.h"

namespace pt {

__constant__ HarmTables<double> c_tab_d;
__constant__ HarmTables<float> c_tab_f;
// the same tables in global memory, for kernels whose lanes read them at
// different m (constant memory would serialise those reads)
__device__ HarmTables<double> g_tab_d;
__device__ HarmTables<float> g_tab_f;
// M2L source offsets per target octant: packed (ox+3)*49 + (oy+3)*7 + (oz+3),
// o = target - source, o_a in [b_a - 3, b_a + 2] with b the octant bits,
// excluding the 27 neighbours.
__constant__ int16_t c_m2l_off[8][189];

template <typename T>
__device__ __forceinline__ const HarmTables<T>& tab();
template <>
__device__ __forceinline__ const HarmTables<double>& tab<double>() { return c_tab_d; }
template <>
__device__ __forceinline__ const HarmTables<float>& tab<float>() { return c_tab_f; }
template <typename T>
__device__ __forceinline__ const HarmTables<T>& gtab();
template <>
__device__ __forceinline__ const HarmTables<double>& gtab<double>() { return g_tab_d; }
template <>
__device__ __forceinline__ const HarmTables<float>& gtab<float>() { return g_tab_f; }

void host_m2l_offsets(int16_t out[8][189]) {
    for (int oct = 0; oct < 8; ++oct) {
        int b[3] = {(oct >> 2) & 1, (oct >> 1) & 1, oct & 1};
        int k = 0;
        for (int ox = b[0] - 3; ox <= b[0] + 2; ++ox)
            for (int oy = b[1] - 3; oy <= b[1] + 2; ++oy)
                for (int oz = b[2] - 3; oz <= b[2] + 2; ++oz) {
                    if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                    out[oct][k++] = (int16_t)((ox + 3) * 49 + (oy + 3) * 7 + (oz + 3));
                }
    }
}


// Sorted ion records (written by the tree build): the FP64 path keeps
// (u, q) in double; the FP32 paths keep u in 30-bit fixed point and q as
// float bits (int4), so that near-field separations are exact integers.
template <typename T>
struct Ion;
template <>
struct Ion<double> {
    using rec = double4_32a;
    static __device__ __forceinline__ void get(const rec& r, double& x, double& y, double& z,
                                               double& q) {
        x = r.x; y = r.y; z = r.z; q = r.w;
    }
    // (x_t - x_s)/s for a source in the leaf at integer offset d from the target's
    static __device__ __forceinline__ void sep(const rec& t, const rec& o, int dx, int dy, int dz,
                                               double& rx, double& ry, double& rz) {
        rx = (t.x - o.x) - dx;
        ry = (t.y - o.y) - dy;
        rz = (t.z - o.z) - dz;
    }
    // a source expressed in the target leaf's frame (u + d)
    static __device__ __forceinline__ rec shifted(const rec& o, int dx, int dy, int dz) {
        return make_double4_32a(o.x + dx, o.y + dy, o.z + dz, o.w);
    }
    static __device__ __forceinline__ void sep_shifted(const rec& t, const rec& o, double& rx,
                                                       double& ry, double& rz, double& q) {
        rx = t.x - o.x;
        ry = t.y - o.y;
        rz = t.z - o.z;
        q = o.w;
    }
};
template <>
struct Ion<float> {
    using rec = int4;
    static __device__ __forceinline__ void get(const rec& r, float& x, float& y, float& z,
                                               float& q) {
        x = __int2float_rn(r.x) * 0x1p-30f;
        y = __int2float_rn(r.y) * 0x1p-30f;
        z = __int2float_rn(r.z) * 0x1p-30f;
        q = __int_as_float(r.w);
    }
    // |t - o| < 2^30 and |d| 2^30 <= 2^30: the integer difference fits in 31 bits
    static __device__ __forceinline__ void sep(const rec& t, const rec& o, int dx, int dy, int dz,
                                               float& rx, float& ry, float& rz) {
        rx = __int2float_rn((t.x - o.x) - dx * (1 << 30)) * 0x1p-30f;
        ry = __int2float_rn((t.y - o.y) - dy * (1 << 30)) * 0x1p-30f;
        rz = __int2float_rn((t.z - o.z) - dz * (1 << 30)) * 0x1p-30f;
    }
    // a source in the target leaf's frame: u + d 2^30 stays within
    // [-2^29 - 2^30, 2^29 - 1 + 2^30], so u_t - (u_s + d 2^30) fits in int32
    static __device__ __forceinline__ rec shifted(const rec& o, int dx, int dy, int dz) {
        return make_int4(o.x + dx * (1 << 30), o.y + dy * (1 << 30), o.z + dz * (1 << 30), o.w);
    }
    static __device__ __forceinline__ void sep_shifted(const rec& t, const rec& o, float& rx,
                                                       float& ry, float& rz, float& q) {
        rx = __int2float_rn(t.x - o.x) * 0x1p-30f;
        ry = __int2float_rn(t.y - o.y) * 0x1p-30f;
        rz = __int2float_rn(t.z - o.z) * 0x1p-30f;
        q = __int_as_float(o.w);
    }
};

// s + v with the rounding error carried in c (Kahan-Babuska / Neumaier).
template <typename T>
__device__ __forceinline__ void kb_add(T& s, T& c, T v) {
    T t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

// Position of a sorted ion in the frame of its ancestor s levels above its
// leaf: o = the leaf's integer position inside the ancestor (0 .. 2^s - 1
// per axis), u_anc = (u_leaf + o + 1/2 - 2^s / 2) / 2^s, in ancestor units.
__device__ __forceinline__ void ion_in_ancestor(const Ion<float>::rec& r, int s, int ox, int oy,
                                                int oz, float& x, float& y, float& z, float& q) {
    const float sc = __int_as_float((127 - 30 - s) << 23);  // 2^-(30+s)
    const int half = 1 << s;
    const long long u = 1ll << 29;  // 1/2 in 30-bit fixed point
    x = __ll2float_rn((long long)r.x + (long long)(2 * ox + 1 - half) * u) * sc;
    y = __ll2float_rn((long long)r.y + (long long)(2 * oy + 1 - half) * u) * sc;
    z = __ll2float_rn((long long)r.z + (long long)(2 * oz + 1 - half) * u) * sc;
    q = __int_as_float(r.w);
}
__device__ __forceinline__ void ion_in_ancestor(const Ion<double>::rec& r, int s, int ox, int oy,
                                                int oz, double& x, double& y, double& z, double& q) {
    const double sc = ldexp(1.0, -s), c = 0.5 - 0.5 * (double)(1 << s);
    x = (r.x + ((double)ox + c)) * sc;
    y = (r.y + ((double)oy + c)) * sc;
    z = (r.z + ((double)oz + c)) * sc;
    q = r.w;
}

constexpr int kP2mThreads = 128;
constexpr int kP2mIons = 32;

// ---------------------------------------------------------------------------
// P2M: one block per leaf.  Each thread evaluates conj(Y^_n^m(u)) q of one ion
// (all n, m, by the column recurrences) into shared memory, then each thread
// owns coefficients and sums them over the leaf's ions in slot order
// (deterministic).  Leaves with more ions than kP2mIons are done in passes.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kP2mThreads) k_p2m(int D, int p, int ld, const LevelInfo* linfo,
                                                     const int32_t* __restrict__ cstart,
                                                     const int32_t* __restrict__ ccount,
                                                     const typename Ion<T>::rec* __restrict__ sorted,
                                                     T* __restrict__ M, uint16_t* Mp) {
    extern __shared__ unsigned char p2m_smem[];
    const int P = (p + 1) * (p + 1);
    T* terms = reinterpret_cast<T*>(p2m_smem);  // [kP2mIons][P]
    const HarmTables<T>& t = tab<T>();
    const int g0 = linfo->gbase[D], g1 = linfo->gbase[D + 1];
    for (int g = g0 + blockIdx.x; g < g1; g += gridDim.x) {
        const int s = cstart[g], k = ccount[g];
        T acc[(kMaxOrder + 1) * (kMaxOrder + 1) / kP2mThreads + 1];
        constexpr int NA = (kMaxOrder + 1) * (kMaxOrder + 1) / kP2mThreads + 1;
#pragma unroll
        for (int r = 0; r < NA; ++r) acc[r] = T(0);
        for (int i0 = 0; i0 < k; i0 += kP2mIons) {
            const int ni = min(kP2mIons, k - i0);
            __syncthreads();
            if (threadIdx.x < ni) {
                T x, y, z, q;
                Ion<T>::get(sorted[s + i0 + threadIdx.x], x, y, z, q);
                T* row = terms + threadIdx.x * P;
                for_each_ups<T>(p, x, y, z, t, [&](int n, int m, T re, T im) {
                    const int idx = re_idx(n, m);
                    row[idx] = q * re;
                    if (m > 0) row[idx + 1] = -q * im;
                });
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < NA; ++r) {
                const int c = threadIdx.x + r * kP2mThreads;
                if (c < P)
                    for (int i = 0; i < ni; ++i) acc[r] += terms[i * P + c];
            }
        }
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            const int c = threadIdx.x + r * kP2mThreads;
            if (c < P) {
                M[(int64_t)g * ld + c] = acc[r];
                if (Mp) store_pieces(Mp, g, ld, c, (float)acc[r]);  // BF16x3 operand
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Direct ancestor multipoles (PT_EXPAND_DIRECT): P2M of every ion about each
// of its cells at levels lmin..D, one block per cell, as k_p2m but with u in
// the cell's frame and units and compensated sums (an ancestor's
// coefficients sum thousands of terms of both signs).  A cell's ions are the
// contiguous slots of its leaves.  Equal to P2M at the leaves followed by the
// M2M shifts, which shift a truncated expansion exactly.
// ---------------------------------------------------------------------------
constexpr int kP2mAncIons = 64;

template <typename T>
__global__ void __launch_bounds__(kP2mThreads) k_p2m_anc(
    int D, int lmin, int p, int ld, const LevelInfo* linfo, const uint32_t* __restrict__ code,
    const int32_t* __restrict__ leaf_start, const int32_t* __restrict__ leaf_of,
    const typename Ion<T>::rec* __restrict__ sorted, T* __restrict__ M, uint16_t* Mp) {
    extern __shared__ unsigned char p2m_smem[];
    const int P = (p + 1) * (p + 1);
    pdl_wait();
    T* terms = reinterpret_cast<T*>(p2m_smem);  // [kP2mAncIons][P]
    const HarmTables<T>& t = tab<T>();
    const int g0 = linfo->gbase[lmin], g1 = linfo->gbase[D + 1];
    for (int g = g0 + blockIdx.x; g < g1; g += gridDim.x) {
        int l = lmin;
        while (l < D && g >= linfo->gbase[l + 1]) ++l;
        const int sh = D - l, mask = (1 << sh) - 1;
        const uint32_t c = code[g];
        const int s = leaf_start[(int64_t)c << (3 * sh)];
        const int k = leaf_start[((int64_t)c + 1) << (3 * sh)] - s;
        constexpr int NA = (kMaxOrder + 1) * (kMaxOrder + 1) / kP2mThreads + 1;
        T acc[NA], cmp[NA];
#pragma unroll
        for (int r = 0; r < NA; ++r) acc[r] = cmp[r] = T(0);
        for (int i0 = 0; i0 < k; i0 += kP2mAncIons) {
            const int ni = min(kP2mAncIons, k - i0);
            __syncthreads();
            if (threadIdx.x < ni) {
                T x, y, z, q;
                const int slot = s + i0 + threadIdx.x;
                int ix, iy, iz;
                demorton3(code[leaf_of[slot]], ix, iy, iz);
                ion_in_ancestor(sorted[slot], sh, ix & mask, iy & mask, iz & mask, x, y, z, q);
                T* row = terms + threadIdx.x * P;
                for_each_ups<T>(p, x, y, z, t, [&](int n, int m, T re, T im) {
                    const int idx = re_idx(n, m);
                    row[idx] = q * re;
                    if (m > 0) row[idx + 1] = -q * im;
                });
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < NA; ++r) {
                const int cc = threadIdx.x + r * kP2mThreads;
                if (cc < P)
                    for (int i = 0; i < ni; ++i) kb_add(acc[r], cmp[r], terms[i * P + cc]);
            }
        }
#pragma unroll
        for (int r = 0; r < NA; ++r) {
            const int cc = threadIdx.x + r * kP2mThreads;
            if (cc < P) {
                const T v = acc[r] + cmp[r];
                M[(int64_t)g * ld + cc] = v;
                if (Mp) store_pieces(Mp, g, ld, cc, (float)v);  // BF16x3 operand
            }
        }
    }
}

// ---------------------------------------------------------------------------
// M2M: one warp per parent; lanes over output coefficients.
//   Tt: [8][P][P] transposed (in-major) so that lanes read consecutively.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_m2m(int l, int P, int ld, const LevelInfo* linfo,
                                             const uint32_t* __restrict__ code,
                                             const int32_t* __restrict__ cid, int64_t off_child,
                                             const T* __restrict__ Tt, T* M) {
    extern __shared__ unsigned char smem_raw[];
    T* sM = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * P;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int g0 = linfo->gbase[l], g1 = linfo->gbase[l + 1];
    constexpr int R = ((kMaxOrder + 1) * (kMaxOrder + 1) + 31) / 32;
    for (int g = g0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); g < g1; g += warps) {
        const uint32_t c = code[g];
        T acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = T(0);
        for (int o = 0; o < 8; ++o) {
            const int gc = cid[off_child + ((c << 3) | o)];
            if (gc < 0) continue;
            __syncwarp();
            for (int k = lane; k < P; k += 32) sM[k] = M[(int64_t)gc * ld + k];
            __syncwarp();
            const T* To = Tt + (int64_t)o * P * P;
            for (int k = 0; k < P; ++k) {
                const T mk = sM[k];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    int row = lane + 32 * r;
                    if (row < P) acc[r] += To[(int64_t)k * P + row] * mk;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int row = lane + 32 * r;
            if (row < P) M[(int64_t)g * ld + row] = acc[r];
        }
    }
}

// ---------------------------------------------------------------------------
// M2M and L2L of the small upper levels on the tensor-core paths, on the CUDA
// cores: out[g][r] (+)= sum_t Op[r][t] x_g[t], with
//   M2M (MODE 0): x_g = the M of parent g's eight children side by side
//                 (t = o P + c; absent children zero), Op = [T_0 ... T_7];
//   L2L (MODE 1): x_g = the L of child g's parent, Op = T_octant(g), added
//                 to the child's own M2L sum already in L.
// A level of a few dozen or hundred cells is latency work: a launch of the
// persistent tensor-core kernel (TMEM and barrier set-up, operator copies
// from DRAM, one partial per octant and a reduction for M2M) costs more than
// the products.  A block holds rows r0 .. r0 + 15 of the operator in shared
// memory (staged before the programmatic wait: operators are constants) and
// applies them to runs of kShCells cells; warp w owns rows w and w + 8, its
// lanes split the dot products and a butterfly sums them (every lane gets the
// same value: the order is fixed, results are deterministic).
// ---------------------------------------------------------------------------
constexpr int kShRows = 16;
constexpr int kShThreads = 256;
template <int MODE>
struct ShCells { static constexpr int v = MODE == 0 ? 8 : 16; };

// 4-byte asynchronous copy global -> shared (zero-filled when !valid): the
// staging loops issue every copy before waiting once
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// row stride of the staged operator: K rounded up to 2 mod 32 (the M2M
// staging writes two values of t for 16 rows per warp without conflicts)
__host__ __device__ inline int sh_stride(int K) { return K + ((2 - K % 32) % 32 + 32) % 32; }

template <typename T, int MODE>
size_t shift_rows_smem(int P) {
    const int K = MODE == 0 ? 8 * P : P;
    return (size_t)(kShRows * sh_stride(K) + ShCells<MODE>::v * K) * sizeof(T);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kShThreads) k_shift_rows(int l, int P, int ld,
                                                           const LevelInfo* linfo,
                                                           const uint32_t* __restrict__ code,
                                                           const int32_t* __restrict__ cid,
                                                           int64_t off_nb,
                                                           const T* __restrict__ Op, T* Y,
                                                           uint16_t* Mp) {
    static_assert(sizeof(T) == 4, "FP32 plans only (4-byte asynchronous copies)");
    constexpr int CG = ShCells<MODE>::v;
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_src[CG * (MODE == 0 ? 8 : 1)];
    const int K = MODE == 0 ? 8 * P : P, S = sh_stride(K);
    T* sOp = reinterpret_cast<T*>(smem_raw);  // [kShRows][S]
    T* sX = sOp + kShRows * S;                // [CG][K]
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.x * kShRows;
    const int oct = MODE == 1 ? (int)blockIdx.y : 0;
    if (MODE == 0) {
        // Op = T_m2m transposed, [o][c][r]: element (r, t = o P + c) at t P + r
        for (int e = tid; e < K * kShRows; e += kShThreads) {
            const int t = e >> 4, rr = e & 15, r = r0 + rr;
            cp_async4(&sOp[rr * S + t], Op + (int64_t)t * P + (r < P ? r : 0), r < P);
        }
    } else {
        const T* To = Op + (int64_t)oct * P * P;  // T_l2l row-major [o][r][c]
        for (int rr = w; rr < kShRows; rr += kShThreads / 32) {
            const int r = r0 + rr;
            for (int c = lane; c < K; c += 32)
                cp_async4(&sOp[rr * S + c], To + (int64_t)(r < P ? r : 0) * P + c, r < P);
        }
    }
    pdl_wait();
    int g0, g1;
    if (MODE == 0) {
        g0 = linfo->gbase[l];
        g1 = linfo->gbase[l + 1];
    } else {
        g0 = linfo->oct_start[l][oct];
        g1 = linfo->oct_start[l][oct + 1];
    }
    const int nch = (g1 - g0 + CG - 1) / CG;
    const int ch0 = MODE == 0 ? (int)blockIdx.y : (int)blockIdx.z;
    const int chs = MODE == 0 ? (int)gridDim.y : (int)gridDim.z;
    const T* op0 = sOp + w * S;
    const T* op1 = sOp + (w + 8) * S;
    for (int ch = ch0; ch < nch; ch += chs) {
        const int gb = g0 + ch * CG, nc = min(CG, g1 - gb);
        __syncthreads();  // the previous run is done with sX and s_src
        if (MODE == 0) {
            if (tid < CG * 8) {
                const int ci = tid >> 3, o = tid & 7;
                s_src[tid] = ci < nc ? cid[off_nb + (((int64_t)code[gb + ci] << 3) | o)] : -1;
            }
        } else if (tid < CG) {
            s_src[tid] = tid < nc ? cid[off_nb + (code[gb + tid] >> 3)] : -1;
        }
        __syncthreads();
        // x rows: (cell, octant) of M2M, one per cell for L2L
        for (int q = w; q < CG * (MODE == 0 ? 8 : 1); q += kShThreads / 32) {
            const int src = s_src[q];
            T* dst = sX + (MODE == 0 ? (q >> 3) * K + (q & 7) * P : q * K);
            const T* from = Y + (int64_t)(src >= 0 ? src : 0) * ld;
            for (int c = lane; c < P; c += 32) cp_async4(&dst[c], from + c, src >= 0);
        }
        cp_async_wait_all();  // this thread's copies (and, first time round, the operator's)
        __syncthreads();
        T a0[CG], a1[CG];
#pragma unroll
        for (int ci = 0; ci < CG; ++ci) a0[ci] = a1[ci] = T(0);
        for (int t = lane; t < K; t += 32) {
            const T u0 = op0[t], u1 = op1[t];
#pragma unroll
            for (int ci = 0; ci < CG; ++ci) {
                const T x = sX[ci * K + t];
                a0[ci] += u0 * x;
                a1[ci] += u1 * x;
            }
        }
        T v0 = T(0), v1 = T(0);
#pragma unroll
        for (int ci = 0; ci < CG; ++ci) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                a0[ci] += __shfl_xor_sync(0xffffffffu, a0[ci], o);
                a1[ci] += __shfl_xor_sync(0xffffffffu, a1[ci], o);
            }
            if (lane == ci) {
                v0 = a0[ci];
                v1 = a1[ci];
            }
        }
        if (lane < nc) {  // lane ci stores cell ci's rows w and w + 8
            T* y = Y + (int64_t)(gb + lane) * ld;
            const int ra = r0 + w, rb = r0 + w + 8;
            if (MODE == 0) {
                if (ra < P) y[ra] = v0;
                if (rb < P) y[rb] = v1;
                if (Mp) {  // BF16x3 operand of the M2L
                    if (ra < P) store_pieces(Mp, gb + lane, ld, ra, (float)v0);
                    if (rb < P) store_pieces(Mp, gb + lane, ld, rb, (float)v1);
                }
            } else {
                if (ra < P) y[ra] += v0;
                if (rb < P) y[rb] += v1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// M2L (+ folded L2L) on the CUDA cores: block = 64 output rows x 32 targets of
// one octant; loops over the 189 offsets (and the parent shift), each a
// 64 x P x 32 product staged through shared memory.
// ---------------------------------------------------------------------------
constexpr int kRT = 64, kNT = 32, kKC = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_m2l_simt(int l, int P, int ld, const LevelInfo* linfo,
                                                  const uint32_t* __restrict__ code,
                                                  const int32_t* __restrict__ cid, int64_t off_l,
                                                  int64_t off_parent, const T* __restrict__ M,
                                                  T* L, const T* __restrict__ Tm2l,
                                                  const T* __restrict__ Tl2l) {
    __shared__ T As[kKC][kRT];
    __shared__ T Bs[kKC][kNT];
    __shared__ const T* src[kNT];
    __shared__ int tile_oct, tile_base, tile_n;
    __shared__ int s_oct[9];
    const int tid = threadIdx.x;
    if (tid < 9) s_oct[tid] = linfo->oct_start[l][tid];
    __syncthreads();
    if (tid == 0) {
        int b = blockIdx.x, acc = 0;
        tile_n = 0;
        for (int o = 0; o < 8; ++o) {
            int s0 = s_oct[o], s1 = s_oct[o + 1];
            int nt = (s1 - s0 + kNT - 1) / kNT;
            if (b < acc + nt) {
                tile_oct = o;
                tile_base = s0 + (b - acc) * kNT;
                tile_n = min(kNT, s1 - tile_base);
                break;
            }
            acc += nt;
        }
    }
    __syncthreads();
    if (tile_n <= 0) return;
    const int oct = tile_oct, base = tile_base, ntile = tile_n;
    const int row0 = blockIdx.y * kRT;
    const int ty = tid >> 4, tx = tid & 15;
    const int lim = 1 << l;
    T acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = T(0);
    const int nterms = 189 + (l >= 3 ? 1 : 0);
    for (int term = 0; term < nterms; ++term) {
        const T* A;
        if (term < 189) {
            const int opi = c_m2l_off[oct][term];
            A = Tm2l + (int64_t)opi * P * P;
            if (tid < kNT) {
                const T* sp = nullptr;
                if (tid < ntile) {
                    int ix, iy, iz;
                    demorton3(code[base + tid], ix, iy, iz);
                    int sx = ix - (opi / 49 - 3), sy = iy - ((opi / 7) % 7 - 3),
                        sz = iz - (opi % 7 - 3);
                    if (sx >= 0 && sx < lim && sy >= 0 && sy < lim && sz >= 0 && sz < lim) {
                        int gs = cid[off_l + morton3(sx, sy, sz)];
                        if (gs >= 0) sp = M + (int64_t)gs * ld;
                    }
                }
                src[tid] = sp;
            }
        } else {
            A = Tl2l + (int64_t)oct * P * P;
            if (tid < kNT) {
                const T* sp = nullptr;
                if (tid < ntile) {
                    int gp = cid[off_parent + (code[base + tid] >> 3)];
                    if (gp >= 0) sp = L + (int64_t)gp * ld;
                }
                src[tid] = sp;
            }
        }
        int any = __syncthreads_or(tid < kNT && src[tid] != nullptr);
        if (!any) continue;
        for (int k0 = 0; k0 < P; k0 += kKC) {
#pragma unroll
            for (int e = 0; e < (kRT * kKC) / 256; ++e) {
                int idx = tid + 256 * e;
                int r = idx / kKC, kk = idx % kKC;
                int row = row0 + r, col = k0 + kk;
                As[kk][r] = (row < P && col < P) ? A[(int64_t)row * P + col] : T(0);
            }
#pragma unroll
            for (int e = 0; e < (kNT * kKC) / 256; ++e) {
                int idx = tid + 256 * e;
                int j = idx / kKC, kk = idx % kKC;
                const T* sp = src[j];
                Bs[kk][j] = (sp != nullptr && k0 + kk < P) ? sp[k0 + kk] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kKC; ++kk) {
                T a0 = As[kk][ty * 4 + 0], a1 = As[kk][ty * 4 + 1], a2 = As[kk][ty * 4 + 2],
                  a3 = As[kk][ty * 4 + 3];
                T b0 = Bs[kk][tx * 2 + 0], b1 = Bs[kk][tx * 2 + 1];
                acc[0][0] += a0 * b0; acc[0][1] += a0 * b1;
                acc[1][0] += a1 * b0; acc[1][1] += a1 * b1;
                acc[2][0] += a2 * b0; acc[2][1] += a2 * b1;
                acc[3][0] += a3 * b0; acc[3][1] += a3 * b1;
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            int row = row0 + ty * 4 + i, j = tx * 2 + jj;
            if (row < P && j < ntile) L[(int64_t)(base + j) * ld + row] = acc[i][jj];
        }
}

// ---------------------------------------------------------------------------
// L2P + P2P, one thread per sorted ion; the result is written in the
// original ion order, scaled to SI (k_e / s^2 for E, k_e / s for phi, with s
// the leaf side).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T inv_sqrt(T r2);
template <>
__device__ __forceinline__ float inv_sqrt<float>(float r2) {
    float y = rsqrtf(r2);
    return y * (1.5f - 0.5f * r2 * y * y);  // one Newton step
}
template <>
__device__ __forceinline__ double inv_sqrt<double>(double r2) {
    return 1.0 / sqrt(r2);
}


// P2P, one block per target leaf: the sources of the 27 adjacent leaves are
// staged in shared memory in the target leaf's frame; thread (target i,
// chunk c) sums every nchunk-th source; the chunk partials are combined in a
// fixed order with compensated sums (deterministic) into near[slot] =
// (E_x, E_y, E_z, phi) in leaf units (k_e = 1, leaf side = 1).
constexpr int kNfThreads = 128;
constexpr int kNfSrc = 1024;   // staged sources per pass

template <typename T>
__global__ void __launch_bounds__(kNfThreads) k_p2p(
    int D, const LevelInfo* linfo, const typename Ion<T>::rec* __restrict__ sorted,
    const uint32_t* __restrict__ code, const int32_t* __restrict__ cid_leaf,
    const int32_t* __restrict__ cstart, const int32_t* __restrict__ ccount, T* __restrict__ near) {
    using R = typename Ion<T>::rec;
    __shared__ R src[kNfSrc];
    __shared__ int nb_start[27], nb_count[27], nb_pre[28];
    __shared__ T part[kNfThreads][4];
    const int tid = threadIdx.x;
    const int lim = 1 << D;
    const int g0 = linfo->gbase[D], g1 = linfo->gbase[D + 1];
    for (int g = g0 + blockIdx.x; g < g1; g += gridDim.x) {
        const int ts = cstart[g], nt = ccount[g];
        int ix, iy, iz;
        demorton3(code[g], ix, iy, iz);
        if (tid < 27) {
            const int dx = tid / 9 - 1, dy = (tid / 3) % 3 - 1, dz = tid % 3 - 1;
            const int nx = ix + dx, ny = iy + dy, nz = iz + dz;
            int st = 0, ct = 0;
            if (nx >= 0 && ny >= 0 && nz >= 0 && nx < lim && ny < lim && nz < lim) {
                const int gn = cid_leaf[morton3(nx, ny, nz)];
                if (gn >= 0) {
                    st = cstart[gn];
                    ct = ccount[gn];
                }
            }
            nb_start[tid] = st;
            nb_count[tid] = ct;
        }
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int k = 0; k < 27; ++k) {
                nb_pre[k] = acc;
                acc += nb_count[k];
            }
            nb_pre[27] = acc;
        }
        __syncthreads();
        const int ns = nb_pre[27];
        for (int t0 = 0; t0 < nt; t0 += kNfThreads) {   // targets in blocks of 128
            const int ntb = min(kNfThreads, nt - t0);
            const int nch = kNfThreads / ntb;            // source chunks per target
            const int ti = tid % ntb, ch = tid / ntb;
            const bool active = ch < nch;
            const R me = sorted[ts + t0 + ti];
            T ex = 0, ey = 0, ez = 0, ph = 0, cex = 0, cey = 0, cez = 0, cph = 0;
            for (int s0 = 0; s0 < ns; s0 += kNfSrc) {    // sources in passes of kNfSrc
                const int nsb = min(kNfSrc, ns - s0);
                __syncthreads();
                for (int j = tid; j < nsb; j += kNfThreads) {
                    const int v = s0 + j;
                    int k = 0;  // largest k with nb_pre[k] <= v (binary search over 28 bounds)
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1)
                        if (k + step <= 26 && nb_pre[k + step] <= v) k += step;
                    const int dx = k / 9 - 1, dy = (k / 3) % 3 - 1, dz = k % 3 - 1;
                    const int slot = nb_start[k] + (v - nb_pre[k]);
                    src[j] = Ion<T>::shifted(sorted[slot], dx, dy, dz);
                }
                __syncthreads();
                if (active) {
                    // the target's own entry: leaf offset d = 0 is neighbour 13
                    const int self = nb_pre[13] + (t0 + ti) - s0;
                    // plain sums over blocks of 64 sources, compensated across blocks
                    for (int jb = ch; jb < nsb; jb += 64 * nch) {
                        const int je = min(nsb, jb + 64 * nch);
                        T px = 0, py = 0, pz = 0, pp = 0;
                        for (int j = jb; j < je; j += nch) {
                            if (j == self) continue;
                            T rx, ry, rz, q;
                            Ion<T>::sep_shifted(me, src[j], rx, ry, rz, q);
                            const T r2 = rx * rx + ry * ry + rz * rz;
                            const T ir = inv_sqrt<T>(r2);
                            const T qi = q * ir;
                            const T q3 = qi * ir * ir;
                            px += q3 * rx;
                            py += q3 * ry;
                            pz += q3 * rz;
                            pp += qi;
                        }
                        kb_add(ex, cex, px);
                        kb_add(ey, cey, py);
                        kb_add(ez, cez, pz);
                        kb_add(ph, cph, pp);
                    }
                }
            }
            part[tid][0] = ex + cex;
            part[tid][1] = ey + cey;
            part[tid][2] = ez + cez;
            part[tid][3] = ph + cph;
            __syncthreads();
            if (tid < ntb) {
                // fixed-order compensated combination of the chunk partials
                T sx = 0, sy = 0, sz = 0, sp = 0, cx = 0, cy = 0, cz = 0, cp = 0;
                for (int c = 0; c < nch; ++c) {
                    const int th = c * ntb + tid;
                    kb_add(sx, cx, part[th][0]);
                    kb_add(sy, cy, part[th][1]);
                    kb_add(sz, cz, part[th][2]);
                    kb_add(sp, cp, part[th][3]);
                }
                T* o = near + 4 * (int64_t)(ts + t0 + tid);
                o[0] = sx + cx;
                o[1] = sy + cy;
                o[2] = sz + cz;
                o[3] = sp + cp;
            }
            __syncthreads();
        }
        __syncthreads();
    }
}

// L2P (Eq. L2P) and the total field, one block per target leaf.
//   * Per leaf, four derived expansions are formed in shared memory from the
//     leaf's local expansion L: for every (n, m) a pair D_k(n, m) such that
//     the potential and the three gradient components are sums over (n, m)
//     of Re D_k Y^_n^m + Im D_k Im Y^_n^m -- the terms of l2p_eval_cols regrouped
//     by the harmonic they multiply (D_phi = w L_{n,m}; D_z = w e L_{n+1,m};
//     D_x, D_y from f L_{n+1,m+1} and g L_{n+1,m-1}).  The leaf's ~10 targets
//     share them.
//   * One target per 16-lane half-warp, lane m holding column m: the
//     diagonal Y^_m^m = prod_{k<=m} (x + i y) c_k is an inclusive prefix
//     product over the lanes (4 shuffle steps), then lane m runs its column
//     recurrence n = m..p adding four dot products per step; a fixed shuffle
//     tree sums the columns (deterministic).
// The near field (if any) is added and the field written in the original ion
// order scaled to SI (k_e / s^2 for E, k_e / s for phi, s = leaf side).
constexpr int kL2pThreads = 128;
constexpr int kPmax = (kMaxOrder + 1) * (kMaxOrder + 1);


// the derived expansions of one local expansion Lr (see k_l2p) into D4[4][P]
template <typename T>
__device__ __forceinline__ void l2p_derive(int p, const T* Lr, const HarmTables<T>& t, T (*D4)[kPmax]) {
    const int C = p + 1;
    for (int q = threadIdx.x; q < C * C; q += kL2pThreads) {
        const int nn = q / C, mm = q % C;
        if (mm > nn) continue;
        const int k = re_idx(nn, mm);
        const T w = mm > 0 ? T(2) : T(1);
        T d0r = w * Lr[k], d0i = mm > 0 ? w * Lr[k + 1] : T(0);
        T dxr = 0, dxi = 0, dyr = 0, dyi = 0, dzr = 0, dzi = 0;
        if (nn + 1 <= p) {
            const int k1 = re_idx(nn + 1, mm);
            const T e = w * t.e[nn][mm];
            dzr = e * Lr[k1];
            dzi = mm > 0 ? e * Lr[k1 + 1] : T(0);
            const int k2 = re_idx(nn + 1, mm + 1);
            const T f = t.f[nn][mm], l2r = Lr[k2], l2i = Lr[k2 + 1];
            dxr = f * l2r;
            dxi = f * l2i;
            dyr = f * l2i;
            dyi = -f * l2r;
            if (mm >= 1) {
                const int k3 = re_idx(nn + 1, mm - 1);
                const T gg = t.g[nn][mm], l3r = Lr[k3], l3i = mm - 1 > 0 ? Lr[k3 + 1] : T(0);
                dxr -= gg * l3r;
                dxi -= gg * l3i;
                dyr += gg * l3i;
                dyi -= gg * l3r;
            }
        }
        D4[0][k] = d0r;
        D4[1][k] = dxr;
        D4[2][k] = dyr;
        D4[3][k] = dzr;
        if (mm > 0) {  // for m = 0 the imaginary parts meet Im Y = 0
            D4[0][k + 1] = d0i;
            D4[1][k + 1] = dxi;
            D4[2][k + 1] = dyi;
            D4[3][k + 1] = dzi;
        }
    }
}

// column m of the potential and gradient at (x, y, z) from derived
// expansions D4; every lane of the half-warp calls it (the prefix product
// shuffles), lanes m > p return zeros.  At p = 16 the last column (m = 16,
// degree 16 only) goes to lane 15 beside its own.
template <typename T>
__device__ __forceinline__ void l2p_columns(int p, int m, unsigned hw_mask, T x, T y, T z,
                                            const HarmTables<T>& t, const T (*D4)[kPmax], T& ph,
                                            T& ax, T& ay, T& az) {
    // diagonal: inclusive prefix product of (x + i y) c_k over k = 1..m
    T dre = m == 0 ? T(1) : x * t.c[m <= p ? m : 0];
    T dim = m == 0 ? T(0) : y * t.c[m <= p ? m : 0];
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
        const T ore = __shfl_up_sync(hw_mask, dre, off, 16);
        const T oim = __shfl_up_sync(hw_mask, dim, off, 16);
        if (m >= off) {
            const T r = ore * dre - oim * dim;
            dim = ore * dim + oim * dre;
            dre = r;
        }
    }
    ph = ax = ay = az = T(0);
    if (m > p) return;
    const T r2 = x * x + y * y + z * z;
    T yr = dre, yi = dim, y1r = 0, y1i = 0;  // Y_n^m, Y_{n-1}^m
    for (int nn = m; nn <= p; ++nn) {
        if (nn == m + 1) {
            y1r = yr;
            y1i = yi;
            yr = z * t.d[m] * y1r;
            yi = z * t.d[m] * y1i;
        } else if (nn > m + 1) {
            const T a = t.a[nn][m] * z, b = t.b[nn][m] * r2;
            const T cr = a * yr - b * y1r, ci = a * yi - b * y1i;
            y1r = yr;
            y1i = yi;
            yr = cr;
            yi = ci;
        }
        const int k = re_idx(nn, m);
        ph += D4[0][k] * yr;
        ax += D4[1][k] * yr;
        ay += D4[2][k] * yr;
        az += D4[3][k] * yr;
        if (m > 0) {
            ph += D4[0][k + 1] * yi;
            ax += D4[1][k + 1] * yi;
            ay += D4[2][k + 1] * yi;
            az += D4[3][k + 1] * yi;
        }
    }
    if (p == 16 && m == 15) {
        // Y_16^16 = c_16 (x + i y) Y_15^15, the one term of column 16
        const T gr = (dre * x - dim * y) * t.c[16], gi = (dre * y + dim * x) * t.c[16];
        const int k = re_idx(16, 16);
        ph += D4[0][k] * gr + D4[0][k + 1] * gi;
        ax += D4[1][k] * gr + D4[1][k + 1] * gi;
        ay += D4[2][k] * gr + D4[2][k + 1] * gi;
        az += D4[3][k] * gr + D4[3][k + 1] * gi;
    }
}

// The same sums on an 8-lane group (p <= 15): lane j takes column j and, if
// p - j > j, column p - j, about p + 2 recurrence steps on every lane instead
// of p + 1 - m on a lane per column (on 16 lanes half the lane steps idle).
// Diagonals: lanes hold w_j = (x + i y) c_j and w_{8+j}; two inclusive prefix
// products over the group give Y_j^j and prod_{k=8..8+j} w_k, and Y_m^m for
// m >= 8 is Y_7^7 times the latter (one more rounding than the sequential
// product; every lane fetches its second diagonal by one shuffle).
template <typename T>
__device__ __forceinline__ void l2p_col_run(int p, int m, T yr, T yi, T z, T r2,
                                            const HarmTables<T>& t, const T (*D4)[kPmax], T& ph,
                                            T& ax, T& ay, T& az) {
    T y1r = 0, y1i = 0;  // Y_{n-1}^m
    for (int nn = m; nn <= p; ++nn) {
        if (nn == m + 1) {
            y1r = yr;
            y1i = yi;
            yr = z * t.d[m] * y1r;
            yi = z * t.d[m] * y1i;
        } else if (nn > m + 1) {
            const T a = t.a[nn][m] * z, b = t.b[nn][m] * r2;
            const T cr = a * yr - b * y1r, ci = a * yi - b * y1i;
            y1r = yr;
            y1i = yi;
            yr = cr;
            yi = ci;
        }
        const int k = re_idx(nn, m);
        ph += D4[0][k] * yr;
        ax += D4[1][k] * yr;
        ay += D4[2][k] * yr;
        az += D4[3][k] * yr;
        if (m > 0) {
            ph += D4[0][k + 1] * yi;
            ax += D4[1][k + 1] * yi;
            ay += D4[2][k + 1] * yi;
            az += D4[3][k + 1] * yi;
        }
    }
}

template <typename T>
__device__ __forceinline__ void l2p_columns8(int p, int j, unsigned gmask, T x, T y, T z,
                                             const HarmTables<T>& t, const T (*D4)[kPmax], T& ph,
                                             T& ax, T& ay, T& az) {
    T ar = T(1), ai = T(0), br = T(1), bi = T(0);
    if (j >= 1 && j <= p) {
        ar = x * t.c[j];
        ai = y * t.c[j];
    }
    if (8 + j <= p) {
        br = x * t.c[8 + j];
        bi = y * t.c[8 + j];
    }
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
        const T oar = __shfl_up_sync(gmask, ar, off, 8), oai = __shfl_up_sync(gmask, ai, off, 8);
        const T obr = __shfl_up_sync(gmask, br, off, 8), obi = __shfl_up_sync(gmask, bi, off, 8);
        if (j >= off) {
            const T r = oar * ar - oai * ai;
            ai = oar * ai + oai * ar;
            ar = r;
            const T s2 = obr * br - obi * bi;
            bi = obr * bi + obi * br;
            br = s2;
        }
    }
    const T d7r = __shfl_sync(gmask, ar, 7, 8), d7i = __shfl_sync(gmask, ai, 7, 8);
    const T er = d7r * br - d7i * bi, ei = d7r * bi + d7i * br;  // Y_{8+j}^{8+j}
    const int m2 = p - j;
    const int src = m2 >= 8 ? m2 - 8 : (m2 >= 0 ? m2 : 0);
    const T gar = __shfl_sync(gmask, ar, src, 8), gai = __shfl_sync(gmask, ai, src, 8);
    const T ger = __shfl_sync(gmask, er, src, 8), gei = __shfl_sync(gmask, ei, src, 8);
    ph = ax = ay = az = T(0);
    const T r2 = x * x + y * y + z * z;
    if (j <= m2) l2p_col_run<T>(p, j, ar, ai, z, r2, t, D4, ph, ax, ay, az);
    if (m2 > j)
        l2p_col_run<T>(p, m2, m2 >= 8 ? ger : gar, m2 >= 8 ? gei : gai, z, r2, t, D4, ph, ax, ay,
                       az);
}

// nlev = 2: the leaf's expansion holds its own M2L sum only, and the
// parent's complete expansion is evaluated at the ion in the parent's frame
// (equal to the L2L shift into the leaf, which shifts a truncated expansion
// exactly), saving the last L2L launch.
template <typename T, int G>
__global__ void __launch_bounds__(kL2pThreads) k_l2p(
    int64_t n, int D, int p, int ld, bool far, int nlev, const RootCube* root,
    const LevelInfo* linfo, const uint32_t* __restrict__ code, const int32_t* __restrict__ cid,
    const typename Ion<T>::rec* __restrict__ sorted, const int32_t* __restrict__ perm,
    const int32_t* __restrict__ cstart, const int32_t* __restrict__ ccount,
    const T* __restrict__ L, const T* __restrict__ near, double* E, double* phi) {
    pdl_wait();
    const int g0 = linfo->gbase[D], g1 = linfo->gbase[D + 1];
    if (g0 + (int)blockIdx.x >= g1) return;  // no leaf for this block
    constexpr int NL = sizeof(T) == 4 ? 3 : 2;  // levels evaluated at most (shared memory)
    __shared__ T sL[NL][kPmax];
    __shared__ T sD[NL][4][kPmax];  // derived expansions: phi, grad x, grad y, grad z
    __shared__ HarmTables<T> t;
    __shared__ double s_f[2];
    {
        const int* src = reinterpret_cast<const int*>(&gtab<T>());
        int* dst = reinterpret_cast<int*>(&t);
        for (int i = threadIdx.x; i < (int)(sizeof(HarmTables<T>) / sizeof(int)); i += kL2pThreads)
            dst[i] = src[i];
    }
    // SI scale factors, once per block: FP64 division is slow on this GPU,
    // and every thread computing them cost more than the L2P itself
    if (threadIdx.x == 0) {
        const double sl = root->side / (double)(1 << D);
        s_f[0] = kCoulomb / (sl * sl);
        s_f[1] = kCoulomb / sl;
    }
    __syncthreads();
    const T tE = (T)s_f[0], tP = (T)s_f[1];
    // a group of G lanes per target: G = 8 (p <= 15, l2p_columns8) or 16
    const int lane = threadIdx.x & 31, m = lane & (G - 1);
    const int slot_in_pass = threadIdx.x / G;         // target of this group
    constexpr int kPerPass = kL2pThreads / G;
    const unsigned hw_mask = (G == 8 ? 0xffu : 0xffffu) << (lane & (32 - G));
    const int P = (p + 1) * (p + 1);
    const int levs = far ? (nlev < NL ? nlev : NL) : 0;
    for (int g = g0 + blockIdx.x; g < g1; g += gridDim.x) {
        const int ts = cstart[g], nt = ccount[g];
        const uint32_t cl = code[g];
        int ix, iy, iz;
        demorton3(cl, ix, iy, iz);
        __syncthreads();  // sL, sD free from the previous leaf
        for (int lv = 0; lv < levs; ++lv) {
            // dense maps of levels 2.. concatenated: level l starts at (8^l - 64) / 7
            const int ga =
                lv == 0 ? g : cid[(((1ll << (3 * (D - lv))) - 64) / 7) + (cl >> (3 * lv))];
            for (int c = threadIdx.x; c < P; c += kL2pThreads) sL[lv][c] = L[(int64_t)ga * ld + c];
        }
        __syncthreads();
        for (int lv = 0; lv < levs; ++lv) l2p_derive<T>(p, sL[lv], t, sD[lv]);
        __syncthreads();
        for (int t0 = 0; t0 < nt; t0 += kPerPass) {
            const int ti = t0 + slot_in_pass;
            if (ti >= nt) continue;  // whole groups only: the shuffles stay within one
            T ex = 0, ey = 0, ez = 0, ph = 0;
            const typename Ion<T>::rec me = sorted[ts + ti];
            for (int lv = 0; lv < levs; ++lv) {
                T x, y, z, q;
                const int am = (1 << lv) - 1;  // the leaf's position inside the ancestor
                ion_in_ancestor(me, lv, ix & am, iy & am, iz & am, x, y, z, q);
                T cph, cax, cay, caz;
                if (G == 8) l2p_columns8<T>(p, m, hw_mask, x, y, z, t, sD[lv], cph, cax, cay, caz);
                else l2p_columns<T>(p, m, hw_mask, x, y, z, t, sD[lv], cph, cax, cay, caz);
                // level units -> leaf units: phi / 2^lv, E / 4^lv (exact)
                const T fp1 = lv == 0 ? T(1) : (lv == 1 ? T(0.5) : T(0.25)), fe1 = fp1 * fp1;
                ph += fp1 * cph;
                ex -= fe1 * cax;
                ey -= fe1 * cay;
                ez -= fe1 * caz;
            }
            // column sums: a fixed shuffle tree over the group
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                ex += __shfl_xor_sync(hw_mask, ex, off, G);
                ey += __shfl_xor_sync(hw_mask, ey, off, G);
                ez += __shfl_xor_sync(hw_mask, ez, off, G);
                ph += __shfl_xor_sync(hw_mask, ph, off, G);
            }
            if (m == 0) {
                // near + far and the SI scale in T: in FP32 one conversion per
                // stored component (FP64 instructions are scarce on this GPU)
                if (near) {
                    const T* o = near + 4 * (int64_t)(ts + ti);
                    ex += o[0];
                    ey += o[1];
                    ez += o[2];
                    ph += o[3];
                }
                const int i = perm[ts + ti];
                E[i] = (double)(tE * ex);
                E[n + i] = (double)(tE * ey);
                E[2 * n + i] = (double)(tE * ez);
                if (phi) phi[i] = (double)(tP * ph);
            }
        }
    }
}

// Direct ancestor local expansions (PT_EXPAND_DIRECT): as k_l2p, but every
// thread evaluates its columns of the M2L-only local expansions of the
// target's cells at levels lmin..D, each at the ion in that cell's frame,
// scaled to leaf units; equal to shifting them down by L2L (which shifts a
// truncated local expansion exactly) and evaluating the leaf's.
template <typename T>
__global__ void __launch_bounds__(kNfThreads) k_l2p_anc(
    int64_t n, int D, int lmin, int p, int ld, const RootCube* root, const LevelInfo* linfo,
    const uint32_t* __restrict__ code, const int32_t* __restrict__ cid,
    const typename Ion<T>::rec* __restrict__ sorted, const int32_t* __restrict__ perm,
    const int32_t* __restrict__ cstart, const int32_t* __restrict__ ccount,
    const T* __restrict__ L, const T* __restrict__ near, double* E, double* phi) {
    __shared__ T part[kNfThreads][4];
    const int tid = threadIdx.x;
    const int lim = 1 << D;
    // SI scale factors, once per block: FP64 division is slow on this GPU,
    // and every thread computing them cost more than the L2P itself
    __shared__ double s_f[2];
    if (threadIdx.x == 0) {
        const double sl = root->side / (double)lim;
        s_f[0] = kCoulomb / (sl * sl);
        s_f[1] = kCoulomb / sl;
    }
    __syncthreads();
    const double fE = s_f[0], fP = s_f[1];
    const int g0 = linfo->gbase[D], g1 = linfo->gbase[D + 1];
    for (int g = g0 + blockIdx.x; g < g1; g += gridDim.x) {
        const int ts = cstart[g], nt = ccount[g];
        const uint32_t cl = code[g];
        int ix, iy, iz;
        demorton3(cl, ix, iy, iz);
        for (int t0 = 0; t0 < nt; t0 += kNfThreads) {
            const int ntb = min(kNfThreads, nt - t0);
            const int nch = kNfThreads / ntb;
            const int ti = tid % ntb, ch = tid / ntb;
            T ex = 0, ey = 0, ez = 0, ph = 0;
            if (ch < nch) {
                const typename Ion<T>::rec me = sorted[ts + t0 + ti];
                for (int l = lmin; l <= D; ++l) {
                    const int sh = D - l, mask = (1 << sh) - 1;
                    // dense maps of levels 2.. concatenated: level l starts at (8^l - 64) / 7
                    const int ga =
                        sh == 0 ? g : cid[(((1ll << (3 * l)) - 64) / 7) + (cl >> (3 * sh))];
                    T fphi, gx, gy, gz, ux, uy, uz, uq;
                    ion_in_ancestor(me, sh, ix & mask, iy & mask, iz & mask, ux, uy, uz, uq);
                    l2p_eval_cols<T>(p, L + (int64_t)ga * ld, ux, uy, uz, tab<T>(), ch, nch, fphi,
                                     gx, gy, gz);
                    // level-l units -> leaf units: phi / 2^sh, E / 4^sh (exact)
                    const T fp1 = (T)1 / (T)(1 << sh), fe1 = fp1 * fp1;
                    ex -= fe1 * gx;
                    ey -= fe1 * gy;
                    ez -= fe1 * gz;
                    ph += fp1 * fphi;
                }
            }
            part[tid][0] = ex;
            part[tid][1] = ey;
            part[tid][2] = ez;
            part[tid][3] = ph;
            __syncthreads();
            if (tid < ntb) {
                T sx = 0, sy = 0, sz = 0, sp = 0, cx = 0, cy = 0, cz = 0, cp = 0;
                for (int c = 0; c < nch; ++c) {
                    const int th = c * ntb + tid;
                    kb_add(sx, cx, part[th][0]);
                    kb_add(sy, cy, part[th][1]);
                    kb_add(sz, cz, part[th][2]);
                    kb_add(sp, cp, part[th][3]);
                }
                double fx = (double)(sx + cx), fy = (double)(sy + cy), fz = (double)(sz + cz),
                       fp = (double)(sp + cp);
                if (near) {
                    const T* o = near + 4 * (int64_t)(ts + t0 + tid);
                    fx += (double)o[0];
                    fy += (double)o[1];
                    fz += (double)o[2];
                    fp += (double)o[3];
                }
                const int i = perm[ts + t0 + tid];
                E[i] = fE * fx;
                E[n + i] = fE * fy;
                E[2 * n + i] = fE * fz;
                if (phi) phi[i] = fP * fp;
            }
            __syncthreads();
        }
    }
}

template <typename T>
static cudaError_t run_fmm(int64_t n, int D, int phases, Workspace& ws, bool use_tc, double* E,
                           double* phi, cudaStream_t s, cudaEvent_t* ev) {
    const int p = ws.p, P = ws.P;
    DenseLayout dl = dense_layout(D);
    T* M = (T*)ws.M;
    T* L = (T*)ws.L;
    T* near = (T*)ws.near;
    const bool far = (phases & PT_PHASE_FAR) && D >= 2;
    const bool nf = (phases & PT_PHASE_NEAR) != 0;
    const int64_t leaves = n < ((int64_t)1 << (3 * D)) ? n : ((int64_t)1 << (3 * D));
    const int leaf_grid = (int)(leaves < 152 * 16 ? (leaves > 0 ? leaves : 1) : 152 * 16);
    // The M2L work list and the near field depend on the tree only: with a
    // side stream they run there, beside the main chain.
    const bool fork = far && nf && ws.side != nullptr;
    cudaStream_t sn = fork ? ws.side : s;
    // ancestor expansions of the tensor-core path directly from the ions
    // instead of the M2M / L2L shifts (an option: a cross-check of the shifts)
    const bool direct = far && use_tc && ws.expand == PT_EXPAND_DIRECT;
    // ancestor levels the leaves' L2P evaluates on the tensor-core paths: the
    // leaf, its parent and grandparent (each shift that L2P replaces is one
    // launch fewer; M2L levels start at 2)
    const int l2p_levels = use_tc ? (D - 1 < 3 ? (D - 1 > 1 ? D - 1 : 1) : 3) : 1;
    cudaError_t e;
    if (fork) {
        if ((e = cudaEventRecord(ws.ev_fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sn, ws.ev_fork, 0)) != cudaSuccess) return e;
    }
    // the M2L work list: the tensor-core schedules, and the pair-packed
    // schedule of the CUDA-core paths
    const bool pairs_simt = far && !use_tc && ws.m2l_pairs;
    if (far && (use_tc || pairs_simt)) {
        if ((e = use_tc ? launch_m2l_tc_worklist(n, D, ws, sn)
                        : launch_m2l_pairs_worklist(n, D, ws, sn)) != cudaSuccess)
            return e;
        if (fork && (e = cudaEventRecord(ws.ev_items, sn)) != cudaSuccess) return e;
    }
    // Multipoles from the ions: at the leaves, and on the tensor-core path also
    // at their parents (a parent holds about eight leaves' ions, cheaper to
    // expand directly than one more M2M launch and its reduction), or at every
    // level >= 2 in the direct mode; M2M shifts the rest up.
    const int lmin_p2m = direct ? 2 : (far && use_tc && D >= 3 ? D - 1 : D);
    // BF16x3: the multipoles' bf16 pieces, the M2L operand, are written by
    // their producers (P2M and the small-level M2M); a split pass covers the
    // levels of the tensor-core M2M (3 .. lmin_p2m - 1)
    uint16_t* Mp = use_tc && ws.tc_bf16 ? ws.M_pieces : nullptr;
    const int split_last = use_tc && ws.tc_bf16 && !direct ? lmin_p2m - 1 : 0;
    if (far && lmin_p2m < D) {
        int64_t cells = 0;
        for (int l = lmin_p2m; l <= D; ++l)
            cells += n < ((int64_t)1 << (3 * l)) ? n : ((int64_t)1 << (3 * l));
        const int grid = (int)(cells < 152 * 16 ? cells : 152 * 16);
        if ((e = launch_pdl(k_p2m_anc<T>, dim3(grid), dim3(kP2mThreads), kP2mAncIons * P * sizeof(T),
                            s, D, lmin_p2m, p, ws.ld, (const LevelInfo*)ws.linfo,
                            (const uint32_t*)ws.code, (const int32_t*)ws.leaf_start,
                            (const int32_t*)ws.leaf_of, (const typename Ion<T>::rec*)ws.sorted,
                            M, Mp)) != cudaSuccess)
            return e;
    } else if (far) {
        int grid = leaf_grid;
        k_p2m<T><<<grid, kP2mThreads, kP2mIons * P * sizeof(T), s>>>(
            D, p, ws.ld, ws.linfo, ws.cstart, ws.ccount, (const typename Ion<T>::rec*)ws.sorted, M,
            Mp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // P2P on the side stream: after P2M on the CUDA-core paths (beside their
    // M2L); on the tensor-core path after the M2L kernel, which needs every
    // SM, beside the slab reduction and the L2L launches, which use few
    // On the tensor-core paths the near field takes a third stream from the
    // fork, beside the upward pass and the work list (both latency-bound).
    const bool near_early = fork && use_tc && ws.side2 != nullptr;
    cudaStream_t snf = near_early ? ws.side2 : sn;
    auto launch_near = [&](bool after_event) -> cudaError_t {
        cudaError_t r;
        if (fork && after_event && (r = cudaStreamWaitEvent(snf, ws.ev_p2m, 0)) != cudaSuccess)
            return r;
        if (ws.kev[2] && (r = record_timing(ws.kev[2], snf)) !=
                             cudaSuccess)
            return r;
        k_p2p<T><<<leaf_grid, kNfThreads, 0, snf>>>(D, ws.linfo,
                                                   (const typename Ion<T>::rec*)ws.sorted, ws.code,
                                                   ws.cid + dl.off[D], ws.cstart, ws.ccount, near);
        if ((r = cudaGetLastError()) != cudaSuccess) return r;
        if (ws.kev[3] && (r = record_timing(ws.kev[3], snf)) !=
                             cudaSuccess)
            return r;
        if (fork && (r = cudaEventRecord(ws.ev_near, snf)) != cudaSuccess) return r;
        return cudaSuccess;
    };
    if (nf && near_early) {
        if ((e = cudaStreamWaitEvent(snf, ws.ev_fork, 0)) != cudaSuccess) return e;
        if ((e = launch_near(false)) != cudaSuccess) return e;
    }
    const bool near_late = fork && use_tc && !near_early;
    if (nf && !near_late && !near_early) {
        if (fork && (e = cudaEventRecord(ws.ev_p2m, s)) != cudaSuccess) return e;
        if ((e = launch_near(true)) != cudaSuccess) return e;
    }
    if (far) {
        for (int l = lmin_p2m - 1; l >= 2; --l) {
            if (use_tc) {
                e = level_cap(n, l) <= kShiftSmallM2M ? launch_shift_small(0, n, D, l, ws, s)
                                                      : launch_m2m_tc(n, D, l, ws, s);
                if (e != cudaSuccess) return e;
                continue;
            }
            int64_t cl = (int64_t)1 << (3 * l);
            int cells = (int)(n < cl ? n : cl);
            int g = (cells + 3) / 4;
            if (g > 152 * 16) g = 152 * 16;
            k_m2m<T><<<g, 128, 4 * P * sizeof(T), s>>>(l, P, ws.ld, ws.linfo, ws.code, ws.cid,
                                                       dl.off[l + 1], (const T*)ws.T_m2m, M);
        }
    }
    if (ev && (e = record_timing(ev[0], s)) != cudaSuccess)
        return e;
    if (far && use_tc) {
        if (fork && (e = cudaStreamWaitEvent(s, ws.ev_items, 0)) != cudaSuccess) return e;
        // L2L down to level D - l2p_levels + 1; the leaves' L2P evaluates the
        // own M2L sums of the leaf and its parent and the complete expansion
        // of the ancestor above them itself (direct mode: no L2L at all)
        if ((e = launch_m2l_tc_run(n, D, ws, direct ? 2 : D + 1 - l2p_levels, split_last, s,
                                   near_late ? ws.ev_p2m : nullptr)) != cudaSuccess)
            return e;
        if (nf && near_late && (e = launch_near(true)) != cudaSuccess) return e;
    } else if (pairs_simt) {
        if (fork && (e = cudaStreamWaitEvent(s, ws.ev_items, 0)) != cudaSuccess) return e;
        // M2L products of the work list, the per-target sums, L2L down to
        // the leaves (their L2P evaluates their own expansion)
        if ((e = launch_m2l_pairs_simt(n, D, ws, direct ? 2 : D, s)) != cudaSuccess) return e;
    } else if (far) {
        if (ws.kev[0] && (e = record_timing(ws.kev[0], s)) !=
                             cudaSuccess)
            return e;
        for (int l = 2; l <= D; ++l) {
            int64_t cl = (int64_t)1 << (3 * l);
            int cells = (int)(n < cl ? n : cl);
            dim3 grid((cells + kNT - 1) / kNT + 8, (P + kRT - 1) / kRT);
            k_m2l_simt<T><<<grid, 256, 0, s>>>(l, P, ws.ld, ws.linfo, ws.code, ws.cid, dl.off[l],
                                               l >= 3 ? dl.off[l - 1] : 0, M, L,
                                               (const T*)ws.T_m2l, (const T*)ws.T_l2l);
        }
        if (ws.kev[1] && (e = record_timing(ws.kev[1], s)) !=
                             cudaSuccess)
            return e;
    }
    if (ev && (e = record_timing(ev[1], s)) != cudaSuccess)
        return e;
    if (fork && (e = cudaStreamWaitEvent(s, ws.ev_near, 0)) != cudaSuccess) return e;
    if (direct)
        k_l2p_anc<T><<<leaf_grid, kNfThreads, 0, s>>>(
            n, D, 2, p, ws.ld, ws.root, ws.linfo, ws.code, ws.cid,
            (const typename Ion<T>::rec*)ws.sorted, ws.perm, ws.cstart, ws.ccount, L,
            nf ? near : nullptr, E, phi);
    else
        e = launch_pdl(p <= 15 ? k_l2p<T, 8> : k_l2p<T, 16>, dim3(leaf_grid), dim3(kL2pThreads),
                       0, s, n, D, p, ws.ld, far,
                       l2p_levels, (const RootCube*)ws.root,
                       (const LevelInfo*)ws.linfo, (const uint32_t*)ws.code,
                       (const int32_t*)ws.cid, (const typename Ion<T>::rec*)ws.sorted,
                       (const int32_t*)ws.perm, (const int32_t*)ws.cstart,
                       (const int32_t*)ws.ccount, (const T*)L, (const T*)(nf ? near : nullptr),
                       E, phi);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev && (e = record_timing(ev[2], s)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

cudaError_t launch_fmm_phased(int64_t n, int D, int phases, Workspace& ws, bool use_tc, double* E,
                              double* phi, cudaStream_t s, cudaEvent_t* ev) {
    if (ws.fp64) return run_fmm<double>(n, D, phases, ws, false, E, phi, s, ev);
    return run_fmm<float>(n, D, phases, ws, use_tc, E, phi, s, ev);
}

cudaError_t launch_fmm(int64_t n, int D, int phases, Workspace& ws, bool use_tc, double* E,
                       double* phi, cudaStream_t s) {
    return launch_fmm_phased(n, D, phases, ws, use_tc, E, phi, s, nullptr);
}

// M2M into level l (mode 0) or L2L into level l (mode 1) of a small level of
// the tensor-core paths on the CUDA cores (k_shift_rows; FP32 plans).
cudaError_t launch_shift_small(int mode, int64_t n, int D, int l, Workspace& ws, cudaStream_t s) {
    const int P = ws.P;
    const DenseLayout dl = dense_layout(D);
    const unsigned rg = (unsigned)((P + kShRows - 1) / kShRows);
    const int64_t cl = (int64_t)1 << (3 * l);
    const int64_t cells = n < cl ? n : cl;
    if (mode == 0) {
        const int64_t ch = (cells + ShCells<0>::v - 1) / ShCells<0>::v;
        return launch_pdl(k_shift_rows<float, 0>, dim3(rg, (unsigned)(ch < 16 ? ch : 16)),
                          dim3(kShThreads), shift_rows_smem<float, 0>(P), s, l, P, ws.ld,
                          (const LevelInfo*)ws.linfo, (const uint32_t*)ws.code,
                          (const int32_t*)ws.cid, dl.off[l + 1], (const float*)ws.T_m2m,
                          (float*)ws.M, ws.tc_bf16 ? ws.M_pieces : (uint16_t*)nullptr);
    }
    // per octant: runs of 16 children, a few blocks per octant
    const int64_t ch = (cells + ShCells<1>::v * 8 - 1) / (ShCells<1>::v * 8);
    return launch_pdl(k_shift_rows<float, 1>, dim3(rg, 8, (unsigned)(ch < 4 ? (ch > 0 ? ch : 1) : 4)),
                      dim3(kShThreads), shift_rows_smem<float, 1>(P), s, l, P, ws.ld,
                      (const LevelInfo*)ws.linfo, (const uint32_t*)ws.code, (const int32_t*)ws.cid,
                      dl.off[l - 1], (const float*)ws.T_l2l, (float*)ws.L, (uint16_t*)nullptr);
}

// ---------------------------------------------------------------------------
// Interaction counts of the current tree (for algorithmic work accounting).
// ---------------------------------------------------------------------------
__global__ void k_tree_stats(int D, const LevelInfo* linfo, const uint32_t* __restrict__ code,
                             const int32_t* __restrict__ cid, DenseLayout dl,
                             const int32_t* __restrict__ ccount, unsigned long long* st) {
    const int lmin = dl.lmin;
    const int g0 = linfo->gbase[lmin], g1 = linfo->gbase[D + 1];
    unsigned long long m2l = 0, p2p = 0, shifts = 0;
    for (int g = g0 + blockIdx.x * blockDim.x + threadIdx.x; g < g1; g += gridDim.x * blockDim.x) {
        int l = lmin;
        while (l < D && g >= linfo->gbase[l + 1]) ++l;
        int ix, iy, iz;
        demorton3(code[g], ix, iy, iz);
        const int lim = 1 << l;
        if (l >= 2) {
            const int oct = code[g] & 7;
            for (int t = 0; t < 189; ++t) {
                int opi = c_m2l_off[oct][t];
                int sx = ix - (opi / 49 - 3), sy = iy - ((opi / 7) % 7 - 3), sz = iz - (opi % 7 - 3);
                if (sx < 0 || sy < 0 || sz < 0 || sx >= lim || sy >= lim || sz >= lim) continue;
                if (cid[dl.off[l] + morton3(sx, sy, sz)] >= 0) ++m2l;
            }
        }
        if (l >= 3) ++shifts;
        if (l == D) {
            long long cnt = ccount[g], nb = 0;
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        int nx = ix + dx, ny = iy + dy, nz = iz + dz;
                        if (nx < 0 || ny < 0 || nz < 0 || nx >= lim || ny >= lim || nz >= lim) continue;
                        int gn = cid[dl.off[D] + morton3(nx, ny, nz)];
                        if (gn >= 0) nb += ccount[gn];
                    }
            p2p += (unsigned long long)(cnt * nb - cnt);
        }
    }
    atomicAdd(&st[0], m2l);
    atomicAdd(&st[1], p2p);
    atomicAdd(&st[2], shifts);
}

cudaError_t launch_tree_stats(int64_t n, int D, Workspace& ws, int64_t* out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ws.stats, 0, sizeof(unsigned long long) * 8, s);
    if (e != cudaSuccess) return e;
    DenseLayout dl = dense_layout(D);
    k_tree_stats<<<152, 256, 0, s>>>(D, ws.linfo, ws.code, ws.cid, dl, ws.ccount, ws.stats);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unsigned long long h[3];
    LevelInfo li;
    if ((e = cudaMemcpyAsync(h, ws.stats, sizeof h, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&li, ws.linfo, sizeof li, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    out[0] = n;
    out[1] = D;
    out[2] = li.gbase[D + 1] - li.gbase[D];
    out[3] = D >= 2 ? li.gbase[D + 1] - li.gbase[2] : 0;
    out[4] = (int64_t)h[0];
    out[5] = (int64_t)h[1];
    out[6] = (int64_t)h[2];
    out[7] = (int64_t)h[2];
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Direct O(N^2) field in FP64 (Eq. hamiltonian), shared-memory source tiles,
// Neumaier-compensated accumulation.
// ---------------------------------------------------------------------------
struct Neu {
    double s = 0, c = 0;
    __device__ __forceinline__ void add(double v) {
        double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ double val() const { return s + c; }
};

__global__ void __launch_bounds__(256) k_direct(int64_t n, const double* __restrict__ pos,
                                                const double* __restrict__ q, double* E,
                                                double* phi) {
    __shared__ double4_32a tile[256];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double xi = 0, yi = 0, zi = 0;
    if (i < n) { xi = pos[i]; yi = pos[n + i]; zi = pos[2 * n + i]; }
    Neu ax, ay, az, ap;
    for (int64_t t0 = 0; t0 < n; t0 += 256) {
        int64_t j = t0 + threadIdx.x;
        tile[threadIdx.x] = j < n ? make_double4_32a(pos[j], pos[n + j], pos[2 * n + j], q[j])
                                  : make_double4_32a(0, 0, 0, 0);
        __syncthreads();
        int cnt = (int)(n - t0 < 256 ? n - t0 : 256);
        for (int k = 0; k < cnt; ++k) {
            if (t0 + k == i) continue;
            double4_32a o = tile[k];
            double dx = xi - o.x, dy = yi - o.y, dz = zi - o.z;
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double ir = 1.0 / r;
            double w = o.w * ir / r2;
            ax.add(w * dx);
            ay.add(w * dy);
            az.add(w * dz);
            ap.add(o.w * ir);
        }
        __syncthreads();
    }
    if (i < n) {
        E[i] = kCoulomb * ax.val();
        E[n + i] = kCoulomb * ay.val();
        E[2 * n + i] = kCoulomb * az.val();
        if (phi) phi[i] = kCoulomb * ap.val();
    }
}

cudaError_t launch_direct(int64_t n, const double* pos, const double* q, double* E, double* phi,
                          cudaStream_t s) {
    int grid = (int)((n + 255) / 256);
    k_direct<<<grid > 0 ? grid : 1, 256, 0, s>>>(n, pos, q, E, phi);
    return cudaGetLastError();
}

cudaError_t upload_harmonic_tables() {
    static HarmTables<double> hd;
    static HarmTables<float> hf;
    static int16_t off[8][189];
    static bool filled = false;
    if (!filled) {
        fill_harm_tables(hd);
        fill_harm_tables(hf);
        host_m2l_offsets(off);
        filled = true;
    }
    cudaError_t e = cudaMemcpyToSymbol(c_tab_d, &hd, sizeof hd);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tab_f, &hf, sizeof hf);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tab_d, &hd, sizeof hd);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tab_f, &hf, sizeof hf);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_m2l_off, off, sizeof off);
    const int pmax = (kMaxOrder + 1) * (kMaxOrder + 1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_p2m<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kP2mIons * pmax * (int)sizeof(double));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_p2m<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kP2mIons * pmax * (int)sizeof(float));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_p2m_anc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kP2mAncIons * pmax * (int)sizeof(double));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_p2m_anc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kP2mAncIons * pmax * (int)sizeof(float));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_shift_rows<float, 0>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)shift_rows_smem<float, 0>(pmax));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_shift_rows<float, 1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)shift_rows_smem<float, 1>(pmax));
    return e;
}

}  // namespace pt
