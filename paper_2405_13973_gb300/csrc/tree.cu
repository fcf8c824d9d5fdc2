// tree.cu -- octree construction on the GPU (Sec. 2.3.2: "the smallest cube
// containing all N ions is found ... recursively divided into octants").
//
// One uniform-depth octree per evaluation, rebuilt from the positions:
//   1. bounding cube (min/max reduction, last-block finalisation);
//   2. leaf Morton keys and a histogram over the 8^D leaf cells;
//   3. exclusive scan of the histogram -> first slot of every leaf;
//   4. scatter ions to slots (a one-digit radix / counting sort on the key);
//   5. compaction of the non-empty cells of every level (octant-major order
//      so that M2L tiles share one octant) into global compact ids;
//   6. per leaf: order its ions by original index (deterministic), gather the
//      leaf-relative scaled coordinates and charges into sorted slots.
// All grids are sized by the plan's capacities, not by device-side counts, so
// the whole sequence can be captured in a CUDA graph.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "harmonics.cuh"
#include "internal.h"
#include "bbox.cuh"

namespace pt {

DenseLayout dense_layout(int D) {
    DenseLayout d;
    d.D = D;
    d.lmin = D < 2 ? D : 2;
    int64_t o = 0;
    for (int l = 0; l <= D + 1; ++l) {
        d.off[l] = o;
        if (l >= d.lmin && l <= D) o += (int64_t)1 << (3 * l);
    }
    d.total = o;
    return d;
}

// ---------------------------------------------------------------------------
// 1. bounding cube
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBboxThreads) k_bbox(const double* __restrict__ x,
                                                      const double* __restrict__ y,
                                                      const double* __restrict__ z, int64_t n,
                                                      int64_t per, unsigned long long* acc,
                                                      unsigned* ticket, RootCube* root, int* err) {
    BboxAcc t;
    const int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) t.add(x[i], y[i], z[i]);
    bbox_commit(t, acc, ticket, root, err);
}

cudaError_t launch_bbox(const double* x, const double* y, const double* z, int64_t n,
                        Workspace& ws, cudaStream_t s) {
    const IonSplit sp = bbox_split(n, ws);
    k_bbox<<<sp.grid, kBboxThreads, 0, s>>>(x, y, z, n, sp.per, ws.bbox_acc, ws.ticket, ws.root,
                                            ws.err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 2. leaf keys and histogram
// ---------------------------------------------------------------------------
__device__ __forceinline__ int leaf_coord(double v, double lo, double side, double scale, int m) {
    double t = __dmul_rn(__ddiv_rn(__dsub_rn(v, lo), side), scale);
    double f = floor(t);
    if (!(f >= 0.0)) return 0;
    if (f > (double)m) return m;
    return (int)f;
}

__global__ void k_keys(const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, int64_t n, int64_t per, int D,
                       const RootCube* root, uint32_t* key, uint32_t* rank, int32_t* leaf_count) {
    pdl_wait();
    const double lo0 = root->lo[0], lo1 = root->lo[1], lo2 = root->lo[2], side = root->side;
    const double scale = (double)(1 << D);
    const int m = (1 << D) - 1;
    const int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        uint32_t k = morton3(leaf_coord(x[i], lo0, side, scale, m),
                             leaf_coord(y[i], lo1, side, scale, m),
                             leaf_coord(z[i], lo2, side, scale, m));
        key[i] = k;
        rank[i] = (uint32_t)atomicAdd(&leaf_count[k], 1);
    }
}

// ---------------------------------------------------------------------------
// 3./5. three-phase exclusive scans with on-the-fly inputs
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = kScanTile / kScanThreads;

__device__ __forceinline__ int block_exclusive_scan(int v, int& total) {
    __shared__ int warp_tot[kScanThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    int before = wid > 0 ? warp_tot[wid - 1] : 0;
    total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

template <class Src>
__global__ void k_scan_reduce(Src src, int64_t total, int32_t* block_sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
        if (i < total) acc += src.load(i);
    }
    int tot;
    block_exclusive_scan(acc, tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_top(int32_t* block_sums, int nb) {
    int carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        int i = base + threadIdx.x;
        int v = i < nb ? block_sums[i] : 0;
        int tot;
        int ex = block_exclusive_scan(v, tot);
        if (i < nb) block_sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) block_sums[nb] = carry;
}

template <class Src>
__global__ void k_scan_apply(Src src, int64_t total, const int32_t* block_sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int vals[kScanItems];
    int acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        vals[k] = i < total ? src.load(i) : 0;
        acc += vals[k];
    }
    int tot;
    int ex = block_exclusive_scan(acc, tot) + block_sums[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < total) src.store(i, ex, vals[k]);
        ex += vals[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) src.finish(block_sums[gridDim.x]);
}

// Small scans in one block of 1024 threads, tile by tile with a carry: one
// launch instead of three (the three-phase scan of a few thousand cells is
// all launch latency).
constexpr int kScan1Threads = 1024;
constexpr int kScan1Items = 8;
constexpr int64_t kScan1Max = 65536;

template <class Src>
__device__ __forceinline__ void scan_single_body(const Src& src, int64_t total) {
    __shared__ int warp_tot[kScan1Threads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int carry = 0;
    for (int64_t t0 = 0; t0 < total; t0 += (int64_t)kScan1Threads * kScan1Items) {
        const int64_t base = t0 + (int64_t)threadIdx.x * kScan1Items;
        int vals[kScan1Items];
        int acc = 0;
#pragma unroll
        for (int k = 0; k < kScan1Items; ++k) {  // all loads in flight at once
            const int64_t i = base + k;
            vals[k] = i < total ? src.load(i) : 0;
        }
#pragma unroll
        for (int k = 0; k < kScan1Items; ++k) acc += vals[k];
        int x = acc;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        int ex = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + x - acc;
        const int tot = warp_tot[kScan1Threads / 32 - 1];
#pragma unroll
        for (int k = 0; k < kScan1Items; ++k) {
            const int64_t i = base + k;
            if (i < total) src.store(i, ex, vals[k]);
            ex += vals[k];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) src.finish(carry);
}

template <class Src>
__global__ void __launch_bounds__(kScan1Threads) k_scan_single(Src src, int64_t total) {
    scan_single_body(src, total);
}

// Two dependent scans in one launch on a cluster of kScanCtas CTAs (the work
// of one block spread over eight SMs): each CTA scans its contiguous
// share in registers, the CTAs' totals are exchanged through distributed
// shared memory after a cluster barrier (each CTA adds those of the lower
// ranks), and a second barrier makes every CTA's stores visible to the whole
// cluster before the next scan loads them (through L2: __ldcg).
constexpr int kScanCtas = 8;
constexpr int kScanCtaThreads = 1024;
constexpr int kScanCtaItems = kScan1Max / (kScanCtas * kScanCtaThreads);

template <class Src>
__device__ __forceinline__ void scan_cluster_body(const Src& src, int64_t total, int* warp_tot,
                                                  int* cta_tot, int* s_tot) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), nr = (int)cl.num_blocks();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t share = (total + nr - 1) / nr;
    const int64_t b0 = min(total, (int64_t)rank * share), b1 = min(total, b0 + share);
    const int ipt = (int)((b1 - b0 + kScanCtaThreads - 1) / kScanCtaThreads);
    const int64_t base = b0 + (int64_t)threadIdx.x * ipt;
    int vals[kScanCtaItems];
    int acc = 0;
#pragma unroll
    for (int k = 0; k < kScanCtaItems; ++k) {  // all loads in flight at once
        const int64_t i = base + k;
        vals[k] = (k < ipt && i < b1) ? src.load(i) : 0;
    }
#pragma unroll
    for (int k = 0; k < kScanCtaItems; ++k) acc += vals[k];
    int x = acc;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    int ex = (wid > 0 ? warp_tot[wid - 1] : 0) + x - acc;
    if (threadIdx.x == 0) *cta_tot = warp_tot[kScanCtaThreads / 32 - 1];
    cl.sync();  // every CTA's total is in its shared memory
    if (threadIdx.x < nr) s_tot[threadIdx.x] = *cl.map_shared_rank(cta_tot, (unsigned)threadIdx.x);
    __syncthreads();
    int all = 0;
    for (int r = 0; r < nr; ++r) {
        if (r == rank) ex += all;
        all += s_tot[r];
    }
#pragma unroll
    for (int k = 0; k < kScanCtaItems; ++k) {
        const int64_t i = base + k;
        if (k < ipt && i < b1) src.store(i, ex, vals[k]);
        ex += vals[k];
    }
    if (rank == nr - 1 && threadIdx.x == 0) src.finish(all);
    cl.sync();  // the stores are visible cluster-wide; cta_tot and s_tot are free again
}

template <class SrcA, class SrcB>
__global__ void __launch_bounds__(kScanCtaThreads) k_scan_cluster2(SrcA a, int64_t total_a, SrcB b,
                                                                  int64_t total_b) {
    __shared__ int warp_tot[kScanCtaThreads / 32];
    __shared__ int cta_tot, s_tot[kScanCtas];
    pdl_wait();
    scan_cluster_body(a, total_a, warp_tot, &cta_tot, s_tot);
    scan_cluster_body(b, total_b, warp_tot, &cta_tot, s_tot);
}

// a cluster launch of kScanCtas CTAs, programmatic (see launch_pdl)
template <typename... KArgs, typename... Args>
static cudaError_t launch_scan_cluster(void (*k)(KArgs...), cudaStream_t s, Args... args) {
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kScanCtas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kScanCtas);
    cfg.blockDim = dim3(kScanCtaThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

template <class Src>
static cudaError_t run_scan(Src src, int64_t total, Workspace& ws, cudaStream_t s) {
    if (total <= kScan1Max) {
        k_scan_single<<<1, kScan1Threads, 0, s>>>(src, total);
        return cudaGetLastError();
    }
    int nb = (int)((total + kScanTile - 1) / kScanTile);
    if (nb < 1) nb = 1;
    if (nb + 1 > ws.block_sums_cap) return cudaErrorInvalidValue;
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(src, total, ws.block_sums);
    k_scan_top<<<1, kScanThreads, 0, s>>>(ws.block_sums, nb);
    k_scan_apply<<<nb, kScanThreads, 0, s>>>(src, total, ws.block_sums);
    return cudaGetLastError();
}

// Leaf histogram -> first slot of every leaf (leaf_start[8^D] = n).  The
// histogram is zeroed as it is read (every element is stored by the thread
// that loaded it, after the load): it is zero again for the next k_keys.
struct LeafCountScan {
    int32_t* count;
    int32_t* start;
    int64_t ncells;
    __device__ int load(int64_t i) const { return count[i]; }
    __device__ void store(int64_t i, int ex, int) const {
        start[i] = ex;
        count[i] = 0;
    }
    __device__ void finish(int tot) const { start[ncells] = tot; }
};

// Non-empty flags of levels lmin..D in octant-major order -> compact ids.
struct CellCompaction {
    const int32_t* leaf_start;
    int32_t* cid;
    uint32_t* code;
    int32_t* cstart;
    int32_t* ccount;
    LevelInfo* linfo;
    int D, lmin;
    int64_t off[kMaxDepth + 2];

    __device__ void locate(int64_t v, int& l, uint32_t& c) const {
        l = lmin;
        while (l < D && v >= off[l + 1]) ++l;
        int64_t j = v - off[l];
        if (l == 0) { c = 0; return; }
        // j = oct * 8^(l-1) + par (octant-major order)
        const int sh = 3 * (l - 1);
        uint32_t oct = (uint32_t)(j >> sh), par = (uint32_t)(j & (((int64_t)1 << sh) - 1));
        c = (par << 3) | oct;
    }
    __device__ int range(int l, uint32_t c, int& first) const {
        int sh = 3 * (D - l);
        int64_t a = (int64_t)c << sh, b = ((int64_t)c + 1) << sh;
        // written by the leaf scan of the same launch, possibly by another
        // CTA of the cluster: read through L2
        first = __ldcg(&leaf_start[a]);
        return __ldcg(&leaf_start[b]) - first;
    }
    __device__ int load(int64_t v) const {
        int l;
        uint32_t c;
        locate(v, l, c);
        int f;
        return range(l, c, f) > 0 ? 1 : 0;
    }
    __device__ void store(int64_t v, int ex, int flag) const {
        int l;
        uint32_t c;
        locate(v, l, c);
        int64_t j = v - off[l];
        cid[off[l] + c] = flag ? ex : -1;
        if (flag) {
            code[ex] = c;
            if (l == D) {
                int f;
                int cnt = range(l, c, f);
                cstart[ex] = f;
                ccount[ex] = cnt;
            }
        }
        if (j == 0) linfo->gbase[l] = ex;
        if (l >= 1) {
            const int sh = 3 * (l - 1);
            if ((j & (((int64_t)1 << sh) - 1)) == 0) linfo->oct_start[l][j >> sh] = ex;
        } else {
            for (int o = 0; o < 8; ++o) linfo->oct_start[0][o] = ex;
        }
        if (v == off[l + 1] - 1 || (l == D && v == off[D + 1] - 1)) {
            linfo->oct_start[l][8] = ex + flag;
            if (l == D) linfo->gbase[D + 1] = ex + flag;
        }
    }
    __device__ void finish(int) const {}
};

// ---------------------------------------------------------------------------
// 4./6. scatter and per-leaf ordering + gather
// ---------------------------------------------------------------------------
__global__ void k_scatter(const uint32_t* __restrict__ key, const uint32_t* __restrict__ rank,
                          const int32_t* __restrict__ leaf_start, int64_t n, int32_t* perm_tmp) {
    pdl_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        perm_tmp[leaf_start[key[i]] + rank[i]] = (int32_t)i;
}

// Sorted ion record: FP64 path (u_x, u_y, u_z, q) in double; FP32 paths
// store u as 30-bit fixed point, u_i = round(u * 2^30) clamped to
// [-2^29, 2^29 - 1], so that the pair differences of the near field are
// formed exactly in integers (see fmm.cu), and q as float bits.
template <typename T4>
__device__ __forceinline__ T4 make4(double a, double b, double c, double d);
template <>
__device__ __forceinline__ int4 make4<int4>(double a, double b, double c, double d) {
    auto fx = [](double u) {
        double r = rint(u * 1073741824.0);
        r = fmin(fmax(r, -536870912.0), 536870911.0);
        return (int)r;
    };
    return make_int4(fx(a), fx(b), fx(c), __float_as_int((float)d));
}
template <>
__device__ __forceinline__ double4_32a make4<double4_32a>(double a, double b, double c, double d) {
    return make_double4_32a(a, b, c, d);
}

// One thread per sorted slot: the slot's ion (in arrival order within its
// leaf) takes the rank of its index among the leaf's ions, so every leaf
// lists its ions by original index (deterministic whatever the atomic order
// of k_keys); the leaf's ions are read from the few cache lines the
// neighbouring threads share.
template <typename T4>
__global__ void k_leaf_gather(const double* __restrict__ x, const double* __restrict__ y,
                              const double* __restrict__ z, const double* __restrict__ q, int64_t n,
                              int64_t per, int D, const RootCube* root,
                              const uint32_t* __restrict__ key,
                              const int32_t* __restrict__ leaf_start,
                              const int32_t* __restrict__ cid_leaf,
                              const int32_t* __restrict__ perm_tmp, int32_t* perm,
                              int32_t* slot_of, int32_t* leaf_of, T4* sorted) {
    pdl_wait();
    const double lo0 = root->lo[0], lo1 = root->lo[1], lo2 = root->lo[2], side = root->side;
    const double scale = (double)(1 << D);
    const int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int idx = perm_tmp[i];
        const uint32_t c = key[idx];
        const int s = leaf_start[c], k = leaf_start[c + 1] - s;
        int r = 0;
        for (int u = 0; u < k; ++u) r += (perm_tmp[s + u] < idx);
        const int slot = s + r;
        int ix, iy, iz;
        demorton3(c, ix, iy, iz);
        perm[slot] = idx;
        slot_of[idx] = slot;
        leaf_of[slot] = cid_leaf[c];
        const double ux = (x[idx] - lo0) / side * scale - (ix + 0.5);
        const double uy = (y[idx] - lo1) / side * scale - (iy + 0.5);
        const double uz = (z[idx] - lo2) / side * scale - (iz + 0.5);
        sorted[slot] = make4<T4>(ux, uy, uz, q[idx]);
    }
}

cudaError_t launch_tree(int64_t n, const double* x, const double* y, const double* z,
                        const double* q, int D, Workspace& ws, cudaStream_t s) {
    const int64_t ncells = (int64_t)1 << (3 * D);
    // the leaf histogram is zero here (zeroed at allocation and by its scans)
    // the per-ion passes (keys, gather) do FP64 divisions: equal shares of
    // the ions per SM (ion_split); the scatter is integer work
    const int grid_ions = (int)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8);
    const IonSplit sp = ion_split(n, 128, ws.sms, (int64_t)1 << 30);
    cudaError_t e = launch_pdl(k_keys, dim3(sp.grid), dim3(128), 0, s, x, y, z, n, sp.per, D,
                               (const RootCube*)ws.root, ws.key, ws.rank, ws.leaf_count);
    if (e != cudaSuccess) return e;
    LeafCountScan ls{ws.leaf_count, ws.leaf_start, ncells};
    DenseLayout dl = dense_layout(D);
    CellCompaction cc;
    cc.leaf_start = ws.leaf_start;
    cc.cid = ws.cid;
    cc.code = ws.code;
    cc.cstart = ws.cstart;
    cc.ccount = ws.ccount;
    cc.linfo = ws.linfo;
    cc.D = D;
    cc.lmin = dl.lmin;
    for (int l = 0; l < kMaxDepth + 2; ++l) cc.off[l] = dl.off[l];
    // the cell compaction reads only the leaf starts: both scans in one
    // cluster launch when they fit, then the scatter
    if (ncells <= kScan1Max && dl.total <= kScan1Max) {
        if ((e = launch_scan_cluster(k_scan_cluster2<LeafCountScan, CellCompaction>, s, ls,
                                     ncells, cc, dl.total)) != cudaSuccess)
            return e;
    } else {
        if ((e = run_scan(ls, ncells, ws, s)) != cudaSuccess) return e;
        if ((e = run_scan(cc, dl.total, ws, s)) != cudaSuccess) return e;
    }
    const int g = grid_ions > 0 ? grid_ions : 1;
    if ((e = launch_pdl(k_scatter, dim3(g), dim3(256), 0, s, (const uint32_t*)ws.key,
                        (const uint32_t*)ws.rank, (const int32_t*)ws.leaf_start, n,
                        ws.perm_tmp)) != cudaSuccess)
        return e;
    const int32_t* cid_leaf = ws.cid + dl.off[D];
    if (ws.fp64)
        return launch_pdl(k_leaf_gather<double4_32a>, dim3(sp.grid), dim3(128), 0, s, x, y, z, q,
                          n, sp.per, D,
                          (const RootCube*)ws.root, (const uint32_t*)ws.key,
                          (const int32_t*)ws.leaf_start, cid_leaf, (const int32_t*)ws.perm_tmp,
                          ws.perm, ws.slot_of, ws.leaf_of, (double4_32a*)ws.sorted);
    return launch_pdl(k_leaf_gather<int4>, dim3(sp.grid), dim3(128), 0, s, x, y, z, q, n, sp.per,
                      D,
                      (const RootCube*)ws.root, (const uint32_t*)ws.key,
                      (const int32_t*)ws.leaf_start, cid_leaf, (const int32_t*)ws.perm_tmp,
                      ws.perm, ws.slot_of, ws.leaf_of, (int4*)ws.sorted);
}

// ---------------------------------------------------------------------------
// Automatic depth: non-empty cell counts of every level up to depth_max.
// ---------------------------------------------------------------------------
__global__ void k_level_nonempty(const int32_t* __restrict__ leaf_start, int Dm,
                                 int32_t* counts) {
    // thread per (level, cell) pair over levels 0..Dm; per-thread counts per
    // level, summed over the warp before one atomic per level and warp
    int64_t total = 0;
    for (int l = 0; l <= Dm; ++l) total += (int64_t)1 << (3 * l);
    int mine[kMaxDepth + 1];
#pragma unroll
    for (int l = 0; l <= kMaxDepth; ++l) mine[l] = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < total;
         v += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        int64_t base = 0;
        while (v >= base + ((int64_t)1 << (3 * l))) { base += (int64_t)1 << (3 * l); ++l; }
        const int64_t c = v - base;
        const int sh = 3 * (Dm - l);
        const int ne = leaf_start[(c + 1) << sh] - leaf_start[c << sh] > 0 ? 1 : 0;
#pragma unroll
        for (int k = 0; k <= kMaxDepth; ++k) mine[k] += (k == l) ? ne : 0;
    }
#pragma unroll
    for (int l = 0; l <= kMaxDepth; ++l) {
        const int w = __reduce_add_sync(0xffffffffu, mine[l]);
        if ((threadIdx.x & 31) == 0 && w > 0) atomicAdd(&counts[l], w);
    }
}

cudaError_t launch_level_counts(int64_t n, const double* x, const double* y, const double* z,
                                int Dm, Workspace& ws, int32_t* host_counts, cudaStream_t s) {
    cudaError_t e = launch_bbox(x, y, z, n, ws, s);
    if (e != cudaSuccess) return e;
    const int64_t ncells = (int64_t)1 << (3 * Dm);
    const IonSplit sk = ion_split(n, 128, ws.sms, (int64_t)1 << 30);
    k_keys<<<sk.grid, 128, 0, s>>>(x, y, z, n, sk.per, Dm, ws.root, ws.key, ws.rank,
                                   ws.leaf_count);
    LeafCountScan ls{ws.leaf_count, ws.leaf_start, ncells};
    if ((e = run_scan(ls, ncells, ws, s)) != cudaSuccess) return e;
    int32_t* d_counts = (int32_t*)ws.block_sums;  // reuse scratch after the scan
    if ((e = cudaMemsetAsync(d_counts, 0, sizeof(int32_t) * (kMaxDepth + 1), s)) != cudaSuccess)
        return e;
    k_level_nonempty<<<152 * 4, 256, 0, s>>>(ws.leaf_start, Dm, d_counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(host_counts, d_counts, sizeof(int32_t) * (Dm + 1),
                             cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(s);
}

}  // namespace pt
