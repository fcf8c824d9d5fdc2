// m2l_tc.cu -- M2L (Eq. FMM_local) on the 5th-generation tensor cores.
//
// Problem: for every target cell t of level l >= 2 and each of the 189
// source offsets o of its octant, L_t += T_o M_{t-o} (Sec. 2.3.2: the
// children of the parent's neighbours that are not neighbours of t).  Cells
// of one (level, octant) share the 189 operators, so a tile of 128 such
// targets is, per offset, one dense product
//     D[128 x N] += A[128 x K] * B[K x N],
//     A row r = M of the source of target r (gathered; zero if empty),
//     B = T_o^T (K = input coefficients, N = output coefficients).
//
// Precision: tensor-core inputs are split into pieces whose products, summed
// in FP32 in tensor memory, rebuild the FP32 (or FP64) operands.
//   3xTF32: x = hi + lo, hi = rna_tf32(x), lo = rna_tf32(x - hi) (22 of
//     FP32's 24 bits); D += A_hi B_hi + A_hi B_lo + A_lo B_hi.  Each product
//     is good to about 2^-21.
//   BF16x3: x = hi + mid + lo with three round-to-nearest bf16 pieces (8 bits
//     each: an FP32 value exactly, an FP64 operator to 2^-24); D += the six
//     products whose piece orders sum to at most 2 (hh, hm, mh, hl, lh, mm).
//     The dropped terms are below 2^-25 of the product, so each product is
//     as good as an FP32 multiply; the BF16 rate is twice the TF32 rate, so
//     six BF16 products take the tensor time of three TF32 ones.
//
// Data movement: the operators are split and laid out on the host in the
// swizzled K-major shared-memory image of each 32-wide K chunk (128-byte
// rows and swizzle for TF32, 64-byte rows and swizzle for BF16), so one
// cp.async.bulk per (offset, chunk) brings every piece of B.  A rows are
// gathered by 256 producer threads: for the BF16x3 M2L, M is split into its
// bf16 pieces once per step (k_split_m) and the producers copy 16-byte units
// of the pieces by cp.async.cg straight into the swizzled stage; in the
// other modes they copy FP32 rows into a per-thread ring, split them and
// store the pieces.  Up to four stages: the loads of later chunks overlap the
// MMAs of chunk i.  One thread issues tcgen05.mma (M = 128, N = P rounded up
// to 16, 32 bytes of K per instruction) and commits to an mbarrier per stage.
//
// The same gathered product serves the two other dense translations:
//   M2M (upward pass): a tile of parents, 8 terms (child octants), A = the
//     children's M, B = the octant's M2M operator;
//   L2L (downward pass): a tile of children of one octant, 1 term, A = the
//     parent's L, B = the octant's L2L operator, and the epilogue adds the
//     child's own M2L result (and the split partials).
// Parallelism: one persistent M2L launch (a CTA per SM) covers every level
// and walks a device work list: per tile its non-empty offsets (k_tc_plan)
// cut into runs of at most four (k_tc_items; the tensor-core accumulation
// rounds with a bias that grows with the products summed into one
// accumulator).  The first run of a tile writes L, the others write partial
// slabs that k_tc_reduce_tiles adds in run order (deterministic); then the
// L2L launches shift level by level.
//
// Every wait on an mbarrier is bounded: on expiry the CTA records
// ERR_TIMEOUT, stops issuing, waits (bounded) for its own work in flight,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "bf16split.cuh"
#include "harmonics.cuh"
#include "internal.h"
#include "m2l_pairs.h"

namespace pt {

namespace {

constexpr int kMaxStages = 4;
constexpr int kTcRows = 128;
constexpr int kMaxSplits = 8;    // M2M: CTAs per tile (one per child octant at most)
constexpr int kChainCap = 4;     // M2L: at most this many offsets per work item
// above this many ions, at most kChainCapLarge: the accumulation error grows
// with the crystal (1e6 ions, BF16x3, p = 12: force error 1.00e-6 with runs
// of 4 offsets, 9.6e-7 with runs of 3, 5 % slower)
constexpr int64_t kChainLargeIons = 262144;
constexpr int kChainCapLarge = 3;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

struct TcGeom {
    int P = 0, Kpad = 0, Npad = 0, kchunks = 0, tmem_cols = 0, acc_cols = 0, pieces = 2,
        row_bytes = 128;
    int a_bytes = 0, b_bytes = 0, stage_bytes = 0, smem_bytes = 0, stages = 2, raw = 2;
    // BF16 pair-packed epilogue: the accumulators pass through shared memory
    // (the producers' raw ring, unused in that mode) in two column halves of
    // epi_half columns, rows epi_stride floats apart
    int epi_half = 0, epi_stride = 0, region = 0;
};

// raw FP32 A chunks in flight per producer thread (cp.async ring): 16 KB a slot
constexpr int kRawSlotBytes = 128 * 32 * 4;

TcGeom tc_geom(int p, bool bf16) {
    TcGeom g;
    g.P = (p + 1) * (p + 1);
    g.Kpad = ((g.P + 31) / 32) * 32;
    g.Npad = ((g.P + 15) / 16) * 16;
    g.kchunks = g.Kpad / 32;
    // two accumulators (leading products | the rest), each a power of two >= 32 columns
    g.acc_cols = 32;
    while (g.acc_cols < g.Npad) g.acc_cols *= 2;
    g.tmem_cols = 2 * g.acc_cols;
    g.pieces = bf16 ? 3 : 2;
    g.row_bytes = bf16 ? 64 : 128;       // 32 K values of one row
    g.a_bytes = kTcRows * g.row_bytes;   // one piece of A for a 32-wide chunk
    g.b_bytes = g.Npad * g.row_bytes;    // one piece of B
    g.stage_bytes = g.pieces * (g.a_bytes + g.b_bytes);
    if (bf16) {
        g.epi_half = ((g.Npad / 16 + 1) / 2) * 16;
        g.epi_stride = 16;  // boxes of 16 columns
    }
    const int epi_bytes = (g.epi_half / 16) * kTcRows * 16 * 4;
    // three raw A slots when three operand stages still fit, else two; the
    // region after the stages also holds the pair epilogue's staging
    g.raw = 3;
    g.region = g.raw * kRawSlotBytes > epi_bytes ? g.raw * kRawSlotBytes : epi_bytes;
    g.stages = (227 * 1024 - 1024 - g.region) / g.stage_bytes;
    if (g.stages < 3) {
        g.raw = 2;
        g.region = g.raw * kRawSlotBytes > epi_bytes ? g.raw * kRawSlotBytes : epi_bytes;
        g.stages = (227 * 1024 - 1024 - g.region) / g.stage_bytes;
    }
    if (g.stages > kMaxStages) g.stages = kMaxStages;
    g.smem_bytes = g.stages * g.stage_bytes + g.region + 1024;
    return g;
}

bool tc_supported(int p, bool bf16) {
    const TcGeom g = tc_geom(p, bf16);
    return g.Npad <= 256 && g.stages >= 2;
}

// byte offset of element (row, k) of a 32-wide chunk in the swizzled K-major
// layouts.  TF32: 128-byte rows, 8-row atoms of 1024 B, 16-byte units XOR-ed
// with row % 8.  BF16: 64-byte rows, 8-row atoms of 512 B, 16-byte units
// XOR-ed with (row % 8) / 2 (address bits 4-5 with bits 7-8).
inline size_t swz_off(int row, int k) {
    return (size_t)(row >> 3) * 1024 + (size_t)(row & 7) * 128 +
           (size_t)(((k >> 2) ^ (row & 7)) << 4) + (size_t)(k & 3) * 4;
}
inline size_t swz64_off(int row, int k) {
    return (size_t)(row >> 3) * 512 + (size_t)(row & 7) * 64 +
           (size_t)(((k >> 3) ^ ((row & 7) >> 1)) << 4) + (size_t)(k & 7) * 2;
}

// round-to-nearest-even FP32 -> BF16 (finite inputs)
inline uint16_t bf16_bits_host(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    b += 0x7FFFu + ((b >> 16) & 1u);
    return (uint16_t)(b >> 16);
}
inline double bf16_value_host(uint16_t h) {
    const uint32_t b = (uint32_t)h << 16;
    float f;
    memcpy(&f, &b, 4);
    return (double)f;
}

inline float rna_tf32_host(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    if ((b & 0x7F800000u) != 0x7F800000u) b = (b + 0x1000u) & 0xFFFFE000u;
    float r;
    memcpy(&r, &b, 4);
    return r;
}


// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait (2 s of %globaltimer); false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
    }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// 16-byte global -> shared copy; src_bytes = 0 fills the 16 bytes with zeros
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
// arrive on an mbarrier once all of this thread's earlier cp.async copies have landed
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
// 16-byte global -> shared copy through L1; src_bytes = 0 fills zeros
__device__ __forceinline__ void cp_async16ca(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
// wait until at most n (1 or 2) of this thread's newest copy groups are pending
__device__ __forceinline__ void cp_async_wait(int n) {
    if (n >= 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else asm volatile("cp.async.wait_group 1;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ uint32_t rna_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// shared-memory matrix descriptor, K-major, descriptor version 1:
//   128-byte swizzle (layout 2), 8-row atoms 1024 B apart, or
//   64-byte swizzle (layout 4), 8-row atoms 512 B apart (stride byte offset).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused with these swizzles)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}
__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;             // 64-byte swizzle
    return d;
}
// instruction descriptors: D f32, A and B K-major, N and M; A/B tf32 (kind::tf32)
// or bf16 (kind::f16)
__host__ __device__ constexpr uint32_t idesc_tf32(int N, int M) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16(int N, int M) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// TMA tensor store of one box (2D: x = column, y = row) from shared memory,
// bulk-group completion, with an L2 eviction-priority hint (a createpolicy
// value)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y,
                                             const void* src, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%1, %2}], "
        "[%3], %4;" ::"l"(reinterpret_cast<uint64_t>(map)),
        "r"(x), "r"(y), "r"(smem_addr(src)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// bulk global -> shared copy with an L2 eviction-priority hint
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the source shared memory of this thread's committed bulk stores may be reused
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// barrier 1 over the N epilogue threads; the variant returns whether any
// of them passed true
template <int N>
__device__ __forceinline__ void epi_bar() {
    asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ bool epi_bar_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
        " selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(N)
        : "memory");
    return r != 0;
}
// tcgen05.ld of 16 columns without the wait (several loads, one wait)
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// tcgen05.st of 16 columns; tmem_wait_st before the columns are read back
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

enum TcMode { MODE_M2L = 0, MODE_M2M = 1, MODE_L2L = 2, MODE_PAIR = 3 };

constexpr int kOpM2M = 343, kOpL2L = 351, kNumOps = 359;  // packed operator indices

// One member of a joined ensemble M2L launch (BF16 pair-packed): its work
// list, its split multipoles and the TMA map of its partial rows.
struct alignas(64) PairMember {
    CUtensorMap map;
    const M2lPairItem* items;
    const M2lPair* pairs;
    const uint16_t* Mp;
    const M2lPairHdr* hdr;
};

struct TcArgs {
    CUtensorMap part_map;  // pair epilogue: TMA descriptor of the partial rows (BF16)
    int mode, level;      // level: the target level of M2M / L2L launches
    int D, P, ld, kchunks, Npad, tmem_cols, acc_cols, splits, stages, raw;
    int bf16, pieces, a_bytes, b_bytes;  // operand format and per-piece tile bytes
    int epi_half, epi_stride;            // BF16 pair epilogue staging (TcGeom)
    int epi_scratch;                     // the second half fits the free TMEM columns
    uint32_t idesc;
    const LevelInfo* linfo;
    const uint32_t* code;
    const int32_t* cid;
    int64_t off[kMaxDepth + 2];
    const float* M;
    float* L;
    float* Mout;           // M2M output (= M, other level)
    float* part;           // M2M: [splits-1][cells][ld]; M2L: [item][128][ld] slabs
    const uint16_t* Mp;    // BF16x3 M2L: M already split, [cell][kPieceRows][ld] bf16 (store_pieces)
    int64_t part_stride;   // cells_max * ld
    const unsigned char* ops;  // [359][kchunks][pieces][Npad rows] swizzled
    int* err;
    // M2L work list (written by k_tc_plan)
    const struct TcTile* tiles;
    const struct TcItem* items;
    const struct TcPlanHdr* hdr;
    // pair-packed M2L work list (k_pp_*) and its partial rows [slot][Npad]
    const M2lPair* pairs;
    const M2lPairItem* pitems;
    const M2lPairHdr* phdr;
    float* ppart;
    // joined ensemble launch (n_pm > 0): the members, and the first item of
    // each (pm_prefix[n_pm] = all items); work item idx belongs to the last
    // member k with pm_prefix[k] <= idx
    const PairMember* pm;
    const int* pm_prefix;
    int n_pm;
};

// One M2L tile (up to 128 targets of one level) and its non-empty offsets,
// as operator indices (ox+3)*49 + (oy+3)*7 + (oz+3) in increasing order; one
// work item = a contiguous run of them.  oct is the targets' common child
// octant, or -1 for a mixed tile (a sparse level's cells of every octant).
// The tile's items are item0 .. item0 + nsplit - 1 of the work list.
constexpr int kMaxTerms = 320;  // >= 316 offsets of [-3,3]^3 outside [-1,1]^3
struct TcTile {
    int level, oct, base, rows, cnt, nsplit, item0, pad1;
    uint16_t terms[kMaxTerms];
};

// Tiles of level l: one group per child octant (the 189 offsets of an octant
// share their operators) when the level is dense; when it holds fewer than
// kMixedCells cells, tiles of consecutive cells of every octant, so that
// sparse upper levels do not run mostly empty 128-row products.
constexpr int kMixedCells = 512;
__host__ __device__ __forceinline__ bool tc_level_mixed(const LevelInfo& li, int l) {
    return li.gbase[l + 1] - li.gbase[l] < kMixedCells;
}
// number of tiles of level l
__host__ __device__ inline int tc_level_tiles(const LevelInfo& li, int l) {
    if (tc_level_mixed(li, l)) return (li.gbase[l + 1] - li.gbase[l] + kTcRows - 1) / kTcRows;
    int nt = 0;
    for (int o = 0; o < 8; ++o) nt += (li.oct_start[l][o + 1] - li.oct_start[l][o] + kTcRows - 1) / kTcRows;
    return nt;
}
// tile t of the M2L launch (levels 2..D in order); false past the last tile
__host__ __device__ inline bool tc_tile(const LevelInfo& li, int D, int t, int& level, int& oct,
                                        int& base, int& rows) {
    int acc = 0;
    for (int l = 2; l <= D; ++l) {
        const bool mixed = tc_level_mixed(li, l);
        for (int o = 0; o < (mixed ? 1 : 8); ++o) {
            const int s0 = mixed ? li.gbase[l] : li.oct_start[l][o];
            const int s1 = mixed ? li.gbase[l + 1] : li.oct_start[l][o + 1];
            const int nt = (s1 - s0 + kTcRows - 1) / kTcRows;
            if (t < acc + nt) {
                level = l;
                oct = mixed ? -1 : o;
                base = s0 + (t - acc) * kTcRows;
                rows = min(kTcRows, s1 - base);
                return true;
            }
            acc += nt;
        }
    }
    return false;
}
// does a target of child octant (bx, by, bz) take offset o?  (its source is a
// child of a neighbour of the target's parent: o_a in [b_a - 3, b_a + 2])
__host__ __device__ __forceinline__ bool tc_admits(int ox, int oy, int oz, int bx, int by, int bz) {
    return ox >= bx - 3 && ox <= bx + 2 && oy >= by - 3 && oy <= by + 2 && oz >= bz - 3 &&
           oz <= bz + 2;
}
struct TcItem {
    int tile, begin, end, rank;
};
struct TcPlanHdr {
    unsigned ticket;
    int n_tiles, n_items, pad;
};

// LevelInfo copied to shared memory by all threads at once (the tile
// enumeration otherwise walks it with a chain of dependent global loads).
__device__ __forceinline__ void stage_linfo(const LevelInfo* g, LevelInfo* s) {
    const int* src = reinterpret_cast<const int*>(g);
    int* dst = reinterpret_cast<int*>(s);
    for (int i = threadIdx.x; i < (int)(sizeof(LevelInfo) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
}

// Warp roles: an operator producer (bulk copies), an MMA issuer, A producers
// (gather + split) and epilogue warps, which have warps of their own so that
// the producers run on into the next work item while the accumulators drain.
// Default: warp 0 = operator producer, warp 1 = MMA issuer, warps 2..9 = A
// producers, warps 10..13 = epilogue (one TMEM lane quarter each).  The BF16
// pair-packed kernel, whose items are short, drains its accumulators with
// two warps per lane quarter: warps 0..7 = epilogue, warp 8 = operator
// producer, warp 9 = MMA issuer, warps 10..11 = A producers (it copies
// pre-split rows only); 384 threads leave 168 registers a thread, room for
// three column groups of both accumulators per TMEM wait.  Warp 0
// allocates and frees TMEM in either layout.
template <int MODE, int BF16>
struct TcLayout {
    static constexpr bool kWide = MODE == 3 && BF16;  // MODE_PAIR
    static constexpr int kThreads = kWide ? 384 : 448;
    static constexpr int kWarpOp = kWide ? 8 : 0;
    static constexpr int kWarpMma = kWide ? 9 : 1;
    static constexpr int kWarpA0 = kWide ? 10 : 2;
    static constexpr int kAWarps = kWide ? 2 : 8;
    static constexpr int kEpiWarps = kWide ? 8 : 4;
};
constexpr int kEpiBoxBytes = kTcRows * 16 * 4;  // one TMA box: 128 rows x 16 FP32

// One unit of work for a CTA: a run [begin, end) of the term list of one tile
// of 128 target cells.  rank > 0 runs of M2L (and split > 0 of M2M) write
// partial sums that a reduction adds afterwards.
struct TcWork {
    int level, oct, base, rows, begin, end, rank, tile, slot, op, pbegin;
};

// Work item idx of this launch: M2L reads the device work list; M2M and L2L
// derive (tile, split) from the block index (one item per CTA).
template <int MODE>
__device__ __forceinline__ bool tc_work(const TcArgs& a, const LevelInfo& li, int idx, TcWork& w) {
    w.rows = 0;
    if (MODE == MODE_PAIR) {
        M2lPairItem it;
        int k = 0;
        if (a.n_pm > 0) {
            int lo = 0, hi = a.n_pm - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.pm_prefix[mid] <= idx) lo = mid;
                else hi = mid - 1;
            }
            k = lo;
            it = a.pm[k].items[idx - a.pm_prefix[k]];
        } else {
            it = a.pitems[idx];
        }
        w.op = it.op;
        w.pbegin = it.begin;
        w.rows = it.rows;
        w.begin = 0;
        w.end = 1;
        w.rank = 0;
        w.tile = k;  // the member of a joined launch
        w.slot = idx;
        w.level = 0;
        w.oct = 0;
        w.base = 0;
        return w.rows > 0;
    }
    if (MODE == MODE_M2L) {
        const TcItem it = a.items[idx];
        const TcTile& tl = a.tiles[it.tile];
        w.level = tl.level;
        w.oct = tl.oct;
        w.base = tl.base;
        w.rows = tl.rows;
        w.begin = it.begin;
        w.end = it.end;
        w.rank = it.rank;
        w.tile = it.tile;
        w.slot = idx;
        return w.rows > 0;
    }
    const int gsplit = MODE == MODE_L2L ? 1 : a.splits;  // CTAs per tile
    const int split = idx % gsplit;
    const int l0 = a.level;
    int t = idx / gsplit, acc = 0;
    const int ngroups = MODE == MODE_M2M ? 1 : 8;
    for (int o = 0; o < ngroups; ++o) {
        int s0, s1;
        if (MODE == MODE_M2M) {
            s0 = li.gbase[l0];
            s1 = li.gbase[l0 + 1];
        } else {
            s0 = li.oct_start[l0][o];
            s1 = li.oct_start[l0][o + 1];
        }
        const int nt = (s1 - s0 + kTcRows - 1) / kTcRows;
        if (t < acc + nt) {
            w.level = l0;
            w.oct = o;
            w.base = s0 + (t - acc) * kTcRows;
            w.rows = min(kTcRows, s1 - w.base);
            break;
        }
        acc += nt;
    }
    const int cnt = MODE == MODE_M2M ? 8 : (l0 >= 3 ? 1 : 0);
    w.begin = (cnt * split) / gsplit;
    w.end = (cnt * (split + 1)) / gsplit;
    w.rank = split;
    w.tile = -1;
    w.slot = -1;
    return w.rows > 0;
}

// packed operator index of term j of a work item
template <int MODE>
__device__ __forceinline__ int tc_op(const TcArgs& a, const TcWork& w, int j) {
    if (MODE == MODE_PAIR) return w.op;
    if (MODE == MODE_M2L) return a.tiles[w.tile].terms[j];
    if (MODE == MODE_M2M) return kOpM2M + j;
    return kOpL2L + w.oct;
}

__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity,
                                                   volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
    }
}

// Pair epilogue helpers.  A row's 16 FP32 values of one column group go to
// its 64-byte line of a TMA box, 16-byte unit q at q ^ rsw (the 64-byte
// swizzle, rsw = (row & 7) >> 1).
__device__ __forceinline__ void epi_put16(unsigned char* b, int rsw, const uint32_t (&v)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(b + ((q ^ rsw) << 4)) =
            make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
// TMEM column of the k-th parked group of 16 (pair_epi_scratch_fits): the
// free columns after the hh accumulator, then after the cross one, then
// after both
__device__ __forceinline__ uint32_t epi_scratch_col(int k, int Npad, int acc_cols) {
    const int W = acc_cols - Npad;
    int c = k * 16;
    if (c < W) return (uint32_t)(Npad + c);
    c -= W;
    if (c < W) return (uint32_t)(acc_cols + Npad + c);
    return (uint32_t)(2 * acc_cols + c - W);
}
template <bool PARK>
__device__ __forceinline__ void epi_sink(int k, const uint32_t (&v)[16], unsigned char* brow,
                                         int rsw, uint32_t trow, int Npad, int acc_cols) {
    if (PARK)
        tmem_st16(trow + epi_scratch_col(k, Npad, acc_cols), v);
    else
        epi_put16(brow + k * kEpiBoxBytes, rsw, v);
}
// column groups [g0, g1) of the two accumulators (hh at trow, cross at trow +
// cross), summed, into boxes 0.. (kEpiBoxBytes apart from brow) or, PARK,
// into the free TMEM columns (k-th group at epi_scratch_col(k)); two groups
// per TMEM wait
template <bool PARK>
__device__ __forceinline__ void epi_drain(uint32_t trow, uint32_t cross, int g0, int g1,
                                          unsigned char* brow, int rsw, int Npad, int acc_cols) {
#pragma unroll 1
    for (int gq = g0; gq < g1; gq += 2) {
        uint32_t h0[16], c0[16], h1[16], c1[16];
        const bool two = gq + 1 < g1;  // uniform
        tmem_ld16_nw(trow + (uint32_t)(gq * 16), h0);
        tmem_ld16_nw(trow + (uint32_t)(gq * 16) + cross, c0);
        if (two) {
            tmem_ld16_nw(trow + (uint32_t)(gq * 16 + 16), h1);
            tmem_ld16_nw(trow + (uint32_t)(gq * 16 + 16) + cross, c1);
        }
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j)
            h0[j] = __float_as_uint(__uint_as_float(h0[j]) + __uint_as_float(c0[j]));
        epi_sink<PARK>(gq - g0, h0, brow, rsw, trow, Npad, acc_cols);
        if (two) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                h1[j] = __float_as_uint(__uint_as_float(h1[j]) + __uint_as_float(c1[j]));
            epi_sink<PARK>(gq - g0 + 1, h1, brow, rsw, trow, Npad, acc_cols);
        }
    }
}
// n parked groups from the free TMEM columns into boxes 0.., two per wait
__device__ __forceinline__ void epi_unpark(uint32_t trow, int n, unsigned char* brow, int rsw,
                                           int Npad, int acc_cols) {
#pragma unroll 1
    for (int k = 0; k < n; k += 2) {
        uint32_t v0[16], v1[16];
        const bool two = k + 1 < n;  // uniform
        tmem_ld16_nw(trow + epi_scratch_col(k, Npad, acc_cols), v0);
        if (two) tmem_ld16_nw(trow + epi_scratch_col(k + 1, Npad, acc_cols), v1);
        tmem_wait_ld();
        epi_put16(brow + k * kEpiBoxBytes, rsw, v0);
        if (two) epi_put16(brow + (k + 1) * kEpiBoxBytes, rsw, v1);
    }
}

// One instantiation per mode and operand format (MODE == MODE, BF16 == BF16):
// each kernel carries only its own paths.
template <int MODE, int BF16>
__global__ void __launch_bounds__((TcLayout<MODE, BF16>::kThreads), 1)
    k_m2l_tc(const __grid_constant__ TcArgs a) {
    using L = TcLayout<MODE, BF16>;
    extern __shared__ unsigned char smem_dyn[];
    pdl_wait();  // launched after its inputs' producer (programmatic launches)
    __shared__ __align__(8) uint64_t fullA_bar[kMaxStages], fullB_bar[kMaxStages],
        empty_bar[kMaxStages], accf_bar, acce_bar, drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    __shared__ LevelInfo li;
    volatile int* abort_v = &abort_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const int a_bytes = a.a_bytes, b_bytes = a.b_bytes, pieces = a.pieces;
    const int stage_bytes = pieces * (a_bytes + b_bytes);
    const int NS = a.stages;
    // work items of this CTA: idx = first, first + stride, ... < count
    int count, first, stride;
    if (MODE == MODE_M2L || MODE == MODE_PAIR) {
        count = MODE == MODE_PAIR ? (a.n_pm > 0 ? a.pm_prefix[a.n_pm] : a.phdr->n_items)
                                  : a.hdr->n_items;
        first = blockIdx.x;
        stride = gridDim.x;
    } else {
        count = blockIdx.x + 1;
        first = blockIdx.x;
        stride = 1;
        stage_linfo(a.linfo, &li);
    }
    if (first >= count) return;  // uniform across the block
    if (tid == 0) {
        abort_sh = 0;
        mbar_init(&accf_bar, 1);
        mbar_init(&acce_bar, L::kEpiWarps * 32);
        mbar_init(&drain_bar, 1);
        for (int s = 0; s < NS; ++s) {
            mbar_init(&fullA_bar[s], L::kAWarps * 32);
            mbar_init(&fullB_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_base_sh)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    int issued_par[kMaxStages];  // operator producer: parity of the last copy per stage
#pragma unroll
    for (int s = 0; s < kMaxStages; ++s) issued_par[s] = -1;

    if (warp == L::kWarpOp) {
        // ---- operator producer
        if (lane == 0) {
            const uint64_t op_l2 = policy_evict_first();
            (void)op_l2;
            int g = 0;
            for (int idx = first; idx < count && !*abort_v; idx += stride) {
                TcWork w;
                if (!tc_work<MODE>(a, li, idx, w)) continue;
                const int n_it = (w.end - w.begin) * a.kchunks;
                for (int it = 0; it < n_it; ++it, ++g) {
                    const int st = g % NS, use = g / NS;
                    if (!mbar_wait_or_abort(&empty_bar[st], (use & 1) ^ 1, abort_v)) {
                        *abort_v = 1;
                        break;
                    }
                    const int j = w.begin + it / a.kchunks, kc = it % a.kchunks;
                    unsigned char* sB = base + st * stage_bytes + pieces * a_bytes;
                    mbar_arrive_expect_tx(&fullB_bar[st], pieces * b_bytes);
                    const unsigned char* src =
                        a.ops + ((size_t)tc_op<MODE>(a, w, j) * a.kchunks + kc) * pieces * b_bytes;
                    if (MODE == MODE_PAIR && BF16)
                        // an offset's items run side by side in one wave: once
                        // read, its operator may leave L2 before the partial rows
                        bulk_g2s_hint(sB, src, pieces * b_bytes, &fullB_bar[st], op_l2);
                    else
                        bulk_g2s(sB, src, pieces * b_bytes, &fullB_bar[st]);
                    issued_par[st] = use & 1;
                }
            }
        }
    } else if (warp == L::kWarpMma) {
        // ---- MMA issuer
        if (lane == 0) {
            int g = 0, jacc = 0;
            for (int idx = first; idx < count && !*abort_v; idx += stride) {
                TcWork w;
                if (!tc_work<MODE>(a, li, idx, w)) continue;
                const int n_it = (w.end - w.begin) * a.kchunks;
                if (n_it == 0) continue;
                // the epilogue of the previous item has read the accumulators
                if (jacc > 0 && !mbar_wait_or_abort(&acce_bar, (jacc - 1) & 1, abort_v)) {
                    *abort_v = 1;
                    break;
                }
                tc_fence_after();
                // accumulator 0 takes only the leading products hi x hi, the
                // rest (2^-8 / 2^-11 of them and smaller) go to accumulator 1
                const uint32_t d0 = tmem, d1 = tmem + (uint32_t)a.acc_cols;
                for (int it = 0; it < n_it; ++it, ++g) {
                    const int st = g % NS, use = g / NS;
                    if (!mbar_wait_or_abort(&fullB_bar[st], use & 1, abort_v) ||
                        !mbar_wait_or_abort(&fullA_bar[st], use & 1, abort_v)) {
                        *abort_v = 1;
                        break;
                    }
                    // pre-split A rows arrive by cp.async (generic proxy): order
                    // them before the tensor core's reads
                    if ((MODE == MODE_M2L || MODE == MODE_PAIR) && BF16) fence_proxy_async();
                    tc_fence_after();
                    const uint32_t ah = smem_addr(base + st * stage_bytes);
                    if (BF16) {
                        // pieces hi, mid, lo of A then of B; 2 K-steps of 16 values
                        const uint32_t am = ah + a_bytes, al = am + a_bytes;
                        const uint32_t bh = ah + 3 * a_bytes, bm = bh + b_bytes, bl = bm + b_bytes;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                            const uint32_t o = 32 * kk;
                            mma_bf16(d1, sdesc64(am + o), sdesc64(bm + o), a.idesc, acc);
                            mma_bf16(d1, sdesc64(ah + o), sdesc64(bl + o), a.idesc, 1u);
                            mma_bf16(d1, sdesc64(al + o), sdesc64(bh + o), a.idesc, 1u);
                            mma_bf16(d1, sdesc64(ah + o), sdesc64(bm + o), a.idesc, 1u);
                            mma_bf16(d1, sdesc64(am + o), sdesc64(bh + o), a.idesc, 1u);
                            mma_bf16(d0, sdesc64(ah + o), sdesc64(bh + o), a.idesc, acc);
                        }
                    } else {
                        const uint32_t al = ah + a_bytes;
                        const uint32_t bh = ah + 2 * a_bytes, bl = bh + b_bytes;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                            mma_tf32(d1, sdesc(ah + 32 * kk), sdesc(bl + 32 * kk), a.idesc, acc);
                            mma_tf32(d1, sdesc(al + 32 * kk), sdesc(bh + 32 * kk), a.idesc, 1u);
                            mma_tf32(d0, sdesc(ah + 32 * kk), sdesc(bh + 32 * kk), a.idesc, acc);
                        }
                    }
                    mma_commit(&empty_bar[st]);  // frees the stage once these MMAs finish
                }
                if (*abort_v) break;
                mma_commit(&accf_bar);  // this item's accumulators are complete
                ++jacc;
            }
        }
    } else if (warp >= L::kWarpA0 && warp < L::kWarpA0 + L::kAWarps) {
        if ((MODE == MODE_M2L || MODE == MODE_PAIR) && BF16) {
            // ---- A producers, BF16x3 M2L: the sources' M rows are already
            // split into bf16 pieces (k_split_m), so each thread copies its
            // 16-byte unit (8 values) of each piece for two rows by cp.async
            // straight into the stage's swizzled layout, and the stage barrier
            // counts its arrival once those copies land; no conversion here.
            // Thread ta owns unit c = ta % 4 of rows ta / 4 + RS j.
            constexpr int RS = L::kAWarps * 8;             // rows per pass
            constexpr int NJ = (kTcRows + RS - 1) / RS;    // passes
            const int ta = tid - L::kWarpA0 * 32;
            const int r0 = ta >> 2, c = ta & 3;
            int g = 0;
            for (int idx = first; idx < count && !*abort_v; idx += stride) {
                TcWork w;
                if (!tc_work<MODE>(a, li, idx, w)) continue;
                const int n_it = (w.end - w.begin) * a.kchunks;
                const int l = w.level, lim = 1 << l;
                int tix[NJ], tiy[NJ], tiz[NJ], pg[NJ];
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    tix[j] = tiy[j] = tiz[j] = 0;
                    pg[j] = -1;
                    if (MODE == MODE_M2L && r0 + RS * j < w.rows)
                        demorton3(a.code[w.base + r0 + RS * j], tix[j], tiy[j], tiz[j]);
                }
                for (int it = 0; it < n_it; ++it) {
                    const int gg = g + it;
                    const int st = gg % NS, use = gg / NS;
                    const int kc = it % a.kchunks;
                    if (MODE == MODE_PAIR && it == 0) {
                        // first piece row of each A row: the source's pieces,
                        // or its mirrored pieces for a pair of -op
                        const M2lPair* pr = a.n_pm > 0 ? a.pm[w.tile].pairs : a.pairs;
#pragma unroll
                        for (int j = 0; j < NJ; ++j) {
                            pg[j] = -1;
                            if (r0 + RS * j < w.rows) {
                                const int sv = pr[w.pbegin + r0 + RS * j].src;
                                pg[j] = (sv & (kPairMirror - 1)) * kPieceRows +
                                        ((sv & kPairMirror) ? 3 : 0);
                            }
                        }
                    } else if (MODE == MODE_M2L && kc == 0) {
                        const int opi = a.tiles[w.tile].terms[w.begin + it / a.kchunks];
                        const int ox = opi / 49 - 3, oy = (opi / 7) % 7 - 3, oz = opi % 7 - 3;
#pragma unroll
                        for (int j = 0; j < NJ; ++j) {
                            int gs = -1;
                            const int sx = tix[j] - ox, sy = tiy[j] - oy, sz = tiz[j] - oz;
                            if (r0 + RS * j < w.rows &&
                                tc_admits(ox, oy, oz, tix[j] & 1, tiy[j] & 1, tiz[j] & 1) &&
                                sx >= 0 && sy >= 0 && sz >= 0 && sx < lim && sy < lim && sz < lim)
                                gs = a.cid[a.off[l] + morton3(sx, sy, sz)];
                            pg[j] = gs >= 0 ? gs * kPieceRows : -1;
                        }
                    }
                    int okw = 1;
                    if (lane == 0) okw = mbar_wait_or_abort(&empty_bar[st], (use & 1) ^ 1, abort_v) ? 1 : 0;
                    okw = __shfl_sync(0xffffffffu, okw, 0);
                    if (!okw) {
                        *abort_v = 1;
                        break;
                    }
                    unsigned char* sA = base + st * stage_bytes;
                    const uint16_t* Mp = MODE == MODE_PAIR && a.n_pm > 0 ? a.pm[w.tile].Mp : a.Mp;
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        const int r = r0 + RS * j;
                        if (r >= kTcRows) break;
                        const int off = (r >> 3) * 512 + (r & 7) * 64 + ((c ^ ((r & 7) >> 1)) << 4);
                        const int gs = pg[j];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const uint16_t* src =
                                gs >= 0 ? Mp + ((int64_t)gs + q) * a.ld + kc * 32 + c * 8 : Mp;
                            cp_async16ca(sA + q * a_bytes + off, src, gs >= 0 ? 16u : 0u);
                        }
                    }
                    cp_async_arrive(&fullA_bar[st]);
                }
                g += n_it;
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
        } else {
        // ---- A producers: each thread owns rows r0 + 32 j (j < 4) and 16-byte unit c.
        // Its raw FP32 values travel by cp.async into its own slots of a ring
        // of a.raw chunks, a.raw - 1 iterations ahead of their split.
        static_assert(L::kWide || L::kAWarps == 8, "the FP32 row ring assumes 256 A threads");
        const int ta = tid - L::kWarpA0 * 32;
        const int r0 = ta >> 3, c = ta & 7;
        const float* src_base = MODE == MODE_L2L ? a.L : a.M;
        unsigned char* raw = base + NS * stage_bytes;  // [slot][j][256 threads][16 B]
        const int R = a.raw;
        int g = 0;
        for (int idx = first; idx < count && !*abort_v; idx += stride) {
            TcWork w;
            if (!tc_work<MODE>(a, li, idx, w)) continue;
            const int n_it = (w.end - w.begin) * a.kchunks;
            const int l = w.level, lim = 1 << l;
            int tix[4], tiy[4], tiz[4];
            uint32_t tcode[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = r0 + 32 * j;
                tcode[j] = 0;
                tix[j] = tiy[j] = tiz[j] = 0;
                if (MODE != MODE_PAIR && r < w.rows) {
                    tcode[j] = a.code[w.base + r];
                    demorton3(tcode[j], tix[j], tiy[j], tiz[j]);
                }
            }
            // source cells of this thread's rows for term t
            int pg[4] = {-1, -1, -1, -1};
            auto sources = [&](int t) {
                int opi = 0, term = t;
                if (MODE == MODE_M2L) opi = a.tiles[w.tile].terms[t];
                const int ox = opi / 49 - 3, oy = (opi / 7) % 7 - 3, oz = opi % 7 - 3;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int gs = -1;
                    if (r0 + 32 * j < w.rows) {
                        if (MODE == MODE_PAIR) {
                            gs = a.pairs[w.pbegin + r0 + 32 * j].src;
                        } else if (MODE == MODE_M2L) {
                            // a mixed tile's rows differ in octant: each takes its own offsets
                            const int sx = tix[j] - ox, sy = tiy[j] - oy, sz = tiz[j] - oz;
                            if (tc_admits(ox, oy, oz, tix[j] & 1, tiy[j] & 1, tiz[j] & 1) &&
                                sx >= 0 && sy >= 0 && sz >= 0 && sx < lim && sy < lim && sz < lim)
                                gs = a.cid[a.off[l] + morton3(sx, sy, sz)];
                        } else if (MODE == MODE_M2M) {
                            gs = a.cid[a.off[l + 1] + ((tcode[j] << 3) | (uint32_t)term)];
                        } else {
                            gs = a.cid[a.off[l - 1] + (tcode[j] >> 3)];
                        }
                    }
                    pg[j] = gs;
                }
            };
            // copies of iteration j into ring slot (g + j) % R; one group per iteration
            // (empty past the end, so that the count of pending groups is fixed)
            auto prefetch = [&](int j) {
                if (j < n_it) {
                    const int kc = j % a.kchunks;
                    if (kc == 0) sources(w.begin + j / a.kchunks);
                    unsigned char* slot = raw + ((g + j) % R) * kRawSlotBytes + ta * 16;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int gs = pg[q];
                        const float* src = gs >= 0 ? src_base + (int64_t)gs * a.ld + kc * 32 + c * 4
                                                   : src_base;
                        cp_async16(slot + q * 4096, src, gs >= 0 ? 16u : 0u);
                    }
                }
                cp_async_commit();
            };
            for (int j = 0; j < R - 1; ++j) prefetch(j);
            for (int it = 0; it < n_it; ++it) {
                prefetch(it + R - 1);
                const int gg = g + it;
                const int st = gg % NS, use = gg / NS;
                cp_async_wait(R - 1);  // this thread's copies of iteration it have landed
                const unsigned char* mine = raw + (gg % R) * kRawSlotBytes + ta * 16;
                float4 v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = *reinterpret_cast<const float4*>(mine + q * 4096);
                // one lane polls the stage barrier for the whole warp
                int okw = 1;
                if (lane == 0) okw = mbar_wait_or_abort(&empty_bar[st], (use & 1) ^ 1, abort_v) ? 1 : 0;
                okw = __shfl_sync(0xffffffffu, okw, 0);
                if (!okw) {
                    *abort_v = 1;
                    break;
                }
                unsigned char* sA_hi = base + st * stage_bytes;
                if (BF16) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int r = r0 + 32 * j;
                        uint32_t h0, h1, h2, h3, m0, m1, m2, m3, l0, l1, l2, l3;
                        split_bf16x3(v[j].x, h0, m0, l0);
                        split_bf16x3(v[j].y, h1, m1, l1);
                        split_bf16x3(v[j].z, h2, m2, l2);
                        split_bf16x3(v[j].w, h3, m3, l3);
                        // 4 values = half a 16-byte unit of the 64-byte row
                        const int off = (r >> 3) * 512 + (r & 7) * 64 +
                                        (((c >> 1) ^ ((r & 7) >> 1)) << 4) + (c & 1) * 8;
                        *reinterpret_cast<uint2*>(sA_hi + off) =
                            make_uint2(h0 | (h1 << 16), h2 | (h3 << 16));
                        *reinterpret_cast<uint2*>(sA_hi + a_bytes + off) =
                            make_uint2(m0 | (m1 << 16), m2 | (m3 << 16));
                        *reinterpret_cast<uint2*>(sA_hi + 2 * a_bytes + off) =
                            make_uint2(l0 | (l1 << 16), l2 | (l3 << 16));
                    }
                } else {
                    unsigned char* sA_lo = sA_hi + a_bytes;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int r = r0 + 32 * j;
                        uint4 hi, lo;
                        hi.x = rna_tf32(v[j].x); lo.x = rna_tf32(v[j].x - __uint_as_float(hi.x));
                        hi.y = rna_tf32(v[j].y); lo.y = rna_tf32(v[j].y - __uint_as_float(hi.y));
                        hi.z = rna_tf32(v[j].z); lo.z = rna_tf32(v[j].z - __uint_as_float(hi.z));
                        hi.w = rna_tf32(v[j].w); lo.w = rna_tf32(v[j].w - __uint_as_float(hi.w));
                        const int off = (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4);
                        *reinterpret_cast<uint4*>(sA_hi + off) = hi;
                        *reinterpret_cast<uint4*>(sA_lo + off) = lo;
                    }
                }
                fence_proxy_async();
                mbar_arrive(&fullA_bar[st]);
            }
            g += n_it;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        }
    } else if (MODE == MODE_PAIR && BF16) {
        // ---- epilogue of the BF16 pair-packed items, warps 0..7: warp w
        // reads TMEM lanes 32 (w % 4) .. + 31 (row = lane = pair), warps 0..3
        // the first half of the column groups, warps 4..7 the rest.  The
        // first half goes to shared memory in boxes of 128 rows x 16 columns
        // (the TMA 64-byte swizzle: 16-byte unit u of row r at
        // u ^ ((r & 7) >> 1), bank-conflict free), the second half to
        // registers, two or three TMEM waits per warp, and the accumulators are
        // released; one thread then stores the boxes with TMA (the item's
        // rows are one 128-row block of the partial array), the second half
        // follows through the same boxes, while the MMAs of the next item
        // run.  The warps decide to stop together (barrier reduction), so
        // their barriers stay matched.
        constexpr int NE = L::kEpiWarps * 32;
        const int quad = warp & 3, second = warp >> 2;
        const int row = quad * 32 + lane;
        const int etid = warp * 32 + lane;
        unsigned char* boxes = base + NS * stage_bytes;  // kEpiBoxBytes apart
        const int ngr = a.Npad / 16, gh = a.epi_half / 16;
        const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
        const uint32_t cross = (uint32_t)a.acc_cols;
        const int rsw = (row & 7) >> 1;
        // the partial rows are read back by the reduction right after this
        // kernel: keep them in L2 ahead of the operators
        const uint64_t keep_l2 = policy_evict_last();
        unsigned char* brow = boxes + row * 64;
        int jacc = 0;
        for (int idx = first; idx < count; idx += stride) {
            TcWork w;
            if (!tc_work<MODE>(a, li, idx, w)) continue;  // uniform: rows >= 1 for every item
            int ok = 1;
            if (lane == 0) ok = mbar_wait_or_abort(&accf_bar, jacc & 1, abort_v) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            // the boxes of the previous item have been read by its stores
            if (etid == 0) bulk_wait_read();
            if (epi_bar_any<NE>(ok == 0)) {
                *abort_v = 1;
                break;
            }
            tc_fence_after();
            // the member's partial rows (joined launch: its map in global
            // memory, written by the host before the launch)
            const CUtensorMap* map = a.n_pm > 0 ? &a.pm[w.tile].map : &a.part_map;
            if (a.n_pm > 0 && etid == 0)
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map)
                             : "memory");
            // the two warp sets take separate branches for the whole item;
            // their barriers match
            if (!second) {
                epi_drain<false>(trow, cross, 0, gh, brow, rsw, a.Npad, a.acc_cols);
                tc_fence_before();
                mbar_arrive(&acce_bar);  // this half of the accumulators read
                // first half out by TMA
                fence_proxy_async();
                epi_bar<NE>();
                if (etid == 0) {
                    for (int gq = 0; gq < gh; ++gq)
                        tma_store_2d(map, gq * 16, w.pbegin, boxes + gq * kEpiBoxBytes, keep_l2);
                    bulk_commit();
                    bulk_wait_read();
                }
                epi_bar<NE>();
                // (the other warps refill the boxes)
                epi_bar<NE>();
                if (etid == 0) {
                    for (int k = 0; k < ngr - gh; ++k)
                        tma_store_2d(map, (gh + k) * 16, w.pbegin, boxes + k * kEpiBoxBytes,
                                     keep_l2);
                    bulk_commit();
                }
            } else if (a.epi_scratch) {  // uniform
                // second half summed into the free TMEM columns, so that the
                // accumulators are released after two waits
                epi_drain<true>(trow, cross, gh, ngr, brow, rsw, a.Npad, a.acc_cols);
                tmem_wait_st();
                tc_fence_before();
                mbar_arrive(&acce_bar);  // the other half read: the issuer may go on
                epi_bar<NE>();
                // (the first half is stored from the boxes)
                epi_bar<NE>();
                tc_fence_after();
                epi_unpark(trow, ngr - gh, brow, rsw, a.Npad, a.acc_cols);
                fence_proxy_async();
                epi_bar<NE>();
            } else {
                // wide rows: the second half straight from TMEM once the
                // first half's boxes are free (the accumulators held longer)
                epi_bar<NE>();
                epi_bar<NE>();
                epi_drain<false>(trow, cross, gh, ngr, brow, rsw, a.Npad, a.acc_cols);
                tc_fence_before();
                mbar_arrive(&acce_bar);
                fence_proxy_async();
                epi_bar<NE>();
            }
            ++jacc;
        }
        // the boxes read before the CTA's shared memory goes away (the
        // stores themselves complete with the grid)
        if (etid == 0) bulk_wait_read();
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = rows of the tile
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        int jacc = 0;
        for (int idx = first; idx < count && !*abort_v; idx += stride) {
            TcWork w;
            if (!tc_work<MODE>(a, li, idx, w)) continue;
            const int n_it = (w.end - w.begin) * a.kchunks;
            float* out;
            int64_t orow;
            if (MODE == MODE_PAIR) {
                out = a.ppart;  // rows in pair order
                orow = (int64_t)w.pbegin + row;
            } else if (MODE == MODE_M2L && w.rank > 0) {
                out = a.part + (int64_t)w.slot * kTcRows * a.ld;  // this item's partial slab
                orow = row;
            } else if (MODE == MODE_M2M && w.rank > 0) {
                out = a.part + (int64_t)(w.rank - 1) * a.part_stride;
                orow = w.base + row;
            } else {
                out = MODE == MODE_M2M ? a.Mout : a.L;
                orow = w.base + row;
            }
            if (n_it > 0) {
                int ok = 1;
                if (lane == 0) ok = mbar_wait_or_abort(&accf_bar, jacc & 1, abort_v) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    *abort_v = 1;
                    break;
                }
                tc_fence_after();
            }
            // columns in groups of 4 x 16; the L2L epilogue's loads of the
            // cell's own M2L result are all issued before the group's stores.
            // Columns P .. Npad-1 hold exact zeros (zero operator rows), so
            // whole 16-byte units are written.
            float* orow_p = out + orow * (MODE == MODE_PAIR ? a.Npad : a.ld);
            const float* own_p = a.L + orow * a.ld;
            const bool live = row < w.rows;
            if (MODE == MODE_PAIR) {
                // two column groups of both accumulators per wait; the row
                // (one pair's partial expansion) goes straight to its slot
                for (int cb = 0; cb * 16 < a.Npad; cb += 2) {
                    const bool two = (cb + 1) * 16 < a.Npad;  // uniform
                    const uint32_t t0 = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cb * 16);
                    uint32_t h0[16], c0[16], h1[16], c1[16];
                    tmem_ld16_nw(t0, h0);
                    tmem_ld16_nw(t0 + (uint32_t)a.acc_cols, c0);
                    if (two) {
                        tmem_ld16_nw(t0 + 16u, h1);
                        tmem_ld16_nw(t0 + 16u + (uint32_t)a.acc_cols, c1);
                    }
                    tmem_wait_ld();
                    if (live) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float4 v;
                            v.x = __uint_as_float(h0[4 * q + 0]) + __uint_as_float(c0[4 * q + 0]);
                            v.y = __uint_as_float(h0[4 * q + 1]) + __uint_as_float(c0[4 * q + 1]);
                            v.z = __uint_as_float(h0[4 * q + 2]) + __uint_as_float(c0[4 * q + 2]);
                            v.w = __uint_as_float(h0[4 * q + 3]) + __uint_as_float(c0[4 * q + 3]);
                            *reinterpret_cast<float4*>(orow_p + cb * 16 + 4 * q) = v;
                        }
                        if (two) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                float4 v;
                                v.x = __uint_as_float(h1[4 * q + 0]) + __uint_as_float(c1[4 * q + 0]);
                                v.y = __uint_as_float(h1[4 * q + 1]) + __uint_as_float(c1[4 * q + 1]);
                                v.z = __uint_as_float(h1[4 * q + 2]) + __uint_as_float(c1[4 * q + 2]);
                                v.w = __uint_as_float(h1[4 * q + 3]) + __uint_as_float(c1[4 * q + 3]);
                                *reinterpret_cast<float4*>(orow_p + (cb + 1) * 16 + 4 * q) = v;
                            }
                        }
                    }
                }
            } else
            for (int cb0 = 0; cb0 * 16 < a.Npad; cb0 += 4) {
                float4 own[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    own[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (MODE == MODE_L2L && live && (cb0 * 16 + q * 4) < a.Npad)
                        own[q] = *reinterpret_cast<const float4*>(own_p + cb0 * 16 + q * 4);
                }
#pragma unroll
                for (int cq = 0; cq < 4; ++cq) {
                    const int cb = cb0 + cq;
                    if (cb * 16 >= a.Npad) break;
                    uint32_t r[16];
                    if (n_it > 0) {
                        const uint32_t t0 = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cb * 16);
                        uint32_t r1[16];
                        tmem_ld16(t0, r);
                        tmem_ld16(t0 + (uint32_t)a.acc_cols, r1);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(r1[j]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) r[j] = 0u;
                    }
                    if (live) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 o = own[cq * 4 + q];
                            float4 v;
                            v.x = __uint_as_float(r[4 * q + 0]) + o.x;
                            v.y = __uint_as_float(r[4 * q + 1]) + o.y;
                            v.z = __uint_as_float(r[4 * q + 2]) + o.z;
                            v.w = __uint_as_float(r[4 * q + 3]) + o.w;
                            *reinterpret_cast<float4*>(orow_p + cb * 16 + 4 * q) = v;
                        }
                    }
                }
            }
            if (n_it > 0) {
                // accumulators read: the issuer may start the next item
                tc_fence_before();
                mbar_arrive(&acce_bar);
                ++jacc;
            }
        }
    }

    __syncthreads();
    if (*abort_v) {
        // drain (bounded): the issuer's MMAs in flight and every bulk copy
        // still owed to a stage
        if (tid == L::kWarpMma * 32) {
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0);
        }
        if (tid == L::kWarpOp * 32) {
            for (int s = 0; s < NS; ++s)
                if (issued_par[s] >= 0) mbar_wait(&fullB_bar[s], (uint32_t)issued_par[s]);
            atomicOr(a.err, ERR_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(a.tmem_cols)
                     : "memory");
}

// Work list of the M2L launch, first part: one block per tile finds the
// offsets with at least one source among the tile's targets and stores them
// in increasing order.  Up to level kBitmapLevel the level's occupancy is a
// bitmap of x-rows (one 64-bit word per (y, z) row) in shared memory, so an
// (offset, target row) test is one shift and one AND; deeper levels test
// each (offset, target) through the cell-id table.
constexpr int kPlanThreads = 512;
constexpr int kWaveItems = 148;
constexpr int kBitmapLevel = 6;

__host__ __device__ inline int tc_plan_smem_bytes(int D) {
    const int l = D < kBitmapLevel ? D : kBitmapLevel;
    return 2 * (1 << (2 * l)) * (int)sizeof(unsigned long long);
}

__global__ void __launch_bounds__(kPlanThreads) k_tc_plan(TcArgs a, TcTile* tiles) {
    extern __shared__ unsigned long long bm[];  // occupancy rows | target rows
    __shared__ uint8_t flag[343];
    __shared__ int rowlist[kTcRows];
    __shared__ int wcnt[kPlanThreads / 32];
    __shared__ int t_level, t_oct, t_base, t_rows, nrows;
    __shared__ LevelInfo li;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    stage_linfo(a.linfo, &li);
    __syncthreads();
    if (tid == 0) {
        if (!tc_tile(li, a.D, blockIdx.x, t_level, t_oct, t_base, t_rows)) t_rows = 0;
        nrows = 0;
    }
    for (int i = tid; i < 343; i += kPlanThreads) flag[i] = 0;
    __syncthreads();
    const int rows = t_rows, l = t_level, base = t_base;
    if (rows <= 0) return;  // uniform
    const int side = 1 << l;
    if (l <= kBitmapLevel) {
        const int nr = side * side;
        unsigned long long* occ = bm;
        unsigned long long* tg = bm + nr;
        for (int i = tid; i < 2 * nr; i += kPlanThreads) bm[i] = 0ull;
        __syncthreads();
        for (int c = li.gbase[l] + tid; c < li.gbase[l + 1]; c += kPlanThreads) {
            int x, y, z;
            demorton3(a.code[c], x, y, z);
            atomicOr(&occ[z * side + y], 1ull << x);
        }
        for (int r = tid; r < rows; r += kPlanThreads) {
            int x, y, z;
            demorton3(a.code[base + r], x, y, z);
            if (atomicOr(&tg[z * side + y], 1ull << x) == 0ull) rowlist[atomicAdd(&nrows, 1)] = z * side + y;
        }
        __syncthreads();
        const int K = nrows;
        for (int i = tid; i < 343 * K; i += kPlanThreads) {
            const int op = i / K;
            if (flag[op]) continue;
            const int ox = op / 49 - 3, oy = (op / 7) % 7 - 3, oz = op % 7 - 3;
            if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
            const int row = rowlist[i % K];
            const int ty = row % side, tz = row / side;
            if (oy < (ty & 1) - 3 || oy > (ty & 1) + 2 || oz < (tz & 1) - 3 || oz > (tz & 1) + 2)
                continue;
            const int sy = ty - oy, sz = tz - oz;
            if (sy < 0 || sz < 0 || sy >= side || sz >= side) continue;
            const unsigned long long src = occ[sz * side + sy];
            const unsigned long long sh = ox >= 0 ? (src << ox) : (src >> -ox);
            unsigned long long tb = tg[row];
            // x parity: offset +3 needs an odd target x, -3 an even one
            if (ox == 3) tb &= 0xAAAAAAAAAAAAAAAAull;
            else if (ox == -3) tb &= 0x5555555555555555ull;
            if (sh & tb) flag[op] = 1;
        }
    } else {
        for (int i = tid; i < 343 * rows; i += kPlanThreads) {
            const int op = i / rows;
            if (flag[op]) continue;
            const int ox = op / 49 - 3, oy = (op / 7) % 7 - 3, oz = op % 7 - 3;
            if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
            int x, y, z;
            demorton3(a.code[base + i % rows], x, y, z);
            if (!tc_admits(ox, oy, oz, x & 1, y & 1, z & 1)) continue;
            const int sx = x - ox, sy = y - oy, sz = z - oz;
            if (sx < 0 || sy < 0 || sz < 0 || sx >= side || sy >= side || sz >= side) continue;
            if (a.cid[a.off[l] + morton3(sx, sy, sz)] >= 0) flag[op] = 1;
        }
    }
    __syncthreads();
    // flagged offsets in increasing order
    const bool f = tid < 343 && flag[tid];
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcnt[wid] = __popc(bal);
    __syncthreads();
    TcTile& tl = tiles[blockIdx.x];
    if (f) {
        int pos = __popc(bal & ((1u << lane) - 1u));
        for (int v = 0; v < wid; ++v) pos += wcnt[v];
        tl.terms[pos] = (uint16_t)tid;
    }
    if (tid == 0) {
        int cnt = 0;
        for (int v = 0; v < kPlanThreads / 32; ++v) cnt += wcnt[v];
        tl.level = l;
        tl.oct = t_oct;
        tl.base = base;
        tl.rows = rows;
        tl.cnt = cnt;
    }
}

// Cuts every tile's list into runs (one work item each), in tile order.
// Run length: short enough that there are about a wave of runs, and never
// more than chain_cap offsets, because the tensor-core accumulator rounds
// every accumulation toward zero and its error grows with the number of
// products summed into it (runs are summed afterwards in FP32 round to
// nearest); long enough that the runs with rank > 0 fit slab_cap partial
// slabs.  One block; tiles in chunks.
constexpr int kItemThreads = 1024;

__global__ void __launch_bounds__(kItemThreads) k_tc_items(int D, const LevelInfo* linfo,
                                                           int ntile_cap, int slab_cap, int chain_cap,
                                                           TcPlanHdr* hdr, TcTile* tiles,
                                                           TcItem* items) {
    __shared__ int warp_sum[32];
    __shared__ int s_total, s_ntile, s_carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        int ntile = 0;  // tiles are numbered densely from 0 (the plan's order)
        for (int l = 2; l <= D; ++l) ntile += tc_level_tiles(*linfo, l);
        s_ntile = ntile < ntile_cap ? ntile : ntile_cap;
        s_carry = 0;
    }
    __syncthreads();
    const int ntile = s_ntile;
    // total non-empty offsets over all tiles
    int part = 0;
    for (int b = tid; b < ntile; b += kItemThreads) part += tiles[b].cnt;
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) warp_sum[wid] = part;
    __syncthreads();
    if (tid == 0) {
        int t = 0;
        for (int w = 0; w < kItemThreads / 32; ++w) t += warp_sum[w];
        s_total = t;
    }
    __syncthreads();
    const int total = s_total;
    int tpi = (total + kWaveItems - 1) / kWaveItems;
    if (tpi > chain_cap) tpi = chain_cap;
    const int tpi_mem = (total + slab_cap - 1) / slab_cap;
    if (tpi < tpi_mem) tpi = tpi_mem;
    if (tpi < 1) tpi = 1;
    // tiles in chunks of kItemThreads: exclusive scan of the run counts
    for (int c0 = 0; c0 < ntile; c0 += kItemThreads) {
        const int b = c0 + tid;
        int cnt = 0, ns = 0;
        if (b < ntile) {
            cnt = tiles[b].cnt;
            ns = (cnt + tpi - 1) / tpi;
            if (ns < 1) ns = 1;
        }
        int x = ns;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncthreads();
        if (lane == 31) warp_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = warp_sum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sum[lane] = w;
        }
        __syncthreads();
        const int off = s_carry + (wid > 0 ? warp_sum[wid - 1] : 0) + x - ns;
        if (b < ntile) {
            tiles[b].nsplit = ns;
            tiles[b].item0 = off;
            for (int k = 0; k < ns; ++k) {
                TcItem it;
                it.tile = b;
                it.begin = (cnt * k) / ns;
                it.end = (cnt * (k + 1)) / ns;
                it.rank = k;
                items[off + k] = it;
            }
        }
        __syncthreads();
        if (tid == 0) s_carry += warp_sum[kItemThreads / 32 - 1];
        __syncthreads();
    }
    if (tid == 0) {
        hdr->n_tiles = ntile;
        hdr->n_items = s_carry;
    }
}

// L += the partial slabs of the M2L items of rank > 0, per tile in rank
// order; 32 blocks per tile, each a slice of its rows, eight slabs in flight.
constexpr int kRedSlices = 32;

__global__ void __launch_bounds__(256) k_tc_reduce_tiles(int ld, const TcPlanHdr* hdr,
                                                         const TcTile* tiles,
                                                         const float4* __restrict__ slabs,
                                                         float4* L) {
    const int n_tiles = hdr->n_tiles;
    const int w = ld / 4;
    const int64_t slab4 = (int64_t)kTcRows * w;
    for (int bb = blockIdx.x; bb < n_tiles * kRedSlices; bb += gridDim.x) {
        const int b = bb / kRedSlices, slice = bb % kRedSlices;
        const int ns = tiles[b].nsplit, base = tiles[b].base, rows = tiles[b].rows;
        if (ns <= 1) continue;
        const float4* first = slabs + (int64_t)(tiles[b].item0 + 1) * slab4;
        const int r0 = (rows * slice) / kRedSlices, r1 = (rows * (slice + 1)) / kRedSlices;
        for (int e = threadIdx.x; e < (r1 - r0) * w; e += blockDim.x) {
            const int64_t local = (int64_t)(r0 + e / w) * w + (e % w);
            const int64_t idx = (int64_t)base * w + local;
            float4 v = L[idx];
            int k = 0;
            for (; k + 8 <= ns - 1; k += 8) {
                float4 q[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) q[u] = first[(k + u) * slab4 + local];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    v.x += q[u].x; v.y += q[u].y; v.z += q[u].z; v.w += q[u].w;
                }
            }
            for (; k < ns - 1; ++k) {
                const float4 q = first[k * slab4 + local];
                v.x += q.x; v.y += q.y; v.z += q.z; v.w += q.w;
            }
            L[idx] = v;
        }
    }
}

// L += the split partials of M2L, for every cell of levels 2..D (fixed order,
// whole padded rows: the partials' padding stays zero from allocation).
__global__ void k_tc_reduce(int lfirst, int llast, int ld, int nparts, const LevelInfo* linfo,
                            const float4* __restrict__ part, int64_t part_stride4, float4* L) {
    pdl_wait();
    const int64_t g0 = linfo->gbase[lfirst], g1 = linfo->gbase[llast + 1];
    const int64_t w = ld / 4;
    for (int64_t e = g0 * w + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g1 * w;
         e += (int64_t)gridDim.x * blockDim.x) {
        float4 v = L[e];
        for (int s = 0; s < nparts; ++s) {
            const float4 q = part[s * part_stride4 + e];
            v.x += q.x;
            v.y += q.y;
            v.z += q.z;
            v.w += q.w;
        }
        L[e] = v;
    }
}

}  // namespace

void host_m2l_offsets(int16_t out[8][189]);

int m2l_tc_npad(int p) { return tc_geom(p, true).Npad; }

// TMA descriptor of the pair-packed partial rows: rows_cap rows of Npad FP32
// values, stored by boxes of 128 rows x 16 columns with the 64-byte swizzle.
cudaError_t m2l_tc_make_part_map(Workspace& ws) {
    ws.pp_map_ok = 0;
    if (!ws.pp_part || !ws.tc_bf16) return cudaSuccess;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const int npad = m2l_tc_npad(ws.p);
    const cuuint64_t dims[2] = {(cuuint64_t)npad, (cuuint64_t)ws.pp_rows_cap};
    const cuuint64_t strides[1] = {(cuuint64_t)npad * sizeof(float)};
    const cuuint32_t box[2] = {16, (cuuint32_t)kTcRows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(reinterpret_cast<CUtensorMap*>(ws.pp_map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        2, ws.pp_part, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    ws.pp_map_ok = 1;
    return cudaSuccess;
}

size_t m2l_tc_operand_bytes(int p, bool bf16) {
    if (!tc_supported(p, bf16)) return 0;
    TcGeom g = tc_geom(p, bf16);
    return (size_t)kNumOps * g.kchunks * g.pieces * g.b_bytes;
}

size_t m2l_tc_partial_splits(int p, int64_t cells_max, int ld) {
    const double budget = 512.0 * 1024 * 1024;
    double per = (double)cells_max * ld * sizeof(float);
    int s = 1 + (int)(budget / per);
    if (s > kMaxSplits) s = kMaxSplits;
    (void)p;
    return (size_t)s;
}

int64_t m2l_tc_slab_cap(int ld, int64_t tiles_cap, int64_t n_max) {
    // 16 KB per ion, within [16 MB, 8 GB]: enough slabs for runs of
    // kChainCap offsets up to about a million ions at p <= 12 (beyond, runs
    // lengthen), small for the small crystals of an ensemble
    double budget = 16384.0 * (double)n_max;
    if (budget < 16.0 * 1024 * 1024) budget = 16.0 * 1024 * 1024;
    if (budget > 8192.0 * 1024 * 1024) budget = 8192.0 * 1024 * 1024;
    int64_t s = (int64_t)(budget / ((double)kTcRows * ld * sizeof(float)));
    if (s > tiles_cap * 189) s = tiles_cap * 189;
    return s > 1 ? s : 1;
}

size_t m2l_tc_part_floats(int64_t cells_max, int ld, int m2m_splits, int64_t tiles_cap,
                          int64_t slab_cap) {
    const size_t m2m = (size_t)(m2m_splits > 1 ? m2m_splits - 1 : 1) * cells_max * ld;
    const size_t m2l = (size_t)(tiles_cap + slab_cap) * kTcRows * ld;
    return m2m > m2l ? m2m : m2l;
}

// Operators 0..342: M2L by offset index; 343..350: M2M by child octant;
// 351..358: L2L by child octant.  Each P x P (out x in) operator T becomes B
// with B[k][n] = T[n][k], split into pieces (TF32 hi/lo or BF16 hi/mid/lo)
// and swizzled per 32-wide K chunk: [op][chunk][piece][Npad rows].
void m2l_tc_pack_operands(int p, bool bf16, const double* T_m2l, const double* T_m2m,
                          const double* T_l2l, void* out) {
    const TcGeom g = tc_geom(p, bf16);
    const int P = g.P;
    unsigned char* bytes = static_cast<unsigned char*>(out);
    for (int opi = 0; opi < kNumOps; ++opi) {
        const double* T = opi < kOpM2M ? T_m2l + (size_t)opi * P * P
                          : opi < kOpL2L ? T_m2m + (size_t)(opi - kOpM2M) * P * P
                                         : T_l2l + (size_t)(opi - kOpL2L) * P * P;
        for (int kc = 0; kc < g.kchunks; ++kc) {
            unsigned char* chunk = bytes + ((size_t)opi * g.kchunks + kc) * g.pieces * g.b_bytes;
            for (int n = 0; n < g.Npad; ++n)
                for (int k = 0; k < 32; ++k) {
                    const int kk = kc * 32 + k;
                    const double t = (n < P && kk < P) ? T[(size_t)n * P + kk] : 0.0;
                    if (bf16) {
                        const uint16_t h = bf16_bits_host((float)t);
                        const double r1 = t - bf16_value_host(h);
                        const uint16_t m = bf16_bits_host((float)r1);
                        const double r2 = r1 - bf16_value_host(m);
                        const uint16_t l = bf16_bits_host((float)r2);
                        const size_t o = swz64_off(n, k);
                        memcpy(chunk + o, &h, 2);
                        memcpy(chunk + g.b_bytes + o, &m, 2);
                        memcpy(chunk + 2 * g.b_bytes + o, &l, 2);
                    } else {
                        const float h = rna_tf32_host((float)t);
                        const float r = rna_tf32_host((float)(t - (double)h));
                        const size_t o = swz_off(n, k);
                        memcpy(chunk + o, &h, 4);
                        memcpy(chunk + g.b_bytes + o, &r, 4);
                    }
                }
        }
    }
}

// pdl: a programmatic dependent launch (launch_pdl); the M2L launches stay
// plain (the ensemble's graph rewrite takes their edges as they are)
template <int MODE>
static cudaError_t tc_launch_mode(const TcArgs& a, unsigned grid, int smem, cudaStream_t s,
                                  bool pdl) {
    if (pdl) {
        if (a.bf16)
            return launch_pdl(k_m2l_tc<MODE, 1>, dim3(grid), dim3(TcLayout<MODE, 1>::kThreads),
                              (size_t)smem, s, a);
        return launch_pdl(k_m2l_tc<MODE, 0>, dim3(grid), dim3(TcLayout<MODE, 0>::kThreads),
                          (size_t)smem, s, a);
    }
    if (a.bf16) k_m2l_tc<MODE, 1><<<grid, TcLayout<MODE, 1>::kThreads, smem, s>>>(a);
    else k_m2l_tc<MODE, 0><<<grid, TcLayout<MODE, 0>::kThreads, smem, s>>>(a);
    return cudaGetLastError();
}
static cudaError_t tc_launch(const TcArgs& a, unsigned grid, int smem, cudaStream_t s,
                             bool pdl = false) {
    if (a.mode == MODE_PAIR) return tc_launch_mode<MODE_PAIR>(a, grid, smem, s, false);
    if (a.mode == MODE_M2L) return tc_launch_mode<MODE_M2L>(a, grid, smem, s, false);
    if (a.mode == MODE_M2M) return tc_launch_mode<MODE_M2M>(a, grid, smem, s, pdl);
    return tc_launch_mode<MODE_L2L>(a, grid, smem, s, pdl);
}

cudaError_t m2l_tc_init() {
    cudaError_t e = cudaFuncSetAttribute(k_tc_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc_plan_smem_bytes(kBitmapLevel));
    if (e != cudaSuccess) return e;
    int most = 0;
    for (int q = 2; q <= kMaxOrder; ++q)
        for (int b = 0; b < 2; ++b)
            if (tc_supported(q, b) && tc_geom(q, b).smem_bytes > most) most = tc_geom(q, b).smem_bytes;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t r = cudaSuccess;
    auto set = [&](const void* f) {
        if (r == cudaSuccess) r = cudaFuncSetAttribute(f, at, most);
    };
    set((const void*)k_m2l_tc<MODE_M2L, 0>);
    set((const void*)k_m2l_tc<MODE_M2L, 1>);
    set((const void*)k_m2l_tc<MODE_PAIR, 0>);
    set((const void*)k_m2l_tc<MODE_PAIR, 1>);
    set((const void*)k_m2l_tc<MODE_M2M, 0>);
    set((const void*)k_m2l_tc<MODE_M2M, 1>);
    set((const void*)k_m2l_tc<MODE_L2L, 0>);
    set((const void*)k_m2l_tc<MODE_L2L, 1>);
    return r;
}

static TcArgs base_args(int64_t n, int D, Workspace& ws, int splits) {
    (void)n;
    const bool bf16 = ws.tc_bf16 != 0;
    TcGeom g = tc_geom(ws.p, bf16);
    TcArgs a;
    memset(&a, 0, sizeof a);
    a.D = D;
    a.P = g.P;
    a.ld = ws.ld;
    a.kchunks = g.kchunks;
    a.Npad = g.Npad;
    a.tmem_cols = g.tmem_cols;
    a.acc_cols = g.acc_cols;
    a.splits = splits;
    a.stages = g.stages;
    a.raw = g.raw;
    a.epi_half = g.epi_half;
    a.epi_stride = g.epi_stride;
    a.bf16 = bf16 ? 1 : 0;
    a.pieces = g.pieces;
    a.a_bytes = g.a_bytes;
    a.b_bytes = g.b_bytes;
    a.idesc = bf16 ? idesc_bf16(g.Npad, kTcRows) : idesc_tf32(g.Npad, kTcRows);
    a.linfo = ws.linfo;
    a.code = ws.code;
    a.cid = ws.cid;
    DenseLayout dl = dense_layout(D);
    for (int l = 0; l < kMaxDepth + 2; ++l) a.off[l] = dl.off[l];
    a.M = (const float*)ws.M;
    a.L = (float*)ws.L;
    a.Mout = (float*)ws.M;
    a.part = ws.tc_part;
    a.part_stride = ws.cells_max * ws.ld;
    a.ops = static_cast<const unsigned char*>(ws.T_m2l_tc);
    a.Mp = ws.M_pieces;
    a.err = ws.err;
    return a;
}

static int64_t level_cells(int64_t n, int l) {
    int64_t cl = (int64_t)1 << (3 * l);
    return n < cl ? n : cl;
}

cudaError_t launch_m2m_tc(int64_t n, int D, int l, Workspace& ws, cudaStream_t s) {
    const int64_t tiles = (level_cells(n, l) + kTcRows - 1) / kTcRows;
    // split the 8 child terms across CTAs when the level has few tiles
    int splits = (int)((152 + tiles - 1) / tiles);
    if (splits > 8) splits = 8;
    if (splits > ws.tc_splits_max) splits = ws.tc_splits_max;
    if (splits < 1) splits = 1;
    TcArgs a = base_args(n, D, ws, splits);
    a.mode = MODE_M2M;
    a.level = l;
    cudaError_t e = tc_launch(a, (unsigned)(tiles * splits), tc_geom(ws.p, ws.tc_bf16 != 0).smem_bytes, s,
                              true);
    if (e != cudaSuccess || splits == 1) return e;
    return launch_pdl(k_tc_reduce, dim3(152 * 2), dim3(256), 0, s, l, l, ws.ld, splits - 1,
                      (const LevelInfo*)ws.linfo, (const float4*)ws.tc_part,
                      (int64_t)(ws.cells_max * ws.ld / 4), (float4*)ws.M);
}

// M of the cells of levels lfirst..llast as bf16 hi/mid/lo pieces
// (split_bf16x3, the split the M2L producers would otherwise repeat for
// every target that gathers the cell), with the mirrored copies that the
// pairs of -o read: Mp[(cell * kPieceRows + q) * ld + k].  The other levels'
// pieces are stored by the kernels that compute their M.
__global__ void k_split_m(int lfirst, int llast, int ld, const LevelInfo* linfo, const float* M,
                          uint16_t* Mp) {
    pdl_wait();
    const int64_t g0 = linfo->gbase[lfirst], g1 = linfo->gbase[llast + 1];
    for (int64_t e = g0 * ld + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g1 * ld;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = e / ld, k = e - cell * ld;
        store_pieces(Mp, cell, ld, (int)k, M[e]);
    }
}

// The M2L work list of the current tree (tiles, their non-empty offsets,
// the work items); it reads the tree only.
static bool tc_worklist_layout(int64_t n, int D, Workspace& ws, int64_t& tiles, TcPlanHdr*& hdr,
                               TcTile*& tl, TcItem*& items) {
    tiles = 0;
    for (int l = 2; l <= D; ++l) tiles += (level_cells(n, l) + kTcRows - 1) / kTcRows + 8;
    hdr = (TcPlanHdr*)ws.tc_work;
    tl = (TcTile*)(hdr + 1);
    items = (TcItem*)(tl + ws.tc_tiles_cap);
    return tiles <= ws.tc_tiles_cap;
}


// Free TMEM columns of the pair kernel (all 512 allocated): after each
// accumulator's Npad columns up to acc_cols, then after both accumulators.
// The BF16 epilogue parks the summed second half of the columns there.
static bool pair_epi_scratch_fits(const TcArgs& a) {
    const int need = a.Npad - a.epi_half;
    const int free = 2 * (a.acc_cols - a.Npad) + (512 - 2 * a.acc_cols);
    return need <= free;
}

static TcArgs pair_args(int64_t n, int D, Workspace& ws) {
    TcArgs a = base_args(n, D, ws, 1);
    a.mode = MODE_PAIR;
    if (a.bf16) {
        a.tmem_cols = 512;
        a.epi_scratch = pair_epi_scratch_fits(a) ? 1 : 0;
    }
    memcpy(&a.part_map, ws.pp_map, sizeof(CUtensorMap));
    PairList L = pair_list(ws);
    a.pairs = L.pairs;
    a.pitems = L.items;
    a.phdr = L.hdr;
    a.ppart = (float*)ws.pp_part;
    return a;
}

cudaError_t launch_m2l_tc_worklist(int64_t n, int D, Workspace& ws, cudaStream_t s) {
    if (D < 2) return cudaSuccess;
    if (ws.m2l_pairs) return launch_m2l_pairs_worklist(n, D, ws, s);
    int64_t tiles;
    TcPlanHdr* hdr;
    TcTile* tl;
    TcItem* items;
    if (!tc_worklist_layout(n, D, ws, tiles, hdr, tl, items)) return cudaErrorInvalidValue;
    TcArgs a = base_args(n, D, ws, 1);
    a.mode = MODE_M2L;
    a.tiles = tl;
    a.items = items;
    a.hdr = hdr;
    k_tc_plan<<<(unsigned)tiles, kPlanThreads, tc_plan_smem_bytes(D), s>>>(a, tl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tc_items<<<1, kItemThreads, 0, s>>>(D, ws.linfo, (int)tiles, (int)ws.tc_slab_cap,
                                          n > kChainLargeIons ? kChainCapLarge : kChainCap, hdr, tl,
                                          items);
    return cudaGetLastError();
}

// L2L shifts level by level, levels 3 .. l2l_last (level 2 has no parent
// expansion); each adds the cell's own M2L result already in L.
static cudaError_t launch_l2l_levels(int64_t n, int D, Workspace& ws, int l2l_last, int smem,
                                     cudaStream_t s) {
    for (int l = 3; l <= l2l_last && l <= D; ++l) {
        if (level_cap(n, l) <= kShiftSmallL2L) {
            cudaError_t e = launch_shift_small(1, n, D, l, ws, s);
            if (e != cudaSuccess) return e;
            continue;
        }
        TcArgs b = base_args(n, D, ws, 1);
        b.mode = MODE_L2L;
        b.level = l;
        const int64_t t2 = (level_cells(n, l) + kTcRows - 1) / kTcRows + 8;
        cudaError_t e = tc_launch(b, (unsigned)t2, smem, s, true);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static int sm_count() {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 152;
}

// CTAs of the persistent M2L launch: one per SM, or the plan's cap
static unsigned m2l_grid(const Workspace& ws) {
    const int sms = sm_count();
    return (unsigned)(ws.m2l_ctas > 0 && ws.m2l_ctas < sms ? ws.m2l_ctas : sms);
}

cudaError_t launch_m2l_tc_run(int64_t n, int D, Workspace& ws, int l2l_last, int split_last,
                              cudaStream_t s, cudaEvent_t after_m2l) {
    if (D < 2) return cudaSuccess;
    const int smem = tc_geom(ws.p, ws.tc_bf16 != 0).smem_bytes;
    if (ws.m2l_pairs) {
        TcArgs a = pair_args(n, D, ws);
        cudaError_t e;
        if (ws.tc_bf16 && split_last >= 3) {
            if ((e = launch_pdl(k_split_m, dim3(152 * 8), dim3(256), 0, s, 3, split_last, ws.ld,
                                (const LevelInfo*)ws.linfo, (const float*)ws.M, ws.M_pieces)) !=
                cudaSuccess)
                return e;
        }
        if (ws.kev[0] && (e = record_timing(ws.kev[0], s)) !=
                             cudaSuccess)
            return e;
        if ((e = tc_launch(a, m2l_grid(ws), smem, s)) != cudaSuccess) return e;
        if (ws.kev[1] && (e = record_timing(ws.kev[1], s)) !=
                             cudaSuccess)
            return e;
        if (after_m2l && (e = cudaEventRecord(after_m2l, s)) != cudaSuccess) return e;
        if ((e = launch_m2l_pairs_reduce(n, D, ws, a.Npad, s)) != cudaSuccess) return e;
        return launch_l2l_levels(n, D, ws, l2l_last, smem, s);
    }
    int64_t tiles;
    TcPlanHdr* hdr;
    TcTile* tl;
    TcItem* items;
    if (!tc_worklist_layout(n, D, ws, tiles, hdr, tl, items)) return cudaErrorInvalidValue;
    TcArgs a = base_args(n, D, ws, 1);
    a.mode = MODE_M2L;
    a.tiles = tl;
    a.items = items;
    a.hdr = hdr;
    cudaError_t e;
    if (ws.tc_bf16) {
        if (split_last >= 3)
            k_split_m<<<152 * 8, 256, 0, s>>>(3, split_last, ws.ld, ws.linfo, (const float*)ws.M,
                                              ws.M_pieces);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // persistent: one CTA per SM walks the work list
    if (ws.kev[0] && (e = record_timing(ws.kev[0], s)) !=
                         cudaSuccess)
        return e;
    if ((e = tc_launch(a, m2l_grid(ws), smem, s)) != cudaSuccess) return e;
    if (ws.kev[1] && (e = record_timing(ws.kev[1], s)) !=
                         cudaSuccess)
        return e;
    if (after_m2l && (e = cudaEventRecord(after_m2l, s)) != cudaSuccess) return e;
    const int64_t rg = tiles * kRedSlices;
    k_tc_reduce_tiles<<<(unsigned)(rg < 152 * 16 ? rg : 152 * 16), 256, 0, s>>>(
        ws.ld, hdr, tl, (const float4*)ws.tc_part, (float4*)ws.L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_l2l_levels(n, D, ws, l2l_last, smem, s);
}

// Work-list counts of the last M2L launch: {tiles, tile-offset products
// (sum of the tiles' non-empty offsets), work items, target rows}.
cudaError_t m2l_tc_work_stats(const Workspace& ws, int64_t* out, cudaStream_t s) {
    for (int k = 0; k < 4; ++k) out[k] = 0;
    if (ws.m2l_pairs) return m2l_pairs_stats(ws, out, s);
    if (!ws.tc_work) return cudaSuccess;
    TcPlanHdr h;
    cudaError_t e = cudaMemcpyAsync(&h, ws.tc_work, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (h.n_tiles <= 0 || h.n_tiles > ws.tc_tiles_cap) return cudaSuccess;
    std::vector<TcTile> t((size_t)h.n_tiles);
    e = cudaMemcpyAsync(t.data(), (const TcPlanHdr*)ws.tc_work + 1, sizeof(TcTile) * t.size(),
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    out[0] = h.n_tiles;
    out[2] = h.n_items;
    for (const TcTile& x : t) {
        out[1] += x.cnt;
        out[3] += x.rows;
    }
    return cudaSuccess;
}

size_t m2l_tc_work_bytes(int64_t tiles_cap, int64_t slab_cap) {
    return sizeof(TcPlanHdr) + (size_t)tiles_cap * sizeof(TcTile) +
           (size_t)(tiles_cap + slab_cap) * sizeof(TcItem);
}

// ---------------------------------------------------------------------------
// Joined M2L of an ensemble.  Every BF16 pair-packed member's M2L launch in
// a captured ensemble graph is replaced by one launch over all members'
// items: a member's partial rows are the same products as in its own launch
// (a row depends on its own source row and the offset's operator only), so
// results are unchanged bit for bit, while the members' M2L phases share the
// SMs instead of each taking all of them in turn.
// ---------------------------------------------------------------------------

// pm_prefix[k] = items of members 0 .. k-1 (a member whose pool overflowed
// has none); one block
constexpr int kJoinThreads = 1024;
__global__ void __launch_bounds__(kJoinThreads) k_pm_prefix(const PairMember* pm, int n,
                                                            int* prefix) {
    __shared__ int s_c[kJoinThreads];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    for (int b = 0; b < n; b += kJoinThreads) {
        const int k = b + (int)threadIdx.x;
        __syncthreads();
        s_c[threadIdx.x] = k < n ? pm[k].hdr->n_items : 0;
        __syncthreads();
        // inclusive scan (Hillis-Steele) over the chunk
        for (int off = 1; off < kJoinThreads; off <<= 1) {
            const int v = threadIdx.x >= (unsigned)off ? s_c[threadIdx.x - off] : 0;
            __syncthreads();
            s_c[threadIdx.x] += v;
            __syncthreads();
        }
        if (k < n) prefix[k + 1] = s_carry + s_c[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == kJoinThreads - 1) s_carry += s_c[kJoinThreads - 1];
    }
    if (threadIdx.x == 0) prefix[0] = 0;
}

size_t m2l_join_member_bytes() { return sizeof(PairMember); }

cudaError_t m2l_join_pair_launches(cudaGraph_t g, void* d_members, int* d_prefix, int cap,
                                   int* joined) {
    *joined = 0;
    size_t nn = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &nn);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn && (e = cudaGraphGetNodes(g, nodes.data(), &nn)) != cudaSuccess) return e;
    const void* fn = (const void*)k_m2l_tc<MODE_PAIR, 1>;
    std::vector<cudaGraphNode_t> found;
    std::vector<TcArgs> args;
    cudaKernelNodeParams first{};
    for (cudaGraphNode_t x : nodes) {
        cudaGraphNodeType t;
        if ((e = cudaGraphNodeGetType(x, &t)) != cudaSuccess) return e;
        if (t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        if ((e = cudaGraphKernelNodeGetParams(x, &kp)) != cudaSuccess) return e;
        if (kp.func != fn) continue;
        if (found.empty()) first = kp;
        found.push_back(x);
        args.push_back(*static_cast<const TcArgs*>(kp.kernelParams[0]));
    }
    const int n = (int)found.size();
    if (n < 2) return cudaSuccess;  // nothing to share
    if (n > cap) return cudaErrorInvalidValue;
    std::vector<PairMember> hm((size_t)n);
    for (int k = 0; k < n; ++k) {
        memset(&hm[k], 0, sizeof(PairMember));
        hm[k].map = args[k].part_map;
        hm[k].items = args[k].pitems;
        hm[k].pairs = args[k].pairs;
        hm[k].Mp = args[k].Mp;
        hm[k].hdr = args[k].phdr;
    }
    if ((e = cudaMemcpy(d_members, hm.data(), sizeof(PairMember) * n, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return e;
    // the joined launch waits for every member's inputs and precedes every
    // member's consumers of its partial rows
    // (an edge to a successor may be programmatic: its edge data is kept)
    std::vector<cudaGraphNode_t> preds, succs;
    std::vector<cudaGraphEdgeData> succ_ed;
    for (cudaGraphNode_t x : found) {
        size_t np = 0, ns = 0;
        if ((e = cudaGraphNodeGetDependencies(x, nullptr, nullptr, &np)) != cudaSuccess ||
            (e = cudaGraphNodeGetDependentNodes(x, nullptr, nullptr, &ns)) != cudaSuccess)
            return e;
        std::vector<cudaGraphNode_t> a(np), b(ns);
        std::vector<cudaGraphEdgeData> ea(np), eb(ns);
        if (np && (e = cudaGraphNodeGetDependencies(x, a.data(), ea.data(), &np)) != cudaSuccess)
            return e;
        if (ns && (e = cudaGraphNodeGetDependentNodes(x, b.data(), eb.data(), &ns)) != cudaSuccess)
            return e;
        for (size_t i = 0; i < np; ++i)
            if (std::find(preds.begin(), preds.end(), a[i]) == preds.end()) preds.push_back(a[i]);
        for (size_t i = 0; i < ns; ++i)
            if (std::find(succs.begin(), succs.end(), b[i]) == succs.end()) {
                succs.push_back(b[i]);
                succ_ed.push_back(eb[i]);
            }
    }
    const PairMember* dm = static_cast<const PairMember*>(d_members);
    int nm = n;
    void* pargs[] = {(void*)&dm, (void*)&nm, (void*)&d_prefix};
    cudaKernelNodeParams pp{};
    pp.func = (void*)k_pm_prefix;
    pp.gridDim = dim3(1);
    pp.blockDim = dim3(kJoinThreads);
    pp.sharedMemBytes = 0;
    pp.kernelParams = pargs;
    cudaGraphNode_t pnode, jnode;
    if ((e = cudaGraphAddKernelNode(&pnode, g, preds.data(), preds.size(), &pp)) != cudaSuccess)
        return e;
    TcArgs ja = args[0];
    ja.pm = dm;
    ja.pm_prefix = d_prefix;
    ja.n_pm = n;
    void* jargs[] = {(void*)&ja};
    cudaKernelNodeParams jp = first;
    jp.kernelParams = jargs;
    jp.extra = nullptr;
    if ((e = cudaGraphAddKernelNode(&jnode, g, &pnode, 1, &jp)) != cudaSuccess) return e;
    for (size_t i = 0; i < succs.size(); ++i)
        if ((e = cudaGraphAddDependencies(g, &jnode, &succs[i], &succ_ed[i], 1)) != cudaSuccess)
            return e;
    for (cudaGraphNode_t x : found)
        if ((e = cudaGraphDestroyNode(x)) != cudaSuccess) return e;
    *joined = n;
    return cudaSuccess;
}

}  // namespace pt
