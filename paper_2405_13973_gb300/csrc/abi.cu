// abi.cu -- the C entry points of libpenning (declared in include/penning.h):
// plan management, host construction of the translation operators, the step
// loop (captured once per configuration as a CUDA graph and replayed per
// step) and the diagnostics.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <set>
#include <vector>

#include "bf16split.cuh"
#include "internal.h"
#include "m2l_pairs.h"
#include "operators.h"

using namespace pt;

namespace {

constexpr int kWallChunk = 4096;  // steps per wall-phase table upload
// tensor-core plans up to this many ions use the pair-packed M2L schedule
// (above it the tile schedule is faster: its rows are already mostly
// pairs, and it has no partial rows to round-trip)
constexpr int64_t kPairsDefaultIons = 65536;
// CUDA-core plans up to this many ions use the pair work list (rotation M2L
// in FP64), which beats the per-level tile kernel at every size measured;
// the bound keeps the FP64 partial-row pool within a few GB
constexpr int64_t kPairsDefaultIonsCudaCore = 262144;

struct GraphKey {
    int D = -1;
    int64_t n = -1;
    const void* ptr[7] = {nullptr};
    PushParams pp{};
    pt_laser laser{};
    bool profile = false;
    int expand = 0;
    int sched = 0;
    int ctas = 0;
    int pool = 0;
    bool operator==(const GraphKey& o) const {
        return D == o.D && n == o.n && profile == o.profile && expand == o.expand &&
               sched == o.sched && ctas == o.ctas && pool == o.pool &&
               memcmp(ptr, o.ptr, sizeof ptr) == 0 &&
               memcmp(&pp, &o.pp, sizeof pp) == 0 && memcmp(&laser, &o.laser, sizeof laser) == 0;
    }
};

}  // namespace

struct fmm_plan_s {
    int device = 0;
    int64_t n_max = 0;
    int p = 0, P = 0, leaf_max = 32, depth = -1, precision = PT_FP64;
    int phases = PT_PHASE_ALL;
    double damping = 0.0;      // artificial damping rate (1/s) of the push; 0 = off
    // time anchor of the trajectory being stepped: step k's time is
    // anc_t + (k - anc_step) dt, whatever calls the steps are split into
    double anc_t = 0.0, anc_dt = 0.0, end_t = 0.0;
    int64_t anc_step = 0, end_step = -1;
    int last_depth = -1;
    int64_t last_n = 0;
    Workspace ws;
    std::vector<void*> allocs;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    GraphKey gkey;
    int* h_err = nullptr;      // pinned
    // pinned host ring for the per-chunk wall-phase tables and step counters
    // (asynchronous steps may have several chunks in flight)
    static constexpr int kSlots = 8;
    double* h_wall[kSlots] = {nullptr};
    StepCounter* h_steps[kSlots] = {nullptr};
    cudaEvent_t slot_ev[kSlots] = {nullptr};
    int next_slot = 0;
    // The wall-phase table on the device covers steps [win_base, win_base +
    // win_count) of the anchor (win_t, win_step, win_dt) at rotation win_wr;
    // dev_next is the step the device counter will start next once the work
    // enqueued so far has run (-1: unknown).  Chunks inside the window that
    // continue the device counter upload nothing.
    double win_t = 0.0, win_dt = 0.0, win_wr = 0.0;
    int64_t win_step = 0, win_base = 0, win_count = 0;
    int64_t dev_next = -1;
    // per-phase device timing (events captured into the step graph)
    bool profile = false;
    static constexpr int kPhases = 6;
    cudaEvent_t ph_ev[kPhases + 1] = {nullptr};
    cudaEvent_t k_ev[4] = {nullptr};   // kernel timing of profiled steps (Workspace::kev)
    bool ops_held = false;     // holds a reference on the shared operator set
    bool dry = false;          // sizing only (fmm_plan_footprint): nothing is allocated
    bool pp_counted = false;   // the pair pool was checked against a real tree
    size_t dry_bytes = 0;
};

namespace {

std::mutex g_tables_mu;
std::set<int> g_tables_dev;

template <typename T>
bool dalloc(fmm_plan_s* pl, T*& p, size_t bytes) {
    void* v = nullptr;
    if (bytes == 0) bytes = 16;
    if (pl->dry) {  // count (at the allocator's 512-byte granularity), allocate nothing
        pl->dry_bytes += (bytes + 511) / 512 * 512;
        p = nullptr;
        return true;
    }
    if (cudaMalloc(&v, bytes) != cudaSuccess) return false;
    pl->allocs.push_back(v);
    p = (T*)v;
    return true;
}

// the two tensor-core modes share every kernel but the operand format
bool is_tc(int precision) {
    return precision == PT_MIXED_TF32X3 || precision == PT_MIXED_BF16X3;
}

int status_from(cudaError_t e) {
    if (e == cudaSuccess) return PT_OK;
    if (e == cudaErrorMemoryAllocation) return PT_ERR_OOM;
    if (e == cudaErrorNotSupported) return PT_ERR_UNSUPPORTED;
    return PT_ERR_CUDA;
}

// Translation operators are read-only and depend only on (device, p,
// precision): plans of the same kind share one copy (an ensemble of hundreds
// of crystals would otherwise hold hundreds of identical 100 MB sets).
struct OpSet {
    int refs = 0;
    void* T_m2m = nullptr;
    void* T_l2l = nullptr;
    void* T_m2l = nullptr;
    void* T_m2l_tc = nullptr;
    void* T_rot = nullptr;   // rotation-based M2L operators (CUDA-core precisions)
};
std::mutex g_ops_mu;
std::map<std::tuple<int, int, int>, OpSet> g_ops;

void release_ops(fmm_plan_s* pl) {
    if (!pl->ops_held) return;
    std::lock_guard<std::mutex> g(g_ops_mu);
    auto it = g_ops.find(std::make_tuple(pl->device, pl->p, pl->precision));
    if (it != g_ops.end() && --it->second.refs == 0) {
        cudaFree(it->second.T_m2m);
        cudaFree(it->second.T_l2l);
        cudaFree(it->second.T_m2l);
        if (it->second.T_m2l_tc) cudaFree(it->second.T_m2l_tc);
        if (it->second.T_rot) cudaFree(it->second.T_rot);
        g_ops.erase(it);
    }
    pl->ops_held = false;
}

// Stream priorities for calls outside a graph: the main chain of a step
// high, the side stream (near field, M2L work list) low, so that freed SMs go
// to the main chain first.  (Step graphs run at the priority of the stream
// they are launched into: measured, node priorities did not help there.)
int prio_high() {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    return hi;
}
int prio_low() {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    return lo;
}

void free_plan(fmm_plan_s* pl) {
    if (!pl) return;
    cudaSetDevice(pl->device);
    cudaDeviceSynchronize();
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    for (void* v : pl->allocs) cudaFree(v);
    release_ops(pl);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    Workspace& ws = pl->ws;
    if (ws.side) cudaStreamDestroy(ws.side);
    if (ws.side2) cudaStreamDestroy(ws.side2);
    for (cudaEvent_t ev : {ws.ev_fork, ws.ev_p2m, ws.ev_items, ws.ev_near})
        if (ev) cudaEventDestroy(ev);
    for (int k = 0; k < fmm_plan_s::kSlots; ++k) {
        if (pl->h_wall[k]) cudaFreeHost(pl->h_wall[k]);
        if (pl->h_steps[k]) cudaFreeHost(pl->h_steps[k]);
        if (pl->slot_ev[k]) cudaEventDestroy(pl->slot_ev[k]);
    }
    for (int k = 0; k <= fmm_plan_s::kPhases; ++k)
        if (pl->ph_ev[k]) cudaEventDestroy(pl->ph_ev[k]);
    for (cudaEvent_t ev : pl->k_ev)
        if (ev) cudaEventDestroy(ev);
    if (pl->h_err) cudaFreeHost(pl->h_err);
    if (ws.h_pp_hdr) cudaFreeHost(ws.h_pp_hdr);
    delete pl;
}

int64_t pow8(int l) { return (int64_t)1 << (3 * l); }

// Uploads operators in the plan's arithmetic type.
template <typename T>
cudaError_t upload_ops(fmm_plan_s* pl, const std::vector<double>& m2m, const std::vector<double>& l2l,
                       const std::vector<double>& m2l) {
    const int P = pl->P;
    std::vector<T> tmp;
    // M2M transposed (in-major) for the warp-per-cell kernel
    tmp.resize((size_t)8 * P * P);
    for (int o = 0; o < 8; ++o)
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c)
                tmp[(size_t)o * P * P + (size_t)c * P + r] = (T)m2m[(size_t)o * P * P + (size_t)r * P + c];
    cudaError_t e = cudaMemcpy(pl->ws.T_m2m, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    tmp.assign(l2l.begin(), l2l.end());
    if ((e = cudaMemcpy(pl->ws.T_l2l, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return e;
    tmp.assign(m2l.begin(), m2l.end());
    return cudaMemcpy(pl->ws.T_m2l, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice);
}

int build_operators(fmm_plan_s* pl) {
    const int p = pl->p, P = pl->P;
    std::vector<double> m2m((size_t)8 * P * P), l2l((size_t)8 * P * P), m2l((size_t)343 * P * P, 0.0);
    for (int o = 0; o < 8; ++o) {
        ops::build_m2m(p, o, &m2m[(size_t)o * P * P]);
        ops::build_l2l(p, o, &l2l[(size_t)o * P * P]);
    }
    for (int ox = -3; ox <= 3; ++ox)
        for (int oy = -3; oy <= 3; ++oy)
            for (int oz = -3; oz <= 3; ++oz) {
                if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                int idx = (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3);
                ops::build_m2l(p, ox, oy, oz, &m2l[(size_t)idx * P * P]);
            }
    cudaError_t e = pl->ws.fp64 ? upload_ops<double>(pl, m2m, l2l, m2l)
                                : upload_ops<float>(pl, m2m, l2l, m2l);
    if (e != cudaSuccess) return status_from(e);
    if (pl->ws.T_rot) {
        // rotation-based M2L operators of every offset index (neighbours zero)
        const int nv = pl->ws.rot_op_vals;
        std::vector<double> rot((size_t)343 * nv, 0.0);
        for (int ox = -3; ox <= 3; ++ox)
            for (int oy = -3; oy <= 3; ++oy)
                for (int oz = -3; oz <= 3; ++oz) {
                    if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                    const int idx = (ox + 3) * 49 + (oy + 3) * 7 + (oz + 3);
                    if (!ops::build_m2l_rotation(p, ox, oy, oz, &rot[(size_t)idx * nv]))
                        return PT_ERR_CUDA;
                }
        if (pl->ws.fp64) {
            e = cudaMemcpy(pl->ws.T_rot, rot.data(), rot.size() * sizeof(double),
                           cudaMemcpyHostToDevice);
        } else {
            std::vector<float> rf(rot.begin(), rot.end());
            e = cudaMemcpy(pl->ws.T_rot, rf.data(), rf.size() * sizeof(float),
                           cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return status_from(e);
    }
    if (is_tc(pl->precision)) {
        const bool bf16 = pl->precision == PT_MIXED_BF16X3;
        std::vector<unsigned char> packed(m2l_tc_operand_bytes(p, bf16));
        m2l_tc_pack_operands(p, bf16, m2l.data(), m2m.data(), l2l.data(), packed.data());
        e = cudaMemcpy(pl->ws.T_m2l_tc, packed.data(), packed.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return status_from(e);
    }
    return PT_OK;
}

// Rotation-based M2L operators: CUDA-core precisions whose operators fit the
// kernel's shared memory.
size_t rot_operator_bytes(const fmm_plan_s* pl) {
    if (is_tc(pl->precision)) return 0;
    const size_t tsz = pl->precision == PT_FP64 ? sizeof(double) : sizeof(float);
    Workspace w = pl->ws;
    w.rot_op_vals = ops::rot_op_vals(pl->p);
    if (m2l_rot_tile(w) == 0) return 0;
    return (size_t)343 * w.rot_op_vals * tsz;
}

// Points the plan at the shared operator set of its (device, p, precision),
// building and uploading it on first use.
int acquire_ops(fmm_plan_s* pl, size_t op_bytes) {
    std::lock_guard<std::mutex> g(g_ops_mu);
    const auto key = std::make_tuple(pl->device, pl->p, pl->precision);
    auto it = g_ops.find(key);
    Workspace& ws = pl->ws;
    if (it == g_ops.end()) {
        OpSet o;
        const size_t tc = is_tc(pl->precision) ? m2l_tc_operand_bytes(pl->p, ws.tc_bf16 != 0) : 0;
        const size_t rot = rot_operator_bytes(pl);
        if (cudaMalloc(&o.T_m2m, 8 * op_bytes) != cudaSuccess ||
            cudaMalloc(&o.T_l2l, 8 * op_bytes) != cudaSuccess ||
            cudaMalloc(&o.T_m2l, 343 * op_bytes) != cudaSuccess ||
            (tc && cudaMalloc(&o.T_m2l_tc, tc) != cudaSuccess) ||
            (rot && cudaMalloc(&o.T_rot, rot) != cudaSuccess)) {
            cudaFree(o.T_m2m);
            cudaFree(o.T_l2l);
            cudaFree(o.T_m2l);
            cudaFree(o.T_m2l_tc);
            return PT_ERR_OOM;
        }
        ws.T_m2m = o.T_m2m;
        ws.T_l2l = o.T_l2l;
        ws.T_m2l = o.T_m2l;
        ws.T_m2l_tc = o.T_m2l_tc;
        ws.T_rot = o.T_rot;
        int r = build_operators(pl);
        if (r != PT_OK) {
            cudaFree(o.T_m2m);
            cudaFree(o.T_l2l);
            cudaFree(o.T_m2l);
            if (o.T_m2l_tc) cudaFree(o.T_m2l_tc);
            if (o.T_rot) cudaFree(o.T_rot);
            ws.T_m2m = ws.T_l2l = ws.T_m2l = ws.T_m2l_tc = ws.T_rot = nullptr;
            return r;
        }
        it = g_ops.emplace(key, o).first;
    }
    it->second.refs++;
    ws.T_m2m = it->second.T_m2m;
    ws.T_l2l = it->second.T_l2l;
    ws.T_m2l = it->second.T_m2l;
    ws.T_m2l_tc = it->second.T_m2l_tc;
    ws.T_rot = it->second.T_rot;
    pl->ops_held = true;
    return PT_OK;
}

int check_err(fmm_plan_s* pl, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(pl->h_err, pl->ws.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_from(e);
    if (*pl->h_err) {
        int v = *pl->h_err;
        cudaMemsetAsync(pl->ws.err, 0, sizeof(int), s);
        cudaStreamSynchronize(s);
        if (v & ERR_NONFINITE) return PT_ERR_NONFINITE;
        if (v & ERR_TIMEOUT) return PT_ERR_TIMEOUT;
        if (v & ERR_CAPACITY) return PT_ERR_OOM;
    }
    return PT_OK;
}

int choose_depth(fmm_plan_s* pl, int64_t n, const double* x, const double* y, const double* z,
                 cudaStream_t s, int* D) {
    if (pl->depth >= 0) {
        *D = pl->depth;
        return PT_OK;
    }
    int32_t counts[kMaxDepth + 1] = {0};
    cudaError_t e = launch_level_counts(n, x, y, z, pl->ws.depth_max, pl->ws, counts, s);
    if (e != cudaSuccess) return status_from(e);
    int r = check_err(pl, s);
    if (r != PT_OK) return r;
    int d = pl->ws.depth_max;
    for (int l = 0; l <= pl->ws.depth_max; ++l) {
        if (counts[l] > 0 && (double)n / (double)counts[l] <= (double)pl->leaf_max) {
            d = l;
            break;
        }
    }
    *D = d;
    return PT_OK;
}

// Pair-packed M2L schedule: the pool of partial rows holds every (target,
// source) pair of a step; 189 sources per cell of levels 2..D bound them.
static int alloc_pairs(fmm_plan_s* pl) {
    Workspace& ws = pl->ws;
    if (ws.pp_work) return PT_OK;
    const int dcap = pl->depth >= 0 ? pl->depth : ws.depth_max;
    int64_t exact = 0;
    for (int l = 2; l <= dcap; ++l) exact += 189 * (pow8(l) < pl->n_max ? pow8(l) : pl->n_max);
    // initial pool: the exact bound, or about twelve pairs per ion if less
    // (the 10,000-ion spheroid has ten); the first call counts its pairs and
    // every later call checks the count of the last step (ensure_pairs)
    int64_t cap = std::min<int64_t>(exact, 12 * pl->n_max + 4096);
    ws.pp_slot_cap = cap > 0 ? cap : 1;
    ws.pp_rows_cap = ws.pp_slot_cap + 343 * 128;
    ws.pp_item_cap = ws.pp_slot_cap / 128 + 344;
    ws.pp_stride = is_tc(pl->precision) ? m2l_tc_npad(pl->p) : ws.ld;
    bool ok = dalloc(pl, ws.pp_work, m2l_pp_work_bytes(ws)) &&
              dalloc(pl, ws.pp_part, m2l_pp_part_bytes(ws));
    if (!ok) {
        ws.pp_work = nullptr;
        ws.pp_part = nullptr;
        return PT_ERR_OOM;
    }
    if (!pl->dry && cudaMemset(ws.pp_work, 0, m2l_pp_work_bytes(ws)) != cudaSuccess)
        return PT_ERR_CUDA;
    if (!pl->dry && ws.tc_bf16 && m2l_tc_make_part_map(ws) != cudaSuccess) return PT_ERR_CUDA;
    if (!pl->dry && !ws.h_pp_hdr) {
        if (cudaMallocHost(&ws.h_pp_hdr, sizeof(M2lPairHdr)) != cudaSuccess) return PT_ERR_CUDA;
        memset(ws.h_pp_hdr, 0, sizeof(M2lPairHdr));
    }
    return PT_OK;
}

// Replaces the pool by one of `cap` pairs (device idle first; graphs that
// captured the old buffers are recaptured through the pool generation).
static int regrow_pairs(fmm_plan_s* pl, int64_t cap) {
    Workspace& ws = pl->ws;
    if (cudaDeviceSynchronize() != cudaSuccess) return PT_ERR_CUDA;
    for (auto it = pl->allocs.begin(); it != pl->allocs.end();) {
        if (*it == ws.pp_work || *it == ws.pp_part) {
            cudaFree(*it);
            it = pl->allocs.erase(it);
        } else {
            ++it;
        }
    }
    ws.pp_work = nullptr;
    ws.pp_part = nullptr;
    ws.pp_slot_cap = cap;
    ws.pp_rows_cap = cap + 343 * 128;
    ws.pp_item_cap = cap / 128 + 344;
    if (!dalloc(pl, ws.pp_work, m2l_pp_work_bytes(ws)) ||
        !dalloc(pl, ws.pp_part, m2l_pp_part_bytes(ws)))
        return PT_ERR_OOM;
    if (cudaMemset(ws.pp_work, 0, m2l_pp_work_bytes(ws)) != cudaSuccess) return PT_ERR_CUDA;
    if (ws.tc_bf16 && m2l_tc_make_part_map(ws) != cudaSuccess) return PT_ERR_CUDA;
    memset(ws.h_pp_hdr, 0, sizeof(M2lPairHdr));
    ++ws.pp_gen;
    return PT_OK;
}

// Pool check of the pair-packed schedule before a call enqueues work: the
// plan's first call counts the pairs of its tree (one synchronising work-list
// pass); later calls read the count that the last step left in pinned host
// memory, and the pool grows by half again once a step used more than 80 %
// of it (a step that overflowed reported PT_ERR_OOM and is counted too).
static int ensure_pairs(fmm_plan_s* pl, int64_t n, const double* x, const double* y,
                        const double* z, const double* q, int D, cudaStream_t s) {
    Workspace& ws = pl->ws;
    if (!ws.m2l_pairs || !ws.h_pp_hdr || D < 2) return PT_OK;
    if (!pl->pp_counted) {
        cudaError_t e = launch_bbox(x, y, z, n, ws, s);
        if (e == cudaSuccess) e = launch_tree(n, x, y, z, q, D, ws, s);
        if (e == cudaSuccess) e = launch_m2l_pairs_worklist(n, D, ws, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return status_from(e);
        int r = check_err(pl, s);  // an overflow of this count is not an error
        if (r != PT_OK && r != PT_ERR_OOM) return r;
        pl->pp_counted = true;
    }
    const M2lPairHdr* h = (const M2lPairHdr*)ws.h_pp_hdr;
    const int64_t used = h->n_pairs;
    if (used > 0 && (h->overflow || 10 * used > 8 * ws.pp_slot_cap))
        return regrow_pairs(pl, used + used / 2 + 4096);
    return PT_OK;
}

// The tile schedule's full pool of partial slabs (plans created for the pair
// schedule hold the minimum).
static int alloc_tile_slabs(fmm_plan_s* pl) {
    Workspace& ws = pl->ws;
    const int64_t want = m2l_tc_slab_cap(ws.ld, ws.tc_tiles_cap, pl->n_max);
    if (ws.tc_slab_cap >= want) return PT_OK;
    const size_t floats = m2l_tc_part_floats(ws.cells_max, ws.ld, ws.tc_splits_max,
                                             ws.tc_tiles_cap, want);
    void *work = nullptr, *part = nullptr;
    if (cudaDeviceSynchronize() != cudaSuccess) return PT_ERR_CUDA;
    if (cudaMalloc(&work, m2l_tc_work_bytes(ws.tc_tiles_cap, want)) != cudaSuccess ||
        cudaMalloc(&part, sizeof(float) * floats) != cudaSuccess) {
        cudaFree(work);
        return PT_ERR_OOM;
    }
    if (cudaMemset(work, 0, m2l_tc_work_bytes(ws.tc_tiles_cap, want)) != cudaSuccess ||
        cudaMemset(part, 0, sizeof(float) * floats) != cudaSuccess) {
        cudaFree(work);
        cudaFree(part);
        return PT_ERR_CUDA;
    }
    for (void*& v : pl->allocs) {
        if (v == ws.tc_work) {
            cudaFree(v);
            v = work;
        } else if (v == (void*)ws.tc_part) {
            cudaFree(v);
            v = part;
        }
    }
    ws.tc_work = work;
    ws.tc_part = (float*)part;
    ws.tc_slab_cap = want;
    ws.tc_part_floats = floats;
    if (pl->graph) {  // captured with the old buffers
        cudaGraphExecDestroy(pl->graph);
        pl->graph = nullptr;
        pl->gkey = GraphKey{};
    }
    return PT_OK;
}

int forces_impl(fmm_plan_s* pl, int64_t n, const double* x, const double* y, const double* z,
                const double* q, double* E, double* phi, cudaStream_t s, int D) {
    int r = ensure_pairs(pl, n, x, y, z, q, D, s);
    if (r != PT_OK) return r;
    // with profiling on, the M2L and near-field kernels are timed as in a step
    for (int k = 0; k < 4; ++k) pl->ws.kev[k] = pl->profile ? pl->k_ev[k] : nullptr;
    cudaError_t e = launch_bbox(x, y, z, n, pl->ws, s);
    if (e == cudaSuccess) e = launch_tree(n, x, y, z, q, D, pl->ws, s);
    if (e == cudaSuccess)
        e = launch_fmm(n, D, pl->phases, pl->ws, is_tc(pl->precision), E, phi, s);
    for (int k = 0; k < 4; ++k) pl->ws.kev[k] = nullptr;
    pl->last_depth = D;
    pl->last_n = n;
    return status_from(e);
}

// One time step: drift + cube, tree, FMM, kick + drift.  With profiling on,
// event records between the phases are captured too.
cudaError_t enqueue_step(fmm_plan_s* pl, const pt_state& st, const PushParams& pp,
                         const pt_laser& laser, int D, cudaStream_t s) {
    Workspace& ws = pl->ws;
    const int64_t n = st.n;
    for (int k = 0; k < 4; ++k) ws.kev[k] = pl->profile ? pl->k_ev[k] : nullptr;
    auto mark = [&](int k) -> cudaError_t {
        return pl->profile ? record_timing(pl->ph_ev[k], s)
                           : cudaSuccess;
    };
    cudaError_t e = mark(0);
    if (e == cudaSuccess) e = launch_drift_bbox(n, st.x, st.y, st.z, st.vx, st.vy, st.vz, pp, ws, s);
    if (e == cudaSuccess) e = mark(1);
    if (e == cudaSuccess) e = launch_tree(n, st.x, st.y, st.z, st.q, D, ws, s);
    if (e == cudaSuccess) e = mark(2);
    if (e == cudaSuccess)
        e = launch_fmm_phased(n, D, PT_PHASE_ALL, ws, is_tc(pl->precision), ws.E,
                              nullptr, s, pl->profile ? pl->ph_ev + 3 : nullptr);
    if (e == cudaSuccess)
        e = launch_kick_drift(n, st.x, st.y, st.z, st.vx, st.vy, st.vz, st.q, ws.E, pp, laser, ws, s);
    if (e == cudaSuccess) e = mark(6);
    for (int k = 0; k < 4; ++k) ws.kev[k] = nullptr;
    return e;
}

PushParams make_push(const pt_trap* trap, double dt, double damping) {
    PushParams pp;
    memset(&pp, 0, sizeof pp);
    pp.h = 0.5 * dt;
    pp.dt = dt;
    pp.wc = trap->charge * trap->B / trap->mass;
    pp.C = cos(pp.wc * pp.h);
    pp.S = sin(pp.wc * pp.h);
    pp.kz = trap->mass * trap->omega_z * trap->omega_z / trap->charge;
    pp.delta = trap->delta;
    pp.mass = trap->mass;
    pp.rk = 1.054571817e-34 / trap->mass;
    pp.damp = damping > 0.0 ? exp(-damping * dt) : 1.0;
    pp.wr = trap->omega_r;
    return pp;
}

// Before a chunk of k steps starting at step step0 + s0: the octree depth
// and, through the next pinned slot, the chunk's wall phases
// cos/sin(2 w_r t_mid) and the device step counter (queued on s).
int prepare_chunk(fmm_plan_s* plan, const pt_state* st, const pt_trap* trap, double dt, double t0,
                  int64_t step0, int64_t s0, int64_t k, bool sync, cudaStream_t s, int* D) {
    Workspace& ws = plan->ws;
    if (sync || plan->depth >= 0) {
        int r = choose_depth(plan, st->n, st->x, st->y, st->z, s, D);
        if (r != PT_OK) return r;
    } else {
        if (plan->last_depth < 0) return PT_ERR_ARG;
        *D = plan->last_depth;
    }
    int rp = ensure_pairs(plan, st->n, st->x, st->y, st->z, st->q, *D, s);
    if (rp != PT_OK) return rp;
    const int64_t first = step0 + s0;  // global index of the chunk's first step
    const bool in_window = plan->win_count > 0 && plan->win_t == t0 && plan->win_step == step0 &&
                           plan->win_dt == dt && plan->win_wr == trap->omega_r &&
                           first >= plan->win_base && first + k <= plan->win_base + plan->win_count;
    if (in_window && plan->dev_next == first) return PT_OK;  // table and counter in place
    const int slot = plan->next_slot;
    plan->next_slot = (slot + 1) % fmm_plan_s::kSlots;
    cudaError_t e = cudaEventSynchronize(plan->slot_ev[slot]);  // slot free again
    if (e != cudaSuccess) return status_from(e);
    plan->dev_next = -1;
    if (!in_window) {
        // a new window of wall_cap steps from this chunk's first (the table
        // depends on the anchor and the step index only)
        double* hw = plan->h_wall[slot];
        for (int64_t j = 0; j < ws.wall_cap; ++j) {
            double tm = (t0 + (double)(s0 + j) * dt) + 0.5 * dt;
            hw[2 * j] = cos(2.0 * trap->omega_r * tm);
            hw[2 * j + 1] = sin(2.0 * trap->omega_r * tm);
        }
        e = cudaMemcpyAsync(ws.wall_cs, hw, sizeof(double) * 2 * ws.wall_cap,
                            cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return status_from(e);
        plan->win_t = t0;
        plan->win_step = step0;
        plan->win_dt = dt;
        plan->win_wr = trap->omega_r;
        plan->win_base = first;
        plan->win_count = ws.wall_cap;
    }
    *plan->h_steps[slot] = StepCounter{0, first, plan->win_base};
    e = cudaMemcpyAsync(ws.steps, plan->h_steps[slot], sizeof(StepCounter), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(plan->slot_ev[slot], s);
    return status_from(e);
}

GraphKey make_key(const fmm_plan_s* plan, const pt_state* st, const PushParams& pp,
                  const pt_laser& lz, int D) {
    GraphKey key;
    key.D = D;
    key.n = st->n;
    const void* ptrs[7] = {st->x, st->y, st->z, st->vx, st->vy, st->vz, st->q};
    memcpy(key.ptr, ptrs, sizeof ptrs);
    key.pp = pp;
    key.laser = lz;
    key.profile = plan->profile;
    key.expand = plan->ws.expand;
    key.sched = plan->ws.m2l_pairs + 2 * plan->ws.m2l_rot + 4 * plan->ws.pp_mirror;
    key.ctas = plan->ws.m2l_ctas;
    key.pool = plan->ws.pp_gen;
    return key;
}

// A call that continues exactly where the plan's last call left the state
// (same step, same t, same dt) keeps the plan's time anchor; any other call
// starts a new one at (state->t, state->step).  Step times then come from the
// global step index alone, so a trajectory is bit for bit the same however
// its steps are split into calls (the serving loop splits them at arbitrary
// points).
void anchor_time(fmm_plan_s* pl, double t0, int64_t step0, double dt) {
    if (!(pl->end_step == step0 && pl->end_t == t0 && pl->anc_dt == dt)) {
        pl->anc_t = t0;
        pl->anc_step = step0;
        pl->anc_dt = dt;
    }
}

double anchored_end(fmm_plan_s* pl, int64_t step_end) {
    pl->end_step = step_end;
    pl->end_t = pl->anc_t + (double)(step_end - pl->anc_step) * pl->anc_dt;
    return pl->end_t;
}

// The step loop shared by pt_step (synchronous) and pt_step_async.
int step_impl(fmm_plan_s* plan, pt_state* st, const pt_trap* trap, const pt_laser* laser,
              double dt, int64_t n_steps, cudaStream_t s, bool sync) {
    Workspace& ws = plan->ws;
    pt_laser lz;
    memset(&lz, 0, sizeof lz);
    if (laser) lz = *laser;
    const PushParams pp = make_push(trap, dt, plan->damping);
    const int64_t step0 = st->step;
    anchor_time(plan, st->t, step0, dt);
    const int64_t off = step0 - plan->anc_step;
    for (int64_t s0 = 0; s0 < n_steps; s0 += ws.wall_cap) {
        const int64_t k = (n_steps - s0) < ws.wall_cap ? (n_steps - s0) : ws.wall_cap;
        int D;
        int r = prepare_chunk(plan, st, trap, dt, plan->anc_t, plan->anc_step, off + s0, k, sync, s,
                              &D);
        if (r != PT_OK) return r;
        cudaError_t e;
        const GraphKey key = make_key(plan, st, pp, lz, D);
        if (!plan->graph || !(key == plan->gkey)) {
            if (plan->graph) {
                cudaGraphExecDestroy(plan->graph);
                plan->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return status_from(e);
            cudaError_t e2 = enqueue_step(plan, *st, pp, lz, D, plan->cap_stream);
            e = cudaStreamEndCapture(plan->cap_stream, &g);
            if (e2 != cudaSuccess || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return status_from(e2 != cudaSuccess ? e2 : e);
            }
            e = cudaGraphInstantiate(&plan->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                plan->graph = nullptr;
                return status_from(e);
            }
            plan->gkey = key;
        }
        for (int64_t j = 0; j < k; ++j) {
            e = cudaGraphLaunch(plan->graph, s);
            if (e != cudaSuccess) {
                plan->dev_next = -1;
                return status_from(e);
            }
        }
        // each launch advances the device's step counter by one
        plan->dev_next = plan->anc_step + off + s0 + k;
        plan->last_depth = D;
        plan->last_n = st->n;
        if (sync) {
            r = check_err(plan, s);
            if (r != PT_OK) return r;
        }
    }
    st->t = anchored_end(plan, step0 + n_steps);
    st->step = step0 + n_steps;
    return PT_OK;
}

}  // namespace

// Independent crystals stepped together: one CUDA graph holds every member's
// time step as a parallel branch, so one graph launch advances the whole
// ensemble by one step and the members' kernels share the GPU.  The members'
// BF16 pair-packed M2L launches are joined into one launch over all their
// work items (m2l_join_pair_launches), unless switched off.
struct pt_ensemble_s {
    int device = 0;
    std::vector<fmm_plan_s*> plans;      // not owned
    std::vector<cudaStream_t> br;        // capture-time branch streams
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::vector<GraphKey> keys;
    bool join_m2l = true;
    int joined = 0;                      // members in the joined M2L launch
    void* d_members = nullptr;           // joined launch: member records
    int* d_prefix = nullptr;             // and their first items
};

namespace {
void free_ensemble(pt_ensemble_s* e) {
    if (!e) return;
    cudaSetDevice(e->device);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    for (cudaStream_t b : e->br)
        if (b) cudaStreamDestroy(b);
    for (cudaEvent_t j : e->join)
        if (j) cudaEventDestroy(j);
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->d_members) cudaFree(e->d_members);
    if (e->d_prefix) cudaFree(e->d_prefix);
    delete e;
}
}  // namespace

extern "C" {

const char* pt_status_str(int status) {
    switch (status) {
        case PT_OK: return "ok";
        case PT_ERR_ARG: return "invalid argument";
        case PT_ERR_OOM: return "device out of memory";
        case PT_ERR_CUDA: return "CUDA runtime error";
        case PT_ERR_NONFINITE: return "non-finite ion position";
        case PT_ERR_ESCAPED: return "ion escaped the domain";
        case PT_ERR_TIMEOUT: return "bounded device wait timed out";
        case PT_ERR_COINCIDENT: return "coincident ions";
        case PT_ERR_UNSUPPORTED: return "unsupported on this device or build";
        default: return "unknown status";
    }
}

static int plan_create_impl(int64_t n_max, int p, int leaf_max, int depth, int precision,
                            fmm_plan* out, bool dry, int64_t* dry_bytes, int64_t* op_bytes);

int fmm_plan_create(int64_t n_max, int p, int leaf_max, int depth, int precision, fmm_plan* out) {
    return plan_create_impl(n_max, p, leaf_max, depth, precision, out, false, nullptr, nullptr);
}

int fmm_plan_set_m2l_schedule(fmm_plan plan, int schedule) {
    if (!plan || (schedule != PT_M2L_TILES && schedule != PT_M2L_PAIRS &&
                  schedule != PT_M2L_ROTATION))
        return PT_ERR_ARG;
    if (schedule == PT_M2L_ROTATION && (is_tc(plan->precision) || !plan->ws.T_rot))
        return PT_ERR_UNSUPPORTED;
    if (cudaSetDevice(plan->device) != cudaSuccess) return PT_ERR_CUDA;
    int r = schedule != PT_M2L_TILES ? alloc_pairs(plan)
            : is_tc(plan->precision) ? alloc_tile_slabs(plan) : PT_OK;
    if (r != PT_OK) return r;
    plan->ws.m2l_pairs = schedule != PT_M2L_TILES ? 1 : 0;
    plan->ws.m2l_rot = schedule == PT_M2L_ROTATION ? 1 : 0;
    return PT_OK;
}

int fmm_plan_set_m2l_ctas(fmm_plan plan, int ctas) {
    if (!plan || ctas < 0) return PT_ERR_ARG;
    plan->ws.m2l_ctas = ctas;
    return PT_OK;
}

int fmm_plan_set_m2l_mirror(fmm_plan plan, int on) {
    if (!plan || (on != 0 && on != 1)) return PT_ERR_ARG;
    if (on && !plan->ws.tc_bf16) return PT_ERR_UNSUPPORTED;
    plan->ws.pp_mirror = on;
    return PT_OK;
}

int fmm_plan_m2l_schedule(fmm_plan plan) {
    if (!plan) return -1;
    if (plan->ws.m2l_rot) return PT_M2L_ROTATION;
    return plan->ws.m2l_pairs ? PT_M2L_PAIRS : PT_M2L_TILES;
}

int fmm_plan_footprint(int64_t n_max, int p, int leaf_max, int depth, int precision,
                       int64_t* plan_bytes, int64_t* operator_bytes) {
    if (!plan_bytes || !operator_bytes) return PT_ERR_ARG;
    fmm_plan dummy = nullptr;
    return plan_create_impl(n_max, p, leaf_max, depth, precision, &dummy, true, plan_bytes,
                            operator_bytes);
}

static int plan_create_impl(int64_t n_max, int p, int leaf_max, int depth, int precision,
                            fmm_plan* out, bool dry, int64_t* dry_bytes, int64_t* op_bytes) {
    if (!out || n_max < 1 || n_max > (int64_t)1 << 30 || p < 2 || p > kMaxOrder || leaf_max < 1 ||
        depth < -1 || depth > kMaxDepth)
        return PT_ERR_ARG;
    if (precision != PT_FP64 && precision != PT_FP32 && !is_tc(precision)) return PT_ERR_ARG;
    *out = nullptr;
    fmm_plan_s* pl = new (std::nothrow) fmm_plan_s;
    if (!pl) return PT_ERR_OOM;
    pl->dry = dry;
    if (dry) {
        if (is_tc(precision) && m2l_tc_operand_bytes(p, precision == PT_MIXED_BF16X3) == 0) {
            delete pl;
            return PT_ERR_UNSUPPORTED;
        }
    } else if (cudaGetDevice(&pl->device) != cudaSuccess) {
        delete pl;
        return PT_ERR_CUDA;
    }
    if (!dry && is_tc(precision)) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, pl->device) != cudaSuccess) {
            delete pl;
            return PT_ERR_CUDA;
        }
        if (prop.major != 10 || prop.minor != 3 ||
            m2l_tc_operand_bytes(p, precision == PT_MIXED_BF16X3) == 0) {
            delete pl;
            return PT_ERR_UNSUPPORTED;
        }
    }
    pl->n_max = n_max;
    pl->p = p;
    pl->P = (p + 1) * (p + 1);
    pl->leaf_max = leaf_max;
    pl->depth = depth;
    pl->precision = precision;
    Workspace& ws = pl->ws;
    ws.n_max = n_max;
    ws.p = p;
    ws.P = pl->P;
    ws.fp64 = (precision == PT_FP64);
    ws.tc_bf16 = (precision == PT_MIXED_BF16X3) ? 1 : 0;
    ws.pp_mirror = ws.tc_bf16;  // offset mirroring: the BF16x3 pair products only
    ws.ld = ws.fp64 ? pl->P : ((pl->P + 31) / 32) * 32;
    ws.rot_op_vals = rot_operator_bytes(pl) > 0 ? ops::rot_op_vals(p) : 0;
    if (depth >= 0) {
        ws.depth_max = depth;
    } else {
        int d = 1;
        while (d < kMaxDepth && pow8(d - 1) < n_max) ++d;
        ws.depth_max = d;
    }
    int64_t cells = 0, dense = 0;
    for (int l = 0; l <= ws.depth_max; ++l) {
        cells += pow8(l) < n_max ? pow8(l) : n_max;
        dense += pow8(l);
    }
    ws.cells_max = cells;
    ws.dense_max = dense;
    ws.block_sums_cap = (dense + kScanTile - 1) / kScanTile + 16;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            sms > 0)
            ws.sms = sms;
    }
    ws.bbox_blocks = ws.sms * 4;
    ws.wall_cap = kWallChunk;
    const size_t tsz = ws.fp64 ? sizeof(double) : sizeof(float);
    const size_t PP = (size_t)pl->P * pl->P;
    bool ok = true;
    if (!dry) {
        // per-device tables and kernel attributes: a failure here is a CUDA
        // error, not a lack of memory
        std::lock_guard<std::mutex> g(g_tables_mu);
        if (!g_tables_dev.count(pl->device)) {
            if (upload_harmonic_tables() != cudaSuccess || m2l_tc_init() != cudaSuccess ||
                m2l_rot_init() != cudaSuccess) {
                free_plan(pl);
                return PT_ERR_CUDA;
            }
            g_tables_dev.insert(pl->device);
        }
    }
    ok = ok && dalloc(pl, ws.key, sizeof(uint32_t) * n_max) && dalloc(pl, ws.rank, sizeof(uint32_t) * n_max) &&
         dalloc(pl, ws.perm_tmp, sizeof(int32_t) * n_max) && dalloc(pl, ws.perm, sizeof(int32_t) * n_max) &&
         dalloc(pl, ws.slot_of, sizeof(int32_t) * n_max) && dalloc(pl, ws.leaf_of, sizeof(int32_t) * n_max) &&
         dalloc(pl, ws.sorted, (ws.fp64 ? sizeof(double4_32a) : sizeof(float4)) * n_max) &&
         dalloc(pl, ws.leaf_count, sizeof(int32_t) * pow8(ws.depth_max)) &&
         dalloc(pl, ws.leaf_start, sizeof(int32_t) * (pow8(ws.depth_max) + 1)) &&
         dalloc(pl, ws.cid, sizeof(int32_t) * dense) && dalloc(pl, ws.code, sizeof(uint32_t) * cells) &&
         dalloc(pl, ws.cstart, sizeof(int32_t) * cells) && dalloc(pl, ws.ccount, sizeof(int32_t) * cells) &&
         dalloc(pl, ws.linfo, sizeof(LevelInfo)) && dalloc(pl, ws.M, tsz * ws.ld * cells) &&
         dalloc(pl, ws.L, tsz * ws.ld * cells) && dalloc(pl, ws.E, sizeof(double) * 3 * n_max) &&
         dalloc(pl, ws.near, tsz * 4 * n_max) &&
         dalloc(pl, ws.block_sums, sizeof(int32_t) * ws.block_sums_cap) &&
         dalloc(pl, ws.root, sizeof(RootCube)) &&
         dalloc(pl, ws.bbox_acc, sizeof(unsigned long long) * 8) &&
         dalloc(pl, ws.ticket, sizeof(unsigned)) && dalloc(pl, ws.err, sizeof(int)) &&
         dalloc(pl, ws.steps, sizeof(StepCounter)) && dalloc(pl, ws.stats, sizeof(unsigned long long) * 8) &&
         dalloc(pl, ws.wall_cs, sizeof(double) * 2 * ws.wall_cap);
    // the leaf histogram starts at zero; every scan of it zeroes what it read
    if (ok && !dry)
        ok = cudaMemset(ws.leaf_count, 0, sizeof(int32_t) * pow8(ws.depth_max)) == cudaSuccess;
    if (ok && is_tc(precision)) {
        ws.tc_splits_max = (int)m2l_tc_partial_splits(p, cells, ws.ld);
        int64_t tcap = 0;
        for (int l = 2; l <= ws.depth_max; ++l) tcap += ((pow8(l) < n_max ? pow8(l) : n_max) + 127) / 128 + 8;
        ws.tc_tiles_cap = tcap > 0 ? tcap : 1;
        // the pair-packed schedule by default up to kPairsDefaultIons; the
        // tile schedule's partial slabs then only at their minimum until it
        // is selected
        const bool pairs = n_max <= kPairsDefaultIons;
        ws.tc_slab_cap = pairs ? 1 : m2l_tc_slab_cap(ws.ld, ws.tc_tiles_cap, n_max);
        ws.tc_part_floats = m2l_tc_part_floats(cells, ws.ld, ws.tc_splits_max, ws.tc_tiles_cap,
                                               ws.tc_slab_cap);
        ok = dalloc(pl, ws.tc_work, m2l_tc_work_bytes(ws.tc_tiles_cap, ws.tc_slab_cap));
        ok = ok && dalloc(pl, ws.tc_part, sizeof(float) * ws.tc_part_floats);
        if (ws.tc_bf16) ok = ok && dalloc(pl, ws.M_pieces, sizeof(uint16_t) * kPieceRows * ws.ld * cells);
        if (ok && pairs) {
            ok = alloc_pairs(pl) == PT_OK;
            ws.m2l_pairs = ok ? 1 : 0;
        }
    } else if (ok && n_max <= kPairsDefaultIonsCudaCore) {
        // CUDA-core precisions: the pair work list by default as well, with
        // the rotation-based M2L for FP64 (a quarter of the dense
        // translation's FP64 operations at p = 12)
        ok = alloc_pairs(pl) == PT_OK;
        ws.m2l_pairs = ok ? 1 : 0;
        ws.m2l_rot = ok && ws.fp64 && ws.rot_op_vals > 0 ? 1 : 0;
    }
    if (dry) {
        *dry_bytes = (int64_t)pl->dry_bytes;
        *op_bytes = (int64_t)(tsz * (8 + 8 + 343) * PP +
                              (is_tc(precision) ? m2l_tc_operand_bytes(p, ws.tc_bf16 != 0) : 0) +
                              rot_operator_bytes(pl));
        delete pl;
        return PT_OK;
    }
    if (!ok) {
        free_plan(pl);
        return PT_ERR_OOM;
    }
    if ((ws.tc_work &&
         cudaMemset(ws.tc_work, 0, m2l_tc_work_bytes(ws.tc_tiles_cap, ws.tc_slab_cap)) != cudaSuccess) ||
        (ws.tc_part && cudaMemset(ws.tc_part, 0, sizeof(float) * ws.tc_part_floats) != cudaSuccess) ||
        cudaMemset(ws.M, 0, tsz * ws.ld * cells) != cudaSuccess ||
        (ws.M_pieces &&
         cudaMemset(ws.M_pieces, 0, sizeof(uint16_t) * kPieceRows * ws.ld * cells) != cudaSuccess) ||
        cudaMemset(ws.L, 0, tsz * ws.ld * cells) != cudaSuccess ||
        cudaMemset(ws.ticket, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(ws.bbox_acc, 0, sizeof(unsigned long long) * 8) != cudaSuccess ||
        cudaMemset(ws.err, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(ws.steps, 0, sizeof(StepCounter)) != cudaSuccess ||
        cudaMallocHost(&pl->h_err, sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithPriority(&pl->cap_stream, cudaStreamNonBlocking, prio_high()) != cudaSuccess ||
        cudaStreamCreateWithPriority(&ws.side, cudaStreamNonBlocking, prio_low()) != cudaSuccess ||
        cudaStreamCreateWithPriority(&ws.side2, cudaStreamNonBlocking, prio_low()) != cudaSuccess ||
        cudaEventCreateWithFlags(&ws.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ws.ev_p2m, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ws.ev_items, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ws.ev_near, cudaEventDisableTiming) != cudaSuccess) {
        free_plan(pl);
        return PT_ERR_CUDA;
    }
    for (int k = 0; k < fmm_plan_s::kSlots; ++k) {
        if (cudaMallocHost(&pl->h_wall[k], sizeof(double) * 2 * ws.wall_cap) != cudaSuccess ||
            cudaMallocHost(&pl->h_steps[k], sizeof(StepCounter)) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->slot_ev[k], cudaEventDisableTiming) != cudaSuccess) {
            free_plan(pl);
            return PT_ERR_CUDA;
        }
    }
    for (int k = 0; k <= fmm_plan_s::kPhases; ++k) {
        if (cudaEventCreate(&pl->ph_ev[k]) != cudaSuccess) {
            free_plan(pl);
            return PT_ERR_CUDA;
        }
    }
    for (cudaEvent_t& ev : pl->k_ev) {
        if (cudaEventCreate(&ev) != cudaSuccess) {
            free_plan(pl);
            return PT_ERR_CUDA;
        }
    }
    int r = acquire_ops(pl, tsz * PP);
    if (r != PT_OK) {
        free_plan(pl);
        return r;
    }
    *out = pl;
    return PT_OK;
}

int fmm_plan_destroy(fmm_plan plan) {
    free_plan(plan);
    return PT_OK;
}

int fmm_plan_set_expansion(fmm_plan plan, int mode) {
    if (!plan || (mode != PT_EXPAND_TREE && mode != PT_EXPAND_DIRECT)) return PT_ERR_ARG;
    plan->ws.expand = mode;
    return PT_OK;
}

int fmm_plan_set_phases(fmm_plan plan, int phases) {
    if (!plan || phases < 1 || phases > 3) return PT_ERR_ARG;
    plan->phases = phases;
    return PT_OK;
}

int fmm_plan_last_depth(fmm_plan plan) { return plan ? plan->last_depth : -1; }

int fmm_forces(fmm_plan plan, int64_t n, const double* pos, const double* q, double* E,
               double* phi, void* stream) {
    if (!plan || !pos || !q || !E || n < 1 || n > plan->n_max) return PT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaSetDevice(plan->device) != cudaSuccess) return PT_ERR_CUDA;
    const double *x = pos, *y = pos + n, *z = pos + 2 * n;
    int D;
    int r = choose_depth(plan, n, x, y, z, s, &D);
    if (r != PT_OK) return r;
    return forces_impl(plan, n, x, y, z, q, E, phi, s, D);
}

int fmm_direct(int64_t n, const double* pos, const double* q, double* E, double* phi,
               void* stream) {
    if (!pos || !q || !E || n < 1) return PT_ERR_ARG;
    return status_from(launch_direct(n, pos, q, E, phi, (cudaStream_t)stream));
}

int pt_laser_kicks(const pt_laser* laser, double mass, int64_t n, const double* x, const double* y,
                   const double* z, const double* vx, const double* vy, const double* vz,
                   int64_t step, double dt, int32_t* counts, double* dv, void* stream) {
    if (!laser || !x || !y || !z || !vx || !vy || !vz || !dv || n < 1 || !(mass > 0) ||
        laser->n_beams < 0 || laser->n_beams > PT_MAX_BEAMS)
        return PT_ERR_ARG;
    const double rk = 1.054571817e-34 / mass;
    return status_from(launch_laser_kicks(*laser, rk, n, x, y, z, vx, vy, vz, step, dt, counts, dv,
                                          (cudaStream_t)stream));
}

static int step_args_ok(fmm_plan plan, const pt_state* st, const pt_trap* trap,
                        const pt_laser* laser, double dt, int64_t n_steps) {
    if (!plan || !st || !trap || !(dt > 0) || n_steps < 0 || st->n < 1 || st->n > plan->n_max ||
        !st->x || !st->y || !st->z || !st->vx || !st->vy || !st->vz || !st->q || !(trap->mass > 0) ||
        trap->charge == 0.0 || trap->B == 0.0)
        return PT_ERR_ARG;
    if (laser && (laser->n_beams < 0 || laser->n_beams > PT_MAX_BEAMS)) return PT_ERR_ARG;
    return PT_OK;
}

int pt_step(fmm_plan plan, pt_state* st, const pt_trap* trap, const pt_laser* laser, double dt,
            int64_t n_steps, void* stream) {
    int r = step_args_ok(plan, st, trap, laser, dt, n_steps);
    if (r != PT_OK) return r;
    if (n_steps == 0) return PT_OK;
    if (cudaSetDevice(plan->device) != cudaSuccess) return PT_ERR_CUDA;
    return step_impl(plan, st, trap, laser, dt, n_steps, (cudaStream_t)stream, true);
}

int pt_step_async(fmm_plan plan, pt_state* st, const pt_trap* trap, const pt_laser* laser,
                  double dt, int64_t n_steps, void* stream) {
    int r = step_args_ok(plan, st, trap, laser, dt, n_steps);
    if (r != PT_OK) return r;
    if (plan->depth < 0 && plan->last_depth < 0) return PT_ERR_ARG;
    if (n_steps == 0) return PT_OK;
    if (cudaSetDevice(plan->device) != cudaSuccess) return PT_ERR_CUDA;
    return step_impl(plan, st, trap, laser, dt, n_steps, (cudaStream_t)stream, false);
}

int pt_sync(fmm_plan plan, void* stream) {
    if (!plan) return PT_ERR_ARG;
    return check_err(plan, (cudaStream_t)stream);
}

int fmm_plan_profile(fmm_plan plan, int enable) {
    if (!plan) return PT_ERR_ARG;
    plan->profile = enable != 0;
    return PT_OK;
}

int fmm_plan_kernel_times(fmm_plan plan, double* ms) {
    if (!plan || !ms || !plan->profile) return PT_ERR_ARG;
    for (int k = 0; k < 2; ++k) {
        float v = 0.f;
        cudaError_t e = cudaEventElapsedTime(&v, plan->k_ev[2 * k], plan->k_ev[2 * k + 1]);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();  // an unrecorded event: not a fault of later launches
            return status_from(e);
        }
        ms[k] = v;
    }
    return PT_OK;
}

int fmm_plan_phase_times(fmm_plan plan, double* ms) {
    if (!plan || !ms || !plan->profile) return PT_ERR_ARG;
    for (int k = 0; k < fmm_plan_s::kPhases; ++k) {
        float v = 0.f;
        cudaError_t e = cudaEventElapsedTime(&v, plan->ph_ev[k], plan->ph_ev[k + 1]);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();  // an unrecorded event: not a fault of later launches
            return status_from(e);
        }
        ms[k] = v;
    }
    return PT_OK;
}

int fmm_plan_stats(fmm_plan plan, int64_t* out, void* stream) {
    if (!plan || !out || plan->last_depth < 0) return PT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_tree_stats(plan->last_n, plan->last_depth, plan->ws, out, s);
    return status_from(e);
}

int fmm_plan_tc_stats(fmm_plan plan, int64_t* out, void* stream) {
    if (!plan || !out || plan->last_depth < 0) return PT_ERR_ARG;
    if (!is_tc(plan->precision) || plan->last_depth < 2) {
        for (int k = 0; k < 4; ++k) out[k] = 0;
        return PT_OK;
    }
    return status_from(m2l_tc_work_stats(plan->ws, out, (cudaStream_t)stream));
}

int pt_energy(fmm_plan plan, const pt_state* st, const pt_trap* trap, double* out, void* stream) {
    if (!st || !trap || !out || st->n < 1 || !st->x || !st->y || !st->z || !st->vx || !st->vy ||
        !st->vz || !st->q || trap->charge == 0.0)
        return PT_ERR_ARG;
    if (plan && st->n > plan->n_max) return PT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = st->n;
    double *pos = nullptr, *E = nullptr, *phi = nullptr, *dout = nullptr;
    size_t bytes = sizeof(double) * (3 * n + 3 * n + n + 4 + 3 * 256);
    if (cudaMalloc(&pos, bytes) != cudaSuccess) return PT_ERR_OOM;
    E = pos + 3 * n;
    phi = E + 3 * n;
    dout = phi + n;
    cudaError_t e = cudaMemcpyAsync(pos, st->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pos + n, st->y, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pos + 2 * n, st->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    int r = PT_OK;
    if (e == cudaSuccess) {
        if (plan) r = fmm_forces(plan, n, pos, st->q, E, phi, s);
        else e = launch_direct(n, pos, st->q, E, phi, s);
    }
    const double kz = trap->mass * trap->omega_z * trap->omega_z / trap->charge;
    if (e == cudaSuccess && r == PT_OK) e = launch_energy_parts(n, *st, *trap, kz, phi, dout, s);
    double h[3] = {0, 0, 0};
    if (e == cudaSuccess && r == PT_OK) e = cudaMemcpyAsync(h, dout, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(pos);
    if (r != PT_OK) return r;
    if (e != cudaSuccess) return status_from(e);
    out[0] = h[0];
    out[1] = h[1];
    out[2] = h[2];
    out[3] = h[0] + h[1] + h[2];
    return PT_OK;
}

int fmm_tree_info(fmm_plan plan, double* root, int32_t* perm, uint32_t* keys, void* stream) {
    if (!plan || !root || plan->last_depth < 0) return PT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = plan->last_n;
    RootCube rc;
    cudaError_t e = cudaMemcpyAsync(&rc, plan->ws.root, sizeof rc, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && perm)
        e = cudaMemcpyAsync(perm, plan->ws.perm, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && keys)
        e = cudaMemcpyAsync(keys, plan->ws.key, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_from(e);
    root[0] = rc.lo[0];
    root[1] = rc.lo[1];
    root[2] = rc.lo[2];
    root[3] = rc.side;
    return PT_OK;
}

int pt_ensemble_create(int n_members, const fmm_plan* plans, pt_ensemble* out) {
    if (!out || !plans || n_members < 1) return PT_ERR_ARG;
    *out = nullptr;
    std::set<fmm_plan> seen;
    for (int b = 0; b < n_members; ++b) {
        if (!plans[b] || !seen.insert(plans[b]).second || plans[b]->device != plans[0]->device)
            return PT_ERR_ARG;
    }
    pt_ensemble_s* e = new (std::nothrow) pt_ensemble_s;
    if (!e) return PT_ERR_OOM;
    e->device = plans[0]->device;
    if (cudaSetDevice(e->device) != cudaSuccess) {
        delete e;
        return PT_ERR_CUDA;
    }
    e->plans.assign(plans, plans + n_members);
    e->br.assign(n_members, nullptr);
    e->join.assign(n_members, nullptr);
    bool ok = cudaStreamCreateWithPriority(&e->cap, cudaStreamNonBlocking, prio_high()) == cudaSuccess &&
              cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; ok && b < n_members; ++b)
        ok = cudaStreamCreateWithPriority(&e->br[b], cudaStreamNonBlocking, prio_high()) == cudaSuccess &&
             cudaEventCreateWithFlags(&e->join[b], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&e->d_members, m2l_join_member_bytes() * (size_t)n_members) == cudaSuccess &&
         cudaMalloc(&e->d_prefix, sizeof(int) * ((size_t)n_members + 1)) == cudaSuccess;
    if (!ok) {
        free_ensemble(e);
        return PT_ERR_CUDA;
    }
    *out = e;
    return PT_OK;
}

int pt_ensemble_destroy(pt_ensemble ens) {
    free_ensemble(ens);
    return PT_OK;
}

int pt_ensemble_step(pt_ensemble ens, pt_state* states, const pt_trap* traps,
                     const pt_laser* lasers, const double* dt, int64_t n_steps, void* stream) {
    if (!ens || !states || !traps || !dt || n_steps < 0) return PT_ERR_ARG;
    const int nm = (int)ens->plans.size();
    for (int b = 0; b < nm; ++b) {
        int r = step_args_ok(ens->plans[b], &states[b], &traps[b], lasers ? &lasers[b] : nullptr,
                             dt[b], n_steps);
        if (r != PT_OK) return r;
    }
    if (n_steps == 0) return PT_OK;
    if (cudaSetDevice(ens->device) != cudaSuccess) return PT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<PushParams> pp(nm);
    std::vector<pt_laser> lz(nm);
    std::vector<int64_t> step0(nm);
    for (int b = 0; b < nm; ++b) {
        pp[b] = make_push(&traps[b], dt[b], ens->plans[b]->damping);
        memset(&lz[b], 0, sizeof(pt_laser));
        if (lasers) lz[b] = lasers[b];
        step0[b] = states[b].step;
        anchor_time(ens->plans[b], states[b].t, step0[b], dt[b]);
    }
    std::vector<int> D(nm);
    std::vector<GraphKey> keys(nm);
    for (int64_t s0 = 0; s0 < n_steps; s0 += kWallChunk) {
        const int64_t k = (n_steps - s0) < kWallChunk ? (n_steps - s0) : kWallChunk;
        for (int b = 0; b < nm; ++b) {
            fmm_plan_s* pl = ens->plans[b];
            // an automatic-depth plan that never chose a depth chooses it now
            int r = prepare_chunk(pl, &states[b], &traps[b], dt[b], pl->anc_t, pl->anc_step,
                                  (step0[b] - pl->anc_step) + s0, k,
                                  pl->depth < 0 && pl->last_depth < 0, s, &D[b]);
            if (r != PT_OK) return r;
            keys[b] = make_key(pl, &states[b], pp[b], lz[b], D[b]);
        }
        bool same = ens->graph != nullptr && ens->keys.size() == keys.size();
        for (int b = 0; same && b < nm; ++b) same = keys[b] == ens->keys[b];
        cudaError_t e;
        if (!same) {
            if (ens->graph) {
                cudaGraphExecDestroy(ens->graph);
                ens->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(ens->cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return status_from(e);
            cudaError_t e2 = cudaEventRecord(ens->fork, ens->cap);
            for (int b = 0; e2 == cudaSuccess && b < nm; ++b) {
                e2 = cudaStreamWaitEvent(ens->br[b], ens->fork, 0);
                if (e2 == cudaSuccess)
                    e2 = enqueue_step(ens->plans[b], states[b], pp[b], lz[b], D[b], ens->br[b]);
                if (e2 == cudaSuccess) e2 = cudaEventRecord(ens->join[b], ens->br[b]);
                if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(ens->cap, ens->join[b], 0);
            }
            e = cudaStreamEndCapture(ens->cap, &g);
            if (e2 != cudaSuccess || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return status_from(e2 != cudaSuccess ? e2 : e);
            }
            ens->joined = 0;
            if (ens->join_m2l &&
                (e = m2l_join_pair_launches(g, ens->d_members, ens->d_prefix, nm, &ens->joined)) !=
                    cudaSuccess) {
                cudaGraphDestroy(g);
                return status_from(e);
            }
            e = cudaGraphInstantiate(&ens->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                ens->graph = nullptr;
                return status_from(e);
            }
            ens->keys = keys;
        }
        for (int64_t j = 0; j < k; ++j) {
            e = cudaGraphLaunch(ens->graph, s);
            if (e != cudaSuccess) {
                for (int b = 0; b < nm; ++b) ens->plans[b]->dev_next = -1;
                return status_from(e);
            }
        }
        for (int b = 0; b < nm; ++b) {
            fmm_plan_s* pl = ens->plans[b];
            pl->dev_next = step0[b] + s0 + k;
            ens->plans[b]->last_depth = D[b];
            ens->plans[b]->last_n = states[b].n;
        }
    }
    for (int b = 0; b < nm; ++b) {
        states[b].t = anchored_end(ens->plans[b], step0[b] + n_steps);
        states[b].step = step0[b] + n_steps;
    }
    return PT_OK;
}

int pt_ensemble_set_joined_m2l(pt_ensemble ens, int on) {
    if (!ens) return PT_ERR_ARG;
    if (ens->join_m2l != (on != 0)) {
        ens->join_m2l = on != 0;
        ens->keys.clear();  // re-capture at the next step
    }
    return PT_OK;
}

int pt_ensemble_joined_m2l(pt_ensemble ens, int* members) {
    if (!ens || !members) return PT_ERR_ARG;
    *members = ens->joined;
    return PT_OK;
}

int pt_ensemble_sync(pt_ensemble ens, void* stream) {
    if (!ens) return PT_ERR_ARG;
    if (cudaSetDevice(ens->device) != cudaSuccess) return PT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PT_ERR_CUDA;
    int first = PT_OK;
    for (fmm_plan_s* pl : ens->plans) {
        int r = check_err(pl, s);
        if (r != PT_OK && first == PT_OK) first = r;
    }
    return first;
}

int pt_set_damping(fmm_plan plan, double gamma) {
    if (!plan || !(gamma >= 0.0)) return PT_ERR_ARG;
    plan->damping = gamma;
    return PT_OK;
}

namespace {
// scratch of the temperature reduction: {T_par, T_perp} and per-block partials
static __device__ __align__(256) double g_diag_scratch[2 + 2 * 256];
std::mutex g_diag_mu;
}  // namespace

int pt_temperatures(const pt_state* st, const pt_trap* trap, double* out, void* stream) {
    if (!st || !trap || !out || st->n < 1 || !st->x || !st->y || !st->vx || !st->vy || !st->vz ||
        !(trap->mass > 0))
        return PT_ERR_ARG;
    std::lock_guard<std::mutex> g(g_diag_mu);
    double* d = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&d, g_diag_scratch);
    cudaStream_t s = (cudaStream_t)stream;
    if (e == cudaSuccess) e = launch_temperatures(st->n, *st, *trap, d, s);
    double h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_from(e);
    out[0] = h[0];
    out[1] = h[1];
    return PT_OK;
}

int pt_mh_scans(const pt_state* st, const pt_trap* trap, double temperature, double dx,
                uint64_t seed, int64_t scan0, int64_t n_scans, int64_t* accepted, double* de_sum,
                void* stream) {
    if (!st || !trap || st->n < 1 || !st->x || !st->y || !st->z || !st->q || !(trap->mass > 0) ||
        trap->charge == 0.0 || !(temperature > 0) || !(dx >= 0) || n_scans < 0 || scan0 < 0)
        return PT_ERR_ARG;
    MhParams mp;
    mp.c = cos(trap->omega_r * st->t);
    mp.s = sin(trap->omega_r * st->t);
    mp.kz = trap->mass * trap->omega_z * trap->omega_z / trap->charge;
    mp.B = trap->B;
    mp.wr = trap->omega_r;
    mp.m = trap->mass;
    mp.delta = trap->delta;
    mp.ke = 1.0 / (4.0 * 3.14159265358979323846 * 8.8541878128e-12);
    mp.kb = 1.380649e-23;
    mp.temp = temperature;
    mp.dx = dx;
    mp.seed = seed;
    std::lock_guard<std::mutex> g(g_diag_mu);
    double* d = nullptr;
    double* scratch = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&d, g_diag_scratch);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t sb = mh_scratch_bytes(st->n);
    if (e == cudaSuccess && sb > 0 && cudaMalloc((void**)&scratch, sb) != cudaSuccess)
        return PT_ERR_OOM;
    if (e == cudaSuccess)
        e = launch_mh_scans(st->n, st->x, st->y, st->z, st->q, mp, scan0, n_scans,
                            (unsigned long long*)d, d + 1, scratch, s);
    double h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (scratch) cudaFree(scratch);
    if (e != cudaSuccess) return status_from(e);
    unsigned long long a;
    memcpy(&a, &h[0], sizeof a);
    if (accepted) *accepted = (int64_t)a;
    if (de_sum) *de_sum = h[1];
    return PT_OK;
}

int pt_position_moments(const pt_state* st, const pt_trap* trap, double* acc, void* stream) {
    if (!st || !trap || !acc || st->n < 1 || !st->x || !st->y || !st->z) return PT_ERR_ARG;
    return status_from(launch_position_moments(st->n, *st, *trap, acc, (cudaStream_t)stream));
}

int pt_rms_displacement(int64_t n, const double* acc, int64_t samples, double* out,
                        void* stream) {
    if (n < 1 || !acc || !out || samples < 1) return PT_ERR_ARG;
    return status_from(launch_rms_displacement(n, acc, samples, out, (cudaStream_t)stream));
}

int pt_potential_temperature(fmm_plan plan, const pt_state* st, const pt_state* ref,
                             const pt_trap* trap, double* out, void* stream) {
    if (!st || !ref || !out || st->n < 1 || ref->n != st->n) return PT_ERR_ARG;
    double e[4], e0[4];
    int r = pt_energy(plan, st, trap, e, stream);
    if (r != PT_OK) return r;
    if ((r = pt_energy(plan, ref, trap, e0, stream)) != PT_OK) return r;
    const double kb = 1.380649e-23;
    *out = (2.0 / 3.0) * ((e[1] + e[2]) - (e0[1] + e0[2])) / ((double)st->n * kb);
    return PT_OK;
}

}  // extern "C"
