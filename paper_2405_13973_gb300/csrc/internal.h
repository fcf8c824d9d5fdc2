// internal.h -- declarations shared by the CUDA translation units of
// libpenning (host launchers and the plan workspace).  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/penning.h"

namespace pt {

// A timing event on s: an external event node while s is being captured
// into a graph (so that the event is recorded when the graph runs), a plain
// record otherwise (the external flag is refused outside a capture).
inline cudaError_t record_timing(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, s);
}

// Programmatic dependent launch: a kernel launched by launch_pdl may be
// scheduled while its predecessor in the stream finishes (its blocks become
// resident, its set-up runs); it calls pdl_wait() before it touches memory
// that earlier work writes or reads, which returns once the predecessor has
// completed and its writes are visible.  In a kernel launched normally,
// pdl_wait() returns at once.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Blocks of a per-ion FP64 pass (FP64 is scarce on this GPU: a few results
// per SM per cycle): a multiple of the SM count where the ions allow, each
// block an equal contiguous share [blockIdx.x * per, min(n, (blockIdx.x + 1) *
// per)) of about `cap` ions at most (at least about 16), so that every SM's
// FP64 pipes get the same work; max_blocks bounds the grid (then per > cap).
struct IonSplit {
    int grid;
    int64_t per;
};
inline IonSplit ion_split(int64_t n, int cap, int sms, int64_t max_blocks) {
    const int64_t w = (int64_t)sms * cap;
    int64_t g = (int64_t)sms * ((n + w - 1) / w);
    const int64_t gmin = (n + 15) / 16;
    if (g > gmin) g = gmin;
    if (g > max_blocks) g = max_blocks;
    if (g < 1) g = 1;
    IonSplit r;
    r.grid = (int)g;
    r.per = (n + g - 1) / g;
    if (r.per < 1) r.per = 1;
    return r;
}

constexpr int kMaxDepth = 8;      // uniform octree depth limit (8^8 leaf cells)
constexpr int kMaxOrder = 16;     // expansion order limit
constexpr int kScanTile = 2048;   // elements per block in the device scans
// 1/(4 pi eps0) with the CODATA 2018 eps0, evaluated as (1 / ((4 pi) eps0))
constexpr double kCoulomb = 1.0 / (4.0 * 3.14159265358979323846 * 8.8541878128e-12);

// Root cube of the octree (Sec. 2.3.2): lower corner and side length.
struct RootCube {
    double lo[3];
    double side;
};

// Per-level bookkeeping written on the device by the compaction pass.
//   gbase[l]        first global compact id of level l (gbase[D+1] = total)
//   oct_start[l][o] first global id of the cells of level l whose Morton code
//                   ends in octant o (cells are grouped octant-major)
struct LevelInfo {
    int32_t gbase[kMaxDepth + 2];
    int32_t oct_start[kMaxDepth + 1][9];
};

// Step counter shared by the kernels of one time step (advanced on the
// device so that a captured step graph can be replayed).
struct StepCounter {
    int64_t cur;    // index of the step being computed
    int64_t next;   // index the next step will take
    int64_t base;   // first step of the current chunk (indexes the wall table)
};

// Device workspace owned by a plan.
struct Workspace {
    int64_t n_max = 0;
    int depth_max = 0;
    int p = 0, P = 0;
    int ld = 0;                 // row stride of M and L (P for FP64, P rounded up to 32 for FP32)
    bool fp64 = true;
    int64_t cells_max = 0;      // capacity of the compact cell arrays
    int sms = 152;              // multiprocessors of the plan's device
    int64_t dense_max = 0;      // capacity of the concatenated dense maps

    uint32_t* key = nullptr;       // [n] leaf key of every ion (original order)
    uint32_t* rank = nullptr;      // [n] arrival rank inside its leaf
    int32_t* perm_tmp = nullptr;   // [n] slot -> ion, unordered inside a leaf
    int32_t* perm = nullptr;       // [n] slot -> ion, ordered by ion index
    int32_t* slot_of = nullptr;    // [n] ion -> slot
    int32_t* leaf_of = nullptr;    // [n] slot -> global compact id of its leaf
    void* sorted = nullptr;        // [n] float4 / double4 (u_x, u_y, u_z, q)
    int32_t* leaf_count = nullptr; // [8^Dmax] ions per leaf code
    int32_t* leaf_start = nullptr; // [8^Dmax + 1] exclusive scan of leaf_count
    int32_t* cid = nullptr;        // [dense_max] dense (level, code) -> global id or -1
    uint32_t* code = nullptr;      // [cells_max] global id -> Morton code
    int32_t* cstart = nullptr;     // [cells_max] first slot of a leaf
    int32_t* ccount = nullptr;     // [cells_max] ions in a leaf
    LevelInfo* linfo = nullptr;    // level bookkeeping (device)
    void* M = nullptr;             // [cells_max][ld] multipole coefficients (padding zero)
    void* L = nullptr;             // [cells_max][ld] local coefficients
    double* E = nullptr;           // [3n] Coulomb field of the last evaluation (SoA, SI)
    void* near = nullptr;          // [n][4] P2P field and potential per sorted slot (leaf units)
    // side stream (lowest priority) of the M2L work list and the near field,
    // which overlap the main chain; events of the fork and the joins
    // (ev_p2m: when the near field may start)
    cudaStream_t side = nullptr;
    cudaStream_t side2 = nullptr;  // the near field of the tensor-core paths
    cudaEvent_t ev_fork = nullptr, ev_p2m = nullptr, ev_items = nullptr, ev_near = nullptr;
    int32_t* block_sums = nullptr; // scan scratch
    int64_t block_sums_cap = 0;
    RootCube* root = nullptr;
    unsigned long long* bbox_acc = nullptr;  // bounding-box accumulator, 8 words, kept zero between passes
    int bbox_blocks = 0;
    unsigned* ticket = nullptr;      // last-block-done counter
    int* err = nullptr;              // device error flags (bit mask)
    StepCounter* steps = nullptr;
    unsigned long long* stats = nullptr;  // [8] interaction counters
    double* wall_cs = nullptr;       // [wall_cap][2] cos, sin of 2 w_r t_mid per step
    int64_t wall_cap = 0;
    // operators (device), P x P each, row-major out x in
    void* T_m2m = nullptr;   // [8][P][P]
    void* T_l2l = nullptr;   // [8][P][P]
    void* T_m2l = nullptr;   // [343][P][P], index (ox+3)*49+(oy+3)*7+(oz+3)
    void* T_m2l_tc = nullptr;   // tensor-core operand tiles (mixed modes)
    uint16_t* M_pieces = nullptr;  // BF16x3: M split into bf16 hi/mid/lo and the same of
                                   // the mirrored M, [cell][kPieceRows = 6][ld]
    int tc_bf16 = 0;            // tensor-core operand format: 0 TF32 hi/lo, 1 BF16 hi/mid/lo
    float* tc_part = nullptr;   // M2M split partials, then M2L item slabs (tc_part_floats)
    size_t tc_part_floats = 0;
    int tc_splits_max = 1;      // M2M CTAs per tile
    int64_t tc_slab_cap = 1;    // M2L items of rank > 0 (partial slabs)
    void* tc_work = nullptr;    // M2L work list (tiles, items)
    int64_t tc_tiles_cap = 0;
    int expand = 0;             // PT_EXPAND_*: ancestor expansions of the tensor-core paths
    // pair-packed M2L schedule (PT_M2L_PAIRS, m2l_pairs.h): work list and the
    // partial rows of every (target, source) pair, [slot][pp_stride] in the
    // path's type (FP32: P rounded up to 16 on the tensor cores, ld on the
    // CUDA cores; FP64: ld)
    int m2l_pairs = 0;
    // rotation-based M2L of the CUDA-core paths (PT_M2L_ROTATION, with the
    // pair work list): per offset index [R^M | R^L | Z_re | Z_im], rot_op_vals
    // values of the path's type
    int m2l_rot = 0;
    // CTAs of the persistent tensor-core M2L kernel (0: one per SM); members
    // of an ensemble may take fewer so that their M2L kernels share the SMs
    int m2l_ctas = 0;
    // BF16x3 pair schedule: the pairs of offsets o and -o share the runs of
    // o (the pairs of -o read the mirrored multipole pieces and their partial
    // rows carry negated odd-degree terms, undone by the per-target sums):
    // half the operators, and fewer runs padded to 128 rows
    int pp_mirror = 0;
    void* T_rot = nullptr;
    int rot_op_vals = 0;
    // kernel timing (profiled steps only, else null): recorded right before
    // and after the M2L kernel(s) [0, 1] and the near-field kernel [2, 3]
    cudaEvent_t kev[4] = {nullptr, nullptr, nullptr, nullptr};
    void* pp_work = nullptr;
    void* pp_part = nullptr;
    void* h_pp_hdr = nullptr;       // pinned copy of the last work list's header (pairs, overflow),
                                    // written by k_pp_scan through the unified address space
    int pp_gen = 0;                 // bumped whenever the pool is reallocated
    int pp_stride = 0;
    int64_t pp_slot_cap = 0;    // pairs the pool holds
    int64_t pp_rows_cap = 0;    // partial rows: pairs, each offset's run padded to 128 rows
    int64_t pp_item_cap = 0;    // work items (runs of up to 128 pairs of one offset)
    // TMA descriptor of the partial rows for the tensor-core epilogue
    // (a CUtensorMap: rows x (P rounded up to 16) FP32, boxes of 128 rows x 16)
    alignas(64) unsigned char pp_map[128] = {0};
    int pp_map_ok = 0;
};

enum ErrBits { ERR_NONFINITE = 1, ERR_TIMEOUT = 2, ERR_CAPACITY = 4 };

// Offsets of the concatenated dense maps: levels lmin..D.
struct DenseLayout {
    int lmin = 0, D = 0;
    int64_t off[kMaxDepth + 2] = {0};
    int64_t total = 0;
};
DenseLayout dense_layout(int D);

// ---- tree (tree.cu) ----------------------------------------------------------
cudaError_t launch_bbox(const double* x, const double* y, const double* z, int64_t n,
                        Workspace& ws, cudaStream_t s);
cudaError_t launch_tree(int64_t n, const double* x, const double* y, const double* z,
                        const double* q, int D, Workspace& ws, cudaStream_t s);
cudaError_t launch_level_counts(int64_t n, const double* x, const double* y, const double* z,
                                int D, Workspace& ws, int32_t* host_counts, cudaStream_t s);

// ---- FMM stages (fmm.cu) -----------------------------------------------------
cudaError_t upload_harmonic_tables();
cudaError_t launch_fmm(int64_t n, int D, int phases, Workspace& ws, bool use_tc, double* E,
                       double* phi, cudaStream_t s);
// As launch_fmm; if ev is not null, records ev[0] after the upward pass,
// ev[1] after M2L/L2L and ev[2] after L2P/P2P.
cudaError_t launch_fmm_phased(int64_t n, int D, int phases, Workspace& ws, bool use_tc, double* E,
                              double* phi, cudaStream_t s, cudaEvent_t* ev);
// Interaction counts of the last tree (synchronises s).  out[8] = {n, D,
// leaves, cells at levels >= 2, M2L pairs, P2P pairs (ordered, i != j),
// L2L shifts, M2M shifts}.
cudaError_t launch_tree_stats(int64_t n, int D, Workspace& ws, int64_t* out, cudaStream_t s);
cudaError_t launch_direct(int64_t n, const double* pos, const double* q, double* E, double* phi,
                          cudaStream_t s);

// ---- tensor-core M2L (m2l_tc.cu) ---------------------------------------------
// The M2L work list of the current tree (reads the tree only), then the M2L
// of every level on the tensor cores with the slab reduction and the L2L
// shifts level by level (L is complete once the second has run).
cudaError_t launch_m2l_tc_worklist(int64_t n, int D, Workspace& ws, cudaStream_t s);
// L2L into levels 3 .. l2l_last; BF16x3: M of levels 3 .. split_last split
// into bf16 pieces first (the other levels' producers store theirs);
// after_m2l (optional) is recorded on s right after the M2L kernel.
cudaError_t launch_m2l_tc_run(int64_t n, int D, Workspace& ws, int l2l_last, int split_last,
                              cudaStream_t s, cudaEvent_t after_m2l = nullptr);
cudaError_t m2l_tc_init();
size_t m2l_tc_operand_bytes(int p, bool bf16);   // 0 if the order is not supported
size_t m2l_tc_partial_splits(int p, int64_t cells_max, int ld);
size_t m2l_tc_work_bytes(int64_t tiles_cap, int64_t slab_cap);
// ---- pair-packed M2L schedule (m2l_pairs.cu) -----------------------------------
// work-list and partial-row bytes for the workspace's cells_max, pp_slot_cap,
// pp_item_cap and pp_stride
size_t m2l_pp_work_bytes(const Workspace& ws);
size_t m2l_pp_part_bytes(const Workspace& ws);
// the work list of the current tree (reads the tree only)
cudaError_t launch_m2l_pairs_worklist(int64_t n, int D, Workspace& ws, cudaStream_t s);
// L of every cell of levels 2..D = the sum of its pairs' partial rows
// (`width` columns)
cudaError_t launch_m2l_pairs_reduce(int64_t n, int D, Workspace& ws, int width, cudaStream_t s);
// CUDA-core paths: the M2L products of the work list, the reduction and the
// L2L shifts into levels 3 .. l2l_last
cudaError_t launch_m2l_pairs_simt(int64_t n, int D, Workspace& ws, int l2l_last, cudaStream_t s);
// {offsets with pairs, work items, work items, pairs} of the last work list
cudaError_t m2l_pairs_stats(const Workspace& ws, int64_t* out, cudaStream_t s);
// rotation-based M2L: pairs per shared-memory tile (0: the operators of
// this order do not fit), per-device kernel set-up
int m2l_rot_tile(const Workspace& ws);
cudaError_t m2l_rot_init();
// the tensor-core partial-row width (P rounded up to 16)
int m2l_tc_npad(int p);
// (re)builds ws.pp_map for the current pp_part / pp_rows_cap (BF16 tensor-core
// plans; others leave it unused)
cudaError_t m2l_tc_make_part_map(Workspace& ws);
// ensembles: replaces the BF16 pair-packed M2L launches of a captured graph
// by one launch over all of them (d_members: room for cap member records of
// m2l_join_member_bytes() each; d_prefix: cap + 1 ints); *joined = members
// joined (0 when fewer than two were found)
size_t m2l_join_member_bytes();
cudaError_t m2l_join_pair_launches(cudaGraph_t g, void* d_members, int* d_prefix, int cap,
                                   int* joined);
cudaError_t m2l_tc_work_stats(const Workspace& ws, int64_t* out, cudaStream_t s);
// partial slabs of the M2L work items (a pool of 16 KB per ion, 16 MB to 8 GB)
int64_t m2l_tc_slab_cap(int ld, int64_t tiles_cap, int64_t n_max);
size_t m2l_tc_part_floats(int64_t cells_max, int ld, int m2m_splits, int64_t tiles_cap,
                          int64_t slab_cap);
void m2l_tc_pack_operands(int p, bool bf16, const double* T_m2l, const double* T_m2m,
                          const double* T_l2l, void* out);
// M2M of one level (targets = parents at level l) on the tensor cores.
cudaError_t launch_m2m_tc(int64_t n, int D, int l, Workspace& ws, cudaStream_t s);
// M2M (mode 0, targets at level l) or L2L (mode 1, into level l) of a small
// level on the CUDA cores, for the FP32 plans of the tensor-core paths: up to
// kShiftSmallM2M parents / kShiftSmallL2L children (capacity bounds).
constexpr int64_t kShiftSmallM2M = 64;
constexpr int64_t kShiftSmallL2L = 512;
inline int64_t level_cap(int64_t n, int l) {
    const int64_t c = (int64_t)1 << (3 * l);
    return n < c ? n : c;
}
cudaError_t launch_shift_small(int mode, int64_t n, int D, int l, Workspace& ws, cudaStream_t s);
void host_m2l_offsets(int16_t out[8][189]);

// ---- push (push.cu) ----------------------------------------------------------
struct PushParams {
    double h;          // dt/2
    double dt;
    double C, S, wc;   // cos(wc h), sin(wc h), q B / m
    double kz;         // m w_z^2 / q
    double delta;
    double mass;
    double t0;         // time of the chunk's first step
    int64_t step0;     // its global index
    double rk;         // hbar / m
    double damp;       // exp(-gamma dt) of the rotating-frame velocity; 1 = no damping
    double wr;         // rotation frequency of the damping's rigid rotor
};
// ---- Metropolis-Hastings initialisation (mh.cu) --------------------------------
struct MhParams {
    double c, s;            // wall phase cos, sin(w_r t)
    double kz, B, wr, m, delta;
    double ke, kb;          // Coulomb and Boltzmann constants (J m / C^2, J / K)
    double temp, dx;        // temperature (K), largest displacement (m)
    uint64_t seed;
};
// scratch: mh_scratch_bytes(n) of device memory (none needed for large n)
size_t mh_scratch_bytes(int64_t n);
cudaError_t launch_mh_scans(int64_t n, double* x, double* y, double* z, const double* q,
                            const MhParams& mp, int64_t scan0, int64_t n_scans,
                            unsigned long long* acc_out, double* de_out, double* scratch,
                            cudaStream_t s);

cudaError_t launch_drift_bbox(int64_t n, double* x, double* y, double* z, double* vx, double* vy,
                              double* vz, const PushParams& pp, Workspace& ws, cudaStream_t s);
cudaError_t launch_kick_drift(int64_t n, double* x, double* y, double* z, double* vx, double* vy,
                              double* vz, const double* q, const double* E, const PushParams& pp,
                              const pt_laser& laser, Workspace& ws, cudaStream_t s);
cudaError_t launch_laser_kicks(const pt_laser& laser, double rk, int64_t n, const double* x,
                               const double* y, const double* z, const double* vx,
                               const double* vy, const double* vz, int64_t step, double dt,
                               int32_t* counts, double* dv, cudaStream_t s);
cudaError_t launch_energy_parts(int64_t n, const pt_state& st, const pt_trap& trap, double kz,
                                const double* phi, double* d_out, cudaStream_t s);
// {T_par, T_perp} into d_out[0..1]; d_out holds 2 + 2 * 256 doubles
cudaError_t launch_temperatures(int64_t n, const pt_state& st, const pt_trap& trap, double* d_out,
                                cudaStream_t s);
// acc[0..n) += x_r, [n, 2n) += y_r, [2n, 3n) += z, [3n, 4n) += |x_r|^2 at time st.t
cudaError_t launch_position_moments(int64_t n, const pt_state& st, const pt_trap& trap,
                                    double* acc, cudaStream_t s);
// out[i] = Delta r_rms of ion i from `samples` accumulations of acc (above)
cudaError_t launch_rms_displacement(int64_t n, const double* acc, int64_t samples, double* out,
                                    cudaStream_t s);

}  // namespace pt
