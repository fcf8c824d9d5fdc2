/*
 * penning.h -- C ABI of libpenning: the FMM Coulomb field of a 3D Penning-trap
 * ion crystal fused with the cyclotronic push, for NVIDIA GB300 (sm_103a).
 *
 * Method: Zaris, Johnson, Shankar, Bollinger & Parker, "Numerical Simulations
 * of 3D Ion Crystal Dynamics in a Penning Trap using the Fast Multipole
 * Method" (arXiv:2405.13973).
 *
 * Conventions shared by every call:
 *   - SI units.  Positions in m, velocities in m/s, charges in C, fields in
 *     V/m, potentials in V, times in s, angular frequencies in rad/s.
 *   - Arrays of 3-vectors are structure-of-arrays: x[0..n), y[0..n), z[0..n)
 *     stored back to back in one buffer of 3n doubles ("SoA 3n").
 *   - Pointers documented "device" must be CUDA device (or managed) memory
 *     of the current device; "host" pointers are ordinary host memory.  The
 *     caller owns every buffer it passes; the library never frees them and
 *     keeps no reference after the call returns (except a plan's captured
 *     launch graph, which is rebuilt when the pointers change).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *     enqueue their work on it and return; results are valid once the stream
 *     is synchronised.  Calls that must read device results on the host
 *     (automatic depth selection, error flags, energies) synchronise the
 *     stream themselves, as documented per call.
 *   - Every call returns a pt_status.  No call aborts the process or throws.
 *     A device-side error (non-finite positions) is latched in the plan and
 *     returned by the next synchronising call on that plan.
 *   - Plans are not thread-safe: one host thread at a time per plan.
 */
#ifndef PENNING_H
#define PENNING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
    PT_OK = 0,
    PT_ERR_ARG = -1,         /* bad argument (null pointer, size, range) */
    PT_ERR_OOM = -2,         /* device allocation failed */
    PT_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    PT_ERR_NONFINITE = -4,   /* a position was NaN or infinite */
    PT_ERR_ESCAPED = -5,     /* reserved: ion outside the plan's domain */
    PT_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
    PT_ERR_COINCIDENT = -7,  /* reserved: two ions at the same point */
    PT_ERR_UNSUPPORTED = -8  /* the library or the device lacks the feature */
} pt_status;

/* Arithmetic of the FMM (positions, velocities and the push are FP64 in
 * every mode).
 *   PT_FP64          : every FMM stage in FP64 on the CUDA cores.
 *   PT_MIXED_TF32X3  : P2M/L2P/P2P in FP32 on the CUDA cores; M2M, M2L and
 *                      L2L on the tensor cores (tcgen05, operands split into
 *                      TF32 hi + lo, three products, FP32 accumulation in
 *                      tensor memory: products good to about 2^-21).
 *   PT_MIXED_BF16X3  : as PT_MIXED_TF32X3 with operands split into three
 *                      BF16 pieces and six products (products good to about
 *                      2^-24, the accuracy of FP32 multiplies) in the same
 *                      tensor time.
 *   PT_FP32          : every FMM stage in FP32 on the CUDA cores. */
typedef enum {
    PT_FP64 = 0,
    PT_MIXED_TF32X3 = 1,
    PT_MIXED_BF16X3 = 2,
    PT_FP32 = 3
} pt_precision;

/* FMM stages run by fmm_forces (bit mask); default PT_PHASE_ALL. */
enum { PT_PHASE_NEAR = 1, PT_PHASE_FAR = 2, PT_PHASE_ALL = 3 };

typedef struct fmm_plan_s* fmm_plan;

/* ---------------------------------------------------------------------------
 * fmm_plan_create -- allocate a plan and its device workspace.
 * Paper: Sec. 2.3.2 (the octree, upward and downward passes) and Eq.
 * multipole_error (the order p of the expansions).
 *   n_max     : largest ion count the plan will see (>= 1).
 *   p         : expansion order, 2 <= p <= 16; (p+1)^2 real coefficients per
 *               cell (Eq. FMM_coul truncated at n = p).
 *   leaf_max  : target mean ion count per non-empty leaf; used when depth = 0.
 *   depth     : octree depth D (0 <= D <= 8) or -1 for automatic: the
 *               smallest D whose mean non-empty-leaf occupancy is <= leaf_max,
 *               chosen from the positions at each fmm_forces call and at the
 *               start of each pt_step call (this synchronises the stream).
 *   precision : a pt_precision value.
 *   out       : receives the plan (host pointer to an fmm_plan).
 * Uses the current CUDA device.  Errors: PT_ERR_ARG, PT_ERR_OOM, PT_ERR_CUDA,
 * PT_ERR_UNSUPPORTED (tensor-core mode on a device that is not sm_103). */
int fmm_plan_create(int64_t n_max, int p, int leaf_max, int depth, int precision, fmm_plan* out);

/* Free a plan and its workspace (NULL is accepted).  Synchronises the device. */
int fmm_plan_destroy(fmm_plan plan);

/* Restrict the stages of fmm_forces to PT_PHASE_NEAR (direct sum over
 * adjacent leaves, Sec. 2.3.2), PT_PHASE_FAR (multipole/local expansions) or
 * both (default).  For testing each stage against its definition. */
int fmm_plan_set_phases(fmm_plan plan, int phases);

/* How the tensor-core precisions obtain the expansions of the cells above
 * the leaves (Sec. 2.3.1):
 *   PT_EXPAND_TREE   (default) the passes: P2M at the leaves and at their
 *                    parents, M2M shifts up from there, M2L, L2L shifts
 *                    down, L2P at the leaves;
 *   PT_EXPAND_DIRECT P2M of every ion about each of its ancestor cells and
 *                    L2P of each ancestor's own M2L sum at the ion -- equal
 *                    to the passes up to rounding, since M2M and L2L shift
 *                    truncated expansions exactly.  It costs D - 1
 *                    expansions per ion and serves as a cross-check of the
 *                    shifts (slower than the passes on the 10k-ion crystal).
 * The CUDA-core precisions always use the passes.  Errors: PT_ERR_ARG. */
#define PT_EXPAND_TREE 0
#define PT_EXPAND_DIRECT 1
int fmm_plan_set_expansion(fmm_plan plan, int mode);

/* How M2L is scheduled (Eq. FMM_local; Sec. 2.3.2's interaction list of 189
 * source cells per target, at most 316 distinct offsets o = target - source
 * per level).  The translation operator depends on the offset only
 * (expansions are stored scaled by the cell size), so:
 *   PT_M2L_TILES     tensor cores: tiles of 128 target cells of one level
 *                    and child octant, per non-empty offset one dense
 *                    product of all 128 rows (rows whose source is empty
 *                    multiply zeros), summed in tensor memory over runs of
 *                    up to four offsets; CUDA cores: per level, tiles of 32
 *                    targets of one octant looping over their 189 offsets
 *                    (and the L2L shift);
 *   PT_M2L_PAIRS     the (target, source) pairs of each offset, gathered
 *                    over all levels, fill products of 128 pairs (tensor
 *                    cores) or 64 x 64 SIMT tiles (CUDA cores); each pair's
 *                    result row is a partial local expansion, and each
 *                    target's partials are summed in increasing offset order
 *                    (deterministic).  Fewer, fuller products on small or flat
 *                    crystals, at the price of a pool of partial rows (P
 *                    rounded up to 16 values on the tensor cores, the row
 *                    stride of M and L on the CUDA cores, per pair).  The
 *                    pool starts at 12 n_max + 4096 pairs (or the exact bound
 *                    189 x the cells of levels 2..depth, if smaller); a
 *                    plan's first call counts the pairs of its tree, and a
 *                    call grows the pool by half again once the last step
 *                    used more than 80 % of it (synchronising the device).  A
 *                    step whose pairs exceed the pool returns PT_ERR_OOM (its
 *                    far field is missing) and the next call grows the pool;
 *   PT_M2L_ROTATION  CUDA-core precisions, p <= 16: the pair work list, each
 *                    translation done by rotating the multipole so that the
 *                    offset points along +z, translating along z (orders m
 *                    do not mix) and rotating back (the point-and-shoot
 *                    factorisation of the dense operator, exact up to
 *                    rounding): O(p^3) instead of (p+1)^4 multiply-adds per
 *                    translation (7.3k instead of 28.6k at p = 12).
 * Default: PT_M2L_PAIRS for the tensor-core precisions up to n_max = 65536;
 * PT_M2L_ROTATION for FP64 and PT_M2L_PAIRS for FP32 up to n_max = 262144;
 * PT_M2L_TILES above.  Selecting another schedule allocates what it needs.
 * Errors: PT_ERR_ARG, PT_ERR_UNSUPPORTED (rotation on the tensor-core
 * precisions or beyond p = 16), PT_ERR_OOM, PT_ERR_CUDA. */
#define PT_M2L_TILES 0
#define PT_M2L_PAIRS 1
#define PT_M2L_ROTATION 2
int fmm_plan_set_m2l_schedule(fmm_plan plan, int schedule);
/* CTAs of the plan's persistent tensor-core M2L kernel: 0 (default) one per
 * SM, else at most `ctas`, so that the M2L kernels of several plans stepped
 * together (an ensemble) can run side by side.  Results do not depend on it:
 * every work item is computed by one CTA whatever the grid.  Errors:
 * PT_ERR_ARG. */
int fmm_plan_set_m2l_ctas(fmm_plan plan, int ctas);
/* Offset mirroring of the BF16x3 pair schedule: 1 (default) or 0.  The M2L
 * operator of Eq. FMM_local obeys T_{-o}[l][j] = (-1)^(j + l) T_o[l][j]
 * (Sec. 2.3.1: the irregular solid harmonic of degree n is even or odd in
 * its argument as n is), so with mirroring on the pairs of offset -o are
 * products with the operator of o: their multipole enters with its
 * odd-degree coefficients negated and their partial local expansion leaves
 * with its odd-degree coefficients negated.  Both negations are exact, so
 * the forces equal those with mirroring off; half the operators are read
 * and fewer 128-row products are padded.  Takes effect at the next call.
 * Errors: PT_ERR_ARG (on not 0 or 1), PT_ERR_UNSUPPORTED (on, on a plan of
 * another precision). */
int fmm_plan_set_m2l_mirror(fmm_plan plan, int on);
/* The plan's M2L schedule (PT_M2L_*), or -1 for a NULL plan. */
int fmm_plan_m2l_schedule(fmm_plan plan);

/* Depth used by the last fmm_forces / pt_step call on this plan (or -1). */
int fmm_plan_last_depth(fmm_plan plan);

/* ---------------------------------------------------------------------------
 * fmm_forces -- Coulomb field (and potential) on every ion by the FMM.
 * Paper: Eq. hamiltonian (the pair sum it approximates: the force on ion i
 * is q_i E_i with E_i = k_e sum_{j!=i} q_j (x_i - x_j)/|x_i - x_j|^3),
 * Sec. 2.3.1-2.3.2 (ME, LE, upward and downward passes).
 *   n    : number of ions, 1 <= n <= n_max.
 *   pos  : device, SoA 3n doubles (m).
 *   q    : device, n doubles (C).
 *   E    : device, SoA 3n doubles, written (V/m).  Coulomb part only.
 *   phi  : device, n doubles (V) or NULL.
 * Asynchronous unless depth is automatic.  Errors: PT_ERR_ARG, PT_ERR_CUDA,
 * PT_ERR_NONFINITE (latched from an earlier call). */
int fmm_forces(fmm_plan plan, int64_t n, const double* pos, const double* q, double* E,
               double* phi, void* stream);

/* ---------------------------------------------------------------------------
 * fmm_direct -- the same field by the O(N^2) pair sum in FP64 on the GPU.
 * Paper: Eq. hamiltonian; the "direct" mode of Sec. 3.  Reference for error
 * measurement at sizes the CPU cannot reach.  Arguments as fmm_forces.
 * Asynchronous.  Errors: PT_ERR_ARG, PT_ERR_CUDA. */
int fmm_direct(int64_t n, const double* pos, const double* q, double* E, double* phi,
               void* stream);

/* ---------------------------------------------------------------------------
 * Trap, beams, laser, state (SI).  Paper: Eqs. pot_trap, pot_wall (k_z =
 * m omega_z^2 / q), B along +z (omega_c = q B / m), Eq. scattering_rate. */
typedef struct {
    double B;        /* axial magnetic field (T), along +z */
    double omega_z;  /* axial trap frequency (rad/s) */
    double omega_r;  /* rotating-wall frequency (rad/s) */
    double delta;    /* rotating-wall strength (dimensionless) */
    double mass;     /* ion mass (kg), the same for every ion */
    double charge;   /* reference charge (C) defining k_z = m omega_z^2 / q */
} pt_trap;

typedef struct {
    double s0;        /* peak saturation parameter S_0 */
    double detuning;  /* Delta_l (rad/s) */
    double kx, ky, kz;/* wave vector k_l (1/m) */
    double waist_y;   /* w_y (m), non-uniform beams */
    double waist_z;   /* w_z (m), non-uniform beams */
    double offset_d;  /* beam centre y = d (m), non-uniform beams */
    int32_t uniform;  /* 1: S = S0 everywhere; 0: S0 exp(-(y-d)^2/w_y^2 - z^2/w_z^2) */
    int32_t pad_;
} pt_beam;

#define PT_MAX_BEAMS 8
typedef struct {
    int32_t n_beams;  /* 0..PT_MAX_BEAMS */
    int32_t enabled;  /* 0: no photon kicks */
    uint64_t seed;    /* Philox4x32-10 key */
    double gamma0;    /* natural linewidth (rad/s), 2 pi 18 MHz for Be+ */
    pt_beam beam[PT_MAX_BEAMS];
} pt_laser;

typedef struct {
    int64_t n;        /* ion count */
    double t;         /* time (s); advanced by pt_step */
    int64_t step;     /* global step index (keys the photon random numbers) */
    double* x;        /* device, n doubles each */
    double* y;
    double* z;
    double* vx;
    double* vy;
    double* vz;
    double* q;        /* device, n charges (C) */
} pt_state;

/* ---------------------------------------------------------------------------
 * pt_step -- advance the crystal by n_steps cyclotronic steps.
 * Paper: Eq. time_ev2, U = U0(dt/2) Ukick(t + dt/2; dt) U0(dt/2), with U0 the
 * exact gyration of Eq. U0 (read for B along +z: the velocity turns
 * clockwise), Ukick of Eq. velocity_kick (Coulomb by the FMM plus trap and
 * wall fields at t + dt/2) and the photon kicks of Eq. laser_kick with
 * Poisson counts of mean gamma_l(x, v) dt (Eq. scattering_rate) at the
 * midpoint state.  Photon random numbers: Philox4x32-10 with key = seed and
 * counter = (ion, beam | slot << 8, step lo, step hi); slot 0 draws the
 * Poisson uniform, slots 1.. the sphere points (Marsaglia 1972).
 *   state : host struct; its device arrays are updated in place and its
 *           t and step fields advanced on return.
 *   trap, laser : host structs (laser may be NULL = no cooling).
 *   dt    : time step (s) > 0.   n_steps >= 0.
 * Synchronises the stream before returning (status of the whole run).
 * Errors: PT_ERR_ARG, PT_ERR_CUDA, PT_ERR_NONFINITE. */
int pt_step(fmm_plan plan, pt_state* state, const pt_trap* trap, const pt_laser* laser,
            double dt, int64_t n_steps, void* stream);

/* ---------------------------------------------------------------------------
 * pt_step_async -- as pt_step but without synchronising: the steps are
 * enqueued on `stream` and the call returns (state->t, state->step are
 * advanced on return).  Needs a fixed octree depth: the plan's `depth`, or,
 * for an automatic plan, the depth chosen by its last synchronising call
 * (PT_ERR_ARG if there was none).  Device errors are latched and returned by
 * pt_sync or the next synchronising call.  Consecutive asynchronous calls on
 * one plan must use one stream.  Paper: Eq. time_ev2 as for pt_step. */
int pt_step_async(fmm_plan plan, pt_state* state, const pt_trap* trap, const pt_laser* laser,
                  double dt, int64_t n_steps, void* stream);

/* Synchronise `stream` and return the plan's latched device error, if any. */
int pt_sync(fmm_plan plan, void* stream);

/* ---------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper).
 * fmm_plan_profile: enable (1) or disable (0) CUDA-event timing of the phases
 *   of every time step (drift + root cube, tree, upward pass, M2L + L2L,
 *   L2P + P2P, kick + drift).  Takes effect at the next step.
 * fmm_plan_phase_times: device milliseconds of those six phases in the last
 *   executed step (host, 6 doubles).  The step must have completed.
 * fmm_plan_stats: interaction counts of the last octree (host, 8 int64):
 *   {n, depth, leaves, cells at levels >= 2, M2L translations (target,
 *   source) with a non-empty source, P2P pair interactions (ordered, i != j),
 *   L2L shifts, M2M shifts}.  Synchronises the stream. */
int fmm_plan_profile(fmm_plan plan, int enable);
int fmm_plan_phase_times(fmm_plan plan, double* ms);
/* fmm_plan_kernel_times: device milliseconds, in the last executed profiled
 *   step or force evaluation (fmm_forces), of the M2L kernel alone (host ms[0]: the tensor-core M2L launch,
 *   or the CUDA-core M2L launches of all levels) and of the near-field (P2P)
 *   kernel (ms[1]), each between events recorded right before and after the
 *   launch on its own stream.  Errors: PT_ERR_ARG (profiling off). */
int fmm_plan_kernel_times(fmm_plan plan, double* ms);
int fmm_plan_stats(fmm_plan plan, int64_t* out, void* stream);

/* fmm_plan_tc_stats: the tensor-core M2L work list of the last evaluation
 * (host, 4 int64): {tiles (up to 128 target cells of one level), tile-offset
 * products (each a dense 128-row translation by one operator, Eq. M2L),
 * work items (runs of products of one tile), target rows (cells at levels
 * >= 2)}.  All zero for the CUDA-core precisions and trees of depth < 2.
 * Synchronises the stream.  Errors: PT_ERR_ARG (no evaluation yet),
 * PT_ERR_CUDA. */
int fmm_plan_tc_stats(fmm_plan plan, int64_t* out, void* stream);

/* ---------------------------------------------------------------------------
 * pt_laser_kicks -- the photon counts and recoil velocity change of one step
 * for a given midpoint state, without applying them.  Paper: Eqs.
 * scattering_rate and laser_kick.  Bit-reproducible definition (see pt_step).
 *   x..vz : device, n doubles each (midpoint positions and velocities).
 *   counts: device, n * n_beams int32 (row-major by ion) or NULL.
 *   dv    : device, SoA 3n doubles (m/s), written.
 * Asynchronous.  Errors: PT_ERR_ARG, PT_ERR_CUDA. */
int pt_laser_kicks(const pt_laser* laser, double mass, int64_t n, const double* x,
                   const double* y, const double* z, const double* vx, const double* vy,
                   const double* vz, int64_t step, double dt, int32_t* counts, double* dv,
                   void* stream);

/* ---------------------------------------------------------------------------
 * pt_energy -- rotating-frame energy of the state at time state->t.
 * Paper: Eq. rotation (x_r = R(omega_r t) x), Eq. pe_rot (first line, from
 * Eqs. pot_trap and pot_wall) and Sec. 3 (energies in the rotating frame):
 *   out[0] kinetic  sum m |v_r|^2 / 2, v_r = (v_x - w_r y, v_y + w_r x, v_z)
 *   out[1] external sum q_i k_z (2z^2 - r^2)/4 + (q_i B w_r - m w_r^2) r^2/2
 *                       + q_i k_z delta (x_r^2 - y_r^2)/4
 *   out[2] Coulomb  (1/2) sum_i q_i phi_i
 *   out[3] total.
 *   plan   : the FMM for phi, or NULL to use the exact FP64 direct sum.
 *   out    : host, 4 doubles (J).
 * Synchronises the stream.  Errors: PT_ERR_ARG, PT_ERR_CUDA, PT_ERR_OOM. */
int pt_energy(fmm_plan plan, const pt_state* state, const pt_trap* trap, double* out,
              void* stream);

/* ---------------------------------------------------------------------------
 * pt_energy_noalloc -- pt_energy with the exact FP64 direct sum (as with a
 * NULL plan), for callers that cannot allocate device memory: real-time
 * loops that cannot afford cudaMalloc's implicit device synchronisation in
 * the middle of a run, and programs whose device memory is reserved up
 * front by their own allocator (a fixed pool that leaves nothing for a
 * library to take).  The paper has no counterpart; this is a service of the
 * library.
 *   state, trap, out, stream : as pt_energy.
 * Allocates nothing: its scratch is a fixed array inside the library
 * (3.5 MiB, held by every GPU that loads the library until exit), which
 * limits state->n to 65536 (larger: PT_ERR_ARG, nothing queued).  The first
 * call on a device looks the array's device address up once (the set-up);
 * make that first call before any stream capture on the device.  All calls
 * on a device share the array and it keeps the last call's contents: calls
 * that overlap on the GPU (other streams or threads) race and must be
 * serialised.  Each call overwrites all the scratch it reads, so nothing
 * needs clearing.  Copies the four results to `out` on the host and
 * synchronises the stream.  Errors: PT_ERR_ARG, PT_ERR_CUDA. */
int pt_energy_noalloc(const pt_state* state, const pt_trap* trap, double* out, void* stream);

/* Human-readable text for a status code (static storage). */
const char* pt_status_str(int status);

/* ---------------------------------------------------------------------------
 * fmm_tree_info -- the octree of the last fmm_forces / pt_step call, for
 * checking the sort (Sec. 2.3.2: root cube = smallest cube around the ions,
 * split into octants; leaf keys are Morton codes of the leaf coordinates,
 * ix the most significant bit of each triple).
 *   root  : host, 4 doubles written: lo_x, lo_y, lo_z, side (m).
 *   perm  : device, n int32 written: perm[k] = original index of the ion in
 *           sorted slot k (sorted by leaf key, ties by index) or NULL.
 *   keys  : device, n uint32 written: leaf key of every ion (original order)
 *           or NULL.
 * Synchronises the stream.  Errors: PT_ERR_ARG, PT_ERR_CUDA. */
int fmm_tree_info(fmm_plan plan, double* root, int32_t* perm, uint32_t* keys, void* stream);

/* ---------------------------------------------------------------------------
 * pt_mh_scans -- Metropolis-Hastings initialisation of the potential energy
 * (Sec. 4, the laser-cooling initialisation): n_scans scans; in each, ion i =
 * 0..n-1 in turn is displaced by a distance uniform in [0, dx) in a uniformly
 * random direction (Marsaglia's disc pick), and the move is kept if the
 * crystal's rotating-frame potential energy (Eq. pe_rot at the state's time
 * t, trap + rotating wall + Coulomb) falls, or else if u < exp(-dE /
 * (k_B temperature)); otherwise the ion goes back.  Random numbers: the
 * Philox stream of pt_laser_kicks with beam field 0xFF and the scan index
 * scan0 + s in place of the step (resume = pass the next scan0).
 *   st          : positions x, y, z updated in place (device); q read;
 *                 velocities untouched.
 *   temperature : K (> 0); dx: m (>= 0).
 *   accepted    : host, the number of accepted moves, or NULL.
 *   de_sum      : host, the sum of the accepted energy changes (J), or NULL.
 * FP64.  Up to 4096 ions: a cluster of 8 CTAs (the Coulomb change of each
 * move summed over the other ions by all of them), with a device scratch of
 * 40 B per ion allocated for the call; larger crystals: one 1024-thread
 * block.  Synchronises the stream; calls on one device are serialised (they
 * share a small device result buffer).
 * Errors: PT_ERR_ARG, PT_ERR_OOM, PT_ERR_CUDA. */
int pt_mh_scans(const pt_state* st, const pt_trap* trap, double temperature, double dx,
                uint64_t seed, int64_t scan0, int64_t n_scans, int64_t* accepted, double* de_sum,
                void* stream);

/* ---------------------------------------------------------------------------
 * Diagnostics of a run (Sec. 5, Eqs. temps and rms_disp) and artificial
 * damping toward equilibria (Sec. 6: the crystal evolves under the trap
 * equations of motion while the ions' motion is slowly removed).
 *
 * pt_set_damping -- from the plan's next step on, after every kick each
 *   ion's velocity relative to the rigid rotation at omega_r (the rotating-
 *   frame velocity (v_x - w_r y, v_y + w_r x, v_z) at the mid-step
 *   position) is scaled by exp(-gamma dt); gamma in 1/s, 0 (the default)
 *   turns damping off and leaves the step exactly as without this call.
 *   Errors: PT_ERR_ARG (NULL plan, gamma < 0 or NaN).
 * pt_temperatures -- out[0] = T_par = m sum v_z^2 / (N k_B) (Eq. temp_ax),
 *   out[1] = T_perp = m sum (w_x^2 + w_y^2) / (2 N k_B) (Eq. temp_pl), in K,
 *   of the velocities relative to the rigid rotation (instantaneous; the
 *   paper's angle brackets average these over time).  state: device
 *   pointers (x, y, vx, vy, vz read); out: host, 2 doubles.  Uses a fixed
 *   scratch array inside the library; calls are serialised by a host lock.
 *   Synchronises the stream.  Errors: PT_ERR_ARG, PT_ERR_CUDA.
 * pt_position_moments -- accumulates the rotating-frame moments of every
 *   ion at time state->t (x_r = R(w_r t) x as in Eq. rotation):
 *   acc[i] += x_r, acc[n+i] += y_r, acc[2n+i] += z, acc[3n+i] += |x_r|^2.
 *   acc: device, 4 n doubles owned and zeroed by the caller.  After K calls,
 *   Delta r_rms of ion i = sqrt(acc[3n+i]/K - |(acc[i], acc[n+i],
 *   acc[2n+i])/K|^2) (Eq. rms_disp).  Asynchronous.  Errors: PT_ERR_ARG,
 *   PT_ERR_CUDA. */
int pt_set_damping(fmm_plan plan, double gamma);
int pt_temperatures(const pt_state* state, const pt_trap* trap, double* out, void* stream);
int pt_position_moments(const pt_state* state, const pt_trap* trap, double* acc, void* stream);

/* ---------------------------------------------------------------------------
 * pt_rms_displacement -- Delta r_rms of every ion (Sec. 5, Eq. rms_disp: the
 * RMS displacement of an ion about its mean rotating-frame position over K
 * samples) from the moments pt_position_moments accumulated K times:
 *   out[i] = sqrt(max(0, acc[3n+i]/K - sum_a (acc[a n+i]/K)^2)).
 *   n       : ions.
 *   acc     : device, 4n doubles (layout of pt_position_moments), read only.
 *   samples : K >= 1.
 *   out     : device, n doubles written (m).
 * Asynchronous on the stream.  Errors: PT_ERR_ARG, PT_ERR_CUDA. */
int pt_rms_displacement(int64_t n, const double* acc, int64_t samples, double* out,
                        void* stream);

/* ---------------------------------------------------------------------------
 * pt_potential_temperature -- T_PE = (2/3)(PE - PE_0)/(N k_B) (Sec. 5, Eq.
 * temp_pe): PE the rotating-frame potential energy (external: trap, rotating
 * wall and rotation terms, plus Coulomb) of `state` and PE_0 that of the
 * reference configuration `ref` (the paper's is a minimised equilibrium),
 * each at its own time, both from pt_energy with `plan` (NULL: the exact
 * direct sum).
 *   out : host, 1 double written (K).
 * Synchronises the stream.  Errors: as pt_energy; PT_ERR_ARG if the ion
 * counts differ. */
int pt_potential_temperature(fmm_plan plan, const pt_state* state, const pt_state* ref,
                             const pt_trap* trap, double* out, void* stream);

/* ---------------------------------------------------------------------------
 * fmm_plan_footprint -- the device memory fmm_plan_create would allocate for
 * these arguments, without allocating anything (no GPU needed): for admission
 * control by memory budget.  The paper has no counterpart (a service of the
 * library, like pt_energy_noalloc).
 *   plan_bytes     : receives the plan's own workspace (octree, expansions,
 *                    work list and partial slabs), at 512-byte granularity.
 *   operator_bytes : receives the translation operators, which all plans of
 *                    one (device, p, precision) share: counted once.
 * Errors: PT_ERR_ARG (as fmm_plan_create), PT_ERR_UNSUPPORTED. */
int fmm_plan_footprint(int64_t n_max, int p, int leaf_max, int depth, int precision,
                       int64_t* plan_bytes, int64_t* operator_bytes);

/* ---------------------------------------------------------------------------
 * Ensembles: many independent crystals (e.g. trajectories of the stochastic
 * laser cooling of Sec. 2.2, or crystals of different ion counts and rotation
 * frequencies) advanced together.  Each member is the step of Eq. time_ev2
 * on its own crystal with its own plan; the members do not interact.
 *
 * pt_ensemble_create -- groups n_members distinct plans of one device.
 *   plans : host array of n_members plans, one per crystal.  The caller keeps
 *           them and must not destroy or use them elsewhere while the
 *           ensemble is stepping them.
 *   out   : receives the ensemble.
 * Members' kernels share the GPU; fmm_plan_set_m2l_ctas lets each member's
 * persistent M2L kernel take fewer CTAs than one per SM.
 * Errors: PT_ERR_ARG (NULL, duplicate plans, mixed devices), PT_ERR_OOM,
 * PT_ERR_CUDA. */
typedef struct pt_ensemble_s* pt_ensemble;
int pt_ensemble_create(int n_members, const fmm_plan* plans, pt_ensemble* out);

/* pt_ensemble_step -- advances every member b by n_steps steps.
 *   states : host array of n_members pt_state (device pointers inside);
 *            member b's t and step advance as with pt_step.
 *   traps  : host array of n_members traps.
 *   lasers : host array of n_members lasers, or NULL for no cooling.
 *   dt     : host array of n_members time steps (s).
 *   stream : CUDA stream (cudaStream_t) or NULL.
 * Every step of the whole ensemble is one launch of one CUDA graph holding
 * each member's step as a parallel branch (captured once, again when a
 * member's depth, buffers or parameters change).  The M2L launches of the
 * members that use the BF16x3 pair-packed schedule (Eq. FMM_local) are
 * replaced in that graph by one launch over all of their work items, which
 * waits for every such member's multipoles and precedes every member's
 * reduction (see pt_ensemble_set_joined_m2l).  A member's result equals
 * the same plan stepped alone by pt_step, bit for bit.  Asynchronous like
 * pt_step_async: automatic-depth plans keep the depth chosen at their first
 * step; device errors are latched and returned by pt_ensemble_sync.
 * Errors: PT_ERR_ARG (any member's arguments as in pt_step), PT_ERR_CUDA. */
int pt_ensemble_step(pt_ensemble ens, pt_state* states, const pt_trap* traps,
                     const pt_laser* lasers, const double* dt, int64_t n_steps, void* stream);

/* pt_ensemble_sync -- waits for the stream and returns the first member's
 * latched device error (PT_ERR_NONFINITE, PT_ERR_TIMEOUT, ...) or PT_OK.
 * A timeout of the joined M2L launch is latched by the first joined member. */
int pt_ensemble_sync(pt_ensemble ens, void* stream);

/* pt_ensemble_set_joined_m2l -- on != 0 (default): the members' BF16x3
 * pair-packed M2L launches run as one launch (pt_ensemble_step); 0: each
 * member launches its own.  Takes effect at the next step (re-capture).
 * Errors: PT_ERR_ARG (NULL). */
int pt_ensemble_set_joined_m2l(pt_ensemble ens, int on);

/* pt_ensemble_joined_m2l -- *members receives how many members the last
 * captured graph's joined M2L launch covers (0: none joined; fewer than two
 * eligible members are never joined).  Errors: PT_ERR_ARG (NULL). */
int pt_ensemble_joined_m2l(pt_ensemble ens, int* members);

/* pt_ensemble_destroy -- frees the ensemble (not its plans). */
int pt_ensemble_destroy(pt_ensemble ens);

#ifdef __cplusplus
}
#endif
#endif /* PENNING_H */
