// mh.cu -- Metropolis-Hastings potential-energy initialisation of a crystal
// (Sec. 4: starting from an equilibrium, ions are displaced one after the
// other by a random distance below dx in a random direction; a move is kept
// if the crystal's potential energy falls, or else with probability
// exp(-dE / (k_B T)); one scan visits every ion once).
//
// Potential energy: the rotating-frame one at the state's time (Eq. pe_rot
// with the wall phase (c, s) = (cos w_r t, sin w_r t) given by the caller):
// per ion U(x) = q k_z (2 z^2 - x^2 - y^2)/4 + (q B w_r - m w_r^2)(x^2 + y^2)/2
// + q k_z delta (x_r^2 - y_r^2)/4, plus the Coulomb pair energy, so moving
// ion i from a to b changes it by
//   dE = (U(b) - U(a)) + k_e q_i sum_{j != i} q_j (1/|b - x_j| - 1/|a - x_j|).
//
// Random numbers (rng.cuh's Philox, the photon-kick stream with beam field
// 0xFF, the scan in place of the step): slot 0 words (0,1) -> the distance
// fraction, (2,3) -> the accept uniform; slots 1, 2, ... -> (v1, v2) pairs of
// Marsaglia's disc pick of the direction.  The distance depends on |b - a|
// only: the proposal is symmetric.
//
// Crystals of up to 4096 ions run on a cluster of 8 CTAs (below), larger ones
// on one 1024-thread block: thread 0 draws the proposal and takes the
// decision, all threads sum the Coulomb change over their share of the other
// ions (FP64), combined by a fixed tree (deterministic).  Compiled with
// -fmad=false like the push, so the proposal and U are the literal IEEE
// sequence; the pair sum (its order, and rsqrt on the cluster path) differs
// from the sequential 1/sqrt sum only in the last bits of dE.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"

namespace pt {

constexpr int kMhThreads = 1024;

__device__ __forceinline__ double mh_u_ext(const MhParams& mp, double qi, double x, double y,
                                           double z) {
    const double xr = mp.c * x - mp.s * y, yr = mp.s * x + mp.c * y, r2 = x * x + y * y;
    return 0.25 * qi * mp.kz * (2.0 * z * z - r2) + 0.5 * (qi * mp.B * mp.wr - mp.m * mp.wr * mp.wr) * r2 +
           0.25 * qi * mp.kz * mp.delta * (xr * xr - yr * yr);
}

__global__ void __launch_bounds__(kMhThreads) k_mh_scans(int64_t n, double* x, double* y, double* z,
                                                         const double* __restrict__ q, MhParams mp,
                                                         int64_t scan0, int64_t n_scans,
                                                         unsigned long long* acc_out,
                                                         double* de_out) {
    __shared__ double prop[4];  // b and the accept uniform
    __shared__ double red[kMhThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    unsigned long long acc = 0;
    double de_sum = 0.0;
    for (int64_t sc = 0; sc < n_scans; ++sc) {
        const uint64_t scan = (uint64_t)(scan0 + sc);
        for (int64_t i = 0; i < n; ++i) {
            if (tid == 0) {
                uint32_t w[4];
                philox4x32_10((uint32_t)i, 0xFFu, (uint32_t)scan, (uint32_t)(scan >> 32),
                              (uint32_t)mp.seed, (uint32_t)(mp.seed >> 32), w);
                const double r = mp.dx * u01(w[0], w[1]);
                const double u = u01(w[2], w[3]);
                double v1 = 0.0, v2 = 0.0, ss = 0.0;
                for (uint32_t slot = 1; slot <= (uint32_t)kMaxTries; ++slot) {
                    philox4x32_10((uint32_t)i, 0xFFu | (slot << 8), (uint32_t)scan,
                                  (uint32_t)(scan >> 32), (uint32_t)mp.seed,
                                  (uint32_t)(mp.seed >> 32), w);
                    v1 = 2.0 * u01(w[0], w[1]) - 1.0;
                    v2 = 2.0 * u01(w[2], w[3]) - 1.0;
                    ss = v1 * v1 + v2 * v2;
                    if (ss < 1.0) break;
                }
                const double f = 2.0 * sqrt(1.0 - ss);
                prop[0] = x[i] + r * (v1 * f);
                prop[1] = y[i] + r * (v2 * f);
                prop[2] = z[i] + r * (1.0 - 2.0 * ss);
                prop[3] = u;
            }
            __syncthreads();
            const double ax = x[i], ay = y[i], az = z[i];
            const double bx = prop[0], by = prop[1], bz = prop[2];
            double part = 0.0;
            for (int64_t j = tid; j < n; j += kMhThreads) {
                if (j == i) continue;
                const double dbx = bx - x[j], dby = by - y[j], dbz = bz - z[j];
                const double dax = ax - x[j], day = ay - y[j], daz = az - z[j];
                part += q[j] * (1.0 / sqrt(dbx * dbx + dby * dby + dbz * dbz) -
                                1.0 / sqrt(dax * dax + day * day + daz * daz));
            }
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) red[wid] = part;
            __syncthreads();
            if (tid == 0) {
                double sum = 0.0;
                for (int k = 0; k < kMhThreads / 32; ++k) sum += red[k];
                const double qi = q[i];
                const double dE = (mh_u_ext(mp, qi, bx, by, bz) - mh_u_ext(mp, qi, ax, ay, az)) +
                                  mp.ke * qi * sum;
                if (dE < 0.0 || prop[3] < pt_exp(-dE / (mp.kb * mp.temp))) {
                    x[i] = bx;
                    y[i] = by;
                    z[i] = bz;
                    ++acc;
                    de_sum += dE;
                }
            }
            __syncthreads();  // the move (or not) is seen by the next proposal
        }
    }
    if (tid == 0) {
        *acc_out = acc;
        *de_out = de_sum;
    }
}

// ---------------------------------------------------------------------------
// The same chain on a cluster of kMhCtas CTAs (crystals of up to kMhClusterIons
// ions).  Each CTA keeps a replica of the positions and charges in shared
// memory.  Per scan, the proposals (b = a + displacement, the accept uniform,
// the external-energy change U(b) - U(a)) are drawn for all ions in parallel:
// they depend only on the moving ion's own position, which no earlier move
// of the scan changes.  Per move, every CTA sums the Coulomb change over its
// share of the other ions (FP64, rsqrt), writes its partial into a
// double-buffered slot, and after one cluster barrier every CTA's thread 0
// adds the partials of all CTAs in rank order (distributed shared memory),
// takes the same decision and updates its replica.  The barrier is the
// hardware cluster barrier; nothing spins.
// ---------------------------------------------------------------------------
constexpr int kMhCtas = 8;
constexpr int kMhCtaThreads = 256;
constexpr int64_t kMhClusterIons = 4096;

__global__ void __launch_bounds__(kMhCtaThreads) k_mh_scans_cluster(
    int64_t n, double* x, double* y, double* z, const double* __restrict__ q, MhParams mp,
    int64_t scan0, int64_t n_scans, double* prop, unsigned long long* acc_out, double* de_out) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), nr = (int)cl.num_blocks();
    extern __shared__ double mh_sm[];
    double* sx = mh_sm;
    double* sy = sx + n;
    double* sz = sy + n;
    double* sq = sz + n;
    __shared__ double slot[2];
    __shared__ double red[kMhCtaThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int64_t j = tid; j < n; j += kMhCtaThreads) {
        sx[j] = x[j];
        sy[j] = y[j];
        sz[j] = z[j];
        sq[j] = q[j];
    }
    __syncthreads();
    unsigned long long acc = 0;
    double de_sum = 0.0;
    const int64_t gt = (int64_t)rank * kMhCtaThreads + tid, gs = (int64_t)nr * kMhCtaThreads;
    for (int64_t sc = 0; sc < n_scans; ++sc) {
        const uint64_t scan = (uint64_t)(scan0 + sc);
        for (int64_t i = gt; i < n; i += gs) {
            uint32_t w[4];
            philox4x32_10((uint32_t)i, 0xFFu, (uint32_t)scan, (uint32_t)(scan >> 32),
                          (uint32_t)mp.seed, (uint32_t)(mp.seed >> 32), w);
            const double r = mp.dx * u01(w[0], w[1]);
            const double u = u01(w[2], w[3]);
            double v1 = 0.0, v2 = 0.0, ss = 0.0;
            for (uint32_t slt = 1; slt <= (uint32_t)kMaxTries; ++slt) {
                philox4x32_10((uint32_t)i, 0xFFu | (slt << 8), (uint32_t)scan,
                              (uint32_t)(scan >> 32), (uint32_t)mp.seed, (uint32_t)(mp.seed >> 32),
                              w);
                v1 = 2.0 * u01(w[0], w[1]) - 1.0;
                v2 = 2.0 * u01(w[2], w[3]) - 1.0;
                ss = v1 * v1 + v2 * v2;
                if (ss < 1.0) break;
            }
            const double f = 2.0 * sqrt(1.0 - ss);
            const double ax = sx[i], ay = sy[i], az = sz[i];
            const double bx = ax + r * (v1 * f), by = ay + r * (v2 * f), bz = az + r * (1.0 - 2.0 * ss);
            double* pr = prop + 5 * i;
            pr[0] = bx;
            pr[1] = by;
            pr[2] = bz;
            pr[3] = u;
            pr[4] = mh_u_ext(mp, sq[i], bx, by, bz) - mh_u_ext(mp, sq[i], ax, ay, az);
        }
        cl.sync();  // the scan's proposals, written by every CTA, are visible
        for (int64_t i = 0; i < n; ++i) {
            const double* pr = prop + 5 * i;
            const double bx = __ldcg(pr), by = __ldcg(pr + 1), bz = __ldcg(pr + 2);
            double u = 0.0, dU = 0.0;
            if (tid == 0) {
                u = __ldcg(pr + 3);
                dU = __ldcg(pr + 4);
            }
            const double ax = sx[i], ay = sy[i], az = sz[i];
            double part = 0.0;
            for (int64_t j = gt; j < n; j += gs) {
                if (j == i) continue;
                const double dbx = bx - sx[j], dby = by - sy[j], dbz = bz - sz[j];
                const double dax = ax - sx[j], day = ay - sy[j], daz = az - sz[j];
                part += sq[j] * (rsqrt(dbx * dbx + dby * dby + dbz * dbz) -
                                 rsqrt(dax * dax + day * day + daz * daz));
            }
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) red[wid] = part;
            __syncthreads();
            if (tid == 0) {
                double p = 0.0;
                for (int k = 0; k < kMhCtaThreads / 32; ++k) p += red[k];
                slot[i & 1] = p;
            }
            cl.sync();  // every CTA's partial of this move is in its slot
            if (tid == 0) {
                double sum = 0.0;
                for (int k = 0; k < nr; ++k) sum += *cl.map_shared_rank(&slot[i & 1], k);
                const double dE = dU + mp.ke * sq[i] * sum;
                const int keep = (dE < 0.0 || u < pt_exp(-dE / (mp.kb * mp.temp))) ? 1 : 0;
                if (keep) {
                    sx[i] = bx;
                    sy[i] = by;
                    sz[i] = bz;
                    ++acc;
                    de_sum += dE;
                }
            }
            __syncthreads();  // the replica is updated before the next move reads it
        }
    }
    if (rank == 0) {
        for (int64_t j = tid; j < n; j += kMhCtaThreads) {
            x[j] = sx[j];
            y[j] = sy[j];
            z[j] = sz[j];
        }
        if (tid == 0) {
            *acc_out = acc;
            *de_out = de_sum;
        }
    }
    cl.sync();  // no CTA leaves while another may still read its slots
}

size_t mh_scratch_bytes(int64_t n) {
    return n <= kMhClusterIons ? sizeof(double) * 5 * (size_t)n : 0;
}

cudaError_t launch_mh_scans(int64_t n, double* x, double* y, double* z, const double* q,
                            const MhParams& mp, int64_t scan0, int64_t n_scans,
                            unsigned long long* acc_out, double* de_out, double* scratch,
                            cudaStream_t s) {
    if (n > kMhClusterIons || !scratch) {
        k_mh_scans<<<1, kMhThreads, 0, s>>>(n, x, y, z, q, mp, scan0, n_scans, acc_out, de_out);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(double) * 4 * (size_t)n;
    cudaError_t e = cudaFuncSetAttribute(k_mh_scans_cluster,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kMhCtas, 1, 1);
    cfg.blockDim = dim3(kMhCtaThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kMhCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mh_scans_cluster, n, x, y, z, q, mp, scan0, n_scans, scratch,
                              acc_out, de_out);
}

}  // namespace pt
