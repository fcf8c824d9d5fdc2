// push.cu -- the cyclotronic push (Eq. time_ev2) and the laser-cooling kicks
// (Eqs. scattering_rate, laser_kick), FP64.
//
// This translation unit is compiled with -fmad=false: every expression below
// is the literal sequence of IEEE double operations written, so that the
// photon counts and recoil kicks are bit-reproducible definitions (the same
// counter-based random numbers give the same kicks on any conforming
// implementation of the same sequence).
//
// Random numbers (rng.cuh): Philox4x32-10, key = (seed lo, seed hi),
// counter = (ion, beam | slot << 8, step lo, step hi); the exponential of
// the rates and Poisson draws is rng.cuh's pt_exp.
#include <cuda_runtime.h>

#include "bbox.cuh"
#include "internal.h"
#include "rng.cuh"

namespace pt {

__device__ __forceinline__ double saturation(const pt_beam& b, double y, double z) {
    if (b.uniform) return b.s0;
    double dy = y - b.offset_d;
    double a = (dy * dy) / (b.waist_y * b.waist_y) + (z * z) / (b.waist_z * b.waist_z);
    return b.s0 * pt_exp(-a);
}

__device__ __forceinline__ double scatter_rate(const pt_beam& b, double gamma0, double y, double z,
                                               double vx, double vy, double vz) {
    double S = saturation(b, y, z);
    double g = 0.5 * gamma0;
    double g2 = g * g;
    double kv = (b.kx * vx + b.ky * vy) + b.kz * vz;
    double det = b.detuning - kv;
    double den = g2 * (1.0 + 2.0 * S) + det * det;
    return ((S * gamma0) * g2) / den;
}

__device__ __forceinline__ int poisson(double lambda, double u) {
    double p = pt_exp(-lambda);
    double F = p;
    int k = 0;
    while (u >= F && k < kMaxPhotons) {
        k = k + 1;
        p = p * lambda / (double)k;
        F = F + p;
    }
    return k;
}

// Photon count of beam l for ion i at its midpoint state: the scattering
// rate of Eq. scattering_rate times dt is the Poisson mean (Eq. laser_kick).
__device__ __forceinline__ int beam_count(const pt_laser& L, int64_t i, int64_t step, double dt,
                                          int l, double y, double z, double vx, double vy,
                                          double vz) {
    const pt_beam& b = L.beam[l];
    double rate = scatter_rate(b, L.gamma0, y, z, vx, vy, vz);
    double lam = rate * dt;
    uint32_t blk[4];
    stream_block(L.seed, step, i, l, 0u, blk);
    return poisson(lam, u01(blk[0], blk[1]));
}

// Recoil of cnt > 0 photons of beam l (Eq. laser_kick): cnt absorptions
// along the beam and cnt isotropic emissions (Marsaglia's disc method),
// added in this order to (ax, ay, az).
__device__ void beam_recoil(const pt_laser& L, double rk, int64_t i, int64_t step, int l, int cnt,
                            double& ax, double& ay, double& az) {
    const pt_beam& b = L.beam[l];
    double kmag = sqrt((b.kx * b.kx + b.ky * b.ky) + b.kz * b.kz);
    double fc = (double)cnt * rk;
    ax = ax + fc * b.kx;
    ay = ay + fc * b.ky;
    az = az + fc * b.kz;
    double em = rk * kmag;
    uint32_t slot = 1;
    uint32_t blk[4];
    for (int j = 0; j < cnt; ++j) {
        double v1 = 0.0, v2 = 0.0, s = 0.0;
        for (int tr = 0; tr < kMaxTries; ++tr) {
            stream_block(L.seed, step, i, l, slot, blk);
            slot = slot + 1;
            v1 = 2.0 * u01(blk[0], blk[1]) - 1.0;
            v2 = 2.0 * u01(blk[2], blk[3]) - 1.0;
            s = v1 * v1 + v2 * v2;
            if (s < 1.0) break;
        }
        double w = 2.0 * sqrt(1.0 - s);
        ax = ax + em * (v1 * w);
        ay = ay + em * (v2 * w);
        az = az + em * (1.0 - 2.0 * s);
    }
}

// Photon counts and recoil of ion i at its midpoint state (Eq. laser_kick),
// the beams in order.
__device__ void laser_ion(const pt_laser& L, double rk, int64_t i, int64_t step, double dt,
                          double y, double z, double vx, double vy, double vz, int32_t* counts_row,
                          double& ax, double& ay, double& az) {
    ax = 0.0;
    ay = 0.0;
    az = 0.0;
    for (int l = 0; l < L.n_beams; ++l) {
        int cnt = beam_count(L, i, step, dt, l, y, z, vx, vy, vz);
        if (counts_row) counts_row[l] = cnt;
        if (cnt == 0) continue;
        beam_recoil(L, rk, i, step, l, cnt, ax, ay, az);
    }
}

// Exact gyration U0(h) (Eq. U0, B along +z: clockwise velocity rotation).
__device__ __forceinline__ void gyrate(const PushParams& pp, double& x, double& y, double& z,
                                       double& vx, double& vy, double vz) {
    double ux = vx, uy = vy;
    x = x + (ux * pp.S + uy * (1.0 - pp.C)) / pp.wc;
    y = y + (uy * pp.S - ux * (1.0 - pp.C)) / pp.wc;
    z = z + vz * pp.h;
    vx = ux * pp.C + uy * pp.S;
    vy = -ux * pp.S + uy * pp.C;
}

// First half-drift of a step, fused with the bounding cube of the midpoint
// positions; the finalising thread also advances the step counter.
__global__ void __launch_bounds__(kBboxThreads) k_drift_bbox(int64_t n, int64_t per, double* x,
                                                             double* y, double* z, double* vx,
                                                             double* vy, const double* vz,
                                                             PushParams pp,
                                                             unsigned long long* acc,
                                                             unsigned* ticket, RootCube* root,
                                                             int* err, StepCounter* steps) {
    BboxAcc t;
    const int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        double px = x[i], py = y[i], pz = z[i], ux = vx[i], uy = vy[i];
        gyrate(pp, px, py, pz, ux, uy, vz[i]);
        x[i] = px;
        y[i] = py;
        z[i] = pz;
        vx[i] = ux;
        vy[i] = uy;
        t.add(px, py, pz);
    }
    if (bbox_commit(t, acc, ticket, root, err)) {
        steps->cur = steps->next;
        steps->next = steps->next + 1;
    }
}

// Kick (Eq. velocity_kick with the laser kicks of Eq. laser_kick) and the
// second half-drift.  A block takes an equal contiguous share of the ions
// (ion_split: FP64 is the bound, so every SM gets the same amount) in runs of
// kKickIons: the block's threads first draw the photon counts of every
// (beam, ion) pair of the run in parallel (the rate and Poisson draw, the
// bulk of the FP64 work), then one thread per ion adds the recoils of the
// beams in order, kicks and drifts, exactly the sequence of laser_ion.
constexpr int kKickIons = 128;
constexpr int kKickThreads = 256;
__global__ void __launch_bounds__(kKickThreads) k_kick_drift(
    int64_t n, int64_t per, double* x, double* y, double* z, double* vx, double* vy, double* vz,
    const double* __restrict__ q, const double* __restrict__ E, PushParams pp, pt_laser laser,
    const StepCounter* steps, const double* __restrict__ wall_cs) {
    pdl_wait();
    __shared__ int s_cnt[PT_MAX_BEAMS][kKickIons];
    const bool lasers = laser.enabled && laser.n_beams > 0;
    const int nb = lasers ? laser.n_beams : 0;
    const int64_t step = steps->cur;
    const int64_t widx = step - steps->base;
    const double c = wall_cs[2 * widx], s = wall_cs[2 * widx + 1];
    const double kw = 0.5 * pp.kz * pp.delta;
    const int64_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
    for (int64_t r0 = b0; r0 < b1; r0 += kKickIons) {
        const int nr = (int)min((int64_t)kKickIons, b1 - r0);
        if (lasers) {
            for (int j = threadIdx.x; j < nb * nr; j += kKickThreads) {
                const int l = j / nr, k = j - l * nr;
                const int64_t i = r0 + k;
                s_cnt[l][k] = beam_count(laser, i, step, pp.dt, l, y[i], z[i], vx[i], vy[i], vz[i]);
            }
            __syncthreads();
        }
        for (int k = threadIdx.x; k < nr; k += kKickThreads) {
            const int64_t i = r0 + k;
            double px = x[i], py = y[i], pz = z[i], ux = vx[i], uy = vy[i], uz = vz[i];
            double etx = 0.5 * pp.kz * px, ety = 0.5 * pp.kz * py, etz = -pp.kz * pz;
            double ewx = -kw * (px * c - py * s);
            double ewy = -kw * (-py * c - px * s);
            double Fx = etx + ewx, Fy = ety + ewy, Fz = etz;
            double dx = 0.0, dy = 0.0, dz = 0.0;
            for (int l = 0; l < nb; ++l) {
                const int cnt = s_cnt[l][k];
                if (cnt != 0) beam_recoil(laser, pp.rk, i, step, l, cnt, dx, dy, dz);
            }
            double qm = q[i] / pp.mass;
            ux = ux + qm * (E[i] + Fx) * pp.dt + dx;
            uy = uy + qm * (E[n + i] + Fy) * pp.dt + dy;
            uz = uz + qm * (E[2 * n + i] + Fz) * pp.dt + dz;
            if (pp.damp != 1.0) {
                // artificial damping: the velocity relative to the rigid rotation
                // at this (mid-step) position shrinks by exp(-gamma dt)
                const double rx = pp.wr * py, ry = -pp.wr * px;
                ux = rx + pp.damp * (ux - rx);
                uy = ry + pp.damp * (uy - ry);
                uz = pp.damp * uz;
            }
            gyrate(pp, px, py, pz, ux, uy, uz);
            x[i] = px;
            y[i] = py;
            z[i] = pz;
            vx[i] = ux;
            vy[i] = uy;
            vz[i] = uz;
        }
        if (lasers) __syncthreads();  // s_cnt is rewritten for the next run
    }
}

__global__ void k_laser_kicks(pt_laser laser, double rk, int64_t n, const double* x,
                              const double* y, const double* z, const double* vx,
                              const double* vy, const double* vz, int64_t step, double dt,
                              int32_t* counts, double* dv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double ax, ay, az;
        laser_ion(laser, rk, i, step, dt, y[i], z[i], vx[i], vy[i], vz[i],
                  counts ? counts + i * laser.n_beams : nullptr, ax, ay, az);
        dv[i] = ax;
        dv[n + i] = ay;
        dv[2 * n + i] = az;
    }
}

static int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    if (g > 152 * 16) g = 152 * 16;
    return g > 0 ? (int)g : 1;
}

cudaError_t launch_drift_bbox(int64_t n, double* x, double* y, double* z, double* vx, double* vy,
                              double* vz, const PushParams& pp, Workspace& ws, cudaStream_t s) {
    const IonSplit sp = bbox_split(n, ws);
    k_drift_bbox<<<sp.grid, kBboxThreads, 0, s>>>(n, sp.per, x, y, z, vx, vy, vz, pp, ws.bbox_acc,
                                                  ws.ticket, ws.root, ws.err, ws.steps);
    return cudaGetLastError();
}

cudaError_t launch_kick_drift(int64_t n, double* x, double* y, double* z, double* vx, double* vy,
                              double* vz, const double* q, const double* E, const PushParams& pp,
                              const pt_laser& laser, Workspace& ws, cudaStream_t s) {
    const IonSplit sp = ion_split(n, kKickIons, ws.sms, (int64_t)1 << 30);
    return launch_pdl(k_kick_drift, dim3(sp.grid), dim3(kKickThreads), 0, s, n, sp.per, x, y, z, vx,
                      vy, vz, q, E, pp, laser, (const StepCounter*)ws.steps,
                      (const double*)ws.wall_cs);
}

cudaError_t launch_laser_kicks(const pt_laser& laser, double rk, int64_t n, const double* x,
                               const double* y, const double* z, const double* vx,
                               const double* vy, const double* vz, int64_t step, double dt,
                               int32_t* counts, double* dv, cudaStream_t s) {
    k_laser_kicks<<<grid_for(n, 128), 128, 0, s>>>(laser, rk, n, x, y, z, vx, vy, vz, step, dt,
                                                    counts, dv);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Rotating-frame energy parts (Eq. rotation, Eq. pe_rot first line), a
// deterministic two-stage reduction with compensated sums.
// ---------------------------------------------------------------------------
struct Neu2 {
    double s = 0, c = 0;
    __device__ void add(double v) {
        double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
};

constexpr int kEnergyBlocks = 256;

__global__ void __launch_bounds__(256) k_energy_partial(int64_t n, pt_state st, pt_trap trap,
                                                        double kz, double c, double s,
                                                        const double* phi, double* partial) {
    __shared__ double sh[3][256];
    Neu2 a[3];
    const double m = trap.mass, wr = trap.omega_r, B = trap.B;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x = st.x[i], y = st.y[i], z = st.z[i];
        double wx = st.vx[i] - wr * y, wy = st.vy[i] + wr * x, vz = st.vz[i];
        a[0].add(0.5 * m * (wx * wx + wy * wy + vz * vz));
        double xr = c * x - s * y, yr = s * x + c * y;
        double r2 = x * x + y * y;
        double qi = st.q[i];
        a[1].add(0.25 * qi * kz * (2.0 * z * z - r2));
        a[1].add(0.5 * (qi * B * wr - m * wr * wr) * r2);
        a[1].add(0.25 * qi * kz * trap.delta * (xr * xr - yr * yr));
        if (phi) a[2].add(0.5 * qi * phi[i]);
    }
    for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] = a[k].s + a[k].c;
    __syncthreads();
    if (threadIdx.x < 3) {
        Neu2 t;
        for (int j = 0; j < (int)blockDim.x; ++j) t.add(sh[threadIdx.x][j]);
        partial[blockIdx.x * 3 + threadIdx.x] = t.s + t.c;
    }
}

__global__ void k_energy_final(const double* partial, int nb, double* out) {
    if (threadIdx.x < 3) {
        Neu2 t;
        for (int b = 0; b < nb; ++b) t.add(partial[b * 3 + threadIdx.x]);
        out[threadIdx.x] = t.s + t.c;
    }
}

cudaError_t launch_energy_parts(int64_t n, const pt_state& st, const pt_trap& trap, double kz,
                                const double* phi, double* d_out, cudaStream_t s) {
    double c = cos(trap.omega_r * st.t), sn = sin(trap.omega_r * st.t);
    double* partial = d_out + 4;  // caller provides 4 + 3 * kEnergyBlocks doubles
    k_energy_partial<<<kEnergyBlocks, 256, 0, s>>>(n, st, trap, kz, c, sn, phi, partial);
    k_energy_final<<<1, 32, 0, s>>>(partial, kEnergyBlocks, d_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Temperatures of the rotating-frame motion (Eqs. temp_ax, temp_pl), the same
// deterministic two-stage compensated reduction as the energy.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_temps_partial(int64_t n, pt_state st, double wr,
                                                       double* partial) {
    __shared__ double sh[2][256];
    Neu2 a[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double wx = st.vx[i] - wr * st.y[i], wy = st.vy[i] + wr * st.x[i], vz = st.vz[i];
        a[0].add(vz * vz);
        a[1].add(wx * wx + wy * wy);
    }
    for (int k = 0; k < 2; ++k) sh[k][threadIdx.x] = a[k].s + a[k].c;
    __syncthreads();
    if (threadIdx.x < 2) {
        Neu2 t;
        for (int j = 0; j < (int)blockDim.x; ++j) t.add(sh[threadIdx.x][j]);
        partial[blockIdx.x * 2 + threadIdx.x] = t.s + t.c;
    }
}

__global__ void k_temps_final(const double* partial, int nb, double m, double nkb, double* out) {
    if (threadIdx.x < 2) {
        Neu2 t;
        for (int b = 0; b < nb; ++b) t.add(partial[b * 2 + threadIdx.x]);
        const double sum = t.s + t.c;
        out[threadIdx.x] = threadIdx.x == 0 ? m * sum / nkb : m * sum / (2.0 * nkb);
    }
}

cudaError_t launch_temperatures(int64_t n, const pt_state& st, const pt_trap& trap, double* d_out,
                                cudaStream_t s) {
    double* partial = d_out + 2;
    k_temps_partial<<<kEnergyBlocks, 256, 0, s>>>(n, st, trap.omega_r, partial);
    k_temps_final<<<1, 32, 0, s>>>(partial, kEnergyBlocks, trap.mass, (double)n * 1.380649e-23,
                                   d_out);
    return cudaGetLastError();
}

// Rotating-frame position moments (Eq. rms_disp accumulates these over time).
__global__ void k_position_moments(int64_t n, pt_state st, double c, double s, double* acc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = st.x[i], y = st.y[i], z = st.z[i];
        const double xr = c * x - s * y, yr = s * x + c * y;
        acc[i] += xr;
        acc[n + i] += yr;
        acc[2 * n + i] += z;
        acc[3 * n + i] += xr * xr + yr * yr + z * z;
    }
}

cudaError_t launch_position_moments(int64_t n, const pt_state& st, const pt_trap& trap,
                                    double* acc, cudaStream_t s) {
    const double c = cos(trap.omega_r * st.t), sn = sin(trap.omega_r * st.t);
    k_position_moments<<<grid_for(n, 256), 256, 0, s>>>(n, st, c, sn, acc);
    return cudaGetLastError();
}

// Delta r_rms of every ion (Eq. rms_disp) from K accumulations of the
// rotating-frame moments: sqrt(<|x_r|^2> - |<x_r>|^2), the variance clamped
// at zero against rounding.
__global__ void k_rms_displacement(int64_t n, const double* __restrict__ acc, double inv_k,
                                   double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double mx = acc[i] * inv_k, my = acc[n + i] * inv_k, mz = acc[2 * n + i] * inv_k;
        const double v = acc[3 * n + i] * inv_k - (mx * mx + my * my + mz * mz);
        out[i] = v > 0.0 ? sqrt(v) : 0.0;
    }
}

cudaError_t launch_rms_displacement(int64_t n, const double* acc, int64_t samples, double* out,
                                    cudaStream_t s) {
    k_rms_displacement<<<grid_for(n, 256), 256, 0, s>>>(n, acc, 1.0 / (double)samples, out);
    return cudaGetLastError();
}

}  // namespace pt
