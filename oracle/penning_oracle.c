/*
 * penning_oracle.c -- plain, slow, FP64 CPU oracle for the Penning-trap
 * ion-crystal time step of Zaris, Johnson, Shankar, Bollinger & Parker,
 * "Numerical Simulations of 3D Ion Crystal Dynamics in a Penning Trap using
 * the Fast Multipole Method" (arXiv:2405.13973).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the CUDA library; where both
 * sides must agree bit for bit (the photon-scattering random numbers and the
 * exponential they feed), each side implements the same published definition
 * on its own.
 *
 * What it computes, each function citing the passage it follows:
 *   - the Coulomb field and potential as the plain O(N^2) pair sum
 *     (Hamiltonian, Eq. hamiltonian; Sec. 2.3 "direct" mode);
 *   - the same sum restricted to pairs in adjacent leaves of a uniform
 *     octree (the near field of the FMM, Sec. 2.3.2);
 *   - the octree root cube and Morton leaf keys (Sec. 2.3.2);
 *   - the external trap and rotating-wall fields (Eqs. pot_trap, pot_wall);
 *   - the exact gyration U0 (Eq. U0, sign reading in the header notes);
 *   - the photon-scattering rate, Poisson counts and recoil kicks
 *     (Eqs. scattering_rate, laser_kick; Sec. 2.2);
 *   - the literal cyclotronic step U0(dt/2) Ukick U0(dt/2) (Eq. time_ev2);
 *   - the rotating-frame energy (Eq. rotation and Eq. pe_rot);
 *   - the Metropolis-Hastings potential-energy initialisation (Sec. 4).
 *
 * Parity status: every function below is pinned by tests/test_oracle_*.py
 * against closed forms, a library routine, or brute force (see the tests).
 *
 * Build: plain C11, -O2 -ffp-contract=off (no fused multiply-add anywhere,
 * so the laser arithmetic is the literal sequence of IEEE operations),
 * OpenMP for the independent target loops only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- physical constants (CODATA 2018, SI) ---------------------------- */
#define ORC_EPS0 8.8541878128e-12
#define ORC_HBAR 1.054571817e-34
#define ORC_PI 3.14159265358979323846

static double orc_ke(void) { return 1.0 / (4.0 * ORC_PI * ORC_EPS0); }

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ======================================================================
 * Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Each round maps
 * (c0,c1,c2,c3) with key (k0,k1) to
 *   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),
 * M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl
 * constants (0x9E3779B9, 0xBB67AE85) between rounds; 10 rounds.
 * ====================================================================== */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform double in [0,1) from two 32-bit words: the top 27 bits of a and
 * the top 26 bits of b form a 53-bit integer k; u = k * 2^-53 (exact). */
double orc_u01(uint32_t a, uint32_t b) {
    uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return (double)k * 0x1.0p-53;
}

/* Counter layout of the photon-scattering stream (both sides implement it):
 *   key = (seed low 32 bits, seed high 32 bits)
 *   ctr = (ion index, beam | (slot << 8), step low 32 bits, step high 32 bits)
 * slot 0 gives the Poisson uniform; slots 1,2,... give one (v1,v2) pair each
 * for the Marsaglia sphere picks of that beam's photons, in order. */
static void orc_stream_block(uint64_t seed, int64_t step, int64_t ion, int beam,
                             uint32_t slot, uint32_t out[4]) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t st = (uint64_t)step;
    uint32_t ctr[4] = {(uint32_t)ion, (uint32_t)beam | (slot << 8), (uint32_t)st,
                       (uint32_t)(st >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* ======================================================================
 * exp(x), written from Cody & Waite's argument reduction ("Software Manual
 * for the Elementary Functions", 1980) and the Taylor series:
 *   k = floor(x/ln2 + 1/2),  r = (x - k*LN2_HI) - k*LN2_LO,  |r| <= ln2/2,
 *   e^r = sum_{j=0}^{13} r^j / j!  (Horner; truncation < 5e-18 relative),
 *   e^x = 2^k e^r  (exponent bits; two steps below the normal range).
 * LN2_HI is ln2 truncated to 40 fraction bits (k*LN2_HI is exact for
 * |k| < 2^13); LN2_LO = ln2 - LN2_HI rounded to double.  The coefficients
 * 1/j! are IEEE quotients of exactly representable integers.
 * ====================================================================== */
static const double ORC_LN2_HI = 0x1.62e42fefa2000p-1;
static const double ORC_LN2_LO = 0x1.9ef35793c7673p-41;
static const double ORC_INV_LN2 = 0x1.71547652b82fep+0;

static double orc_pow2i(int k) { /* 2^k for -1022 <= k <= 1023 */
    uint64_t bits = (uint64_t)(k + 1023) << 52;
    double d;
    memcpy(&d, &bits, sizeof d);
    return d;
}

double orc_exp(double x) {
    if (x != x) return x;
    if (x > 709.8) return INFINITY;
    if (x < -745.2) return 0.0;
    double kf = floor(x * ORC_INV_LN2 + 0.5);
    double r = (x - kf * ORC_LN2_HI) - kf * ORC_LN2_LO;
    double fact = 1.0;
    double c[14];
    for (int j = 0; j <= 13; ++j) {
        if (j > 0) fact = fact * (double)j;
        c[j] = 1.0 / fact;
    }
    double p = c[13];
    for (int j = 12; j >= 0; --j) p = p * r + c[j];
    int k = (int)kf;
    if (k >= -1022) return p * orc_pow2i(k);
    /* subnormal result: scale in two exact-then-rounded steps */
    return (p * orc_pow2i(k + 600)) * orc_pow2i(-600);
}

/* ======================================================================
 * Coulomb field and potential, direct pair sum (Eq. hamiltonian; the force on
 * ion i is -dH/dx_i = q_i k_e sum_{j!=i} q_j (x_i-x_j)/|x_i-x_j|^3 with
 * k_e = 1/(4 pi eps0); the 1/(8 pi eps0) in H is the double-count half).
 * E_i = k_e sum_{j!=i} q_j (x_i-x_j)/r^3,   phi_i = k_e sum_{j!=i} q_j/r.
 * Neumaier-compensated accumulation; OpenMP over target ions only.
 * If mask_depth >= 0, only pairs whose leaves (at that depth of the uniform
 * octree on the given root cube) are adjacent or equal are summed: the FMM
 * near field (Sec. 2.3.2: adjacent cubes are "calculated directly").
 * ====================================================================== */
typedef struct { double s, c; } orc_acc;
static void acc_add(orc_acc* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static double acc_val(const orc_acc* a) { return a->s + a->c; }

static int64_t orc_leaf_coord(double x, double lo, double side, int depth) {
    double t = ((x - lo) / side) * (double)((int64_t)1 << depth);
    double f = floor(t);
    int64_t m = ((int64_t)1 << depth) - 1;
    if (!(f >= 0.0)) return 0;
    if (f > (double)m) return m;
    return (int64_t)f;
}

static void orc_coulomb_impl(int64_t n, const double* x, const double* y, const double* z,
                             const double* q, double* Ex, double* Ey, double* Ez, double* phi,
                             const double* lo, double side, int mask_depth) {
    const double ke = orc_ke();
    int64_t* cx = NULL;
    if (mask_depth >= 0) {
        cx = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) {
            cx[3 * i + 0] = orc_leaf_coord(x[i], lo[0], side, mask_depth);
            cx[3 * i + 1] = orc_leaf_coord(y[i], lo[1], side, mask_depth);
            cx[3 * i + 2] = orc_leaf_coord(z[i], lo[2], side, mask_depth);
        }
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        orc_acc ax = {0, 0}, ay = {0, 0}, az = {0, 0}, ap = {0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (cx) {
                if (llabs(cx[3 * i] - cx[3 * j]) > 1 || llabs(cx[3 * i + 1] - cx[3 * j + 1]) > 1 ||
                    llabs(cx[3 * i + 2] - cx[3 * j + 2]) > 1)
                    continue;
            }
            double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double inv_r = 1.0 / r;
            double w = q[j] * inv_r / r2; /* q_j / r^3 */
            acc_add(&ax, w * dx);
            acc_add(&ay, w * dy);
            acc_add(&az, w * dz);
            acc_add(&ap, q[j] * inv_r);
        }
        Ex[i] = ke * acc_val(&ax);
        Ey[i] = ke * acc_val(&ay);
        Ez[i] = ke * acc_val(&az);
        if (phi) phi[i] = ke * acc_val(&ap);
    }
    free(cx);
}

void orc_coulomb_direct(int64_t n, const double* x, const double* y, const double* z,
                        const double* q, double* Ex, double* Ey, double* Ez, double* phi) {
    orc_coulomb_impl(n, x, y, z, q, Ex, Ey, Ez, phi, NULL, 1.0, -1);
}

/* The same sum (Eq. hamiltonian's pair term) at m chosen targets only:
 * target k is ion idx[k]; every other ion j != idx[k] is a source.  Same
 * pair expression and compensated accumulation in ascending j, so at a full
 * sample it reproduces orc_coulomb_direct bit for bit.  Serves the large-N
 * checks, where the all-pairs sum is out of reach on the host. */
void orc_coulomb_targets(int64_t n, const double* x, const double* y, const double* z,
                         const double* q, int64_t m, const int64_t* idx, double* Ex, double* Ey,
                         double* Ez, double* phi) {
    const double ke = orc_ke();
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < m; ++k) {
        const int64_t i = idx[k];
        orc_acc ax = {0, 0}, ay = {0, 0}, az = {0, 0}, ap = {0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double inv_r = 1.0 / r;
            double w = q[j] * inv_r / r2; /* q_j / r^3 */
            acc_add(&ax, w * dx);
            acc_add(&ay, w * dy);
            acc_add(&az, w * dz);
            acc_add(&ap, q[j] * inv_r);
        }
        Ex[k] = ke * acc_val(&ax);
        Ey[k] = ke * acc_val(&ay);
        Ez[k] = ke * acc_val(&az);
        if (phi) phi[k] = ke * acc_val(&ap);
    }
}

/* ======================================================================
 * Octree root cube and leaf keys (Sec. 2.3.2: "the smallest cube containing
 * all N ions is found" and is divided recursively into octants).
 * Root cube: per axis the min and max of the positions; side = the largest
 * extent (1.0 if every ion coincides); centre = (min+max)/2 per axis;
 * lo = centre - side/2.  Leaf coordinate on axis a at depth D:
 * floor(((x_a - lo_a)/side) * 2^D), clamped to [0, 2^D - 1].
 * Morton key: bits of (ix, iy, iz) interleaved, ix the most significant of
 * each triple:  key = sum_b ix_b 2^(3b+2) + iy_b 2^(3b+1) + iz_b 2^(3b).
 * ====================================================================== */
void orc_root_cube(int64_t n, const double* x, const double* y, const double* z, double lo[3],
                   double* side) {
    const double* p[3] = {x, y, z};
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = n > 0 ? p[a][0] : 0.0;
        mx[a] = mn[a];
        for (int64_t i = 1; i < n; ++i) {
            if (p[a][i] < mn[a]) mn[a] = p[a][i];
            if (p[a][i] > mx[a]) mx[a] = p[a][i];
        }
    }
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
        if (mx[a] - mn[a] > s) s = mx[a] - mn[a];
    if (!(s > 0.0)) s = 1.0;
    for (int a = 0; a < 3; ++a) lo[a] = 0.5 * (mn[a] + mx[a]) - 0.5 * s;
    *side = s;
}

void orc_leaf_keys(int64_t n, const double* x, const double* y, const double* z, int depth,
                   uint64_t* key, double lo_out[3], double* side_out) {
    double lo[3], side;
    orc_root_cube(n, x, y, z, lo, &side);
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3] = {orc_leaf_coord(x[i], lo[0], side, depth),
                        orc_leaf_coord(y[i], lo[1], side, depth),
                        orc_leaf_coord(z[i], lo[2], side, depth)};
        uint64_t k = 0;
        for (int b = 0; b < depth; ++b) {
            k |= (uint64_t)((c[0] >> b) & 1) << (3 * b + 2);
            k |= (uint64_t)((c[1] >> b) & 1) << (3 * b + 1);
            k |= (uint64_t)((c[2] >> b) & 1) << (3 * b);
        }
        key[i] = k;
    }
    if (lo_out) memcpy(lo_out, lo, sizeof lo);
    if (side_out) *side_out = side;
}

/* Near field of the uniform octree of depth D on the root cube above: the
 * pair sum restricted to ions whose leaves are equal or adjacent. */
void orc_coulomb_near(int64_t n, const double* x, const double* y, const double* z,
                      const double* q, int depth, double* Ex, double* Ey, double* Ez,
                      double* phi) {
    double lo[3], side;
    orc_root_cube(n, x, y, z, lo, &side);
    orc_coulomb_impl(n, x, y, z, q, Ex, Ey, Ez, phi, lo, side, depth);
}

/* ======================================================================
 * Trap parameters, passed as double[6] = {B, omega_z, omega_r, delta, m, q}
 * (SI; q is the reference charge that defines k_z = m omega_z^2 / q).
 * ====================================================================== */
enum { T_B = 0, T_WZ, T_WR, T_DELTA, T_M, T_Q };

/* External field at time t (Eqs. pot_trap and pot_wall):
 *   phi_trap = k_z (2z^2 - x^2 - y^2)/4       -> E = (k_z/2)(x, y, -2z)
 *   phi_wall = (k_z delta/4)[(x^2-y^2) cos 2w_r t - 2xy sin 2w_r t]
 *                                             -> E = -(k_z delta/2)(x c - y s, -y c - x s, 0)
 * with c = cos(2 w_r t), s = sin(2 w_r t), k_z = m w_z^2 / q. */
void orc_external_field(int64_t n, const double* trap, double t, const double* x,
                        const double* y, const double* z, double* Ex, double* Ey, double* Ez) {
    double kz = trap[T_M] * trap[T_WZ] * trap[T_WZ] / trap[T_Q];
    double c = cos(2.0 * trap[T_WR] * t), s = sin(2.0 * trap[T_WR] * t);
    double kw = 0.5 * kz * trap[T_DELTA];
    for (int64_t i = 0; i < n; ++i) {
        double etx = 0.5 * kz * x[i], ety = 0.5 * kz * y[i], etz = -kz * z[i];
        double ewx = -kw * (x[i] * c - y[i] * s);
        double ewy = -kw * (-y[i] * c - x[i] * s);
        Ex[i] = etx + ewx;
        Ey[i] = ety + ewy;
        Ez[i] = etz;
    }
}

/* ======================================================================
 * Exact gyration U0(h) in B = +B z (Eq. U0).  With q > 0 and B along +z the
 * Lorentz force dv/dt = (q/m) v x B turns the velocity clockwise seen from
 * +z, which is the crystal's rotation sense (v_x = +w_r y, Eq. rotation).  The
 * printed matrix turns it counter-clockwise and prints a zero last row; the
 * reading used is the printed matrix with w_c -> -w_c and v_z' = v_z:
 *   x' = x + (v_x S + v_y (1-C))/w_c,   v_x' =  v_x C + v_y S,
 *   y' = y + (v_y S - v_x (1-C))/w_c,   v_y' = -v_x S + v_y C,
 *   z' = z + v_z h,                     v_z' =  v_z,
 * with C = cos(w_c h), S = sin(w_c h), w_c = q B / m.
 * ====================================================================== */
void orc_u0(int64_t n, double h, double wc, double* x, double* y, double* z, double* vx,
            double* vy, double* vz) {
    double C = cos(wc * h), S = sin(wc * h);
    for (int64_t i = 0; i < n; ++i) {
        double ux = vx[i], uy = vy[i];
        x[i] = x[i] + (ux * S + uy * (1.0 - C)) / wc;
        y[i] = y[i] + (uy * S - ux * (1.0 - C)) / wc;
        z[i] = z[i] + vz[i] * h;
        vx[i] = ux * C + uy * S;
        vy[i] = -ux * S + uy * C;
    }
}

/* ======================================================================
 * Laser cooling (Sec. 2.2, Eqs. scattering_rate and laser_kick).
 * A beam is double[9] = {S0, detuning Delta (rad/s), kx, ky, kz (1/m),
 *                        w_y, w_z, d, uniform(0/1)}.
 * Saturation S(x): uniform beams S0; otherwise (a beam along x, Sec. 4)
 *   S = S0 exp(-((y-d)^2/w_y^2 + z^2/w_z^2)).
 * Rate (Eq. scattering_rate), with g = gamma0/2:
 *   gamma = S gamma0 g^2 / (g^2 (1 + 2S) + (Delta - k.v)^2).
 * Count n ~ Poisson(gamma dt) by inversion of the cumulative sum against the
 * slot-0 uniform (cap 64); recoil (Eq. laser_kick): n hbar k/m plus, per
 * photon, hbar |k|/m times a unit vector from Marsaglia's (1972) disc-to-
 * sphere map of (v1,v2) uniform in the unit disc:
 *   q = (2 v1 sqrt(1-s), 2 v2 sqrt(1-s), 1 - 2s),  s = v1^2 + v2^2 < 1.
 * The literal order of operations is part of the definition (bit-exact
 * agreement with the GPU is required); the file is compiled without FMA.
 * ====================================================================== */
enum { B_S0 = 0, B_DET, B_KX, B_KY, B_KZ, B_WY, B_WZ, B_D, B_UNI };
#define ORC_MAX_PHOTONS 64
#define ORC_MAX_TRIES 64

double orc_saturation(const double* beam, double y, double z) {
    if (beam[B_UNI] != 0.0) return beam[B_S0];
    double dy = y - beam[B_D];
    double a = (dy * dy) / (beam[B_WY] * beam[B_WY]) + (z * z) / (beam[B_WZ] * beam[B_WZ]);
    return beam[B_S0] * orc_exp(-a);
}

double orc_scatter_rate(const double* beam, double gamma0, double y, double z, double vx,
                        double vy, double vz) {
    double S = orc_saturation(beam, y, z);
    double g = 0.5 * gamma0;
    double g2 = g * g;
    double kv = (beam[B_KX] * vx + beam[B_KY] * vy) + beam[B_KZ] * vz;
    double det = beam[B_DET] - kv;
    double den = g2 * (1.0 + 2.0 * S) + det * det;
    return ((S * gamma0) * g2) / den;
}

int orc_poisson(double lambda, double u) {
    double p = orc_exp(-lambda);
    double F = p;
    int k = 0;
    while (u >= F && k < ORC_MAX_PHOTONS) {
        k = k + 1;
        p = p * lambda / (double)k;
        F = F + p;
    }
    return k;
}

/* Photon counts and recoil velocity change of every ion for one step.
 * x,v are the midpoint state (after the first U0(dt/2), before the kick).
 * counts: n * n_beams ints (or NULL); dv: velocity change (m/s). */
void orc_laser_kick(int64_t n, const double* beams, int n_beams, double gamma0, double mass,
                    uint64_t seed, int64_t step, double dt, const double* x, const double* y,
                    const double* z, const double* vx, const double* vy, const double* vz,
                    int32_t* counts, double* dvx, double* dvy, double* dvz) {
    (void)x;
    for (int64_t i = 0; i < n; ++i) {
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int l = 0; l < n_beams; ++l) {
            const double* b = beams + 9 * l;
            double rate = orc_scatter_rate(b, gamma0, y[i], z[i], vx[i], vy[i], vz[i]);
            double lam = rate * dt;
            uint32_t blk[4];
            orc_stream_block(seed, step, i, l, 0u, blk);
            int cnt = orc_poisson(lam, orc_u01(blk[0], blk[1]));
            if (counts) counts[i * n_beams + l] = cnt;
            if (cnt == 0) continue;
            double rk = ORC_HBAR / mass;
            double kmag = sqrt((b[B_KX] * b[B_KX] + b[B_KY] * b[B_KY]) + b[B_KZ] * b[B_KZ]);
            double fc = (double)cnt * rk;
            ax = ax + fc * b[B_KX];
            ay = ay + fc * b[B_KY];
            az = az + fc * b[B_KZ];
            double em = rk * kmag;
            uint32_t slot = 1;
            for (int j = 0; j < cnt; ++j) {
                double v1 = 0.0, v2 = 0.0, s = 0.0;
                for (int tr = 0; tr < ORC_MAX_TRIES; ++tr) {
                    orc_stream_block(seed, step, i, l, slot, blk);
                    slot = slot + 1;
                    v1 = 2.0 * orc_u01(blk[0], blk[1]) - 1.0;
                    v2 = 2.0 * orc_u01(blk[2], blk[3]) - 1.0;
                    s = v1 * v1 + v2 * v2;
                    if (s < 1.0) break;
                }
                double w = 2.0 * sqrt(1.0 - s);
                ax = ax + em * (v1 * w);
                ay = ay + em * (v2 * w);
                az = az + em * (1.0 - 2.0 * s);
            }
        }
        dvx[i] = ax;
        dvy[i] = ay;
        dvz[i] = az;
    }
}

/* ======================================================================
 * One literal cyclotronic step per iteration (Eq. time_ev2):
 *   (x,v) <- U0(dt/2)(x,v);  E = Coulomb(x) + external(x, t + dt/2);
 *   v <- v + (q_i/m) E dt + dv_lasers(x, v, step);  (x,v) <- U0(dt/2)(x,v);
 *   t <- t + dt.
 * Trap parameters as above; beams as above (n_beams may be 0); laser_on
 * switches the kicks; t0 and step0 are the time and step index at entry.
 * ====================================================================== */
/* The step above with optional artificial damping (Sec. 6: damping the
 * ions' motion to find crystal equilibria): after the kick, each ion's
 * velocity relative to the rigid rotation at w_r (the rotating-frame
 * velocity w = (v_x - w_r y, v_y + w_r x, v_z) at the mid-step position) is
 * scaled by f = exp(-gamma dt):  v <- (w_r y, -w_r x, 0) + f w.  f = 1 is the
 * undamped step.  The rotating-frame energy (orc_energy_rot) then falls by
 * gamma m |w|^2 per unit time (magnetic and Coriolis forces do no work), so
 * the crystal relaxes to a minimum of the rotating-frame potential. */
static void orc_step_impl(int64_t n, double* x, double* y, double* z, double* vx, double* vy,
                          double* vz, const double* q, const double* trap, const double* beams,
                          int n_beams, double gamma0, uint64_t seed, int laser_on, double dt,
                          double t0, int64_t step0, int64_t n_steps, double damp);

void orc_step(int64_t n, double* x, double* y, double* z, double* vx, double* vy, double* vz,
              const double* q, const double* trap, const double* beams, int n_beams,
              double gamma0, uint64_t seed, int laser_on, double dt, double t0, int64_t step0,
              int64_t n_steps) {
    orc_step_impl(n, x, y, z, vx, vy, vz, q, trap, beams, n_beams, gamma0, seed, laser_on, dt, t0,
                  step0, n_steps, 1.0);
}

void orc_step_damped(int64_t n, double* x, double* y, double* z, double* vx, double* vy,
                     double* vz, const double* q, const double* trap, const double* beams,
                     int n_beams, double gamma0, uint64_t seed, int laser_on, double dt, double t0,
                     int64_t step0, int64_t n_steps, double damping) {
    orc_step_impl(n, x, y, z, vx, vy, vz, q, trap, beams, n_beams, gamma0, seed, laser_on, dt, t0,
                  step0, n_steps, exp(-damping * dt));
}

static void orc_step_impl(int64_t n, double* x, double* y, double* z, double* vx, double* vy,
                          double* vz, const double* q, const double* trap, const double* beams,
                          int n_beams, double gamma0, uint64_t seed, int laser_on, double dt,
                          double t0, int64_t step0, int64_t n_steps, double damp) {
    double m = trap[T_M];
    double wc = trap[T_Q] * trap[T_B] / m;
    size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double *Ex = malloc(sz), *Ey = malloc(sz), *Ez = malloc(sz);
    double *Fx = malloc(sz), *Fy = malloc(sz), *Fz = malloc(sz);
    double *dvx = malloc(sz), *dvy = malloc(sz), *dvz = malloc(sz);
    for (int64_t s = 0; s < n_steps; ++s) {
        double t = t0 + (double)s * dt;
        orc_u0(n, 0.5 * dt, wc, x, y, z, vx, vy, vz);
        orc_coulomb_direct(n, x, y, z, q, Ex, Ey, Ez, NULL);
        orc_external_field(n, trap, t + 0.5 * dt, x, y, z, Fx, Fy, Fz);
        if (laser_on && n_beams > 0)
            orc_laser_kick(n, beams, n_beams, gamma0, m, seed, step0 + s, dt, x, y, z, vx, vy, vz,
                           NULL, dvx, dvy, dvz);
        else
            for (int64_t i = 0; i < n; ++i) dvx[i] = dvy[i] = dvz[i] = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double qm = q[i] / m;
            vx[i] = vx[i] + qm * (Ex[i] + Fx[i]) * dt + dvx[i];
            vy[i] = vy[i] + qm * (Ey[i] + Fy[i]) * dt + dvy[i];
            vz[i] = vz[i] + qm * (Ez[i] + Fz[i]) * dt + dvz[i];
        }
        if (damp != 1.0) {
            const double wr = trap[T_WR];
            for (int64_t i = 0; i < n; ++i) {
                const double rx = wr * y[i], ry = -wr * x[i];
                vx[i] = rx + damp * (vx[i] - rx);
                vy[i] = ry + damp * (vy[i] - ry);
                vz[i] = damp * vz[i];
            }
        }
        orc_u0(n, 0.5 * dt, wc, x, y, z, vx, vy, vz);
    }
    free(Ex); free(Ey); free(Ez); free(Fx); free(Fy); free(Fz);
    free(dvx); free(dvy); free(dvz);
}

/* ======================================================================
 * Rotating-frame energy at time t (Eq. rotation, Eq. pe_rot, Sec. 3):
 *   x_r = R(w_r t) x,  v_r = R(w_r t)(v_x - w_r y, v_y + w_r x),
 *   E_r = sum_i [ m|v_r|^2/2
 *               + q_i k_z (2 z^2 - x^2 - y^2)/4            (trap)
 *               + (q_i B w_r - m w_r^2)(x^2 + y^2)/2        (Lorentz + centrifugal)
 *               + q_i k_z delta (x_r^2 - y_r^2)/4 ]         (wall)
 *         + (1/2) sum_i q_i phi_i                            (Coulomb).
 * For q_i = q the planar terms are the first line of Eq. pe_rot.  out[4] =
 * {kinetic, external potential, Coulomb, total}.
 * ====================================================================== */
void orc_energy_rot(int64_t n, const double* x, const double* y, const double* z,
                    const double* vx, const double* vy, const double* vz, const double* q,
                    const double* trap, double t, double out[4]) {
    double m = trap[T_M], wr = trap[T_WR], B = trap[T_B];
    double kz = m * trap[T_WZ] * trap[T_WZ] / trap[T_Q];
    double c = cos(wr * t), s = sin(wr * t);
    size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double *Ex = malloc(sz), *Ey = malloc(sz), *Ez = malloc(sz), *phi = malloc(sz);
    orc_coulomb_direct(n, x, y, z, q, Ex, Ey, Ez, phi);
    orc_acc ke = {0, 0}, pe = {0, 0}, ce = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double wx = vx[i] - wr * y[i], wy = vy[i] + wr * x[i];
        acc_add(&ke, 0.5 * m * (wx * wx + wy * wy + vz[i] * vz[i]));
        double xr = c * x[i] - s * y[i], yr = s * x[i] + c * y[i];
        double r2 = x[i] * x[i] + y[i] * y[i];
        acc_add(&pe, 0.25 * q[i] * kz * (2.0 * z[i] * z[i] - r2));
        acc_add(&pe, 0.5 * (q[i] * B * wr - m * wr * wr) * r2);
        acc_add(&pe, 0.25 * q[i] * kz * trap[T_DELTA] * (xr * xr - yr * yr));
        acc_add(&ce, 0.5 * q[i] * phi[i]);
    }
    out[0] = acc_val(&ke);
    out[1] = acc_val(&pe);
    out[2] = acc_val(&ce);
    out[3] = out[0] + out[1] + out[2];
    free(Ex); free(Ey); free(Ez); free(phi);
}

/* ======================================================================
 * Temperatures of the rotating-frame motion (Eqs. temp_ax, temp_pl):
 *   T_par  = m sum_i w_z^2 / (N k_B),
 *   T_perp = m sum_i (w_x^2 + w_y^2) / (2 N k_B),
 * with w the velocity relative to the rigid rotation (w_x = v_x - w_r y,
 * w_y = v_y + w_r x, w_z = v_z); the rotation into the rotating frame
 * leaves w_x^2 + w_y^2 unchanged.  Instantaneous values (the paper's
 * angle brackets are time averages of these).  out[2] = {T_par, T_perp} (K).
 * ====================================================================== */
void orc_temperatures(int64_t n, const double* x, const double* y, const double* vx,
                      const double* vy, const double* vz, const double* trap, double out[2]) {
    const double m = trap[T_M], wr = trap[T_WR], kb = 1.380649e-23;
    orc_acc a = {0, 0}, b = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        const double wx = vx[i] - wr * y[i], wy = vy[i] + wr * x[i];
        acc_add(&a, vz[i] * vz[i]);
        acc_add(&b, wx * wx + wy * wy);
    }
    out[0] = m * acc_val(&a) / ((double)n * kb);
    out[1] = m * acc_val(&b) / (2.0 * (double)n * kb);
}

/* ======================================================================
 * Metropolis-Hastings potential-energy initialisation (Sec. 4, the laser-
 * cooling initialisation following Shankar et al. 2020): ions are visited in
 * order; ion i is displaced by a distance uniform in [0, dx) in a uniformly
 * random direction; with dE the change of the crystal's potential energy
 * the move is kept if dE < 0, or else if u < exp(-dE / (k_B T)), u uniform in
 * [0, 1); otherwise the ion goes back.  One scan visits every ion once.
 *
 * Potential energy (rotating frame at the state's time, wall phase given as
 * (c, s) = (cos w_r t, sin w_r t)): per ion
 *   U(x) = q k_z (2 z^2 - x^2 - y^2)/4 + (q B w_r - m w_r^2)(x^2 + y^2)/2
 *        + q k_z delta (x_r^2 - y_r^2)/4,   x_r = c x - s y, y_r = s x + c y,
 * plus the Coulomb pair energy; moving ion i from a to b changes it by
 *   dE = (U(b) - U(a)) + k_e q_i sum_{j != i} q_j (1/|b - x_j| - 1/|a - x_j|)
 * (the j sum in index order).
 *
 * Random numbers: the Philox stream of the photon kicks with the beam field
 * set to 0xFF (no beam uses it), the scan index in place of the step:
 *   ctr = (ion, 0xFF | (slot << 8), scan low, scan high), key = seed;
 * slot 0: words (0,1) -> the distance fraction, words (2,3) -> u;
 * slots 1, 2, ...: one (v1, v2) pair each for Marsaglia's disc pick of the
 * direction (v in (-1,1)^2 until s = v1^2 + v2^2 < 1; direction
 * (2 v1 sqrt(1-s), 2 v2 sqrt(1-s), 1 - 2 s)), at most 64 tries.
 * The proposal depends on |b - a| only, so it is symmetric and the plain
 * Metropolis test samples exp(-E / k_B T).
 *
 * Positions are updated in place; out[0] = accepted moves, out[1] = the sum
 * of the accepted dE (J).
 * ====================================================================== */
void orc_mh_scans(int64_t n, double* x, double* y, double* z, const double* q,
                  const double* trap, double c, double s, double temp, double dx, uint64_t seed,
                  int64_t scan0, int64_t n_scans, double out[2]) {
    const double m = trap[T_M], wr = trap[T_WR], B = trap[T_B], delta = trap[T_DELTA];
    const double kz = m * trap[T_WZ] * trap[T_WZ] / trap[T_Q];
    const double ke = orc_ke(), kb = 1.380649e-23;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t acc = 0;
    double de_sum = 0.0;
    for (int64_t sc = 0; sc < n_scans; ++sc) {
        const uint64_t scan = (uint64_t)(scan0 + sc);
        for (int64_t i = 0; i < n; ++i) {
            uint32_t ctr[4] = {(uint32_t)i, 0xFFu, (uint32_t)scan, (uint32_t)(scan >> 32)};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            const double r = dx * orc_u01(w[0], w[1]);
            const double u = orc_u01(w[2], w[3]);
            double v1 = 0.0, v2 = 0.0, ss = 0.0;
            for (uint32_t slot = 1; slot <= 64; ++slot) {
                uint32_t c2[4] = {(uint32_t)i, 0xFFu | (slot << 8), (uint32_t)scan,
                                  (uint32_t)(scan >> 32)};
                orc_philox4x32_10(c2, key, w);
                v1 = 2.0 * orc_u01(w[0], w[1]) - 1.0;
                v2 = 2.0 * orc_u01(w[2], w[3]) - 1.0;
                ss = v1 * v1 + v2 * v2;
                if (ss < 1.0) break;
            }
            const double f = 2.0 * sqrt(1.0 - ss);
            const double ax = x[i], ay = y[i], az = z[i];
            const double bx = ax + r * (v1 * f), by = ay + r * (v2 * f), bz = az + r * (1.0 - 2.0 * ss);
            /* external part */
            double ua, ub;
            {
                const double xr = c * ax - s * ay, yr = s * ax + c * ay, r2 = ax * ax + ay * ay;
                ua = 0.25 * q[i] * kz * (2.0 * az * az - r2) + 0.5 * (q[i] * B * wr - m * wr * wr) * r2 +
                     0.25 * q[i] * kz * delta * (xr * xr - yr * yr);
            }
            {
                const double xr = c * bx - s * by, yr = s * bx + c * by, r2 = bx * bx + by * by;
                ub = 0.25 * q[i] * kz * (2.0 * bz * bz - r2) + 0.5 * (q[i] * B * wr - m * wr * wr) * r2 +
                     0.25 * q[i] * kz * delta * (xr * xr - yr * yr);
            }
            /* Coulomb part, j in index order */
            double sum = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                const double dbx = bx - x[j], dby = by - y[j], dbz = bz - z[j];
                const double dax = ax - x[j], day = ay - y[j], daz = az - z[j];
                sum += q[j] * (1.0 / sqrt(dbx * dbx + dby * dby + dbz * dbz) -
                               1.0 / sqrt(dax * dax + day * day + daz * daz));
            }
            const double dE = (ub - ua) + ke * q[i] * sum;
            if (dE < 0.0 || u < orc_exp(-dE / (kb * temp))) {
                x[i] = bx;
                y[i] = by;
                z[i] = bz;
                ++acc;
                de_sum += dE;
            }
        }
    }
    out[0] = (double)acc;
    out[1] = de_sum;
}
