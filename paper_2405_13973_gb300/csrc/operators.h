// operators.h -- host construction of the FMM translation operators as dense
// real (p+1)^2 x (p+1)^2 matrices in the normalised storage of
// harmonics.cuh.  Built once per plan in FP64.
//
// With the conventions of harmonics.cuh (addition theorems verified
// numerically when this code was written) and cell-size scaling (cell side s
// at the level of the expansion, M~ = M / s^n, L~ = L s^{n+1}), the
// translations are level independent:
//   M2M (child -> parent, Sec. 2.3.2 upward pass), d = (c_child - c_parent)/S:
//        M'_n^m = sum_{j,k} 2^{-j} M_j^k conj(Y_{n-j}^{m-k}(d))
//   M2L (Eq. FMM_local), o = (c_target - c_source)/s, an integer vector:
//        L_l^h = (-1)^l sum_{j,k} M_j^k Th_{j+l}^{k+h}(o)
//   L2L (parent -> child, downward pass), d = (c_child - c_parent)/S:
//        L'_a^b = 2^{-(a+1)} sum_{l>=a,h} L_l^h conj(Y_{l-a}^{h-b}(d))
// All sums are truncated at order p.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace pt {
namespace ops {

using cd = std::complex<double>;

struct Harm {
    int nmax = 0;
    std::vector<cd> v;  // [n][m], m = 0..n
    cd get(int n, int m) const {
        if (n < 0 || n > nmax || m > n || -m > n) return cd(0, 0);
        if (m < 0) return ((-m) & 1 ? -1.0 : 1.0) * std::conj(v[n * (nmax + 1) - m]);
        return v[n * (nmax + 1) + m];
    }
};

inline Harm regular(int nmax, double x, double y, double z) {
    Harm h;
    h.nmax = nmax;
    h.v.assign((size_t)(nmax + 1) * (nmax + 1), cd(0, 0));
    auto at = [&](int n, int m) -> cd& { return h.v[n * (nmax + 1) + m]; };
    cd w(x, y);
    double r2 = x * x + y * y + z * z;
    at(0, 0) = 1.0;
    for (int m = 0; m <= nmax; ++m) {
        if (m > 0) at(m, m) = at(m - 1, m - 1) * w / (2.0 * m);
        if (m + 1 <= nmax) at(m + 1, m) = z * at(m, m);
        for (int n = m + 2; n <= nmax; ++n)
            at(n, m) = ((2.0 * n - 1.0) * z * at(n - 1, m) - r2 * at(n - 2, m)) /
                       ((double)(n + m) * (double)(n - m));
    }
    return h;
}

inline Harm irregular(int nmax, double x, double y, double z) {
    Harm h;
    h.nmax = nmax;
    h.v.assign((size_t)(nmax + 1) * (nmax + 1), cd(0, 0));
    auto at = [&](int n, int m) -> cd& { return h.v[n * (nmax + 1) + m]; };
    cd w(x, y);
    double r2 = x * x + y * y + z * z, ir2 = 1.0 / r2;
    at(0, 0) = std::sqrt(ir2);
    for (int m = 0; m <= nmax; ++m) {
        if (m > 0) at(m, m) = at(m - 1, m - 1) * (2.0 * m - 1.0) * w * ir2;
        if (m + 1 <= nmax) at(m + 1, m) = (2.0 * m + 1.0) * z * ir2 * at(m, m);
        for (int n = m + 2; n <= nmax; ++n)
            at(n, m) = ((2.0 * n - 1.0) * z * at(n - 1, m) -
                        ((double)(n - 1) * (n - 1) - (double)m * m) * at(n - 2, m)) * ir2;
    }
    return h;
}

inline double norm_s(int n, int m) {  // sqrt((n+m)!(n-m)!)
    return std::exp(0.5 * (std::lgamma(n + m + 1.0) + std::lgamma(n - m + 1.0)));
}

// Assemble the real matrix (row-major out x in) of a complex-linear map given
// coef(n_out, m_out >= 0, n_in, k_in signed).  kind_out/kind_in: 0 = M-type
// (stored M^ = s M), 1 = L-type (stored L^ = L / s).
template <class Coef>
inline void assemble(int p, Coef coef, int kind_out, int kind_in, double* T) {
    const int P = (p + 1) * (p + 1);
    for (int i = 0; i < P * P; ++i) T[i] = 0.0;
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m)
            for (int j = 0; j <= p; ++j)
                for (int k = 0; k <= j; ++k) {
                    cd A = coef(n, m, j, k);
                    cd B = (k > 0) ? coef(n, m, j, -k) * ((k & 1) ? -1.0 : 1.0) : cd(0, 0);
                    cd S = A + B, D = A - B;
                    double so = norm_s(n, m), si = norm_s(j, k);
                    double sc = (kind_out == 0 ? so : 1.0 / so) / (kind_in == 0 ? si : 1.0 / si);
                    int ro = n * n + (m == 0 ? 0 : 2 * m - 1);
                    int ri = j * j + (k == 0 ? 0 : 2 * k - 1);
                    T[ro * P + ri] += sc * S.real();
                    if (k > 0) T[ro * P + ri + 1] += sc * (-D.imag());
                    if (m > 0) {
                        T[(ro + 1) * P + ri] += sc * S.imag();
                        if (k > 0) T[(ro + 1) * P + ri + 1] += sc * D.real();
                    }
                }
}

// Octant o = 4 bx + 2 by + bz (Morton order of the children); child centre
// offset from the parent centre in parent units: (b - 1/2)/2 per axis.
inline void child_offset(int o, double d[3]) {
    int b[3] = {(o >> 2) & 1, (o >> 1) & 1, o & 1};
    for (int a = 0; a < 3; ++a) d[a] = (b[a] - 0.5) * 0.5;
}

inline void build_m2m(int p, int o, double* T) {
    double d[3];
    child_offset(o, d);
    Harm Y = regular(p, d[0], d[1], d[2]);
    assemble(p,
             [&](int n, int m, int j, int k) -> cd {
                 if (j > n) return cd(0, 0);
                 return std::ldexp(1.0, -j) * std::conj(Y.get(n - j, m - k));
             },
             0, 0, T);
}

inline void build_l2l(int p, int o, double* T) {
    double d[3];
    child_offset(o, d);
    Harm Y = regular(p, d[0], d[1], d[2]);
    assemble(p,
             [&](int a, int b, int l, int h) -> cd {
                 if (l < a) return cd(0, 0);
                 return std::ldexp(1.0, -(a + 1)) * std::conj(Y.get(l - a, h - b));
             },
             1, 1, T);
}

inline void build_m2l(int p, int ox, int oy, int oz, double* T) {
    Harm Th = irregular(2 * p, (double)ox, (double)oy, (double)oz);
    assemble(p,
             [&](int l, int h, int j, int k) -> cd {
                 return ((l & 1) ? -1.0 : 1.0) * Th.get(j + l, k + h);
             },
             1, 0, T);
}

}  // namespace ops
}  // namespace pt

// ---------------------------------------------------------------------------
// Rotation-based M2L ("point and shoot", the O(p^3) alternative to the dense
// O(p^4) translation): with Q a rotation taking the offset direction o/|o| to
// +z, R^M(Q) and R^L(Q) the (degree-block-diagonal) maps of stored multipole
// and local coefficients under Q, and T_z(d) the M2L along +z by d = |o|:
//        T_o = R^L(Q)^{-1} T_z(|o|) R^M(Q) = R^L(Q^T) T_z(|o|) R^M(Q),
// because the M2L map commutes with rotating the whole configuration.  T_z
// couples only equal orders m (Re to Re and Im to Im), so one translation
// costs sum_n (2n+1)^2 twice plus sum_m (p+1-m)^2 (x 2 for m > 0)
// multiply-adds instead of (p+1)^4.
namespace pt {
namespace ops {

// Q (row-major 3 x 3) with Q (v/|v|) = +z (Rodrigues' formula about v x z).
inline void rotation_to_z(double vx, double vy, double vz, double Q[9]) {
    const double r = std::sqrt(vx * vx + vy * vy + vz * vz);
    const double x = vx / r, y = vy / r, z = vz / r;
    // axis a = v x z = (y, -x, 0), sin = |a|, cos = z
    const double ax = y, ay = -x, s2 = ax * ax + ay * ay;
    for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? 1.0 : 0.0;
    if (s2 < 1e-28) {
        if (z < 0) {  // v = -z: half turn about x
            Q[4] = -1.0;
            Q[8] = -1.0;
        }
        return;
    }
    const double c = z, k = (1.0 - c) / s2;
    // Q = I + [a]x + k [a]x^2, [a]x = [[0, 0, ay], [0, 0, -ax], [-ay, ax, 0]]
    const double A[9] = {0, 0, ay, 0, 0, -ax, -ay, ax, 0};
    double A2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double t = 0;
            for (int l = 0; l < 3; ++l) t += A[3 * i + l] * A[3 * l + j];
            A2[3 * i + j] = t;
        }
    for (int i = 0; i < 9; ++i) Q[i] += A[i] + k * A2[i];
}

// stored coefficients of degree n (2n+1 reals: Re m=0, then Re/Im for
// m = 1..n) of a unit charge at u: multipole M^ = s conj(Y(u)), or local
// L^ = Th(u) / s
inline void degree_coeffs(int n, bool local, const double u[3], double* out) {
    if (local) {
        Harm T = irregular(n, u[0], u[1], u[2]);
        for (int m = 0; m <= n; ++m) {
            const cd v = T.get(n, m) / norm_s(n, m);
            if (m == 0) {
                out[0] = v.real();
            } else {
                out[2 * m - 1] = v.real();
                out[2 * m] = v.imag();
            }
        }
    } else {
        Harm Y = regular(n, u[0], u[1], u[2]);
        for (int m = 0; m <= n; ++m) {
            const cd v = std::conj(Y.get(n, m)) * norm_s(n, m);
            if (m == 0) {
                out[0] = v.real();
            } else {
                out[2 * m - 1] = v.real();
                out[2 * m] = v.imag();
            }
        }
    }
}

// Solve G X = B in place (G k x k, B k x r; Gaussian elimination with
// partial pivoting); false if G is singular.
inline bool solve_dense(int k, int r, double* G, double* B) {
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int i = c + 1; i < k; ++i)
            if (std::fabs(G[i * k + c]) > std::fabs(G[piv * k + c])) piv = i;
        if (std::fabs(G[piv * k + c]) < 1e-300) return false;
        if (piv != c) {
            for (int j = 0; j < k; ++j) std::swap(G[c * k + j], G[piv * k + j]);
            for (int j = 0; j < r; ++j) std::swap(B[c * r + j], B[piv * r + j]);
        }
        for (int i = c + 1; i < k; ++i) {
            const double f = G[i * k + c] / G[c * k + c];
            if (f == 0.0) continue;
            for (int j = c; j < k; ++j) G[i * k + j] -= f * G[c * k + j];
            for (int j = 0; j < r; ++j) B[i * r + j] -= f * B[c * r + j];
        }
    }
    for (int c = k - 1; c >= 0; --c) {
        for (int j = 0; j < r; ++j) {
            double t = B[c * r + j];
            for (int i = c + 1; i < k; ++i) t -= G[c * k + i] * B[i * r + j];
            B[c * r + j] = t / G[c * k + c];
        }
    }
    return true;
}

// R (degree blocks, row-major, packed n = 0..p: block n at n (4n^2 - 1) / 3)
// with coeffs(Q u) = R coeffs(u) for every u, fitted by least squares on
// 3 (2n + 1) points spread over the unit sphere (exact up to rounding: the
// coefficients of degree n of a rotated point are a linear map of those of
// the point).
inline bool rotation_blocks(int p, const double Q[9], bool local, double* R) {
    for (int n = 0; n <= p; ++n) {
        const int k = 2 * n + 1, K = 3 * k;
        std::vector<double> X((size_t)k * K), Y((size_t)k * K), cu(k), cq(k);
        for (int s = 0; s < K; ++s) {
            // Fibonacci sphere point s of K, slightly off the poles
            const double zz = 1.0 - (2.0 * s + 1.0) / K;
            const double rr = std::sqrt(std::max(0.0, 1.0 - zz * zz));
            const double ph = 2.399963229728653 * s + 0.3;
            const double u[3] = {rr * std::cos(ph), rr * std::sin(ph), zz};
            const double qu[3] = {Q[0] * u[0] + Q[1] * u[1] + Q[2] * u[2],
                                  Q[3] * u[0] + Q[4] * u[1] + Q[5] * u[2],
                                  Q[6] * u[0] + Q[7] * u[1] + Q[8] * u[2]};
            degree_coeffs(n, local, u, cu.data());
            degree_coeffs(n, local, qu, cq.data());
            for (int i = 0; i < k; ++i) {
                X[(size_t)i * K + s] = cu[i];
                Y[(size_t)i * K + s] = cq[i];
            }
        }
        // R X = Y in least squares: (X X^T) R^T = X Y^T
        std::vector<double> G((size_t)k * k, 0.0), B((size_t)k * k, 0.0);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                double g = 0, b = 0;
                for (int s = 0; s < K; ++s) {
                    g += X[(size_t)i * K + s] * X[(size_t)j * K + s];
                    b += X[(size_t)i * K + s] * Y[(size_t)j * K + s];
                }
                G[(size_t)i * k + j] = g;
                B[(size_t)i * k + j] = b;
            }
        if (!solve_dense(k, k, G.data(), B.data())) return false;  // B = R^T
        double* blk = R + (size_t)n * (4 * n * n - 1) / 3;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) blk[(size_t)i * k + j] = B[(size_t)j * k + i];
    }
    return true;
}

// Sizes of the packed rotation-M2L operator of one offset.
inline int rot_block_vals(int p) { return (p + 1) * (4 * (p + 1) * (p + 1) - 1) / 3; }
inline int rot_z_vals(int p) {
    int t = 0;
    for (int m = 0; m <= p; ++m) t += (p + 1 - m) * (p + 1 - m);
    return t;
}
inline int rot_op_vals(int p) { return 2 * rot_block_vals(p) + 2 * rot_z_vals(p); }

// Packed rotation-M2L operator of offset o: [R^M(Q) | R^L(Q^T) | Z_re | Z_im],
// Z_re (Z_im) the Re -> Re (Im -> Im) coupling of T_z(|o|) per order m,
// rows l = m..p, columns j = m..p, orders in turn.  False if a fit failed or
// T_z couples anything else.
inline bool build_m2l_rotation(int p, int ox, int oy, int oz, double* out) {
    const int P = (p + 1) * (p + 1);
    double Q[9], Qt[9];
    rotation_to_z(ox, oy, oz, Q);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Qt[3 * i + j] = Q[3 * j + i];
    const int nb = rot_block_vals(p), nz = rot_z_vals(p);
    if (!rotation_blocks(p, Q, false, out)) return false;
    if (!rotation_blocks(p, Qt, true, out + nb)) return false;
    const double d = std::sqrt((double)(ox * ox + oy * oy + oz * oz));
    Harm Th = irregular(2 * p, 0.0, 0.0, d);
    std::vector<double> Tz((size_t)P * P);
    assemble(p,
             [&](int l, int h, int j, int k) -> cd {
                 return ((l & 1) ? -1.0 : 1.0) * Th.get(j + l, k + h);
             },
             1, 0, Tz.data());
    double* zr = out + 2 * nb;
    double* zi = zr + nz;
    double big = 0;
    for (double v : Tz) big = std::max(big, std::fabs(v));
    std::vector<char> used((size_t)P * P, 0);
    int o = 0;
    for (int m = 0; m <= p; ++m)
        for (int l = m; l <= p; ++l)
            for (int j = m; j <= p; ++j, ++o) {
                const int ro = l * l + (m == 0 ? 0 : 2 * m - 1), ri = j * j + (m == 0 ? 0 : 2 * m - 1);
                zr[o] = Tz[(size_t)ro * P + ri];
                used[(size_t)ro * P + ri] = 1;
                zi[o] = 0.0;
                if (m > 0) {
                    zi[o] = Tz[(size_t)(ro + 1) * P + ri + 1];
                    used[(size_t)(ro + 1) * P + ri + 1] = 1;
                }
            }
    for (size_t i = 0; i < Tz.size(); ++i)
        if (!used[i] && std::fabs(Tz[i]) > 1e-13 * big) return false;
    return true;
}

}  // namespace ops
}  // namespace pt
