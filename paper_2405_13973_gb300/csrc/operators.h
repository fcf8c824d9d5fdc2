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
