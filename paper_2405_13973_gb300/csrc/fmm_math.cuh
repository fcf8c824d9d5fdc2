// fmm_math.cuh -- per-ion P2M and L2P in the normalised real storage of
// harmonics.cuh (host and device).
//
// P2M (Eq. FMM_coul2): M^_n^m += q conj(Y^_n^m(u)), u = (x - c)/s.
// L2P (Sec. 2.3.2 downward pass, "the potential at the location of each ion
// is then easily computed"): phi~ = sum L^_n^m conj(Y^_n^m(u)) and its
// gradient from the order-1 local expansion shifted to u:
//   d/dz         = sum_{n,m} w_m Re(L_{n+1}^m conj(Y_n^m))
//   d/dx + i d/dy = sum_{n,m} [L_{n+1}^{m+1} conj(Y_n^m) - conj(L_{n+1}^{m-1}) Y_n^m]
// (w_0 = 1, w_m = 2; the second bracket term only for m >= 1), each term
// carrying the ratio of normalisations s_{n+1,m'} / s_{n,m}.
#pragma once
#include "harmonics.cuh"

namespace pt {

// Visit Y^_n^m(u) for m = 0..p, n = m..p in column order; fn(n, m, re, im).
template <typename T, class Fn>
PT_HD void for_each_ups(int p, T x, T y, T z, const HarmTables<T>& t, Fn fn) {
    T r2 = x * x + y * y + z * z;
    T dre = 1, dim = 0;  // Y^_m^m
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            T nre = (dre * x - dim * y) * t.c[m];
            T nim = (dre * y + dim * x) * t.c[m];
            dre = nre;
            dim = nim;
        }
        fn(m, m, dre, dim);
        if (m + 1 > p) break;
        T p2re = dre, p2im = dim;
        T p1re = z * t.d[m] * dre, p1im = z * t.d[m] * dim;
        fn(m + 1, m, p1re, p1im);
        for (int n = m + 2; n <= p; ++n) {
            T a = t.a[n][m] * z, b = t.b[n][m] * r2;
            T cre = a * p1re - b * p2re;
            T cim = a * p1im - b * p2im;
            fn(n, m, cre, cim);
            p2re = p1re;
            p2im = p1im;
            p1re = cre;
            p1im = cim;
        }
    }
}

// As for_each_ups, but the columns m = m0, m0 + mstep, ... only (the diagonal
// Y^_m^m is still carried through every m): lets several threads share one
// point's harmonics, each taking every mstep-th column.
template <typename T, typename Fn>
PT_HD void for_each_ups_cols(int p, T x, T y, T z, const HarmTables<T>& t, int m0, int mstep,
                             Fn fn) {
    T r2 = x * x + y * y + z * z;
    T dre = 1, dim = 0;  // Y^_m^m
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            T nre = (dre * x - dim * y) * t.c[m];
            T nim = (dre * y + dim * x) * t.c[m];
            dre = nre;
            dim = nim;
        }
        if (m < m0 || (m - m0) % mstep != 0) continue;
        fn(m, m, dre, dim);
        if (m + 1 > p) continue;
        T p2re = dre, p2im = dim;
        T p1re = z * t.d[m] * dre, p1im = z * t.d[m] * dim;
        fn(m + 1, m, p1re, p1im);
        for (int n = m + 2; n <= p; ++n) {
            T a = t.a[n][m] * z, b = t.b[n][m] * r2;
            T cre = a * p1re - b * p2re;
            T cim = a * p1im - b * p2im;
            fn(n, m, cre, cim);
            p2re = p1re;
            p2im = p1im;
            p1re = cre;
            p1im = cim;
        }
    }
}

// L2P over the columns m0, m0 + mstep, ... of the local expansion (see
// for_each_ups_cols); summing the mstep parts gives the whole L2P (Eq. L2P):
// the potential and the gradient of the local expansion at (x, y, z).
template <typename T>
PT_HD void l2p_eval_cols(int p, const T* Lh, T x, T y, T z, const HarmTables<T>& t, int m0,
                         int mstep, T& phi, T& gx, T& gy, T& gz) {
    T ph = 0, ax = 0, ay = 0, az = 0;
    for_each_ups_cols(p, x, y, z, t, m0, mstep, [&](int n, int m, T yr, T yi) {
        int k = re_idx(n, m);
        T lr = Lh[k], li = m > 0 ? Lh[k + 1] : T(0);
        T w = m > 0 ? T(2) : T(1);
        ph += w * (lr * yr + li * yi);
        if (n + 1 <= p) {
            int k1 = re_idx(n + 1, m);
            T l1r = Lh[k1], l1i = m > 0 ? Lh[k1 + 1] : T(0);
            az += w * t.e[n][m] * (l1r * yr + l1i * yi);
            int k2 = re_idx(n + 1, m + 1);
            T l2r = Lh[k2], l2i = Lh[k2 + 1];
            ax += t.f[n][m] * (l2r * yr + l2i * yi);
            ay += t.f[n][m] * (l2i * yr - l2r * yi);
            if (m >= 1) {
                int k3 = re_idx(n + 1, m - 1);
                T l3r = Lh[k3], l3i = (m - 1) > 0 ? Lh[k3 + 1] : T(0);
                ax -= t.g[n][m] * (l3r * yr + l3i * yi);
                ay -= t.g[n][m] * (l3r * yi - l3i * yr);
            }
        }
    });
    phi = ph;
    gx = ax;
    gy = ay;
    gz = az;
}

}  // namespace pt
