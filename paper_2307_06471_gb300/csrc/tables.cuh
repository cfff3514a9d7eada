// Compile-time Legendre bases and Gauss--Legendre rules on the reference cell.
//
// The DG space V_h (Sec. 2.1) holds P^k or Q^k polynomials per cell; the
// modal basis on [-1,1]^d is P_i(xi) P_j(eta).  Everything here is constexpr:
// after full unrolling of the kernels' mode and point loops every table entry
// is an immediate, so zero entries (e.g. d/dxi of a mode with i = 0) vanish
// from the generated code.  Gauss nodes and weights are the closed forms for
// n <= 4; square roots are evaluated by a constexpr Newton iteration.
#pragma once

namespace crk {

constexpr double csqrt(double x) {
    if (x <= 0.0) return 0.0;
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 200; ++i) r = 0.5 * (r + x / r);
    return r;
}

struct GaussRule {
    double x[4];
    double w[4];
};

// n-point Gauss--Legendre rule on [-1, 1], ascending nodes, 1 <= n <= 4
constexpr GaussRule gauss_rule(int n) {
    GaussRule g{};
    if (n == 1) {
        g.x[0] = 0.0; g.w[0] = 2.0;
    } else if (n == 2) {
        const double a = 1.0 / csqrt(3.0);
        g.x[0] = -a; g.x[1] = a; g.w[0] = 1.0; g.w[1] = 1.0;
    } else if (n == 3) {
        const double a = csqrt(0.6);
        g.x[0] = -a; g.x[1] = 0.0; g.x[2] = a;
        g.w[0] = 5.0 / 9.0; g.w[1] = 8.0 / 9.0; g.w[2] = 5.0 / 9.0;
    } else {
        const double r = csqrt(6.0 / 5.0);
        const double a = csqrt(3.0 / 7.0 - 2.0 / 7.0 * r);
        const double b = csqrt(3.0 / 7.0 + 2.0 / 7.0 * r);
        const double wa = (18.0 + csqrt(30.0)) / 36.0;
        const double wb = (18.0 - csqrt(30.0)) / 36.0;
        g.x[0] = -b; g.x[1] = -a; g.x[2] = a; g.x[3] = b;
        g.w[0] = wb; g.w[1] = wa; g.w[2] = wa; g.w[3] = wb;
    }
    return g;
}

// Legendre P_n(x) by the three-term recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}
constexpr double legP(int n, double x) {
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// P_n'(x) = sum over k = n-1, n-3, ... >= 0 of (2k+1) P_k(x)
constexpr double legdP(int n, double x) {
    double s = 0.0;
    for (int k = n - 1; k >= 0; k -= 2) s += (2.0 * k + 1.0) * legP(k, x);
    return s;
}

constexpr int n_modes_2d(int K, int B) { return B == 0 ? (K + 1) * (K + 2) / 2 : (K + 1) * (K + 1); }

// (i, j) of mode m: by total degree ascending, within a degree i descending;
// P (B = 0): i + j <= K; Q (B = 1): i, j <= K.
constexpr void mode_ij(int K, int B, int m, int& mi, int& mj) {
    int c = 0;
    const int dmax = B == 0 ? K : 2 * K;
    for (int d = 0; d <= dmax; ++d)
        for (int i = d; i >= 0; --i) {
            const int j = d - i;
            if (i <= K && j <= K) {
                if (c == m) { mi = i; mj = j; return; }
                ++c;
            }
        }
    mi = 0; mj = 0;
}

// 2D tables for P^K / Q^K with the (K+1)-point rule per direction.
// Volume point q = a*NQ + b sits at (xi_a, eta_b); face point p of the E/W
// faces sits at eta_p, of the N/S faces at xi_p.
template <int K, int B>
struct Tab2D {
    static constexpr int NQ = K + 1;
    static constexpr int NQV = NQ * NQ;
    static constexpr int NM = n_modes_2d(K, B);
    double phi[NQV][NM];   // phi_m(q)
    double gx[NQV][NM];    // w_q dphi_m/dxi (q)
    double gy[NQV][NM];    // w_q dphi_m/deta (q)
    double tE[NQ][NM], tW[NQ][NM], tN[NQ][NM], tS[NQ][NM];   // phi_m at face points
    double pE[NQ][NM], pW[NQ][NM], pN[NQ][NM], pS[NQ][NM];   // w_p phi_m at face points
    double sN[NM];         // sum_p pN[p][m] = int phi_m(xi, 1) dxi = 2 if i = 0, else 0 (exact rule)
    int ip[NM], jp[NM];    // parities of i and j: phi_m(-1, eta) = (-1)^i phi_m(1, eta), likewise in eta
    double cm[NM];         // (2i+1)(2j+1)/2 = inverse mass / (2|K|) factor
    double pw[NQV][NM];    // projection weights 1/4 w_q phi_m(q) / mass_m
    double xq[NQ];         // Gauss nodes
};

template <int K, int B>
constexpr Tab2D<K, B> make_tab2d() {
    Tab2D<K, B> t{};
    constexpr int NQ = K + 1;
    const GaussRule g = gauss_rule(NQ);
    for (int a = 0; a < NQ; ++a) t.xq[a] = g.x[a];
    for (int m = 0; m < Tab2D<K, B>::NM; ++m) {
        int i = 0, j = 0;
        mode_ij(K, B, m, i, j);
        const double mass = 1.0 / ((2.0 * i + 1.0) * (2.0 * j + 1.0));
        t.cm[m] = 0.5 / mass;
        t.sN[m] = i == 0 ? 2.0 : 0.0;
        t.ip[m] = i & 1;
        t.jp[m] = j & 1;
        for (int a = 0; a < NQ; ++a)
            for (int b = 0; b < NQ; ++b) {
                const int q = a * NQ + b;
                const double xi = g.x[a], eta = g.x[b], wq = g.w[a] * g.w[b];
                t.phi[q][m] = legP(i, xi) * legP(j, eta);
                t.gx[q][m] = wq * legdP(i, xi) * legP(j, eta);
                t.gy[q][m] = wq * legP(i, xi) * legdP(j, eta);
                t.pw[q][m] = 0.25 * wq * legP(i, xi) * legP(j, eta) / mass;
            }
        for (int p = 0; p < NQ; ++p) {
            const double s = g.x[p], w = g.w[p];
            t.tE[p][m] = legP(i, 1.0) * legP(j, s);
            t.tW[p][m] = legP(i, -1.0) * legP(j, s);
            t.tN[p][m] = legP(i, s) * legP(j, 1.0);
            t.tS[p][m] = legP(i, s) * legP(j, -1.0);
            t.pE[p][m] = w * t.tE[p][m];
            t.pW[p][m] = w * t.tW[p][m];
            t.pN[p][m] = w * t.tN[p][m];
            t.pS[p][m] = w * t.tS[p][m];
        }
    }
    return t;
}

// 1D tables for P^K with the (K+1)-point rule.
template <int K>
struct Tab1D {
    static constexpr int NQ = K + 1;
    static constexpr int NM = K + 1;
    double phi[NQ][NM];
    double g[NQ][NM];      // w_q P_m'(xi_q)
    double tR[NM], tL[NM]; // P_m(+1), P_m(-1)
    double cm[NM];         // (2m+1)
    double pw[NQ][NM];     // (2m+1)/2 w_q P_m(xi_q)
    double xq[NQ];
};

template <int K>
constexpr Tab1D<K> make_tab1d() {
    Tab1D<K> t{};
    const GaussRule g = gauss_rule(K + 1);
    for (int a = 0; a <= K; ++a) t.xq[a] = g.x[a];
    for (int m = 0; m <= K; ++m) {
        t.tR[m] = legP(m, 1.0);
        t.tL[m] = legP(m, -1.0);
        t.cm[m] = 2.0 * m + 1.0;
        for (int q = 0; q <= K; ++q) {
            t.phi[q][m] = legP(m, g.x[q]);
            t.g[q][m] = g.w[q] * legdP(m, g.x[q]);
            t.pw[q][m] = 0.5 * (2.0 * m + 1.0) * g.w[q] * legP(m, g.x[q]);
        }
    }
    return t;
}

}  // namespace crk
