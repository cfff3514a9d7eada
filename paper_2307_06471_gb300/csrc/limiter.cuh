// TVB-minmod limiter in characteristic fields on Cartesian cells (Sec. 4.2,
// Remark 2.2; the limiter of Cockburn and Shu for multidimensional systems,
// which the paper cites without printing it).  Reading implemented:
//   per direction (x: slope mode (1,0), neighbours E/W, mesh size dx;
//                  y: slope mode (0,1), neighbours N/S, mesh size dy):
//     a1 = slope coefficient, a2 = ubar_E - ubar, a3 = ubar - ubar_W,
//     projected on characteristic fields with L = R^{-1} at the cell average
//     (scalar problems: no projection);
//     mt = a1 if |a1| <= M h^2 else minmod(a1, a2, a3)
//   troubled if mt != a1 in any field of either direction; then the slope
//   modes become R mt, every other non-constant mode becomes 0, and the
//   average is kept.
#pragma once
#include "common.cuh"

// 1: the two directions' characteristic projections as packed FP32x2 FMAs
#ifndef CRK_LIM_PACKED
#define CRK_LIM_PACKED 1
#endif

namespace crk {

template <class T>
__device__ __forceinline__ T minmod3(T a, T b, T c) {
    const bool pos = a > T(0) && b > T(0) && c > T(0);
    const bool neg = a < T(0) && b < T(0) && c < T(0);
    T m = fabs(a);
    m = fabs(b) < m ? fabs(b) : m;
    m = fabs(c) < m ? fabs(c) : m;
    return pos ? m : (neg ? -m : T(0));
}

template <class T>
__device__ __forceinline__ T tvb_minmod(T a1, T a2, T a3, T Mh2) {
    return fabs(a1) <= Mh2 ? a1 : minmod3(a1, a2, a3);
}

// a0 = fma(x0, y0, a0), a1 = fma(x1, y1, a1): one packed FP32x2 FMA for an
// FP32 pair (each lane rounds like the scalar FMA)
template <class T>
__device__ __forceinline__ void fma_pair(T& a0, T& a1, T x0, T x1, T y0, T y1) {
    if constexpr (sizeof(T) == 4) {
        const float2 r = __ffma2_rn(make_float2(x0, x1), make_float2(y0, y1), make_float2(a0, a1));
        a0 = r.x;
        a1 = r.y;
    } else {
        a0 = fma(x0, y0, a0);
        a1 = fma(x1, y1, a1);
    }
}

// The scalars both directions' eigenvectors share at one state: velocity,
// |vel|^2, sound speed and its inverse, (gamma-1)/c^2 and its kinetic
// multiple, total enthalpy -- one reciprocal of rho, one square root, one
// reciprocal of c per cell for x and y together.
template <class T>
struct EulerEig {
    T w, v, q2, c, ic, b1, b2, H;
};

template <class T>
__device__ __forceinline__ EulerEig<T> euler_eig_scalars(const T* u, T gamma) {
    EulerEig<T> e;
    const T gm1 = gamma - T(1);
    const T ir = T(1) / u[0];
    e.w = u[1] * ir;
    e.v = u[2] * ir;
    e.q2 = e.w * e.w + e.v * e.v;
    const T p = gm1 * (u[3] - T(0.5) * u[0] * e.q2);
    const T c2 = gamma * p * ir;
    e.c = sqrt(c2 > T(0) ? c2 : T(0));
    e.ic = T(1) / e.c;
    e.b1 = gm1 * e.ic * e.ic;
    e.b2 = T(0.5) * e.b1 * e.q2;
    e.H = (u[3] + p) * ir;
    return e;
}

// rows of R^{-1} along AXIS (left eigenvectors) from the shared scalars
template <class T, int AXIS>
__device__ __forceinline__ void euler_left_of(const EulerEig<T>& e, T L[4][4]) {
    const T vn = AXIS == 0 ? e.w : e.v;
    const T vt = AXIS == 0 ? e.v : e.w;
    const int in = 1 + AXIS, it = 2 - AXIS;
    L[0][0] = T(0.5) * (e.b2 + vn * e.ic);
    L[0][in] = -T(0.5) * (e.b1 * vn + e.ic);
    L[0][it] = -T(0.5) * e.b1 * vt;
    L[0][3] = T(0.5) * e.b1;
    L[1][0] = T(1) - e.b2;
    L[1][in] = e.b1 * vn;
    L[1][it] = e.b1 * vt;
    L[1][3] = -e.b1;
    L[2][0] = -vt;
    L[2][in] = T(0);
    L[2][it] = T(1);
    L[2][3] = T(0);
    L[3][0] = T(0.5) * (e.b2 - vn * e.ic);
    L[3][in] = -T(0.5) * (e.b1 * vn - e.ic);
    L[3][it] = -T(0.5) * e.b1 * vt;
    L[3][3] = T(0.5) * e.b1;
}

// columns = right eigenvectors along AXIS, for the eigenvalues (vn - c, vn, vn, vn + c)
template <class T, int AXIS>
__device__ __forceinline__ void euler_right_of(const EulerEig<T>& e, T R[4][4]) {
    const T vn = AXIS == 0 ? e.w : e.v;
    const T vt = AXIS == 0 ? e.v : e.w;
    const int in = 1 + AXIS, it = 2 - AXIS;
    R[0][0] = T(1); R[0][1] = T(1); R[0][2] = T(0); R[0][3] = T(1);
    R[in][0] = vn - e.c; R[in][1] = vn; R[in][2] = T(0); R[in][3] = vn + e.c;
    R[it][0] = vt; R[it][1] = vt; R[it][2] = T(1); R[it][3] = vt;
    R[3][0] = e.H - vn * e.c; R[3][1] = T(0.5) * e.q2; R[3][2] = vt; R[3][3] = e.H + vn * e.c;
}

// Limit one cell in place.  u[v][m] modal coefficients, nb* neighbour
// averages.  Returns true if the cell was troubled.
// mode -1: the TVB test decides; 0: leave the cell; 1: limit it (slopes
// become the modified-minmod values, higher modes 0) -- modes 0 and 1 carry
// the decision of a learned indicator.
template <class T, int NV, int NM>
__device__ __forceinline__ bool tvb_limit_cell(T (&u)[NV][NM], const T* nbW, const T* nbE, const T* nbS,
                                               const T* nbN, T Mdx2, T Mdy2, T gamma, int mode = -1) {
    if (NM < 3) return false;
    T avg[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) avg[v] = u[v][0];
    T mx[NV], my[NV];
    bool flag = false;
    if (NV == 4) {
        T L[4][4], mxc[4], myc[4];
        const EulerEig<T> eg = euler_eig_scalars<T>(avg, gamma);
#if CRK_LIM_PACKED
        // both directions' characteristic values at once, x in the first
        // lane of each pair and y in the second, each sum in the order of v
        T Ly[4][4];
        euler_left_of<T, 0>(eg, L);
        euler_left_of<T, 1>(eg, Ly);
        T dE[4], dW[4], dN[4], dS[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            dE[v] = nbE[v] - avg[v];
            dN[v] = nbN[v] - avg[v];
            dW[v] = avg[v] - nbW[v];
            dS[v] = avg[v] - nbS[v];
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            T x1 = 0, y1 = 0, x2 = 0, y2 = 0, x3 = 0, y3 = 0;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                fma_pair(x1, y1, L[f][v], Ly[f][v], u[v][1], u[v][2]);
                fma_pair(x2, y2, L[f][v], Ly[f][v], dE[v], dN[v]);
                fma_pair(x3, y3, L[f][v], Ly[f][v], dW[v], dS[v]);
            }
            mxc[f] = tvb_minmod(x1, x2, x3, Mdx2);
            myc[f] = tvb_minmod(y1, y2, y3, Mdy2);
            flag |= (mxc[f] != x1) || (myc[f] != y1);
        }
#else
        // x direction: characteristic values and the modified minmod
        euler_left_of<T, 0>(eg, L);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            T s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                s1 += L[f][v] * u[v][1];
                s2 += L[f][v] * (nbE[v] - avg[v]);
                s3 += L[f][v] * (avg[v] - nbW[v]);
            }
            mxc[f] = tvb_minmod(s1, s2, s3, Mdx2);
            flag |= (mxc[f] != s1);
        }
        // y direction
        euler_left_of<T, 1>(eg, L);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            T s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                s1 += L[f][v] * u[v][2];
                s2 += L[f][v] * (nbN[v] - avg[v]);
                s3 += L[f][v] * (avg[v] - nbS[v]);
            }
            myc[f] = tvb_minmod(s1, s2, s3, Mdy2);
            flag |= (myc[f] != s1);
        }
#endif
        if (mode >= 0) flag = mode == 1;
        if (flag) {
            // back to conserved variables only for limited cells
            T R[4][4];
            euler_right_of<T, 0>(eg, R);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T s = 0;
#pragma unroll
                for (int f = 0; f < 4; ++f) s += R[v][f] * mxc[f];
                mx[v] = s;
            }
            euler_right_of<T, 1>(eg, R);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T s = 0;
#pragma unroll
                for (int f = 0; f < 4; ++f) s += R[v][f] * myc[f];
                my[v] = s;
            }
        }
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            mx[v] = tvb_minmod(u[v][1], nbE[v] - avg[v], avg[v] - nbW[v], Mdx2);
            my[v] = tvb_minmod(u[v][2], nbN[v] - avg[v], avg[v] - nbS[v], Mdy2);
            flag |= (mx[v] != u[v][1]) || (my[v] != u[v][2]);
        }
    }
    if (mode >= 0) flag = mode == 1;
    if (flag) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            u[v][1] = mx[v];
            u[v][2] = my[v];
#pragma unroll
            for (int m = 3; m < NM; ++m) u[v][m] = T(0);
        }
    }
    return flag;
}

}  // namespace crk

namespace crk {

// Positivity-preserving scaling of Zhang and Shu (J. Comput. Phys. 229,
// 2010) -- an option outside the paper's method, applied after the TVB
// limiter at the same final stage.  Points: the volume Gauss points and the
// Gauss points of the four faces.  Step 1 scales the density's non-constant
// modes so that rho >= eps at every point; step 2 scales every non-constant
// mode by the smallest t in (0, 1] with p(ubar + t (u_q - ubar)) = eps over
// the points where p(u_q) < eps (a quadratic in t after multiplying by rho).
// The cell average is unchanged.  Returns true if the cell was scaled.
template <class T, int NV, int NM, int K, int B>
__device__ __forceinline__ bool positivity_cell(T (&u)[NV][NM], T gamma, T eps) {
    if constexpr (NV != 4 || NM < 2) {
        return false;
    } else {
        constexpr Tab2D<K, B> tb = make_tab2d<K, B>();
        constexpr int NQ = K + 1, NQV = NQ * NQ, NPT = NQV + 4 * NQ;
        auto phi = [&](int q, int m) -> T {
            if (q < NQV) return T(tb.phi[q][m]);
            const int f = (q - NQV) / NQ, p = (q - NQV) % NQ;
            return T(f == 0 ? tb.tE[p][m] : f == 1 ? tb.tW[p][m] : f == 2 ? tb.tN[p][m] : tb.tS[p][m]);
        };
        // Shortcut: |phi_m| <= 1 on the reference cell, so rho >= rho_lo =
        // rhobar - sum |rho_m| and p >= (gamma-1)(E_lo - (Mx^2 + My^2)/(2 rho_lo))
        // at every point.  When both bounds clear eps by a margin far above
        // the rounding of the point values, the scaling below would change
        // nothing: return at once.
        {
            T sr = T(0), se = T(0), sx = T(0), sy = T(0);
#pragma unroll
            for (int m = 1; m < NM; ++m) {
                sr += fabs(u[0][m]);
                sx += fabs(u[1][m]);
                sy += fabs(u[2][m]);
                se += fabs(u[3][m]);
            }
            const T rlo = u[0][0] - sr;
            const T elo = u[3][0] - se;
            const T mx = fabs(u[1][0]) + sx, my = fabs(u[2][0]) + sy;
            const T margin = T(1e-4);
            if (rlo > eps + margin * (fabs(u[0][0]) + sr)) {
                const T plo = (gamma - T(1)) * (elo - (mx * mx + my * my) / (T(2) * rlo));
                if (plo > eps + margin * (gamma - T(1)) * (fabs(u[3][0]) + se)) return false;
            }
        }
        bool changed = false;
        // step 1: density
        const T rbar = u[0][0];
        T rmin = rbar;
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            T r = T(0);
#pragma unroll
            for (int m = 0; m < NM; ++m) r += u[0][m] * phi(q, m);
            rmin = r < rmin ? r : rmin;
        }
        if (rmin < eps) {
            T den = rbar - rmin;
            T th = den > T(0) ? (rbar - eps) / den : T(0);
            th = th < T(1) ? (th > T(0) ? th : T(0)) : T(1);
#pragma unroll
            for (int m = 1; m < NM; ++m) u[0][m] *= th;
            changed = true;
        }
        // step 2: pressure
        const T kk = eps / (gamma - T(1));
        const T rb = u[0][0], mxb = u[1][0], myb = u[2][0], eb = u[3][0];
        const T c = rb * eb - T(0.5) * (mxb * mxb + myb * myb) - kk * rb;
        T th2 = T(1);
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            T d[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T s = T(0);
#pragma unroll
                for (int m = 1; m < NM; ++m) s += u[v][m] * phi(q, m);
                s += u[v][0] * phi(q, 0) - u[v][0];
                d[v] = s;
            }
            const T a = d[0] * d[3] - T(0.5) * (d[1] * d[1] + d[2] * d[2]);
            const T b = rb * d[3] + eb * d[0] - (mxb * d[1] + myb * d[2]) - kk * d[0];
            if (a + b + c < T(0)) {
                T disc = b * b - T(4) * a * c;
                disc = sqrt(disc > T(0) ? disc : T(0));
                const T qq = T(-0.5) * (b + (b >= T(0) ? disc : -disc));
                T r = T(1e30);
                if (qq != T(0)) {
                    const T r1 = c / qq;
                    if (r1 > T(0) && r1 <= T(1)) r = r1;
                }
                if (a != T(0)) {
                    const T r2 = qq / a;
                    if (r2 > T(0) && r2 <= T(1) && r2 < r) r = r2;
                }
                if (r > T(1)) r = T(0);
                th2 = r < th2 ? r : th2;
            }
        }
        if (th2 < T(1)) {
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 1; m < NM; ++m) u[v][m] *= th2;
            changed = true;
        }
        return changed;
    }
}

}  // namespace crk
