// Fused cRKDG time step for the linear flux f(u) = (bx u, by u) in modal form.
//
// With a linear flux and the Lax--Friedrichs flux of speed alpha = |beta . n|
// (the upwind flux), both operators of the cRKDG step (eq. (2.8)) are fixed
// linear maps of the modal coefficients, and the quadrature forms of
// step2d.cuh evaluate them exactly:
//   - the local operator (eq. (2.7)) of a P^k / Q^k state w is beta . grad w
//     itself (its derivative stays in the space), i.e.
//     L_loc(w) = (2 bx / dx) d/dxi w + (2 by / dy) d/deta w with the Legendre
//     derivative d/dxi P_i = sum_{i' = i-1, i-3, ...} (2i'+1) P_i';
//   - the DG operator (eq. (2.3)) is the local operator plus, on each inflow
//     face (beta . n < 0), (beta . n)(w_ext - w_int) lifted to the modes:
//     (2i+1) P_i(+-1) / dx per trace coefficient on the E/W faces,
//     (2j+1) P_j(+-1) / dy on the N/S faces; the trace coefficients are
//     sums of the modes with P_i(+-1) = (+-1)^i;
//   - being linear, the final stage sum_i b_i L_DG(u^(i)) equals
//     L_DG(sum_i b_i u^(i)) (the identity behind Theorem 3.3), so the face
//     coupling is needed once per step, for wbar = sum_i b_i u^(i).
// The work decomposition is step2d.cuh's (marching warps, 30 columns + 2 halo
// lanes, segments of rows, the row below finished when the current row's
// south trace is known) with a tenth of its arithmetic, so the step is bound
// by HBM.  Boundary sides: periodic, or an exterior state affine in the
// interior one (outflow, wall, constant state; BCSide::affine).
#pragma once
#include "step2d.cuh"

// blocks of 256 threads per SM the FP32 modal step is compiled for (tuning knob)
#ifndef CRK_LIN_MINB
#define CRK_LIN_MINB 2
#endif

namespace crk {

// Degrees of mode m and the entries of the Legendre derivative matrices,
// as constexpr functions (called with constant-expression arguments only)
template <int K, int B>
constexpr int lin_mi(int m) {
    int i = 0, j = 0;
    mode_ij(K, B, m, i, j);
    return i;
}
template <int K, int B>
constexpr int lin_mj(int m) {
    int i = 0, j = 0;
    mode_ij(K, B, m, i, j);
    return j;
}
// d/dxi phi_c = sum_r lin_dxi(r, c) phi_r, d/deta likewise
template <int K, int B>
constexpr double lin_dxi(int r, int c) {
    const int ir = lin_mi<K, B>(r), jr = lin_mj<K, B>(r), ic = lin_mi<K, B>(c), jc = lin_mj<K, B>(c);
    return (jc == jr && ic > ir && (ic - ir) % 2 == 1) ? 2.0 * ir + 1.0 : 0.0;
}
template <int K, int B>
constexpr double lin_deta(int r, int c) {
    const int ir = lin_mi<K, B>(r), jr = lin_mj<K, B>(r), ic = lin_mi<K, B>(c), jc = lin_mj<K, B>(c);
    return (ic == ir && jc > jr && (jc - jr) % 2 == 1) ? 2.0 * jr + 1.0 : 0.0;
}

// private shared memory per thread (none: the stages are combined in registers)
template <class T, int K, int B>
__host__ __device__ constexpr int linear_smem_per_thread(int) {
    return 0;
}

template <class T, int K, int B>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? CRK_LIN_MINB : 1) step2d_linear_kernel(const StepArgs a) {
    constexpr int NM = n_modes_2d(K, B);
    constexpr int NT = K + 1;   // trace coefficients per face
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;

    allow_dependent_launch();
    const int gw = blockIdx.x * (nthr >> 5) + (tid >> 5);
    const int total_warps = a.n_strips * a.n_segs;
    if (gw >= total_warps) return;   // whole warp leaves; no block barriers
    const ArgsView<T> pv{a, a.dt_from_dev ? a.ds->t : a.t, a.dt_from_dev ? a.ds->dt : a.dt};

    const int nx = a.nx, ny = a.ny;
    const size_t plane = (size_t)nx * ny;
    const T* __restrict__ uin = static_cast<const T*>(a.uin);
    T* __restrict__ uout = static_cast<T*>(a.uout);
    const double dt = pv.dt();
    const double t0 = pv.t();

    const int strip = gw % a.n_strips;
    const int seg = gw / a.n_strips;
    const int xs = strip * 30;
    const int col = xs - 1 + lane;
    const bool perx = a.bc[0].type == BC_PERIODIC;
    const bool pery = a.bc[2].type == BC_PERIODIC;
    int xl = ((col % nx) + nx) % nx;
    if (!perx) xl = col < 0 ? 0 : (col >= nx ? nx - 1 : col);
    const bool outlane = lane >= 1 && lane <= 30 && col < nx;
    const int r0 = (int)(((long long)seg * ny) / a.n_segs);
    const int r1 = (int)(((long long)(seg + 1) * ny) / a.n_segs);
    const int rstart = (r0 > 0 || pery) ? r0 - 1 : r0;
    const int rend = (r1 < ny || pery) ? r1 : r1 - 1;

    if (!(dt > 0.0)) {   // a non-positive dt leaves the state unchanged
        if (outlane)
            for (int r = r0; r < r1; ++r)
                for (int m = 0; m < NM; ++m) uout[m * plane + (size_t)r * nx + col] = uin[m * plane + (size_t)r * nx + col];
        return;
    }

    const T tdt = T(dt);
    // launch constants made on the host (set_derived): no FP64 divisions per warp
    constexpr bool F32 = sizeof(T) == 4;
    auto kc = [&](int i) -> T { return F32 ? T(a.lin_kf[i]) : T(a.lin_k[i]); };
    const T cx = kc(0), cy = kc(1);
    // lifts of the inflow-face jumps: W (bx > 0), E (bx < 0), S (by > 0), N (by < 0)
    // integer flags (set on the host): tests on the FP64 launch parameters
    // would be re-evaluated on GB300's narrow FP64 pipe at every use
    const int inflow = a.lin_inflow;
    const bool inW = inflow & 1, inE = inflow & 2, inS = inflow & 4, inN = inflow & 8;
    const T kW = kc(2), kE = kc(3), kS = kc(4), kN = kc(5);
    const int S = a.s;
    // out = D w: the local operator (2 bx / dx) d/dxi + (2 by / dy) d/deta
    auto applyD = [&](const T* w, T* out) {
        static_for<NM>([&](auto mr) {
            constexpr int m = decltype(mr)::value;
            T acc = T(0);
            static_for<NM>([&](auto cc) {
                constexpr int c = decltype(cc)::value;
                constexpr double ex = lin_dxi<K, B>(m, c), ey = lin_deta<K, B>(m, c);
                if constexpr (ex != 0.0) acc += (cx * T(ex)) * w[c];
                if constexpr (ey != 0.0) acc += (cy * T(ey)) * w[c];
            });
            out[m] = acc;
        });
    };
    // exterior trace at a non-periodic side: m * interior + constant state
    auto bc_trace = [&](int side, const T* in, T* out) {
        const BCSide& b = a.bc[side];
        const T c = sizeof(T) == 4 ? T(b.cf[0]) : T(b.cd[0]);
#pragma unroll
        for (int q = 0; q < NT; ++q) out[q] = T(b.m[0]) * in[q] + (q == 0 ? c : T(0));
    };

    T cs_hi = T(0), cs_lo = T(0);   // compensated column total
    unsigned status = 0;
    T prevN[NT];                    // north trace of wbar, row below
    T P[NM];                        // row below: u^{n+1} without its north-face term
#pragma unroll
    for (int q = 0; q < NT; ++q) prevN[q] = T(0);
#pragma unroll
    for (int m = 0; m < NM; ++m) P[m] = T(0);

    auto write_row = [&](int rw) {
        if (!outlane) return;
        const size_t o = (size_t)rw * nx + col;
#pragma unroll
        for (int m = 0; m < NM; ++m) uout[m * plane + o] = P[m];
        const T sum = cs_hi + P[0];   // TwoSum
        const T bv = sum - cs_hi;
        cs_lo += (cs_hi - (sum - bv)) + (P[0] - bv);
        cs_hi = sum;
        if (!(P[0] == P[0])) status |= ST_NAN;
    };

    // u^n of the next row is loaded while the current row computes
    auto row_index = [&](int r) -> size_t {
        const int ry = r < 0 ? r + ny : (r >= ny ? r - ny : r);
        return (size_t)ry * nx + xl;
    };
    T unext[NM];
    {
        const size_t c0 = row_index(rstart);
#pragma unroll
        for (int m = 0; m < NM; ++m) unext[m] = uin[m * plane + c0];
    }
    for (int r = rstart; r <= rend; ++r) {
        const bool out_row = r >= r0 && r < r1;
        const bool south_bc = (r == 0) && !pery;
        T un[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) un[m] = unext[m];
        if (r < rend) {
            const size_t cn = row_index(r + 1);
#pragma unroll
            for (int m = 0; m < NM; ++m) unext[m] = uin[m * plane + cn];
        }

        // stages (eq. (2.8), first line) combined: with the local operator the
        // fixed linear map D, u^(i) = sum_l (A^l 1)_i (-dt D)^l u^n, hence
        // wbar = sum_i b_i u^(i) = sum_l gamma_l (-dt D)^l u^n, gamma_l =
        // b^T A^l 1 (Horner: s - 1 applications of D)
        T wbar[NM];
        bool started = false;
#pragma unroll
        for (int l = MAXS - 1; l >= 0; --l) {
            if (l < S) {
                const T gl = sizeof(T) == 4 ? T(a.lin_gammaf[l]) : T(a.lin_gamma[l]);
                if (started) {
                    T d[NM];
                    applyD(wbar, d);
#pragma unroll
                    for (int m = 0; m < NM; ++m) wbar[m] = gl * un[m] - tdt * d[m];
                } else {
#pragma unroll
                    for (int m = 0; m < NM; ++m) wbar[m] = gl * un[m];
                    started = true;
                }
            }
        }

        // DG operator of wbar: local part, then the inflow-face jumps
        T Lw[NM];
        applyD(wbar, Lw);
        T tE[NT], tW[NT], tN[NT], tS[NT];
#pragma unroll
        for (int q = 0; q < NT; ++q) tE[q] = tW[q] = tN[q] = tS[q] = T(0);
        static_for<NM>([&](auto mc) {
            constexpr int m = decltype(mc)::value;
            constexpr int i = lin_mi<K, B>(m), j = lin_mj<K, B>(m);
            tE[j] += wbar[m];
            tN[i] += wbar[m];
            if constexpr (i % 2) tW[j] -= wbar[m];
            else tW[j] += wbar[m];
            if constexpr (j % 2) tS[i] -= wbar[m];
            else tS[i] += wbar[m];
        });
        T extW[NT], extE[NT];
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            extW[q] = shfl_up(tE[q], 1);     // west neighbour's east trace
            extE[q] = shfl_down(tW[q], 1);   // east neighbour's west trace
        }
        if (!perx && col == 0) bc_trace(0, tW, extW);
        if (!perx && col == nx - 1) bc_trace(1, tE, extE);
        if (inW) {
            static_for<NM>([&](auto mc) {
                constexpr int m = decltype(mc)::value;
                constexpr int i = lin_mi<K, B>(m), j = lin_mj<K, B>(m);
                constexpr double f = (2.0 * i + 1.0) * ((i % 2) ? -1.0 : 1.0);
                Lw[m] += (kW * T(f)) * (extW[j] - tW[j]);
            });
        }
        if (inE) {
            static_for<NM>([&](auto mc) {
                constexpr int m = decltype(mc)::value;
                constexpr int i = lin_mi<K, B>(m), j = lin_mj<K, B>(m);
                Lw[m] += (kE * T(2.0 * i + 1.0)) * (extE[j] - tE[j]);
            });
        }
        if (inS && (r > rstart || south_bc)) {
            T extS[NT];
            if (south_bc) {
                bc_trace(2, tS, extS);
            } else {
#pragma unroll
                for (int q = 0; q < NT; ++q) extS[q] = prevN[q];
            }
            static_for<NM>([&](auto mc) {
                constexpr int m = decltype(mc)::value;
                constexpr int i = lin_mi<K, B>(m), j = lin_mj<K, B>(m);
                constexpr double f = (2.0 * j + 1.0) * ((j % 2) ? -1.0 : 1.0);
                Lw[m] += (kS * T(f)) * (extS[i] - tS[i]);
            });
        }

        // the row below: its north face is this row's south face
        if (r > rstart && r - 1 >= r0 && r - 1 < r1) {
            if (inN) {
                static_for<NM>([&](auto mc) {
                    constexpr int m = decltype(mc)::value;
                    constexpr int i = lin_mi<K, B>(m), j = lin_mj<K, B>(m);
                    P[m] -= tdt * ((kN * T(2.0 * j + 1.0)) * (tS[i] - prevN[i]));
                });
            }
            write_row(r - 1);
        }
        if (out_row) {
#pragma unroll
            for (int m = 0; m < NM; ++m) P[m] = un[m] - tdt * Lw[m];
            if (r == ny - 1 && !pery) {   // top boundary: north face from the boundary state
                if (inN) {
                    T extN[NT];
                    bc_trace(3, tN, extN);
                    static_for<NM>([&](auto mc) {
                        constexpr int m = decltype(mc)::value;
                        constexpr int i = lin_mi<K, B>(m), j = lin_mj<K, B>(m);
                        P[m] -= tdt * ((kN * T(2.0 * j + 1.0)) * (extN[i] - tN[i]));
                    });
                }
                write_row(r);
            }
        }
#pragma unroll
        for (int q = 0; q < NT; ++q) prevN[q] = tN[q];
    }

    double red_max = (outlane && r0 < r1) ? a.adv_speed : 0.0;
    double red_sum[1] = {double(cs_hi) + double(cs_lo)};
    step_epilogue<1, 3>(a, pv, gw, lane, total_warps, red_max, red_sum, 0u, status, a.cell, t0, dt);
}

}  // namespace crk
