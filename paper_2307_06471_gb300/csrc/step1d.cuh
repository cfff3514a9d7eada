// Fused cRKDG time step on a 1D mesh (eq. (2.8)).  A warp owns 30 cells plus
// one halo cell on each side; each lane runs all RK stages of its cell with
// the local operator (eq. (2.7)), exchanges the final-stage face traces with
// its neighbour lane by shuffles and writes u^{n+1}.  With n_steps > 1 (one
// block only) the block marches n_steps steps in one launch, ping-ponging
// between the two state buffers with a block barrier between steps.
#pragma once
#include "common.cuh"

namespace crk {

template <class T, int K, int PHYS>
__global__ void __launch_bounds__(1024) step1d_kernel(StepArgs a, int n_steps) {
    constexpr Tab1D<K> tb = make_tab1d<K>();
    constexpr int NM = K + 1;
    constexpr int NV = Phys<T, PHYS>::NV;
    constexpr int NQ = K + 1;
    constexpr int NDOF = NV * NM;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int nthr = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    auto slot = [&](int k) -> T& { return sm[k * nthr + tid]; };

    const int nx = a.nx;
    const int gw = blockIdx.x * (nthr >> 5) + (tid >> 5);
    const int xs = gw * 30;
    const int col = xs - 1 + lane;
    const bool per = a.bc[0].type == BC_PERIODIC;
    int xl = ((col % nx) + nx) % nx;
    if (!per) xl = col < 0 ? 0 : (col >= nx ? nx - 1 : col);
    const bool outlane = lane >= 1 && lane <= 30 && col < nx && xs < nx;
    const bool has_bcW = !per && xs == 0;
    const bool has_bcE = !per && xs + 30 >= nx;

    Phys<T, PHYS> ph;
    if constexpr (PHYS == PHYS_ADV) {
        ph.bx = T(a.beta[0]);
        ph.by = T(0);
    } else {
        ph.gamma = T(a.gamma);
        ph.gm1 = T(a.gamma - 1.0);
    }
    const double dt = a.dt;
    const T tdt = T(dt), rx = T(1.0 / a.dx);
    const int S = a.s;
    const T* src = static_cast<const T*>(a.uin);
    T* dst = static_cast<T*>(a.uout);

    for (int step = 0; step < n_steps; ++step) {
        const double t0 = a.t + step * dt;
        T un[NV][NM];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int m = 0; m < NM; ++m) un[v][m] = src[(size_t)(v * NM + m) * nx + xl];
        T V[NV][NM], FR[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            FR[v] = T(0);
#pragma unroll
            for (int m = 0; m < NM; ++m) V[v][m] = T(0);
        }
        for (int i = 0; i < S; ++i) {
            const double bid = tab_b(a, i);
            const T bi = T(bid);
            const bool need_L = i < S - 1;
            if (!need_L && bid == 0.0) continue;
            const double ti = t0 + tab_c(a, i) * dt;
            T w[NV][NM];
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 0; m < NM; ++m) w[v][m] = un[v][m];
            for (int j = 0; j < i; ++j) {
                const double ad = tab_a(a, i, j);
                if (ad == 0.0) continue;
                const T aij = T(ad) * tdt;
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int m = 0; m < NM; ++m) w[v][m] -= aij * slot(j * NDOF + v * NM + m);
            }
            // volume term sum_q w_q f(u_q) P_m'(xi_q) (scaled by 1/dx)
            T vol[NV][NM];
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 0; m < NM; ++m) vol[v][m] = T(0);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                T uq[NV], f[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    T s = T(0);
#pragma unroll
                    for (int m = 0; m < NM; ++m) s += w[v][m] * T(tb.phi[q][m]);
                    uq[v] = s;
                }
                ph.template fluxn<0>(uq, f);
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int m = 0; m < NM; ++m)
                        if (tb.g[q][m] != 0.0) vol[v][m] += rx * f[v] * T(tb.g[q][m]);
            }
            T tR[NV], tL[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                T r = 0, l = 0;
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    r += w[v][m] * T(tb.tR[m]);
                    l += w[v][m] * T(tb.tL[m]);
                }
                tR[v] = r;
                tL[v] = l;
            }
            if (need_L) {
                T fr[NV], fl[NV];
                ph.template fluxn<0>(tR, fr);
                ph.template fluxn<0>(tL, fl);
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int m = 0; m < NM; ++m)
                        slot(i * NDOF + v * NM + m) =
                            T(tb.cm[m]) * (rx * (fr[v] * T(tb.tR[m]) - fl[v] * T(tb.tL[m])) - vol[v][m]);
            }
            if (bid == 0.0) continue;
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 0; m < NM; ++m) V[v][m] += bi * vol[v][m];
            T tLn[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) tLn[v] = shfl_down(tL[v], 1);
            if (has_bcW && lane == 0)
                bc_exterior<T, NV>(a.bc[0], 0, tLn, [&](double& x, double& y, double& t) { x = a.x0; y = 0.0; t = ti; }, tR);
            if (has_bcE && col == nx - 1)
                bc_exterior<T, NV>(a.bc[1], 0, tR, [&](double& x, double& y, double& t) { x = a.x0 + nx * a.dx; y = 0.0; t = ti; },
                                   tLn);
            T F[NV];
            llf<T, PHYS, 0>(ph, tR, tLn, F);
#pragma unroll
            for (int v = 0; v < NV; ++v) FR[v] += bi * F[v];
        }
        T FL[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) FL[v] = shfl_up(FR[v], 1);
        if (outlane) {
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    const T face = FR[v] * T(tb.tR[m]) - FL[v] * T(tb.tL[m]);
                    dst[(size_t)(v * NM + m) * nx + col] =
                        un[v][m] - tdt * T(tb.cm[m]) * (rx * face - V[v][m]);
                }
        }
        if (step + 1 < n_steps) {
            __syncthreads();
            const T* tmp = src;
            src = dst;
            dst = const_cast<T*>(tmp);
        }
    }
}

}  // namespace crk
