// Shared device definitions: launch arguments, device state, physical
// fluxes, the Lax--Friedrichs flux (Sec. 2.1) and boundary exterior states.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "tables.cuh"

namespace crk {

constexpr int MAXS = 6;
enum { PHYS_ADV = 0, PHYS_EULER = 1, PHYS_EULER1D = 2 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2, BC_DIRICHLET = 3 };
enum { FN_CONST = 0, FN_SINE = 1, FN_SINE_PROD = 2, FN_DMR_BOTTOM = 3, FN_DMR_TOP = 4 };
enum { ST_NONPHYSICAL = 1u, ST_NAN = 2u, ST_TIMEOUT = 4u };

// Device-resident run state.  The fused reduction of every step writes the
// FP64 wave-speed maximum and totals of the new cell averages here and, for
// device-driven runs, the next dt = min(cfl / maxspeed, t_end - t).
struct DevState {
    double t, dt, t_end, cfl;
    double maxspeed;
    double sums[4];
    double troubled;          // troubled cells flagged in the last step
    unsigned status;          // ST_* bits
    unsigned counter;         // arrival counter of a batched problem's last-warp reduction
    unsigned long long steps;
    unsigned long long lim_count;   // cells flagged by a separate limiter pass since the last step
};

struct BCSide {
    int type;
    int fn;
    double p[16];
    float pf[4];              // FP32 copy of p[0..3] (the constant exterior state of FN_CONST)
    // affine form u_ext = m * u_int + c of the sides whose exterior state
    // depends on nothing else (outflow, reflecting wall, constant state);
    // affine = 0: the general function (set_bc_affine fills these)
    int affine;
    float m[4];
    float cf[4];
    double cd[4];
};

struct StepArgs {
    const void* uin;
    void* uout;
    int nx, ny;
    double x0, y0, dx, dy;
    double t, dt;             // used when dt_from_dev == 0
    int dt_from_dev;
    DevState* ds;
    double* partials;         // per-warp reduction slots
    int s;
    const double* tab;        // device tableau buffer, layout of pack_tableau
    BCSide bc[4];             // W, E, S, N
    int seg_len, n_strips, n_segs;
    int limit;                // 1: limit u^n on load (final-stage limiters of the previous step)
    double M;                 // TVB parameter; < 0: no TVB limiter
    double pp_eps;            // > 0: positivity-preserving scaling with this floor
    double gamma;
    double beta[2];
    // sum_i b_i u^(i) = sum_l lin_gamma[l] (-dt D)^l u^n for a linear local
    // operator D: lin_gamma[l] = b^T A^l 1 (the modal linear step)
    double lin_gamma[MAXS];
    float lin_gammaf[MAXS];
    int lin_inflow;           // inflow faces of every cell: bit 0 W, 1 E, 2 S, 3 N (the modal linear step)
    // limiter parameters as the one-thread-per-cell limiter pass takes them
    // (filled by set_limiter_params at its launch)
    float Mdx2f, Mdy2f, gammaf, pp_epsf;
    int tvb_on, pp_on;
    // constants derived from the fields above, filled on the host by
    // set_derived at every launch: no warp recomputes them (FP64 divisions
    // run on GB300's narrow FP64 pipe, and every warp of a launch reaches its
    // prologue at the same time)
    double rx, ry, cell, adv_speed;   // 1/dx, 1/dy, dx dy, |bx|/dx + |by|/dy
    float rxf, ryf, gm1f;
    double lin_k[6];                  // modal step: 2bx/dx, 2by/dy, -bx/dx, bx/dx, -by/dy, by/dy
    float lin_kf[6];
    const float* mlp;         // learned indicator parameters (device), or null
    float mlp_zlo, mlp_zhi;   // logit band in which the TVB test decides
    float mlp_scale;          // M h^2, h = max(dx, dy): the features' scale reference (set_derived)
};

// One problem of a batched ensemble (problem table, device)
struct BatchProblem {
    long long offset;      // element offset of the problem's planes in each buffer
    int nx, ny;
    double x0, y0, dx, dy;
    double rx, ry;         // 1/dx, 1/dy (host)
    int n_strips, n_segs;
    int warp0;             // first task / reduction slot of the problem
    int sq;                // 1: square cells (dx == dy), the square-cell form of the step
};

// -------------------------------------------------------------------------
// Physical flux along one axis and the wave speed |f'(u).nu| for nu = e_axis.
template <class T, int PHYS> struct Phys;

template <class T> struct Phys<T, PHYS_ADV> {
    static constexpr int NV = 1;
    T bx, by;
    __device__ __forceinline__ void flux2(const T* u, T* fx, T* fy) const {
        fx[0] = bx * u[0];
        fy[0] = by * u[0];
    }
    template <int AXIS>
    __device__ __forceinline__ T fluxn(const T* u, T* f) const {
        const T b = AXIS == 0 ? bx : by;
        f[0] = b * u[0];
        return fabs(b);
    }
};

template <class T> struct Phys<T, PHYS_EULER> {
    static constexpr int NV = 4;
    T gm1, gamma;
    __device__ __forceinline__ void flux2(const T* u, T* fx, T* fy) const {
        const T ir = T(1) / u[0];
        const T w = u[1] * ir, v = u[2] * ir;
        const T p = gm1 * (u[3] - T(0.5) * (u[1] * w + u[2] * v));
        const T ep = u[3] + p;
        const T muv = u[1] * v;   // rho u v, the x flux of rho v and the y flux of rho u
        fx[0] = u[1]; fx[1] = u[1] * w + p; fx[2] = muv; fx[3] = w * ep;
        fy[0] = u[2]; fy[1] = muv; fy[2] = u[2] * v + p; fy[3] = v * ep;
    }
    // normal flux and wave speed |v_n| + c
    template <int AXIS>
    __device__ __forceinline__ T fluxn(const T* u, T* f) const {
        const T ir = T(1) / u[0];
        const T w = u[1] * ir, v = u[2] * ir;
        const T p = gm1 * (u[3] - T(0.5) * (u[1] * w + u[2] * v));
        const T vn = AXIS == 0 ? w : v;
        f[0] = u[1 + AXIS];
        f[1] = u[1] * vn + (AXIS == 0 ? p : T(0));
        f[2] = u[2] * vn + (AXIS == 1 ? p : T(0));
        f[3] = vn * (u[3] + p);
        const T c2 = gamma * p * ir;
        return fabs(vn) + sqrt(c2 > T(0) ? c2 : T(0));
    }
};

// 1D Euler: (rho, rho w, E)
template <class T> struct Phys<T, PHYS_EULER1D> {
    static constexpr int NV = 3;
    T gm1, gamma;
    template <int AXIS>
    __device__ __forceinline__ T fluxn(const T* u, T* f) const {
        const T ir = T(1) / u[0];
        const T w = u[1] * ir;
        const T p = gm1 * (u[2] - T(0.5) * u[1] * w);
        f[0] = u[1];
        f[1] = u[1] * w + p;
        f[2] = w * (u[2] + p);
        const T c2 = gamma * p * ir;
        return fabs(w) + sqrt(c2 > T(0) ? c2 : T(0));
    }
};

// 2D Euler fluxes in deviation form.  A state is held as its deviation d
// from a base state c (per cell: the FP32 high part of the cell's average at
// t^n), and every flux as the deviation f(c + d) - f(c), computed from
// exact algebraic differences in which each term is a base or full quantity
// times a deviation:
//   du = (d_m - u0 d_rho) / rho1,  dv = (d_n - v0 d_rho) / rho1,
//   d(m u) = d_m u0 + m1 du,  d(n v) = d_n v0 + n1 dv,
//   dp = (gamma - 1)(d_E - (d(m u) + d(n v)) / 2),
//   d((E + p) u) = (d_E + dp) u0 + (E1 + p1) du,  ...
// with u0 = m0 / rho0 (any rounding of u0 only perturbs a term that is
// already multiplied by a deviation), m1 = m0 + d_m, E1 + p1 = E0 + p0 +
// d_E + dp.  The FP32 rounding error of a flux is then a few ulps of the
// deviation, O(eps |f(u) - f(c)|) = O(eps h |f_x|), instead of a few ulps of
// the flux itself, O(eps |f|).  A DG operator applied to deviation fluxes
// equals the operator applied to the fluxes (the constant f(c) has zero
// discrete divergence: the Gauss rules integrate grad phi_m and phi_m on the
// faces exactly), so div^loc f and div^DG f come out with errors relative to
// their own size, as Sec. 3.3's perturbed-RK estimate assumes of a
// full-accuracy final stage.  Only the base changes from cell to cell:
// face states and face fluxes are moved between two cells' bases by the
// deviation of the base difference.
template <class T>
struct EulerDev {
    static constexpr int NV = 4;
    T gm1, gamma;
    T r0, u0, v0, m0, n0, p0, ep0;   // base: rho, velocity, momentum, pressure, E + p
    __device__ __forceinline__ void set_base(const T* c) {
        r0 = c[0];
        m0 = c[1];
        n0 = c[2];
        const T ir = T(1) / c[0];
        u0 = c[1] * ir;
        v0 = c[2] * ir;
        p0 = gm1 * (c[3] - T(0.5) * (c[1] * u0 + c[2] * v0));
        ep0 = c[3] + p0;
    }
    // the deviation's primitive increments: 1 / rho1, du, dv, d(m u), d(n v), dp, m1, n1
    struct Inc {
        T r1i, du, dv, dmu, dnv, dp, m1, n1;
    };
    __device__ __forceinline__ Inc inc(const T* d) const {
        Inc q;
        q.r1i = T(1) / (r0 + d[0]);
        q.du = (d[1] - u0 * d[0]) * q.r1i;
        q.dv = (d[2] - v0 * d[0]) * q.r1i;
        q.m1 = m0 + d[1];
        q.n1 = n0 + d[2];
        q.dmu = fma(d[1], u0, q.m1 * q.du);
        q.dnv = fma(d[2], v0, q.n1 * q.dv);
        q.dp = gm1 * (d[3] - T(0.5) * (q.dmu + q.dnv));
        return q;
    }
    // deviations of both fluxes at a state of deviation d
    __device__ __forceinline__ void flux2(const T* d, T* fx, T* fy) const {
        const Inc q = inc(d);
        const T dep = d[3] + q.dp;
        const T ep1 = ep0 + dep;
        fx[0] = d[1];
        fx[1] = q.dmu + q.dp;
        fx[2] = fma(d[2], u0, q.n1 * q.du);
        fx[3] = fma(dep, u0, ep1 * q.du);
        fy[0] = d[2];
        fy[1] = fma(d[1], v0, q.m1 * q.dv);
        fy[2] = q.dnv + q.dp;
        fy[3] = fma(dep, v0, ep1 * q.dv);
    }
    // deviation of the normal flux along +e_AXIS and the full state's wave
    // speed |v_n| + c
    template <int AXIS>
    __device__ __forceinline__ T fluxn(const T* d, T* f) const {
        const Inc q = inc(d);
        const T dep = d[3] + q.dp;
        const T ep1 = ep0 + dep;
        if (AXIS == 0) {
            f[0] = d[1];
            f[1] = q.dmu + q.dp;
            f[2] = fma(d[2], u0, q.n1 * q.du);
            f[3] = fma(dep, u0, ep1 * q.du);
        } else {
            f[0] = d[2];
            f[1] = fma(d[1], v0, q.m1 * q.dv);
            f[2] = q.dnv + q.dp;
            f[3] = fma(dep, v0, ep1 * q.dv);
        }
        const T vn = AXIS == 0 ? u0 + q.du : v0 + q.dv;
        const T c2 = gamma * (p0 + q.dp) * q.r1i;
        return fabs(vn) + sqrt(c2 > T(0) ? c2 : T(0));
    }
};

// Lax--Friedrichs flux through a face with normal +e_AXIS from the state on
// the low side uL to the state on the high side uR; alpha is local to the
// point: max of |f'.nu| over both traces.
// HALF = false: twice the flux (the factor 1/2 left to the caller's weights)
template <class T, int PHYS, int AXIS, bool HALF = true>
__device__ __forceinline__ void llf(const Phys<T, PHYS>& ph, const T* uL, const T* uR, T* F) {
    constexpr int NV = Phys<T, PHYS>::NV;
    T fL[NV], fR[NV];
    const T sL = ph.template fluxn<AXIS>(uL, fL);
    const T sR = ph.template fluxn<AXIS>(uR, fR);
    const T al = sL > sR ? sL : sR;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = (HALF ? T(0.5) : T(1)) * ((fL[v] + fR[v]) - al * (uR[v] - uL[v]));
}

// The same flux in deviation form: uL, uR and F are deviations from the
// base of ph (F = fhat - f(c).nu; the jump uR - uL is the same).
template <class T, int AXIS, bool HALF = true>
__device__ __forceinline__ void llf(const EulerDev<T>& ph, const T* uL, const T* uR, T* F) {
    T fL[4], fR[4];
    const T sL = ph.template fluxn<AXIS>(uL, fL);
    const T sR = ph.template fluxn<AXIS>(uR, fR);
    const T al = sL > sR ? sL : sR;
#pragma unroll
    for (int v = 0; v < 4; ++v) F[v] = (HALF ? T(0.5) : T(1)) * ((fL[v] + fR[v]) - al * (uR[v] - uL[v]));
}

// llf for either kind of flux object (physical fluxes or deviation form)
template <int AXIS, bool HALF = true, class T, int PHYS>
__device__ __forceinline__ void llf_ax(const Phys<T, PHYS>& ph, const T* uL, const T* uR, T* F) {
    llf<T, PHYS, AXIS, HALF>(ph, uL, uR, F);
}
template <int AXIS, bool HALF = true, class T>
__device__ __forceinline__ void llf_ax(const EulerDev<T>& ph, const T* uL, const T* uR, T* F) {
    llf<T, AXIS, HALF>(ph, uL, uR, F);
}

// The Lax--Friedrichs flux of llf from states whose normal fluxes and wave
// speeds are already known (the same arithmetic as llf).
template <class T, int NV>
__device__ __forceinline__ void lf_from_fluxes(const T* uL, const T* fL, T sL, const T* uR, const T* fR, T sR, T* F) {
    const T al = sL > sR ? sL : sR;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = T(0.5) * ((fL[v] + fR[v]) - al * (uR[v] - uL[v]));
}

// Value of the sine boundary data (FN_SINE, FN_SINE_PROD); kept out of line
// so that the double-precision sines are not inlined at every call site.
static __device__ __noinline__ double bc_sine_value(int prod, double p0, double p1, double p2, double p3, double p4,
                                             double x, double y, double t) {
    return prod ? p0 * sin(p1 * (x - p2 * t)) * sin(p3 * (y - p4 * t)) : p0 * sin(p1 * x + p2 * y - p3 * t + p4);
}

// Exterior state at a boundary point from the interior state; axis is the
// axis normal to the boundary.  xyt(x, y, t) yields the point and time; it is
// called only by the boundary functions that depend on them, so outflow,
// reflecting and constant-state sides cost no FP64 arithmetic.
template <class T, int NV, class XYT>
__device__ __forceinline__ void bc_exterior(const BCSide& bc, int axis, const T* uin, const XYT& xyt, T* uext) {
#pragma unroll
    for (int v = 0; v < NV; ++v) uext[v] = uin[v];
    if (bc.type == BC_OUTFLOW) return;
    if (bc.type == BC_REFLECT) {
        if (NV >= 3) uext[1 + axis] = -uin[1 + axis];
        return;
    }
    const double* p = bc.p;
    if (bc.fn == FN_CONST) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if constexpr (sizeof(T) == 4) uext[v] = bc.pf[v];
            else uext[v] = T(p[v]);
        }
        return;
    }
    double x, y, t;
    xyt(x, y, t);
    switch (bc.fn) {
        case FN_SINE:
        case FN_SINE_PROD:
            uext[0] = T(bc_sine_value(bc.fn == FN_SINE_PROD, p[0], p[1], p[2], p[3], p[4], x, y, t));
            break;
        case FN_DMR_BOTTOM:
            if (x < p[4]) {
#pragma unroll
                for (int v = 0; v < NV; ++v) uext[v] = T(p[v]);
            } else if (NV >= 3) {
                uext[1 + axis] = -uin[1 + axis];
            }
            break;
        case FN_DMR_TOP: {
            const double xs = p[8] + p[9] * y + p[10] * t;
            const double* st = x < xs ? p : p + 4;
#pragma unroll
            for (int v = 0; v < NV; ++v) uext[v] = T(st[v]);
        } break;
        default:
            break;
    }
}

// Affine forms of the boundary sides (see BCSide); the kernels fall back to
// bc_exterior where affine is 0.
inline void set_bc_affine(BCSide* bc, int nv) {
    for (int s = 0; s < 4; ++s) {
        BCSide& b = bc[s];
        b.affine = 0;
        for (int v = 0; v < 4; ++v) { b.m[v] = 1.f; b.cf[v] = 0.f; b.cd[v] = 0.0; }
        if (b.type == BC_OUTFLOW) {
            b.affine = 1;
        } else if (b.type == BC_REFLECT) {
            b.affine = 1;
            if (nv >= 3) b.m[1 + (s < 2 ? 0 : 1)] = -1.f;
        } else if (b.type == BC_DIRICHLET && b.fn == FN_CONST) {
            b.affine = 1;
            for (int v = 0; v < 4; ++v) { b.m[v] = 0.f; b.cf[v] = (float)b.p[v]; b.cd[v] = b.p[v]; }
        }
    }
}

// FP32 copies and switches of the limiter parameters, so that a kernel with
// one thread per cell does no FP64 arithmetic for them
inline void set_limiter_params(StepArgs& a) {
    a.Mdx2f = (float)(a.M * a.dx * a.dx);
    a.Mdy2f = (float)(a.M * a.dy * a.dy);
    a.gammaf = (float)a.gamma;
    a.pp_epsf = (float)a.pp_eps;
    a.tvb_on = a.M >= 0.0;
    a.pp_on = a.pp_eps > 0.0;
}

// Every derived constant of a launch (the limiter parameters included), in
// the same arithmetic the kernels would use: FP64, rounded once to FP32.
inline void set_derived(StepArgs& a) {
    set_limiter_params(a);
    a.rx = 1.0 / a.dx;
    a.ry = 1.0 / a.dy;
    a.cell = a.dx * a.dy;
    a.adv_speed = (a.beta[0] < 0 ? -a.beta[0] : a.beta[0]) / a.dx + (a.beta[1] < 0 ? -a.beta[1] : a.beta[1]) / a.dy;
    a.rxf = (float)a.rx;
    a.ryf = (float)a.ry;
    a.gm1f = (float)(a.gamma - 1.0);
    a.lin_k[0] = 2.0 * a.beta[0] / a.dx;
    a.lin_k[1] = 2.0 * a.beta[1] / a.dy;
    a.lin_k[2] = -a.beta[0] / a.dx;
    a.lin_k[3] = a.beta[0] / a.dx;
    a.lin_k[4] = -a.beta[1] / a.dy;
    a.lin_k[5] = a.beta[1] / a.dy;
    for (int i = 0; i < 6; ++i) a.lin_kf[i] = (float)a.lin_k[i];
    const double hh = a.dx > a.dy ? a.dx : a.dy;
    a.mlp_scale = (float)(a.M * hh * hh);
}

// Device tableau buffer: FP64 a (MAXS x MAXS, row-major), b, c, followed by
// FP32 copies of a and b rounded once on the host, so that FP32 kernels take
// their stage weights without FP64 loads or conversions.
constexpr int TAB_F64 = MAXS * MAXS + 2 * MAXS;
constexpr int TAB_F32 = MAXS * MAXS + MAXS;
constexpr size_t TAB_BYTES = TAB_F64 * sizeof(double) + TAB_F32 * sizeof(float);
inline void pack_tableau(int s, const double* A, const double* b, const double* c, unsigned char* out) {
    double d[TAB_F64] = {0};
    float f[TAB_F32] = {0};
    for (int i = 0; i < s; ++i) {
        for (int j = 0; j < s; ++j) d[i * MAXS + j] = A[i * MAXS + j];
        d[MAXS * MAXS + i] = b[i];
        d[MAXS * MAXS + MAXS + i] = c[i];
    }
    for (int i = 0; i < MAXS * MAXS + MAXS; ++i) f[i] = (float)d[i];
    for (size_t k = 0; k < sizeof(d); ++k) out[k] = reinterpret_cast<const unsigned char*>(d)[k];
    for (size_t k = 0; k < sizeof(f); ++k) out[sizeof(d) + k] = reinterpret_cast<const unsigned char*>(f)[k];
}

__device__ __forceinline__ double tab_a(const StepArgs& a, int i, int j) { return __ldg(a.tab + i * MAXS + j); }
__device__ __forceinline__ double tab_b(const StepArgs& a, int i) { return __ldg(a.tab + MAXS * MAXS + i); }
__device__ __forceinline__ double tab_c(const StepArgs& a, int i) { return __ldg(a.tab + MAXS * MAXS + MAXS + i); }
// the same weights in the kernel's arithmetic type T
template <class T>
__device__ __forceinline__ T tab_aT(const StepArgs& a, int i, int j) {
    if constexpr (sizeof(T) == 4) return __ldg(reinterpret_cast<const float*>(a.tab + TAB_F64) + i * MAXS + j);
    else return tab_a(a, i, j);
}
template <class T>
__device__ __forceinline__ T tab_bT(const StepArgs& a, int i) {
    if constexpr (sizeof(T) == 4) return __ldg(reinterpret_cast<const float*>(a.tab + TAB_F64) + MAXS * MAXS + i);
    else return tab_b(a, i);
}

// Entry of a rarely taken branch (boundary data): no ordinary memory access is
// hoisted above it into the common path, where it would run (predicated or
// speculated) on every row.  Arithmetic on launch parameters and read-only
// loads can still move across it; the branch's indices pass through opaque().
__device__ __forceinline__ void cold_branch() { asm volatile("" ::: "memory"); }
// v, opaque to the compiler.  In a cold branch: arithmetic on the result
// (boundary coordinates and stage times from a row, column or stage index)
// cannot be speculated above the branch.  On a launch constant: the value is
// held in a register from that point, as a computed one would be.
__device__ __forceinline__ int opaque(int v) {
    asm volatile("" : "+r"(v));
    return v;
}
__device__ __forceinline__ float opaque(float v) {
    asm volatile("" : "+f"(v));
    return v;
}
__device__ __forceinline__ double opaque(double v) {
    asm volatile("" : "+d"(v));
    return v;
}

// f(std::integral_constant<int, i>) for i = 0 .. N-1: loops whose index must
// be a constant expression (table entries folded at compile time)
template <class F, int... I>
__device__ __forceinline__ void static_for_seq(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_seq(f, std::make_integer_sequence<int, N>{});
}

template <class T>
__device__ __forceinline__ T shfl_down(T v, int d) {
    return __shfl_down_sync(0xffffffffu, v, d);
}
template <class T>
__device__ __forceinline__ T shfl_up(T v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}

}  // namespace crk
