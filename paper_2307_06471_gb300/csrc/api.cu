// C ABI of the cRKDG library (include/crkdg.h): context management, argument
// checking, state transfer, and the enqueueing of the step, limiter,
// reduction and projection kernels on the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/crkdg.h"
#include "launch.h"

using crk::DevState;
using crk::StepArgs;

const float* crkdg_mlp_device_params(const crkdg_mlp* m);
int crkdg_features_impl(const StepArgs& a, int precision, int k, int basis, const void* u, float* X, float* y,
                        double Mh2, cudaStream_t st);

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(CRKDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct GraphKey {
    int n, start, lim_first, lim_rest;
    bool operator<(const GraphKey& o) const {
        return std::tie(n, start, lim_first, lim_rest) < std::tie(o.n, o.start, o.lim_first, o.lim_rest);
    }
};

}  // namespace

struct crkdg_ctx {
    crkdg_mesh mesh;
    int dim, k, basis, flux, physics, precision;
    double gamma, beta[2];
    crkdg_tableau tab;
    int nv, nm, nqv;
    size_t ncell, elems;
    size_t esize;
    int planes;
    void* u[2];
    int cur;
    double* d_tab;
    DevState* d_state;
    double* d_partials;
    size_t partials_cap;
    unsigned long long* d_flags;
    cudaStream_t stream;
    double t;
    bool t_known;
    bool limiter_on;
    double M;
    bool pending;
    double M_pending;
    double pp_eps;        // positivity floor for following steps (0: off)
    double pp_pending;    // positivity floor of the pending limit
    int seg_rows, wpb;
    int kphys;   // kernel physics id
    void* u3 = nullptr;           // third state copy (RKDG baseline), allocated on first use
    double* d_tab_fe = nullptr;   // forward-Euler tableau (RKDG stages)
    const float* mlp = nullptr;   // learned indicator parameters (device), owned by a crkdg_mlp
    float mlp_zlo = 0.f, mlp_zhi = 0.f;
    int mlp_engine = CRKDG_MLP_TCGEN05;   // crkdg_set_indicator_engine (the limiter pass's inference)
    int limit_mode = CRKDG_LIMIT_PASS;   // where a pending limit runs (crkdg_set_limit_mode)
    double* d_stage = nullptr;            // FP64 staging of state I/O for FP32 states (first use)
    int op_form = CRKDG_FORM_AUTO;        // crkdg_set_operator_form
    int lin_seg_rows = 0, lin_wpb = 0;    // launch shape of the modal linear step (first use)
    bool owns_state = true;               // false: u[0], u[1] are the caller's (crkdg_create_on_buffers)
    std::map<GraphKey, cudaGraphExec_t> graphs;
};

namespace {

// hi + lo FP32 planes: the compensated state, with or without deviation fluxes
bool compensated(int precision) { return precision == CRKDG_F32C || precision == CRKDG_F32D; }

int n_modes(int dim, int k, int basis) {
    if (dim == 1) return k + 1;
    return basis == CRKDG_BASIS_P ? (k + 1) * (k + 2) / 2 : (k + 1) * (k + 1);
}

double dx_of(const crkdg_ctx* c) { return (c->mesh.x1 - c->mesh.x0) / c->mesh.nx; }
double dy_of(const crkdg_ctx* c) { return c->dim == 1 ? 1.0 : (c->mesh.y1 - c->mesh.y0) / c->mesh.ny; }

StepArgs base_args(const crkdg_ctx* c) {
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nx = c->mesh.nx;
    a.ny = c->dim == 1 ? 1 : c->mesh.ny;
    a.x0 = c->mesh.x0;
    a.y0 = c->mesh.y0;
    a.dx = dx_of(c);
    a.dy = dy_of(c);
    a.ds = c->d_state;
    a.partials = c->d_partials;
    a.s = c->tab.s;
    a.tab = c->d_tab;
    for (int s = 0; s < 4; ++s) {
        a.bc[s].type = c->mesh.bc[s];
        a.bc[s].fn = c->mesh.bc_fn[s];
        for (int j = 0; j < 16; ++j) a.bc[s].p[j] = c->mesh.bc_params[s][j];
        for (int j = 0; j < 4; ++j) a.bc[s].pf[j] = (float)a.bc[s].p[j];
    }
    crk::set_bc_affine(a.bc, c->nv);
    a.gamma = c->gamma;
    a.beta[0] = c->beta[0];
    a.beta[1] = c->beta[1];
    return a;
}

// launch geometry of the 2D step
void strips_segs(const crkdg_ctx* c, int seg_rows, int* ns, int* nseg) {
    *ns = (c->mesh.nx + 29) / 30;
    *nseg = (c->mesh.ny + seg_rows - 1) / seg_rows;
}

int ensure_partials(crkdg_ctx* c, size_t n) {
    if (n <= c->partials_cap) return CRKDG_OK;
    if (c->d_partials) cudaFree(c->d_partials);
    c->d_partials = nullptr;
    CK(cudaMalloc(&c->d_partials, n * sizeof(double)));
    c->partials_cap = n;
    return CRKDG_OK;
}

int max_wpb(crkdg_ctx* c) {
    crk::KernelInfo ki;
    CK(crk::info_step2d(c->kphys, c->precision, c->k, c->basis, c->tab.s, &ki));
    int by_regs = std::max(1, ki.max_threads / 32);
    int by_smem = std::max(1, (227 * 1024) / (ki.smem_per_thread * 32));
    return std::min(8, std::min(by_regs, by_smem));
}

// Segment rows for which the step kernel's warps fill the resident slots of
// the device's SMs `waves` times over (registers and private shared memory of the
// kernel decide the slots; blocks of w warps), segments of >= 1 row.  On a
// mesh too small to fill the slots the segments get short: a warp marches
// through its rows one after another, so the step takes about (rows + 2)
// row times however few warps run (the vortex Q^2 RK4 step at 80^2 took
// 2.94 ms in FP64 and 0.185 ms in the deviation form with 8-row segments,
// 0.78 and 0.052 ms with 1-row segments).
int wave_rows(crkdg_ctx* c, int w, int waves, int* rows) {
    const int ns = (c->mesh.nx + 29) / 30;
    crk::KernelInfo ki;
    CK(crk::info_step2d(c->kphys, c->precision, c->k, c->basis, c->tab.s, &ki));
    const int regs_warp = ((ki.regs + 7) / 8) * 8 * 32;
    const int by_regs = 65536 / regs_warp;
    const int by_smem = (228 * 1024) / std::max(1, ki.smem_per_thread * 32);
    int resident = std::min(64, std::min(by_regs, by_smem));
    resident = std::max(w, resident / w * w);
    const long target = (long)std::max(1, crk::sm_count()) * resident * waves;
    const long nseg = std::max(1L, target / ns);
    int L = (int)std::max(1L, ((long)c->mesh.ny + nseg - 1) / nseg);
    *rows = std::min(L, c->mesh.ny);
    return CRKDG_OK;
}

int default_launch(crkdg_ctx* c) {
    if (c->dim != 2) return CRKDG_OK;
    int w = max_wpb(c);
    if (w < 0) return w;
    c->wpb = std::min(w, 4);
    // one wave: as many warps as the SMs hold at once
    return wave_rows(c, c->wpb, 1, &c->seg_rows);
}

int enqueue_reduce(crkdg_ctx* c, int set_dt) {
    const int blocks = 4 * std::max(1, crk::sm_count());
    int r = ensure_partials(c, (size_t)blocks * 8 * 8);
    if (r) return r;
    CK(crk::launch_reduce(c->dim, c->kphys, c->precision, c->u[c->cur], c->mesh.nx, c->dim == 1 ? 1 : c->mesh.ny, c->nm,
                          dx_of(c), dy_of(c), c->gamma, c->beta[0], c->beta[1], c->d_state, c->d_partials, blocks,
                          set_dt, c->stream));
    return CRKDG_OK;
}

// the modal step applies: linear flux, 2D, FP32/FP64, every non-periodic side
// affine (outflow, wall, constant state), not switched off
bool use_linear(const crkdg_ctx* c) {
    if (c->op_form != CRKDG_FORM_AUTO || c->kphys != crk::PHYS_ADV || c->dim != 2 ||
        compensated(c->precision))
        return false;
    crk::BCSide bc[4];
    for (int s = 0; s < 4; ++s) {
        bc[s].type = c->mesh.bc[s];
        bc[s].fn = c->mesh.bc_fn[s];
        for (int j = 0; j < 16; ++j) bc[s].p[j] = c->mesh.bc_params[s][j];
    }
    crk::set_bc_affine(bc, 1);
    for (int s = 0; s < 4; ++s)
        if (bc[s].type != crk::BC_PERIODIC && !bc[s].affine) return false;
    return true;
}

// one wave of the modal step: as many warps as its registers and shared
// memory let the device's SMs hold, segments of >= 1 row
int linear_shape(crkdg_ctx* c) {
    if (c->lin_seg_rows > 0) return CRKDG_OK;
    crk::KernelInfo ki;
    CK(crk::info_step2d_linear(c->precision, c->k, c->basis, c->tab.s, &ki));
    const int wpb = std::max(1, std::min(4, ki.max_threads / 32));
    const int regs_warp = ((ki.regs + 7) / 8) * 8 * 32;
    const int by_regs = 65536 / regs_warp;
    const int by_smem = (228 * 1024) / std::max(1, ki.smem_per_thread * 32);
    int resident = std::min(64, std::min(by_regs, by_smem));
    resident = std::max(wpb, resident / wpb * wpb);
    const int ns = (c->mesh.nx + 29) / 30;
    const long nseg = std::max(1L, (long)std::max(1, crk::sm_count()) * resident / ns);
    const int L = (int)std::max(1L, ((long)c->mesh.ny + nseg - 1) / nseg);
    c->lin_seg_rows = std::min(L, c->mesh.ny);
    c->lin_wpb = wpb;
    return CRKDG_OK;
}

// the pending limit as an in-place pass over u[cur]; troubled cells are
// counted into the run state, where the next step's epilogue reports them
int enqueue_limit_pass(crkdg_ctx* c, double M, int dt_from_dev) {
    StepArgs a = base_args(c);
    a.M = M;
    a.pp_eps = c->pp_pending;
    a.t = c->t;
    a.dt_from_dev = dt_from_dev;
    if (c->mlp && M >= 0.0) {
        // the learned indicator decides (TVB test in its uncertainty band)
        a.mlp = c->mlp;
        a.mlp_zlo = c->mlp_zlo;
        a.mlp_zhi = c->mlp_zhi;
        if (c->mlp_engine == CRKDG_MLP_TCGEN05)
            CK(crk::limit2d_euler_f32_mlp_tc(c->k, c->basis, a, c->u[c->cur], &c->d_state->lim_count, c->stream));
        else
            CK(crk::limit2d_euler_f32_mlp(c->k, c->basis, a, c->u[c->cur], &c->d_state->lim_count, c->stream));
        return CRKDG_OK;
    }
    CK(crk::launch_limit2d(c->kphys, c->precision, c->k, c->basis, a, c->u[c->cur], &c->d_state->lim_count,
                           c->stream));
    return CRKDG_OK;
}

int enqueue_limit(crkdg_ctx* c, double M) {
    StepArgs a = base_args(c);
    a.M = M;
    a.pp_eps = c->pp_pending;
    a.t = c->t;
    CK(crk::launch_limit2d(c->kphys, c->precision, c->k, c->basis, a, c->u[c->cur], c->d_flags, c->stream));
    return CRKDG_OK;
}

// enqueue one 2D/1D step from u[cur] into u[cur^1]
int enqueue_step(crkdg_ctx* c, double dt, int dt_from_dev, int limit, double M) {
    StepArgs a = base_args(c);
    a.uin = c->u[c->cur];
    a.uout = c->u[c->cur ^ 1];
    a.t = c->t;
    a.dt = dt;
    a.dt_from_dev = dt_from_dev;
    a.limit = limit;
    a.M = M;
    a.pp_eps = limit ? c->pp_pending : 0.0;
    if (c->dim == 2) {
        int ns, nseg;
        strips_segs(c, c->seg_rows, &ns, &nseg);
        a.seg_len = c->seg_rows;
        a.n_strips = ns;
        a.n_segs = nseg;
        int r = ensure_partials(c, (size_t)ns * nseg * 8);
        if (r) return r;
        a.partials = c->d_partials;
        if (c->mlp && limit && M >= 0.0 && c->limit_mode == CRKDG_LIMIT_FUSED) {
            a.mlp = c->mlp;
            a.mlp_zlo = c->mlp_zlo;
            a.mlp_zhi = c->mlp_zhi;
            CK(crk::step2d_euler_f32_mlp(c->k, c->basis, a, c->wpb, c->stream));
        } else {
            if (limit && c->limit_mode == CRKDG_LIMIT_PASS) {
                // the pending limit as its own in-place pass over u^n; the
                // step then loads the limited state as it is
                int r = enqueue_limit_pass(c, M, dt_from_dev);
                if (r) return r;
                a.limit = 0;
            }
            if (!a.limit && use_linear(c)) {
                int r = linear_shape(c);
                if (r) return r;
                int lns, lnseg;
                strips_segs(c, c->lin_seg_rows, &lns, &lnseg);
                a.seg_len = c->lin_seg_rows;
                a.n_strips = lns;
                a.n_segs = lnseg;
                r = ensure_partials(c, (size_t)lns * lnseg * 8);
                if (r) return r;
                a.partials = c->d_partials;
                // gamma_l = b^T A^l 1 of the tableau (FP64, host)
                const int s = c->tab.s;
                double v[crk::MAXS];
                for (int i = 0; i < s; ++i) v[i] = 1.0;
                for (int l = 0; l < crk::MAXS; ++l) {
                    double g = 0.0;
                    if (l < s)
                        for (int i = 0; i < s; ++i) g += c->tab.b[i] * v[i];
                    a.lin_gamma[l] = g;
                    a.lin_gammaf[l] = (float)g;
                    double nv[crk::MAXS];
                    for (int i = 0; i < s; ++i) {
                        nv[i] = 0.0;
                        for (int j = 0; j < s; ++j) nv[i] += c->tab.a[i * CRKDG_MAX_STAGES + j] * v[j];
                    }
                    for (int i = 0; i < s; ++i) v[i] = nv[i];
                }
                a.lin_inflow = (a.beta[0] > 0.0 ? 1 : 0) | (a.beta[0] < 0.0 ? 2 : 0) | (a.beta[1] > 0.0 ? 4 : 0) |
                               (a.beta[1] < 0.0 ? 8 : 0);
                CK(crk::launch_step2d_linear(c->precision, c->k, c->basis, a, c->lin_wpb, c->stream));
            } else {
                CK(crk::launch_step2d(c->kphys, c->precision, c->k, c->basis, a, c->wpb, c->stream));
            }
        }
    } else {
        const int warps = (c->mesh.nx + 29) / 30;
        const int blocks = (warps + 7) / 8;
        CK(crk::launch_step1d(c->kphys, c->precision, c->k, a, 1, blocks == 1 ? warps * 32 : 256, blocks, c->stream));
    }
    c->cur ^= 1;
    return CRKDG_OK;
}

int check_ctx(const crkdg_ctx* c) { return c ? CRKDG_OK : fail(CRKDG_EINVAL, "null context"); }

__global__ void set_run_params(DevState* ds, double cfl, double t_end) {
    ds->cfl = cfl;
    ds->t_end = t_end;
}

}  // namespace

namespace {

// the values of one state copy for these arguments (host arithmetic only)
size_t state_values(const crkdg_mesh* mesh, int k, int basis, int physics, int precision) {
    const int dim = mesh->dim;
    const size_t ncell = (size_t)mesh->nx * (dim == 2 ? mesh->ny : 1);
    const int nv = physics == CRKDG_ADVECTION ? 1 : (dim == 1 ? 3 : 4);
    const int nm = n_modes(dim, k, dim == 1 ? CRKDG_BASIS_P : basis);
    return ncell * nv * nm * (compensated(precision) ? 2 : 1);
}

}  // namespace

namespace {

int create_impl(const crkdg_mesh* mesh, int k, int basis, int flux, const crkdg_tableau* tab, double gamma,
                int physics, int precision, const double* phys_params, void* stream, void* buf_a, void* buf_b,
                crkdg_ctx** out) {
    if (!mesh || !tab || !out) return fail(CRKDG_EINVAL, "null argument");
    *out = nullptr;
    if (mesh->dim != 1 && mesh->dim != 2) return fail(CRKDG_EINVAL, "dim must be 1 or 2");
    if (mesh->nx < 1 || (mesh->dim == 2 && mesh->ny < 1)) return fail(CRKDG_EINVAL, "mesh must have cells");
    if (!(mesh->x1 > mesh->x0) || (mesh->dim == 2 && !(mesh->y1 > mesh->y0)))
        return fail(CRKDG_EINVAL, "empty domain");
    if ((long long)mesh->nx * (mesh->dim == 2 ? mesh->ny : 1) > (1LL << 30))
        return fail(CRKDG_EINVAL, "mesh too large (more than 2^30 cells)");
    if (k < 0 || k > 3) return fail(CRKDG_EUNSUPPORTED, "k must be 0..3");
    if (basis != CRKDG_BASIS_P && basis != CRKDG_BASIS_Q) return fail(CRKDG_EINVAL, "basis must be P or Q");
    if (flux != CRKDG_FLUX_LLF) return fail(CRKDG_EINVAL, "flux must be CRKDG_FLUX_LLF");
    if (physics != CRKDG_ADVECTION && physics != CRKDG_EULER) return fail(CRKDG_EINVAL, "unknown physics");
    if (precision != CRKDG_F32 && precision != CRKDG_F64 && !compensated(precision))
        return fail(CRKDG_EINVAL, "unknown precision");
    if (compensated(precision) && (physics != CRKDG_EULER || mesh->dim != 2))
        return fail(CRKDG_EUNSUPPORTED, "the compensated FP32 state is built for 2D Euler");
    if (tab->s < 1 || tab->s > CRKDG_MAX_STAGES) return fail(CRKDG_EINVAL, "tableau stages must be 1..6");
    for (int i = 0; i < tab->s; ++i)
        for (int j = i; j < CRKDG_MAX_STAGES; ++j)
            if (tab->a[i * CRKDG_MAX_STAGES + j] != 0.0)
                return fail(CRKDG_EINVAL, "tableau must be explicit (a strictly lower triangular)");
    if (physics == CRKDG_EULER && !(gamma > 1.0)) return fail(CRKDG_EINVAL, "gamma must exceed 1");
    if (physics == CRKDG_ADVECTION && !phys_params) return fail(CRKDG_EINVAL, "advection needs beta");
    const int ns = mesh->dim == 1 ? 2 : 4;
    for (int s = 0; s < ns; ++s) {
        const int b = mesh->bc[s];
        if (b < 0 || b > 3) return fail(CRKDG_EINVAL, "unknown boundary condition");
        if (b == CRKDG_BC_REFLECT && physics != CRKDG_EULER) return fail(CRKDG_EINVAL, "reflect needs Euler");
        if (b == CRKDG_BC_DIRICHLET && (mesh->bc_fn[s] < 0 || mesh->bc_fn[s] > 4))
            return fail(CRKDG_EINVAL, "unknown boundary function");
    }
    if ((mesh->bc[0] == CRKDG_BC_PERIODIC) != (mesh->bc[1] == CRKDG_BC_PERIODIC))
        return fail(CRKDG_EINVAL, "periodic W/E must come in pairs");
    if (mesh->dim == 2 && (mesh->bc[2] == CRKDG_BC_PERIODIC) != (mesh->bc[3] == CRKDG_BC_PERIODIC))
        return fail(CRKDG_EINVAL, "periodic S/N must come in pairs");

    crkdg_ctx* c = new crkdg_ctx();
    c->mesh = *mesh;
    if (mesh->dim == 1) {
        c->mesh.ny = 1;
        c->mesh.y0 = 0.0;
        c->mesh.y1 = 1.0;
        c->mesh.bc[2] = c->mesh.bc[3] = CRKDG_BC_PERIODIC;
    }
    c->dim = mesh->dim;
    c->k = k;
    c->basis = mesh->dim == 1 ? CRKDG_BASIS_P : basis;
    c->flux = flux;
    c->physics = physics;
    c->precision = precision;
    c->gamma = gamma;
    c->beta[0] = phys_params && physics == CRKDG_ADVECTION ? phys_params[0] : 0.0;
    c->beta[1] = phys_params && physics == CRKDG_ADVECTION && mesh->dim == 2 ? phys_params[1] : 0.0;
    c->tab = *tab;
    c->nv = physics == CRKDG_ADVECTION ? 1 : (mesh->dim == 1 ? 3 : 4);
    c->nm = n_modes(mesh->dim, k, c->basis);
    c->nqv = mesh->dim == 1 ? k + 1 : (k + 1) * (k + 1);
    c->ncell = (size_t)c->mesh.nx * c->mesh.ny;
    c->elems = c->ncell * c->nv * c->nm;
    c->esize = precision == CRKDG_F64 ? 8 : 4;
    c->planes = compensated(precision) ? 2 : 1;   // compensated: hi planes then lo planes
    c->kphys = physics == CRKDG_ADVECTION ? crk::PHYS_ADV : (mesh->dim == 1 ? crk::PHYS_EULER1D : crk::PHYS_EULER);
    c->stream = static_cast<cudaStream_t>(stream);
    c->t = 0.0;
    c->t_known = true;
    c->M = -1.0;
    c->seg_rows = 8;
    c->wpb = 4;
    auto bail = [&](int code) {
        crkdg_destroy(c);
        return code;
    };
    if (buf_a) {   // the caller's copies: kept as they are (the state starts as buf_a's contents)
        c->owns_state = false;
        c->u[0] = buf_a;
        c->u[1] = buf_b;
    } else {
        for (int b = 0; b < 2; ++b) {
            if (cudaMalloc(&c->u[b], c->elems * c->esize * c->planes) != cudaSuccess)
                return bail(fail(CRKDG_ENOMEM, "cudaMalloc of the state failed"));
            cudaMemsetAsync(c->u[b], 0, c->elems * c->esize * c->planes, c->stream);
        }
    }
    unsigned char htab[crk::TAB_BYTES];
    crk::pack_tableau(tab->s, tab->a, tab->b, tab->c, htab);
    if (cudaMalloc(&c->d_tab, sizeof(htab)) != cudaSuccess ||
        cudaMalloc(&c->d_state, sizeof(DevState)) != cudaSuccess ||
        cudaMalloc(&c->d_flags, sizeof(unsigned long long)) != cudaSuccess)
        return bail(fail(CRKDG_ENOMEM, "cudaMalloc failed"));
    if (cudaMemcpy(c->d_tab, htab, sizeof(htab), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(CRKDG_ECUDA, "copy of the tableau failed"));
    DevState ds;
    std::memset(&ds, 0, sizeof(ds));
    if (cudaMemcpy(c->d_state, &ds, sizeof(ds), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_flags, 0, sizeof(unsigned long long)) != cudaSuccess)
        return bail(fail(CRKDG_ECUDA, "initialisation of the device state failed"));
    int r = ensure_partials(c, 4096);
    if (r) return bail(r);
    r = default_launch(c);
    if (r) return bail(r);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(fail(CRKDG_ECUDA, "stream sync failed"));
    *out = c;
    return CRKDG_OK;
}

}  // namespace

extern "C" {

const char* crkdg_last_error(void) { return g_err.c_str(); }
const char* crkdg_version(void) { return "crkdg-gb300 1.0 (sm_103a)"; }


int crkdg_state_bytes(const crkdg_mesh* mesh, int k, int basis, int physics, int precision, size_t* bytes) {
    if (!mesh || !bytes) return fail(CRKDG_EINVAL, "null argument");
    if ((mesh->dim != 1 && mesh->dim != 2) || mesh->nx < 1 || (mesh->dim == 2 && mesh->ny < 1) || k < 0 || k > 3 ||
        (basis != CRKDG_BASIS_P && basis != CRKDG_BASIS_Q) ||
        (physics != CRKDG_ADVECTION && physics != CRKDG_EULER) ||
        (precision != CRKDG_F32 && precision != CRKDG_F64 && !compensated(precision)))
        return fail(CRKDG_EINVAL, "bad mesh, degree, basis, physics or precision");
    *bytes = state_values(mesh, k, basis, physics, precision) * (precision == CRKDG_F64 ? 8 : 4);
    return CRKDG_OK;
}

int crkdg_create(const crkdg_mesh* mesh, int k, int basis, int flux, const crkdg_tableau* tab, double gamma,
                 int physics, int precision, const double* phys_params, void* stream, crkdg_ctx** out) {
    return create_impl(mesh, k, basis, flux, tab, gamma, physics, precision, phys_params, stream, nullptr, nullptr,
                       out);
}

int crkdg_create_on_buffers(const crkdg_mesh* mesh, int k, int basis, int flux, const crkdg_tableau* tab,
                            double gamma, int physics, int precision, const double* phys_params, void* stream,
                            void* state_a, void* state_b, crkdg_ctx** out) {
    if (!out) return fail(CRKDG_EINVAL, "null argument");
    *out = nullptr;
    if (!state_a || !state_b) return fail(CRKDG_EINVAL, "null state buffer");
    size_t bytes = 0;
    int r = crkdg_state_bytes(mesh, k, basis, physics, precision, &bytes);
    if (r) return r;
    const uintptr_t a = reinterpret_cast<uintptr_t>(state_a), b = reinterpret_cast<uintptr_t>(state_b);
    if (a % 16 != 0 || b % 16 != 0) return fail(CRKDG_EINVAL, "state buffers must be 16-byte aligned");
    if ((a < b ? b - a : a - b) < bytes) return fail(CRKDG_EINVAL, "state buffers overlap");
    // both must be device memory of the current device
    for (void* p : {state_a, state_b}) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return fail(CRKDG_EINVAL, "state buffers must be device memory");
        }
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess || at.device != dev)
            return fail(CRKDG_EINVAL, "state buffers must be on the current device");
    }
    return create_impl(mesh, k, basis, flux, tab, gamma, physics, precision, phys_params, stream, state_a, state_b,
                       out);
}

int crkdg_current_state(const crkdg_ctx* c, int* which, void** dev_ptr) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (which) *which = c->cur;
    if (dev_ptr) *dev_ptr = c->u[c->cur];
    return CRKDG_OK;
}


void crkdg_destroy(crkdg_ctx* c) {
    if (!c) return;
    if (c->stream || true) cudaStreamSynchronize(c->stream);
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    if (c->owns_state)
        for (int b = 0; b < 2; ++b)
            if (c->u[b]) cudaFree(c->u[b]);
    if (c->d_tab) cudaFree(c->d_tab);
    if (c->d_state) cudaFree(c->d_state);
    if (c->d_partials) cudaFree(c->d_partials);
    if (c->d_flags) cudaFree(c->d_flags);
    if (c->u3) cudaFree(c->u3);
    if (c->d_stage) cudaFree(c->d_stage);
    if (c->d_tab_fe) cudaFree(c->d_tab_fe);
    delete c;
}

int crkdg_sizes(const crkdg_ctx* c, int* n_cells, int* n_modes_, int* n_vars, int* n_qp) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (n_cells) *n_cells = (int)c->ncell;
    if (n_modes_) *n_modes_ = c->nm;
    if (n_vars) *n_vars = c->nv;
    if (n_qp) *n_qp = c->nqv;
    return CRKDG_OK;
}

int crkdg_quadrature_points(const crkdg_ctx* c, double* xy) {
    if (check_ctx(c) || !xy) return fail(CRKDG_EINVAL, "null argument");
    const crk::GaussRule g = crk::gauss_rule(c->k + 1);
    const double dx = dx_of(c), dy = dy_of(c);
    const int nq = c->k + 1;
    size_t o = 0;
    for (int y = 0; y < c->mesh.ny; ++y)
        for (int x = 0; x < c->mesh.nx; ++x) {
            const double xc = c->mesh.x0 + (x + 0.5) * dx, yc = c->mesh.y0 + (y + 0.5) * dy;
            if (c->dim == 1) {
                for (int q = 0; q < nq; ++q) xy[o++] = xc + 0.5 * dx * g.x[q];
            } else {
                for (int a = 0; a < nq; ++a)
                    for (int b = 0; b < nq; ++b) {
                        xy[o++] = xc + 0.5 * dx * g.x[a];
                        xy[o++] = yc + 0.5 * dy * g.x[b];
                    }
            }
        }
    return CRKDG_OK;
}

int crkdg_project_ic(crkdg_ctx* c, const double* values) {
    if (check_ctx(c) || !values) return fail(CRKDG_EINVAL, "null argument");
    const size_t n = c->ncell * c->nqv * c->nv;
    double* d = nullptr;
    if (cudaMalloc(&d, n * sizeof(double)) != cudaSuccess) return fail(CRKDG_ENOMEM, "cudaMalloc failed");
    cudaError_t e = cudaMemcpyAsync(d, values, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = crk::launch_project(c->dim, c->kphys, c->precision, c->k, c->basis, d, c->u[c->cur], (int)c->ncell,
                                c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(CRKDG_ECUDA, std::string("project_ic: ") + cudaGetErrorString(e));
    c->t = 0.0;
    c->t_known = true;
    c->pending = false;
    CK(cudaMemcpy(&c->d_state->t, &c->t, sizeof(double), cudaMemcpyHostToDevice));
    return CRKDG_OK;
}

int crkdg_set_state(crkdg_ctx* c, const double* h, double t) {
    if (check_ctx(c) || !h) return fail(CRKDG_EINVAL, "null argument");
    if (c->precision == CRKDG_F64) {
        CK(cudaMemcpyAsync(c->u[c->cur], h, c->elems * 8, cudaMemcpyHostToDevice, c->stream));
    } else {
        // FP64 over the link, rounded to the FP32 state on the GPU
        if (!c->d_stage && cudaMalloc(&c->d_stage, c->elems * 8) != cudaSuccess) {
            c->d_stage = nullptr;
            return fail(CRKDG_ENOMEM, "cudaMalloc of the state staging buffer failed");
        }
        CK(cudaMemcpyAsync(c->d_stage, h, c->elems * 8, cudaMemcpyHostToDevice, c->stream));
        CK(crk::launch_f64_to_f32(c->d_stage, static_cast<float*>(c->u[c->cur]), c->elems, c->planes == 2, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    c->t = t;
    c->t_known = true;
    c->pending = false;
    CK(cudaMemcpyAsync(&c->d_state->t, &c->t, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return CRKDG_OK;
}

int crkdg_get_state(crkdg_ctx* c, double* h) {
    if (check_ctx(c) || !h) return fail(CRKDG_EINVAL, "null argument");
    if (c->pending && c->dim == 2) {
        if (!c->t_known) {
            CK(cudaMemcpyAsync(&c->t, &c->d_state->t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            c->t_known = true;
        }
        int r = enqueue_limit(c, c->M_pending);
        if (r) return r;
        c->pending = false;
    }
    if (c->precision == CRKDG_F64) {
        CK(cudaMemcpyAsync(h, c->u[c->cur], c->elems * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        // widened to FP64 on the GPU, FP64 over the link
        if (!c->d_stage && cudaMalloc(&c->d_stage, c->elems * 8) != cudaSuccess) {
            c->d_stage = nullptr;
            return fail(CRKDG_ENOMEM, "cudaMalloc of the state staging buffer failed");
        }
        CK(crk::launch_f32_to_f64(static_cast<const float*>(c->u[c->cur]), c->d_stage, c->elems, c->planes == 2,
                                  c->stream));
        CK(cudaMemcpyAsync(h, c->d_stage, c->elems * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return CRKDG_OK;
}

int crkdg_cfl_dt(crkdg_ctx* c, double cfl, double* dt_out) {
    if (check_ctx(c) || !dt_out) return fail(CRKDG_EINVAL, "null argument");
    if (!(cfl > 0.0)) return fail(CRKDG_EINVAL, "cfl must be positive");
    int r = enqueue_reduce(c, 0);
    if (r) return r;
    double ms = 0.0;
    CK(cudaMemcpyAsync(&ms, &c->d_state->maxspeed, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (!(ms > 0.0) || !std::isfinite(ms)) return fail(CRKDG_ENONPHYSICAL, "wave speed is zero or not finite");
    *dt_out = cfl / ms;
    return CRKDG_OK;
}

int crkdg_step(crkdg_ctx* c, double dt) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(CRKDG_EINVAL, "dt must be positive and finite");
    if (!c->t_known) {
        CK(cudaMemcpyAsync(&c->t, &c->d_state->t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->t_known = true;
    }
    const int lim = c->pending && c->dim == 2;
    int r = enqueue_step(c, dt, 0, lim, lim ? c->M_pending : 0.0);
    if (r) return r;
    c->t += dt;
    c->pending = (c->limiter_on || c->pp_eps > 0.0) && c->dim == 2;
    c->M_pending = c->M;
    c->pp_pending = c->pp_eps;
    return CRKDG_OK;
}

int crkdg_advance(crkdg_ctx* c, int n_steps, double cfl, double t_end, int capture) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (c->dim != 2) return fail(CRKDG_EUNSUPPORTED, "crkdg_advance is 2D only (use crkdg_run_fixed in 1D)");
    if (n_steps < 0) return fail(CRKDG_EINVAL, "n_steps must be >= 0");
    if (!(cfl > 0.0)) return fail(CRKDG_EINVAL, "cfl must be positive");
    if (n_steps == 0) return CRKDG_OK;
    // run parameters and the first dt from the current state
    set_run_params<<<1, 1, 0, c->stream>>>(c->d_state, cfl, t_end);
    CK(cudaGetLastError());
    int r = enqueue_reduce(c, 1);
    if (r) return r;
    const int lim_first = c->pending ? 1 : 0;
    const int lim_rest = (c->limiter_on || c->pp_eps > 0.0) ? 1 : 0;
    const double M_first = c->M_pending, M_rest = c->M;
    const double pp_first = c->pp_pending, pp_rest = c->pp_eps;
    int ns, nseg;
    strips_segs(c, c->seg_rows, &ns, &nseg);
    r = ensure_partials(c, (size_t)ns * nseg * 8);
    if (r) return r;
    if (use_linear(c)) {   // slots of the modal step too: nothing may allocate while a graph is captured
        r = linear_shape(c);
        if (r) return r;
        strips_segs(c, c->lin_seg_rows, &ns, &nseg);
        r = ensure_partials(c, (size_t)ns * nseg * 8);
        if (r) return r;
    }
    auto enqueue_all = [&]() -> int {
        for (int i = 0; i < n_steps; ++i) {
            const int lim = i == 0 ? lim_first : lim_rest;
            c->pp_pending = i == 0 ? pp_first : pp_rest;
            int rr = enqueue_step(c, 0.0, 1, lim, i == 0 ? M_first : M_rest);
            if (rr) return rr;
        }
        return CRKDG_OK;
    };
    if (!capture) {
        r = enqueue_all();
        if (r) return r;
    } else {
        GraphKey key{n_steps, c->cur, lim_first, lim_rest};
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            if (c->stream == nullptr) return fail(CRKDG_EINVAL, "graph capture needs a non-default stream");
            const int cur0 = c->cur;
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            r = enqueue_all();
            cudaError_t e = cudaStreamEndCapture(c->stream, &g);
            if (r) return r;
            if (e != cudaSuccess) return fail(CRKDG_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
            cudaGraphExec_t ge;
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(CRKDG_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
            it = c->graphs.emplace(key, ge).first;
            c->cur = cur0;   // capture recorded but did not run the steps
        }
        CK(cudaGraphLaunch(it->second, c->stream));
        if (n_steps % 2) c->cur ^= 1;
    }
    c->t_known = false;
    c->pending = c->limiter_on || c->pp_eps > 0.0;
    c->M_pending = c->M;
    c->pp_pending = c->pp_eps;
    return CRKDG_OK;
}

int crkdg_step_device(crkdg_ctx* c) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (c->dim != 2) return fail(CRKDG_EUNSUPPORTED, "crkdg_step_device is 2D only");
    const int lim = c->pending ? 1 : 0;
    int r = enqueue_step(c, 0.0, 1, lim, c->M_pending);
    if (r) return r;
    c->t_known = false;
    c->pending = c->limiter_on || c->pp_eps > 0.0;
    c->M_pending = c->M;
    c->pp_pending = c->pp_eps;
    return CRKDG_OK;
}

// one forward-Euler DG step out = in - dt div^DG f(in) at time t (the
// fused step kernel with a one-stage tableau), no limiting on load
static int enqueue_fe(crkdg_ctx* c, const void* in, void* out, double t, double dt) {
    StepArgs a = base_args(c);
    a.uin = in;
    a.uout = out;
    a.t = t;
    a.dt = dt;
    a.s = 1;
    a.tab = c->d_tab_fe;
    int ns, nseg;
    strips_segs(c, c->seg_rows, &ns, &nseg);
    a.seg_len = c->seg_rows;
    a.n_strips = ns;
    a.n_segs = nseg;
    int r = ensure_partials(c, (size_t)ns * nseg * 8);
    if (r) return r;
    a.partials = c->d_partials;
    CK(crk::launch_step2d(c->kphys, c->precision, c->k, c->basis, a, c->wpb, c->stream));
    return CRKDG_OK;
}

static int enqueue_limit_buf(crkdg_ctx* c, void* u, double t, double M, double pp) {
    if (M < 0.0 && !(pp > 0.0)) return CRKDG_OK;
    StepArgs a = base_args(c);
    a.M = M;
    a.pp_eps = pp;
    a.t = t;
    CK(crk::launch_limit2d(c->kphys, c->precision, c->k, c->basis, a, u, c->d_flags, c->stream));
    return CRKDG_OK;
}

int crkdg_rkdg_step(crkdg_ctx* c, double dt, int order) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (c->dim != 2 || compensated(c->precision)) return fail(CRKDG_EUNSUPPORTED, "RKDG is built for 2D FP32/FP64");
    if (order != 2 && order != 3) return fail(CRKDG_EINVAL, "order must be 2 or 3 (Shu--Osher SSP forms)");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(CRKDG_EINVAL, "dt must be positive and finite");
    if (!c->u3) {
        if (cudaMalloc(&c->u3, c->elems * c->esize) != cudaSuccess) return fail(CRKDG_ENOMEM, "cudaMalloc failed");
        const double fa[crk::MAXS * crk::MAXS] = {0}, fb[crk::MAXS] = {1.0}, fc[crk::MAXS] = {0};
        unsigned char fe[crk::TAB_BYTES];
        crk::pack_tableau(1, fa, fb, fc, fe);   // forward Euler: s = 1, b_1 = 1, c_1 = 0
        if (cudaMalloc(&c->d_tab_fe, sizeof(fe)) != cudaSuccess) return fail(CRKDG_ENOMEM, "cudaMalloc failed");
        CK(cudaMemcpy(c->d_tab_fe, fe, sizeof(fe), cudaMemcpyHostToDevice));
    }
    if (!c->t_known) {
        CK(cudaMemcpyAsync(&c->t, &c->d_state->t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->t_known = true;
    }
    const double t = c->t;
    void* U = c->u[c->cur];
    void* A = c->u[c->cur ^ 1];
    void* B = c->u3;
    const double M = c->limiter_on ? c->M : -1.0, pp = c->pp_eps;
    int r = CRKDG_OK;
    // u^n as stored is pending the limiter of the previous step
    if (c->pending) r = enqueue_limit_buf(c, U, t, c->M_pending, c->pp_pending);
    // u1 = Lim(u^n + dt L(u^n)), boundary data at t
    if (!r) r = enqueue_fe(c, U, A, t, dt);
    if (!r) r = enqueue_limit_buf(c, A, t + dt, M, pp);
    if (order == 2) {
        // u^{n+1} = Lim(1/2 u^n + 1/2 (u1 + dt L(u1))), data at t + dt
        if (!r) r = enqueue_fe(c, A, B, t + dt, dt);
        if (!r) CK(crk::launch_axpby(c->precision, A, U, B, 0.5, 0.5, c->elems, c->stream));
    } else {
        // u2 = Lim(3/4 u^n + 1/4 (u1 + dt L(u1))), data at t + dt
        if (!r) r = enqueue_fe(c, A, B, t + dt, dt);
        if (!r) CK(crk::launch_axpby(c->precision, A, U, B, 0.75, 0.25, c->elems, c->stream));
        if (!r) r = enqueue_limit_buf(c, A, t + 0.5 * dt, M, pp);
        // u^{n+1} = Lim(1/3 u^n + 2/3 (u2 + dt L(u2))), data at t + dt/2
        if (!r) r = enqueue_fe(c, A, B, t + 0.5 * dt, dt);
        if (!r) CK(crk::launch_axpby(c->precision, A, U, B, 1.0 / 3.0, 2.0 / 3.0, c->elems, c->stream));
    }
    if (r) return r;
    CK(crk::launch_set_time(c->d_state, t + dt, c->stream));
    c->cur ^= 1;
    c->t = t + dt;
    c->pending = (c->limiter_on || c->pp_eps > 0.0);
    c->M_pending = c->M;
    c->pp_pending = c->pp_eps;
    return CRKDG_OK;
}

int crkdg_run_fixed(crkdg_ctx* c, int n_steps, double dt) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (n_steps < 0 || !(dt > 0.0)) return fail(CRKDG_EINVAL, "need n_steps >= 0 and dt > 0");
    if (c->dim == 2) {
        for (int i = 0; i < n_steps; ++i) {
            int r = crkdg_step(c, dt);
            if (r) return r;
        }
        return CRKDG_OK;
    }
    const int warps = (c->mesh.nx + 29) / 30;
    if (warps > 32) {
        for (int i = 0; i < n_steps; ++i) {
            int r = crkdg_step(c, dt);
            if (r) return r;
        }
        return CRKDG_OK;
    }
    // whole run in one single-block launch
    if (n_steps == 0) return CRKDG_OK;
    StepArgs a = base_args(c);
    a.uin = c->u[c->cur];
    a.uout = c->u[c->cur ^ 1];
    a.t = c->t;
    a.dt = dt;
    CK(crk::launch_step1d(c->kphys, c->precision, c->k, a, n_steps, warps * 32, 1, c->stream));
    if (n_steps % 2) c->cur ^= 1;
    c->t += n_steps * dt;
    return CRKDG_OK;
}

int crkdg_limit(crkdg_ctx* c, double M) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (c->dim != 2) return fail(CRKDG_EUNSUPPORTED, "the TVB limiter is built for 2D meshes");
    if (compensated(c->precision) && M >= 0.0)
        return fail(CRKDG_EUNSUPPORTED, "limiters are not built for the compensated FP32 state");
    if (M >= 0.0) {
        c->limiter_on = true;
        c->M = M;
        c->pending = true;
        c->M_pending = M;
        c->pp_pending = c->pp_eps;
    } else {
        c->limiter_on = false;
        c->M = -1.0;
    }
    return CRKDG_OK;
}

int crkdg_positivity(crkdg_ctx* c, double eps) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (c->dim != 2 || c->physics != CRKDG_EULER)
        return fail(CRKDG_EUNSUPPORTED, "positivity scaling is built for 2D Euler");
    if (compensated(c->precision) && eps > 0.0)
        return fail(CRKDG_EUNSUPPORTED, "limiters are not built for the compensated FP32 state");
    if (eps > 0.0) {
        c->pp_eps = eps;
        if (!c->pending) {
            c->pending = true;
            c->M_pending = -1.0;
        }
        c->pp_pending = eps;
    } else {
        c->pp_eps = 0.0;
    }
    return CRKDG_OK;
}

int crkdg_set_indicator(crkdg_ctx* c, const crkdg_mlp* net, double z_lo, double z_hi) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (!net) {
        c->mlp = nullptr;
        return CRKDG_OK;
    }
    if (c->dim != 2 || c->physics != CRKDG_EULER || c->precision != CRKDG_F32 || c->k != 2)
        return fail(CRKDG_EUNSUPPORTED, "the learned indicator is built for 2D Euler, k = 2, FP32");
    if (!(z_lo <= z_hi)) return fail(CRKDG_EINVAL, "need z_lo <= z_hi");
    c->mlp = crkdg_mlp_device_params(net);
    c->mlp_zlo = (float)z_lo;
    c->mlp_zhi = (float)z_hi;
    return CRKDG_OK;
}

int crkdg_set_indicator_engine(crkdg_ctx* c, int engine) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (engine != CRKDG_MLP_TCGEN05 && engine != CRKDG_MLP_MMA_SYNC)
        return fail(CRKDG_EINVAL, "unknown indicator engine");
    c->mlp_engine = engine;
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    return CRKDG_OK;
}

int crkdg_features(crkdg_ctx* c, float* X_dev, float* y_dev, double M) {
    if (check_ctx(c) || !X_dev || !y_dev) return fail(CRKDG_EINVAL, "null argument");
    if (c->dim != 2 || c->physics != CRKDG_EULER || compensated(c->precision))
        return fail(CRKDG_EUNSUPPORTED, "features are built for 2D Euler FP32/FP64 states");
    if (!(M >= 0.0)) return fail(CRKDG_EINVAL, "M must be >= 0");
    if (!c->t_known) {
        CK(cudaMemcpyAsync(&c->t, &c->d_state->t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->t_known = true;
    }
    StepArgs a = base_args(c);
    a.t = c->t;
    a.M = M;
    const double h = std::max(dx_of(c), dy_of(c));
    int r = crkdg_features_impl(a, c->precision, c->k, c->basis, c->u[c->cur], X_dev, y_dev, M * h * h, c->stream);
    if (r) return fail(r, crkdg_mlp_last_error());
    CK(cudaStreamSynchronize(c->stream));
    return CRKDG_OK;
}

int crkdg_conservation(crkdg_ctx* c, double* sums) {
    if (check_ctx(c) || !sums) return fail(CRKDG_EINVAL, "null argument");
    int r = enqueue_reduce(c, 0);
    if (r) return r;
    CK(cudaMemcpyAsync(sums, c->d_state->sums, c->nv * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return CRKDG_OK;
}

int crkdg_troubled_count(crkdg_ctx* c, unsigned long long* count) {
    if (check_ctx(c) || !count) return fail(CRKDG_EINVAL, "null argument");
    double tr = 0.0;
    CK(cudaMemcpyAsync(&tr, &c->d_state->troubled, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *count = (unsigned long long)tr;
    return CRKDG_OK;
}

int crkdg_sync(crkdg_ctx* c, unsigned* device_status) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    unsigned st = 0;
    CK(cudaMemcpy(&st, &c->d_state->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    CK(cudaMemset(&c->d_state->status, 0, sizeof(unsigned)));
    if (device_status) *device_status = st;
    if (st & crk::ST_TIMEOUT) return fail(CRKDG_ETIMEOUT, "a bounded device wait ran out");
    if (st) return fail(CRKDG_ENONPHYSICAL, "non-physical or NaN state seen on the device");
    return CRKDG_OK;
}

int crkdg_time(const crkdg_ctx* cc, double* t) {
    crkdg_ctx* c = const_cast<crkdg_ctx*>(cc);
    if (check_ctx(c) || !t) return fail(CRKDG_EINVAL, "null argument");
    if (!c->t_known) {
        CK(cudaMemcpyAsync(&c->t, &c->d_state->t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->t_known = true;
    }
    *t = c->t;
    return CRKDG_OK;
}

int crkdg_step_count(crkdg_ctx* c, unsigned long long* steps) {
    if (check_ctx(c) || !steps) return fail(CRKDG_EINVAL, "null argument");
    if (c->dim != 2) return fail(CRKDG_EUNSUPPORTED, "the step counter is kept by the 2D step");
    CK(cudaMemcpyAsync(steps, &c->d_state->steps, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return CRKDG_OK;
}

int crkdg_run_state_async(crkdg_ctx* c, double* out) {
    if (check_ctx(c) || !out) return fail(CRKDG_EINVAL, "null argument");
    static_assert(offsetof(DevState, maxspeed) == 4 * sizeof(double), "run state layout");
    CK(cudaMemcpyAsync(out, c->d_state, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return CRKDG_OK;
}

int crkdg_set_launch(crkdg_ctx* c, int seg_rows, int wpb) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (seg_rows < 0 || wpb < 0) return fail(CRKDG_EINVAL, "negative launch shape");
    if (wpb > 0) {
        const int mx = max_wpb(c);
        if (mx < 0) return mx;
        if (wpb > mx) return fail(CRKDG_EINVAL, "warps per block exceeds the kernel's register/shared-memory limit");
        c->wpb = wpb;
    }
    if (seg_rows > 0) c->seg_rows = std::min(seg_rows, c->mesh.ny);
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    return CRKDG_OK;
}

int crkdg_apply_limit(crkdg_ctx* c) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (c->dim != 2 || !c->pending) return CRKDG_OK;
    int r = enqueue_limit_pass(c, c->M_pending, c->t_known ? 0 : 1);
    if (r) return r;
    c->pending = false;
    return CRKDG_OK;
}

int crkdg_set_limit_mode(crkdg_ctx* c, int mode) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (mode != CRKDG_LIMIT_FUSED && mode != CRKDG_LIMIT_PASS) return fail(CRKDG_EINVAL, "unknown limit mode");
    c->limit_mode = mode;
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    return CRKDG_OK;
}

int crkdg_set_operator_form(crkdg_ctx* c, int form) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (form != CRKDG_FORM_QUADRATURE && form != CRKDG_FORM_AUTO) return fail(CRKDG_EINVAL, "unknown operator form");
    c->op_form = form;
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    return CRKDG_OK;
}

int crkdg_get_operator_form(const crkdg_ctx* c, int* form) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (form) *form = c->op_form;
    return CRKDG_OK;
}

int crkdg_get_limit_mode(const crkdg_ctx* c, int* mode) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (mode) *mode = c->limit_mode;
    return CRKDG_OK;
}

int crkdg_get_launch(const crkdg_ctx* c, int* seg_rows, int* wpb) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (seg_rows) *seg_rows = c->seg_rows;
    if (wpb) *wpb = c->wpb;
    return CRKDG_OK;
}

int crkdg_autotune(crkdg_ctx* c, double* best_us) {
    if (check_ctx(c)) return CRKDG_EINVAL;
    if (c->dim != 2) return fail(CRKDG_EUNSUPPORTED, "autotune is for the 2D step");
    // time candidate shapes on the current state; u[cur] is only read, the
    // device run state is saved and restored around the trials.  A limit
    // pending in pass mode is applied first (in place, as the next step
    // would), so the trials time the step kernel as a pass-mode step runs it
    if (c->pending && c->limit_mode == CRKDG_LIMIT_PASS) {
        if (!c->t_known) {
            CK(cudaMemcpy(&c->t, &c->d_state->t, sizeof(double), cudaMemcpyDeviceToHost));
            c->t_known = true;
        }
        int r = enqueue_limit_pass(c, c->M_pending, 0);
        if (r) return r;
        c->pending = false;
    }
    DevState saved;
    CK(cudaMemcpyAsync(&saved, c->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int mx = max_wpb(c);
    if (mx < 0) return mx;
    // candidates: the current shape first (tuning never makes it worse), the
    // one- and two-wave shapes of every block size, then a fixed ladder
    const int rows[] = {4, 6, 8, 12, 16, 24, 32, 48, 64, 96};
    const int wpbs[] = {1, 2, 4, 8};
    std::vector<std::pair<int, int>> cand;
    auto add = [&](int L, int w) {
        L = std::max(1, std::min(L, c->mesh.ny));
        for (auto& p : cand)
            if (p.first == L && p.second == w) return;
        cand.emplace_back(L, w);
    };
    add(c->seg_rows, c->wpb);
    for (int w : wpbs) {
        if (w > mx) continue;
        for (int waves = 1; waves <= 2; ++waves) {
            int L = 0;
            int r = wave_rows(c, w, waves, &L);
            if (r) return r;
            add(L, w);
        }
    }
    for (int L : rows) {
        if (L > c->mesh.ny && L != rows[0]) continue;
        for (int w : wpbs)
            if (w <= mx) add(L, w);
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // trials run from a cold L2, as a long run sees it: a 256 MiB buffer is
    // written before every timed launch; the median of 5 launches counts
    void* flush = nullptr;
    const size_t flush_bytes = 256u << 20;
    if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) flush = nullptr;
    double best = 1e30;
    int bl = c->seg_rows, bw = c->wpb;
    const int cur0 = c->cur;
    double dt = 0.0;
    {
        int r = enqueue_reduce(c, 0);
        if (r) return r;
        double ms = 0.0;
        CK(cudaMemcpy(&ms, &c->d_state->maxspeed, sizeof(double), cudaMemcpyDeviceToHost));
        dt = ms > 0 ? 0.05 / ms : 1e-6;
    }
    for (const auto& cw : cand) {
        {
            const int w = cw.second;
            c->seg_rows = cw.first;
            c->wpb = w;
            float t[6];
            for (int it = 0; it < 6; ++it) {
                c->cur = cur0;
                if (flush) CK(cudaMemsetAsync(flush, it, flush_bytes, c->stream));
                CK(cudaEventRecord(e0, c->stream));
                int r = enqueue_step(c, dt, 0, c->pending, c->M_pending);
                if (r) return r;
                CK(cudaEventRecord(e1, c->stream));
                CK(cudaEventSynchronize(e1));
                CK(cudaEventElapsedTime(&t[it], e0, e1));
            }
            std::sort(t + 1, t + 6);
            const double us = 1000.0 * t[3];
            if (us < best) {
                best = us;
                bl = c->seg_rows;
                bw = w;
            }
        }
    }
    if (flush) cudaFree(flush);
    c->cur = cur0;
    c->seg_rows = bl;
    c->wpb = bw;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaMemcpy(c->d_state, &saved, sizeof(DevState), cudaMemcpyHostToDevice));
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    if (best_us) *best_us = best;
    return CRKDG_OK;
}

int crkdg_save(crkdg_ctx* c, const char* path) {
    if (check_ctx(c) || !path) return fail(CRKDG_EINVAL, "null argument");
    std::vector<double> h(c->elems);
    const bool pend = c->pending;
    const double Mp = c->M_pending;
    // save the stored (not yet limited) state and the pending flag
    c->pending = false;
    int r = crkdg_get_state(c, h.data());
    c->pending = pend;
    if (r) return r;
    double t;
    r = crkdg_time(c, &t);
    if (r) return r;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(CRKDG_EINVAL, std::string("cannot open ") + path);
    const int hdr[8] = {0x43524b44, 1, c->dim, c->mesh.nx, c->mesh.ny, c->nv, c->nm, c->precision};
    const double dh[6] = {t, pend ? 1.0 : 0.0, Mp, c->limiter_on ? c->M : -1.0, c->pp_pending, c->pp_eps};
    bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(dh, sizeof(dh), 1, f) == 1 &&
              std::fwrite(h.data(), sizeof(double), h.size(), f) == h.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? CRKDG_OK : fail(CRKDG_EINVAL, "write failed");
}

int crkdg_load(crkdg_ctx* c, const char* path) {
    if (check_ctx(c) || !path) return fail(CRKDG_EINVAL, "null argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(CRKDG_EINVAL, std::string("cannot open ") + path);
    int hdr[8];
    double dh[6];
    std::vector<double> h(c->elems);
    bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(dh, sizeof(dh), 1, f) == 1;
    ok = ok && hdr[0] == 0x43524b44 && hdr[2] == c->dim && hdr[3] == c->mesh.nx && hdr[4] == c->mesh.ny &&
         hdr[5] == c->nv && hdr[6] == c->nm;
    ok = ok && std::fread(h.data(), sizeof(double), h.size(), f) == h.size();
    std::fclose(f);
    if (!ok) return fail(CRKDG_EINVAL, "checkpoint does not match this context");
    int r = crkdg_set_state(c, h.data(), dh[0]);
    if (r) return r;
    c->pending = dh[1] != 0.0;
    c->M_pending = dh[2];
    c->limiter_on = dh[3] >= 0.0;
    c->M = dh[3];
    c->pp_pending = dh[4];
    c->pp_eps = dh[5];
    return CRKDG_OK;
}

}  // extern "C"
