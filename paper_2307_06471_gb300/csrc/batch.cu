// Batched ensembles of 2D Euler problems of uneven sizes (C ABI part of
// include/crkdg.h): one problem table, one state allocation, one batched step
// kernel per step covering every problem's tiles, per-problem FP64 dt, and a
// CUDA graph of K steps replayed until every problem reaches t_end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/crkdg.h"
#include "launch.h"
#include "step2d.cuh"

int crkdg_features_impl(const crk::StepArgs& a, int precision, int k, int basis, const void* u, float* X, float* y,
                        double Mh2, cudaStream_t st);
extern "C" const char* crkdg_mlp_last_error(void);

using crk::BatchProblem;
using crk::DevState;
using crk::StepArgs;

namespace {

thread_local std::string g_berr;
int bfail(int code, const std::string& m) {
    g_berr = m;
    return code;
}
#define BCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return bfail(CRKDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// per-problem start of a run: cfl, t_end and the first dt from a block-wide
// FP64 reduction of the problem's averages (one block per problem)
template <class T>
__global__ void batch_start_kernel(const BatchProblem* probs, const T* bufA, const T* bufB, const int* curs,
                                   int nm, double gamma, double cfl, double t_end, DevState* states,
                                   unsigned* done) {
    const int p = blockIdx.x;
    const BatchProblem pb = probs[p];
    const T* u = (curs[p] ? bufB : bufA) + pb.offset;
    const size_t plane = (size_t)pb.nx * pb.ny;
    double mx = 0.0;
    for (size_t c = threadIdx.x; c < plane; c += blockDim.x) {
        const double r = u[c], mu = u[(size_t)nm * plane + c], mv = u[(size_t)2 * nm * plane + c],
                     E = u[(size_t)3 * nm * plane + c];
        const double ir = 1.0 / r;
        const double w = mu * ir, v = mv * ir;
        const double pr = (gamma - 1.0) * (E - 0.5 * (mu * w + mv * v));
        const double cs = sqrt(fmax(gamma * pr * ir, 0.0));
        mx = fmax(mx, (fabs(w) + cs) / pb.dx + (fabs(v) + cs) / pb.dy);
    }
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
        DevState* ds = states + p;
        ds->cfl = cfl;
        ds->t_end = t_end;
        ds->maxspeed = m;
        ds->counter = 0;
        const double rem = t_end - ds->t;
        double d = m > 0.0 ? cfl / m : 0.0;
        if (d > rem) d = rem;
        if (rem <= 1e-12 * fmax(1.0, fabs(t_end))) {
            d = 0.0;
            atomicAdd(done, 1u);
        }
        ds->dt = d;
    }
}

}  // namespace

struct crkdg_batch {
    int n, k, basis, precision, nv, nm;
    int bc[4];
    crkdg_tableau tab;
    double gamma;
    size_t esize, elems;
    std::vector<BatchProblem> probs;
    std::vector<int2> tasks;
    void* buf[2] = {nullptr, nullptr};
    BatchProblem* d_probs = nullptr;
    int2* d_tasks = nullptr;
    DevState* d_states = nullptr;
    int* d_curs = nullptr;
    unsigned* d_done = nullptr;
    double* d_partials = nullptr;
    double* d_tab = nullptr;
    unsigned long long* d_flags = nullptr;
    cudaStream_t stream = nullptr;
    int seg_rows = 32, wpb = 4;
    int4* d_rows = nullptr;                // limiter-pass row tiles: (problem, row, first column)
    int n_rows = 0;
    int limit_mode = CRKDG_LIMIT_PASS;     // crkdg_batch_set_limit_mode
    bool limiter_on = false, pending = false;
    double M = -1.0, pp_eps = 0.0, M_pending = -1.0, pp_pending = 0.0;
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
};

namespace {

StepArgs batch_args(const crkdg_batch* b) {
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.s = b->tab.s;
    a.tab = b->d_tab;
    for (int s = 0; s < 4; ++s) a.bc[s].type = b->bc[s];
    crk::set_bc_affine(a.bc, 4);
    a.gamma = b->gamma;
    a.seg_len = b->seg_rows;
    a.partials = b->d_partials;
    return a;
}

// rebuild the task table for the current segment length
int build_tasks(crkdg_batch* b) {
    b->tasks.clear();
    int warp0 = 0;
    for (int p = 0; p < b->n; ++p) {
        BatchProblem& pb = b->probs[p];
        pb.n_strips = (pb.nx + 29) / 30;
        pb.n_segs = (pb.ny + b->seg_rows - 1) / b->seg_rows;
        pb.warp0 = warp0;
        const int w = pb.n_strips * pb.n_segs;
        for (int i = 0; i < w; ++i) b->tasks.push_back(make_int2(p, i));
        warp0 += w;
    }
    // the limiter pass's tiles: 128 cells of one row of one problem
    std::vector<int4> rows;
    for (int p = 0; p < b->n; ++p)
        for (int y = 0; y < b->probs[p].ny; ++y)
            for (int x = 0; x < b->probs[p].nx; x += 128) rows.push_back(make_int4(p, y, x, 0));
    if (b->d_tasks) cudaFree(b->d_tasks);
    if (b->d_partials) cudaFree(b->d_partials);
    if (b->d_rows) cudaFree(b->d_rows);
    b->d_tasks = nullptr;
    b->d_partials = nullptr;
    b->d_rows = nullptr;
    b->n_rows = (int)rows.size();
    BCK(cudaMalloc(&b->d_rows, rows.size() * sizeof(int4)));
    BCK(cudaMemcpy(b->d_rows, rows.data(), rows.size() * sizeof(int4), cudaMemcpyHostToDevice));
    BCK(cudaMalloc(&b->d_tasks, b->tasks.size() * sizeof(int2)));
    BCK(cudaMalloc(&b->d_partials, (size_t)warp0 * 8 * sizeof(double)));
    BCK(cudaMemcpy(b->d_tasks, b->tasks.data(), b->tasks.size() * sizeof(int2), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_probs, b->probs.data(), b->n * sizeof(BatchProblem), cudaMemcpyHostToDevice));
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    return CRKDG_OK;
}

int enqueue_batch_step(crkdg_batch* b, int limit, double M, double pp) {
    StepArgs a = batch_args(b);
    a.limit = limit;
    a.M = M;
    a.pp_eps = limit ? pp : 0.0;
    if (limit && b->limit_mode == CRKDG_LIMIT_PASS) {
        // the pending limit of every running problem as one in-place pass;
        // the batched step then loads the limited states as they are
        cudaError_t e = b->precision == CRKDG_F32
                            ? crk::blimit2d_euler_f32(b->k, b->basis, a, b->d_probs, b->d_rows, b->n_rows,
                                                      b->d_states, b->d_curs, b->buf[0], b->buf[1], b->stream)
                            : crk::blimit2d_euler_f64(b->k, b->basis, a, b->d_probs, b->d_rows, b->n_rows,
                                                      b->d_states, b->d_curs, b->buf[0], b->buf[1], b->stream);
        if (e != cudaSuccess) return bfail(CRKDG_ECUDA, std::string("batched limiter pass: ") + cudaGetErrorString(e));
        a.limit = 0;
    }
    cudaError_t e = b->precision == CRKDG_F32
                        ? crk::batch2d_euler_f32(b->k, b->basis, a, b->d_probs, b->d_tasks, (int)b->tasks.size(),
                                                 b->d_states, b->d_curs, b->d_done, b->buf[0], b->buf[1], b->wpb,
                                                 b->stream)
                        : crk::batch2d_euler_f64(b->k, b->basis, a, b->d_probs, b->d_tasks, (int)b->tasks.size(),
                                                 b->d_states, b->d_curs, b->d_done, b->buf[0], b->buf[1], b->wpb,
                                                 b->stream);
    if (e != cudaSuccess) return bfail(CRKDG_ECUDA, std::string("batched step: ") + cudaGetErrorString(e));
    return CRKDG_OK;
}

int get_cur(const crkdg_batch* b, int p, int* cur) {
    BCK(cudaStreamSynchronize(b->stream));
    BCK(cudaMemcpy(cur, b->d_curs + p, sizeof(int), cudaMemcpyDeviceToHost));
    return CRKDG_OK;
}

StepArgs problem_args(const crkdg_batch* b, int p) {
    StepArgs a = batch_args(b);
    const BatchProblem& pb = b->probs[p];
    a.nx = pb.nx;
    a.ny = pb.ny;
    a.x0 = pb.x0;
    a.y0 = pb.y0;
    a.dx = pb.dx;
    a.dy = pb.dy;
    return a;
}

}  // namespace

extern "C" {

const char* crkdg_batch_last_error(void) { return g_berr.c_str(); }

int crkdg_batch_create(const crkdg_batch_problem* probs, int n, const int* bc, int k, int basis,
                       const crkdg_tableau* tab, double gamma, int precision, void* stream, crkdg_batch** out) {
    if (!probs || !bc || !tab || !out || n < 1) return bfail(CRKDG_EINVAL, "null argument or empty batch");
    *out = nullptr;
    if (k < 0 || k > 3) return bfail(CRKDG_EUNSUPPORTED, "k must be 0..3");
    if (basis != CRKDG_BASIS_P && basis != CRKDG_BASIS_Q) return bfail(CRKDG_EINVAL, "basis must be P or Q");
    if (precision != CRKDG_F32 && precision != CRKDG_F64) return bfail(CRKDG_EINVAL, "unknown precision");
    if (tab->s < 1 || tab->s > CRKDG_MAX_STAGES) return bfail(CRKDG_EINVAL, "tableau stages must be 1..6");
    if (!(gamma > 1.0)) return bfail(CRKDG_EINVAL, "gamma must exceed 1");
    for (int s = 0; s < 4; ++s)
        if (bc[s] != CRKDG_BC_PERIODIC && bc[s] != CRKDG_BC_OUTFLOW && bc[s] != CRKDG_BC_REFLECT)
            return bfail(CRKDG_EINVAL, "batched problems take periodic, outflow or reflect boundaries");
    if ((bc[0] == CRKDG_BC_PERIODIC) != (bc[1] == CRKDG_BC_PERIODIC) ||
        (bc[2] == CRKDG_BC_PERIODIC) != (bc[3] == CRKDG_BC_PERIODIC))
        return bfail(CRKDG_EINVAL, "periodic sides must come in pairs");
    crkdg_batch* b = new crkdg_batch();
    b->n = n;
    b->k = k;
    b->basis = basis;
    b->precision = precision;
    b->nv = 4;
    b->nm = basis == CRKDG_BASIS_P ? (k + 1) * (k + 2) / 2 : (k + 1) * (k + 1);
    for (int s = 0; s < 4; ++s) b->bc[s] = bc[s];
    b->tab = *tab;
    b->gamma = gamma;
    b->esize = precision == CRKDG_F32 ? 4 : 8;
    b->stream = static_cast<cudaStream_t>(stream);
    size_t off = 0;
    for (int p = 0; p < n; ++p) {
        const crkdg_batch_problem& q = probs[p];
        if (q.nx < 1 || q.ny < 1 || !(q.x1 > q.x0) || !(q.y1 > q.y0)) {
            delete b;
            return bfail(CRKDG_EINVAL, "problem " + std::to_string(p) + " has an empty mesh or domain");
        }
        BatchProblem pb;
        std::memset(&pb, 0, sizeof(pb));
        pb.offset = (long long)off;
        pb.nx = q.nx;
        pb.ny = q.ny;
        pb.x0 = q.x0;
        pb.y0 = q.y0;
        pb.dx = (q.x1 - q.x0) / q.nx;
        pb.dy = (q.y1 - q.y0) / q.ny;
        pb.rx = 1.0 / pb.dx;
        pb.ry = 1.0 / pb.dy;
        pb.sq = pb.dx == pb.dy ? 1 : 0;
        b->probs.push_back(pb);
        off += (size_t)q.nx * q.ny * b->nv * b->nm;
    }
    b->elems = off;
    auto bail = [&](int code) {
        crkdg_batch_destroy(b);
        return code;
    };
    for (int i = 0; i < 2; ++i)
        if (cudaMalloc(&b->buf[i], b->elems * b->esize) != cudaSuccess)
            return bail(bfail(CRKDG_ENOMEM, "cudaMalloc of the batch state failed"));
    unsigned char htab[crk::TAB_BYTES];
    crk::pack_tableau(tab->s, tab->a, tab->b, tab->c, htab);
    if (cudaMalloc(&b->d_probs, n * sizeof(BatchProblem)) != cudaSuccess ||
        cudaMalloc(&b->d_states, n * sizeof(DevState)) != cudaSuccess ||
        cudaMalloc(&b->d_curs, n * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_done, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&b->d_tab, sizeof(htab)) != cudaSuccess ||
        cudaMalloc(&b->d_flags, sizeof(unsigned long long)) != cudaSuccess)
        return bail(bfail(CRKDG_ENOMEM, "cudaMalloc failed"));
    if (cudaMemcpy(b->d_tab, htab, sizeof(htab), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_states, 0, n * sizeof(DevState)) != cudaSuccess ||
        cudaMemset(b->d_curs, 0, n * sizeof(int)) != cudaSuccess ||
        cudaMemset(b->d_done, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(b->d_flags, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(b->buf[0], 0, b->elems * b->esize) != cudaSuccess ||
        cudaMemset(b->buf[1], 0, b->elems * b->esize) != cudaSuccess)
        return bail(bfail(CRKDG_ECUDA, "initialisation failed"));
    int r = build_tasks(b);
    if (r) return bail(r);
    *out = b;
    return CRKDG_OK;
}

void crkdg_batch_destroy(crkdg_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (int i = 0; i < 2; ++i)
        if (b->buf[i]) cudaFree(b->buf[i]);
    for (void* p : {(void*)b->d_probs, (void*)b->d_tasks, (void*)b->d_states, (void*)b->d_curs, (void*)b->d_done,
                    (void*)b->d_partials, (void*)b->d_tab, (void*)b->d_flags, (void*)b->d_rows})
        if (p) cudaFree(p);
    delete b;
}

int crkdg_batch_quadrature_points(const crkdg_batch* b, int p, double* xy) {
    if (!b || !xy || p < 0 || p >= b->n) return bfail(CRKDG_EINVAL, "bad argument");
    const crk::GaussRule g = crk::gauss_rule(b->k + 1);
    const BatchProblem& pb = b->probs[p];
    const int nq = b->k + 1;
    size_t o = 0;
    for (int y = 0; y < pb.ny; ++y)
        for (int x = 0; x < pb.nx; ++x) {
            const double xc = pb.x0 + (x + 0.5) * pb.dx, yc = pb.y0 + (y + 0.5) * pb.dy;
            for (int a = 0; a < nq; ++a)
                for (int c = 0; c < nq; ++c) {
                    xy[o++] = xc + 0.5 * pb.dx * g.x[a];
                    xy[o++] = yc + 0.5 * pb.dy * g.x[c];
                }
        }
    return CRKDG_OK;
}

int crkdg_batch_project_ic(crkdg_batch* b, int p, const double* values) {
    if (!b || !values || p < 0 || p >= b->n) return bfail(CRKDG_EINVAL, "bad argument");
    int cur = 0;
    int r = get_cur(b, p, &cur);
    if (r) return r;
    const BatchProblem& pb = b->probs[p];
    const size_t ncell = (size_t)pb.nx * pb.ny;
    const size_t n = ncell * (b->k + 1) * (b->k + 1) * b->nv;
    double* d = nullptr;
    if (cudaMalloc(&d, n * sizeof(double)) != cudaSuccess) return bfail(CRKDG_ENOMEM, "cudaMalloc failed");
    char* base = static_cast<char*>(b->buf[cur]) + pb.offset * b->esize;
    cudaError_t e = cudaMemcpyAsync(d, values, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = crk::launch_project(2, crk::PHYS_EULER, b->precision, b->k, b->basis, d, base, (int)ncell, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d);
    if (e != cudaSuccess) return bfail(CRKDG_ECUDA, std::string("project: ") + cudaGetErrorString(e));
    DevState ds;
    std::memset(&ds, 0, sizeof(ds));
    BCK(cudaMemcpy(b->d_states + p, &ds, sizeof(ds), cudaMemcpyHostToDevice));
    return CRKDG_OK;
}

int crkdg_batch_set_state(crkdg_batch* b, int p, const double* h, double t) {
    if (!b || !h || p < 0 || p >= b->n) return bfail(CRKDG_EINVAL, "bad argument");
    int cur = 0;
    int r = get_cur(b, p, &cur);
    if (r) return r;
    const BatchProblem& pb = b->probs[p];
    const size_t n = (size_t)pb.nx * pb.ny * b->nv * b->nm;
    char* base = static_cast<char*>(b->buf[cur]) + pb.offset * b->esize;
    if (b->precision == CRKDG_F64) {
        BCK(cudaMemcpy(base, h, n * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(n);
        for (size_t i = 0; i < n; ++i) f[i] = (float)h[i];
        BCK(cudaMemcpy(base, f.data(), n * 4, cudaMemcpyHostToDevice));
    }
    DevState ds;
    std::memset(&ds, 0, sizeof(ds));
    ds.t = t;
    BCK(cudaMemcpy(b->d_states + p, &ds, sizeof(ds), cudaMemcpyHostToDevice));
    return CRKDG_OK;
}

int crkdg_batch_get_state(crkdg_batch* b, int p, double* h) {
    if (!b || !h || p < 0 || p >= b->n) return bfail(CRKDG_EINVAL, "bad argument");
    int cur = 0;
    int r = get_cur(b, p, &cur);
    if (r) return r;
    const BatchProblem& pb = b->probs[p];
    const size_t n = (size_t)pb.nx * pb.ny * b->nv * b->nm;
    char* base = static_cast<char*>(b->buf[cur]) + pb.offset * b->esize;
    if (b->pending) {
        // the stored state is pending the limiter of its last step: apply it to a copy
        void* tmp = nullptr;
        if (cudaMalloc(&tmp, n * b->esize) != cudaSuccess) return bfail(CRKDG_ENOMEM, "cudaMalloc failed");
        cudaError_t e = cudaMemcpyAsync(tmp, base, n * b->esize, cudaMemcpyDeviceToDevice, b->stream);
        StepArgs a = problem_args(b, p);
        DevState ds;
        if (e == cudaSuccess) e = cudaMemcpy(&ds, b->d_states + p, sizeof(ds), cudaMemcpyDeviceToHost);
        a.t = ds.t;
        a.M = b->M_pending;
        a.pp_eps = b->pp_pending;
        if (e == cudaSuccess)
            e = crk::launch_limit2d(crk::PHYS_EULER, b->precision, b->k, b->basis, a, tmp, b->d_flags, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e == cudaSuccess) {
            if (b->precision == CRKDG_F64) {
                e = cudaMemcpy(h, tmp, n * 8, cudaMemcpyDeviceToHost);
            } else {
                std::vector<float> f(n);
                e = cudaMemcpy(f.data(), tmp, n * 4, cudaMemcpyDeviceToHost);
                for (size_t i = 0; i < n; ++i) h[i] = f[i];
            }
        }
        cudaFree(tmp);
        if (e != cudaSuccess) return bfail(CRKDG_ECUDA, std::string("get_state: ") + cudaGetErrorString(e));
        return CRKDG_OK;
    }
    if (b->precision == CRKDG_F64) {
        BCK(cudaMemcpy(h, base, n * 8, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> f(n);
        BCK(cudaMemcpy(f.data(), base, n * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) h[i] = f[i];
    }
    return CRKDG_OK;
}

int crkdg_batch_features(crkdg_batch* b, int p, float* X_dev, float* y_dev, double M) {
    if (!b || !X_dev || !y_dev || p < 0 || p >= b->n || !(M >= 0.0)) return bfail(CRKDG_EINVAL, "bad argument");
    int cur = 0;
    int r = get_cur(b, p, &cur);
    if (r) return r;
    const BatchProblem& pb = b->probs[p];
    StepArgs a = problem_args(b, p);
    DevState ds;
    BCK(cudaMemcpy(&ds, b->d_states + p, sizeof(ds), cudaMemcpyDeviceToHost));
    a.t = ds.t;
    a.M = M;
    const double h = std::max(pb.dx, pb.dy);
    const char* base = static_cast<const char*>(b->buf[cur]) + pb.offset * b->esize;
    r = crkdg_features_impl(a, b->precision, b->k, b->basis, base, X_dev, y_dev, M * h * h, b->stream);
    if (r) return bfail(r, crkdg_mlp_last_error());
    BCK(cudaStreamSynchronize(b->stream));
    return CRKDG_OK;
}

int crkdg_batch_limit(crkdg_batch* b, double M) {
    if (!b) return bfail(CRKDG_EINVAL, "null batch");
    if (M >= 0.0) {
        b->limiter_on = true;
        b->M = M;
        b->pending = true;
        b->M_pending = M;
        b->pp_pending = b->pp_eps;
    } else {
        b->limiter_on = false;
        b->M = -1.0;
    }
    return CRKDG_OK;
}

int crkdg_batch_positivity(crkdg_batch* b, double eps) {
    if (!b) return bfail(CRKDG_EINVAL, "null batch");
    if (eps > 0.0) {
        b->pp_eps = eps;
        if (!b->pending) {
            b->pending = true;
            b->M_pending = -1.0;
        }
        b->pp_pending = eps;
    } else {
        b->pp_eps = 0.0;
    }
    return CRKDG_OK;
}

int crkdg_batch_run(crkdg_batch* b, double cfl, double t_end, int steps_per_graph, int max_graphs, int* n_done) {
    if (!b || !(cfl > 0.0) || steps_per_graph < 1 || max_graphs < 1) return bfail(CRKDG_EINVAL, "bad argument");
    if (!b->stream) return bfail(CRKDG_EINVAL, "batched runs need a non-default stream (graph capture)");
    BCK(cudaMemsetAsync(b->d_done, 0, sizeof(unsigned), b->stream));
    if (b->precision == CRKDG_F32)
        batch_start_kernel<float><<<b->n, 256, 0, b->stream>>>(b->d_probs, (const float*)b->buf[0],
                                                               (const float*)b->buf[1], b->d_curs, b->nm, b->gamma,
                                                               cfl, t_end, b->d_states, b->d_done);
    else
        batch_start_kernel<double><<<b->n, 256, 0, b->stream>>>(b->d_probs, (const double*)b->buf[0],
                                                                (const double*)b->buf[1], b->d_curs, b->nm, b->gamma,
                                                                cfl, t_end, b->d_states, b->d_done);
    BCK(cudaGetLastError());
    unsigned done = 0;
    for (int g = 0; g < max_graphs; ++g) {
        const int lim_first = b->pending ? 1 : 0;
        const int lim_rest = (b->limiter_on || b->pp_eps > 0.0) ? 1 : 0;
        auto key = std::make_tuple(steps_per_graph, lim_first, lim_rest);
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t gr;
            BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            int r = CRKDG_OK;
            for (int i = 0; i < steps_per_graph && r == CRKDG_OK; ++i)
                r = enqueue_batch_step(b, i == 0 ? lim_first : lim_rest, i == 0 ? b->M_pending : b->M,
                                       i == 0 ? b->pp_pending : b->pp_eps);
            cudaError_t e = cudaStreamEndCapture(b->stream, &gr);
            if (r) return r;
            if (e != cudaSuccess) return bfail(CRKDG_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
            cudaGraphExec_t ge;
            e = cudaGraphInstantiate(&ge, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) return bfail(CRKDG_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
            it = b->graphs.emplace(key, ge).first;
        }
        BCK(cudaGraphLaunch(it->second, b->stream));
        b->pending = b->limiter_on || b->pp_eps > 0.0;
        b->M_pending = b->M;
        b->pp_pending = b->pp_eps;
        BCK(cudaMemcpyAsync(&done, b->d_done, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
        if ((int)done >= b->n) break;
    }
    if (n_done) *n_done = (int)done;
    return CRKDG_OK;
}

int crkdg_batch_problem_info(crkdg_batch* b, int p, double* t, unsigned long long* steps, unsigned* status) {
    if (!b || p < 0 || p >= b->n) return bfail(CRKDG_EINVAL, "bad argument");
    DevState ds;
    BCK(cudaStreamSynchronize(b->stream));
    BCK(cudaMemcpy(&ds, b->d_states + p, sizeof(ds), cudaMemcpyDeviceToHost));
    if (t) *t = ds.t;
    if (steps) *steps = ds.steps;
    if (status) *status = ds.status;
    return CRKDG_OK;
}

int crkdg_batch_sizes(const crkdg_batch* b, int* n_problems, long long* total_cells, int* n_modes, int* n_tasks) {
    if (!b) return bfail(CRKDG_EINVAL, "null batch");
    long long c = 0;
    for (const auto& p : b->probs) c += (long long)p.nx * p.ny;
    if (n_problems) *n_problems = b->n;
    if (total_cells) *total_cells = c;
    if (n_modes) *n_modes = b->nm;
    if (n_tasks) *n_tasks = (int)b->tasks.size();
    return CRKDG_OK;
}

int crkdg_batch_set_limit_mode(crkdg_batch* b, int mode) {
    if (!b) return bfail(CRKDG_EINVAL, "null batch");
    if (mode != CRKDG_LIMIT_FUSED && mode != CRKDG_LIMIT_PASS) return bfail(CRKDG_EINVAL, "unknown limit mode");
    b->limit_mode = mode;
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    return CRKDG_OK;
}

int crkdg_batch_set_launch(crkdg_batch* b, int seg_rows, int wpb) {
    if (!b || seg_rows < 0 || wpb < 0 || wpb > 8) return bfail(CRKDG_EINVAL, "bad launch shape");
    if (wpb > 0) {
        crk::KernelInfo ki;
        cudaError_t e = b->precision == CRKDG_F32 ? crk::binfo2d_euler_f32(b->k, b->basis, b->tab.s, &ki)
                                                  : crk::binfo2d_euler_f64(b->k, b->basis, b->tab.s, &ki);
        if (e != cudaSuccess) return bfail(CRKDG_ECUDA, cudaGetErrorString(e));
        if (wpb * 32 > ki.max_threads || (size_t)ki.smem_per_thread * wpb * 32 > 227 * 1024)
            return bfail(CRKDG_EINVAL, "warps per block exceeds the kernel's limits");
        b->wpb = wpb;
    }
    if (seg_rows > 0 && seg_rows != b->seg_rows) {
        b->seg_rows = seg_rows;
        return build_tasks(b);
    }
    return CRKDG_OK;
}

int crkdg_batch_autotune(crkdg_batch* b, double cfl, double* best_us) {
    if (!b || !(cfl > 0.0)) return bfail(CRKDG_EINVAL, "bad argument");
    if (!b->stream) return bfail(CRKDG_EINVAL, "batched runs need a non-default stream");
    // trial steps advance the run state and flip buffers: save and restore
    std::vector<DevState> st(b->n);
    std::vector<int> cu(b->n);
    BCK(cudaStreamSynchronize(b->stream));
    BCK(cudaMemcpy(st.data(), b->d_states, b->n * sizeof(DevState), cudaMemcpyDeviceToHost));
    BCK(cudaMemcpy(cu.data(), b->d_curs, b->n * sizeof(int), cudaMemcpyDeviceToHost));
    const int rows[] = {8, 16, 32, 64};
    const int wpbs[] = {2, 4, 8};
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    double best = 1e30;
    int bl = b->seg_rows, bw = b->wpb;
    for (int L : rows)
        for (int w : wpbs) {
            if (crkdg_batch_set_launch(b, L, w) != CRKDG_OK) continue;
            float t[4];
            for (int it = 0; it < 4; ++it) {
                BCK(cudaMemcpy(b->d_states, st.data(), b->n * sizeof(DevState), cudaMemcpyHostToDevice));
                BCK(cudaMemcpy(b->d_curs, cu.data(), b->n * sizeof(int), cudaMemcpyHostToDevice));
                if (b->precision == CRKDG_F32)
                    batch_start_kernel<float><<<b->n, 256, 0, b->stream>>>(
                        b->d_probs, (const float*)b->buf[0], (const float*)b->buf[1], b->d_curs, b->nm, b->gamma, cfl,
                        1e30, b->d_states, b->d_done);
                else
                    batch_start_kernel<double><<<b->n, 256, 0, b->stream>>>(
                        b->d_probs, (const double*)b->buf[0], (const double*)b->buf[1], b->d_curs, b->nm, b->gamma,
                        cfl, 1e30, b->d_states, b->d_done);
                BCK(cudaEventRecord(e0, b->stream));
                int r = enqueue_batch_step(b, b->pending, b->M_pending, b->pp_pending);
                if (r) return r;
                BCK(cudaEventRecord(e1, b->stream));
                BCK(cudaEventSynchronize(e1));
                BCK(cudaEventElapsedTime(&t[it], e0, e1));
            }
            std::sort(t + 1, t + 4);
            const double us = 1000.0 * t[2];
            if (us < best) {
                best = us;
                bl = L;
                bw = w;
            }
        }
    BCK(cudaMemcpy(b->d_states, st.data(), b->n * sizeof(DevState), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_curs, cu.data(), b->n * sizeof(int), cudaMemcpyHostToDevice));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int r = crkdg_batch_set_launch(b, bl, bw);
    if (r) return r;
    if (best_us) *best_us = best;
    return CRKDG_OK;
}

}  // extern "C"
