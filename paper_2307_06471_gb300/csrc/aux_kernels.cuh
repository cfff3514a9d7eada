// Auxiliary kernels: FP64 reductions of the cell averages (CFL wave speed and
// conserved totals, eq. (3.4)), the L2 projection of point values onto the
// modal basis (the Pi of Sec. 2.2) and the standalone TVB limiter.
#pragma once
#include "common.cuh"
#include "limiter.cuh"
#include "mlp_tc.cuh"
#include "mlp_warp.cuh"

// resident blocks per SM the limiter pass is compiled for (tuning knob)
#ifndef CRK_LIMIT_MINB
#define CRK_LIMIT_MINB 7
#endif

namespace crk {

// max_K wave speed (2D: s_x/dx + s_y/dy; 1D: |f'|/dx) and sum_K |K| ubar_K,
// from the mode-0 planes.  Per-warp slots, then the last warp reduces them in
// a fixed order (deterministic) and writes DevState.
template <class T, int PHYS, int NV, bool COMP = false>
__global__ void reduce_state_kernel(const T* __restrict__ u, int nx, int ny, int nm, double dx, double dy,
                                    double gamma, double bx, double by, DevState* ds, double* partials,
                                    int set_dt) {
    const size_t plane = (size_t)nx * ny;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int total_warps = gridDim.x * (blockDim.x >> 5);
    double mx = 0.0, sm[NV];
    unsigned st = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) sm[v] = 0.0;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < plane; c += (size_t)gridDim.x * blockDim.x) {
        double av[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            av[v] = double(u[(size_t)(v * nm) * plane + c]);
            if (COMP) av[v] += double(u[(size_t)(NV * nm) * plane + (size_t)(v * nm) * plane + c]);
            sm[v] += av[v];
        }
        double sp;
        if constexpr (PHYS == PHYS_EULER) {
            const double ir = 1.0 / av[0];
            const double w = av[1] * ir, v = av[2] * ir;
            const double p = (gamma - 1.0) * (av[3] - 0.5 * (av[1] * w + av[2] * v));
            const double cs = sqrt(fmax(gamma * p * ir, 0.0));
            sp = (fabs(w) + cs) / dx + (fabs(v) + cs) / dy;
            if (!(av[0] > 0.0) || !(p > 0.0)) st |= ST_NONPHYSICAL;
        } else if constexpr (PHYS == PHYS_EULER1D) {
            const double ir = 1.0 / av[0];
            const double w = av[1] * ir;
            const double p = (gamma - 1.0) * (av[2] - 0.5 * av[1] * w);
            sp = (fabs(w) + sqrt(fmax(gamma * p * ir, 0.0))) / dx;
            if (!(av[0] > 0.0) || !(p > 0.0)) st |= ST_NONPHYSICAL;
        } else {
            sp = fabs(bx) / dx + (ny > 1 ? fabs(by) / dy : 0.0);
        }
        if (!(sp == sp)) st |= ST_NAN;
        mx = fmax(mx, sp);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
#pragma unroll
        for (int v = 0; v < NV; ++v) sm[v] += __shfl_xor_sync(0xffffffffu, sm[v], off);
        st |= __shfl_xor_sync(0xffffffffu, st, off);
    }
    unsigned prev = 0;
    if (lane == 0) {
        double* q = partials + (size_t)gw * (NV + 2);
        q[0] = mx;
#pragma unroll
        for (int v = 0; v < NV; ++v) q[1 + v] = sm[v] * dx * dy;
        if (st) atomicOr(&ds->status, st);
        __threadfence();
        prev = atomicAdd(&ds->counter, 1u);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != (unsigned)total_warps - 1) return;
    __threadfence();
    double M = 0.0, Sm[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Sm[v] = 0.0;
    for (int wi = lane; wi < total_warps; wi += 32) {
        const double* q = partials + (size_t)wi * (NV + 2);
        M = fmax(M, __ldcg(q));
#pragma unroll
        for (int v = 0; v < NV; ++v) Sm[v] += __ldcg(q + 1 + v);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        M = fmax(M, __shfl_xor_sync(0xffffffffu, M, off));
#pragma unroll
        for (int v = 0; v < NV; ++v) Sm[v] += __shfl_xor_sync(0xffffffffu, Sm[v], off);
    }
    if (lane == 0) {
        ds->maxspeed = M;
#pragma unroll
        for (int v = 0; v < NV; ++v) ds->sums[v] = Sm[v];
        if (set_dt) {
            double d = ds->cfl > 0.0 && M > 0.0 ? ds->cfl / M : 0.0;
            const double rem = ds->t_end - ds->t;
            ds->dt = d < rem ? d : rem;
        }
        ds->counter = 0;
    }
}

// u_m = sum_q pw[q][m] g(x_q) per cell, values[cell][q][v] (FP64, device).
// COMP: store hi = T(u_m) and lo = T(u_m - hi) in the planes after the hi planes.
template <class T, int K, int B, int NV, bool COMP = false>
__global__ void project2d_kernel(const double* __restrict__ vals, T* __restrict__ u, int ncell) {
    constexpr Tab2D<K, B> tb = make_tab2d<K, B>();
    constexpr int NQV = Tab2D<K, B>::NQV, NM = Tab2D<K, B>::NM;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const size_t plane = ncell;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < NQV; ++q) s += tb.pw[q][m] * vals[((size_t)c * NQV + q) * NV + v];
            const T hi = T(s);
            u[(size_t)(v * NM + m) * plane + c] = hi;
            if (COMP) u[(size_t)(NV * NM) * plane + (size_t)(v * NM + m) * plane + c] = T(s - double(hi));
        }
}

template <class T, int K, int NV>
__global__ void project1d_kernel(const double* __restrict__ vals, T* __restrict__ u, int ncell) {
    constexpr Tab1D<K> tb = make_tab1d<K>();
    constexpr int NQ = K + 1, NM = K + 1;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < NQ; ++q) s += tb.pw[q][m] * vals[((size_t)c * NQ + q) * NV + v];
            u[(size_t)(v * NM + m) * ncell + c] = T(s);
        }
}

// Standalone TVB limiter, in place: a thread reads its own modes and the
// neighbours' averages (mode 0) and writes only its own modes 1.. , so no
// thread writes anything another thread reads.  The x neighbours' averages
// come from the neighbouring lanes by shuffle (loads only at a warp's ends
// and at the domain's sides).  Returns whether the cell was troubled.
// The state's time (for time-dependent ghost averages) comes from the device
// run state when the run is device driven.  (x, y): the thread's cell; lanes
// past the east side (x >= nx) take part in the shuffles (and, with MLPI, in
// the warp's network evaluation) and limit nothing.
// MLPK: where the troubled-cell decision comes from.  0: the TVB test.  1
// and 2: the learned indicator (limit if the logit exceeds zhi, keep if it is
// below zlo, TVB test in between), evaluated for the warp's 32 cells with
// mma.sync (1: weights mw, the warp's staging area) or for the block's 128
// cells on the tcgen05 tensor cores (2: tcs, its barrier phase; *tc_ok turns
// false, for the whole block, once a bounded wait ran out, and the TVB test
// decides from then on).
// The mesh a limiter pass works on: a single problem's (from the launch
// arguments) or one problem of a batch (from its table entry), the time of
// its ghost data (tsrc: the device run state, or null for a.t) and its TVB
// thresholds M dx^2, M dy^2 in the kernel's arithmetic.
struct LimMesh {
    int nx, ny;
    double x0, y0, dx, dy;
    const DevState* tsrc;
    double Mdx2, Mdy2;
};

// Ghost averages beyond the non-periodic sides for cell (x, y) of the mesh
// (its own average `own` gives the exterior state where the boundary
// condition wants it); the loaded neighbour averages there are replaced.
template <class T, int NV>
__device__ __forceinline__ void limit2d_ghosts(const StepArgs& a, const LimMesh& g, int x, int y, const T* own,
                                               T* nbW, T* nbE, T* nbS, T* nbN) {
    const bool perx = a.bc[0].type == BC_PERIODIC, pery = a.bc[2].type == BC_PERIODIC;
    // ghost average beyond a non-periodic side (cx, cy: the ghost cell)
    auto ghost = [&](int side, int cx, int cy, T* out) {
        cold_branch();
        const int cxc = opaque(cx), cyc = opaque(cy);
        bc_exterior<T, NV>(a.bc[side], side < 2 ? 0 : 1, own, [&](double& xg, double& yg, double& tg) {
            xg = g.x0 + (cxc + 0.5) * g.dx;
            yg = g.y0 + (cyc + 0.5) * g.dy;
            tg = g.tsrc ? g.tsrc->t : a.t;
        }, out);
    };
    if (!perx && x == 0) ghost(0, -1, y, nbW);
    if (!perx && x == g.nx - 1) ghost(1, g.nx, y, nbE);
    if (!pery && y == 0) ghost(2, x, -1, nbS);
    if (!pery && y == g.ny - 1) ghost(3, x, g.ny, nbN);
}

// TVB-minmod test and limit (mode: -1 the test decides, 0 keep, 1 limit),
// then the positivity scaling, of cell (x, y) with modes c and neighbour
// averages nb*; modes 1.. of a changed cell are written back to u.  Returns
// whether the cell was troubled.
template <class T, int K, int B, int NV, int NM>
__device__ __forceinline__ bool limit2d_apply(const StepArgs& a, const LimMesh& g, T* __restrict__ u, int x, int y,
                                              T (&c)[NV][NM], const T* nbW, const T* nbE, const T* nbS,
                                              const T* nbN, int mode) {
    const size_t plane = (size_t)g.nx * g.ny;
    const T Mdx2 = T(g.Mdx2), Mdy2 = T(g.Mdy2);
    T gam, ppe;
    if constexpr (sizeof(T) == 4) {
        gam = a.gammaf; ppe = a.pp_epsf;
    } else {
        gam = a.gamma; ppe = a.pp_eps;
    }
    bool fl = false;
    if (a.tvb_on) fl = tvb_limit_cell<T, NV, NM>(c, nbW, nbE, nbS, nbN, Mdx2, Mdy2, gam, mode);
    bool sc = false;
    if (a.pp_on) sc = positivity_cell<T, NV, NM, K, B>(c, gam, ppe);
    if (fl || sc)
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int m = 1; m < NM; ++m) u[(size_t)(v * NM + m) * plane + (size_t)y * g.nx + x] = c[v][m];
    return fl;
}

template <class T, int K, int B, int PHYS, int MLPK>
__device__ __forceinline__ bool limit2d_cell(const StepArgs& a, const LimMesh& g, T* __restrict__ u, int x, int y,
                                             const MlpSmem* mw, __nv_bfloat16* stage, MlpTcSmem* tcs = nullptr,
                                             uint32_t* phase = nullptr, bool* tc_ok = nullptr) {
    constexpr int NM = Tab2D<K, B>::NM;
    constexpr int NV = Phys<T, PHYS>::NV;
    const int nx = g.nx, ny = g.ny;
    const size_t plane = (size_t)nx * ny;
    const int lane = threadIdx.x & 31;
    const bool inside = x < nx;
    const int xc = inside ? x : nx - 1;   // lanes past the east side mirror the last cell (shuffles only)
    const bool perx = a.bc[0].type == BC_PERIODIC, pery = a.bc[2].type == BC_PERIODIC;
    // every load first, at addresses that are always valid (wrapped or
    // clamped indices), so that the neighbours' averages are in flight with
    // the cell's own coefficients; ghost averages replace them afterwards
    const int ys = y > 0 ? y - 1 : (pery ? ny - 1 : 0);
    const int yn = y < ny - 1 ? y + 1 : (pery ? 0 : ny - 1);
    const int xw = x > 0 ? x - 1 : (perx ? nx - 1 : 0);
    const int xe = x < nx - 1 ? x + 1 : (perx ? 0 : nx - 1);
    const bool needW = inside && (lane == 0 || x == 0), needE = inside && (lane == 31 || x == nx - 1);
    T c[NV][NM], own[NV], nbW[NV], nbE[NV], nbS[NV], nbN[NV];
    // each address one plane (or one variable's NM planes) past the last:
    // a running pointer per row instead of an index formed per load
    const T* pc = u + ((size_t)y * nx + xc);
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            c[v][m] = *pc;
            pc += plane;
        }
    const T* ps = u + ((size_t)ys * nx + xc);
    const T* pn = u + ((size_t)yn * nx + xc);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        nbS[v] = *ps;
        nbN[v] = *pn;
        ps += NM * plane;
        pn += NM * plane;
    }
    T ldW[NV], ldE[NV];
    const T* pw = u + ((size_t)y * nx + xw);
    const T* pe = u + ((size_t)y * nx + xe);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        ldW[v] = needW ? *pw : T(0);
        ldE[v] = needE ? *pe : T(0);
        pw += NM * plane;
        pe += NM * plane;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        own[v] = c[v][0];
        nbW[v] = shfl_up(own[v], 1);
        nbE[v] = shfl_down(own[v], 1);
        if (needW) nbW[v] = ldW[v];
        if (needE) nbE[v] = ldE[v];
    }
    if (inside) limit2d_ghosts<T, NV>(a, g, x, y, own, nbW, nbE, nbS, nbN);
    int mode = -1;
    if constexpr (MLPK != 0) {
        // every lane of the warp (MLPK 2: of the block) takes part (lanes
        // past the side on a copy of the last cell); features of the cell and
        // its four neighbours
        float feat[MLP_IN];
        mlp_features<T, NM>(c, nbE, nbW, nbN, nbS, a.mlp_scale, feat);
        float z;
        if constexpr (MLPK == 1) {
            z = mlp_warp_logit(*mw, feat, stage);
        } else {
            z = __int_as_float(0x7fc00000);   // NaN: neither band, the TVB test decides
            if (*tc_ok) *tc_ok = mlp_tc_logit(*tcs, feat, *phase, z);   // block-uniform
        }
        mode = z > a.mlp_zhi ? 1 : (z < a.mlp_zlo ? 0 : -1);
    }
    return inside ? limit2d_apply<T, K, B, NV, NM>(a, g, u, x, y, c, nbW, nbE, nbS, nbN, mode) : false;
}

// the mesh view of a single-problem launch: thresholds as set_limiter_params
// made them (FP32 state) or in FP64
template <class T>
__device__ __forceinline__ LimMesh single_mesh(const StepArgs& a) {
    LimMesh g;
    g.nx = a.nx;
    g.ny = a.ny;
    g.x0 = a.x0;
    g.y0 = a.y0;
    g.dx = a.dx;
    g.dy = a.dy;
    g.tsrc = a.dt_from_dev ? a.ds : nullptr;
    g.Mdx2 = sizeof(T) == 4 ? double(a.Mdx2f) : a.M * a.dx * a.dx;
    g.Mdy2 = sizeof(T) == 4 ? double(a.Mdy2f) : a.M * a.dy * a.dy;
    return g;
}

// The limiter pass: 128 threads per block along x, one block row per mesh
// row.  Counts troubled cells (one atomic per warp that has any).  7 blocks
// per SM (72 registers, a few bytes of spills): on the 1920x480 P^2 state
// 0.0306 ms per pass against 0.0311 at 6 blocks (80 registers, none); 8
// blocks spill more and measured slower, 5 slower still.
template <class T, int K, int B, int PHYS>
__global__ void __launch_bounds__(128, CRK_LIMIT_MINB) limit2d_kernel(const StepArgs a, T* __restrict__ u,
                                                                      unsigned long long* flag_count) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const bool fl = limit2d_cell<T, K, B, PHYS, 0>(a, single_mesh<T>(a), u, x, blockIdx.y, nullptr, nullptr);
    const unsigned b = __ballot_sync(0xffffffffu, fl);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(flag_count, (unsigned long long)__popc(b));
}

// The limiter pass with the learned indicator (2D Euler): a grid of a few
// blocks per SM loads the network's BF16 weights into shared memory once per
// block and then walks the mesh in tiles of one row x blockDim.x cells
// (grid-stride), each warp evaluating the network for its 32 cells on the
// tensor cores.  Shared memory: the weights, then one staging area per warp.
constexpr int LIMIT_MLP_THREADS = 256;
template <class T, int K, int B>
__global__ void __launch_bounds__(LIMIT_MLP_THREADS) limit2d_mlp_kernel(const StepArgs a, T* __restrict__ u,
                                                                        unsigned long long* flag_count) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& mw = *reinterpret_cast<MlpSmem*>(smem_raw);
    __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(smem_raw + sizeof(MlpSmem)) +
                           (threadIdx.x >> 5) * (32 * MLP_INP + 64);
    mlp_load_smem(mw, a.mlp);
    __syncthreads();
    const LimMesh g = single_mesh<T>(a);
    const int xt = (a.nx + LIMIT_MLP_THREADS - 1) / LIMIT_MLP_THREADS;
    const long long tiles = (long long)xt * a.ny;
    unsigned cnt = 0;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int y = (int)(tile / xt);
        const int x = (int)(tile % xt) * LIMIT_MLP_THREADS + threadIdx.x;
        const bool fl = limit2d_cell<T, K, B, PHYS_EULER, 1>(a, g, u, x, y, &mw, stage);
        cnt += __popc(__ballot_sync(0xffffffffu, fl));
    }
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(flag_count, (unsigned long long)cnt);
}

// The same pass with the network on the tcgen05 tensor cores (mlp_tc.cuh):
// blocks of 512 threads, one tile of 512 cells of a row per iteration
// (grid-stride), each tile's network four M = 128 products per layer.  Each
// block holds the BF16 weights in shared memory and its accumulator columns
// of tensor memory for its whole walk.  A bounded wait that runs out makes
// the TVB test decide for the rest of the block's walk and sets ST_TIMEOUT
// in the run state.
template <class T, int K, int B>
__global__ void __launch_bounds__(MLPTC_CELLS) limit2d_mlp_tc_kernel(const StepArgs a, T* __restrict__ u,
                                                                 unsigned long long* flag_count) {
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    MlpTcSmem& tcs = *reinterpret_cast<MlpTcSmem*>(smem_tc);
    mlp_tc_setup(tcs, a.mlp);
    const LimMesh g = single_mesh<T>(a);
    const int xt = (a.nx + MLPTC_CELLS - 1) / MLPTC_CELLS;
    const long long tiles = (long long)xt * a.ny;
    uint32_t phase = 0;
    bool tc_ok = true;
    unsigned cnt = 0;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int y = (int)(tile / xt);
        const int x = (int)(tile % xt) * MLPTC_CELLS + threadIdx.x;
        const bool fl = limit2d_cell<T, K, B, PHYS_EULER, 2>(a, g, u, x, y, nullptr, nullptr, &tcs, &phase, &tc_ok);
        cnt += __popc(__ballot_sync(0xffffffffu, fl));
    }
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(flag_count, (unsigned long long)cnt);
    if (!tc_ok && threadIdx.x == 0) atomicOr(&a.ds->status, ST_TIMEOUT);
    mlp_tc_teardown(tcs);
}

// The limiter pass of a batched ensemble: one block of 128 threads per row
// tile of one problem (rows[b] = problem, row, first column), each problem's
// current buffer limited in place; problems that reached t_end (dt 0) are
// left as they are.  Troubled cells count into the problem's run state.
template <class T, int K, int B>
__global__ void __launch_bounds__(128, CRK_LIMIT_MINB)
    batch_limit2d_kernel(const StepArgs a, const BatchProblem* __restrict__ probs, const int4* __restrict__ rows,
                         DevState* states, const int* curs, T* bufA, T* bufB) {
    const int4 rt = rows[blockIdx.x];
    DevState* ds = states + rt.x;
    if (!(ds->dt > 0.0)) return;   // the whole block: one problem
    const BatchProblem pb = probs[rt.x];
    T* u = (curs[rt.x] ? bufB : bufA) + pb.offset;
    LimMesh g;
    g.nx = pb.nx;
    g.ny = pb.ny;
    g.x0 = pb.x0;
    g.y0 = pb.y0;
    g.dx = pb.dx;
    g.dy = pb.dy;
    g.tsrc = ds;
    // the thresholds in the arithmetic set_limiter_params uses for a single problem
    const double mx2 = a.M * pb.dx * pb.dx, my2 = a.M * pb.dy * pb.dy;
    g.Mdx2 = sizeof(T) == 4 ? double(float(mx2)) : mx2;
    g.Mdy2 = sizeof(T) == 4 ? double(float(my2)) : my2;
    const bool fl = limit2d_cell<T, K, B, PHYS_EULER, 0>(a, g, u, rt.z + threadIdx.x, rt.y, nullptr, nullptr);
    const unsigned b = __ballot_sync(0xffffffffu, fl);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&ds->lim_count, (unsigned long long)__popc(b));
}

// out = alpha * x + beta * y over n elements (RKDG Shu--Osher combinations)
template <class T>
__global__ void axpby_kernel(T* __restrict__ out, const T* __restrict__ x, const T* __restrict__ y, double alpha,
                             double beta, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = T(alpha) * x[i] + T(beta) * y[i];
}

}  // namespace crk
