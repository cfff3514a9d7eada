// Fused cRKDG time step on a 2D Cartesian mesh (eq. (2.8)).
//
// Work decomposition ("marching warps"): a warp owns a strip of 30 columns
// plus one halo column on each side (lane l holds column x0 - 1 + l) and
// marches up a segment of rows.  For every row each lane
//   1. loads u^n of its cell (planes [v][m][y][x]: one coalesced 128-byte
//      line per (v, m) for the warp) and, if a limit is pending, applies the
//      TVB limiter of the previous step to it (limit-on-load);
//   2. runs every RK stage cell-locally (eq. (2.8), first line): stage states
//      u^(i) and div^loc f(u^(i)) (eq. (2.7)) stay in registers and in the
//      thread's private shared-memory slots; nothing of a stage reaches HBM;
//   3. forms the final-stage face fluxes sum_i b_i fhat(u^(i)) (eq. (2.8),
//      second line): east/west faces with the neighbouring lane through
//      warp shuffles, south faces with the north traces of the row below,
//      kept per stage in the same thread's shared-memory slot;
//   4. completes the update of the row below (its north face is the current
//      row's south face) and writes u^{n+1} of that row once.
// Halo columns and one extra row at each segment end are recomputed instead
// of exchanged: the compactness of cRKDG (Sec. 3.1) means one ring suffices.
// Boundary data enter only the final-stage fluxes, at t^n + c_i dt (Sec. 3.4).
// The FP64 epilogue reduces the new cell averages (max wave speed, totals;
// eq. (3.4)) per warp; finalize_step_kernel (a batch: the problem's last warp)
// combines the warps' slots and updates the device run state.
#pragma once
#include "common.cuh"
#include "limiter.cuh"
#include "mlp_warp.cuh"

// where the per-row accumulator sum_i b_i vol_i lives: 0 registers, 1 the
// thread's shared-memory slot (tuning knob)
#ifndef CRK_V_SMEM
#define CRK_V_SMEM 0
#endif
// 1: stages with a local operator form the east/south Lax--Friedrichs fluxes
// from the physical fluxes that operator already computed (own traces), the
// neighbouring lane's (shuffle) and the row below's (kept in shared memory).
// Off: measured slower (fewer instructions, more shuffle and shared-memory
// latency in the inner loop: 0.269 against 0.260 ms per step kernel)
#ifndef CRK_LF_REUSE
#define CRK_LF_REUSE 0
#endif
// launch bounds of the single-problem step kernel (tuning knobs)
#ifndef CRK_STEP_MAXT
#define CRK_STEP_MAXT 256
#endif
#ifndef CRK_STEP_MINB2
#define CRK_STEP_MINB2 1
#endif
// blocks per SM the scalar (advection) step is compiled for: its live state
// is a quarter of the Euler step's, so it can trade registers for warps
#ifndef CRK_STEP_MINB_ADV
#define CRK_STEP_MINB_ADV 2
#endif

namespace crk {

// a0 += x0 * c, a1 += x1 * c: one packed FP32x2 FMA on sm_100+ for float
// (the same fused rounding as two scalar FMAs), two FMAs for double
template <class T>
__device__ __forceinline__ void pfma(T& a0, T& a1, T x0, T x1, T c) {
    if constexpr (sizeof(T) == 4) {
        const float2 r = __ffma2_rn(make_float2(x0, x1), make_float2(c, c), make_float2(a0, a1));
        a0 = r.x;
        a1 = r.y;
    } else {
        a0 = fma(x0, c, a0);
        a1 = fma(x1, c, a1);
    }
}

// packed sum, difference and scaling of pairs: one FP32x2 instruction each
// on sm_100+ for float (rounding as the scalar operations), scalar for double
template <class T>
__device__ __forceinline__ void padd(T& r0, T& r1, T a0, T a1, T b0, T b1) {
    if constexpr (sizeof(T) == 4) {
        const float2 r = __fadd2_rn(make_float2(a0, a1), make_float2(b0, b1));
        r0 = r.x;
        r1 = r.y;
    } else {
        r0 = a0 + b0;
        r1 = a1 + b1;
    }
}
template <class T>
__device__ __forceinline__ void psub(T& r0, T& r1, T a0, T a1, T b0, T b1) {
    if constexpr (sizeof(T) == 4) {
        const float2 r = __ffma2_rn(make_float2(b0, b1), make_float2(-1.f, -1.f), make_float2(a0, a1));
        r0 = r.x;
        r1 = r.y;
    } else {
        r0 = a0 - b0;
        r1 = a1 - b1;
    }
}
template <class T>
__device__ __forceinline__ void pmul(T& a0, T& a1, T c) {
    if constexpr (sizeof(T) == 4) {
        const float2 r = __fmul2_rn(make_float2(a0, a1), make_float2(c, c));
        a0 = r.x;
        a1 = r.y;
    } else {
        a0 *= c;
        a1 *= c;
    }
}

template <class T, int K, int B, int PHYS>
struct Step2D {
    using TB = Tab2D<K, B>;
    static constexpr int NQ = TB::NQ;
    static constexpr int NQV = TB::NQV;
    static constexpr int NM = TB::NM;
    static constexpr int NV = Phys<T, PHYS>::NV;
    static constexpr int NDOF = NV * NM;
    static constexpr int NRED = NV + 2;   // reduction slots: maxspeed, sums[NV], troubled

    // T elements of private shared memory per thread for s stages: L_j
    // (j < s-1), north traces per stage, pending update, (CRK_V_SMEM) the
    // row's sum_i b_i vol_i, and (CRK_LF_REUSE) the north traces' normal
    // fluxes and wave speeds per stage
    static __host__ __device__ constexpr int smem_per_thread(int s) {
        return (s - 1) * NDOF + s * NQ * NV + NDOF + (CRK_V_SMEM ? NDOF : 0) + (CRK_LF_REUSE ? s * NQ * (NV + 1) : 0);
    }
};

// Per-problem view of one step.  The single-problem kernel reads the mesh
// straight from its launch arguments (kernel-parameter constant bank, no
// registers held); the batched kernel reads it from the problem table.
template <class T>
struct ArgsView {
    const StepArgs& a;
    double t_, dt_;
    __device__ __forceinline__ const T* uin() const { return static_cast<const T*>(a.uin); }
    __device__ __forceinline__ T* uout() const { return static_cast<T*>(a.uout); }
    __device__ __forceinline__ int nx() const { return a.nx; }
    __device__ __forceinline__ int ny() const { return a.ny; }
    __device__ __forceinline__ double x0() const { return a.x0; }
    __device__ __forceinline__ double y0() const { return a.y0; }
    __device__ __forceinline__ double dx() const { return a.dx; }
    __device__ __forceinline__ double dy() const { return a.dy; }
    __device__ __forceinline__ double t() const { return t_; }
    __device__ __forceinline__ double dt() const { return dt_; }
    __device__ __forceinline__ int n_strips() const { return a.n_strips; }
    __device__ __forceinline__ int n_segs() const { return a.n_segs; }
    __device__ __forceinline__ int seg_len() const { return a.seg_len; }
    __device__ __forceinline__ int total_warps() const { return a.n_strips * a.n_segs; }
    __device__ __forceinline__ double* partials() const { return a.partials; }
    __device__ __forceinline__ DevState* ds() const { return a.ds; }
    __device__ __forceinline__ int* cur() const { return nullptr; }
    __device__ __forceinline__ unsigned* done() const { return nullptr; }
    __device__ __forceinline__ bool copy_if_idle() const { return true; }
    static constexpr bool kLastWarp = false;   // finalize_step_kernel ends the step
    // derived constants, computed on the host (set_derived)
    __device__ __forceinline__ T rxT() const {
        if constexpr (sizeof(T) == 4) return a.rxf;
        else return T(a.rx);
    }
    __device__ __forceinline__ T ryT() const {
        if constexpr (sizeof(T) == 4) return a.ryf;
        else return T(a.ry);
    }
    __device__ __forceinline__ T Mdx2T() const {
        if constexpr (sizeof(T) == 4) return a.Mdx2f;
        else return T(a.M * a.dx * a.dx);
    }
    __device__ __forceinline__ T Mdy2T() const {
        if constexpr (sizeof(T) == 4) return a.Mdy2f;
        else return T(a.M * a.dy * a.dy);
    }
    __device__ __forceinline__ double cell() const { return a.cell; }
    __device__ __forceinline__ double adv_speed() const { return a.adv_speed; }
};

template <class T>
struct ProbView {
    const T* uin_;
    T* uout_;
    int nx_, ny_;
    double x0_, y0_, dx_, dy_;
    double t_, dt_;
    int n_strips_, n_segs_, seg_len_, total_warps_;
    double* partials_;    // this problem's per-warp reduction slots
    DevState* ds_;        // this problem's run state
    int* cur_;            // this problem's buffer index (flipped by its last warp)
    unsigned* done_;      // count of problems that reached t_end
    __device__ __forceinline__ const T* uin() const { return uin_; }
    __device__ __forceinline__ T* uout() const { return uout_; }
    __device__ __forceinline__ int nx() const { return nx_; }
    __device__ __forceinline__ int ny() const { return ny_; }
    __device__ __forceinline__ double x0() const { return x0_; }
    __device__ __forceinline__ double y0() const { return y0_; }
    __device__ __forceinline__ double dx() const { return dx_; }
    __device__ __forceinline__ double dy() const { return dy_; }
    __device__ __forceinline__ double t() const { return t_; }
    __device__ __forceinline__ double dt() const { return dt_; }
    __device__ __forceinline__ int n_strips() const { return n_strips_; }
    __device__ __forceinline__ int n_segs() const { return n_segs_; }
    __device__ __forceinline__ int seg_len() const { return seg_len_; }
    __device__ __forceinline__ int total_warps() const { return total_warps_; }
    __device__ __forceinline__ double* partials() const { return partials_; }
    __device__ __forceinline__ DevState* ds() const { return ds_; }
    __device__ __forceinline__ int* cur() const { return cur_; }
    __device__ __forceinline__ unsigned* done() const { return done_; }
    __device__ __forceinline__ bool copy_if_idle() const { return false; }
    static constexpr bool kLastWarp = true;    // the problem's last warp ends its step
    // per-problem constants, in the arithmetic of set_derived (1/dx and 1/dy
    // from the problem table, made on the host)
    double rx_, ry_, M_, bx_, by_;
    __device__ __forceinline__ T rxT() const { return T(rx_); }
    __device__ __forceinline__ T ryT() const { return T(ry_); }
    __device__ __forceinline__ T Mdx2T() const { return T(M_ * dx_ * dx_); }
    __device__ __forceinline__ T Mdy2T() const { return T(M_ * dy_ * dy_); }
    __device__ __forceinline__ double cell() const { return dx_ * dy_; }
    __device__ __forceinline__ double adv_speed() const { return fabs(bx_) / dx_ + fabs(by_) / dy_; }
};

// Device run-state update after a step from the reduced slots: t, the next
// dt = min(cfl / max speed, t_end - t), totals, troubled count.
// cfl, t_end, lim_count: the run state's values (not written by the step)
__device__ __forceinline__ void finish_run_state(const StepArgs& a, DevState* ds, double mx, const double* sm_,
                                                 int nv, double tr, double t0, double dt, double cfl,
                                                 double t_end, unsigned lim_count, int* cur, unsigned* done) {
    ds->maxspeed = mx;
    for (int v = 0; v < nv; ++v) ds->sums[v] = sm_[v];
    // troubled cells: this step's limit-on-load, else a separate pass over u^n
    ds->troubled = a.limit ? tr : double(lim_count);
    ds->lim_count = 0;
    const double tn = t0 + dt;
    ds->t = tn;
    double dn = cfl > 0.0 && mx > 0.0 ? cfl / mx : dt;
    const double rem = t_end - tn;
    const bool reached = rem <= 1e-12 * fmax(1.0, fabs(t_end));
    if (dn > rem) dn = rem;
    if (reached) dn = 0.0;
    ds->dt = dn;
    ds->steps += 1;
    ds->counter = 0;
    if (cur) *cur ^= 1;
    if (done && reached) atomicAdd(done, 1u);
}

// FP64 epilogue of a step: warp reduction of the lane accumulators (max
// wave speed, NV totals, troubled count, status bits) into the warp's slot
// (NV + 2 doubles).  Single problems (PV::kLastWarp false) leave the rest to
// finalize_step_kernel, launched after the step; in a batch the last warp of
// a problem to arrive (atomic counter, no waiting) reduces that problem's
// slots in a fixed order and updates its run state.
template <int NV, int NRED, class PV>
__device__ __forceinline__ void step_epilogue(const StepArgs& a, const PV& pv, int gw, int lane, int total_warps,
                                              double red_max, double* red_sum, unsigned red_trouble,
                                              unsigned status, double cell, double t0, double dt) {
    static_assert(NRED == NV + 2, "slot layout: max speed, NV totals, troubled count");
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        red_max = fmax(red_max, __shfl_xor_sync(0xffffffffu, red_max, off));
#pragma unroll
        for (int v = 0; v < NV; ++v) red_sum[v] += __shfl_xor_sync(0xffffffffu, red_sum[v], off);
        red_trouble += __shfl_xor_sync(0xffffffffu, red_trouble, off);
        status |= __shfl_xor_sync(0xffffffffu, status, off);
    }
    double* slotp = pv.partials() + (size_t)gw * NRED;
    unsigned prev = 0;
    if (lane == 0) {
        slotp[0] = red_max;
#pragma unroll
        for (int v = 0; v < NV; ++v) slotp[1 + v] = red_sum[v] * cell;
        slotp[1 + NV] = __longlong_as_double((long long)red_trouble);   // an integer, stored bitwise
        if (status) atomicOr(&pv.ds()->status, status);
        if constexpr (PV::kLastWarp) {
            __threadfence();
            prev = atomicAdd(&pv.ds()->counter, 1u);
        }
    }
    if constexpr (!PV::kLastWarp) {
        return;
    } else {
        prev = __shfl_sync(0xffffffffu, prev, 0);
        if (prev != (unsigned)total_warps - 1) return;
        // last warp: fixed-order reduction of all per-warp slots (deterministic)
        __threadfence();
        double mx = 0.0, sm_[NV], tr = 0.0;
#pragma unroll
        for (int v = 0; v < NV; ++v) sm_[v] = 0.0;
        for (int wi = lane; wi < total_warps; wi += 32) {
            const double* q = pv.partials() + (size_t)wi * NRED;
            mx = fmax(mx, __ldcg(q));
#pragma unroll
            for (int v = 0; v < NV; ++v) sm_[v] += __ldcg(q + 1 + v);
            tr += double(__double_as_longlong(__ldcg(q + 1 + NV)));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
#pragma unroll
            for (int v = 0; v < NV; ++v) sm_[v] += __shfl_xor_sync(0xffffffffu, sm_[v], off);
            tr += __shfl_xor_sync(0xffffffffu, tr, off);
        }
        if (lane == 0) {
            DevState* ds = pv.ds();
            finish_run_state(a, ds, mx, sm_, NV, tr, t0, dt, ds->cfl, ds->t_end, ds->lim_count, pv.cur(), pv.done());
        }
    }
}

// The end of a single-problem step, as its own launch of one block (the
// step's slots are complete when it starts): each thread reduces a run of
// slots with their loads in flight together, then fixed-order trees
// (deterministic); thread 0 updates the device run state.  A last warp of the
// step itself would reduce ~1,000-2,400 slots alone while the rest of the GPU
// idles.  The block runs on one SM, whose FP64 pipe (1/64 of the FP32 rate)
// would bound it: only the NV totals are added in FP64; the maximum wave
// speed is taken on the bit patterns (non-negative doubles order as integers)
// and the troubled count is an integer.
constexpr int FINALIZE_THREADS = 256;

// a slot's speed as an ordered key: NaN (ignored, as fmax does) and -0 map to 0
__device__ __forceinline__ unsigned long long speed_key(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const bool neg = b >> 63, nan = (b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
    return neg || nan ? 0ull : b;
}

template <int NV>
__global__ void __launch_bounds__(FINALIZE_THREADS) finalize_step_kernel(const StepArgs a, int total_warps) {
    constexpr int NRED = NV + 2;
    // launched as a programmatic dependent of the step: wait here until the
    // step grid has completed and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    DevState* ds = a.ds;
    // every load is issued before any result is needed: the run state (none
    // of these fields is written by the step) and the thread's slots
    const double t0 = a.dt_from_dev ? ds->t : a.t;
    const double dt = a.dt_from_dev ? ds->dt : a.dt;
    const double cfl = ds->cfl, t_end = ds->t_end;
    const unsigned lim_count = ds->lim_count;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long mk = 0, tr = 0;
    double sm_[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) sm_[v] = 0.0;
    // chunks of PER slots per thread, loaded unconditionally from valid
    // addresses (slot 0 past the end, masked) so that all are in flight at once
    constexpr int PER = 8;
    for (int base = threadIdx.x; base < total_warps; base += PER * FINALIZE_THREADS) {
        double qv[PER][NRED];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int wi = base + k * FINALIZE_THREADS;
            const double* q = a.partials + (size_t)(wi < total_warps ? wi : 0) * NRED;
#pragma unroll
            for (int e = 0; e < NRED; ++e) qv[k][e] = q[e];
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (base + k * FINALIZE_THREADS >= total_warps) break;
            const unsigned long long key = speed_key(qv[k][0]);
            mk = key > mk ? key : mk;
#pragma unroll
            for (int v = 0; v < NV; ++v) sm_[v] += qv[k][1 + v];
            tr += (unsigned long long)__double_as_longlong(qv[k][1 + NV]);
        }
    }
    auto warp_tree = [&]() {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long k = __shfl_xor_sync(0xffffffffu, mk, off);
            mk = k > mk ? k : mk;
#pragma unroll
            for (int v = 0; v < NV; ++v) sm_[v] += __shfl_xor_sync(0xffffffffu, sm_[v], off);
            tr += __shfl_xor_sync(0xffffffffu, tr, off);
        }
    };
    if (!(dt > 0.0)) return;   // the step left the state and the run state unchanged
    warp_tree();
    constexpr int NW = FINALIZE_THREADS / 32;
    __shared__ unsigned long long red_k[NW], red_t[NW];
    __shared__ double red_s[NW][NV];
    if (lane == 0) {
        red_k[w] = mk;
        red_t[w] = tr;
#pragma unroll
        for (int v = 0; v < NV; ++v) red_s[w][v] = sm_[v];
    }
    __syncthreads();
    if (w != 0) return;
    mk = lane < NW ? red_k[lane] : 0ull;
    tr = lane < NW ? red_t[lane] : 0ull;
#pragma unroll
    for (int v = 0; v < NV; ++v) sm_[v] = lane < NW ? red_s[lane][v] : 0.0;
    warp_tree();
    if (lane == 0)
        finish_run_state(a, ds, __longlong_as_double((long long)mk), sm_, NV, double(tr), t0, dt, cfl, t_end, lim_count,
                         nullptr, nullptr);
}

// launch of finalize_step_kernel after a single-problem step launched with b,
// as a programmatic dependent launch: the step's blocks allow it early
// (griddepcontrol.launch_dependents), so its block is scheduled as soon as an
// SM has room and only waits for the step's completion, without a launch gap
template <int NV>
inline cudaError_t launch_finalize(const StepArgs& b, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(FINALIZE_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, finalize_step_kernel<NV>, b, b.n_strips * b.n_segs);
}

// In a step kernel: its dependent finalize launch may be scheduled now
__device__ __forceinline__ void allow_dependent_launch() { asm volatile("griddepcontrol.launch_dependents;"); }

// COMP = true: compensated FP32 state.  The buffers hold hi planes followed
// by lo planes (u = hi + lo); every stage computes in T from hi, and only the
// final update u^{n+1} = u^n + Delta is accumulated exactly (TwoSum of hi and
// Delta + lo), so the state does not collect one rounding of its own size
// per step.  Used without limiters.
// MLPI = true: the troubled-cell decision of the limit-on-load comes from the
// learned indicator (BF16 tensor-core MLP over the warp's 32 cells): limit if
// the logit exceeds mlp_zhi, keep if it is below mlp_zlo, and let the TVB test
// decide in between.  The weights sit in shared memory after the threads'
// private slots, followed by one staging area per warp.
template <class T, int K, int B, int PHYS>
__host__ __device__ constexpr size_t mlp_smem_offset(int s, int nthr) {
    return ((size_t)Step2D<T, K, B, PHYS>::smem_per_thread(s) * sizeof(T) * nthr + 15) / 16 * 16;
}
constexpr size_t mlp_smem_bytes(int nthr) {
    return sizeof(MlpSmem) + (size_t)(nthr / 32) * (32 * MLP_INP + 64) * sizeof(__nv_bfloat16);
}

// LIM = false: an instantiation without the limit-on-load code, for steps
// whose u^n needs no limiting here (none pending, or a separate pass did it).
// DEV = true (with COMP, 2D Euler, FP32): every state is held as its
// deviation from the cell's base state (the high part of its average at t^n)
// and every flux in deviation form (EulerDev), so that the stage operators
// and the final stage carry FP32 errors relative to their own size; the
// compensated state then accumulates increments that are accurate to a few
// ulps of themselves.  Face traces and face fluxes that cross to a
// neighbouring cell move to its base by the deviation of the base
// difference.  Inner stages, final stage and the update all run on the FP32
// pipe.
// SQ = true (square cells, dx == dy, so 1/dx == 1/dy): the face terms
// accumulate without the 1/dx factors, applied once to each local-operator
// value and to the update (rx (sx + sy) - V for rx sx + ry sy - V): 4 packed
// multiplications per face point fewer.
template <class T, int K, int B, int PHYS, bool COMP = false, bool MLPI = false, bool LIM = true, bool DEV = false,
          bool SQ = false, class PV>
__device__ __forceinline__ void step2d_body(const StepArgs& a, const PV& pv, const int gw) {
    static_assert(!DEV || (COMP && PHYS == PHYS_EULER && sizeof(T) == 4 && !MLPI && !LIM && !CRK_LF_REUSE),
                  "the deviation form is built for the compensated FP32 2D Euler step without limiters");
    static_assert(!SQ || !CRK_LF_REUSE, "the square-cell form is built without the reused face fluxes");
    using C = Step2D<T, K, B, PHYS>;
    using TBL = typename C::TB;
    constexpr int NQ = C::NQ, NQV = C::NQV, NM = C::NM, NV = C::NV;
    constexpr TBL tb = make_tab2d<K, B>();

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;
    const int S = a.s;
    const int offN = (S - 1) * C::NDOF;
    const int offP = offN + S * NQ * NV;
    const int offV = offP + C::NDOF;
    const int offNF = offV + (CRK_V_SMEM ? C::NDOF : 0);   // north fluxes + speeds (CRK_LF_REUSE)
    // the thread's private slots: its warp holds smem_per_thread(S) rows of
    // 32 values, one column per lane (consecutive lanes in consecutive banks),
    // so that slot k sits k * 32 values past the thread's own base
    T* const smt = sm + (size_t)(tid >> 5) * (C::smem_per_thread(S) * 32) + (tid & 31);
    auto slot = [&](int k) -> T& { return smt[k * 32]; };

    const int lane = tid & 31;
    const int total_warps = pv.total_warps();

    const int nx = pv.nx(), ny = pv.ny();
    const size_t plane = (size_t)nx * ny;
    const T* __restrict__ uin = pv.uin();
    T* __restrict__ uout = pv.uout();

    const double dt = pv.dt();
    const double t0 = pv.t();

    const int strip = gw % pv.n_strips();
    const int seg = gw / pv.n_strips();
    const int xs = strip * 30;
    const int col = xs - 1 + lane;
    const bool perx = a.bc[0].type == BC_PERIODIC;
    const bool pery = a.bc[2].type == BC_PERIODIC;
    int xl = ((col % nx) + nx) % nx;
    if (!perx) xl = col < 0 ? 0 : (col >= nx ? nx - 1 : col);
    const bool outlane = lane >= 1 && lane <= 30 && col < nx;
    const bool has_bcW = !perx && xs == 0;
    const bool has_bcE = !perx && xs + 30 >= nx;

    // rows split evenly over the segments (each at most seg_len rows)
    const int r0 = (int)(((long long)seg * ny) / pv.n_segs());
    const int r1 = (int)(((long long)(seg + 1) * ny) / pv.n_segs());
    const int rstart = (r0 > 0 || pery) ? r0 - 1 : r0;
    const int rend = (r1 < ny || pery) ? r1 : r1 - 1;

    // a non-positive dt leaves the state unchanged (runs past t_end)
    if (!(dt > 0.0)) {
        if (pv.copy_if_idle() && outlane)
            for (int r = r0; r < r1; ++r)
                for (int d = 0; d < (COMP ? 2 : 1) * C::NDOF; ++d)
                    uout[d * plane + (size_t)r * nx + col] = uin[d * plane + (size_t)r * nx + col];
        return;
    }

    // launch constants: 1/dx, 1/dy and the limiter thresholds made on the host
    // (set_derived), no FP64 division per warp
    constexpr bool F32 = sizeof(T) == 4;
    std::conditional_t<DEV, EulerDev<T>, Phys<T, PHYS>> ph;
    if constexpr (PHYS == PHYS_EULER) {
        ph.gamma = T(a.gamma);
        ph.gm1 = T(a.gamma - 1.0);
    } else {
        ph.bx = T(a.beta[0]);
        ph.by = T(a.beta[1]);
    }
    const T rx = opaque(pv.rxT()), ry = opaque(pv.ryT());   // held in registers, as when computed
    // the factors of the face terms (SQ: 1, applied later); the volume
    // term keeps its factors, whose products also form the register pairs of
    // its packed accumulation
    const T rxv = SQ ? T(1) : rx, ryv = SQ ? T(1) : ry;
    const T tdt = T(dt);
    const T Mdx2 = pv.Mdx2T(), Mdy2 = pv.Mdy2T();
    const T gam = T(a.gamma);
    const bool do_tvb = a.tvb_on, do_pp = a.pp_on;
    const T pp_eps = F32 ? T(a.pp_epsf) : T(a.pp_eps);

    // FP32 state (plain or compensated): the per-cell wave speed and status
    // tests of the epilogue run in FP32 (GB300's FP64 pipe is 1/64 of its FP32
    // rate), the column totals in compensated FP32 (TwoSum; a compensated
    // state adds its lo parts into the error term), converted to FP64 once per
    // warp
    constexpr bool F32R = sizeof(T) == 4;
    T cs_hi[NV], cs_lo[NV];
    T red_maxT = T(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) cs_hi[v] = cs_lo[v] = T(0);
    const double adv_speed = PHYS == PHYS_EULER ? 0.0 : pv.adv_speed();

    // reduction accumulators (FP64)
    double red_max = 0.0;
    double red_sum[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) red_sum[v] = 0.0;
    unsigned red_trouble = 0;
    unsigned status = 0;

    // limiter: rolling neighbour averages of this column
    T avg_prev[NV], avg_next[NV];
    auto load_avg = [&](int r, T* out) {
        // average of (column xl, row r), r in [-1, ny]; beyond a non-periodic
        // side: ghost average from the boundary cell (at time t^n)
        int rr = r;
        bool ghost = false;
        if (r < 0) { if (pery) rr = r + ny; else { rr = 0; ghost = true; } }
        if (r >= ny) { if (pery) rr = r - ny; else { rr = ny - 1; ghost = true; } }
        T own[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) own[v] = uin[(size_t)(v * NM) * plane + (size_t)rr * nx + xl];
        if (!ghost) {
#pragma unroll
            for (int v = 0; v < NV; ++v) out[v] = own[v];
        } else {
            cold_branch();
            const int side = r < 0 ? 2 : 3;
            const int colc = opaque(col);
            bc_exterior<T, NV>(a.bc[side], 1, own, [&](double& x, double& y, double& t) {
                x = pv.x0() + (colc + 0.5) * pv.dx();
                y = r < 0 ? pv.y0() - 0.5 * pv.dy() : pv.y0() + (ny + 0.5) * pv.dy();
                t = t0;
            }, out);
        }
    };
    auto load_avg_x = [&](int c, int r, T* out) {
        // average of column c (may be -1 .. nx) in row r (0..ny-1)
        T own[NV];
        int cc = perx ? ((c % nx) + nx) % nx : (c < 0 ? 0 : (c >= nx ? nx - 1 : c));
#pragma unroll
        for (int v = 0; v < NV; ++v) own[v] = uin[(size_t)(v * NM) * plane + (size_t)r * nx + cc];
        if (perx || (c >= 0 && c < nx)) {
#pragma unroll
            for (int v = 0; v < NV; ++v) out[v] = own[v];
        } else {
            cold_branch();
            const int side = c < 0 ? 0 : 1;
            const int rc = opaque(r);
            bc_exterior<T, NV>(a.bc[side], 0, own, [&](double& x, double& y, double& t) {
                x = c < 0 ? pv.x0() - 0.5 * pv.dx() : pv.x0() + (nx + 0.5) * pv.dx();
                y = pv.y0() + (rc + 0.5) * pv.dy();
                t = t0;
            }, out);
        }
    };
    if (LIM && a.limit) load_avg(rstart - 1, avg_prev);
    T cprev[NV];   // DEV: base state of the row below (the previous row of the march)
#pragma unroll
    for (int v = 0; v < NV; ++v) cprev[v] = T(0);
    const double hh_ = pv.dx() > pv.dy() ? pv.dx() : pv.dy();
    const double mlp_scale = a.M * hh_ * hh_;

    for (int r = rstart; r <= rend; ++r) {
        const int ry_ = r < 0 ? r + ny : (r >= ny ? r - ny : r);
        const bool out_row = r >= r0 && r < r1;
        const bool south_bc = (r == 0) && !pery;
        const bool do_south = (r > rstart) || south_bc;   // flux through this row's south face
        const bool keep_north = r < rend || (r == ny - 1 && !pery && out_row);

        // ---- load u^n (and limit on load) -------------------------------------
        T un[NV][NM];
        const size_t cidx = (size_t)ry_ * nx + xl;
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int m = 0; m < NM; ++m) un[v][m] = uin[(size_t)(v * NM + m) * plane + cidx];

        // DEV: the base cb = hi part of the average; un becomes the deviation
        // (lo of the average, hi + lo of the higher modes); cS is the base of
        // the row below.  The neighbours' bases minus this cell's are formed
        // where they are used (fewer live registers)
        T cb[NV], cS[NV];
        if constexpr (DEV) {
            const size_t lo_off = (size_t)C::NDOF * plane;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                cb[v] = un[v][0];
                un[v][0] = uin[lo_off + (size_t)(v * NM) * plane + cidx];
#pragma unroll
                for (int m = 1; m < NM; ++m) un[v][m] += uin[lo_off + (size_t)(v * NM + m) * plane + cidx];
            }
            ph.set_base(cb);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                cS[v] = cprev[v];
                cprev[v] = cb[v];
            }
        }
        // exterior state at a boundary point from an interior trace (DEV:
        // both as deviations from this cell's base; the affine sides exactly)
        auto bcx = [&](const BCSide& bc, int axis, const T* din, auto&& xyt, T* out) {
            if constexpr (DEV) {
                if (bc.affine) {
#pragma unroll
                    for (int v = 0; v < NV; ++v)
                        out[v] = fma(T(bc.m[v]), din[v], fma(T(bc.m[v]) - T(1), cb[v], T(bc.cf[v])));
                } else {
                    T full[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) full[v] = cb[v] + din[v];
                    bc_exterior<T, NV>(bc, axis, full, xyt, out);
#pragma unroll
                    for (int v = 0; v < NV; ++v) out[v] -= cb[v];
                }
            } else {
                bc_exterior<T, NV>(bc, axis, din, xyt, out);
            }
        };

        if (LIM && a.limit) {
            T avg_cur[NV], nbW[NV], nbE[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) avg_cur[v] = un[v][0];
            load_avg(r + 1, avg_next);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                nbE[v] = shfl_down(avg_cur[v], 1);
                nbW[v] = shfl_up(avg_cur[v], 1);
            }
            if (lane == 0) load_avg_x(col - 1, ry_, nbW);
            if (lane == 31) load_avg_x(col + 1, ry_, nbE);
            if (!perx && col == 0) load_avg_x(-1, ry_, nbW);
            if (!perx && col == nx - 1) load_avg_x(nx, ry_, nbE);
            const bool real = perx ? true : (col >= 0 && col < nx);
            bool fl = false;
            int mode = -1;
            if constexpr (MLPI) {
                // every lane takes part in the warp's MLP evaluation
                unsigned char* base = smem_raw + mlp_smem_offset<T, K, B, PHYS>(S, nthr);
                const MlpSmem& mw = *reinterpret_cast<const MlpSmem*>(base);
                __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(base + sizeof(MlpSmem)) +
                                       (tid >> 5) * (32 * MLP_INP + 64);
                float feat[MLP_IN];
                mlp_features<T, NM>(un, nbE, nbW, avg_next, avg_prev, mlp_scale, feat);
                const float z = mlp_warp_logit(mw, feat, stage);
                mode = z > a.mlp_zhi ? 1 : (z < a.mlp_zlo ? 0 : -1);
            }
            if (real && do_tvb)
                fl = tvb_limit_cell<T, NV, NM>(un, nbW, nbE, avg_prev, avg_next, Mdx2, Mdy2, gam, mode);
            if (real && do_pp) positivity_cell<T, NV, NM, K, B>(un, gam, pp_eps);
            if (out_row && outlane && fl) ++red_trouble;
#pragma unroll
            for (int v = 0; v < NV; ++v) avg_prev[v] = avg_cur[v];
        }

        // ---- stages ---------------------------------------------------------------
        T Vr[CRK_V_SMEM ? 1 : NV][CRK_V_SMEM ? 1 : NM];   // sum_i b_i * volume term (registers)
        auto V = [&](int v, int m) -> T& {
            if constexpr (CRK_V_SMEM) return slot(offV + v * NM + m);
            else return Vr[v][m];
        };
        T FE[NQ][NV];     // sum_i b_i fhat on the east face
        T FS[NQ][NV];     // sum_i b_i fhat on the south face
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int m = 0; m < NM; ++m) V(v, m) = T(0);
#pragma unroll
        for (int p = 0; p < NQ; ++p)
#pragma unroll
            for (int v = 0; v < NV; ++v) FE[p][v] = FS[p][v] = T(0);

        for (int i = 0; i < S; ++i) {
            const T bi = tab_bT<T>(a, i);
            const T hbi = T(0.5) * bi;   // the weight of the east and south fluxes formed without their 1/2
            const bool need_L = i < S - 1;
            const bool need_flux = bi != T(0);
            if (!need_L && !need_flux) continue;
            // stage state u^(i) = u^n - dt sum_{j<i} a_ij L_j
            T w[NV][NM];
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 0; m < NM; ++m) w[v][m] = un[v][m];
            for (int j = 0; j < i; ++j) {
                const T aijT = tab_aT<T>(a, i, j);
                if (aijT == T(0)) continue;
                const T aij = aijT * tdt;
                if constexpr (NV % 2 == 0) {
#pragma unroll
                    for (int v = 0; v < NV; v += 2)
#pragma unroll
                        for (int m = 0; m < NM; ++m)
                            pfma(w[v][m], w[v + 1][m], slot(j * C::NDOF + v * NM + m),
                                 slot(j * C::NDOF + (v + 1) * NM + m), -aij);
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v)
#pragma unroll
                        for (int m = 0; m < NM; ++m) w[v][m] -= aij * slot(j * C::NDOF + v * NM + m);
                }
            }
            // volume term  sum_q w_q (rx f_x dphi/dxi + ry f_y dphi/deta)
            T vol[NV][NM];
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 0; m < NM; ++m) vol[v][m] = T(0);
            // flux and projection of the point values uq at volume point q
            auto vol_point = [&](const int q, const T (&uq)[NV]) {
                T fx[NV], fy[NV];
                ph.flux2(uq, fx, fy);
                if constexpr (NV % 2 == 0) {
#pragma unroll
                    for (int v = 0; v < NV; v += 2) {
                        const T gx0 = rx * fx[v], gx1 = rx * fx[v + 1], gy0 = ry * fy[v], gy1 = ry * fy[v + 1];
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            if (tb.gx[q][m] != 0.0) pfma(vol[v][m], vol[v + 1][m], gx0, gx1, T(tb.gx[q][m]));
                            if (tb.gy[q][m] != 0.0) pfma(vol[v][m], vol[v + 1][m], gy0, gy1, T(tb.gy[q][m]));
                        }
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const T gxv = rx * fx[v], gyv = ry * fy[v];
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            if (tb.gx[q][m] != 0.0) vol[v][m] += gxv * T(tb.gx[q][m]);
                            if (tb.gy[q][m] != 0.0) vol[v][m] += gyv * T(tb.gy[q][m]);
                        }
                    }
                }
            };
            // a mirrored pair of points (q at xi, its mirror at -xi): w_q dphi/dxi
            // changes sign with (-1)^(i-1) and w_q dphi/deta with (-1)^i, so
            // each mode takes the sum or the difference of the two points'
            // fluxes: one product per mode and direction for both points
            auto vol_pair = [&](const int q, const T (&uq)[NV], const T (&uqm)[NV]) {
                T fx[NV], fy[NV], hx[NV], hy[NV];
                ph.flux2(uq, fx, fy);
                ph.flux2(uqm, hx, hy);
                if constexpr (NV % 2 == 0) {
#pragma unroll
                    for (int v = 0; v < NV; v += 2) {
                        T sx0, sx1, dx0, dx1, sy0, sy1, dy0, dy1;
                        padd(sx0, sx1, fx[v], fx[v + 1], hx[v], hx[v + 1]);
                        psub(dx0, dx1, fx[v], fx[v + 1], hx[v], hx[v + 1]);
                        padd(sy0, sy1, fy[v], fy[v + 1], hy[v], hy[v + 1]);
                        psub(dy0, dy1, fy[v], fy[v + 1], hy[v], hy[v + 1]);
                        pmul(sx0, sx1, rx);
                        pmul(dx0, dx1, rx);
                        pmul(sy0, sy1, ry);
                        pmul(dy0, dy1, ry);
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            if (tb.gx[q][m] != 0.0) {
                                if (tb.ip[m] == 0) pfma(vol[v][m], vol[v + 1][m], dx0, dx1, T(tb.gx[q][m]));
                                else pfma(vol[v][m], vol[v + 1][m], sx0, sx1, T(tb.gx[q][m]));
                            }
                            if (tb.gy[q][m] != 0.0) {
                                if (tb.ip[m] == 0) pfma(vol[v][m], vol[v + 1][m], sy0, sy1, T(tb.gy[q][m]));
                                else pfma(vol[v][m], vol[v + 1][m], dy0, dy1, T(tb.gy[q][m]));
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const T sxv = rx * (fx[v] + hx[v]), dxv = rx * (fx[v] - hx[v]);
                        const T syv = ry * (fy[v] + hy[v]), dyv = ry * (fy[v] - hy[v]);
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            if (tb.gx[q][m] != 0.0) vol[v][m] += (tb.ip[m] == 0 ? dxv : sxv) * T(tb.gx[q][m]);
                            if (tb.gy[q][m] != 0.0) vol[v][m] += (tb.ip[m] == 0 ? syv : dyv) * T(tb.gy[q][m]);
                        }
                    }
                }
            };
            // point values in mirrored pairs: phi_m(-xi, eta) = (-1)^i phi_m(xi,
            // eta), so the values at xi_a and at -xi_a are the sum and the
            // difference of the even-i and odd-i parts of one contraction (the
            // middle column xi = 0 has no odd part)
#pragma unroll
            for (int q = 0; q < NQV; ++q) {
                const int qa = q / NQ, qb = q % NQ, qm = (NQ - 1 - qa) * NQ + qb;
                if (qa > NQ - 1 - qa) continue;   // evaluated with its mirror point
                T uq[NV], uqm[NV];
                if constexpr (NV % 2 == 0) {
#pragma unroll
                    for (int v = 0; v < NV; v += 2) {
                        T e0 = T(0), e1 = T(0), o0 = T(0), o1 = T(0);
#pragma unroll
                        for (int m = 0; m < NM; ++m)   // (P_1 vanishes at the middle Gauss point)
                            if (tb.phi[q][m] != 0.0) {
                                if (tb.ip[m] == 0) pfma(e0, e1, w[v][m], w[v + 1][m], T(tb.phi[q][m]));
                                else pfma(o0, o1, w[v][m], w[v + 1][m], T(tb.phi[q][m]));
                            }
                        padd(uq[v], uq[v + 1], e0, e1, o0, o1);
                        psub(uqm[v], uqm[v + 1], e0, e1, o0, o1);
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        T e = T(0), o = T(0);
#pragma unroll
                        for (int m = 0; m < NM; ++m)
                            if (tb.phi[q][m] != 0.0) {
                                if (tb.ip[m] == 0) e += w[v][m] * T(tb.phi[q][m]);
                                else o += w[v][m] * T(tb.phi[q][m]);
                            }
                        uq[v] = e + o;
                        uqm[v] = e - o;
                    }
                }
                if (qa < NQ - 1 - qa) vol_pair(q, uq, uqm);
                else vol_point(q, uq);
            }
            if (need_flux && out_row) {
                if constexpr (NV % 2 == 0) {
#pragma unroll
                    for (int v = 0; v < NV; v += 2)
#pragma unroll
                        for (int m = 0; m < NM; ++m) pfma(V(v, m), V(v + 1, m), vol[v][m], vol[v + 1][m], bi);
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v)
#pragma unroll
                        for (int m = 0; m < NM; ++m) V(v, m) += bi * vol[v][m];
                }
            }
            // face traces.  phi_m(-1, eta) = (-1)^i phi_m(1, eta): the east and
            // west traces are the sum and difference of the even-i and odd-i
            // parts of one contraction (north and south likewise in j)
            T tE[NQ][NV], tW[NQ][NV], tN[NQ][NV], tS[NQ][NV];
            if constexpr (NV % 2 == 0) {
#pragma unroll
                for (int p = 0; p < NQ; ++p)
#pragma unroll
                    for (int v = 0; v < NV; v += 2) {
                        T xe0 = 0, xe1 = 0, xo0 = 0, xo1 = 0, ye0 = 0, ye1 = 0, yo0 = 0, yo1 = 0;
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            if (tb.tE[p][m] != 0.0) {
                                if (tb.ip[m] == 0) pfma(xe0, xe1, w[v][m], w[v + 1][m], T(tb.tE[p][m]));
                                else pfma(xo0, xo1, w[v][m], w[v + 1][m], T(tb.tE[p][m]));
                            }
                            if (tb.tN[p][m] != 0.0) {
                                if (tb.jp[m] == 0) pfma(ye0, ye1, w[v][m], w[v + 1][m], T(tb.tN[p][m]));
                                else pfma(yo0, yo1, w[v][m], w[v + 1][m], T(tb.tN[p][m]));
                            }
                        }
                        padd(tE[p][v], tE[p][v + 1], xe0, xe1, xo0, xo1);
                        psub(tW[p][v], tW[p][v + 1], xe0, xe1, xo0, xo1);
                        padd(tN[p][v], tN[p][v + 1], ye0, ye1, yo0, yo1);
                        psub(tS[p][v], tS[p][v + 1], ye0, ye1, yo0, yo1);
                    }
            } else {
#pragma unroll
            for (int p = 0; p < NQ; ++p)
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    T e = 0, ww = 0, n = 0, s = 0;
#pragma unroll
                    for (int m = 0; m < NM; ++m) {
                        e += w[v][m] * T(tb.tE[p][m]);
                        ww += w[v][m] * T(tb.tW[p][m]);
                        n += w[v][m] * T(tb.tN[p][m]);
                        s += w[v][m] * T(tb.tS[p][m]);
                    }
                    tE[p][v] = e; tW[p][v] = ww; tN[p][v] = n; tS[p][v] = s;
                }
            }
            // east/south Lax--Friedrichs fluxes formed inside the local operator's
            // point loop (boundary strips and rows keep the separate path below)
            const bool fuseE = CRK_LF_REUSE && need_L && need_flux && out_row && !has_bcW && !has_bcE;
            const bool fuseS = CRK_LF_REUSE && need_L && need_flux && do_south && !south_bc;
            T tWn[NQ][NV];
            if (fuseE) {
#pragma unroll
                for (int p = 0; p < NQ; ++p)
#pragma unroll
                    for (int v = 0; v < NV; ++v) tWn[p][v] = shfl_down(tW[p][v], 1);
            }
            // local operator L_i = cm (face_loc - vol), eq. (2.7)
            if (need_L) {
                T floc[NV][NM];
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int m = 0; m < NM; ++m) floc[v][m] = T(0);
#pragma unroll
                for (int p = 0; p < NQ; ++p) {
                    T fe[NV], fw[NV], fn[NV], fs[NV];
                    const T sE = ph.template fluxn<0>(tE[p], fe);
                    const T sW = ph.template fluxn<0>(tW[p], fw);
                    const T sN = ph.template fluxn<1>(tN[p], fn);
                    const T sS = ph.template fluxn<1>(tS[p], fs);
                    if (fuseE) {   // own east trace vs. the right lane's west trace
                        T fwn[NV], F[NV];
#pragma unroll
                        for (int v = 0; v < NV; ++v) fwn[v] = shfl_down(fw[v], 1);
                        const T sWn = shfl_down(sW, 1);
                        lf_from_fluxes<T, NV>(tE[p], fe, sE, tWn[p], fwn, sWn, F);
#pragma unroll
                        for (int v = 0; v < NV; ++v) FE[p][v] += bi * F[v];
                    }
                    if (fuseS) {   // the row below's north trace vs. own south trace
                        T lo[NV], flo[NV], F[NV];
#pragma unroll
                        for (int v = 0; v < NV; ++v) {
                            lo[v] = slot(offN + (i * NQ + p) * NV + v);
                            flo[v] = slot(offNF + (i * NQ + p) * (NV + 1) + v);
                        }
                        const T slo = slot(offNF + (i * NQ + p) * (NV + 1) + NV);
                        lf_from_fluxes<T, NV>(lo, flo, slo, tS[p], fs, sS, F);
#pragma unroll
                        for (int v = 0; v < NV; ++v) FS[p][v] += bi * F[v];
                    }
                    if (CRK_LF_REUSE && keep_north) {
#pragma unroll
                        for (int v = 0; v < NV; ++v) slot(offNF + (i * NQ + p) * (NV + 1) + v) = fn[v];
                        slot(offNF + (i * NQ + p) * (NV + 1) + NV) = sN;
                    }
                    if constexpr (NV % 2 == 0) {
                        // pW = (-1)^i pE, pS = (-1)^j pN: fe pE - fw pW = pE (fe -+ fw)
#pragma unroll
                        for (int v = 0; v < NV; v += 2) {
                            T xm0, xm1, xp0, xp1, ym0, ym1, yp0, yp1;
                            psub(xm0, xm1, fe[v], fe[v + 1], fw[v], fw[v + 1]);
                            padd(xp0, xp1, fe[v], fe[v + 1], fw[v], fw[v + 1]);
                            psub(ym0, ym1, fn[v], fn[v + 1], fs[v], fs[v + 1]);
                            padd(yp0, yp1, fn[v], fn[v + 1], fs[v], fs[v + 1]);
                            if constexpr (!SQ) {
                                pmul(xm0, xm1, rx);
                                pmul(xp0, xp1, rx);
                                pmul(ym0, ym1, ry);
                                pmul(yp0, yp1, ry);
                            }
#pragma unroll
                            for (int m = 0; m < NM; ++m) {
                                if (tb.pE[p][m] != 0.0) {
                                    if (tb.ip[m] == 0) pfma(floc[v][m], floc[v + 1][m], xm0, xm1, T(tb.pE[p][m]));
                                    else pfma(floc[v][m], floc[v + 1][m], xp0, xp1, T(tb.pE[p][m]));
                                }
                                if (tb.pN[p][m] != 0.0) {
                                    if (tb.jp[m] == 0) pfma(floc[v][m], floc[v + 1][m], ym0, ym1, T(tb.pN[p][m]));
                                    else pfma(floc[v][m], floc[v + 1][m], yp0, yp1, T(tb.pN[p][m]));
                                }
                            }
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < NV; ++v)
#pragma unroll
                            for (int m = 0; m < NM; ++m)
                                floc[v][m] += rxv * (fe[v] * T(tb.pE[p][m]) - fw[v] * T(tb.pW[p][m])) +
                                              ryv * (fn[v] * T(tb.pN[p][m]) - fs[v] * T(tb.pS[p][m]));
                    }
                }
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int m = 0; m < NM; ++m)
                        slot(i * C::NDOF + v * NM + m) =
                            T(tb.cm[m]) * (SQ ? fma(rx, floc[v][m], -vol[v][m]) : floc[v][m] - vol[v][m]);
            }
            if (!need_flux) continue;
            // east face: own east trace vs. the west trace of the lane to the right
            if (out_row && !fuseE) {
                T dcE[NV];   // DEV: east neighbour's base minus this cell's
                if constexpr (DEV) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) dcE[v] = shfl_down(cb[v], 1) - cb[v];
                }
#pragma unroll
                for (int p = 0; p < NQ; ++p)
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        tWn[p][v] = shfl_down(tW[p][v], 1);
                        if constexpr (DEV) tWn[p][v] += dcE[v];
                    }
                // boundary strips: the whole warp forms the exterior states (no
                // divergent branch), only the lane at the boundary keeps them
                if (has_bcW) {
                    const bool edge = lane == 0;
                    const BCSide& bcw = a.bc[0];
                    if (bcw.affine) {
#pragma unroll
                        for (int p = 0; p < NQ; ++p)
#pragma unroll
                            for (int v = 0; v < NV; ++v) {
                                T k0 = sizeof(T) == 4 ? T(bcw.cf[v]) : T(bcw.cd[v]);
                                if constexpr (DEV) k0 = fma(T(bcw.m[v]) - T(1), cb[v], k0);
                                const T ext = fma(T(bcw.m[v]), tWn[p][v], k0);
                                tE[p][v] = edge ? ext : tE[p][v];
                            }
                    } else {
                        cold_branch();
                        const int ryc = opaque(ry_), ic = opaque(i);
#pragma unroll
                        for (int p = 0; p < NQ; ++p) {
                            T ext[NV];
                            bcx(bcw, 0, tWn[p], [&](double& x, double& y, double& t) {
                                x = pv.x0();
                                y = pv.y0() + (ryc + 0.5 + 0.5 * tb.xq[p]) * pv.dy();
                                t = t0 + tab_c(a, ic) * dt;
                            }, ext);
#pragma unroll
                            for (int v = 0; v < NV; ++v) tE[p][v] = edge ? ext[v] : tE[p][v];
                        }
                    }
                }
                if (has_bcE) {
                    const bool edge = col == nx - 1;
                    const BCSide& bce = a.bc[1];
                    if (bce.affine) {
#pragma unroll
                        for (int p = 0; p < NQ; ++p)
#pragma unroll
                            for (int v = 0; v < NV; ++v) {
                                T k0 = sizeof(T) == 4 ? T(bce.cf[v]) : T(bce.cd[v]);
                                if constexpr (DEV) k0 = fma(T(bce.m[v]) - T(1), cb[v], k0);
                                const T ext = fma(T(bce.m[v]), tE[p][v], k0);
                                tWn[p][v] = edge ? ext : tWn[p][v];
                            }
                    } else {
                        cold_branch();
                        const int ryc = opaque(ry_), ic = opaque(i);
#pragma unroll
                        for (int p = 0; p < NQ; ++p) {
                            T ext[NV];
                            bcx(bce, 0, tE[p], [&](double& x, double& y, double& t) {
                                x = pv.x0() + nx * pv.dx();
                                y = pv.y0() + (ryc + 0.5 + 0.5 * tb.xq[p]) * pv.dy();
                                t = t0 + tab_c(a, ic) * dt;
                            }, ext);
#pragma unroll
                            for (int v = 0; v < NV; ++v) tWn[p][v] = edge ? ext[v] : tWn[p][v];
                        }
                    }
                }
#pragma unroll
                for (int p = 0; p < NQ; ++p) {
                    T F[NV];
                    llf_ax<0, false>(ph, tE[p], tWn[p], F);
#pragma unroll
                    for (int v = 0; v < NV; ++v) FE[p][v] += hbi * F[v];
                }
            }
            // south face: north trace of the row below (stored) vs. own south trace
            if (do_south && !fuseS) {
                T lo[NQ][NV];
                if (south_bc) {   // row 0 without periodic wrap: boundary data (one uniform branch per row)
                    cold_branch();
                    const int colc = opaque(col), ic = opaque(i);
#pragma unroll
                    for (int p = 0; p < NQ; ++p)
                        bcx(a.bc[2], 1, tS[p], [&](double& x, double& y, double& t) {
                            x = pv.x0() + (colc + 0.5) * pv.dx() + 0.5 * pv.dx() * tb.xq[p];
                            y = pv.y0();
                            t = t0 + tab_c(a, ic) * dt;
                        }, lo[p]);
                } else {
#pragma unroll
                    for (int p = 0; p < NQ; ++p)
#pragma unroll
                        for (int v = 0; v < NV; ++v) {
                            lo[p][v] = slot(offN + (i * NQ + p) * NV + v);
                            if constexpr (DEV) lo[p][v] += cS[v] - cb[v];
                        }
                }
#pragma unroll
                for (int p = 0; p < NQ; ++p) {
                    T F[NV];
                    llf_ax<1, false>(ph, lo[p], tS[p], F);
#pragma unroll
                    for (int v = 0; v < NV; ++v) FS[p][v] += hbi * F[v];
                }
            }
            if (keep_north) {
#pragma unroll
                for (int p = 0; p < NQ; ++p)
#pragma unroll
                    for (int v = 0; v < NV; ++v) slot(offN + (i * NQ + p) * NV + v) = tN[p][v];
            }
        }

        // ---- finish the row below: its north face is this row's south face --------
        auto finish = [&](T (&P)[NV][NM], int rw) {
            // write u^{n+1} of row rw and accumulate the FP64 reductions
            if (!outlane) return;
            const size_t o = (size_t)rw * nx + col;
            if constexpr (F32R) {
                T avl[NV];   // COMP: lo part of the new averages
                if constexpr (COMP) {
                    // P holds Delta: u^{n+1} = (hi + lo) + Delta, hi' + lo' by
                    // TwoSum; P[v][0] becomes hi' of the average
                    const size_t lo_off = (size_t)C::NDOF * plane;
#pragma unroll
                    for (int v = 0; v < NV; ++v)
#pragma unroll
                        for (int m = 0; m < NM; ++m) {
                            const size_t ix = (size_t)(v * NM + m) * plane + o;
                            const T hi = uin[ix], lo = uin[lo_off + ix];
                            const T d = P[v][m] + lo;
                            const T sum = hi + d;
                            const T bv = sum - hi;
                            const T err = (hi - (sum - bv)) + (d - bv);
                            uout[ix] = sum;
                            uout[lo_off + ix] = err;
                            if (m == 0) {
                                P[v][0] = sum;
                                avl[v] = err;
                            }
                        }
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v)
#pragma unroll
                        for (int m = 0; m < NM; ++m) uout[(size_t)(v * NM + m) * plane + o] = P[v][m];
                }
#pragma unroll
                for (int v = 0; v < NV; ++v) {   // TwoSum: cs_hi + cs_lo += P[v][0] exactly
                    const T x = P[v][0];
                    const T sum = cs_hi[v] + x;
                    const T bv = sum - cs_hi[v];
                    cs_lo[v] += (cs_hi[v] - (sum - bv)) + (x - bv);
                    if constexpr (COMP) cs_lo[v] += avl[v];
                    cs_hi[v] = sum;
                }
                if constexpr (PHYS == PHYS_EULER) {
                    const T ir = T(1) / P[0][0];
                    const T w = P[1][0] * ir, vv = P[2][0] * ir;
                    const T p = ph.gm1 * (P[3][0] - T(0.5) * (P[1][0] * w + P[2][0] * vv));
                    const T c = sqrt(fmax(gam * p * ir, T(0)));
                    const T sp = (fabs(w) + c) * rx + (fabs(vv) + c) * ry;
                    if (!(P[0][0] > T(0)) || !(p > T(0))) status |= ST_NONPHYSICAL;
                    if (!(sp == sp)) status |= ST_NAN;
                    red_maxT = fmax(red_maxT, sp);
                } else {
                    if (!(P[0][0] == P[0][0])) status |= ST_NAN;
                }
                return;
            }
            double av[NV];
            if constexpr (COMP) {
                // P holds Delta: u^{n+1} = (hi + lo) + Delta, hi' + lo' by TwoSum
                const size_t lo_off = (size_t)C::NDOF * plane;
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int m = 0; m < NM; ++m) {
                        const size_t ix = (size_t)(v * NM + m) * plane + o;
                        const T hi = uin[ix], lo = uin[lo_off + ix];
                        const T d = P[v][m] + lo;
                        const T sum = hi + d;
                        const T bv = sum - hi;
                        const T err = (hi - (sum - bv)) + (d - bv);
                        uout[ix] = sum;
                        uout[lo_off + ix] = err;
                        if (m == 0) av[v] = double(sum) + double(err);
                    }
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int m = 0; m < NM; ++m) uout[(size_t)(v * NM + m) * plane + o] = P[v][m];
#pragma unroll
                for (int v = 0; v < NV; ++v) av[v] = double(P[v][0]);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) red_sum[v] += av[v];
            double sp;
            if constexpr (PHYS == PHYS_EULER) {
                const double ir = 1.0 / av[0];
                const double w = av[1] * ir, vv = av[2] * ir;
                const double p = (a.gamma - 1.0) * (av[3] - 0.5 * (av[1] * w + av[2] * vv));
                const double c = sqrt(fmax(a.gamma * p * ir, 0.0));
                sp = (fabs(w) + c) / pv.dx() + (fabs(vv) + c) / pv.dy();
                if (!(av[0] > 0.0) || !(p > 0.0)) status |= ST_NONPHYSICAL;
                if (!(sp == sp)) status |= ST_NAN;
            } else {
                sp = adv_speed;
                if (!(av[0] == av[0])) status |= ST_NAN;
            }
            red_max = fmax(red_max, sp);
        };
        if (do_south && r - 1 >= r0 && r - 1 < r1) {
            // DEV: FS is relative to this row's base; the row below takes it
            // relative to its own: minus f_y(c_below) - f_y(c) (sum_i b_i = 1)
            T gS[NV];
            if constexpr (DEV) {
                T dcS[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) dcS[v] = cS[v] - cb[v];
                ph.template fluxn<1>(dcS, gS);
            }
            T P[NV][NM];
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    T s = T(0);
#pragma unroll
                    for (int p = 0; p < NQ; ++p)
                        if (tb.pN[p][m] != 0.0) s += FS[p][v] * T(tb.pN[p][m]);
                    if constexpr (DEV) {
                        if (tb.sN[m] != 0.0) s -= gS[v] * T(tb.sN[m]);
                    }
                    P[v][m] = slot(offP + v * NM + m) - tdt * T(tb.cm[m]) * (ry * s);
                }
            finish(P, r - 1);
        }
        if (!out_row) continue;

        // ---- this row: east/west/south faces and the volume term ----------------------
        // DEV: FE of the lane to the left is relative to its base; moved to this
        // cell's: plus f_x(c_west) - f_x(c)
        T FW[NQ][NV];
#pragma unroll
        for (int p = 0; p < NQ; ++p)
#pragma unroll
            for (int v = 0; v < NV; ++v) FW[p][v] = shfl_up(FE[p][v], 1);
        if constexpr (DEV) {
            T gW[NV], dcW[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) dcW[v] = shfl_up(cb[v], 1) - cb[v];
            ph.template fluxn<0>(dcW, gW);
#pragma unroll
            for (int p = 0; p < NQ; ++p)
#pragma unroll
                for (int v = 0; v < NV; ++v) FW[p][v] += gW[v];
        }
        // east and west faces: pW = (-1)^i pE, so FE pE - FW pW = pE (FE -+ FW)
        T FEm[NQ][NV], FEp[NQ][NV];
#pragma unroll
        for (int p = 0; p < NQ; ++p)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                FEm[p][v] = FE[p][v] - FW[p][v];
                FEp[p][v] = FE[p][v] + FW[p][v];
            }
        T P[NV][NM];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                T sx = T(0), sy = T(0);
#pragma unroll
                for (int p = 0; p < NQ; ++p) {
                    if (tb.pE[p][m] != 0.0) sx += (tb.ip[m] == 0 ? FEm[p][v] : FEp[p][v]) * T(tb.pE[p][m]);
                    if (tb.pS[p][m] != 0.0) sy -= FS[p][v] * T(tb.pS[p][m]);
                }
                const T fsum = SQ ? fma(rx, sx + sy, -V(v, m)) : rx * sx + ry * sy - V(v, m);
                P[v][m] = (COMP ? T(0) : un[v][m]) - tdt * T(tb.cm[m]) * fsum;
            }
        if (r == ny - 1 && !pery) {
            // top boundary: north face flux from the stored north traces
            cold_branch();
            const int colc = opaque(col);
            T FN[NQ][NV];
#pragma unroll
            for (int p = 0; p < NQ; ++p)
#pragma unroll
                for (int v = 0; v < NV; ++v) FN[p][v] = T(0);
            for (int i = 0; i < S; ++i) {
                const T bi = tab_bT<T>(a, i);
                if (bi == T(0)) continue;
                const double ti = t0 + tab_c(a, i) * dt;
#pragma unroll
                for (int p = 0; p < NQ; ++p) {
                    T lo[NV], hi[NV], F[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) lo[v] = slot(offN + (i * NQ + p) * NV + v);
                    bcx(a.bc[3], 1, lo, [&](double& x, double& y, double& t) {
                        x = pv.x0() + (colc + 0.5) * pv.dx() + 0.5 * pv.dx() * tb.xq[p];
                        y = pv.y0() + ny * pv.dy();
                        t = ti;
                    }, hi);
                    llf_ax<1>(ph, lo, hi, F);
#pragma unroll
                    for (int v = 0; v < NV; ++v) FN[p][v] += bi * F[v];
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    T s = T(0);
#pragma unroll
                    for (int p = 0; p < NQ; ++p) s += FN[p][v] * T(tb.pN[p][m]);
                    P[v][m] -= tdt * T(tb.cm[m]) * (ry * s);
                }
            finish(P, r);
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int m = 0; m < NM; ++m) slot(offP + v * NM + m) = P[v][m];
        }
    }

    // ---- FP64 reductions: warp -> per-warp slot -> finalize (batch: last warp) -------
    const double cell = pv.cell();
    if constexpr (F32R) {
        red_max = PHYS == PHYS_EULER ? double(red_maxT) : (outlane && r0 < r1 ? adv_speed : 0.0);
#pragma unroll
        for (int v = 0; v < NV; ++v) red_sum[v] = double(cs_hi[v]) + double(cs_lo[v]);
    }
    step_epilogue<NV, C::NRED>(a, pv, gw, lane, total_warps, red_max, red_sum, red_trouble, status, cell, t0, dt);
}

// One problem: the launch arguments describe the mesh; dt and t come from
// the arguments or from the device run state (device-driven runs).
template <class T, int K, int B, int PHYS, bool COMP = false, bool MLPI = false, bool LIM = true, bool DEV = false,
          bool SQ = false>
__global__ void __launch_bounds__(CRK_STEP_MAXT, PHYS == PHYS_ADV ? CRK_STEP_MINB_ADV : CRK_STEP_MINB2)
    step2d_kernel(const StepArgs a) {
    if constexpr (MLPI) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        MlpSmem& mw = *reinterpret_cast<MlpSmem*>(smem_raw + mlp_smem_offset<T, K, B, PHYS>(a.s, blockDim.x));
        mlp_load_smem(mw, a.mlp);
        __syncthreads();
    }
    allow_dependent_launch();
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= a.n_strips * a.n_segs) return;   // whole warp leaves; no block barriers
    const ArgsView<T> pv{a, a.dt_from_dev ? a.ds->t : a.t, a.dt_from_dev ? a.ds->dt : a.dt};
    step2d_body<T, K, B, PHYS, COMP, MLPI, LIM, DEV, SQ>(a, pv, gw);
}

// Batched ensemble: problems of different sizes and domains share the
// scheme, tableau and boundary types; each has its own state slice, run state
// (t, dt from its own FP64 wave-speed reduction, t_end, status) and buffer
// index.  Warps take (problem, warp) tasks from a flattened table.  A problem
// whose dt is 0 (it reached t_end) costs nothing: its warps return at once.
// SQ: problems with square cells (pb.sq) take the square-cell form of the
// step (a branch per task, uniform over the warp), the others the general one.

template <class T, int K, int B, int PHYS, bool LIM = true, bool SQ = false>
__global__ void __launch_bounds__(256) batch_step2d_kernel(const StepArgs a, const BatchProblem* __restrict__ probs,
                                                           const int2* __restrict__ tasks, int n_tasks,
                                                           DevState* states, int* curs, unsigned* done,
                                                           const T* bufA, T* bufB) {
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= n_tasks) return;
    const int2 tk = tasks[gw];
    const BatchProblem pb = probs[tk.x];
    DevState* ds = states + tk.x;
    const int cur = curs[tk.x];
    ProbView<T> pv;
    T* A = const_cast<T*>(bufA) + pb.offset;
    T* Bb = bufB + pb.offset;
    pv.uin_ = cur ? Bb : A;
    pv.uout_ = cur ? A : Bb;
    pv.nx_ = pb.nx;
    pv.ny_ = pb.ny;
    pv.x0_ = pb.x0;
    pv.y0_ = pb.y0;
    pv.dx_ = pb.dx;
    pv.dy_ = pb.dy;
    pv.rx_ = pb.rx;
    pv.ry_ = pb.ry;
    pv.M_ = a.M;
    pv.bx_ = a.beta[0];
    pv.by_ = a.beta[1];
    pv.t_ = ds->t;
    pv.dt_ = ds->dt;
    pv.n_strips_ = pb.n_strips;
    pv.n_segs_ = pb.n_segs;
    pv.seg_len_ = a.seg_len;
    pv.total_warps_ = pb.n_strips * pb.n_segs;
    pv.partials_ = a.partials + (size_t)pb.warp0 * Step2D<T, K, B, PHYS>::NRED;
    pv.ds_ = ds;
    pv.cur_ = curs + tk.x;
    pv.done_ = done;
    if constexpr (SQ) {
        if (pb.sq) {
            step2d_body<T, K, B, PHYS, false, false, LIM, false, true>(a, pv, tk.y);
            return;
        }
    }
    step2d_body<T, K, B, PHYS, false, false, LIM, false, false>(a, pv, tk.y);
}

}  // namespace crk
