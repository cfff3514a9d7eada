// Internal launcher interface between the C ABI (api.cu) and the kernel
// translation units (one per physics x precision, compiled in parallel).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace crk {

// Streaming multiprocessors of the current device (queried once per device
// ordinal; 0 if the query fails).
inline int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev] = n;
    }
    return cache[dev];
}

struct KernelInfo {
    int regs;              // registers per thread of the step kernel
    int max_threads;       // max threads per block it can launch with
    int smem_per_thread;   // bytes of private shared memory per thread (for a.s stages)
};

// 2D fused step (step2d.cuh); wpb = warps per block
cudaError_t launch_step2d(int phys, int prec, int k, int basis, const StepArgs& a, int wpb, cudaStream_t st);
cudaError_t info_step2d(int phys, int prec, int k, int basis, int s, KernelInfo* info);
// standalone TVB limiter (in place)
cudaError_t launch_limit2d(int phys, int prec, int k, int basis, const StepArgs& a, void* u,
                           unsigned long long* flags, cudaStream_t st);
// projection of point values (device FP64 [cell][q][v])
cudaError_t launch_project(int dim, int phys, int prec, int k, int basis, const double* vals, void* u, int ncell,
                           cudaStream_t st);
// 1D fused step; n_steps > 1 requires one block
cudaError_t launch_step1d(int phys, int prec, int k, const StepArgs& a, int n_steps, int threads, int blocks,
                          cudaStream_t st);
cudaError_t info_step1d(int phys, int prec, int k, int s, KernelInfo* info);
// FP64 reduction of the averages into DevState (set_dt: also dt = cfl/max)
cudaError_t launch_reduce(int dim, int phys, int prec, const void* u, int nx, int ny, int nm, double dx, double dy,
                          double gamma, double bx, double by, DevState* ds, double* partials, int blocks, int set_dt,
                          cudaStream_t st);

// per-(phys, prec) entry points defined in the kernel translation units
#define CRK_DECL_2D(NAME)                                                                                  \
    cudaError_t step2d_##NAME(int k, int basis, const StepArgs& a, int wpb, cudaStream_t st);            \
    cudaError_t info2d_##NAME(int k, int basis, int s, KernelInfo* info);                                \
    cudaError_t limit2d_##NAME(int k, int basis, const StepArgs& a, void* u, unsigned long long* flags,  \
                               cudaStream_t st);                                                         \
    cudaError_t project2d_##NAME(int k, int basis, const double* vals, void* u, int ncell, cudaStream_t st);
// compensated FP32 state (hi + lo planes), 2D Euler only
cudaError_t step2d_euler_f32c(int k, int basis, const StepArgs& a, int wpb, cudaStream_t st);
cudaError_t info2d_euler_f32c(int k, int basis, int s, KernelInfo* info);
cudaError_t project2d_euler_f32c(int k, int basis, const double* vals, void* u, int ncell, cudaStream_t st);
cudaError_t reduce_euler_f32c(const void* u, int nx, int ny, int nm, double dx, double dy, double gamma, DevState* ds,
                              double* partials, int blocks, int set_dt, cudaStream_t st);

// compensated FP32 state with deviation-form fluxes (same planes as f32c)
cudaError_t step2d_euler_f32d(int k, int basis, const StepArgs& a, int wpb, cudaStream_t st);
cudaError_t info2d_euler_f32d(int k, int basis, int s, KernelInfo* info);

// FP32 2D Euler k = 2 step with the fused learned indicator, and the
// limiter pass that evaluates the indicator
cudaError_t step2d_euler_f32_mlp(int k, int basis, const StepArgs& a, int wpb, cudaStream_t st);
// 2D Euler, k = 2, square cells (dx == dy), no limit on load, FP32 / FP64
cudaError_t step2d_sq_euler_f32(int basis, const StepArgs& a, int wpb, cudaStream_t st);
cudaError_t step2d_sq_euler_f64(int basis, const StepArgs& a, int wpb, cudaStream_t st);
cudaError_t limit2d_euler_f32_mlp(int k, int basis, const StepArgs& a, void* u, unsigned long long* flags,
                                  cudaStream_t st);
// the pass with the network on the tcgen05 tensor cores
cudaError_t limit2d_euler_f32_mlp_tc(int k, int basis, const StepArgs& a, void* u, unsigned long long* flags,
                                     cudaStream_t st);

// out = alpha x + beta y (n elements of the state precision), and DevState.t = t
cudaError_t launch_axpby(int prec, void* out, const void* x, const void* y, double alpha, double beta, size_t n,
                         cudaStream_t st);
cudaError_t launch_set_time(DevState* ds, double t, cudaStream_t st);
// the modal step for linear advection (step2d_linear.cuh); prec 0 FP32, 1 FP64
cudaError_t launch_step2d_linear(int prec, int k, int basis, const StepArgs& a, int wpb, cudaStream_t st);
cudaError_t info_step2d_linear(int prec, int k, int basis, int s, KernelInfo* info);
// FP64 staging <-> FP32 state of n elements: one plane set (comp = 0) or the
// compensated hi + lo plane sets (comp = 1, lo at offset n)
cudaError_t launch_f64_to_f32(const double* in, float* out, size_t n, int comp, cudaStream_t st);
cudaError_t launch_f32_to_f64(const float* in, double* out, size_t n, int comp, cudaStream_t st);

struct BatchProblem;
#define CRK_DECL_B(NAME)                                                                                     \
    cudaError_t batch2d_##NAME(int k, int basis, const StepArgs& a, const BatchProblem* probs, const int2* tasks, \
                               int n_tasks, DevState* states, int* curs, unsigned* done, const void* bufA,    \
                               void* bufB, int wpb, cudaStream_t st);                                         \
    cudaError_t binfo2d_##NAME(int k, int basis, int s, KernelInfo* info);                                 \
    cudaError_t blimit2d_##NAME(int k, int basis, const StepArgs& a, const BatchProblem* probs, const int4* rows, \
                                int n_rows, DevState* states, const int* curs, void* bufA, void* bufB,        \
                                cudaStream_t st);
CRK_DECL_B(euler_f32)
CRK_DECL_B(euler_f64)
#undef CRK_DECL_B

CRK_DECL_2D(euler_f32)
CRK_DECL_2D(euler_f64)
CRK_DECL_2D(adv_f32)
CRK_DECL_2D(adv_f64)
#undef CRK_DECL_2D

}  // namespace crk
