// 2D Euler step, projection and reduction with the compensated FP32 state
// (hi + lo planes; see step2d.cuh).
#include <mutex>

#include "aux_kernels.cuh"
#include "launch.h"
#include "step2d.cuh"

namespace crk {
namespace {

template <int K, int B>
cudaError_t run_step_c(const StepArgs& a, int wpb, cudaStream_t st) {
    using C = Step2D<float, K, B, PHYS_EULER>;
    auto kern = step2d_kernel<float, K, B, PHYS_EULER, true, false, false>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int threads = wpb * 32;
    const size_t smem = (size_t)C::smem_per_thread(a.s) * sizeof(float) * threads;
    const int total = a.n_strips * a.n_segs;
    StepArgs b = a;
    set_derived(b);
    kern<<<(total + wpb - 1) / wpb, threads, smem, st>>>(b);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_finalize<4>(b, st);
}

template <int K, int B>
cudaError_t run_info_c(int s, KernelInfo* info) {
    using C = Step2D<float, K, B, PHYS_EULER>;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step2d_kernel<float, K, B, PHYS_EULER, true, false, false>);
    if (e != cudaSuccess) return e;
    info->regs = fa.numRegs;
    info->max_threads = fa.maxThreadsPerBlock;
    info->smem_per_thread = C::smem_per_thread(s) * (int)sizeof(float);
    return cudaSuccess;
}

template <int K, int B>
cudaError_t run_project_c(const double* vals, void* u, int ncell, cudaStream_t st) {
    project2d_kernel<float, K, B, 4, true><<<(ncell + 127) / 128, 128, 0, st>>>(vals, static_cast<float*>(u), ncell);
    return cudaGetLastError();
}

}  // namespace

#define CRK_SWITCH(FN, ...)                                      \
    switch (k * 2 + (k == 0 ? 0 : basis)) {                       \
        case 0: return FN<0, 0>(__VA_ARGS__);                     \
        case 2: return FN<1, 0>(__VA_ARGS__);                     \
        case 3: return FN<1, 1>(__VA_ARGS__);                     \
        case 4: return FN<2, 0>(__VA_ARGS__);                     \
        case 5: return FN<2, 1>(__VA_ARGS__);                     \
        case 6: return FN<3, 0>(__VA_ARGS__);                     \
        case 7: return FN<3, 1>(__VA_ARGS__);                     \
        default: return cudaErrorInvalidValue;                    \
    }

cudaError_t step2d_euler_f32c(int k, int basis, const StepArgs& a, int wpb, cudaStream_t st) {
    CRK_SWITCH(run_step_c, a, wpb, st)
}
cudaError_t info2d_euler_f32c(int k, int basis, int s, KernelInfo* info) { CRK_SWITCH(run_info_c, s, info) }
cudaError_t project2d_euler_f32c(int k, int basis, const double* vals, void* u, int ncell, cudaStream_t st) {
    CRK_SWITCH(run_project_c, vals, u, ncell, st)
}
cudaError_t reduce_euler_f32c(const void* u, int nx, int ny, int nm, double dx, double dy, double gamma, DevState* ds,
                              double* partials, int blocks, int set_dt, cudaStream_t st) {
    reduce_state_kernel<float, PHYS_EULER, 4, true><<<blocks, 256, 0, st>>>(
        static_cast<const float*>(u), nx, ny, nm, dx, dy, gamma, 0.0, 0.0, ds, partials, set_dt);
    return cudaGetLastError();
}

}  // namespace crk
