// 2D Euler step with the compensated FP32 state and deviation-form fluxes
// (step2d.cuh, DEV); the projection and reduction of its hi + lo planes are
// those of the compensated state (k2d_euler_f32c.cu).
#include <mutex>

#include "launch.h"
#include "step2d.cuh"

namespace crk {
namespace {

template <int K, int B, bool SQ>
cudaError_t run_step_dt(const StepArgs& a, int wpb, cudaStream_t st) {
    using C = Step2D<float, K, B, PHYS_EULER>;
    auto kern = step2d_kernel<float, K, B, PHYS_EULER, true, false, false, true, SQ>;
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

// square cells (dx == dy) take the square-cell form for k = 2
template <int K, int B>
cudaError_t run_step_d(const StepArgs& a, int wpb, cudaStream_t st) {
#ifndef CRK_SQ_STEP_OFF
    if constexpr (K == 2)
        if (a.dx == a.dy) return run_step_dt<K, B, true>(a, wpb, st);
#endif
    return run_step_dt<K, B, false>(a, wpb, st);
}

template <int K, int B>
cudaError_t run_info_d(int s, KernelInfo* info) {
    using C = Step2D<float, K, B, PHYS_EULER>;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step2d_kernel<float, K, B, PHYS_EULER, true, false, false, true>);
    if (e != cudaSuccess) return e;
    info->regs = fa.numRegs;
    info->max_threads = fa.maxThreadsPerBlock;
    info->smem_per_thread = C::smem_per_thread(s) * (int)sizeof(float);
    return cudaSuccess;
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

cudaError_t step2d_euler_f32d(int k, int basis, const StepArgs& a, int wpb, cudaStream_t st) {
    CRK_SWITCH(run_step_d, a, wpb, st)
}
cudaError_t info2d_euler_f32d(int k, int basis, int s, KernelInfo* info) { CRK_SWITCH(run_info_d, s, info) }

}  // namespace crk
