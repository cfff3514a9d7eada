// The modal step for linear advection (step2d_linear.cuh), FP32 and FP64,
// for every (k, basis), and its launcher.
#include <mutex>

#include "launch.h"
#include "step2d_linear.cuh"

namespace crk {
namespace {

template <class T, int K, int B>
cudaError_t run_linear(const StepArgs& a, int wpb, cudaStream_t st) {
    auto kern = step2d_linear_kernel<T, K, B>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int threads = wpb * 32;
    const size_t smem = (size_t)linear_smem_per_thread<T, K, B>(a.s) * sizeof(T) * threads;
    const int grid = (a.n_strips * a.n_segs + wpb - 1) / wpb;
    StepArgs b = a;
    set_derived(b);
    kern<<<grid, threads, smem, st>>>(b);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_finalize<1>(b, st);
}

template <class T, int K, int B>
cudaError_t info_linear(int s, KernelInfo* info) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step2d_linear_kernel<T, K, B>);
    if (e != cudaSuccess) return e;
    info->regs = fa.numRegs;
    info->max_threads = fa.maxThreadsPerBlock;
    info->smem_per_thread = linear_smem_per_thread<T, K, B>(s) * (int)sizeof(T);
    return cudaSuccess;
}

template <class T>
cudaError_t linear_switch(int k, int basis, const StepArgs* a, int wpb, cudaStream_t st, int s, KernelInfo* info) {
    switch (k * 2 + (k == 0 ? 0 : basis)) {
        case 0: return a ? run_linear<T, 0, 0>(*a, wpb, st) : info_linear<T, 0, 0>(s, info);
        case 2: return a ? run_linear<T, 1, 0>(*a, wpb, st) : info_linear<T, 1, 0>(s, info);
        case 3: return a ? run_linear<T, 1, 1>(*a, wpb, st) : info_linear<T, 1, 1>(s, info);
        case 4: return a ? run_linear<T, 2, 0>(*a, wpb, st) : info_linear<T, 2, 0>(s, info);
        case 5: return a ? run_linear<T, 2, 1>(*a, wpb, st) : info_linear<T, 2, 1>(s, info);
        case 6: return a ? run_linear<T, 3, 0>(*a, wpb, st) : info_linear<T, 3, 0>(s, info);
        case 7: return a ? run_linear<T, 3, 1>(*a, wpb, st) : info_linear<T, 3, 1>(s, info);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_step2d_linear(int prec, int k, int basis, const StepArgs& a, int wpb, cudaStream_t st) {
    return prec == 1 ? linear_switch<double>(k, basis, &a, wpb, st, a.s, nullptr)
                     : linear_switch<float>(k, basis, &a, wpb, st, a.s, nullptr);
}

cudaError_t info_step2d_linear(int prec, int k, int basis, int s, KernelInfo* info) {
    return prec == 1 ? linear_switch<double>(k, basis, nullptr, 0, nullptr, s, info)
                     : linear_switch<float>(k, basis, nullptr, 0, nullptr, s, info);
}

}  // namespace crk
