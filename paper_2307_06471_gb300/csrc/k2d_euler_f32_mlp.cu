// 2D Euler FP32 step with the learned troubled-cell indicator fused into the
// limit-on-load (P^2 and Q^2).
#include <mutex>

#include "launch.h"
#include "step2d.cuh"

namespace crk {
namespace {

template <int B>
cudaError_t run_step_mlp(const StepArgs& a, int wpb, cudaStream_t st) {
    auto kern = step2d_kernel<float, 2, B, PHYS_EULER, false, true>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int threads = wpb * 32;
    const size_t smem = mlp_smem_offset<float, 2, B, PHYS_EULER>(a.s, threads) + mlp_smem_bytes(threads);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    const int total = a.n_strips * a.n_segs;
    StepArgs b = a;
    set_derived(b);
    kern<<<(total + wpb - 1) / wpb, threads, smem, st>>>(b);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_finalize<4>(b, st);
}

}  // namespace

cudaError_t step2d_euler_f32_mlp(int k, int basis, const StepArgs& a, int wpb, cudaStream_t st) {
    if (k != 2) return cudaErrorInvalidValue;
    return basis == 0 ? run_step_mlp<0>(a, wpb, st) : run_step_mlp<1>(a, wpb, st);
}

}  // namespace crk
