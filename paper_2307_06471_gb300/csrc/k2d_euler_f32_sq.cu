// The FP32 2D Euler step for square cells (dx == dy) without a limit on
// load: step2d_kernel<..., SQ = true> for k = 2 (P^2 and Q^2), launched as
// the plain kernel is, with its one-block finalize.  Its own translation
// unit so that it compiles beside the others.
#include <mutex>

#include "launch.h"
#include "step2d.cuh"

namespace crk {
namespace {

template <int B>
cudaError_t run_step_sq(const StepArgs& a, int wpb, cudaStream_t st) {
    using C = Step2D<float, 2, B, PHYS_EULER>;
    auto kern = step2d_kernel<float, 2, B, PHYS_EULER, false, false, false, false, true>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int threads = wpb * 32;
    const size_t smem = (size_t)C::smem_per_thread(a.s) * sizeof(float) * threads;
    const int total = a.n_strips * a.n_segs;
    const int grid = (total + wpb - 1) / wpb;
    StepArgs b = a;
    set_derived(b);
    kern<<<grid, threads, smem, st>>>(b);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_finalize<C::NV>(b, st);
}

}  // namespace

cudaError_t step2d_euler_f32_sq(int basis, const StepArgs& a, int wpb, cudaStream_t st) {
    return basis == 0 ? run_step_sq<0>(a, wpb, st) : run_step_sq<1>(a, wpb, st);
}

}  // namespace crk
