// 2D Euler FP32 with the learned troubled-cell indicator (P^2 and Q^2): the
// limiter pass that evaluates it (the default limit mode) and the step with
// it fused into the limit-on-load (CRKDG_LIMIT_FUSED).
#include <mutex>

#include "aux_kernels.cuh"
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

template <int B>
cudaError_t run_limit_mlp(const StepArgs& a, void* u, unsigned long long* flags, cudaStream_t st) {
    auto kern = limit2d_mlp_kernel<float, 2, B>;
    const size_t smem = sizeof(MlpSmem) + (size_t)(LIMIT_MLP_THREADS / 32) * (32 * MLP_INP + 64) * sizeof(__nv_bfloat16);
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int per_sm = 1;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (attr_err == cudaSuccess)
            attr_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LIMIT_MLP_THREADS, smem);
    });
    if (attr_err != cudaSuccess) return attr_err;
    // one wave of resident blocks; each loads the weights once and walks the mesh
    const int grid = std::max(1, per_sm) * std::max(1, sm_count());
    StepArgs b = a;
    set_derived(b);
    kern<<<grid, LIMIT_MLP_THREADS, smem, st>>>(b, static_cast<float*>(u), flags);
    return cudaGetLastError();
}

template <int B>
cudaError_t run_limit_mlp_tc(const StepArgs& a, void* u, unsigned long long* flags, cudaStream_t st) {
    auto kern = limit2d_mlp_tc_kernel<float, 2, B>;
    const size_t smem = sizeof(MlpTcSmem) + MLPTC_SMEM_SLACK;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int per_sm = 1;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (attr_err == cudaSuccess)
            attr_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, MLPTC_CELLS, smem);
    });
    if (attr_err != cudaSuccess) return attr_err;
    // resident blocks only (each holds its tensor-memory columns for its walk)
    const int blocks_sm = std::max(1, std::min(per_sm, 512 / MLPTC_TMEM_COLS));
    const int grid = blocks_sm * std::max(1, sm_count());
    StepArgs b = a;
    set_derived(b);
    kern<<<grid, MLPTC_CELLS, smem, st>>>(b, static_cast<float*>(u), flags);
    return cudaGetLastError();
}

}  // namespace

cudaError_t limit2d_euler_f32_mlp_tc(int k, int basis, const StepArgs& a, void* u, unsigned long long* flags,
                                     cudaStream_t st) {
    if (k != 2) return cudaErrorInvalidValue;
    return basis == 0 ? run_limit_mlp_tc<0>(a, u, flags, st) : run_limit_mlp_tc<1>(a, u, flags, st);
}

cudaError_t limit2d_euler_f32_mlp(int k, int basis, const StepArgs& a, void* u, unsigned long long* flags,
                                  cudaStream_t st) {
    if (k != 2) return cudaErrorInvalidValue;
    return basis == 0 ? run_limit_mlp<0>(a, u, flags, st) : run_limit_mlp<1>(a, u, flags, st);
}

cudaError_t step2d_euler_f32_mlp(int k, int basis, const StepArgs& a, int wpb, cudaStream_t st) {
    if (k != 2) return cudaErrorInvalidValue;
    return basis == 0 ? run_step_mlp<0>(a, wpb, st) : run_step_mlp<1>(a, wpb, st);
}

}  // namespace crk
