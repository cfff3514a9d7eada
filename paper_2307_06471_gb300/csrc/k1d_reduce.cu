// 1D step kernels, projections and FP64 reductions for every physics and
// precision, plus the dispatchers of launch.h.
#include <mutex>

#include "aux_kernels.cuh"
#include "launch.h"
#include "step1d.cuh"

namespace crk {
namespace {

template <class T, int K, int PHYS>
cudaError_t run_step1d(const StepArgs& a, int n_steps, int threads, int blocks, cudaStream_t st) {
    constexpr int NDOF = Phys<T, PHYS>::NV * (K + 1);
    auto kern = step1d_kernel<T, K, PHYS>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const size_t smem = (size_t)(a.s > 1 ? a.s - 1 : 1) * NDOF * sizeof(T) * threads;
    StepArgs b = a;
    set_derived(b);
    kern<<<blocks, threads, smem, st>>>(b, n_steps);
    return cudaGetLastError();
}

template <class T, int K, int PHYS>
cudaError_t run_info1d(int s, KernelInfo* info) {
    constexpr int NDOF = Phys<T, PHYS>::NV * (K + 1);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, step1d_kernel<T, K, PHYS>);
    if (e != cudaSuccess) return e;
    info->regs = fa.numRegs;
    info->max_threads = fa.maxThreadsPerBlock;
    info->smem_per_thread = (s > 1 ? s - 1 : 1) * NDOF * (int)sizeof(T);
    return cudaSuccess;
}

template <class T, int PHYS>
cudaError_t step1d_k(int k, const StepArgs& a, int n, int th, int bl, cudaStream_t st) {
    switch (k) {
        case 0: return run_step1d<T, 0, PHYS>(a, n, th, bl, st);
        case 1: return run_step1d<T, 1, PHYS>(a, n, th, bl, st);
        case 2: return run_step1d<T, 2, PHYS>(a, n, th, bl, st);
        case 3: return run_step1d<T, 3, PHYS>(a, n, th, bl, st);
        default: return cudaErrorInvalidValue;
    }
}

template <class T, int PHYS>
cudaError_t info1d_k(int k, int s, KernelInfo* info) {
    switch (k) {
        case 0: return run_info1d<T, 0, PHYS>(s, info);
        case 1: return run_info1d<T, 1, PHYS>(s, info);
        case 2: return run_info1d<T, 2, PHYS>(s, info);
        case 3: return run_info1d<T, 3, PHYS>(s, info);
        default: return cudaErrorInvalidValue;
    }
}

template <class T, int NV>
cudaError_t project1d_k(int k, const double* vals, void* u, int ncell, cudaStream_t st) {
    const int g = (ncell + 127) / 128;
    T* o = static_cast<T*>(u);
    switch (k) {
        case 0: project1d_kernel<T, 0, NV><<<g, 128, 0, st>>>(vals, o, ncell); break;
        case 1: project1d_kernel<T, 1, NV><<<g, 128, 0, st>>>(vals, o, ncell); break;
        case 2: project1d_kernel<T, 2, NV><<<g, 128, 0, st>>>(vals, o, ncell); break;
        case 3: project1d_kernel<T, 3, NV><<<g, 128, 0, st>>>(vals, o, ncell); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class T, int PHYS, int NV>
cudaError_t reduce_t(const void* u, int nx, int ny, int nm, double dx, double dy, double gamma, double bx,
                     double by, DevState* ds, double* partials, int blocks, int set_dt, cudaStream_t st) {
    reduce_state_kernel<T, PHYS, NV><<<blocks, 256, 0, st>>>(static_cast<const T*>(u), nx, ny, nm, dx, dy, gamma,
                                                              bx, by, ds, partials, set_dt);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step1d(int phys, int prec, int k, const StepArgs& a, int n_steps, int threads, int blocks,
                          cudaStream_t st) {
    if (phys == PHYS_ADV)
        return prec == 0 ? step1d_k<float, PHYS_ADV>(k, a, n_steps, threads, blocks, st)
                         : step1d_k<double, PHYS_ADV>(k, a, n_steps, threads, blocks, st);
    return prec == 0 ? step1d_k<float, PHYS_EULER1D>(k, a, n_steps, threads, blocks, st)
                     : step1d_k<double, PHYS_EULER1D>(k, a, n_steps, threads, blocks, st);
}

cudaError_t info_step1d(int phys, int prec, int k, int s, KernelInfo* info) {
    if (phys == PHYS_ADV)
        return prec == 0 ? info1d_k<float, PHYS_ADV>(k, s, info) : info1d_k<double, PHYS_ADV>(k, s, info);
    return prec == 0 ? info1d_k<float, PHYS_EULER1D>(k, s, info) : info1d_k<double, PHYS_EULER1D>(k, s, info);
}

cudaError_t launch_reduce(int dim, int phys, int prec, const void* u, int nx, int ny, int nm, double dx, double dy,
                          double gamma, double bx, double by, DevState* ds, double* partials, int blocks, int set_dt,
                          cudaStream_t st) {
    if (prec == 2 || prec == 3) return reduce_euler_f32c(u, nx, ny, nm, dx, dy, gamma, ds, partials, blocks, set_dt, st);
#define CRK_R(T, P, NV) reduce_t<T, P, NV>(u, nx, ny, nm, dx, dy, gamma, bx, by, ds, partials, blocks, set_dt, st)
    if (phys == PHYS_ADV) return prec == 0 ? CRK_R(float, PHYS_ADV, 1) : CRK_R(double, PHYS_ADV, 1);
    if (dim == 1) return prec == 0 ? CRK_R(float, PHYS_EULER1D, 3) : CRK_R(double, PHYS_EULER1D, 3);
    return prec == 0 ? CRK_R(float, PHYS_EULER, 4) : CRK_R(double, PHYS_EULER, 4);
#undef CRK_R
}

cudaError_t launch_project(int dim, int phys, int prec, int k, int basis, const double* vals, void* u, int ncell,
                           cudaStream_t st) {
    if (dim == 1) {
        if (phys == PHYS_ADV)
            return prec == 0 ? project1d_k<float, 1>(k, vals, u, ncell, st) : project1d_k<double, 1>(k, vals, u, ncell, st);
        return prec == 0 ? project1d_k<float, 3>(k, vals, u, ncell, st) : project1d_k<double, 3>(k, vals, u, ncell, st);
    }
    if (prec == 2 || prec == 3) return project2d_euler_f32c(k, basis, vals, u, ncell, st);
    if (phys == PHYS_EULER)
        return prec == 0 ? project2d_euler_f32(k, basis, vals, u, ncell, st)
                         : project2d_euler_f64(k, basis, vals, u, ncell, st);
    return prec == 0 ? project2d_adv_f32(k, basis, vals, u, ncell, st) : project2d_adv_f64(k, basis, vals, u, ncell, st);
}

cudaError_t launch_axpby(int prec, void* out, const void* x, const void* y, double alpha, double beta, size_t n,
                         cudaStream_t st) {
    const int blocks = 4 * std::max(1, sm_count());
    if (prec == 1)
        axpby_kernel<double><<<blocks, 256, 0, st>>>(static_cast<double*>(out), static_cast<const double*>(x),
                                                     static_cast<const double*>(y), alpha, beta, n);
    else
        axpby_kernel<float><<<blocks, 256, 0, st>>>(static_cast<float*>(out), static_cast<const float*>(x),
                                                    static_cast<const float*>(y), alpha, beta, n);
    return cudaGetLastError();
}

namespace {
__global__ void set_time_kernel(DevState* ds, double t) { ds->t = t; }

// round to nearest; comp: lo = the rounding remainder, also rounded
__global__ void f64_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, size_t n, int comp) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double x = in[i];
        const float hi = __double2float_rn(x);
        out[i] = hi;
        if (comp) out[n + i] = __double2float_rn(x - (double)hi);
    }
}

__global__ void f32_to_f64_kernel(const float* __restrict__ in, double* __restrict__ out, size_t n, int comp) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = comp ? (double)in[i] + (double)in[n + i] : (double)in[i];
}
}  // namespace

cudaError_t launch_f64_to_f32(const double* in, float* out, size_t n, int comp, cudaStream_t st) {
    f64_to_f32_kernel<<<8 * std::max(1, sm_count()), 256, 0, st>>>(in, out, n, comp);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* in, double* out, size_t n, int comp, cudaStream_t st) {
    f32_to_f64_kernel<<<8 * std::max(1, sm_count()), 256, 0, st>>>(in, out, n, comp);
    return cudaGetLastError();
}

cudaError_t launch_set_time(DevState* ds, double t, cudaStream_t st) {
    set_time_kernel<<<1, 1, 0, st>>>(ds, t);
    return cudaGetLastError();
}

cudaError_t launch_step2d(int phys, int prec, int k, int basis, const StepArgs& a, int wpb, cudaStream_t st) {
    if (prec == 2) return step2d_euler_f32c(k, basis, a, wpb, st);
    if (prec == 3) return step2d_euler_f32d(k, basis, a, wpb, st);
    if (phys == PHYS_EULER)
        return prec == 0 ? step2d_euler_f32(k, basis, a, wpb, st) : step2d_euler_f64(k, basis, a, wpb, st);
    return prec == 0 ? step2d_adv_f32(k, basis, a, wpb, st) : step2d_adv_f64(k, basis, a, wpb, st);
}

cudaError_t info_step2d(int phys, int prec, int k, int basis, int s, KernelInfo* info) {
    if (prec == 2) return info2d_euler_f32c(k, basis, s, info);
    if (prec == 3) return info2d_euler_f32d(k, basis, s, info);
    if (phys == PHYS_EULER)
        return prec == 0 ? info2d_euler_f32(k, basis, s, info) : info2d_euler_f64(k, basis, s, info);
    return prec == 0 ? info2d_adv_f32(k, basis, s, info) : info2d_adv_f64(k, basis, s, info);
}

cudaError_t launch_limit2d(int phys, int prec, int k, int basis, const StepArgs& a, void* u,
                           unsigned long long* flags, cudaStream_t st) {
    if (phys == PHYS_EULER)
        return prec == 0 ? limit2d_euler_f32(k, basis, a, u, flags, st) : limit2d_euler_f64(k, basis, a, u, flags, st);
    return prec == 0 ? limit2d_adv_f32(k, basis, a, u, flags, st) : limit2d_adv_f64(k, basis, a, u, flags, st);
}

}  // namespace crk
