// A reduction entry point that allocates nothing, for callers that cannot
// call cudaMalloc: code running inside a host framework that owns the device
// memory pool (and forbids raw allocations), or code that must not allocate
// while a CUDA graph is being captured or in a real-time loop where an
// allocation could stall.  The caller passes the state and an output buffer
// it already owns; the reduction's scratch lives in a file-scope device array
// of fixed size, so the call itself needs no device memory of its own.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/crkdg.h"
#include "aux_kernels.cuh"

namespace {

// Scratch of the reduction: the run-state block (arrival counter, results)
// and one slot of 8 doubles per warp.  The grid is capped at 128 blocks of
// 256 threads (1024 warps): larger meshes are covered by the kernel's
// grid-stride loop, so the array never needs to grow.
constexpr int kNoAllocBlocks = 128;
constexpr int kNoAllocWarps = kNoAllocBlocks * 8;
constexpr int kSlot = 8;
constexpr long long kMaxCells = 1LL << 30;

struct NoAllocScratch {
    crk::DevState ds;
    double partials[kNoAllocWarps * kSlot];
};

// about 64 KiB, held by every GPU that loads the library until the process exits
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of the array, looked up once per device.  In host code the
// symbol name is only a host-side stand-in; the address must come from
// cudaGetSymbolAddress with that device current.
constexpr int kMaxDevices = 64;
NoAllocScratch* g_addr[kMaxDevices] = {nullptr};
std::mutex g_mtx;
thread_local std::string g_msg;

int fail(int code, const std::string& m) {
    g_msg = m;
    return code;
}

__global__ void copy_results(const crk::DevState* ds, int nv, double* out) {
    if (threadIdx.x == 0) {
        out[0] = ds->maxspeed;
        for (int v = 0; v < nv; ++v) out[1 + v] = ds->sums[v];
    }
}

}  // namespace

extern "C" const char* crkdg_noalloc_last_error(void) { return g_msg.c_str(); }

extern "C" int crkdg_reduce_state_noalloc(const void* u_dev, int dim, int nx, int ny, int n_modes, int physics,
                                          int precision, double dx, double dy, double gamma, const double* beta,
                                          double* out_dev, void* stream) {
    if (!u_dev || !out_dev) return fail(CRKDG_EINVAL, "null state or output pointer");
    if (dim != 1 && dim != 2) return fail(CRKDG_EINVAL, "dim must be 1 or 2");
    if (dim == 1) ny = 1;
    if (nx < 1 || ny < 1 || n_modes < 1) return fail(CRKDG_EINVAL, "mesh and modes must be positive");
    if ((long long)nx * ny > kMaxCells)
        return fail(CRKDG_EINVAL, "mesh exceeds the 2^30-cell maximum of crkdg_reduce_state_noalloc");
    if (physics != CRKDG_ADVECTION && physics != CRKDG_EULER) return fail(CRKDG_EINVAL, "unknown physics");
    if (precision != CRKDG_F32 && precision != CRKDG_F64) return fail(CRKDG_EINVAL, "unknown precision");
    if (!(dx > 0.0) || !(dy > 0.0)) return fail(CRKDG_EINVAL, "dx and dy must be positive");
    if (physics == CRKDG_ADVECTION && !beta) return fail(CRKDG_EINVAL, "advection needs beta");
    if (physics == CRKDG_EULER && !(gamma > 1.0)) return fail(CRKDG_EINVAL, "gamma must exceed 1");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(CRKDG_ECUDA, "no usable current device");
    NoAllocScratch* s = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mtx);
        if (!g_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fail(CRKDG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[dev] = static_cast<NoAllocScratch*>(p);
        }
        s = g_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: the counter and results
    // must start at zero
    cudaError_t e = cudaMemsetAsync(&s->ds, 0, sizeof(crk::DevState), st);
    if (e != cudaSuccess) return fail(CRKDG_ECUDA, std::string("clearing scratch: ") + cudaGetErrorString(e));
    const double bx = beta ? beta[0] : 0.0, by = beta && dim == 2 ? beta[1] : 0.0;
    const int kphys = physics == CRKDG_ADVECTION ? crk::PHYS_ADV : (dim == 1 ? crk::PHYS_EULER1D : crk::PHYS_EULER);
    int nv = 1;
#define CRK_NA(T, P, NV)                                                                                     \
    crk::reduce_state_kernel<T, P, NV><<<kNoAllocBlocks, 256, 0, st>>>(static_cast<const T*>(u_dev), nx, ny,  \
                                                                      n_modes, dx, dy, gamma, bx, by, &s->ds, \
                                                                      s->partials, 0);                       \
    nv = NV;
    if (kphys == crk::PHYS_ADV) {
        if (precision == CRKDG_F32) { CRK_NA(float, crk::PHYS_ADV, 1) } else { CRK_NA(double, crk::PHYS_ADV, 1) }
    } else if (kphys == crk::PHYS_EULER1D) {
        if (precision == CRKDG_F32) { CRK_NA(float, crk::PHYS_EULER1D, 3) } else { CRK_NA(double, crk::PHYS_EULER1D, 3) }
    } else {
        if (precision == CRKDG_F32) { CRK_NA(float, crk::PHYS_EULER, 4) } else { CRK_NA(double, crk::PHYS_EULER, 4) }
    }
#undef CRK_NA
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CRKDG_ECUDA, std::string("reduction launch: ") + cudaGetErrorString(e));
    copy_results<<<1, 32, 0, st>>>(&s->ds, nv, out_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CRKDG_ECUDA, std::string("result copy: ") + cudaGetErrorString(e));
    return CRKDG_OK;
}
