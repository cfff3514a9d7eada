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

// Device address of the array.  In host code the symbol name is only a
// host-side stand-in; the address must come from cudaGetSymbolAddress with
// that device current.  It is looked up again at every call made outside a
// stream capture (so a context that was reset and recreated gets its own
// array's address, not a stale one); a call made while its stream is being
// captured uses the address the last uncaptured call on that device found.
constexpr int kMaxDevices = 64;
NoAllocScratch* g_addr[kMaxDevices] = {nullptr};
std::mutex g_mtx;
thread_local std::string g_msg;

int fail(int code, const std::string& m) {
    g_msg = m;
    return code;
}

// results of the reduction and its status bits, which the next call's
// clearing would otherwise erase
__global__ void copy_results(const crk::DevState* ds, int nv, double* out) {
    if (threadIdx.x == 0) {
        out[0] = ds->maxspeed;
        for (int v = 0; v < nv; ++v) out[1 + v] = ds->sums[v];
        out[1 + nv] = double(ds->status);
    }
}

}  // namespace

extern "C" const char* crkdg_noalloc_last_error(void) { return g_msg.c_str(); }

extern "C" int crkdg_reduce_state_noalloc(const void* u_dev, int dim, int nx, int ny, int n_modes, int physics,
                                          int precision, double dx, double dy, double gamma, const double* beta,
                                          double* out_dev, void* stream) {
    if (!u_dev || !out_dev) return fail(CRKDG_EINVAL, "null state or output pointer");
    if (dim != 1 && dim != 2) return fail(CRKDG_EINVAL, "dim must be 1 or 2");
    // a 1D mesh is one row of cells of unit height (as crkdg_create makes it)
    if (dim == 1) {
        ny = 1;
        dy = 1.0;
    }
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
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();   // a query refused during another stream's capture: treat as capturing
        cap = cudaStreamCaptureStatusActive;
    }
    NoAllocScratch* s = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mtx);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fail(CRKDG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[dev] = static_cast<NoAllocScratch*>(p);
        } else if (!g_addr[dev]) {
            return fail(CRKDG_EINVAL, "the first call on a device must come before any stream capture");
        }
        s = g_addr[dev];
    }
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
