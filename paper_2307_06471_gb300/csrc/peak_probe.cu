// Measured arithmetic peaks of the GPU the library runs on.  The fused step
// is bound by FP32 fused multiply-add issue, not by HBM, so its roofline
// fraction needs an FP32 peak; the FP64 peak bounds the FP64 path.  Each
// probe is a grid of independent FMA chains (enough chains per thread and
// warps per SM to cover the pipe latency), timed by CUDA events on the
// caller's stream.  No counterpart in the paper: a measuring instrument.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/crkdg.h"
#include "launch.h"

namespace {

thread_local std::string g_msg;

int fail(int code, const std::string& m) {
    g_msg = m;
    return code;
}

constexpr int kChains = 8;          // independent chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;     // 64 warps per SM

// x <- x * b + c on kChains independent chains, iters times.  b slightly
// below 1 and c small keep the values bounded; the conditional store keeps
// the chains alive without writing in practice.
__global__ void __launch_bounds__(kThreads) probe_f32(float b, float c, int iters, float* sink) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0f + 1e-3f * i + 1e-7f * threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll 8
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.0f) sink[blockIdx.x] = s;
}

// the packed form: one instruction does two FP32 FMAs per lane
__global__ void __launch_bounds__(kThreads) probe_f32x2(float b, float c, int iters, float* sink) {
    float2 x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = make_float2(1.0f + 1e-3f * i, 1.0f - 1e-3f * i + 1e-7f * threadIdx.x);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll 8
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], bb, cc);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
    if (s == -1.0f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) probe_f64(double b, double c, int iters, float* sink) {
    double x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0 + 1e-3 * i + 1e-7 * threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll 8
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.0) sink[blockIdx.x] = (float)s;
}

}  // namespace

extern "C" const char* crkdg_probe_last_error(void) { return g_msg.c_str(); }

extern "C" int crkdg_alu_peak(int kind, int reps, void* stream, double* tflops, double* ms_per_launch,
                              int* n_sms) {
    if (!tflops || reps < 1) return fail(CRKDG_EINVAL, "null output or reps < 1");
    if (kind < CRKDG_PEAK_F32 || kind > CRKDG_PEAK_F64) return fail(CRKDG_EINVAL, "unknown probe kind");
    const int sms = crk::sm_count();
    if (sms < 1) return fail(CRKDG_ECUDA, "cannot query the SM count");
    const int blocks = sms * kBlocksPerSM;
    // about 0.3-1 ms per launch: 2048 x 8 x 8 FP32 FMAs per thread, 1/16 of that in FP64
    const int iters = kind == CRKDG_PEAK_F64 ? 128 : 2048;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* sink = nullptr;
    if (cudaMalloc(&sink, blocks * sizeof(float)) != cudaSuccess) return fail(CRKDG_ENOMEM, "cudaMalloc failed");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&]() {
        if (kind == CRKDG_PEAK_F32) probe_f32<<<blocks, kThreads, 0, st>>>(0.9999999f, 1e-7f, iters, sink);
        else if (kind == CRKDG_PEAK_F32X2) probe_f32x2<<<blocks, kThreads, 0, st>>>(0.9999999f, 1e-7f, iters, sink);
        else probe_f64<<<blocks, kThreads, 0, st>>>(0.9999999999, 1e-12, iters, sink);
    };
    launch();   // warm-up (clocks, instruction cache)
    std::vector<float> t(reps);
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t[r], e0, e1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return fail(CRKDG_ECUDA, std::string("probe: ") + cudaGetErrorString(e));
    std::sort(t.begin(), t.end());
    const double med = t[reps / 2];
    const double fma_per_thread = (double)iters * 8 * kChains * (kind == CRKDG_PEAK_F32X2 ? 2 : 1);
    *tflops = 2.0 * fma_per_thread * (double)blocks * kThreads / (med * 1e-3) / 1e12;
    if (ms_per_launch) *ms_per_launch = med;
    if (n_sms) *n_sms = sms;
    return CRKDG_OK;
}
