// Learned troubled-cell indicator on the fifth-generation tensor cores
// (tcgen05): the 40 -> 64 -> 64 -> 64 -> 1 ReLU network for a tile of
// MLPTC_CELLS = 512 cells per CTA of 512 threads (one cell per thread).
// Each layer is MLPTC_NT = 4 products of M = 128 rows on the tensor core --
// [128 x K] activations (BF16, shared memory) times the layer's [N x K]
// weights (BF16, shared memory), FP32 accumulators in tensor memory
// (columns 64 j .. 64 j + 63 for the tile's cells 128 j .. 128 j + 127) --
// issued by one thread and committed to one barrier; every thread then
// reads its cell's row of the accumulator (tcgen05.ld), applies ReLU while
// rounding it to BF16 (one cvt.relu per pair) and writes the row back to
// shared memory as the next layer's A operand.  The biases ride in the
// products: every A operand carries a column of ones (column 40 of the
// input layer's K = 48, column 64 of the hidden layers' K = 80) against a
// weight column holding the bias (in BF16).  Four products per round trip
// through the barrier: measured 2.43 ms per 2048^2 shock-vortex step with
// one (128 cells), 1.64 with two, 1.46 with four.
//
// Shared-memory operands use the tensor core's K-major layout without
// swizzling: 8 x 8 BF16 core matrices of 128 contiguous bytes (8 rows of 16
// bytes), core matrix (row group r, column group c) of a [rows x K] operand
// at byte (r * K/8 + c) * 128.  Descriptor: leading byte offset (between
// core matrices along K) 128, stride byte offset (between row groups)
// K/8 * 128.
//
// Every wait on the tensor core's completion barrier is bounded; a wait
// that runs out sets a status flag, no further product is issued, the
// tensor memory is freed and the logits are NaN.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include "mlp_warp.cuh"

namespace crk {

constexpr int MLPTC_M = 128;      // rows of one product (its M)
constexpr int MLPTC_NT = 4;       // products per layer
constexpr int MLPTC_CELLS = MLPTC_M * MLPTC_NT;   // cells per tile = threads per CTA
// tensor-memory columns per CTA: the layers' accumulators (64 columns per
// product; 16 for the output layer): 256, two CTAs of an SM hold theirs
constexpr int MLPTC_TMEM_COLS = 64 * MLPTC_NT;
// dynamic shared memory of a CTA beyond the operands
constexpr size_t MLPTC_SMEM_SLACK = 0;
constexpr unsigned MLPTC_WAIT_LIMIT = 1u << 22;
// tensor-memory loads (16 columns each) in flight per wait in the epilogue:
// 1, 2 or 4 (tuning knob)
#ifndef MLPTC_LD
#define MLPTC_LD 2
#endif
static_assert(MLPTC_LD == 1 || MLPTC_LD == 2 || MLPTC_LD == 4, "MLPTC_LD divides 4");
// K of the hidden and output layers' products: 64 activations, a column of
// ones (the bias) and 15 zero columns
constexpr int MLPTC_KH = MLP_H + 16;

struct __align__(128) MlpTcSmem {
    __nv_bfloat16 act1[MLPTC_CELLS * MLP_INP];   // input layer's A: 40 features, 1, zeros (K = 48)
    __nv_bfloat16 acth[MLPTC_CELLS * MLPTC_KH];  // hidden layers' A: 64 activations, 1, zeros (K = 80)
    __nv_bfloat16 W1[MLP_H * MLP_INP];           // B operands: N x K, the bias in the ones column
    __nv_bfloat16 W2[MLP_H * MLPTC_KH];
    __nv_bfloat16 W3[MLP_H * MLPTC_KH];
    __nv_bfloat16 W4[16 * MLPTC_KH];             // output row 0, rows 1..15 zero
    unsigned tmem;                               // tensor-memory address from tcgen05.alloc
    unsigned long long bar;                      // completion barrier of the products
};

// element index of (row, k) in a [rows x K] operand of the core-matrix layout
__host__ __device__ constexpr int tc_idx(int row, int k, int K) {
    return ((row >> 3) * (K >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

// two FP32 values rounded to BF16 (round to nearest even), packed: x0 in the
// low half
__device__ __forceinline__ uint32_t bf16x2_bits(float x0, float x1) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(x0, x1);
    uint32_t u;
    memcpy(&u, &b, sizeof u);
    return u;
}
// ReLU of two FP32 values rounded to BF16 (max(x, 0), round to nearest
// even) in one conversion, packed: x0 in the low half
__device__ __forceinline__ uint32_t bf16x2_relu_bits(float x0, float x1) {
    uint32_t u;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(x1), "f"(x0));
    return u;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor of a K-major operand without swizzling
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, int K) {
    const uint64_t start = (addr >> 4) & 0x3FFFu;
    const uint64_t lbo = (128u >> 4) & 0x3FFFu;
    const uint64_t sbo = ((uint32_t)(K / 8) * 128u >> 4) & 0x3FFFu;
    return start | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// instruction descriptor: BF16 A and B (K-major), FP32 accumulator, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
    for (unsigned i = 0; i < MLPTC_WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's tensor-memory lane (issued
// only: tc_ld_wait() before the values are used)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tc_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// tensor-memory address of the accumulator row of tile row `row`: lane
// row % 128 (a warp reads the 32 lanes of its quarter), columns from
// 64 (row / 128)
__device__ __forceinline__ uint32_t tc_row_addr(uint32_t tmem, int row) {
    return tmem + ((uint32_t)(row & 96) << 16) + (uint32_t)(row >> 7) * 64u;
}

// Block set-up (all threads): tensor memory (warp 0), the barrier, the
// weights in BF16 in the core-matrix layout and the biases.
__device__ __forceinline__ void mlp_tc_setup(MlpTcSmem& s, const float* __restrict__ prm) {
    const float* W1 = prm;
    const float* b1 = W1 + MLP_H * MLP_IN;
    const float* W2 = b1 + MLP_H;
    const float* b2 = W2 + MLP_H * MLP_H;
    const float* W3 = b2 + MLP_H;
    const float* b3 = W3 + MLP_H * MLP_H;
    const float* W4 = b3 + MLP_H;
    const float* b4 = W4 + MLP_H;
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem)),
                     "r"(MLPTC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < MLP_H * MLP_INP; i += blockDim.x) {
        const int n = i / MLP_INP, k = i % MLP_INP;
        const float w = k < MLP_IN ? W1[n * MLP_IN + k] : (k == MLP_IN ? b1[n] : 0.f);
        s.W1[tc_idx(n, k, MLP_INP)] = __float2bfloat16_rn(w);
    }
    for (int i = threadIdx.x; i < MLP_H * MLPTC_KH; i += blockDim.x) {
        const int n = i / MLPTC_KH, k = i % MLPTC_KH;
        const bool wk = k < MLP_H, bk = k == MLP_H;
        s.W2[tc_idx(n, k, MLPTC_KH)] = __float2bfloat16_rn(wk ? W2[n * MLP_H + k] : (bk ? b2[n] : 0.f));
        s.W3[tc_idx(n, k, MLPTC_KH)] = __float2bfloat16_rn(wk ? W3[n * MLP_H + k] : (bk ? b3[n] : 0.f));
    }
    for (int i = threadIdx.x; i < 16 * MLPTC_KH; i += blockDim.x) {
        const int n = i / MLPTC_KH, k = i % MLPTC_KH;
        const float w = n != 0 ? 0.f : (k < MLP_H ? W4[k] : (k == MLP_H ? b4[0] : 0.f));
        s.W4[tc_idx(n, k, MLPTC_KH)] = __float2bfloat16_rn(w);
    }
    // the hidden layers' ones and zero columns (64 .. 79), written once: the
    // epilogues write columns 0 .. 63 only
    for (int r = threadIdx.x; r < MLPTC_CELLS; r += blockDim.x) {
        *reinterpret_cast<uint4*>(&s.acth[tc_idx(r, MLP_H, MLPTC_KH)]) = make_uint4(bf16x2_bits(1.f, 0.f), 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(&s.acth[tc_idx(r, MLP_H + 8, MLPTC_KH)]) = make_uint4(0u, 0u, 0u, 0u);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// One layer: thread 0 issues acc = A [128 x K] * W^T [K x N] into tensor
// memory for each of the tile's row blocks and commits to the barrier; every
// thread waits (bounded).
__device__ __forceinline__ bool mlp_tc_layer(MlpTcSmem& s, const __nv_bfloat16* A, const __nv_bfloat16* W, int K,
                                             int N, uint32_t& phase) {
    const uint32_t bar = smem_u32(&s.bar);
    if (threadIdx.x == 0) {
        const uint32_t a0 = smem_u32(A), b0 = smem_u32(W);
        const uint32_t idesc = tc_idesc(MLPTC_M, N);
        for (int rb = 0; rb < MLPTC_NT; ++rb)      // rows 128 rb ..: 128 K BF16 further, accumulator columns + 64 rb
            for (int ks = 0; ks < K / 16; ++ks)    // K = 16 per product: two core matrices along K
                tc_mma(s.tmem + 64 * rb, tc_desc(a0 + rb * MLPTC_M * K * 2 + ks * 256, K),
                       tc_desc(b0 + ks * 256, K), idesc, ks > 0);
        tc_commit(bar);
    }
    // every thread waits; the block agrees on the outcome (a uniform branch)
    const bool ok = __syncthreads_and(tc_wait(bar, phase)) != 0;
    phase ^= 1u;
    tc_fence_after();
    return ok;
}

// ReLU(acc) of this thread's row (the bias is in acc) -> BF16 columns 0 .. 63
// of its row of the next A operand, then make the writes visible to the
// tensor core
__device__ __forceinline__ void mlp_tc_hidden(MlpTcSmem& s) {
    const int row = threadIdx.x;
    const uint32_t lane_addr = tc_row_addr(s.tmem, row);
    // the row's 64 accumulator columns in groups of MLPTC_LD loads of 16
    // columns in flight; one 16-byte store per core matrix: the eight rows of
    // a warp's row group fill the core matrix's 128 bytes, one shared-memory
    // wavefront
    constexpr int G = MLPTC_LD;
#pragma unroll
    for (int half = 0; half < 4 / G; ++half) {
        uint32_t r[G][16];
#pragma unroll
        for (int q = 0; q < G; ++q) tc_ld16(lane_addr + 16 * G * half + 16 * q, r[q]);
        tc_ld_wait();
#pragma unroll
        for (int q = 0; q < G; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    w[j] = bf16x2_relu_bits(__uint_as_float(r[q][8 * h + 2 * j]),
                                            __uint_as_float(r[q][8 * h + 2 * j + 1]));
                *reinterpret_cast<uint4*>(&s.acth[tc_idx(row, 16 * G * half + 16 * q + 8 * h, MLPTC_KH)]) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Logit of this thread's cell (row threadIdx.x of the tile) from its 40
// features; all MLPTC_CELLS threads of the block call it.  Returns false if a wait
// ran out (the logit is then NaN).
__device__ __forceinline__ bool mlp_tc_logit(MlpTcSmem& s, const float* feat, uint32_t& phase, float& z) {
    const int row = threadIdx.x;
#pragma unroll
    for (int k = 0; k < MLP_INP; k += 8) {    // 16 bytes (one core-matrix row) per store
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k0 = k + 2 * j;   // features, then the ones column (the bias), then zeros
            w[j] = bf16x2_bits(k0 < MLP_IN ? feat[k0] : (k0 == MLP_IN ? 1.f : 0.f),
                               k0 + 1 < MLP_IN ? feat[k0 + 1] : 0.f);
        }
        *reinterpret_cast<uint4*>(&s.act1[tc_idx(row, k, MLP_INP)]) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    z = __int_as_float(0x7fc00000);
    if (!mlp_tc_layer(s, s.act1, s.W1, MLP_INP, MLP_H, phase)) return false;
    mlp_tc_hidden(s);
    if (!mlp_tc_layer(s, s.acth, s.W2, MLPTC_KH, MLP_H, phase)) return false;
    mlp_tc_hidden(s);
    if (!mlp_tc_layer(s, s.acth, s.W3, MLPTC_KH, MLP_H, phase)) return false;
    mlp_tc_hidden(s);
    if (!mlp_tc_layer(s, s.acth, s.W4, MLPTC_KH, 16, phase)) return false;
    uint32_t v[16];
    tc_ld16(tc_row_addr(s.tmem, row), v);
    tc_ld_wait();
    z = __uint_as_float(v[0]);
    // the accumulator is read before the tile's next product overwrites it
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return true;
}

// Block tear-down: free the tensor memory (warp 0) once every thread is done
__device__ __forceinline__ void mlp_tc_teardown(MlpTcSmem& s) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "r"(MLPTC_TMEM_COLS)
                     : "memory");
}

}  // namespace crk
