// Learned troubled-cell indicator (not in the paper): a 40 -> 64 -> 64 -> 64
// -> 1 ReLU network evaluated by one warp for 32 cells at a time on the tensor
// cores (mma.sync m16n8k16, BF16 inputs, FP32 accumulation).  Layers chain in
// registers: the FP32 accumulator fragments of two adjacent 8-column tiles
// are, after ReLU and conversion, exactly the BF16 A fragment of one 16-wide
// k slice of the next layer.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace crk {

constexpr int MLP_IN = 40, MLP_INP = 48, MLP_H = 64;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + 2 * (MLP_H * MLP_H + MLP_H) + MLP_H + 1;   // 11009

// Weights as the tensor cores read them (B operands are W rows: k contiguous)
struct MlpSmem {
    __nv_bfloat16 W1[MLP_H * MLP_INP];   // layer 1, input padded 40 -> 48 with zeros
    __nv_bfloat16 W2[MLP_H * MLP_H];
    __nv_bfloat16 W3[MLP_H * MLP_H];
    __nv_bfloat16 W4[8 * MLP_H];         // output row 0, rows 1..7 zero
    float b1[MLP_H], b2[MLP_H], b3[MLP_H], b4[8];
};

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// C fragments of n-tiles 2t and 2t+1 (bias added, ReLU) -> A fragment of k slice t
__device__ __forceinline__ void c_to_a(const float (&c0)[4], const float (&c1)[4], uint32_t (&a)[4]) {
    a[0] = pack_bf16(fmaxf(c0[0], 0.f), fmaxf(c0[1], 0.f));
    a[1] = pack_bf16(fmaxf(c0[2], 0.f), fmaxf(c0[3], 0.f));
    a[2] = pack_bf16(fmaxf(c1[0], 0.f), fmaxf(c1[1], 0.f));
    a[3] = pack_bf16(fmaxf(c1[2], 0.f), fmaxf(c1[3], 0.f));
}

// One hidden layer: acc[nt] = bias + A * W^T over KS k-slices of 16
template <int KS>
__device__ __forceinline__ void mlp_layer(const uint32_t (&a)[KS][4], const __nv_bfloat16* W, const float* bias,
                                          int ldw, float (&acc)[8][4], int g, int tig) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float b0 = bias[nt * 8 + 2 * tig], b1 = bias[nt * 8 + 2 * tig + 1];
        acc[nt][0] = b0;
        acc[nt][1] = b1;
        acc[nt][2] = b0;
        acc[nt][3] = b1;
        const __nv_bfloat16* wr = W + (size_t)(nt * 8 + g) * ldw;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            const uint32_t bb0 = *reinterpret_cast<const uint32_t*>(wr + ks * 16 + 2 * tig);
            const uint32_t bb1 = *reinterpret_cast<const uint32_t*>(wr + ks * 16 + 8 + 2 * tig);
            mma_bf16(acc[nt], a[ks], bb0, bb1);
        }
    }
}

// Logits of the 32 cells held by the warp's lanes.  feat: this lane's 40
// features; stage: the warp's 32 x 48 BF16 staging area (+ 32 floats after it).
__device__ __forceinline__ float mlp_warp_logit(const MlpSmem& w, const float* feat, __nv_bfloat16* stage) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, tig = lane & 3;
    float* lout = reinterpret_cast<float*>(stage + 32 * MLP_INP);
#pragma unroll
    for (int f = 0; f < MLP_INP; f += 2)
        *reinterpret_cast<uint32_t*>(stage + lane * MLP_INP + f) =
            pack_bf16(f < MLP_IN ? feat[f] : 0.f, f + 1 < MLP_IN ? feat[f + 1] : 0.f);
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        uint32_t a1[3][4];
        const __nv_bfloat16* r0 = stage + (mt * 16 + g) * MLP_INP;
        const __nv_bfloat16* r1 = stage + (mt * 16 + g + 8) * MLP_INP;
#pragma unroll
        for (int ks = 0; ks < 3; ++ks) {
            a1[ks][0] = *reinterpret_cast<const uint32_t*>(r0 + ks * 16 + 2 * tig);
            a1[ks][1] = *reinterpret_cast<const uint32_t*>(r1 + ks * 16 + 2 * tig);
            a1[ks][2] = *reinterpret_cast<const uint32_t*>(r0 + ks * 16 + 8 + 2 * tig);
            a1[ks][3] = *reinterpret_cast<const uint32_t*>(r1 + ks * 16 + 8 + 2 * tig);
        }
        float acc[8][4];
        uint32_t ah[4][4];
        mlp_layer<3>(a1, w.W1, w.b1, MLP_INP, acc, g, tig);
#pragma unroll
        for (int t = 0; t < 4; ++t) c_to_a(acc[2 * t], acc[2 * t + 1], ah[t]);
        mlp_layer<4>(ah, w.W2, w.b2, MLP_H, acc, g, tig);
#pragma unroll
        for (int t = 0; t < 4; ++t) c_to_a(acc[2 * t], acc[2 * t + 1], ah[t]);
        mlp_layer<4>(ah, w.W3, w.b3, MLP_H, acc, g, tig);
#pragma unroll
        for (int t = 0; t < 4; ++t) c_to_a(acc[2 * t], acc[2 * t + 1], ah[t]);
        // output layer: one 8-column tile, column 0 is the logit
        float o[4] = {w.b4[2 * tig], w.b4[2 * tig + 1], w.b4[2 * tig], w.b4[2 * tig + 1]};
        const __nv_bfloat16* wr = w.W4 + (size_t)g * MLP_H;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const uint32_t bb0 = *reinterpret_cast<const uint32_t*>(wr + ks * 16 + 2 * tig);
            const uint32_t bb1 = *reinterpret_cast<const uint32_t*>(wr + ks * 16 + 8 + 2 * tig);
            mma_bf16(o, ah[ks], bb0, bb1);
        }
        if (tig == 0) {
            lout[mt * 16 + g] = o[0];
            lout[mt * 16 + g + 8] = o[2];
        }
    }
    __syncwarp();
    const float z = lout[lane];
    __syncwarp();
    return z;
}

// Load the BF16 weights and FP32 biases of a packed parameter vector (device,
// FP32, order W1 b1 W2 b2 W3 b3 W4 b4, W row-major out x in) into shared
// memory; every thread of the block takes part.
__device__ __forceinline__ void mlp_load_smem(MlpSmem& w, const float* __restrict__ prm) {
    const float* W1 = prm;
    const float* b1 = W1 + MLP_H * MLP_IN;
    const float* W2 = b1 + MLP_H;
    const float* b2 = W2 + MLP_H * MLP_H;
    const float* W3 = b2 + MLP_H;
    const float* b3 = W3 + MLP_H * MLP_H;
    const float* W4 = b3 + MLP_H;
    const float* b4 = W4 + MLP_H;
    for (int i = threadIdx.x; i < MLP_H * MLP_INP; i += blockDim.x) {
        const int r = i / MLP_INP, c = i % MLP_INP;
        w.W1[i] = __float2bfloat16_rn(c < MLP_IN ? W1[r * MLP_IN + c] : 0.f);
    }
    for (int i = threadIdx.x; i < MLP_H * MLP_H; i += blockDim.x) {
        w.W2[i] = __float2bfloat16_rn(W2[i]);
        w.W3[i] = __float2bfloat16_rn(W3[i]);
    }
    for (int i = threadIdx.x; i < 8 * MLP_H; i += blockDim.x) w.W4[i] = __float2bfloat16_rn(i < MLP_H ? W4[i] : 0.f);
    for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) {
        w.b1[i] = b1[i];
        w.b2[i] = b2[i];
        w.b3[i] = b3[i];
    }
    if (threadIdx.x < 8) w.b4[threadIdx.x] = threadIdx.x == 0 ? b4[0] : 0.f;
}

// The 40 input features of one P^2 (or richer) Euler cell: per variable q the
// four neighbour-average differences and the five non-constant P^2 modes,
// divided by their largest magnitude s_q, then log10(s_q / (M h^2)) clipped
// to [-8, 8] for each q.  Order: 9 normalised values of q = 0..3, then the
// four scale values.
template <class T, int NM>
__device__ __forceinline__ void mlp_features(const T (&u)[4][NM], const T* nbE, const T* nbW, const T* nbN,
                                             const T* nbS, double Mh2, float* f) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float avg = float(u[q][0]);
        float d[9] = {float(nbE[q]) - avg, float(nbW[q]) - avg, float(nbN[q]) - avg, float(nbS[q]) - avg,
                      float(u[q][1]), float(u[q][2]), NM > 3 ? float(u[q][NM > 3 ? 3 : 0]) : 0.f,
                      NM > 4 ? float(u[q][NM > 4 ? 4 : 0]) : 0.f, NM > 5 ? float(u[q][NM > 5 ? 5 : 0]) : 0.f};
        float s = 1e-30f;
#pragma unroll
        for (int i = 0; i < 9; ++i) s = fmaxf(s, fabsf(d[i]));
        const float is = 1.0f / s;
#pragma unroll
        for (int i = 0; i < 9; ++i) f[q * 9 + i] = d[i] * is;
        float sc = log10f(s / float(Mh2));
        f[36 + q] = fminf(fmaxf(sc, -8.f), 8.f);
    }
}

}  // namespace crk
