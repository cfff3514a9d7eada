// Learned troubled-cell indicator (no counterpart in the paper): training
// kernels (FP32 forward/backward with a deterministic gradient reduction,
// Adam), BF16 tensor-core inference, and the feature/label extraction from a
// solver state.  C ABI part of include/crkdg.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/crkdg.h"
#include "aux_kernels.cuh"
#include "launch.h"
#include "mlp_warp.cuh"
#include "mlp_tc.cuh"

using crk::MLP_H;
using crk::MLP_IN;
using crk::MLP_NPARAM;
using crk::StepArgs;

namespace {

thread_local std::string g_merr;
int mfail(int code, const std::string& m) {
    g_merr = m;
    return code;
}
#define MCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return mfail(CRKDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int TILE = 64;   // samples per block in training

// offsets of the packed parameter vector
constexpr int OW1 = 0, OB1 = OW1 + MLP_H * MLP_IN, OW2 = OB1 + MLP_H, OB2 = OW2 + MLP_H * MLP_H,
              OW3 = OB2 + MLP_H, OB3 = OW3 + MLP_H * MLP_H, OW4 = OB3 + MLP_H, OB4 = OW4 + MLP_H;

// Forward and backward of the mean class-weighted BCE over a tile of TILE
// samples (rows idx[i] of X, labels y); writes this block's gradient
// contribution (already divided by n) and loss sum.
__global__ void __launch_bounds__(256) mlp_fwdbwd_kernel(const float* __restrict__ prm, const float* __restrict__ X,
                                                         const float* __restrict__ y, const int* __restrict__ idx,
                                                         int n, float pos_weight, float* __restrict__ gpart,
                                                         float* __restrict__ lpart) {
    extern __shared__ float sh[];
    float* P = sh;                                  // parameters
    float* Xs = P + MLP_NPARAM;                     // TILE x 40
    float* H1 = Xs + TILE * MLP_IN;                 // TILE x 64 each
    float* H2 = H1 + TILE * MLP_H;
    float* H3 = H2 + TILE * MLP_H;
    float* G = H3 + TILE * MLP_H;                   // TILE x 64 (current delta)
    float* G2 = G + TILE * MLP_H;                   // TILE x 64 (next delta)
    float* dz = G2 + TILE * MLP_H;                  // TILE
    const int tid = threadIdx.x, nth = blockDim.x;
    const int s0 = blockIdx.x * TILE;
    const int ns = min(TILE, n - s0);
    for (int i = tid; i < MLP_NPARAM; i += nth) P[i] = prm[i];
    for (int i = tid; i < TILE * MLP_IN; i += nth) {
        const int s = i / MLP_IN, k = i % MLP_IN;
        Xs[i] = s < ns ? X[(size_t)idx[s0 + s] * MLP_IN + k] : 0.f;
    }
    __syncthreads();
    // forward
    auto dense = [&](const float* in, int nin, const float* W, const float* b, float* out) {
        for (int i = tid; i < TILE * MLP_H; i += nth) {
            const int s = i / MLP_H, j = i % MLP_H;
            float a = b[j];
            for (int k = 0; k < nin; ++k) a = fmaf(in[s * nin + k], W[j * nin + k], a);
            out[i] = fmaxf(a, 0.f);
        }
        __syncthreads();
    };
    dense(Xs, MLP_IN, P + OW1, P + OB1, H1);
    dense(H1, MLP_H, P + OW2, P + OB2, H2);
    dense(H2, MLP_H, P + OW3, P + OB3, H3);
    float lsum = 0.f;
    for (int s = tid; s < TILE; s += nth) {
        float z = P[OB4];
        for (int k = 0; k < MLP_H; ++k) z = fmaf(H3[s * MLP_H + k], P[OW4 + k], z);
        if (s < ns) {
            const float yy = y[idx[s0 + s]];
            const float ls = -log1pf(expf(-fabsf(z))) + fminf(z, 0.f);       // log sigma(z)
            const float l1s = -log1pf(expf(-fabsf(z))) + fminf(-z, 0.f);     // log(1 - sigma(z))
            lsum += -(pos_weight * yy * ls + (1.f - yy) * l1s);
            const float sg = 1.f / (1.f + expf(-z));
            dz[s] = (pos_weight * yy * (sg - 1.f) + (1.f - yy) * sg) / float(n);
        } else {
            dz[s] = 0.f;
        }
    }
    __syncthreads();
    float* gb = gpart + (size_t)blockIdx.x * MLP_NPARAM;
    // output layer
    for (int k = tid; k < MLP_H; k += nth) {
        float a = 0.f;
        for (int s = 0; s < TILE; ++s) a = fmaf(dz[s], H3[s * MLP_H + k], a);
        gb[OW4 + k] = a;
    }
    if (tid == 0) {
        float a = 0.f;
        for (int s = 0; s < TILE; ++s) a += dz[s];
        gb[OB4] = a;
    }
    for (int i = tid; i < TILE * MLP_H; i += nth) {
        const int s = i / MLP_H, j = i % MLP_H;
        G[i] = H3[i] > 0.f ? dz[s] * P[OW4 + j] : 0.f;
    }
    __syncthreads();
    // hidden layers: G is the delta at the output of the layer
    auto back = [&](const float* in, int nin, const float* W, int ow, int ob, const float* hin, float* gout) {
        for (int i = tid; i < MLP_H * nin; i += nth) {
            const int j = i / nin, k = i % nin;
            float a = 0.f;
            for (int s = 0; s < TILE; ++s) a = fmaf(G[s * MLP_H + j], in[s * nin + k], a);
            gb[ow + i] = a;
        }
        for (int j = tid; j < MLP_H; j += nth) {
            float a = 0.f;
            for (int s = 0; s < TILE; ++s) a += G[s * MLP_H + j];
            gb[ob + j] = a;
        }
        if (gout) {
            for (int i = tid; i < TILE * nin; i += nth) {
                const int s = i / nin, k = i % nin;
                float a = 0.f;
                for (int j = 0; j < MLP_H; ++j) a = fmaf(G[s * MLP_H + j], W[j * nin + k], a);
                gout[i] = hin[i] > 0.f ? a : 0.f;
            }
        }
        __syncthreads();
    };
    back(H2, MLP_H, P + OW3, OW3, OB3, H2, G2);
    for (int i = tid; i < TILE * MLP_H; i += nth) G[i] = G2[i];
    __syncthreads();
    back(H1, MLP_H, P + OW2, OW2, OB2, H1, G2);
    for (int i = tid; i < TILE * MLP_H; i += nth) G[i] = G2[i];
    __syncthreads();
    back(Xs, MLP_IN, P + OW1, OW1, OB1, nullptr, nullptr);
    // loss partial
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    __shared__ float lred[32];
    if ((tid & 31) == 0) lred[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float a = 0.f;
        for (int i = 0; i < (nth >> 5); ++i) a += lred[i];
        lpart[blockIdx.x] = a;
    }
}

// grad[p] = sum over blocks, in block order (deterministic)
__global__ void mlp_reduce_kernel(const float* __restrict__ gpart, int nblocks, float* __restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_NPARAM) return;
    float a = 0.f;
    for (int b = 0; b < nblocks; ++b) a += gpart[(size_t)b * MLP_NPARAM + p];
    grad[p] = a;
}

// Adam (Kingma and Ba): m, v moments, bias-corrected step
__global__ void mlp_adam_kernel(float* __restrict__ prm, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_NPARAM) return;
    const float gi = g[p];
    const float mi = b1 * m[p] + (1.f - b1) * gi;
    const float vi = b2 * v[p] + (1.f - b2) * gi * gi;
    m[p] = mi;
    v[p] = vi;
    prm[p] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 tensor-core inference, one warp per 32 samples
__global__ void __launch_bounds__(128) mlp_predict_kernel(const float* __restrict__ prm, const float* __restrict__ X,
                                                          int n, float* __restrict__ logits) {
    extern __shared__ __align__(16) unsigned char smb[];
    crk::MlpSmem& w = *reinterpret_cast<crk::MlpSmem*>(smb);
    __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(smb + sizeof(crk::MlpSmem)) +
                           (threadIdx.x >> 5) * (32 * crk::MLP_INP + 64);
    crk::mlp_load_smem(w, prm);
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float f[MLP_IN];
    for (int k = 0; k < MLP_IN; ++k) f[k] = s < n ? X[(size_t)s * MLP_IN + k] : 0.f;
    const float z = crk::mlp_warp_logit(w, f, stage);
    if (s < n) logits[s] = z;
}

// The same inference on the fifth-generation tensor cores (mlp_tc.cuh): one
// tile of 128 samples per block iteration, grid-stride over the tiles; a
// bounded wait that ran out sets ST_TIMEOUT in *status.
__global__ void __launch_bounds__(crk::MLPTC_CELLS) mlp_predict_tc_kernel(const float* __restrict__ prm,
                                                             const float* __restrict__ X, int n,
                                                             float* __restrict__ logits, unsigned* status) {
    extern __shared__ __align__(1024) unsigned char smt[];
    crk::MlpTcSmem& s = *reinterpret_cast<crk::MlpTcSmem*>(smt);
    crk::mlp_tc_setup(s, prm);
    uint32_t phase = 0;
    bool ok = true;
    for (int tile = blockIdx.x; ok && (long long)tile * crk::MLPTC_CELLS < n; tile += gridDim.x) {
        const int i = tile * crk::MLPTC_CELLS + threadIdx.x;
        float f[MLP_IN];
        for (int k = 0; k < MLP_IN; ++k) f[k] = i < n ? X[(size_t)i * MLP_IN + k] : 0.f;
        float z;
        ok = crk::mlp_tc_logit(s, f, phase, z);
        if (i < n) logits[i] = z;
    }
    if (!ok && threadIdx.x == 0) atomicOr(status, crk::ST_TIMEOUT);
    crk::mlp_tc_teardown(s);
}

// Features and TVB labels of every cell of a P^2 2D Euler state (one thread
// per cell).  Label 1 when the TVB-minmod test of the limiter flags the cell.
template <class T, int K, int B>
__global__ void features_kernel(const StepArgs a, const T* __restrict__ u, float* __restrict__ X,
                                float* __restrict__ y, double Mh2) {
    constexpr int NM = crk::Tab2D<K, B>::NM;
    const int nx = a.nx, ny = a.ny;
    const size_t plane = (size_t)nx * ny;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int yy = blockIdx.y;
    if (x >= nx) return;
    const bool perx = a.bc[0].type == crk::BC_PERIODIC, pery = a.bc[2].type == crk::BC_PERIODIC;
    T c[4][NM];
    for (int v = 0; v < 4; ++v)
        for (int m = 0; m < NM; ++m) c[v][m] = u[(size_t)(v * NM + m) * plane + (size_t)yy * nx + x];
    T own[4], nb[4][4];
    for (int v = 0; v < 4; ++v) own[v] = c[v][0];
    const int xs[4] = {x - 1, x + 1, x, x};
    const int ys[4] = {yy, yy, yy - 1, yy + 1};
    for (int s = 0; s < 4; ++s) {
        int cx = xs[s], cy = ys[s];
        const bool out = (s < 2 && !perx && (cx < 0 || cx >= nx)) || (s >= 2 && !pery && (cy < 0 || cy >= ny));
        if (out) {
            crk::bc_exterior<T, 4>(a.bc[s], s < 2 ? 0 : 1, own, [&](double& xc, double& yc, double& tc) {
                xc = a.x0 + (cx + 0.5) * a.dx;
                yc = a.y0 + (cy + 0.5) * a.dy;
                tc = a.t;
            }, nb[s]);
        } else {
            cx = (cx + nx) % nx;
            cy = (cy + ny) % ny;
            for (int v = 0; v < 4; ++v) nb[s][v] = u[(size_t)(v * NM) * plane + (size_t)cy * nx + cx];
        }
    }
    float f[MLP_IN];
    crk::mlp_features<T, NM>(c, nb[1], nb[0], nb[3], nb[2], Mh2, f);
    const size_t cell = (size_t)yy * nx + x;
    for (int k = 0; k < MLP_IN; ++k) X[cell * MLP_IN + k] = f[k];
    const bool fl = crk::tvb_limit_cell<T, 4, NM>(c, nb[0], nb[1], nb[2], nb[3], T(a.M * a.dx * a.dx),
                                                  T(a.M * a.dy * a.dy), T(a.gamma));
    y[cell] = fl ? 1.f : 0.f;
}

uint64_t splitmix(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

}  // namespace

struct crkdg_mlp {
    unsigned* d_status = nullptr;   // ST_TIMEOUT of a tensor-core wait that ran out
    float* d_prm = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    float* d_grad = nullptr;
    cudaStream_t stream = nullptr;
    long long adam_t = 0;
};

// exported for the step kernels' MLP indicator
const float* crkdg_mlp_device_params(const crkdg_mlp* m) { return m ? m->d_prm : nullptr; }

extern "C" {

const char* crkdg_mlp_last_error(void) { return g_merr.c_str(); }

int crkdg_mlp_create(unsigned long long seed, void* stream, crkdg_mlp** out) {
    if (!out) return mfail(CRKDG_EINVAL, "null argument");
    crkdg_mlp* m = new crkdg_mlp();
    m->stream = static_cast<cudaStream_t>(stream);
    std::vector<float> h(MLP_NPARAM, 0.f);
    uint64_t s = seed;
    auto he = [&](int off, int nout, int nin) {
        const double sd = std::sqrt(2.0 / nin);
        for (int i = 0; i < nout * nin; ++i) {
            // Box--Muller normal from two uniforms
            const double u1 = uniform01(s), u2 = uniform01(s);
            h[off + i] = float(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    };
    he(OW1, MLP_H, MLP_IN);
    he(OW2, MLP_H, MLP_H);
    he(OW3, MLP_H, MLP_H);
    he(OW4, 1, MLP_H);
    if (cudaMalloc(&m->d_prm, MLP_NPARAM * 4) != cudaSuccess || cudaMalloc(&m->d_m, MLP_NPARAM * 4) != cudaSuccess ||
        cudaMalloc(&m->d_v, MLP_NPARAM * 4) != cudaSuccess || cudaMalloc(&m->d_grad, MLP_NPARAM * 4) != cudaSuccess) {
        crkdg_mlp_destroy(m);
        return mfail(CRKDG_ENOMEM, "cudaMalloc failed");
    }
    if (cudaMalloc(&m->d_status, sizeof(unsigned)) != cudaSuccess) {
        crkdg_mlp_destroy(m);
        return mfail(CRKDG_ENOMEM, "cudaMalloc failed");
    }
    cudaMemset(m->d_status, 0, sizeof(unsigned));
    cudaMemcpy(m->d_prm, h.data(), MLP_NPARAM * 4, cudaMemcpyHostToDevice);
    cudaMemset(m->d_m, 0, MLP_NPARAM * 4);
    cudaMemset(m->d_v, 0, MLP_NPARAM * 4);
    *out = m;
    return CRKDG_OK;
}

void crkdg_mlp_destroy(crkdg_mlp* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    for (float* p : {m->d_prm, m->d_m, m->d_v, m->d_grad})
        if (p) cudaFree(p);
    if (m->d_status) cudaFree(m->d_status);
    delete m;
}

int crkdg_mlp_n_params(void) { return MLP_NPARAM; }

int crkdg_mlp_set_params(crkdg_mlp* m, const float* host) {
    if (!m || !host) return mfail(CRKDG_EINVAL, "null argument");
    MCK(cudaMemcpy(m->d_prm, host, MLP_NPARAM * 4, cudaMemcpyHostToDevice));
    MCK(cudaMemset(m->d_m, 0, MLP_NPARAM * 4));
    MCK(cudaMemset(m->d_v, 0, MLP_NPARAM * 4));
    m->adam_t = 0;
    return CRKDG_OK;
}

int crkdg_mlp_get_params(const crkdg_mlp* m, float* host) {
    if (!m || !host) return mfail(CRKDG_EINVAL, "null argument");
    MCK(cudaStreamSynchronize(m->stream));
    MCK(cudaMemcpy(host, m->d_prm, MLP_NPARAM * 4, cudaMemcpyDeviceToHost));
    return CRKDG_OK;
}

// Mean loss and its gradient over the n samples (rows of X_dev, labels y_dev,
// device FP32); grad_dev (device, MLP_NPARAM floats) may be NULL.
static int loss_grad(crkdg_mlp* m, const float* X, const float* y, const int* idx, int n, double pw, double* loss,
                     float* grad_dev) {
    const int nb = (n + TILE - 1) / TILE;
    float *gpart = nullptr, *lpart = nullptr;
    if (cudaMalloc(&gpart, (size_t)nb * MLP_NPARAM * 4) != cudaSuccess || cudaMalloc(&lpart, nb * 4) != cudaSuccess) {
        if (gpart) cudaFree(gpart);
        return mfail(CRKDG_ENOMEM, "cudaMalloc failed");
    }
    const size_t smem = (size_t)(MLP_NPARAM + TILE * MLP_IN + 5 * TILE * MLP_H + TILE) * 4;
    cudaFuncSetAttribute(mlp_fwdbwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mlp_fwdbwd_kernel<<<nb, 256, smem, m->stream>>>(m->d_prm, X, y, idx, n, (float)pw, gpart, lpart);
    mlp_reduce_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, m->stream>>>(gpart, nb, grad_dev ? grad_dev : m->d_grad);
    cudaError_t e = cudaGetLastError();
    std::vector<float> lp(nb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lp.data(), lpart, nb * 4, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    cudaFree(gpart);
    cudaFree(lpart);
    if (e != cudaSuccess) return mfail(CRKDG_ECUDA, std::string("loss/grad: ") + cudaGetErrorString(e));
    double l = 0.0;
    for (float v : lp) l += v;
    if (loss) *loss = l / n;
    return CRKDG_OK;
}

int crkdg_mlp_loss_grad(crkdg_mlp* m, const float* X_dev, const float* y_dev, int n, double pos_weight, double* loss,
                        float* grad_host) {
    if (!m || !X_dev || !y_dev || n < 1) return mfail(CRKDG_EINVAL, "bad argument");
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    int* d_idx = nullptr;
    MCK(cudaMalloc(&d_idx, n * sizeof(int)));
    cudaMemcpy(d_idx, idx.data(), n * sizeof(int), cudaMemcpyHostToDevice);
    int r = loss_grad(m, X_dev, y_dev, d_idx, n, pos_weight, loss, nullptr);
    cudaFree(d_idx);
    if (r) return r;
    if (grad_host) MCK(cudaMemcpy(grad_host, m->d_grad, MLP_NPARAM * 4, cudaMemcpyDeviceToHost));
    return CRKDG_OK;
}

int crkdg_mlp_train(crkdg_mlp* m, const float* X_dev, const float* y_dev, int n, int epochs, int batch, double lr,
                    double pos_weight, unsigned long long seed, double* last_epoch_loss) {
    if (!m || !X_dev || !y_dev || n < 1 || epochs < 0 || batch < 1 || !(lr > 0.0))
        return mfail(CRKDG_EINVAL, "bad argument");
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    int* d_idx = nullptr;
    MCK(cudaMalloc(&d_idx, n * sizeof(int)));
    uint64_t s = seed;
    double el = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = n - 1; i > 0; --i) {   // Fisher--Yates shuffle
            const int j = (int)(splitmix(s) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        cudaMemcpyAsync(d_idx, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, m->stream);
        el = 0.0;
        int nb = 0;
        for (int b0 = 0; b0 < n; b0 += batch) {
            const int nbatch = std::min(batch, n - b0);
            double l = 0.0;
            int r = loss_grad(m, X_dev, y_dev, d_idx + b0, nbatch, pos_weight, &l, nullptr);
            if (r) {
                cudaFree(d_idx);
                return r;
            }
            m->adam_t += 1;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - std::pow(b1, (double)m->adam_t), c2 = 1.f - std::pow(b2, (double)m->adam_t);
            mlp_adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, m->stream>>>(m->d_prm, m->d_grad, m->d_m, m->d_v,
                                                                             (float)lr, b1, b2, 1e-8f, c1, c2);
            el += l;
            ++nb;
        }
        el /= nb;
    }
    cudaError_t e = cudaStreamSynchronize(m->stream);
    cudaFree(d_idx);
    if (e != cudaSuccess) return mfail(CRKDG_ECUDA, std::string("train: ") + cudaGetErrorString(e));
    if (last_epoch_loss) *last_epoch_loss = el;
    return CRKDG_OK;
}

int crkdg_mlp_predict(crkdg_mlp* m, const float* X_dev, int n, float* logits_dev) {
    if (!m || !X_dev || !logits_dev || n < 1) return mfail(CRKDG_EINVAL, "bad argument");
    const size_t smem = sizeof(crk::MlpSmem) + 4 * (32 * crk::MLP_INP + 64) * sizeof(__nv_bfloat16);
    cudaFuncSetAttribute(mlp_predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mlp_predict_kernel<<<(n + 127) / 128, 128, smem, m->stream>>>(m->d_prm, X_dev, n, logits_dev);
    MCK(cudaGetLastError());
    MCK(cudaStreamSynchronize(m->stream));
    return CRKDG_OK;
}

int crkdg_mlp_predict_tc(crkdg_mlp* m, const float* X_dev, int n, float* logits_dev) {
    if (!m || !X_dev || !logits_dev || n < 1) return mfail(CRKDG_EINVAL, "bad argument");
    const size_t smem = sizeof(crk::MlpTcSmem) + crk::MLPTC_SMEM_SLACK;
    MCK(cudaFuncSetAttribute(mlp_predict_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long tiles = ((long long)n + crk::MLPTC_CELLS - 1) / crk::MLPTC_CELLS;
    const int grid = (int)std::min<long long>(tiles, 4LL * std::max(1, crk::sm_count()));
    MCK(cudaMemsetAsync(m->d_status, 0, sizeof(unsigned), m->stream));
    mlp_predict_tc_kernel<<<grid, crk::MLPTC_CELLS, smem, m->stream>>>(m->d_prm, X_dev, n, logits_dev, m->d_status);
    MCK(cudaGetLastError());
    unsigned st = 0;
    MCK(cudaMemcpyAsync(&st, m->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    if (st) return mfail(CRKDG_ETIMEOUT, "a bounded wait for the tensor core ran out");
    return CRKDG_OK;
}

}  // extern "C"

// features of a state slice (used by the context and batch entry points)
int crkdg_features_impl(const StepArgs& a, int precision, int k, int basis, const void* u, float* X, float* y,
                        double Mh2, cudaStream_t st) {
    if (k != 2) return mfail(CRKDG_EUNSUPPORTED, "the learned indicator is built for k = 2");
    dim3 grid((a.nx + 127) / 128, a.ny);
    if (precision == CRKDG_F64) {
        if (basis == CRKDG_BASIS_P)
            features_kernel<double, 2, 0><<<grid, 128, 0, st>>>(a, (const double*)u, X, y, Mh2);
        else
            features_kernel<double, 2, 1><<<grid, 128, 0, st>>>(a, (const double*)u, X, y, Mh2);
    } else {
        if (basis == CRKDG_BASIS_P)
            features_kernel<float, 2, 0><<<grid, 128, 0, st>>>(a, (const float*)u, X, y, Mh2);
        else
            features_kernel<float, 2, 1><<<grid, 128, 0, st>>>(a, (const float*)u, X, y, Mh2);
    }
    MCK(cudaGetLastError());
    return CRKDG_OK;
}
