// Training and inference kernels of the learned brancher (no counterpart in the paper: the
// brancher is an addition to the method that changes only the exploration order).
//
//   csp_mlp_pack     flat bf16 parameters -> fragment-ordered block (see mlp.cuh)
//   csp_mlp_forward  scores of a batch of feature rows with the tensor-core tile (mma.sync)
//   csp_mlp_grad     mean-squared-error loss and gradient of a batch (fp32; weights and
//                    activations rounded to bf16 at the same points as the inference tile)
//   csp_mlp_adam     Adam step on fp32 master weights, refreshing the bf16 copy
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/cubics.h"
#include "mlp.cuh"

namespace cubics {

__global__ void mlp_pack_kernel(const uint16_t *params, uint32_t *packed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < PK_WORDS) packed[i] = pack_word(params, i);
}

__global__ void mlp_forward_kernel(const uint32_t *packed, const float *X, int rows, float *out) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int tile = warp; tile * 16 < rows; tile += nwarps) {
        const int r0 = tile * 16;
        auto x = [&](int r, int c) -> uint32_t {
            const int row = r0 + r;
            if (row >= rows) return 0u;
            return pack_bf16(X[(size_t)row * 16 + c], X[(size_t)row * 16 + c + 1]);
        };
        auto pk = [&](int i) -> uint32_t { return __ldg(packed + i); };
        float lo, hi;
        mlp_tile(x, pk, lo, hi);
        if ((lane & 3) == 0) {
            const int g = lane >> 2;
            if (r0 + g < rows) out[r0 + g] = lo;
            if (r0 + g + 8 < rows) out[r0 + g + 8] = hi;
        }
    }
}

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

constexpr int TR = 32;   // rows per block iteration of the gradient kernel

// smem: weights (5313), gradient accumulators (5313), X (TR x 16), Z1, H1, Z2, H2, dZ2, dZ1
// (TR x 64 each), s, ds (TR each)
__global__ void __launch_bounds__(256) mlp_grad_kernel(const float *master, const float *X,
                                                        const float *y, int rows, float *grad,
                                                        float *loss) {
    extern __shared__ float F[];
    float *Wt = F;
    float *G = Wt + MLP_PARAMS;
    float *Xs = G + MLP_PARAMS;
    float *Z1 = Xs + TR * 16, *H1 = Z1 + TR * 64, *Z2 = H1 + TR * 64, *H2 = Z2 + TR * 64;
    float *dZ2 = H2 + TR * 64, *dZ1 = dZ2 + TR * 64, *s = dZ1 + TR * 64, *ds = s + TR;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < MLP_PARAMS; i += nt) {
        Wt[i] = bf16r(master[i]);            // weights and biases are stored as bf16
        G[i] = 0.f;
    }
    float my_loss = 0.f;
    const float inv_b = 1.f / (float)rows;
    __syncthreads();
    for (int r0 = blockIdx.x * TR; r0 < rows; r0 += gridDim.x * TR) {
        const int nr = min(TR, rows - r0);
        for (int i = tid; i < TR * 16; i += nt)
            Xs[i] = (i / 16 < nr) ? bf16r(X[(size_t)r0 * 16 + i]) : 0.f;
        __syncthreads();
        for (int i = tid; i < TR * 64; i += nt) {            // layer 1
            const int r = i / 64, c = i % 64;
            float a = Wt[MLP_OFF_B1 + c];
            for (int k = 0; k < 16; ++k) a = fmaf(Xs[r * 16 + k], Wt[MLP_OFF_W1 + k * 64 + c], a);
            Z1[i] = a;
            H1[i] = bf16r(fmaxf(a, 0.f));
        }
        __syncthreads();
        for (int i = tid; i < TR * 64; i += nt) {            // layer 2
            const int r = i / 64, c = i % 64;
            float a = Wt[MLP_OFF_B2 + c];
            for (int k = 0; k < 64; ++k) a = fmaf(H1[r * 64 + k], Wt[MLP_OFF_W2 + k * 64 + c], a);
            Z2[i] = a;
            H2[i] = bf16r(fmaxf(a, 0.f));
        }
        __syncthreads();
        if (tid < TR) {                                      // layer 3 and the loss
            float a = Wt[MLP_OFF_B3];
            for (int k = 0; k < 64; ++k) a = fmaf(H2[tid * 64 + k], Wt[MLP_OFF_W3 + k], a);
            s[tid] = a;
            const float res = tid < nr ? a - y[r0 + tid] : 0.f;
            ds[tid] = 2.f * res * inv_b;
            my_loss += res * res;
        }
        __syncthreads();
        for (int i = tid; i < TR * 64; i += nt) {            // dZ2 = ds w3 relu'(Z2)
            const int r = i / 64, c = i % 64;
            dZ2[i] = Z2[i] > 0.f ? ds[r] * Wt[MLP_OFF_W3 + c] : 0.f;
        }
        __syncthreads();
        for (int i = tid; i < TR * 64; i += nt) {            // dZ1 = (dZ2 W2^T) relu'(Z1)
            const int r = i / 64, c = i % 64;
            float a = 0.f;
            for (int k = 0; k < 64; ++k) a = fmaf(dZ2[r * 64 + k], Wt[MLP_OFF_W2 + c * 64 + k], a);
            dZ1[i] = Z1[i] > 0.f ? a : 0.f;
        }
        __syncthreads();
        for (int i = tid; i < 64 * 64; i += nt) {            // dW2 = H1^T dZ2
            const int a_ = i / 64, c = i % 64;
            float acc = 0.f;
            for (int r = 0; r < nr; ++r) acc = fmaf(H1[r * 64 + a_], dZ2[r * 64 + c], acc);
            G[MLP_OFF_W2 + i] += acc;
        }
        for (int i = tid; i < 16 * 64; i += nt) {            // dW1 = X^T dZ1
            const int k = i / 64, c = i % 64;
            float acc = 0.f;
            for (int r = 0; r < nr; ++r) acc = fmaf(Xs[r * 16 + k], dZ1[r * 64 + c], acc);
            G[MLP_OFF_W1 + i] += acc;
        }
        if (tid < 64) {                                      // dw3, db2, db1
            float a3 = 0.f, a2 = 0.f, a1 = 0.f;
            for (int r = 0; r < nr; ++r) {
                a3 = fmaf(H2[r * 64 + tid], ds[r], a3);
                a2 += dZ2[r * 64 + tid];
                a1 += dZ1[r * 64 + tid];
            }
            G[MLP_OFF_W3 + tid] += a3;
            G[MLP_OFF_B2 + tid] += a2;
            G[MLP_OFF_B1 + tid] += a1;
        }
        if (tid == 64) {
            float a = 0.f;
            for (int r = 0; r < nr; ++r) a += ds[r];
            G[MLP_OFF_B3] += a;
        }
        __syncthreads();
    }
    for (int i = tid; i < MLP_PARAMS; i += nt) atomicAdd(&grad[i], G[i]);
    for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
    if ((tid & 31) == 0 && loss) atomicAdd(loss, my_loss * inv_b);
}

__global__ void mlp_adam_kernel(float *master, float *m, float *v, const float *grad, int step,
                                float lr, uint16_t *params) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_PARAMS) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)step));
    const float vh = vi / (1.f - powf(b2, (float)step));
    const float w = master[i] - lr * mh / (sqrtf(vh) + eps);
    master[i] = w;
    if (params) {
        __nv_bfloat16 h = __float2bfloat16_rn(w);
        params[i] = *reinterpret_cast<uint16_t *>(&h);
    }
}

cudaError_t mlp_pack(const uint16_t *params, uint32_t *packed, cudaStream_t st) {
    mlp_pack_kernel<<<(PK_WORDS + 255) / 256, 256, 0, st>>>(params, packed);
    return cudaGetLastError();
}

}  // namespace cubics

using namespace cubics;

static int cstat(cudaError_t e) {
    if (e == cudaSuccess) return CSP_OK;
    cudaGetLastError();
    return CSP_ECUDA;
}

extern "C" {

int csp_mlp_pack(const uint16_t *params_dev, uint32_t *packed_dev, void *cuda_stream) {
    if (!params_dev || !packed_dev) return CSP_EINVAL;
    return cstat(mlp_pack(params_dev, packed_dev, (cudaStream_t)cuda_stream));
}

int csp_mlp_forward(const uint32_t *packed_dev, const float *X_dev, int32_t rows, float *scores_dev,
                    void *cuda_stream) {
    if (!packed_dev || rows < 0 || (rows > 0 && (!X_dev || !scores_dev))) return CSP_EINVAL;
    if (rows == 0) return CSP_OK;
    const int tiles = (rows + 15) / 16;
    const int blocks = (tiles + 7) / 8;
    mlp_forward_kernel<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(packed_dev, X_dev, rows, scores_dev);
    return cstat(cudaGetLastError());
}

int csp_mlp_grad(const float *master_dev, const float *X_dev, const float *y_dev, int32_t rows,
                 float *grad_dev, float *loss_dev, void *cuda_stream) {
    if (!master_dev || !grad_dev || rows < 1 || !X_dev || !y_dev) return CSP_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t smem = (size_t)(2 * MLP_PARAMS + TR * 16 + 6 * TR * 64 + 2 * TR) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(grad_dev, 0, MLP_PARAMS * sizeof(float), st);
    if (e == cudaSuccess && loss_dev) e = cudaMemsetAsync(loss_dev, 0, sizeof(float), st);
    if (e != cudaSuccess) return cstat(e);
    const int blocks = std::min(304, (rows + TR - 1) / TR);
    mlp_grad_kernel<<<blocks, 256, smem, st>>>(master_dev, X_dev, y_dev, rows, grad_dev, loss_dev);
    return cstat(cudaGetLastError());
}

int csp_mlp_adam(float *master_dev, float *m_dev, float *v_dev, const float *grad_dev, int32_t step,
                 float lr, uint16_t *params_dev, void *cuda_stream) {
    if (!master_dev || !m_dev || !v_dev || !grad_dev || step < 1) return CSP_EINVAL;
    mlp_adam_kernel<<<(MLP_PARAMS + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(
        master_dev, m_dev, v_dev, grad_dev, step, lr, params_dev);
    return cstat(cudaGetLastError());
}

}  // extern "C"
