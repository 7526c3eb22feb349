// MLP surrogate of the parameter search: (OF, WR, log2 N) standardised -> 128 -> 128 ->
// 128 -> 128 -> 1 (predicted log10 Airy score), exact GELU, BF16 weights with FP32
// activations and accumulation, FP32 master weights updated by Adam.  Not in the paper:
// it learns the sweep's scores so that the search verifies only promising parameter sets.
//
// Parameter layout (floats, GBD_MLP_PARAMS = 50,177): W1[128][3] b1[128] W2[128][128] b2
// W3 b3 W4 b4 W5[1][128] b5[1]; the BF16 copy has the same layout.  The contractions are
// 32-sample x 128 x 128 per CTA: small enough that the step is bound by launch latency, so
// they run on the FP32 pipe with the layer's weights staged in shared memory.  Every
// reduction runs in a fixed order, so training is deterministic.
#include <cuda_bf16.h>
#include <math.h>

#include "gbd_internal.cuh"

namespace {

constexpr int H = 128;
constexpr int TB = 32;  // samples per CTA
// offsets of the weight matrix and bias of layer l (0-based) in the parameter vector
__host__ __device__ constexpr int off_w(int l) {
    return l == 0 ? 0 : l == 1 ? 512 : l == 2 ? 17024 : l == 3 ? 33536 : 50048;
}
__host__ __device__ constexpr int off_b(int l) {
    return l == 0 ? 384 : l == 1 ? 16896 : l == 2 ? 33408 : l == 3 ? 49920 : 50176;
}
constexpr int NPARAM = 50177;

__device__ __forceinline__ float bf(uint16_t w) { return __uint_as_float((uint32_t)w << 16); }
__device__ __forceinline__ float gelu(float x) {
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
           x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Forward pass of TB samples per CTA; thread o owns hidden unit o.  z (pre-activations
// of the four hidden layers) is stored for the backward pass when zbuf is non-null.
constexpr int WPAD = H + 2;  // padded row of the transposed weight tile (no bank conflicts)
constexpr size_t kFwdSmem = sizeof(float) * TB * H + sizeof(uint16_t) * H * WPAD;
constexpr size_t kBwdSmem = sizeof(float) * TB * H + sizeof(uint16_t) * H * H + sizeof(float) * TB;

__global__ void __launch_bounds__(H) mlp_fwd_kernel(const uint16_t* __restrict__ W,
                                                    const float* __restrict__ x, int B,
                                                    float* __restrict__ zbuf, float* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    float(*act)[H] = reinterpret_cast<float(*)[H]>(smem);
    uint16_t(*wt)[WPAD] = reinterpret_cast<uint16_t(*)[WPAD]>(smem + sizeof(float) * TB * H);
    const int o = threadIdx.x, b0 = blockIdx.x * TB;
    const int nb = min(TB, B - b0);
    {
        const float w0 = bf(W[off_w(0) + o * 3]), w1 = bf(W[off_w(0) + o * 3 + 1]),
                    w2 = bf(W[off_w(0) + o * 3 + 2]), bias = bf(W[off_b(0) + o]);
        for (int b = 0; b < TB; ++b) {
            float z = 0.f;
            if (b < nb) {
                const float* xb = x + (size_t)(b0 + b) * 3;
                z = fmaf(w2, xb[2], fmaf(w1, xb[1], fmaf(w0, xb[0], bias)));
                if (zbuf) zbuf[(size_t)(b0 + b) * H + o] = z;
            }
            act[b][o] = b < nb ? gelu(z) : 0.f;
        }
    }
    for (int l = 1; l < 4; ++l) {
        __syncthreads();
        const uint16_t* Wl = W + off_w(l);
        for (int e = o; e < H * H; e += H) wt[e % H][e / H] = Wl[e];  // Wl[row][col] -> wt[col][row]
        __syncthreads();
        float acc[TB];
        const float bias = bf(W[off_b(l) + o]);
#pragma unroll
        for (int b = 0; b < TB; ++b) acc[b] = bias;
        for (int i = 0; i < H; i += 4) {
            const float w0 = bf(wt[i][o]), w1 = bf(wt[i + 1][o]), w2 = bf(wt[i + 2][o]),
                        w3 = bf(wt[i + 3][o]);
#pragma unroll
            for (int b = 0; b < TB; ++b) {
                const float4 a = *reinterpret_cast<const float4*>(&act[b][i]);
                acc[b] = fmaf(a.w, w3, fmaf(a.z, w2, fmaf(a.y, w1, fmaf(a.x, w0, acc[b]))));
            }
        }
        __syncthreads();
        float* zl = zbuf ? zbuf + (size_t)l * B * H : nullptr;
#pragma unroll
        for (int b = 0; b < TB; ++b) {
            if (b < nb && zl) zl[(size_t)(b0 + b) * H + o] = acc[b];
            act[b][o] = b < nb ? gelu(acc[b]) : 0.f;
        }
    }
    __syncthreads();
    if (o < nb) {
        float s = bf(W[off_b(4)]);
        for (int i = 0; i < H; ++i) s = fmaf(bf(W[off_w(4) + i]), act[o][i], s);
        y[b0 + o] = s;
    }
}

// Backward pass of TB samples per CTA: output error of the mean squared loss, then the
// error of every hidden layer (thread i owns unit i).  dbuf[l] = dL/dz_l, dout = dL/dy.
__global__ void __launch_bounds__(H) mlp_bwd_kernel(const uint16_t* __restrict__ W,
                                                    const float* __restrict__ zbuf,
                                                    const float* __restrict__ y,
                                                    const float* __restrict__ target, int B,
                                                    float* __restrict__ dbuf,
                                                    float* __restrict__ dout) {
    extern __shared__ __align__(16) unsigned char smem[];
    float(*dn)[H] = reinterpret_cast<float(*)[H]>(smem);  // error of the layer above
    uint16_t(*ws)[H] = reinterpret_cast<uint16_t(*)[H]>(smem + sizeof(float) * TB * H);  // [o][i]
    float* dy = reinterpret_cast<float*>(smem + sizeof(float) * TB * H + sizeof(uint16_t) * H * H);
    const int i = threadIdx.x, b0 = blockIdx.x * TB;
    const int nb = min(TB, B - b0);
    if (i < TB) {
        float d = 0.f;
        if (i < nb) d = 2.0f * (y[b0 + i] - target[b0 + i]) / (float)B;
        dy[i] = d;
        if (i < nb) dout[b0 + i] = d;
    }
    __syncthreads();
    // layer 4 (feeds the output unit)
    {
        const float w = bf(W[off_w(4) + i]);
        const float* z = zbuf + (size_t)3 * B * H;
        for (int b = 0; b < TB; ++b) {
            float d = 0.f;
            if (b < nb) {
                d = dy[b] * w * gelu_grad(z[(size_t)(b0 + b) * H + i]);
                dbuf[(size_t)3 * B * H + (size_t)(b0 + b) * H + i] = d;
            }
            dn[b][i] = d;
        }
    }
    for (int l = 2; l >= 0; --l) {
        __syncthreads();
        const uint16_t* Wn = W + off_w(l + 1);  // weights from layer l to layer l+1
        for (int e = i; e < H * H; e += H) ws[e / H][e % H] = Wn[e];
        __syncthreads();
        float acc[TB];
#pragma unroll
        for (int b = 0; b < TB; ++b) acc[b] = 0.f;
        for (int o = 0; o < H; o += 4) {
            const float w0 = bf(ws[o][i]), w1 = bf(ws[o + 1][i]), w2 = bf(ws[o + 2][i]),
                        w3 = bf(ws[o + 3][i]);
#pragma unroll
            for (int b = 0; b < TB; ++b) {
                const float4 d = *reinterpret_cast<const float4*>(&dn[b][o]);
                acc[b] = fmaf(d.w, w3, fmaf(d.z, w2, fmaf(d.y, w1, fmaf(d.x, w0, acc[b]))));
            }
        }
        __syncthreads();
        const float* z = zbuf + (size_t)l * B * H;
#pragma unroll
        for (int b = 0; b < TB; ++b) {
            float d = 0.f;
            if (b < nb) {
                d = acc[b] * gelu_grad(z[(size_t)(b0 + b) * H + i]);
                dbuf[(size_t)l * B * H + (size_t)(b0 + b) * H + i] = d;
            }
            dn[b][i] = d;
        }
    }
}

// Deterministic sum over the block's threads (fixed tree).
__device__ float block_sum(float v, float* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
}

// Weight and bias gradients: CTA (layer, o) sums over the batch in sample order.
// blockIdx.x: 0..127 layer 1, 128..511 layers 2-4, 512 output layer (also the loss).
__global__ void __launch_bounds__(H) mlp_wgrad_kernel(const float* __restrict__ x,
                                                      const float* __restrict__ zbuf,
                                                      const float* __restrict__ dbuf,
                                                      const float* __restrict__ dout,
                                                      const float* __restrict__ y,
                                                      const float* __restrict__ target, int B,
                                                      float* __restrict__ grad,
                                                      float* __restrict__ loss) {
    __shared__ float red[H / 32];
    const int i = threadIdx.x;
    const int blk = blockIdx.x;
    if (blk < 128) {  // layer 1: inputs x (3 features)
        const int o = blk;
        const float* d = dbuf;  // layer-1 error
        if (i < 3) {
            float g = 0.f;
            for (int b = 0; b < B; ++b) g = fmaf(d[(size_t)b * H + o], x[(size_t)b * 3 + i], g);
            grad[off_w(0) + o * 3 + i] = g;
        }
        float s = 0.f;
        for (int b = i; b < B; b += H) s += d[(size_t)b * H + o];
        s = block_sum(s, red);
        if (i == 0) grad[off_b(0) + o] = s;
    } else if (blk < 512) {  // layers 2..4: inputs gelu(z_{l-1})
        const int l = 1 + (blk - 128) / H, o = (blk - 128) % H;
        const float* d = dbuf + (size_t)l * B * H;
        const float* zp = zbuf + (size_t)(l - 1) * B * H;
        float g = 0.f;
        for (int b = 0; b < B; ++b) g = fmaf(d[(size_t)b * H + o], gelu(zp[(size_t)b * H + i]), g);
        grad[off_w(l) + o * H + i] = g;
        float s = 0.f;
        for (int b = i; b < B; b += H) s += d[(size_t)b * H + o];
        s = block_sum(s, red);
        if (i == 0) grad[off_b(l) + o] = s;
    } else {  // output unit: inputs gelu(z_4); and the loss
        const float* zp = zbuf + (size_t)3 * B * H;
        float g = 0.f;
        for (int b = 0; b < B; ++b) g = fmaf(dout[b], gelu(zp[(size_t)b * H + i]), g);
        grad[off_w(4) + i] = g;
        float s = 0.f, l2 = 0.f;
        for (int b = i; b < B; b += H) {
            s += dout[b];
            const float e = y[b] - target[b];
            l2 = fmaf(e, e, l2);
        }
        s = block_sum(s, red);
        l2 = block_sum(l2, red);
        if (i == 0) {
            grad[off_b(4)] = s;
            if (loss) *loss = l2 / (float)B;
        }
    }
}

// Adam (Kingma & Ba) with bias correction on the FP32 master weights; writes the BF16
// copy (round to nearest even).
__global__ void __launch_bounds__(256) mlp_adam_kernel(float* __restrict__ p, uint16_t* __restrict__ w,
                                                       float* __restrict__ m, float* __restrict__ v,
                                                       const float* __restrict__ g, float lr,
                                                       float beta1, float beta2, float eps,
                                                       float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    const float gk = g[k];
    const float mk = beta1 * m[k] + (1.0f - beta1) * gk;
    const float vk = beta2 * v[k] + (1.0f - beta2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    p[k] = pk;
    w[k] = __bfloat16_as_ushort(__float2bfloat16_rn(pk));
}

__global__ void __launch_bounds__(256) mlp_pack_kernel(const float* __restrict__ p,
                                                       uint16_t* __restrict__ w) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NPARAM) w[k] = __bfloat16_as_ushort(__float2bfloat16_rn(p[k]));
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

cudaError_t set_smem_attrs() {
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFwdSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kBwdSmem);
    return e;
}

}  // namespace

extern "C" {

size_t gbd_mlp_workspace_bytes(int32_t batch) {
    if (batch < 1) return 0;
    const size_t act = (size_t)4 * batch * H * sizeof(float);
    return 2 * align256(act) + 2 * align256((size_t)batch * sizeof(float)) +
           align256((size_t)NPARAM * sizeof(float));
}

gbd_status gbd_mlp_pack(const float* master, uint16_t* weights, void* stream) {
    if (!master || !weights) return gbd_set_error(GBD_EINVAL, "NULL parameter buffer");
    mlp_pack_kernel<<<(NPARAM + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(master,
                                                                                         weights);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBD_OK : gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
}

gbd_status gbd_mlp_forward(const uint16_t* weights, const float* x, int32_t batch, float* y,
                           void* stream) {
    if (!weights || !x || !y) return gbd_set_error(GBD_EINVAL, "NULL buffer");
    if (batch < 1 || batch > (1 << 24)) return gbd_set_error(GBD_EINVAL, "batch out of range");
    cudaError_t e = set_smem_attrs();
    if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
    mlp_fwd_kernel<<<(batch + TB - 1) / TB, H, kFwdSmem, static_cast<cudaStream_t>(stream)>>>(
        weights, x, batch, nullptr, y);
    e = cudaGetLastError();
    return e == cudaSuccess ? GBD_OK : gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
}

gbd_status gbd_mlp_grad(const uint16_t* weights, const float* x, const float* target,
                        int32_t batch, float* grad, float* loss, void* workspace, size_t bytes,
                        void* stream) {
    if (!weights || !x || !target || !grad || !workspace)
        return gbd_set_error(GBD_EINVAL, "NULL buffer");
    if (batch < 1 || batch > (1 << 20)) return gbd_set_error(GBD_EINVAL, "batch out of range");
    if (bytes < gbd_mlp_workspace_bytes(batch)) return gbd_set_error(GBD_ENOMEM, "workspace too small");
    if (reinterpret_cast<uintptr_t>(workspace) & 255u)
        return gbd_set_error(GBD_EINVAL, "workspace must be 256-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(workspace);
    const size_t act = align256((size_t)4 * batch * H * sizeof(float));
    float* zbuf = reinterpret_cast<float*>(w);
    float* dbuf = reinterpret_cast<float*>(w + act);
    float* y = reinterpret_cast<float*>(w + 2 * act);
    float* dout = reinterpret_cast<float*>(w + 2 * act + align256((size_t)batch * sizeof(float)));
    const int blocks = (batch + TB - 1) / TB;
    cudaError_t e = set_smem_attrs();
    if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
    mlp_fwd_kernel<<<blocks, H, kFwdSmem, s>>>(weights, x, batch, zbuf, y);
    mlp_bwd_kernel<<<blocks, H, kBwdSmem, s>>>(weights, zbuf, y, target, batch, dbuf, dout);
    mlp_wgrad_kernel<<<513, H, 0, s>>>(x, zbuf, dbuf, dout, y, target, batch, grad, loss);
    e = cudaGetLastError();
    return e == cudaSuccess ? GBD_OK : gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
}

gbd_status gbd_mlp_adam(float* master, uint16_t* weights, float* m, float* v, const float* grad,
                        float lr, float beta1, float beta2, float eps, int32_t step, void* stream) {
    if (!master || !weights || !m || !v || !grad) return gbd_set_error(GBD_EINVAL, "NULL buffer");
    if (step < 1) return gbd_set_error(GBD_EINVAL, "step counts from 1");
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return gbd_set_error(GBD_EINVAL, "bad Adam hyper-parameters");
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    mlp_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        master, weights, m, v, grad, lr, beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBD_OK : gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
}

gbd_status gbd_mlp_train_step(float* master, uint16_t* weights, float* m, float* v,
                              const float* x, const float* target, int32_t batch, float lr,
                              float beta1, float beta2, float eps, int32_t step, float* loss,
                              void* workspace, size_t bytes, void* stream) {
    if (bytes < gbd_mlp_workspace_bytes(batch)) return gbd_set_error(GBD_ENOMEM, "workspace too small");
    const size_t act = align256((size_t)4 * batch * H * sizeof(float));
    float* grad = reinterpret_cast<float*>(static_cast<char*>(workspace) + 2 * act +
                                           2 * align256((size_t)batch * sizeof(float)));
    gbd_status st = gbd_mlp_grad(weights, x, target, batch, grad, loss, workspace, bytes, stream);
    if (st != GBD_OK) return st;
    return gbd_mlp_adam(master, weights, m, v, grad, lr, beta1, beta2, eps, step, stream);
}

}  // extern "C"
