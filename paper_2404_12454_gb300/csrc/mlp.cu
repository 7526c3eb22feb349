// MLP surrogate of the parameter search: (OF, WR, log2 N) standardised -> 128 -> 128 ->
// 128 -> 128 -> 1 (predicted log10 Airy score), exact GELU, BF16 weights with FP32
// activations and accumulation, FP32 master weights updated by Adam.  Not in the paper:
// it learns the sweep's scores so that the search verifies only promising parameter sets.
//
// Parameter layout (floats, GBD_MLP_PARAMS = 50,177): W1[128][3] b1[128] W2[128][128] b2
// W3 b3 W4 b4 W5[1][128] b5[1]; the BF16 copy has the same layout.  A training batch of
// ~1000 samples is 1000 x 128 x 128 per layer: far too small for the tensor cores to
// matter, so the step is shaped for latency on the FP32 pipe: few samples per CTA (enough
// CTAs to cover the SMs), all three hidden-layer weight matrices staged in shared memory
// once per CTA, the activations and GELU derivatives stored by the forward pass (the
// weight gradients never recompute GELU), the weight gradients split over sample chunks
// and the chunks summed in chunk order by the optimizer.  Every reduction runs in a fixed
// order, so training is deterministic.
#include <cuda_bf16.h>
#include <math.h>

#include "gbd_internal.cuh"

namespace {

constexpr int H = 128;
// offsets of the weight matrix and bias of layer l (0-based) in the parameter vector
__host__ __device__ constexpr int off_w(int l) {
    return l == 0 ? 0 : l == 1 ? 512 : l == 2 ? 17024 : l == 3 ? 33536 : 50048;
}
__host__ __device__ constexpr int off_b(int l) {
    return l == 0 ? 384 : l == 1 ? 16896 : l == 2 ? 33408 : l == 3 ? 49920 : 50176;
}
constexpr int NPARAM = 50177;
constexpr int PART = NPARAM + 1;  // one chunk's gradient partial plus its squared-error sum
constexpr int MAX_CHUNKS = 16;
constexpr int CHUNK_MIN = 128;  // samples per chunk below which no further chunk is made
constexpr int WPAD = H + 8;     // forward weight rows padded to 272 B (conflict-free rows)

__device__ __forceinline__ float bf(uint16_t w) { return __uint_as_float((uint32_t)w << 16); }
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float gelu(float x) {
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
           x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Number of sample chunks the weight gradients are split into, and their length.
__host__ __device__ inline int n_chunks(int B) {
    const int c = (B + CHUNK_MIN - 1) / CHUNK_MIN;
    return c < MAX_CHUNKS ? c : MAX_CHUNKS;
}
__host__ __device__ inline int chunk_len(int B) {
    const int c = n_chunks(B);
    return (B + c - 1) / c;
}

template <int TB>
constexpr size_t fwd_smem() {
    return sizeof(uint16_t) * 3 * H * WPAD + sizeof(float) * 2 * TB * H;
}
template <int TB>
constexpr size_t bwd_smem() {
    return sizeof(uint16_t) * 3 * H * H + sizeof(float) * 2 * TB * H + sizeof(float) * TB;
}

// Asynchronous global -> shared copies (cp.async): every copy of a CTA is in flight at
// once, and the CTA waits for all of them with one cp.async.wait_all + __syncthreads.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Start copying the three 128 x 128 hidden-layer matrices (W2, W3, W4) into shared memory
// with a row stride of `stride` elements (16-byte pieces, the whole CTA).
__device__ __forceinline__ void stage_hidden_weights(const uint16_t* __restrict__ W, uint16_t* ws,
                                                     int stride) {
    constexpr int PER_MAT = H * H / 8;  // 16-byte pieces per matrix
    for (int e = threadIdx.x; e < 3 * PER_MAT; e += blockDim.x) {
        const int l = e / PER_MAT, r = (e % PER_MAT) / (H / 8), c = (e % (H / 8)) * 8;
        cp_async16(ws + (size_t)(l * H + r) * stride + c, W + off_w(l + 1) + r * H + c);
    }
}

// Forward pass of TB samples per CTA in G = TB / SPT groups of 128 threads: thread (g, o)
// owns hidden unit o of samples g SPT .. g SPT + SPT - 1 (the groups share the staged
// weights; more warps per SM hide the latency of the short per-sample chains).  When abuf
// is non-null (training) the activations gelu(z_l) and derivatives gelu'(z_l) of the four
// hidden layers are stored, [layer][sample][unit].
template <int TB, int SPT>
__global__ void __launch_bounds__(H * (TB / SPT)) mlp_fwd_kernel(const uint16_t* __restrict__ W,
                                                                 const float* __restrict__ x, int B,
                                                                 float* __restrict__ abuf,
                                                                 float* __restrict__ gbuf,
                                                                 float* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t* ws = reinterpret_cast<uint16_t*>(smem);
    float(*act)[TB][H] =
        reinterpret_cast<float(*)[TB][H]>(smem + sizeof(uint16_t) * 3 * H * WPAD);
    const int o = threadIdx.x & (H - 1), bs = (threadIdx.x >> 7) * SPT;
    const int b0 = blockIdx.x * TB;
    const int nb = min(TB, B - b0);
    stage_hidden_weights(W, ws, WPAD);
    {
        const float w0 = bf(W[off_w(0) + o * 3]), w1 = bf(W[off_w(0) + o * 3 + 1]),
                    w2 = bf(W[off_w(0) + o * 3 + 2]), bias = bf(W[off_b(0) + o]);
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            const int b = bs + k;
            float a = 0.f;
            if (b < nb) {
                const float* xb = x + (size_t)(b0 + b) * 3;
                const float z = fmaf(w2, xb[2], fmaf(w1, xb[1], fmaf(w0, xb[0], bias)));
                a = gelu(z);
                if (abuf) {
                    abuf[(size_t)(b0 + b) * H + o] = a;
                    gbuf[(size_t)(b0 + b) * H + o] = gelu_grad(z);
                }
            }
            act[0][b][o] = a;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    for (int l = 1; l < 4; ++l) {
        const float(*cur)[H] = act[(l - 1) & 1];
        float(*nxt)[H] = act[l & 1];
        const uint16_t* wrow = ws + (size_t)((l - 1) * H + o) * WPAD;
        float acc[SPT];
        const float bias = bf(W[off_b(l) + o]);
#pragma unroll
        for (int k = 0; k < SPT; ++k) acc[k] = bias;
#pragma unroll 4
        for (int i = 0; i < H; i += 8) {
            const uint4 wv = *reinterpret_cast<const uint4*>(wrow + i);
            const float w0 = bf_lo(wv.x), w1 = bf_hi(wv.x), w2 = bf_lo(wv.y), w3 = bf_hi(wv.y),
                        w4 = bf_lo(wv.z), w5 = bf_hi(wv.z), w6 = bf_lo(wv.w), w7 = bf_hi(wv.w);
#pragma unroll
            for (int k = 0; k < SPT; ++k) {
                const float4 a = *reinterpret_cast<const float4*>(&cur[bs + k][i]);
                const float4 c = *reinterpret_cast<const float4*>(&cur[bs + k][i + 4]);
                float s = fmaf(a.x, w0, acc[k]);
                s = fmaf(a.y, w1, s);
                s = fmaf(a.z, w2, s);
                s = fmaf(a.w, w3, s);
                s = fmaf(c.x, w4, s);
                s = fmaf(c.y, w5, s);
                s = fmaf(c.z, w6, s);
                acc[k] = fmaf(c.w, w7, s);
            }
        }
        float* al = abuf ? abuf + (size_t)l * B * H : nullptr;
        float* gl = gbuf ? gbuf + (size_t)l * B * H : nullptr;
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            const int b = bs + k;
            float a = 0.f;
            if (b < nb) {
                a = gelu(acc[k]);
                if (al) {
                    al[(size_t)(b0 + b) * H + o] = a;
                    gl[(size_t)(b0 + b) * H + o] = gelu_grad(acc[k]);
                }
            }
            nxt[b][o] = a;
        }
        __syncthreads();
    }
    // output unit: warp w takes samples w, w + warps, ...; lane k the inputs 4k .. 4k + 3
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint2 w5 = *reinterpret_cast<const uint2*>(W + off_w(4) + lane * 4);
    const float v0 = bf_lo(w5.x), v1 = bf_hi(w5.x), v2 = bf_lo(w5.y), v3 = bf_hi(w5.y);
    const float bias5 = bf(W[off_b(4)]);
    for (int b = warp; b < nb; b += (int)(blockDim.x >> 5)) {
        const float4 a = *reinterpret_cast<const float4*>(&act[1][b][lane * 4]);
        float s = fmaf(a.w, v3, fmaf(a.z, v2, fmaf(a.y, v1, a.x * v0)));
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) y[b0 + b] = s + bias5;
    }
}

// Backward pass of TB samples per CTA, grouped like the forward pass (thread (g, i) owns
// unit i of its group's samples): output error of the mean squared loss, then the error
// of every hidden layer.  dbuf[l] = dL/dz_l, dout = dL/dy.
template <int TB, int SPT>
__global__ void __launch_bounds__(H * (TB / SPT)) mlp_bwd_kernel(const uint16_t* __restrict__ W,
                                                                 const float* __restrict__ gbuf,
                                                                 const float* __restrict__ y,
                                                                 const float* __restrict__ target,
                                                                 int B, float* __restrict__ dbuf,
                                                                 float* __restrict__ dout) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t* ws = reinterpret_cast<uint16_t*>(smem);  // [3][o][i], W2..W4
    float(*dn)[TB][H] = reinterpret_cast<float(*)[TB][H]>(smem + sizeof(uint16_t) * 3 * H * H);
    float* dy = reinterpret_cast<float*>(smem + sizeof(uint16_t) * 3 * H * H +
                                         sizeof(float) * 2 * TB * H);
    const int i = threadIdx.x & (H - 1), bs = (threadIdx.x >> 7) * SPT;
    const int b0 = blockIdx.x * TB;
    const int nb = min(TB, B - b0);
    stage_hidden_weights(W, ws, H);
    if (threadIdx.x < TB) {
        const int b = threadIdx.x;
        float d = 0.f;
        if (b < nb) {
            d = 2.0f * (y[b0 + b] - target[b0 + b]) / (float)B;
            dout[b0 + b] = d;
        }
        dy[b] = d;
    }
    cp_async_wait_all();
    __syncthreads();
    {  // layer 4 (feeds the output unit)
        const float w = bf(W[off_w(4) + i]);
        const float* g = gbuf + (size_t)3 * B * H;
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            const int b = bs + k;
            float d = 0.f;
            if (b < nb) {
                d = dy[b] * w * g[(size_t)(b0 + b) * H + i];
                dbuf[(size_t)3 * B * H + (size_t)(b0 + b) * H + i] = d;
            }
            dn[0][b][i] = d;
        }
    }
    __syncthreads();
    for (int l = 2; l >= 0; --l) {
        const float(*cur)[H] = dn[(2 - l) & 1];
        float(*nxt)[H] = dn[(3 - l) & 1];
        const uint16_t* Wn = ws + (size_t)l * H * H;  // W_{l+1}[o][i]: layer l -> l + 1
        const float* g = gbuf + (size_t)l * B * H;
        float acc[SPT], gv[SPT];
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            acc[k] = 0.f;
            gv[k] = bs + k < nb ? g[(size_t)(b0 + bs + k) * H + i] : 0.f;  // in flight during the sum
        }
#pragma unroll 4
        for (int o = 0; o < H; o += 4) {
            const float w0 = bf(Wn[o * H + i]), w1 = bf(Wn[(o + 1) * H + i]),
                        w2 = bf(Wn[(o + 2) * H + i]), w3 = bf(Wn[(o + 3) * H + i]);
#pragma unroll
            for (int k = 0; k < SPT; ++k) {
                const float4 d = *reinterpret_cast<const float4*>(&cur[bs + k][o]);
                acc[k] = fmaf(d.w, w3, fmaf(d.z, w2, fmaf(d.y, w1, fmaf(d.x, w0, acc[k]))));
            }
        }
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            const int b = bs + k;
            float d = 0.f;
            if (b < nb) {
                d = acc[k] * gv[k];
                dbuf[(size_t)l * B * H + (size_t)(b0 + b) * H + i] = d;
            }
            nxt[b][i] = d;
        }
        __syncthreads();
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

// Weight and bias gradients over one chunk of samples (blockIdx.y), written to that
// chunk's partial vector part[chunk][PART] in the parameter layout (the last entry is the
// chunk's sum of squared errors).  blockIdx.x 0..11: hidden layer 2 + x / 4, output units
// 32 (x % 4) .. + 31; 12: the first layer; 13: the output unit, its bias and the loss.
// The chunk is walked in sub-chunks of CHUNK_MIN samples copied to shared memory by
// cp.async; every sum runs over the samples in order.
constexpr int WG_TILE = 32;
constexpr int WG_THREADS = 256;
constexpr int WG_TASKS = 14;
constexpr size_t kWgradSmem =
    sizeof(float) * (CHUNK_MIN * H + CHUNK_MIN * WG_TILE + CHUNK_MIN * 4);
__global__ void __launch_bounds__(WG_THREADS) mlp_wgrad_kernel(const float* __restrict__ x,
                                                               const float* __restrict__ abuf,
                                                               const float* __restrict__ dbuf,
                                                               const float* __restrict__ dout,
                                                               const float* __restrict__ y,
                                                               const float* __restrict__ target,
                                                               int B, float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem[];
    float(*at)[H] = reinterpret_cast<float(*)[H]>(smem);  // sub-chunk x 128 inputs
    float(*dt)[WG_TILE] = reinterpret_cast<float(*)[WG_TILE]>(smem + sizeof(float) * CHUNK_MIN * H);
    float* xs = reinterpret_cast<float*>(smem + sizeof(float) * (CHUNK_MIN * H + CHUNK_MIN * WG_TILE));
    __shared__ float red[WG_THREADS / 32];
    const int t = threadIdx.x, i = t & (H - 1);
    const int L = chunk_len(B);
    const int s0 = blockIdx.y * L, s1 = min(B, s0 + L);
    float* pc = part + (size_t)blockIdx.y * PART;
    const int task = blockIdx.x;
    if (task < 12) {
        // thread t: input unit i, output units o0 + jh .. o0 + jh + 15
        const int l = 1 + task / 4, o0 = (task % 4) * WG_TILE, jh = (t >> 7) * (WG_TILE / 2);
        const float* d = dbuf + (size_t)l * B * H;
        const float* a = abuf + (size_t)(l - 1) * B * H;
        float acc[WG_TILE / 2];
#pragma unroll
        for (int j = 0; j < WG_TILE / 2; ++j) acc[j] = 0.f;
        float bacc = 0.f;
        for (int s = s0; s < s1; s += CHUNK_MIN) {
            const int n = min(CHUNK_MIN, s1 - s);
            __syncthreads();  // the previous sub-chunk is consumed
            for (int e = t; e < n * (H / 4); e += WG_THREADS)
                cp_async16(&at[e / (H / 4)][(e % (H / 4)) * 4], a + (size_t)(s + e / (H / 4)) * H + (e % (H / 4)) * 4);
            for (int e = t; e < n * (WG_TILE / 4); e += WG_THREADS)
                cp_async16(&dt[e / (WG_TILE / 4)][(e % (WG_TILE / 4)) * 4],
                           d + (size_t)(s + e / (WG_TILE / 4)) * H + o0 + (e % (WG_TILE / 4)) * 4);
            cp_async_wait_all();
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < n; ++k) {
                const float ak = at[k][i];
#pragma unroll
                for (int j = 0; j < WG_TILE / 2; j += 4) {
                    const float4 dk = *reinterpret_cast<const float4*>(&dt[k][jh + j]);
                    acc[j] = fmaf(dk.x, ak, acc[j]);
                    acc[j + 1] = fmaf(dk.y, ak, acc[j + 1]);
                    acc[j + 2] = fmaf(dk.z, ak, acc[j + 2]);
                    acc[j + 3] = fmaf(dk.w, ak, acc[j + 3]);
                }
                if (t < WG_TILE) bacc += dt[k][t];
            }
        }
#pragma unroll
        for (int j = 0; j < WG_TILE / 2; ++j) pc[off_w(l) + (o0 + jh + j) * H + i] = acc[j];
        if (t < WG_TILE) pc[off_b(l) + o0 + t] = bacc;
        return;
    }
    if (task == 12) {  // first layer: unit i, inputs x; threads 128..255 only copy
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, gb = 0.f;
        for (int s = s0; s < s1; s += CHUNK_MIN) {
            const int n = min(CHUNK_MIN, s1 - s);
            __syncthreads();
            for (int e = t; e < n * (H / 4); e += WG_THREADS)
                cp_async16(&at[e / (H / 4)][(e % (H / 4)) * 4], dbuf + (size_t)(s + e / (H / 4)) * H + (e % (H / 4)) * 4);
            for (int e = t; e < n * 3; e += WG_THREADS) cp_async4(xs + e, x + (size_t)s * 3 + e);
            cp_async_wait_all();
            __syncthreads();
            if (t < H) {
#pragma unroll 4
                for (int k = 0; k < n; ++k) {
                    const float dk = at[k][i];
                    g0 = fmaf(dk, xs[3 * k], g0);
                    g1 = fmaf(dk, xs[3 * k + 1], g1);
                    g2 = fmaf(dk, xs[3 * k + 2], g2);
                    gb += dk;
                }
            }
        }
        if (t < H) {
            pc[off_w(0) + i * 3] = g0;
            pc[off_w(0) + i * 3 + 1] = g1;
            pc[off_w(0) + i * 3 + 2] = g2;
            pc[off_b(0) + i] = gb;
        }
        return;
    }
    // output unit (input i), its bias and the chunk's squared error
    const float* a3 = abuf + (size_t)3 * B * H;
    float g5 = 0.f;
    for (int s = s0; s < s1; s += CHUNK_MIN) {
        const int n = min(CHUNK_MIN, s1 - s);
        __syncthreads();
        for (int e = t; e < n * (H / 4); e += WG_THREADS)
            cp_async16(&at[e / (H / 4)][(e % (H / 4)) * 4], a3 + (size_t)(s + e / (H / 4)) * H + (e % (H / 4)) * 4);
        for (int e = t; e < n; e += WG_THREADS) cp_async4(xs + e, dout + s + e);
        cp_async_wait_all();
        __syncthreads();
        if (t < H) {
#pragma unroll 4
            for (int k = 0; k < n; ++k) g5 = fmaf(xs[k], at[k][i], g5);
        }
    }
    if (t < H) pc[off_w(4) + i] = g5;
    float sd = 0.f, l2 = 0.f;
    for (int b = s0 + t; b < s1; b += WG_THREADS) {
        sd += dout[b];
        const float e = y[b] - target[b];
        l2 = fmaf(e, e, l2);
    }
    sd = block_sum(sd, red);
    l2 = block_sum(l2, red);
    if (t == 0) {
        pc[off_b(4)] = sd;
        pc[NPARAM] = l2;
    }
}

// Sum of the chunk partials in chunk order.
__device__ __forceinline__ float chunk_sum(const float* __restrict__ part, int chunks, int k) {
    float g = part[k];
    for (int c = 1; c < chunks; ++c) g += part[(size_t)c * PART + k];
    return g;
}

__global__ void __launch_bounds__(256) mlp_reduce_kernel(const float* __restrict__ part, int chunks,
                                                         int B, float* __restrict__ grad,
                                                         float* __restrict__ loss) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NPARAM) grad[k] = chunk_sum(part, chunks, k);
    else if (k == NPARAM && loss) *loss = chunk_sum(part, chunks, k) / (float)B;
}

// Adam (Kingma & Ba) with bias correction on the FP32 master weights; writes the BF16
// copy (round to nearest even).  The gradient is the chunk-ordered sum of `chunks` rows
// of `stride` floats (one row: a plain gradient vector); with a loss pointer the entry
// after the parameters is summed too and divided by B.
__global__ void __launch_bounds__(256) mlp_adam_kernel(float* __restrict__ p, uint16_t* __restrict__ w,
                                                       float* __restrict__ m, float* __restrict__ v,
                                                       const float* __restrict__ g, int chunks,
                                                       float lr, float beta1, float beta2, float eps,
                                                       float c1, float c2, int B,
                                                       float* __restrict__ loss) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == NPARAM && loss) *loss = chunk_sum(g, chunks, k) / (float)B;
    if (k >= NPARAM) return;
    const float gk = chunks == 1 ? g[k] : chunk_sum(g, chunks, k);
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

// Samples per forward/backward CTA: 8 while that leaves SMs idle, else 32 (fewer
// re-stagings of the weights per sample); either way four groups of 128 threads.
constexpr int kSmallTB = 8, kLargeTB = 32, kGroups = 4;
constexpr int kSmallSPT = kSmallTB / kGroups, kLargeSPT = kLargeTB / kGroups;
bool use_large_tb(int B) { return B >= 152 * kLargeTB; }

cudaError_t set_smem_attrs() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* fn, size_t bytes) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void*)mlp_fwd_kernel<kSmallTB, kSmallSPT>, fwd_smem<kSmallTB>());
    set((const void*)mlp_fwd_kernel<kLargeTB, kLargeSPT>, fwd_smem<kLargeTB>());
    set((const void*)mlp_bwd_kernel<kSmallTB, kSmallSPT>, bwd_smem<kSmallTB>());
    set((const void*)mlp_bwd_kernel<kLargeTB, kLargeSPT>, bwd_smem<kLargeTB>());
    set((const void*)mlp_wgrad_kernel, kWgradSmem);
    return e;
}

void launch_forward(const uint16_t* W, const float* x, int B, float* abuf, float* gbuf, float* y,
                    cudaStream_t s) {
    if (use_large_tb(B))
        mlp_fwd_kernel<kLargeTB, kLargeSPT><<<(B + kLargeTB - 1) / kLargeTB, H * kGroups,
                                              fwd_smem<kLargeTB>(), s>>>(W, x, B, abuf, gbuf, y);
    else
        mlp_fwd_kernel<kSmallTB, kSmallSPT><<<(B + kSmallTB - 1) / kSmallTB, H * kGroups,
                                              fwd_smem<kSmallTB>(), s>>>(W, x, B, abuf, gbuf, y);
}

struct TrainBuffers {
    float *abuf, *gbuf, *dbuf, *y, *dout, *part;
};

TrainBuffers carve(void* workspace, int B) {
    char* w = static_cast<char*>(workspace);
    const size_t act = align256((size_t)4 * B * H * sizeof(float));
    const size_t vec = align256((size_t)B * sizeof(float));
    TrainBuffers t;
    t.abuf = reinterpret_cast<float*>(w);
    t.gbuf = reinterpret_cast<float*>(w + act);
    t.dbuf = reinterpret_cast<float*>(w + 2 * act);
    t.y = reinterpret_cast<float*>(w + 3 * act);
    t.dout = reinterpret_cast<float*>(w + 3 * act + vec);
    t.part = reinterpret_cast<float*>(w + 3 * act + 2 * vec);
    return t;
}

// Forward, backward and weight-gradient launches of one step; the gradient is left as
// chunk partials in t.part.
void launch_gradient(const uint16_t* W, const float* x, const float* target, int B,
                     const TrainBuffers& t, cudaStream_t s) {
    launch_forward(W, x, B, t.abuf, t.gbuf, t.y, s);
    if (use_large_tb(B))
        mlp_bwd_kernel<kLargeTB, kLargeSPT><<<(B + kLargeTB - 1) / kLargeTB, H * kGroups,
                                              bwd_smem<kLargeTB>(), s>>>(W, t.gbuf, t.y, target, B,
                                                                         t.dbuf, t.dout);
    else
        mlp_bwd_kernel<kSmallTB, kSmallSPT><<<(B + kSmallTB - 1) / kSmallTB, H * kGroups,
                                              bwd_smem<kSmallTB>(), s>>>(W, t.gbuf, t.y, target, B,
                                                                         t.dbuf, t.dout);
    mlp_wgrad_kernel<<<dim3(WG_TASKS, n_chunks(B)), WG_THREADS, kWgradSmem, s>>>(
        x, t.abuf, t.dbuf, t.dout, t.y, target, B, t.part);
}

gbd_status check_adam(float lr, float beta1, float beta2, float eps, int32_t step) {
    if (step < 1) return gbd_set_error(GBD_EINVAL, "step counts from 1");
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return gbd_set_error(GBD_EINVAL, "bad Adam hyper-parameters");
    return GBD_OK;
}

gbd_status check_train(const uint16_t* weights, const float* x, const float* target,
                       int32_t batch, void* workspace, size_t bytes) {
    if (!weights || !x || !target || !workspace) return gbd_set_error(GBD_EINVAL, "NULL buffer");
    if (batch < 1 || batch > (1 << 20)) return gbd_set_error(GBD_EINVAL, "batch out of range");
    if (reinterpret_cast<uintptr_t>(weights) & 15u)
        return gbd_set_error(GBD_EINVAL, "weights must be 16-byte aligned");
    if (bytes < gbd_mlp_workspace_bytes(batch)) return gbd_set_error(GBD_ENOMEM, "workspace too small");
    if (reinterpret_cast<uintptr_t>(workspace) & 255u)
        return gbd_set_error(GBD_EINVAL, "workspace must be 256-byte aligned");
    return GBD_OK;
}

void launch_adam(float* master, uint16_t* weights, float* m, float* v, const float* g, int chunks,
                 float lr, float beta1, float beta2, float eps, int32_t step, int B, float* loss,
                 cudaStream_t s) {
    // bias corrections in double: for beta2 = 0.999 the FP32 power loses digits by 1e4 steps
    const float c1 = (float)(1.0 - pow((double)beta1, (double)step)),
                c2 = (float)(1.0 - pow((double)beta2, (double)step));
    mlp_adam_kernel<<<(NPARAM + 1 + 255) / 256, 256, 0, s>>>(master, weights, m, v, g, chunks, lr,
                                                             beta1, beta2, eps, c1, c2, B, loss);
}

gbd_status last_error() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBD_OK : gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
}

}  // namespace

extern "C" {

size_t gbd_mlp_workspace_bytes(int32_t batch) {
    if (batch < 1) return 0;
    const size_t act = (size_t)4 * batch * H * sizeof(float);
    return 3 * align256(act) + 2 * align256((size_t)batch * sizeof(float)) +
           align256((size_t)MAX_CHUNKS * PART * sizeof(float));
}

gbd_status gbd_mlp_pack(const float* master, uint16_t* weights, void* stream) {
    if (!master || !weights) return gbd_set_error(GBD_EINVAL, "NULL parameter buffer");
    mlp_pack_kernel<<<(NPARAM + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(master,
                                                                                         weights);
    return last_error();
}

gbd_status gbd_mlp_forward(const uint16_t* weights, const float* x, int32_t batch, float* y,
                           void* stream) {
    GBD_NVTX_RANGE("gbd_mlp_forward");
    if (!weights || !x || !y) return gbd_set_error(GBD_EINVAL, "NULL buffer");
    if (batch < 1 || batch > (1 << 24)) return gbd_set_error(GBD_EINVAL, "batch out of range");
    if (reinterpret_cast<uintptr_t>(weights) & 15u)
        return gbd_set_error(GBD_EINVAL, "weights must be 16-byte aligned");
    cudaError_t e = set_smem_attrs();
    if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
    launch_forward(weights, x, batch, nullptr, nullptr, y, static_cast<cudaStream_t>(stream));
    return last_error();
}

gbd_status gbd_mlp_grad(const uint16_t* weights, const float* x, const float* target,
                        int32_t batch, float* grad, float* loss, void* workspace, size_t bytes,
                        void* stream) {
    GBD_NVTX_RANGE("gbd_mlp_grad");
    if (!grad) return gbd_set_error(GBD_EINVAL, "NULL buffer");
    gbd_status st = check_train(weights, x, target, batch, workspace, bytes);
    if (st != GBD_OK) return st;
    cudaError_t e = set_smem_attrs();
    if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const TrainBuffers t = carve(workspace, batch);
    launch_gradient(weights, x, target, batch, t, s);
    mlp_reduce_kernel<<<(NPARAM + 1 + 255) / 256, 256, 0, s>>>(t.part, n_chunks(batch), batch, grad,
                                                               loss);
    return last_error();
}

gbd_status gbd_mlp_adam(float* master, uint16_t* weights, float* m, float* v, const float* grad,
                        float lr, float beta1, float beta2, float eps, int32_t step, void* stream) {
    GBD_NVTX_RANGE("gbd_mlp_adam");
    if (!master || !weights || !m || !v || !grad) return gbd_set_error(GBD_EINVAL, "NULL buffer");
    gbd_status st = check_adam(lr, beta1, beta2, eps, step);
    if (st != GBD_OK) return st;
    launch_adam(master, weights, m, v, grad, 1, lr, beta1, beta2, eps, step, 1, nullptr,
                static_cast<cudaStream_t>(stream));
    return last_error();
}

gbd_status gbd_mlp_train(float* master, uint16_t* weights, float* m, float* v, const float* x,
                         const float* target, int32_t batch, float lr, float beta1, float beta2,
                         float eps, int32_t first_step, int32_t steps, float* loss,
                         void* workspace, size_t bytes, void* stream) {
    GBD_NVTX_RANGE("gbd_mlp_train");
    if (!master || !m || !v) return gbd_set_error(GBD_EINVAL, "NULL buffer");
    if (steps < 0 || first_step > INT32_MAX - steps)
        return gbd_set_error(GBD_EINVAL, "step count out of range");
    gbd_status st = check_train(weights, x, target, batch, workspace, bytes);
    if (st == GBD_OK) st = check_adam(lr, beta1, beta2, eps, first_step);
    if (st != GBD_OK) return st;
    cudaError_t e = set_smem_attrs();
    if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const TrainBuffers t = carve(workspace, batch);
    for (int32_t k = 0; k < steps; ++k) {
        launch_gradient(weights, x, target, batch, t, s);
        launch_adam(master, weights, m, v, t.part, n_chunks(batch), lr, beta1, beta2, eps,
                    first_step + k, batch, k + 1 == steps ? loss : nullptr, s);
    }
    return last_error();
}

gbd_status gbd_mlp_train_step(float* master, uint16_t* weights, float* m, float* v,
                              const float* x, const float* target, int32_t batch, float lr,
                              float beta1, float beta2, float eps, int32_t step, float* loss,
                              void* workspace, size_t bytes, void* stream) {
    return gbd_mlp_train(master, weights, m, v, x, target, batch, lr, beta1, beta2, eps, step, 1,
                         loss, workspace, bytes, stream);
}

}  // extern "C"
