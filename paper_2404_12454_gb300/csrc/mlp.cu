// MLP surrogate of the parameter search: (OF, WR, log2 N) standardised -> 128 -> 128 ->
// 128 -> 128 -> 1 (predicted log10 Airy score), GELU, BF16 weights with FP32 activations
// and accumulation, FP32 master weights updated by Adam.  Not in the paper: it learns the
// sweep's scores so that the search verifies only promising parameter sets.
//
// Parameter layout (floats, GBD_MLP_PARAMS = 50,177): W1[128][3] b1[128] W2[128][128] b2
// W3 b3 W4 b4 W5[1][128] b5[1]; the BF16 copy has the same layout.
//
// The three 128 x 128 layers run on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation).  The weights are BF16 already, so they enter exactly; an FP32
// operand v (activation or error) is split into BF16 parts v = hi + mid + lo (each the
// rounding of what the previous parts leave; |v - hi - mid - lo| <= 2^-27 |v|) or
// v ~ hi + lo (2^-18 |v|), and W v is the sum of one product per part:
//   forward   z_l = W_l a_{l-1}:     a in three parts (inference: FP32-accurate
//                                    activations) or two (training);
//   backward  e = W_l^T d_l:         d in two parts;
//   gradient  dW_l = sum_n d_l a_{l-1}^T: d and a in two parts each, the products
//             hi.hi + (hi.lo + lo.hi) (the dropped lo.lo is below 2^-17 relative).
// The first layer (3 inputs), the output unit and the biases stay on the FP32 pipe.  GELU's
// normal CDF is Abramowitz & Stegun's 7.1.26 (absolute error <= 1.5e-7).
//
// A training call is one persistent cooperative kernel over all its steps (512 threads,
// one CTA per SM); each step is
//   phase A (sample-parallel): the CTA stages the weight image (bulk copies; the image in
//     the workspace is kept current by Adam) and takes items of 8 samples (the mma's n):
//     forward pass (gelu'(z) kept in shared memory), output, backward pass, each 128 x 128
//     layer split over K between the two warps of a 16-unit m-tile; the activations and
//     errors the weight gradients need go to the workspace, blocked per gradient tile;
//   grid barrier;
//   phase B (parameter-parallel): 112 tasks, each owning a set of parameters and summing
//     its gradient over the whole batch in a fixed order: 96 tiles of 16 x 32 hidden
//     weights (mma over the samples, streamed 256 samples at a time by bulk copies), 8
//     first-layer and 8 output-unit tasks of 16 units (FP32 sums); each task applies Adam
//     to its parameters at once (or writes the gradient, for gbd_mlp_grad);
//   grid barrier (before the next step stages the updated weights).
// Every sum runs in an order fixed by the batch size alone (not by the grid), so training
// is deterministic.  Data written inside the kernel by other CTAs is read through L2 only
// (bulk copies after a proxy fence, ld.global.cg): L1 is not coherent across CTAs.
#include <cuda_bf16.h>
#include <math.h>

#include "gbd_internal.cuh"

__device__ unsigned int g_mlp_status = 0;

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

constexpr int NS = 8;          // samples per phase-A item (the mma's n)
constexpr int THREADS = 512;   // 16 warps: a pair per 16-unit m-tile, splitting K
constexpr int NWARP = THREADS / 32;
constexpr int WP = H + 8;      // padded BF16 row of staged weights and operand planes
constexpr int GP = H + 4;      // padded FP32 row of GELU derivatives and the last activations
constexpr int KI = 32;         // items (of NS samples) per staged block of a gradient tile
constexpr int TO = 16, TI = 32;  // weight-gradient tile: output units x input units
constexpr int kHiddenTasks = 3 * (H / TO) * (H / TI);  // 96
constexpr int kFirstTasks = H / 16;                    // W1 and b1, 16 units each
constexpr int kOutTasks = H / 16;                      // W5, 16 inputs each (+ b5, loss)
constexpr int kTasks = kHiddenTasks + kFirstTasks + kOutTasks;

// Shared memory of phase A (byte offsets).  Phase B reuses the same bytes.
constexpr size_t kOffWs = 0;                                     // [3][H][WP] bf16
constexpr size_t kOffPl = kOffWs + sizeof(uint16_t) * 3 * H * WP;  // [2][3][NS][WP] bf16
constexpr size_t kOffG = kOffPl + sizeof(uint16_t) * 2 * 3 * NS * WP;  // [4][NS][GP] f32
constexpr size_t kOffA4 = kOffG + sizeof(float) * 4 * NS * GP;  // [NS][GP] f32
constexpr size_t kOffW1 = kOffA4 + sizeof(float) * NS * GP;     // [H][3] f32
constexpr size_t kOffBias = kOffW1 + sizeof(float) * H * 3;     // [4][H] f32
constexpr size_t kOffW5 = kOffBias + sizeof(float) * 4 * H;     // [H] f32
constexpr size_t kOffMisc = kOffW5 + sizeof(float) * H;  // b5, dy[NS], x[NS][3], target[NS]
constexpr size_t kOffXch = kOffMisc + 256;  // [2 K-halves][8 m-tiles][32 lanes] float2
constexpr size_t kSmemA = kOffXch + sizeof(float2) * 2 * 8 * 32;
// The weight image in the workspace: the small parameters as FP32 in the shared-memory
// order from kOffW1 (W1, b1..b4, W5, b5, padding: one bulk copy), then W2..W4 as BF16 rows
// padded to WP (the kOffWs bytes: one bulk copy).
constexpr int kImgSmall = 3 * H + 4 * H + H + 4;  // floats
constexpr uint32_t kImgSmallBytes = sizeof(float) * kImgSmall;
constexpr uint32_t kImgBigBytes = sizeof(uint16_t) * 3 * H * WP;
constexpr size_t kImgBigOff = 4352;  // 256-aligned offset of the BF16 rows in the image
static_assert(kImgSmallBytes % 16 == 0 && kImgSmallBytes <= kImgBigOff, "image layout");
static_assert(kOffW1 % 16 == 0 && kOffMisc == kOffW1 + sizeof(float) * (3 * H + 4 * H + H),
              "the small parameters are contiguous in shared memory");
// phase B: a ring of NBUF staged blocks, each [KI][TO][NS] x 2 parts of d, [KI][TI][NS] x 2 of a
constexpr int NBUF = 4;
constexpr size_t kDBytes = sizeof(uint16_t) * KI * TO * NS;
constexpr size_t kABytes = sizeof(uint16_t) * KI * TI * NS;
constexpr size_t kStageBytes = 2 * kDBytes + 2 * kABytes;
constexpr int RP = TI + 8;  // padded row of the warps' partial tiles (conflict-free float2)
// after a task's blocks are consumed, the ring's first bytes hold the warps' partial tiles
// and the small tasks' scratch
constexpr size_t kOffRed = 0;                                           // [NWARP][TO][RP] f32
constexpr size_t kOffBsum = kOffRed + sizeof(float) * NWARP * TO * RP;  // 2048 f32 scratch
constexpr size_t kSmemB = NBUF * kStageBytes;
static_assert(kOffBsum + sizeof(float) * 2048 <= kSmemB, "phase-B scratch");
// mbarriers (weights: small parameters, W2, W3, W4; ring: NBUF) after both phases' bytes
constexpr int kWBars = 4;
constexpr size_t kOffBars = kSmemA > kSmemB ? kSmemA : kSmemB;
constexpr size_t kSmemStep = kOffBars + 8 * (kWBars + NBUF);
static_assert(kSmemStep <= 227 * 1024, "shared memory");
static_assert(kOffBars % 8 == 0 && kSmemA % 8 == 0, "mbarrier alignment");

__device__ __forceinline__ float bf2f(uint16_t w) { return __uint_as_float((uint32_t)w << 16); }
__device__ __forceinline__ uint16_t f2bf(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// gelu(x) = x Phi(x) and gelu'(x) = Phi(x) + x phi(x).  Phi(-|x|) = erfc(u) / 2, u = |x| / sqrt 2,
// by Abramowitz & Stegun 7.1.26 (Hastings' rational approximation, |error| <= 1.5e-7):
//   erfc(u) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^(-u^2),  t = 1 / (1 + p u),
// where e^(-u^2) = e^(-x^2/2) is also the normal density's exponential (one ex2, one rcp).
__device__ __forceinline__ float gelu_and_grad(float x, float& grad) {
    const float u = fabsf(x) * 0.70710678118654752f;
    const float t = rcp_approx(fmaf(0.3275911f, u, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f),
                         -0.284496736f),
                 0.254829592f);
    const float e = gbd::mufu_ex2(-0.72134752044448170f * x * x);  // e^(-x^2/2)
    const float tail = 0.5f * poly * e;                               // Phi(-|x|)
    const float cdf = x >= 0.f ? 1.0f - tail : tail;
    grad = fmaf(x * 0.39894228040143268f, e, cdf);
    return x * cdf;
}
// v = hi + mid + lo (each a BF16 rounding of the remainder; the subtractions are exact)
__device__ __forceinline__ void split3(float v, uint16_t& hi, uint16_t& mid, uint16_t& lo) {
    hi = f2bf(v);
    const float r = v - bf2f(hi);
    mid = f2bf(r);
    lo = f2bf(r - bf2f(mid));
}
__device__ __forceinline__ void split2(float v, uint16_t& hi, uint16_t& lo) {
    hi = f2bf(v);
    lo = f2bf(v - bf2f(hi));
}
__device__ __forceinline__ uint32_t pack2(uint16_t lo_k, uint16_t hi_k) {
    return (uint32_t)lo_k | ((uint32_t)hi_k << 16);
}

// Adam's bias corrections c1 = 1 - beta1^t, c2 = 1 - beta2^t: beta^t by binary powering
// in double with explicitly rounded operations (no contraction), so that every kernel
// computing them gets the same bits; one thread per CTA (the FP64 pipe is narrow).
__device__ __forceinline__ float bias_correction(float beta, int t) {
    double r = 1.0, b = (double)beta;
    while (t > 0) {
        if (t & 1) r = __dmul_rn(r, b);
        b = __dmul_rn(b, b);
        t >>= 1;
    }
    return (float)__dsub_rn(1.0, r);
}

// ---------------------------------------------------------------- PTX wrappers --
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(gbd::smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(gbd::smem_addr(p)));
}
// c += a b (m16n8k16, A row-major 16 x 16, B column-major 16 x 8, BF16, FP32 accumulate)
__device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t lds32(const uint16_t* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}
// Orders this thread's generic-proxy view of global memory (data published by other CTAs
// before a grid barrier) before its next asynchronous-proxy (bulk) copies.
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Bounded wait (every thread) for the copies signalled on `bar`; a block-uniform result.  On
// giving up it records a timeout and waits again with the default limit, so that no copy
// is left writing into shared memory when the CTA returns.
__device__ bool wait_copies(uint64_t* bar, uint32_t parity, uint32_t spins) {
    const bool ok = gbd::mbar_wait_bounded(bar, parity, spins);
    if (!__syncthreads_or(!ok)) return true;
    if (threadIdx.x == 0) atomicOr(&g_mlp_status, gbd::kStatusTimeout);
    gbd::mbar_wait_bounded(bar, parity, gbd::kDefaultWaitSpins);
    return false;
}

// ----------------------------------------------------------- kernel arguments --
// Workspace of a training call.  Items are the batch's groups of NS samples (the batch is
// padded to Bp, a multiple of 16, with zero-error samples).  The operands of the hidden
// weight gradients are stored in two BF16 parts, blocked so that a gradient tile's block
// of items is one contiguous run:
//   d part: [unit / 16][item][unit % 16][NS]    a part: [unit / 32][item][unit % 32][NS]
// a_4 and d_1 (FP32, summed on the FP32 pipe) are [item][unit][NS].
struct Planes {
    uint16_t* a[3][2];  // a_1 .. a_3 = gelu(z_1 .. z_3): hi, lo
    uint16_t* d[3][2];  // d_2 .. d_4 = dL/dz_2 .. dL/dz_4: hi, lo
    float* a4;          // gelu(z_4)
    float* d1;          // dL/dz_1
    float* y;           // [Bp] network outputs
    float* dout;        // [Bp] dL/dy
    unsigned* bar;      // grid barrier: arrival count
    float* img_small;   // weight image (see kImgSmall), kept current by Adam
    uint16_t* img_big;
};

// Element (unit u, padded sample n) of a d part, an a part and an FP32 plane.
__device__ __forceinline__ size_t d_index(int u, int n, int items) {
    return (((size_t)(u / TO) * items + (n >> 3)) * TO + u % TO) * NS + (n & 7);
}
__device__ __forceinline__ size_t a_index(int u, int n, int items) {
    return (((size_t)(u / TI) * items + (n >> 3)) * TI + u % TI) * NS + (n & 7);
}
__device__ __forceinline__ size_t f_index(int u, int n) {
    return ((size_t)(n >> 3) * H + u) * NS + (n & 7);
}

struct StepArgs {
    float* master;
    uint16_t* w;  // BF16 weights (read by phase A; rewritten by Adam)
    float* m;
    float* v;
    float* grad;  // gradient output (gbd_mlp_grad) instead of Adam
    const float* x;
    const float* target;
    float* loss;
    float lr, beta1, beta2, eps;
    int B, Bp, first_step, steps;
    uint32_t spins;
    Planes pl;
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }
__host__ __device__ inline int padded_batch(int B) { return (B + 15) / 16 * 16; }

// ----------------------------------------------------------------- grid barrier --
// Barrier over the co-resident CTAs of a cooperative launch on a monotonic arrival count
// (zeroed before the launch): barrier e (1, 2, ...) is passed once the count reaches
// e x gridDim.x.  Thread 0 publishes the CTA's writes (fence, then a relaxed add) and
// polls the count with acquire loads; after `spins` polls it records a timeout and the
// barrier returns false.
// `side`, if given, runs on thread 32 (warp 1, idle during the wait) before the block
// leaves the barrier.
template <typename Side>
__device__ bool grid_sync(unsigned* count, unsigned& epoch, uint32_t spins, Side side) {
    __shared__ int ok;
    ++epoch;
    __syncthreads();
    if (threadIdx.x == 32) side();
    if (threadIdx.x == 0) {
        const unsigned target = epoch * gridDim.x;
        asm volatile("fence.acq_rel.gpu;\n\tred.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(count)
                     : "memory");
        int good = 1;
        uint32_t it = 0;
        for (;;) {
            unsigned now;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(now) : "l"(count) : "memory");
            if ((int)(now - target) >= 0) break;
            if (++it >= spins) {
                good = 0;
                atomicOr(&g_mlp_status, gbd::kStatusTimeout);
                break;
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// ------------------------------------------------------------------- phase A --
struct SmemA {
    uint16_t* ws;   // W2..W4 [3][H][WP]
    uint16_t* pl;   // operand planes [2 buffers][3 parts][NS][WP] ([sample][unit])
    float* g;       // gelu'(z_1..z_4) [4][NS][GP]
    float* a4;      // gelu(z_4) [NS][GP]
    float* w1;      // [H][3]
    float* bias;    // b1..b4 [4][H]
    float* w5;      // [H]
    float* misc;    // [0] b5, [8..15] dL/dy, [16..39] x, [40..47] targets of the item
    float2* xch;    // K-half partial sums exchanged by the two warps of an m-tile
    __device__ explicit SmemA(unsigned char* s)
        : ws(reinterpret_cast<uint16_t*>(s + kOffWs)),
          pl(reinterpret_cast<uint16_t*>(s + kOffPl)),
          g(reinterpret_cast<float*>(s + kOffG)),
          a4(reinterpret_cast<float*>(s + kOffA4)),
          w1(reinterpret_cast<float*>(s + kOffW1)),
          bias(reinterpret_cast<float*>(s + kOffBias)),
          w5(reinterpret_cast<float*>(s + kOffW5)),
          misc(reinterpret_cast<float*>(s + kOffMisc)),
          xch(reinterpret_cast<float2*>(s + kOffXch)) {}
    __device__ uint16_t* plane(int buf, int part) const { return pl + (buf * 3 + part) * NS * WP; }
};

// Start copying the weight image into shared memory (thread 0, bulk copies): bars[0]
// signals the small parameters, bars[1 + l] the rows of W_{l+2}, so that each layer waits
// only for its own matrix.  The caller has ordered the image's latest writes before this
// (kernel start or a grid barrier).
__device__ void stage_weights(const Planes& pl, const SmemA& S, uint64_t* bars) {
    if (threadIdx.x == 0) {
        proxy_fence();
        gbd::mbar_arrive_expect_tx(bars, kImgSmallBytes);
        gbd::bulk_copy_g2s(S.w1, pl.img_small, kImgSmallBytes, bars);
        constexpr uint32_t mat = kImgBigBytes / 3;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            gbd::mbar_arrive_expect_tx(bars + 1 + l, mat);
            gbd::bulk_copy_g2s(S.ws + (size_t)l * H * WP, pl.img_big + (size_t)l * H * WP, mat,
                               bars + 1 + l);
        }
    }
}

// Gives up waiting for the weight copies from bars[from] on: drains them all (default
// limit) so that no copy is left writing into shared memory.
__device__ void drain_weights(uint64_t* bars, int from, uint32_t parity) {
    for (int b = from; b < kWBars; ++b)
        gbd::mbar_wait_bounded(bars + b, parity, gbd::kDefaultWaitSpins);
}

// Inference: the weights straight from the BF16 vector (16-byte loads), once per CTA.
__device__ void load_weights(const uint16_t* __restrict__ W, const SmemA& S) {
    constexpr int PER_ROW = H / 8, PER_MAT = H * PER_ROW;
    for (int e = threadIdx.x; e < 3 * PER_MAT; e += THREADS) {
        const int l = e / PER_MAT, r = (e % PER_MAT) / PER_ROW, c = (e % PER_ROW) * 8;
        *reinterpret_cast<uint4*>(S.ws + (size_t)(l * H + r) * WP + c) =
            __ldg(reinterpret_cast<const uint4*>(W + off_w(l + 1) + r * H + c));
    }
    for (int e = threadIdx.x; e < 3 * H; e += THREADS) S.w1[e] = bf2f(__ldg(W + off_w(0) + e));
    for (int e = threadIdx.x; e < 4 * H; e += THREADS)
        S.bias[e] = bf2f(__ldg(W + off_b(e / H) + e % H));
    for (int e = threadIdx.x; e < H; e += THREADS) S.w5[e] = bf2f(__ldg(W + off_w(4) + e));
    if (threadIdx.x == 0) S.misc[0] = bf2f(__ldg(W + off_b(4)));
}

// Half (kh) of z = W_l a for the 16 units of m-tile mt and the item's 8 samples:
// acc[p] = W_l (part p of a) over inputs 64 kh .. 64 kh + 63, p < NP; in = the input
// planes [NS][WP].
template <int NP>
__device__ __forceinline__ void fwd_mma(const uint16_t* Wl, const uint16_t* in0,
                                        const uint16_t* in1, const uint16_t* in2, int mt,
                                        int kh, int lane, float (&acc)[3][4]) {
    const int g = lane >> 2, q = lane & 3;
    const uint16_t* arow = Wl + (size_t)(16 * mt + (lane & 15)) * WP + (lane >> 4) * 8;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[p][e] = 0.f;
#pragma unroll
    for (int kk = 4 * kh; kk < 4 * kh + 4; ++kk) {
        uint32_t a[4];
        ldsm_x4(a, arow + 16 * kk);
        const int o = g * WP + 16 * kk + 2 * q;
        mma(acc[0], a, lds32(in0 + o), lds32(in0 + o + 8));
        mma(acc[1], a, lds32(in1 + o), lds32(in1 + o + 8));
        if (NP == 3) mma(acc[2], a, lds32(in2 + o), lds32(in2 + o + 8));
    }
}

// Half (kh: outputs 64 kh ..) of e = W_l^T d for the 16 input units of m-tile mt and the
// item's 8 samples (d in two parts).
__device__ __forceinline__ void bwd_mma(const uint16_t* Wl, const uint16_t* in0,
                                        const uint16_t* in1, int mt, int kh, int lane,
                                        float (&acc)[2][4]) {
    const int g = lane >> 2, q = lane & 3;
    // ldmatrix.trans of W rows o (the k index) and 8 consecutive input units (the m index)
    const uint16_t* arow =
        Wl + (size_t)(((lane >> 4) << 3) + (lane & 7)) * WP + 16 * mt + ((lane >> 3) & 1) * 8;
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[p][e] = 0.f;
#pragma unroll
    for (int kk = 4 * kh; kk < 4 * kh + 4; ++kk) {
        uint32_t a[4];
        ldsm_x4_t(a, arow + (size_t)16 * kk * WP);
        const int o = g * WP + 16 * kk + 2 * q;
        mma(acc[0], a, lds32(in0 + o), lds32(in0 + o + 8));
        mma(acc[1], a, lds32(in1 + o), lds32(in1 + o + 8));
    }
}

// The two K-halves of an m-tile's 16 x 8 result: warp kh keeps rows 8 kh .. 8 kh + 7 (its
// lane's samples 2q, 2q + 1) and receives the other warp's partial sums of them; the
// result is (half 0) + (half 1) in both warps.  Ends with the block synchronised.
__device__ __forceinline__ float2 join_halves(const SmemA& S, const float (&part)[4], int mt,
                                              int kh, int lane) {
    S.xch[(kh * 8 + mt) * 32 + lane] =
        kh == 0 ? make_float2(part[2], part[3]) : make_float2(part[0], part[1]);
    __syncthreads();
    const float2 o = S.xch[((kh ^ 1) * 8 + mt) * 32 + lane];
    return kh == 0 ? make_float2(part[0] + o.x, part[1] + o.y)
                   : make_float2(o.x + part[2], o.y + part[3]);
}

// Forward pass of one item (samples n0 .. n0 + 7 of the padded batch).  Inference splits
// the activations into three BF16 parts (FP32-accurate outputs); training into two
// (2^-18 relative, far inside the gradient's error budget) and also stores a_1..a_3 (two
// parts) and a_4 in the workspace.  Leaves gelu(z_4) in S.a4, gelu'(z_l) in
// S.g, and returns with the block synchronised.  `first`: the step's first item, which
// waits for the staged parameters (bars[0] before layer 1, bars[1] after it); false if a
// wait gave up.
template <bool TRAIN>
__device__ bool forward_item(const SmemA& S, const float* __restrict__ x,
                             const float* __restrict__ target, int B, int n0, const Planes& pl,
                             int Bp, bool first, uint64_t* bars, uint32_t parity,
                             uint32_t spins) {
    const int items = Bp / NS;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t < NS * 3) {
        const int n = t / 3;
        S.misc[16 + t] = n0 + n < B ? __ldg(x + (size_t)n0 * 3 + t) : 0.f;
    } else if (TRAIN && t < NS * 4) {
        const int n = t - NS * 3;
        S.misc[40 + n] = n0 + n < B ? __ldg(target + n0 + n) : 0.f;
    }
    if (first && !wait_copies(bars, parity, spins)) {
        drain_weights(bars, 1, parity);
        return false;
    }
    __syncthreads();
    {  // layer 1 (3 inputs): unit u, samples ns, ns + 1
        const int u = t & (H - 1), ns = (t >> 7) * 2;
        const float w0 = S.w1[u * 3], w1 = S.w1[u * 3 + 1], w2 = S.w1[u * 3 + 2], b = S.bias[u];
        uint16_t hi[2], mid[2], lo[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int n = ns + k;
            const float* xn = S.misc + 16 + 3 * n;
            const float z = fmaf(w2, xn[2], fmaf(w1, xn[1], fmaf(w0, xn[0], b)));
            float gd;
            const float a = gelu_and_grad(z, gd);
            S.g[n * GP + u] = gd;
            if (TRAIN) {
                split2(a, hi[k], mid[k]);
            } else {
                split3(a, hi[k], mid[k], lo[k]);
                S.plane(0, 2)[n * WP + u] = lo[k];
            }
            S.plane(0, 0)[n * WP + u] = hi[k];
            S.plane(0, 1)[n * WP + u] = mid[k];
        }
        if (TRAIN) {
            const size_t off = a_index(u, n0 + ns, items);
            *reinterpret_cast<uint32_t*>(pl.a[0][0] + off) = pack2(hi[0], hi[1]);
            *reinterpret_cast<uint32_t*>(pl.a[0][1] + off) = pack2(mid[0], mid[1]);
        }
    }
    __syncthreads();
    const int g = lane >> 2, q = lane & 3, mt = warp & 7, kh = warp >> 3;
    constexpr int NP = TRAIN ? 2 : 3;
    for (int l = 2; l <= 4; ++l) {
        const int cur = l & 1, nxt = cur ^ 1;  // layer 2 reads buffer 0
        if (first && !wait_copies(bars + l - 1, parity, spins)) {
            drain_weights(bars, l, parity);
            return false;
        }
        float acc[3][4];
        fwd_mma<NP>(S.ws + (size_t)(l - 2) * H * WP, S.plane(cur, 0), S.plane(cur, 1),
                    S.plane(cur, 2), mt, kh, lane, acc);
        float part[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
            part[c] = (NP == 3 ? acc[2][c] + acc[1][c] : acc[1][c]) + acc[0][c];
        const float2 zz = join_halves(S, part, mt, kh, lane);
        {
            const int u = 16 * mt + g + 8 * kh;
            const float b = S.bias[(l - 1) * H + u];
            float av[2];
            uint16_t hi[2], mid[2], lo[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int n = 2 * q + e;
                const float z = (e ? zz.y : zz.x) + b;
                float gd;
                av[e] = gelu_and_grad(z, gd);
                S.g[((l - 1) * NS + n) * GP + u] = gd;
                if (l < 4) {
                    if (TRAIN) {
                        split2(av[e], hi[e], mid[e]);
                    } else {
                        split3(av[e], hi[e], mid[e], lo[e]);
                        S.plane(nxt, 2)[n * WP + u] = lo[e];
                    }
                    S.plane(nxt, 0)[n * WP + u] = hi[e];
                    S.plane(nxt, 1)[n * WP + u] = mid[e];
                } else {
                    S.a4[n * GP + u] = av[e];
                }
            }
            if (TRAIN) {  // one 128-byte line per warp and part
                if (l < 4) {
                    const size_t off = a_index(u, n0 + 2 * q, items);
                    *reinterpret_cast<uint32_t*>(pl.a[l - 1][0] + off) = pack2(hi[0], hi[1]);
                    *reinterpret_cast<uint32_t*>(pl.a[l - 1][1] + off) = pack2(mid[0], mid[1]);
                } else {
                    *reinterpret_cast<float2*>(pl.a4 + f_index(u, n0 + 2 * q)) =
                        make_float2(av[0], av[1]);
                }
            }
        }
        __syncthreads();
    }
    return true;
}

// y of the item's samples: warp w takes sample w, lane k units 4k .. 4k + 3.
__device__ __forceinline__ float output_unit(const SmemA& S, int n, int lane) {
    const float4 a = *reinterpret_cast<const float4*>(S.a4 + n * GP + 4 * lane);
    const float4 v = *reinterpret_cast<const float4*>(S.w5 + 4 * lane);
    float s = fmaf(a.w, v.w, fmaf(a.z, v.z, fmaf(a.y, v.y, a.x * v.x)));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return s + S.misc[0];
}

// Output, loss derivative and backward pass of one item after forward_item<true>.
__device__ void backward_item(const SmemA& S, int B, int n0, const Planes& pl, int Bp) {
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int items = Bp / NS;
    if (warp < NS) {
        const int n = warp;
        const float y = output_unit(S, n, lane);
        if (lane == 0) {
            const float d = n0 + n < B ? 2.0f * (y - S.misc[40 + n]) / (float)B : 0.f;
            S.misc[8 + n] = d;
            pl.y[n0 + n] = y;
            pl.dout[n0 + n] = d;
        }
    }
    __syncthreads();
    {  // d_4 = dL/dy w5 gelu'(z_4): unit u, samples ns, ns + 1
        const int u = t & (H - 1), ns = (t >> 7) * 2;
        const float w = S.w5[u];
        uint16_t hi[2], lo[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int n = ns + k;
            const float d = S.misc[8 + n] * w * S.g[(3 * NS + n) * GP + u];
            split2(d, hi[k], lo[k]);
            S.plane(0, 0)[n * WP + u] = hi[k];
            S.plane(0, 1)[n * WP + u] = lo[k];
        }
        const size_t off = d_index(u, n0 + ns, items);
        *reinterpret_cast<uint32_t*>(pl.d[2][0] + off) = pack2(hi[0], hi[1]);
        *reinterpret_cast<uint32_t*>(pl.d[2][1] + off) = pack2(lo[0], lo[1]);
    }
    __syncthreads();
    const int g = lane >> 2, q = lane & 3, mt = warp & 7, kh = warp >> 3;
    for (int l = 4; l >= 2; --l) {  // W_l: d_l -> d_{l-1}
        const int cur = l & 1, nxt = cur ^ 1;  // d_4 sits in buffer 0
        float acc[2][4];
        bwd_mma(S.ws + (size_t)(l - 2) * H * WP, S.plane(cur, 0), S.plane(cur, 1), mt, kh, lane,
                acc);
        float part[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) part[c] = acc[1][c] + acc[0][c];
        const float2 ee = join_halves(S, part, mt, kh, lane);
        {
            const int i = 16 * mt + g + 8 * kh;
            float dv[2];
            uint16_t hi[2], lo[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int n = 2 * q + e;
                dv[e] = (e ? ee.y : ee.x) * S.g[((l - 2) * NS + n) * GP + i];
                if (l > 2) {
                    split2(dv[e], hi[e], lo[e]);
                    S.plane(nxt, 0)[n * WP + i] = hi[e];
                    S.plane(nxt, 1)[n * WP + i] = lo[e];
                }
            }
            if (l > 2) {
                const size_t off = d_index(i, n0 + 2 * q, items);
                *reinterpret_cast<uint32_t*>(pl.d[l - 3][0] + off) = pack2(hi[0], hi[1]);
                *reinterpret_cast<uint32_t*>(pl.d[l - 3][1] + off) = pack2(lo[0], lo[1]);
            } else {
                *reinterpret_cast<float2*>(pl.d1 + f_index(i, n0 + 2 * q)) =
                    make_float2(dv[0], dv[1]);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------- phase B --
// Adam (Kingma & Ba) with bias correction on one FP32 master weight; writes the BF16
// copy (round to nearest even).  c1 = 1 - beta1^t, c2 = 1 - beta2^t.  The state is loaded
// (adam_load) when a task starts, so that its latency hides behind the task's sums.
struct AdamState {
    float m, v, p;
};
__device__ __forceinline__ float ld_cg_pinned(const float* p) {
    float v;
    asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ AdamState adam_load(const float* __restrict__ p,
                                               const float* __restrict__ m,
                                               const float* __restrict__ v, int k) {
    // issued where they stand (not sunk to their use), so the latency overlaps the task
    return {ld_cg_pinned(m + k), ld_cg_pinned(v + k), ld_cg_pinned(p + k)};
}
__device__ __forceinline__ uint16_t adam_store(float* __restrict__ p, uint16_t* __restrict__ w,
                                               float* __restrict__ m, float* __restrict__ v,
                                               int k, const AdamState& st, float gk, float lr,
                                               float beta1, float beta2, float eps, float c1,
                                               float c2) {
    const float mk = beta1 * st.m + (1.0f - beta1) * gk;
    const float vk = beta2 * st.v + (1.0f - beta2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float pk = st.p - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    p[k] = pk;
    const uint16_t wb = f2bf(pk);
    w[k] = wb;
    return wb;
}

// Parameter k's new BF16 value into the weight image.
__device__ void image_store(const Planes& pl, int k, uint16_t wb) {
    if (k < off_w(1)) {  // W1, b1
        pl.img_small[k] = bf2f(wb);
    } else if (k >= off_w(4)) {  // W5, b5
        pl.img_small[7 * H + (k - off_w(4))] = bf2f(wb);
    } else {
        const int l = k < off_w(2) ? 1 : k < off_w(3) ? 2 : 3, r = k - off_w(l);
        if (r < H * H)
            pl.img_big[((size_t)(l - 1) * H + r / H) * WP + r % H] = wb;
        else
            pl.img_small[3 * H + l * H + (r - H * H)] = bf2f(wb);
    }
}

// Parameter k's state (training) and its update or gradient output.
template <bool TRAIN>
__device__ __forceinline__ AdamState prefetch(const StepArgs& A, int k) {
    if (TRAIN) return adam_load(A.master, A.m, A.v, k);
    return {0.f, 0.f, 0.f};
}
template <bool TRAIN>
__device__ __forceinline__ void emit(const StepArgs& A, int k, const AdamState& st, float gk,
                                     float c1, float c2) {
    if (TRAIN)
        image_store(A.pl, k, adam_store(A.master, A.w, A.m, A.v, k, st, gk, A.lr, A.beta1,
                                        A.beta2, A.eps, c1, c2));
    else
        A.grad[k] = gk;
}

// Gradient of a 16 x 32 tile of W_{L+2} (L = 0..2) over the whole batch:
// dW[o][i] = sum_n d[o][n] a[i][n].  The tile's operands arrive KI items at a time (four
// bulk copies per block) through a ring of NBUF buffers, each with its mbarrier (phase
// parities in *ring); warp w takes k-step (item pair) w of each block and the
// warps' sums are added in warp order.  The tile with ib == 0 also sums the bias gradient
// of its 16 units.  False if a wait gave up.
template <bool TRAIN>
__device__ bool hidden_task(const StepArgs& A, unsigned char* smem, uint64_t* ring,
                            uint32_t& ringpar, bool& fenced, int task, float c1, float c2) {
    const int L = task / ((H / TO) * (H / TI)), ob = (task / (H / TI)) % (H / TO),
              ib = task % (H / TI);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int items = A.Bp / NS;
    const int wbase = off_w(L + 1), bbase = off_b(L + 1);
    // this thread's parameters: tile entry t (row-major 16 x 32), bias t < 16
    static_assert(THREADS == TO * TI, "one tile entry per thread");
    const int k0 = wbase + (TO * ob + t / TI) * H + TI * ib + t % TI;
    const bool has_bias = ib == 0 && t < TO;
    const AdamState st0 = prefetch<TRAIN>(A, k0);
    const AdamState stb = has_bias ? prefetch<TRAIN>(A, bbase + TO * ob + t) : AdamState{};
    const uint16_t* dsrc0 = A.pl.d[L][0] + (size_t)ob * items * TO * NS;
    const uint16_t* dsrc1 = A.pl.d[L][1] + (size_t)ob * items * TO * NS;
    const uint16_t* asrc0 = A.pl.a[L][0] + (size_t)ib * items * TI * NS;
    const uint16_t* asrc1 = A.pl.a[L][1] + (size_t)ib * items * TI * NS;
    const int nblk = (items + KI - 1) / KI;
    auto buffer = [&](int buf) { return smem + buf * kStageBytes; };
    auto stage = [&](int blk) {  // thread 0
        const int it0 = blk * KI, ni = min(KI, items - it0);
        const int buf = blk % NBUF;
        unsigned char* b = buffer(buf);
        const uint32_t db = ni * TO * NS * sizeof(uint16_t), ab = ni * TI * NS * sizeof(uint16_t);
        gbd::mbar_arrive_expect_tx(ring + buf, 2 * (db + ab));
        gbd::bulk_copy_g2s(b, dsrc0 + (size_t)it0 * TO * NS, db, ring + buf);
        gbd::bulk_copy_g2s(b + kDBytes, dsrc1 + (size_t)it0 * TO * NS, db, ring + buf);
        gbd::bulk_copy_g2s(b + 2 * kDBytes, asrc0 + (size_t)it0 * TI * NS, ab, ring + buf);
        gbd::bulk_copy_g2s(b + 2 * kDBytes + kABytes, asrc1 + (size_t)it0 * TI * NS, ab,
                           ring + buf);
    };
    float acc[4][4], crs[4][4];  // hi.hi and hi.lo + lo.hi per n-tile of 8 inputs
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j][e] = crs[j][e] = 0.f;
    float bsum = 0.f;  // bias: unit t & 15, item pair t >> 4 of each block
    if (t == 0) {
        if (!fenced) proxy_fence();  // the operands were written by other CTAs this step
        for (int blk = 0; blk < NBUF - 1 && blk < nblk; ++blk) stage(blk);
    }
    fenced = true;
    for (int blk = 0; blk < nblk; ++blk) {
        if (t == 0 && blk + NBUF - 1 < nblk)
            stage(blk + NBUF - 1);  // its buffer was last read in block blk - 1
        const int buf = blk % NBUF;
        if (!wait_copies(ring + buf, (ringpar >> buf) & 1u, A.spins)) {
            for (int b = blk + 1; b < nblk && b < blk + NBUF; ++b)
                gbd::mbar_wait_bounded(ring + b % NBUF, (ringpar >> (b % NBUF)) & 1u,
                                       gbd::kDefaultWaitSpins);
            return false;
        }
        ringpar ^= 1u << buf;
        const int ks = min(KI, items - blk * KI) / 2;
        const unsigned char* b = buffer(buf);
        const uint16_t* dh = reinterpret_cast<const uint16_t*>(b);
        const uint16_t* dl = reinterpret_cast<const uint16_t*>(b + kDBytes);
        const uint16_t* ah = reinterpret_cast<const uint16_t*>(b + 2 * kDBytes);
        const uint16_t* al = reinterpret_cast<const uint16_t*>(b + 2 * kDBytes + kABytes);
        for (int kk = warp; kk < ks; kk += NWARP) {
            uint32_t Ah[4], Al[4];
            const int ao = ((2 * kk + (lane >> 4)) * TO + (lane & 15)) * NS;
            ldsm_x4(Ah, dh + ao);
            ldsm_x4(Al, dl + ao);
#pragma unroll
            for (int jp = 0; jp < 2; ++jp) {
                uint32_t Bh[4], Bl[4];
                const int bo = ((2 * kk + ((lane >> 3) & 1)) * TI + 16 * jp + ((lane >> 4) << 3) +
                                (lane & 7)) * NS;
                ldsm_x4(Bh, ah + bo);
                ldsm_x4(Bl, al + bo);
                mma(acc[2 * jp], Ah, Bh[0], Bh[1]);
                mma(crs[2 * jp], Ah, Bl[0], Bl[1]);
                mma(crs[2 * jp], Al, Bh[0], Bh[1]);
                mma(acc[2 * jp + 1], Ah, Bh[2], Bh[3]);
                mma(crs[2 * jp + 1], Ah, Bl[2], Bl[3]);
                mma(crs[2 * jp + 1], Al, Bh[2], Bh[3]);
            }
        }
        if (ib == 0) {  // unit o = t & 15, item pair kk = t >> 4: 16 samples in order
            const int o = t & 15, kk = t >> 4;
            if (kk < ks) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int off = ((2 * kk + h) * TO + o) * NS;
                    const uint4 vh = *reinterpret_cast<const uint4*>(dh + off);
                    const uint4 vl = *reinterpret_cast<const uint4*>(dl + off);
                    const uint32_t wh[4] = {vh.x, vh.y, vh.z, vh.w}, wl[4] = {vl.x, vl.y, vl.z, vl.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        bsum += __uint_as_float(wh[e] << 16) + __uint_as_float(wl[e] << 16);
                        bsum += __uint_as_float(wh[e] & 0xffff0000u) +
                                __uint_as_float(wl[e] & 0xffff0000u);
                    }
                }
            }
        }
        __syncthreads();  // the buffer is refilled NBUF - 1 blocks on
    }
    float* red = reinterpret_cast<float*>(smem + kOffRed);  // [NWARP][TO][RP]
    float* bs = reinterpret_cast<float*>(smem + kOffBsum);  // [16 item pairs][TO]
    {
        const int g = lane >> 2, q = lane & 3;
        float* rw = red + warp * TO * RP;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            *reinterpret_cast<float2*>(rw + g * RP + 8 * j + 2 * q) =
                make_float2(crs[j][0] + acc[j][0], crs[j][1] + acc[j][1]);
            *reinterpret_cast<float2*>(rw + (g + 8) * RP + 8 * j + 2 * q) =
                make_float2(crs[j][2] + acc[j][2], crs[j][3] + acc[j][3]);
        }
        if (ib == 0) bs[t] = bsum;
    }
    __syncthreads();
    const int r0 = (t / TI) * RP + t % TI;
    float s0 = red[r0];
#pragma unroll
    for (int w = 1; w < NWARP; ++w) s0 += red[w * TO * RP + r0];
    emit<TRAIN>(A, k0, st0, s0, c1, c2);
    if (has_bias) {
        float s = bs[t];
        for (int k = 1; k < THREADS / TO; ++k) s += bs[k * TO + t];
        emit<TRAIN>(A, bbase + TO * ob + t, stb, s, c1, c2);
    }
    __syncthreads();  // shared memory is reused by the next task
    return true;
}

// First layer: dW1[u][c] = sum_n d_1[u][n] x[n][c], db1[u] = sum_n d_1[u][n] for 16 units;
// thread (o, q) takes samples q, q + 32, ...; the 32 partial sums are added in q order.
template <bool TRAIN>
__device__ void first_task(const StepArgs& A, unsigned char* smem, int f, float c1, float c2) {
    const int t = threadIdx.x, o = t >> 5, q = t & 31, u = 16 * f + o;
    // thread t < 64 owns parameter (unit 16 f + t / 4, column t % 4; column 3 = bias)
    const int pu = 16 * f + (t >> 2), pc = t & 3;
    const int pk = pc < 3 ? off_w(0) + pu * 3 + pc : off_b(0) + pu;
    const AdamState st = t < 64 ? prefetch<TRAIN>(A, pk) : AdamState{};
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, gb = 0.f;
#pragma unroll 8
    for (int n = q; n < A.B; n += 32) {
        const float dn = __ldcg(A.pl.d1 + f_index(u, n));
        const float* xn = A.x + (size_t)n * 3;
        g0 = fmaf(dn, __ldg(xn), g0);
        g1 = fmaf(dn, __ldg(xn + 1), g1);
        g2 = fmaf(dn, __ldg(xn + 2), g2);
        gb += dn;
    }
    float* bs = reinterpret_cast<float*>(smem + kOffBsum);  // [16 units][32 q][4]
    float4* b4 = reinterpret_cast<float4*>(bs);
    b4[t] = make_float4(g0, g1, g2, gb);
    __syncthreads();
    if (t < 64) {
        const int uo = t >> 2;
        float s = bs[(uo * 32) * 4 + pc];
        for (int k = 1; k < 32; ++k) s += bs[(uo * 32 + k) * 4 + pc];
        emit<TRAIN>(A, pk, st, s, c1, c2);
    }
    __syncthreads();
}

// Deterministic sum over the block's threads (fixed tree).
__device__ float block_sum(float v, float* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < THREADS / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Output unit: dW5[u] = sum_n dL/dy[n] a_4[u][n] for 16 inputs; the first of these tasks
// also sums db5 = sum_n dL/dy[n] and, on the last step, the loss.
template <bool TRAIN>
__device__ void out_task(const StepArgs& A, unsigned char* smem, int f, float c1, float c2,
                         bool last) {
    const int t = threadIdx.x, o = t >> 5, q = t & 31, u = 16 * f + o;
    const AdamState st = t < 16 ? prefetch<TRAIN>(A, off_w(4) + 16 * f + t) : AdamState{};
    const AdamState stb = f == 0 && t == 0 ? prefetch<TRAIN>(A, off_b(4)) : AdamState{};
    float g = 0.f;
#pragma unroll 8
    for (int n = q; n < A.B; n += 32)
        g = fmaf(__ldcg(A.pl.dout + n), __ldcg(A.pl.a4 + f_index(u, n)), g);
    float* bs = reinterpret_cast<float*>(smem + kOffBsum);
    bs[t] = g;
    __syncthreads();
    if (t < 16) {
        float s = bs[t * 32];
        for (int k = 1; k < 32; ++k) s += bs[t * 32 + k];
        emit<TRAIN>(A, off_w(4) + 16 * f + t, st, s, c1, c2);
    }
    if (f == 0) {
        float sd = 0.f, l2 = 0.f;
        for (int n = t; n < A.B; n += THREADS) {
            sd += __ldcg(A.pl.dout + n);
            const float e = __ldcg(A.pl.y + n) - __ldg(A.target + n);
            l2 = fmaf(e, e, l2);
        }
        float* red = bs + THREADS;
        sd = block_sum(sd, red);
        l2 = block_sum(l2, red);
        if (t == 0) {
            emit<TRAIN>(A, off_b(4), stb, sd, c1, c2);
            if (last && A.loss) *A.loss = l2 / (float)A.B;
        }
    }
    __syncthreads();
}

__device__ void init_bars(uint64_t* bars, int n) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) gbd::mbar_init(bars + i, 1);
        gbd::mbar_fence_init();
    }
    __syncthreads();
}

// One cooperative launch: `steps` training steps (TRAIN) or one gradient evaluation.
template <bool TRAIN>
__global__ void __launch_bounds__(THREADS, 1) mlp_step_kernel(const StepArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ float corr[2];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBars);  // weights, then the ring
    init_bars(bars, kWBars + NBUF);
    const int items = A.Bp / NS;
    unsigned epoch = 0;
    uint32_t wpar = 0, ringpar = 0;
    for (int s = 0; s < A.steps; ++s) {
        if ((int)blockIdx.x < items) {
            const SmemA S(smem);
            stage_weights(A.pl, S, bars);
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                if (!forward_item<true>(S, A.x, A.target, A.B, it * NS, A.pl, A.Bp,
                                        it == (int)blockIdx.x, bars, wpar, A.spins))
                    return;
                backward_item(S, A.B, it * NS, A.pl, A.Bp);
            }
            wpar ^= 1u;
        }
        // Adam's bias corrections of this step, computed while the barrier waits
        if (!grid_sync(A.pl.bar, epoch, A.spins, [&] {
                if (TRAIN) {
                    corr[0] = bias_correction(A.beta1, A.first_step + s);
                    corr[1] = bias_correction(A.beta2, A.first_step + s);
                }
            }))
            return;
        const float c1 = TRAIN ? corr[0] : 1.f, c2 = TRAIN ? corr[1] : 1.f;
        bool fenced = false;
        for (int task = blockIdx.x; task < kTasks; task += gridDim.x) {
            if (task < kHiddenTasks) {
                if (!hidden_task<TRAIN>(A, smem, bars + kWBars, ringpar, fenced, task, c1, c2))
                    return;
            } else if (task < kHiddenTasks + kFirstTasks) {
                first_task<TRAIN>(A, smem, task - kHiddenTasks, c1, c2);
            } else {
                out_task<TRAIN>(A, smem, task - kHiddenTasks - kFirstTasks, c1, c2,
                                s + 1 == A.steps);
            }
        }
        if (s + 1 < A.steps && !grid_sync(A.pl.bar, epoch, A.spins, [] {})) return;
    }
}

// Inference: items of 8 samples, grid-strided; weights staged once per CTA.
__global__ void __launch_bounds__(THREADS, 1) mlp_forward_kernel(const uint16_t* __restrict__ W,
                                                                 const float* __restrict__ x,
                                                                 int B, float* __restrict__ y) {
    extern __shared__ __align__(128) unsigned char smem[];
    const SmemA S(smem);
    const int items = (B + NS - 1) / NS;
    load_weights(W, S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Planes none{};
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        forward_item<false>(S, x, nullptr, B, it * NS, none, 0, false, nullptr, 0u, 0u);
        if (warp < NS) {
            const float v = output_unit(S, warp, lane);
            if (lane == 0 && it * NS + warp < B) y[it * NS + warp] = v;
        }
        __syncthreads();  // S.a4 and the input samples are rewritten by the next item
    }
}

__global__ void __launch_bounds__(256) mlp_adam_kernel(float* __restrict__ p, uint16_t* __restrict__ w,
                                                       float* __restrict__ m, float* __restrict__ v,
                                                       const float* __restrict__ g, float lr,
                                                       float beta1, float beta2, float eps,
                                                       int step) {
    __shared__ float corr[2];
    if (threadIdx.x == 0) {
        corr[0] = bias_correction(beta1, step);
        corr[1] = bias_correction(beta2, step);
    }
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NPARAM)
        adam_store(p, w, m, v, k, adam_load(p, m, v, k), g[k], lr, beta1, beta2, eps, corr[0],
                   corr[1]);
}

// The weight image of a training call from the BF16 vector (padding columns zero).
__global__ void __launch_bounds__(256) mlp_image_kernel(const uint16_t* __restrict__ W,
                                                        float* __restrict__ small,
                                                        uint16_t* __restrict__ big) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < 3 * H * WP) {
        const int r = e / WP, c = e % WP;
        big[e] = c < H ? W[off_w(1 + r / H) + (r % H) * H + c] : (uint16_t)0;
    }
    if (e < kImgSmall) {
        float v = 0.f;
        if (e < 3 * H) v = bf2f(W[off_w(0) + e]);
        else if (e < 7 * H) v = bf2f(W[off_b((e - 3 * H) / H) + (e - 3 * H) % H]);
        else if (e < 8 * H) v = bf2f(W[off_w(4) + e - 7 * H]);
        else if (e == 8 * H) v = bf2f(W[off_b(4)]);
        small[e] = v;
    }
}

__global__ void __launch_bounds__(256) mlp_pack_kernel(const float* __restrict__ p,
                                                       uint16_t* __restrict__ w) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NPARAM) w[k] = f2bf(p[k]);
}

// ---------------------------------------------------------------------- host --
Planes carve(void* workspace, int B) {
    char* w = static_cast<char*>(workspace);
    const int Bp = padded_batch(B);
    const size_t half = align256((size_t)H * Bp * sizeof(uint16_t));
    const size_t full = align256((size_t)H * Bp * sizeof(float));
    const size_t vec = align256((size_t)Bp * sizeof(float));
    Planes p;
    p.bar = reinterpret_cast<unsigned*>(w);
    w += 256;
    for (int l = 0; l < 3; ++l)
        for (int h = 0; h < 2; ++h, w += half) p.a[l][h] = reinterpret_cast<uint16_t*>(w);
    for (int l = 0; l < 3; ++l)
        for (int h = 0; h < 2; ++h, w += half) p.d[l][h] = reinterpret_cast<uint16_t*>(w);
    p.a4 = reinterpret_cast<float*>(w);
    w += full;
    p.d1 = reinterpret_cast<float*>(w);
    w += full;
    p.y = reinterpret_cast<float*>(w);
    w += vec;
    p.dout = reinterpret_cast<float*>(w);
    w += vec;
    p.img_small = reinterpret_cast<float*>(w);
    p.img_big = reinterpret_cast<uint16_t*>(w + kImgBigOff);
    return p;
}

size_t workspace_bytes(int B) {
    const int Bp = padded_batch(B);
    return 256 + 12 * align256((size_t)H * Bp * sizeof(uint16_t)) +
           2 * align256((size_t)H * Bp * sizeof(float)) + 2 * align256((size_t)Bp * sizeof(float)) +
           align256(kImgBigOff + kImgBigBytes);
}

struct Occupancy {
    int device = -1, step_grid = 0, grad_grid = 0, fwd_grid = 0;
};
thread_local Occupancy t_occ;

// Co-resident grid of each kernel on the current device (the cooperative launch needs
// every CTA resident at once), after raising the shared-memory limits.
cudaError_t occupancy(Occupancy& o) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (o.device == dev) return cudaSuccess;
    int sms = 0, coop = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess)
        return e;
    if (!coop) return cudaErrorNotSupported;
    auto fit = [&](const void* fn, size_t smem, int* grid) {
        if (e != cudaSuccess) return;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nb = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, THREADS, smem);
        *grid = nb * sms;
        if (e == cudaSuccess && nb < 1) e = cudaErrorInvalidConfiguration;
    };
    fit((const void*)mlp_step_kernel<true>, kSmemStep, &o.step_grid);
    fit((const void*)mlp_step_kernel<false>, kSmemStep, &o.grad_grid);
    fit((const void*)mlp_forward_kernel, kSmemA, &o.fwd_grid);
    if (e == cudaSuccess) o.device = dev;
    return e;
}

gbd_status cuda_status(cudaError_t e) {
    return e == cudaSuccess ? GBD_OK : gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
}

gbd_status last_error() { return cuda_status(cudaGetLastError()); }

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

// Grid of a step launch: every CTA resident; at least one CTA per phase-A item or
// phase-B task, as far as residency allows.
int step_grid(int resident, int B) {
    const int items = padded_batch(B) / NS;
    const int want = items > kTasks ? items : kTasks;
    return want < resident ? want : resident;
}

template <bool TRAIN>
gbd_status launch_steps(StepArgs& a, int resident, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.pl.bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_status(e);
    mlp_image_kernel<<<(3 * H * WP + 255) / 256, 256, 0, s>>>(a.w, a.pl.img_small, a.pl.img_big);
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)mlp_step_kernel<TRAIN>,
                                    dim3(step_grid(resident, a.B)), dim3(THREADS), args,
                                    kSmemStep, s);
    return cuda_status(e);
}

}  // namespace

// The status word: copied into pinned host memory on the caller's stream (gbd_sync), and
// cleared once it has been reported.
cudaError_t gbd_mlp_status_fetch(unsigned* host, cudaStream_t s) {
    return cudaMemcpyFromSymbolAsync(host, g_mlp_status, sizeof(unsigned), 0,
                                     cudaMemcpyDeviceToHost, s);
}
void gbd_mlp_status_clear() {
    const unsigned zero = 0;
    cudaMemcpyToSymbol(g_mlp_status, &zero, sizeof(zero));
}

extern "C" {

size_t gbd_mlp_workspace_bytes(int32_t batch) {
    if (batch < 1) return 0;
    return workspace_bytes(batch);
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
    cudaError_t e = occupancy(t_occ);
    if (e != cudaSuccess) return cuda_status(e);
    const int items = (batch + NS - 1) / NS;
    const int grid = items < t_occ.fwd_grid ? items : t_occ.fwd_grid;
    mlp_forward_kernel<<<grid, THREADS, kSmemA, static_cast<cudaStream_t>(stream)>>>(weights, x,
                                                                                     batch, y);
    return last_error();
}

gbd_status gbd_mlp_grad(const uint16_t* weights, const float* x, const float* target,
                        int32_t batch, float* grad, float* loss, void* workspace, size_t bytes,
                        void* stream) {
    GBD_NVTX_RANGE("gbd_mlp_grad");
    if (!grad) return gbd_set_error(GBD_EINVAL, "NULL buffer");
    gbd_status st = check_train(weights, x, target, batch, workspace, bytes);
    if (st != GBD_OK) return st;
    cudaError_t e = occupancy(t_occ);
    if (e != cudaSuccess) return cuda_status(e);
    StepArgs a{};
    a.w = const_cast<uint16_t*>(weights);  // read only in gradient mode
    a.grad = grad;
    a.x = x;
    a.target = target;
    a.loss = loss;
    a.B = batch;
    a.Bp = padded_batch(batch);
    a.first_step = 1;
    a.steps = 1;
    a.spins = gbd_wait_spins();
    a.pl = carve(workspace, batch);
    return launch_steps<false>(a, t_occ.grad_grid, static_cast<cudaStream_t>(stream));
}

gbd_status gbd_mlp_adam(float* master, uint16_t* weights, float* m, float* v, const float* grad,
                        float lr, float beta1, float beta2, float eps, int32_t step, void* stream) {
    GBD_NVTX_RANGE("gbd_mlp_adam");
    if (!master || !weights || !m || !v || !grad) return gbd_set_error(GBD_EINVAL, "NULL buffer");
    gbd_status st = check_adam(lr, beta1, beta2, eps, step);
    if (st != GBD_OK) return st;
    mlp_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        master, weights, m, v, grad, lr, beta1, beta2, eps, step);
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
    if (steps == 0) return GBD_OK;
    cudaError_t e = occupancy(t_occ);
    if (e != cudaSuccess) return cuda_status(e);
    StepArgs a{};
    a.master = master;
    a.w = weights;
    a.m = m;
    a.v = v;
    a.x = x;
    a.target = target;
    a.loss = loss;
    a.lr = lr;
    a.beta1 = beta1;
    a.beta2 = beta2;
    a.eps = eps;
    a.B = batch;
    a.Bp = padded_batch(batch);
    a.first_step = first_step;
    a.steps = steps;
    a.spins = gbd_wait_spins();
    a.pl = carve(workspace, batch);
    return launch_steps<true>(a, t_occ.step_grid, static_cast<cudaStream_t>(stream));
}

gbd_status gbd_mlp_train_step(float* master, uint16_t* weights, float* m, float* v,
                              const float* x, const float* target, int32_t batch, float lr,
                              float beta1, float beta2, float eps, int32_t step, float* loss,
                              void* workspace, size_t bytes, void* stream) {
    return gbd_mlp_train(master, weights, m, v, x, target, batch, lr, beta1, beta2, eps, step, 1,
                         loss, workspace, bytes, stream);
}

}  // extern "C"
