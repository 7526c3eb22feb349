// Throughput probes of the pipes the field kernels are bound by: MUFU ex2 / sin / cos
// (XU pipe), FP32 FMA and FP64 FMA.  Each thread runs eight independent dependency
// chains so that latency is hidden and the pipe, not the chain, limits the rate.  The
// values stay bounded (fixed points of exp2(-x), sin, cos and an affine map).
#include "gbd_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int OP>
__device__ __forceinline__ float step(float x) {
    if (OP == 0) return gbd::mufu_ex2(-x);
    if (OP == 1) return gbd::mufu_sin(x);
    if (OP == 2) return gbd::mufu_cos(x);
    return fmaf(x, 0.99993f, 0.00007f);
}

template <int OP>
__global__ void __launch_bounds__(kThreads) probe_f32(float* sink, int iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.3f + 1e-3f * c + 1e-7f * threadIdx.x;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = step<OP>(x[c]);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) probe_f64(double* sink, int iters) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.3 + 1e-3 * c + 1e-7 * threadIdx.x;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], 0.99993, 0.00007);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) sink[threadIdx.x] = s;
}

template <typename F>
cudaError_t time_best(F launch, double ops, double* rate) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) return e;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a, 0);
        launch();
        cudaEventRecord(b, 0);
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *rate = ops / (best * 1e-3);
    return cudaSuccess;
}

}  // namespace

cudaError_t gbd_run_probes(double* out) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8;
    void* sink = nullptr;
    if ((e = cudaMalloc(&sink, kThreads * sizeof(double))) != cudaSuccess) return e;
    const double threads = (double)blocks * kThreads;
    const int it_mufu = 2048, it_fma = 8192, it_dfma = 1024;
    e = time_best([&] { probe_f32<0><<<blocks, kThreads>>>((float*)sink, it_mufu); },
                  threads * kChains * it_mufu, &out[0]);
    if (e == cudaSuccess)
        e = time_best([&] { probe_f32<1><<<blocks, kThreads>>>((float*)sink, it_mufu); },
                      threads * kChains * it_mufu, &out[1]);
    if (e == cudaSuccess)
        e = time_best([&] { probe_f32<2><<<blocks, kThreads>>>((float*)sink, it_mufu); },
                      threads * kChains * it_mufu, &out[2]);
    if (e == cudaSuccess)
        e = time_best([&] { probe_f32<3><<<blocks, kThreads>>>((float*)sink, it_fma); },
                      threads * kChains * it_fma, &out[3]);
    if (e == cudaSuccess)
        e = time_best([&] { probe_f64<<<blocks, kThreads>>>((double*)sink, it_dfma); },
                      threads * kChains * it_dfma, &out[4]);
    cudaFree(sink);
    return e;
}
