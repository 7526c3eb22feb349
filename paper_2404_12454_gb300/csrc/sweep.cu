// Batched parameter sweep (Sec. 6): many GBD instances sharing the optics and detector but
// differing in beamlets across, overlap factor and waist ratio, each scored by the RMS
// difference of |E|/|E(centre)| to the Airy amplitude inside the third dark ring.
//
// One sweep = a batched trace + projection kernel writing every instance's records at
// tile-aligned offsets, one persistent field kernel, and a finalize kernel.  The field
// kernel runs one CTA per resident slot; each CTA takes (instance, pixel block) work
// items from an atomic counter in longest-first order (instances with the most beamlet
// tiles first), evaluates the instance's beamlets on its pixels exactly as
// field_mixed_kernel does, and folds the score's moments over its pixels
// (S2 = sum |E|^2, S1 = sum |E| A, S0 = sum A^2, n, and |E| at the centre pixel) into a
// per-item slot.  The finalize kernel sums each instance's items in pixel-block order,
// so the result does not depend on which CTA ran which item:
//     score = sqrt((S2/e0^2 - 2 S1/e0 + S0) / n).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "field_core.cuh"
#include "gbd_internal.cuh"

namespace {

using gbd::kStages;
using gbd::kThreads;
using gbd::kWarps;

__device__ unsigned int g_sweep_status = 0;

// Score regions: region 0 is the disc inside the third dark ring (r <= j_{1,3} lambda F#/pi),
// regions 1.. are optional annular zones lo <= r/(lambda F#) < hi.  Per region the
// moments S2 = sum |E|^2, S1 = sum |E| A, S0 = sum A^2 and the pixel count n.
constexpr int kMaxRegions = 8;

struct Regions {
    int n;
    double lo[kMaxRegions], hi[kMaxRegions];  // in lambda F# (region 0: [0, r3] closed)
};

// Per pixel: |2 J1(x)/x| with x = pi r / (lambda F#), and the bit mask of the regions the
// pixel belongs to.
__global__ void __launch_bounds__(256) airy_table_kernel(int nx, int ny, double px, double py,
                                                         double lam_fnum, Regions R,
                                                         double2* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nx * ny) return;
    const int i = p % nx, j = p / nx;
    const double sx = (i - nx / 2) * px, sy = (j - ny / 2) * py;
    const double r = hypot(sx, sy);
    const double x = M_PI * r / lam_fnum;
    const double a = x == 0.0 ? 1.0 : fabs(2.0 * j1(x) / x);
    const double u = r / lam_fnum;
    unsigned mask = u <= R.hi[0] ? 1u : 0u;
    for (int z = 1; z < R.n; ++z)
        if (u >= R.lo[z] && u < R.hi[z]) mask |= 1u << z;
    out[p] = make_double2(a, (double)mask);
}

// Epilogue of one work item: the moments per region of the item's pixels (|E| from
// mag_of(r, c) for the thread's pixel (row0 + 8 r, col0 + 32 c)), reduced by warp
// shuffles, then across warps in a fixed order into the item's slot: e0, then 4 moments
// per region.  Every thread of the CTA calls it.
template <int RB, int CB, class Mag>
__device__ __forceinline__ void item_moments(Mag mag_of, int2 it, int row0, int col0, int nx,
                                             int ny, const double2* __restrict__ airy,
                                             int n_regions, int n_blocks,
                                             double* __restrict__ moments,
                                             double (*red)[kMaxRegions][4], double* red_e0) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double e0 = -1.0;
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c)
            if (row0 + 8 * r == ny / 2 && col0 + 32 * c == nx / 2) e0 = mag_of(r, c);
    for (int o = 16; o > 0; o >>= 1) e0 = fmax(e0, __shfl_xor_sync(0xffffffffu, e0, o));
    if (lane == 0) red_e0[warp] = e0;
    for (int z = 0; z < n_regions; ++z) {
        double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const int row = row0 + 8 * r, col = col0 + 32 * c;
                if (row >= ny || col >= nx) continue;
                const double2 A = airy[(size_t)row * nx + col];
                if (!((unsigned)A.y & (1u << z))) continue;
                const double mg = mag_of(r, c);
                m0 += mg * mg;
                m1 += mg * A.x;
                m2 += A.x * A.x;
                m3 += 1.0;
            }
        for (int o = 16; o > 0; o >>= 1) {
            m0 += __shfl_xor_sync(0xffffffffu, m0, o);
            m1 += __shfl_xor_sync(0xffffffffu, m1, o);
            m2 += __shfl_xor_sync(0xffffffffu, m2, o);
            m3 += __shfl_xor_sync(0xffffffffu, m3, o);
        }
        if (lane == 0) {
            red[warp][z][0] = m0;
            red[warp][z][1] = m1;
            red[warp][z][2] = m2;
            red[warp][z][3] = m3;
        }
    }
    __syncthreads();
    // one slot per item: e0, then 4 moments per region, summed over warps in order
    const int stride = 1 + 4 * n_regions;
    double* dst = moments + ((size_t)it.x * n_blocks + it.y) * stride;
    if (tid == 0) {
        double s = -1.0;
        for (int w = 0; w < kWarps; ++w) s = fmax(s, red_e0[w]);
        dst[0] = s;
    }
    if (tid < 4 * n_regions) {
        const int z = tid / 4, q = tid % 4;
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += red[w][z][q];
        dst[1 + tid] = s;
    }
}

// WIDE, PAIR: as in field_mixed_kernel (several instantiations are launched; each returns
// at once unless the projection's flag word masked by `mask` equals `want`).  SMEM keeps
// the compensation pairs in dynamic shared memory after the record stages (2 x 8 blocks).
template <int RB, int CB, bool WIDE, bool PAIR, bool SMEM, bool CROSS = true>
__global__ void __launch_bounds__(kThreads, 2)
    sweep_kernel(const float4* __restrict__ coef, const int2* __restrict__ inst_tiles,
                 const int2* __restrict__ items, int n_items, int tiles_x, int n_blocks, int nx,
                 int ny, const double2* __restrict__ airy, int n_regions,
                 double* __restrict__ moments, int* __restrict__ counter,
                 const unsigned* __restrict__ flags, unsigned mask, unsigned want, unsigned anyof,
                 uint32_t spins) {
    static_assert(!PAIR || RB == 2, "row pairs need two rows per thread");
    const unsigned fw = *flags;
    if ((fw & mask) != want || (anyof != 0u && (fw & anyof) == 0u)) return;
    constexpr int kTileF4 = gbd::kMixedFields * gbd::kTile;
    extern __shared__ __align__(128) float4 sweep_dyn[];
    float4(*stage)[kTileF4] = reinterpret_cast<float4(*)[kTileF4]>(sweep_dyn);
    float4* comp = sweep_dyn + kStages * kTileF4;  // SMEM: [RB * CB][kThreads]
    // SMEM: then each warp's row terms of the current tile (narrow row pairs)
    float4* ent = comp + RB * CB * kThreads + (threadIdx.x >> 5) * (gbd::kPairRowF4 * gbd::kTile);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
    __shared__ int flag, s_item;
    __shared__ double red[kWarps][kMaxRegions][4];
    __shared__ double red_e0[kWarps];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    gbd::init_stream_barriers(full, empty, tid);
    int g = 0;  // tiles this CTA has streamed so far (keeps the barrier phases in step)
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const int2 it = items[item];           // (instance, pixel block)
        const int2 tt = inst_tiles[it.x];      // (first tile, tiles)
        gbd::TileStream<float4, kTileF4> ts{stage, full, empty, coef + (size_t)tt.x * kTileF4,
                                            tt.y, g, gbd::kMixedTileBytes, 0};
        bool ok = ts.start(tid, spins, &flag);

        const int col0 = (it.y % tiles_x) * (32 * CB) + lane;
        const int row0 = (it.y / tiles_x) * (8 * RB) + warp;
        float colf[CB], rowf[RB];
#pragma unroll
        for (int c = 0; c < CB; ++c) colf[c] = (float)(col0 + 32 * c);
#pragma unroll
        for (int r = 0; r < RB; ++r) rowf[r] = (float)(row0 + 8 * r);
        float2 acc[RB][CB], hi[RB][CB], lo[RB][CB];
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                acc[r][c] = hi[r][c] = lo[r][c] = make_float2(0.f, 0.f);
                if constexpr (SMEM) comp[(r * CB + c) * kThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
            }

        int k = 0;
        for (; ok && k < ts.nt; ++k) {
            if (!ts.acquire(k, spins)) {
                ok = false;
                break;
            }
            if constexpr (PAIR && SMEM && !WIDE) {
                __syncwarp();  // every lane is done with the previous tile's row terms
                gbd::mixed_pair_rows<CROSS>(ts.tile(k), rowf[0], ent, lane);
                __syncwarp();
                gbd::mixed_tile_pair_rows<CB, CROSS>(ts.tile(k), ent, colf, acc);
            } else if constexpr (PAIR)
                gbd::mixed_tile_pair<CB, WIDE>(ts.tile(k), colf, rowf[0], acc);
            else
                gbd::mixed_tile<RB, CB, WIDE>(ts.tile(k), colf, rowf, acc);
            if constexpr (SMEM)
                gbd::mixed_fold_smem<RB, CB>(acc, comp, tid);
            else
                gbd::mixed_fold<RB, CB>(acc, hi, lo);
            if (!ts.release(k, lane, warp, spins)) {
                ok = false;
                ++k;
                break;
            }
        }
        // every thread reaches this vote (failed waits end their loops), so the CTA
        // leaves together when any warp gave up
        if (!__syncthreads_and(ok)) {
            atomicOr(&g_sweep_status, gbd::kStatusTimeout);
            if (tid == 0) ts.drain(k, spins);
            return;
        }
        g += ts.nt;

        // epilogue: per region the moments of this item's pixels; |E| is recomputed per
        // region rather than kept, which holds the wide blocks' register use down
        auto mag_of = [&](int r, int c) -> double {
            double re, im;
            if constexpr (SMEM) {
                const float4 v = comp[(r * CB + c) * kThreads + tid];
                re = (double)v.x + (double)v.z;
                im = (double)v.y + (double)v.w;
            } else {
                re = (double)hi[r][c].x + (double)lo[r][c].x;
                im = (double)hi[r][c].y + (double)lo[r][c].y;
            }
            return sqrt(re * re + im * im);
        };
        item_moments<RB, CB>(mag_of, it, row0, col0, nx, ny, airy, n_regions, n_blocks, moments,
                             red, red_e0);
    }
}

// Row triples (3 x CB pixels per thread, rows 8 apart) on work items of 256 x 24 pixels.
// FAST: fields without multi-row steepness (the warp's row terms computed per 32-beamlet
// half tile): without a uv term mixed_tile_rows, with one (CROSS) mixed_tile_rows_cross
// with the per-column row factors, folded after every tile like the direct instantiation
// (real-ray traced fields); otherwise every pixel is evaluated directly with its phase
// reduced exactly (mixed_tile<3, CB, true>), which holds for any field.
// The sums run in FP32 registers for at most kRowsChunkTiles tiles and are then folded
// with TwoSum into a compensated pair per pixel in shared memory: hi as FP32, the much
// smaller lo as BF16 (its rounding, 2^-9 of lo, is 2^-33 of hi), which makes 24 pixels a
// thread fit next to two CTAs per SM.  The direct instantiation folds after every tile: its
// fields (uv terms, real-ray traces) near the centre add ~1,000 nearly equal in-phase terms
// per 16 tiles onto a sum 50 times larger, whose FP32 rounding then drifts one way (scores
// 1e-3 high at 51k beamlets; folding per tile costs under 1 % there).  Dynamic shared memory: the kStages record stages,
// hi [3 CB][kThreads] float2, lo [3 CB][kThreads] bf16x2, then (FAST) each warp's row
// terms of 32 beamlets.
constexpr int kRowsChunkTiles = 16;
template <int CB, bool FAST, bool CROSS = false>
__global__ void __launch_bounds__(kThreads, 2)
    sweep_rows_kernel(const float4* __restrict__ coef, const int2* __restrict__ inst_tiles,
                      const int2* __restrict__ items, int n_items, int tiles_x, int n_blocks,
                      int nx, int ny, const double2* __restrict__ airy, int n_regions,
                      double* __restrict__ moments, int* __restrict__ counter,
                      const unsigned* __restrict__ flags, unsigned mask, unsigned want,
                      unsigned anyof, uint32_t spins) {
    constexpr int RB = 3;
    const unsigned fw = *flags;
    if ((fw & mask) != want || (anyof != 0u && (fw & anyof) == 0u)) return;
    constexpr int kTileF4 = gbd::kMixedFields * gbd::kTile;
    extern __shared__ __align__(128) float4 sweep_dyn[];
    float4(*stage)[kTileF4] = reinterpret_cast<float4(*)[kTileF4]>(sweep_dyn);
    float2* hi = reinterpret_cast<float2*>(sweep_dyn + kStages * kTileF4);  // [RB CB][kThreads]
    uint32_t* lo = reinterpret_cast<uint32_t*>(hi + RB * CB * kThreads);     // [RB CB][kThreads]
    constexpr int kEntF4 = CROSS ? gbd::kRowsCrossF4<RB> : gbd::kRowsF4;
    float4* ent = reinterpret_cast<float4*>(lo + RB * CB * kThreads) +
                  (threadIdx.x >> 5) * (kEntF4 * 32);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
    __shared__ int flag, s_item;
    __shared__ double red[kWarps][kMaxRegions][4];
    __shared__ double red_e0[kWarps];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    gbd::init_stream_barriers(full, empty, tid);
    int g = 0;  // tiles this CTA has streamed so far (keeps the barrier phases in step)
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const int2 it = items[item];           // (instance, pixel block)
        const int2 tt = inst_tiles[it.x];      // (first tile, tiles)
        gbd::TileStream<float4, kTileF4> ts{stage, full, empty, coef + (size_t)tt.x * kTileF4,
                                            tt.y, g, gbd::kMixedTileBytes, 0};
        bool ok = ts.start(tid, spins, &flag);

        const int col0 = (it.y % tiles_x) * (32 * CB) + lane;
        const int row0 = (it.y / tiles_x) * (8 * RB) + warp;
        float colf[CB], rowf[RB];
#pragma unroll
        for (int c = 0; c < CB; ++c) colf[c] = (float)(col0 + 32 * c);
#pragma unroll
        for (int r = 0; r < RB; ++r) rowf[r] = (float)(row0 + 8 * r);
        float2 acc[RB][CB];
#pragma unroll
        for (int m = 0; m < RB * CB; ++m) {
            acc[m / CB][m % CB] = make_float2(0.f, 0.f);
            hi[m * kThreads + tid] = make_float2(0.f, 0.f);
            lo[m * kThreads + tid] = 0u;
        }

        int k = 0;
        for (; ok && k < ts.nt; ++k) {
            if (!ts.acquire(k, spins)) {
                ok = false;
                break;
            }
            if constexpr (FAST) {
#pragma unroll 1
                for (int h = 0; h < gbd::kTile / 32; ++h) {
                    __syncwarp();  // every lane is done with the previous row terms
                    if constexpr (CROSS) {
                        gbd::mixed_rows_cross_term<RB>(ts.tile(k), 32 * h + lane, rowf[0], ent,
                                                       lane, 32);
                        __syncwarp();
                        gbd::mixed_tile_rows_cross<RB, CB, 32>(ent, colf, acc);
                    } else {
                        gbd::mixed_rows_term<RB>(ts.tile(k), 32 * h + lane, rowf[0], ent, lane,
                                                 32);
                        __syncwarp();
                        gbd::mixed_tile_rows<RB, CB, 32>(ent, colf, acc);
                    }
                }
            } else {
                gbd::mixed_tile<RB, CB, true>(ts.tile(k), colf, rowf, acc);
            }
            constexpr int kChunk = FAST && !CROSS ? kRowsChunkTiles : 1;
            if ((k + 1) % kChunk == 0 || k + 1 == ts.nt) {
#pragma unroll
                for (int m = 0; m < RB * CB; ++m) {
                    const int q = m * kThreads + tid;
                    const float2 h2 = hi[q];
                    const uint32_t l2 = lo[q];
                    float sx, ex, sy, ey;
                    gbd::two_sum(h2.x, acc[m / CB][m % CB].x, sx, ex);
                    gbd::two_sum(h2.y, acc[m / CB][m % CB].y, sy, ey);
                    hi[q] = make_float2(sx, sy);
                    const float lx = __uint_as_float(l2 << 16) + ex;
                    const float ly = __uint_as_float(l2 & 0xffff0000u) + ey;
                    const __nv_bfloat162 lb = __floats2bfloat162_rn(lx, ly);
                    lo[q] = *reinterpret_cast<const uint32_t*>(&lb);
                    acc[m / CB][m % CB] = make_float2(0.f, 0.f);
                }
            }
            if (!ts.release(k, lane, warp, spins)) {
                ok = false;
                ++k;
                break;
            }
        }
        // every thread reaches this vote (failed waits end their loops), so the CTA
        // leaves together when any warp gave up
        if (!__syncthreads_and(ok)) {
            atomicOr(&g_sweep_status, gbd::kStatusTimeout);
            if (tid == 0) ts.drain(k, spins);
            return;
        }
        g += ts.nt;
        auto mag_of = [&](int r, int c) -> double {
            const int q = (r * CB + c) * kThreads + tid;
            const float2 h2 = hi[q];
            const uint32_t l2 = lo[q];
            const double re = (double)h2.x + (double)__uint_as_float(l2 << 16);
            const double im = (double)h2.y + (double)__uint_as_float(l2 & 0xffff0000u);
            return sqrt(re * re + im * im);
        };
        item_moments<RB, CB>(mag_of, it, row0, col0, nx, ny, airy, n_regions, n_blocks, moments,
                             red, red_e0);
    }
}

constexpr size_t sweep_rows_smem(int cb, bool cross = false) {
    return (size_t)kStages * gbd::kMixedTileBytes + (size_t)3 * cb * kThreads * (8 + 4) +
           (size_t)kWarps * (cross ? gbd::kRowsCrossF4<3> : gbd::kRowsF4) * 32 * sizeof(float4);
}

// Per instance, the moments of its pixel blocks summed in block order, then one score per
// region: scores[k * n_regions + z].
__global__ void __launch_bounds__(128) sweep_finalize_kernel(const double* __restrict__ moments,
                                                             int n_inst, int n_blocks,
                                                             int n_regions,
                                                             double* __restrict__ scores) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_inst) return;
    const int stride = 1 + 4 * n_regions;
    double e0 = -1.0;
    for (int t = 0; t < n_blocks; ++t) e0 = fmax(e0, moments[((size_t)k * n_blocks + t) * stride]);
    for (int z = 0; z < n_regions; ++z) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int t = 0; t < n_blocks; ++t) {
            const double* m = moments + ((size_t)k * n_blocks + t) * stride + 1 + 4 * z;
            for (int q = 0; q < 4; ++q) s[q] += m[q];
        }
        double score = nan("");
        if (e0 > 0.0 && s[3] > 0.0)
            score = sqrt(fmax(0.0, (s[0] / (e0 * e0) - 2.0 * s[1] / e0 + s[2]) / s[3]));
        scores[(size_t)k * n_regions + z] = score;
    }
}

typedef cudaError_t (*sweep_launch_fn)(dim3, cudaStream_t, const float4*, const int2*, const int2*,
                                       int, int, int, int, int, const double2*, int, double*, int*,
                                       const unsigned*, uint32_t);

constexpr size_t sweep_smem(int rb, int cb, bool smem) {
    return (size_t)kStages * gbd::kMixedTileBytes +
           (smem ? (size_t)rb * cb * kThreads * sizeof(float4) +
                       (size_t)kWarps * gbd::kPairRowF4 * gbd::kTile * sizeof(float4)
                 : 0);
}

template <int RB, int CB, bool WIDE, bool PAIR, bool SMEM, bool CROSS = true>
cudaError_t launch_one(dim3 grid, cudaStream_t s, const float4* coef, const int2* it_tiles,
                       const int2* items, int n_items, int tiles_x, int n_blocks, int nx, int ny,
                       const double2* airy, int n_regions, double* moments, int* counter,
                       const unsigned* flags, unsigned mask, unsigned want, unsigned anyof,
                       uint32_t spins) {
    constexpr size_t smem = sweep_smem(RB, CB, SMEM);
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<RB, CB, WIDE, PAIR, SMEM, CROSS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep_kernel<RB, CB, WIDE, PAIR, SMEM, CROSS><<<grid, kThreads, smem, s>>>(
        coef, it_tiles, items, n_items, tiles_x, n_blocks, nx, ny, airy, n_regions, moments,
        counter, flags, mask, want, anyof, spins);
    return cudaGetLastError();
}

// Direct evaluation: the narrow- and wide-phase instantiations.
template <int RB, int CB>
cudaError_t launch_sweep(dim3 grid, cudaStream_t s, const float4* coef, const int2* it_tiles,
                         const int2* items, int n_items, int tiles_x, int n_blocks, int nx, int ny,
                         const double2* airy, int n_regions, double* moments, int* counter,
                         const unsigned* flags, uint32_t spins) {
    using gbd::kFlagWide;
    cudaError_t e = launch_one<RB, CB, false, false, false>(
        grid, s, coef, it_tiles, items, n_items, tiles_x, n_blocks, nx, ny, airy, n_regions,
        moments, counter, flags, kFlagWide, 0u, 0u, spins);
    if (e == cudaSuccess)
        e = launch_one<RB, CB, true, false, false>(grid, s, coef, it_tiles, items, n_items, tiles_x,
                                                   n_blocks, nx, ny, airy, n_regions, moments,
                                                   counter, flags, kFlagWide, kFlagWide, 0u, spins);
    return e;
}

// Row pairs on 2 x CB pixels, with direct evaluation on the same pixel blocks as the
// fallback for steep beamlets; SMEM for the 2 x 8 blocks.  Exactly one instantiation
// runs: narrow phase, then wide phase or column-steep, then the steep fallbacks.
template <int CB>
cudaError_t launch_sweep_pair(dim3 grid, cudaStream_t s, const float4* coef, const int2* it_tiles,
                              const int2* items, int n_items, int tiles_x, int n_blocks, int nx,
                              int ny, const double2* airy, int n_regions, double* moments,
                              int* counter, const unsigned* flags, uint32_t spins) {
    using gbd::kFlagColSteep;
    using gbd::kFlagCross;
    using gbd::kFlagSteep;
    using gbd::kFlagWide;
    constexpr unsigned kBoth = kFlagWide | kFlagSteep, kAll = kBoth | kFlagColSteep;
    constexpr bool kSmem = CB >= 8;
    cudaError_t e = cudaSuccess;
    if constexpr (kSmem) {  // the shared-memory form has a no-uv-term instantiation
        e = launch_one<2, CB, false, true, kSmem, false>(
            grid, s, coef, it_tiles, items, n_items, tiles_x, n_blocks, nx, ny, airy, n_regions,
            moments, counter, flags, kAll | kFlagCross, 0u, 0u, spins);
        if (e == cudaSuccess)
            e = launch_one<2, CB, false, true, kSmem>(
                grid, s, coef, it_tiles, items, n_items, tiles_x, n_blocks, nx, ny, airy,
                n_regions, moments, counter, flags, kAll, 0u, kFlagCross, spins);
    } else {
        e = launch_one<2, CB, false, true, kSmem>(
            grid, s, coef, it_tiles, items, n_items, tiles_x, n_blocks, nx, ny, airy, n_regions,
            moments, counter, flags, kAll, 0u, 0u, spins);
    }
    if (e == cudaSuccess)
        e = launch_one<2, CB, true, true, kSmem>(grid, s, coef, it_tiles, items, n_items, tiles_x,
                                                 n_blocks, nx, ny, airy, n_regions, moments,
                                                 counter, flags, kFlagSteep, 0u,
                                                 kFlagWide | kFlagColSteep, spins);
    if (e == cudaSuccess)
        e = launch_one<2, CB, false, false, kSmem>(grid, s, coef, it_tiles, items, n_items,
                                                   tiles_x, n_blocks, nx, ny, airy, n_regions,
                                                   moments, counter, flags, kBoth, kFlagSteep,
                                                   0u, spins);
    if (e == cudaSuccess)
        e = launch_one<2, CB, true, false, kSmem>(grid, s, coef, it_tiles, items, n_items, tiles_x,
                                                  n_blocks, nx, ny, airy, n_regions, moments,
                                                  counter, flags, kBoth, kBoth, 0u, spins);
    return e;
}

// Row triples on 3 x CB pixels (work items of 256 x 24 pixels): the fast instantiations
// for fields without multi-row steepness (without a uv term, then with one), the direct
// one (every phase reduced) for all other fields.  Exactly one runs.
template <int CB>
cudaError_t launch_sweep_rows(dim3 grid, cudaStream_t s, const float4* coef, const int2* it_tiles,
                              const int2* items, int n_items, int tiles_x, int n_blocks, int nx,
                              int ny, const double2* airy, int n_regions, double* moments,
                              int* counter, const unsigned* flags, uint32_t spins) {
    constexpr unsigned kAny = gbd::kFlagWide | gbd::kFlagSteep | gbd::kFlagColSteep |
                              gbd::kFlagCross | gbd::kFlagSteepRows;
    constexpr size_t smem = sweep_rows_smem(CB), smem_x = sweep_rows_smem(CB, true);
    cudaError_t e = cudaFuncSetAttribute(sweep_rows_kernel<CB, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_rows_kernel<CB, true, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_x);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_rows_kernel<CB, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sweep_rows_kernel<CB, true><<<grid, kThreads, smem, s>>>(
        coef, it_tiles, items, n_items, tiles_x, n_blocks, nx, ny, airy, n_regions, moments,
        counter, flags, kAny, 0u, 0u, spins);
    sweep_rows_kernel<CB, true, true><<<grid, kThreads, smem_x, s>>>(
        coef, it_tiles, items, n_items, tiles_x, n_blocks, nx, ny, airy, n_regions, moments,
        counter, flags, kAny, gbd::kFlagCross, 0u, spins);
    sweep_rows_kernel<CB, false><<<grid, kThreads, smem, s>>>(
        coef, it_tiles, items, n_items, tiles_x, n_blocks, nx, ny, airy, n_regions, moments,
        counter, flags, 0u, 0u, kAny & ~gbd::kFlagCross, spins);
    return cudaGetLastError();
}

struct SweepShape {
    int rb, cb, scheme;
    sweep_launch_fn fn;
    const void* kernel;
    size_t smem;
};

const SweepShape kSweepShapes[] = {
    {1, 4, GBD_SCHEME_DIRECT, launch_sweep<1, 4>, (const void*)sweep_kernel<1, 4, false, false, false>,
     sweep_smem(1, 4, false)},
    {2, 2, GBD_SCHEME_DIRECT, launch_sweep<2, 2>, (const void*)sweep_kernel<2, 2, false, false, false>,
     sweep_smem(2, 2, false)},
    {2, 4, GBD_SCHEME_DIRECT, launch_sweep<2, 4>, (const void*)sweep_kernel<2, 4, false, false, false>,
     sweep_smem(2, 4, false)},
    {4, 2, GBD_SCHEME_DIRECT, launch_sweep<4, 2>, (const void*)sweep_kernel<4, 2, false, false, false>,
     sweep_smem(4, 2, false)},
    {2, 4, GBD_SCHEME_ROW_PAIR, launch_sweep_pair<4>,
     (const void*)sweep_kernel<2, 4, false, true, false>, sweep_smem(2, 4, false)},
    {2, 8, GBD_SCHEME_ROW_PAIR, launch_sweep_pair<8>,
     (const void*)sweep_kernel<2, 8, false, true, true, false>, sweep_smem(2, 8, true)},
    {3, 8, GBD_SCHEME_ROW_PAIR, launch_sweep_rows<8>, (const void*)sweep_rows_kernel<8, true>,
     sweep_rows_smem(8)},
};

const SweepShape* find_sweep_shape(int rb, int cb, int scheme) {
    for (const auto& e : kSweepShapes)
        if (e.rb == rb && e.cb == cb && e.scheme == scheme) return &e;
    return nullptr;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// ------------------------------------------------------------------- plan --

struct gbd_sweep_plan {
    gbd_trace_params tp;
    bool mirrors = false;   // trace through `mp` (real rays) instead of the thin lens `tp`
    gbd_mirror_params mp{};
    gbd_project_params pp{};
    double lam_fnum, r3;
    Regions regions;
    int n_inst, max_n, rb, cb, scheme, tiles_x, tiles_y, n_blocks, n_items;
    int64_t total_tiles, total_beamlets;
    double evals;
    std::vector<gbd_instance_dev> inst;
    std::vector<int> rbase, rows;  // per-instance row tables of the batched trace
    std::vector<int2> inst_tiles;
    std::vector<int2> items;
    size_t off_inst, off_itiles, off_items, off_airy, off_moments, off_counter, off_coef, bytes;
    size_t off_rbase, off_rows;
    char* ws = nullptr;
    int device = -1;
    cudaGraphExec_t graph = nullptr;
    double* graph_scores = nullptr;
    cudaStream_t graph_stream = nullptr;
    uint32_t graph_spins = 0;  // wait limit baked into the captured launch
    int graph_device = -1;     // device whose SM count and occupancy sized its grid
};

// The status word: copied into pinned host memory on the caller's stream (gbd_sync), and
// cleared once it has been reported.
cudaError_t gbd_sweep_status_fetch(unsigned* host, cudaStream_t s) {
    return cudaMemcpyFromSymbolAsync(host, g_sweep_status, sizeof(unsigned), 0,
                                     cudaMemcpyDeviceToHost, s);
}
void gbd_sweep_status_clear() {
    const unsigned zero = 0;
    cudaMemcpyToSymbol(g_sweep_status, &zero, sizeof(zero));
}

static gbd_status sweep_enqueue(gbd_sweep_plan* P, double* scores, cudaStream_t s) {
    const SweepShape* sh = find_sweep_shape(P->rb, P->cb, P->scheme);
    int occ = 0;
    cudaFuncSetAttribute(sh->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh->smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sh->kernel, kThreads, sh->smem) !=
            cudaSuccess ||
        occ < 1)
        occ = 1;
    char* w = P->ws;
    // the first 256 bytes hold the work counter (offset 0) and the wide-phase flag (64)
    int* counter = reinterpret_cast<int*>(w + P->off_counter);
    unsigned* wide = reinterpret_cast<unsigned*>(w + P->off_counter + 64);
    float4* coef = reinterpret_cast<float4*>(w + P->off_coef);
    cudaError_t e = cudaMemsetAsync(w + P->off_counter, 0, 256, s);
    if (e == cudaSuccess)
        e = gbd_launch_trace_project(P->tp, P->mirrors ? &P->mp : nullptr, P->n_inst,
                                     reinterpret_cast<const gbd_instance_dev*>(w + P->off_inst),
                                     reinterpret_cast<const int*>(w + P->off_rbase),
                                     reinterpret_cast<const int*>(w + P->off_rows),
                                     P->total_tiles * gbd::kTile, P->pp, coef, wide, s);
    if (e == cudaSuccess) {
        const int grid = std::max(1, std::min(P->n_items, occ * gbd_sm_count()));
        e = sh->fn(dim3(grid), s, coef, reinterpret_cast<const int2*>(w + P->off_itiles),
                   reinterpret_cast<const int2*>(w + P->off_items), P->n_items, P->tiles_x,
                   P->n_blocks, P->pp.nx, P->pp.ny, reinterpret_cast<const double2*>(w + P->off_airy),
                   P->regions.n, reinterpret_cast<double*>(w + P->off_moments), counter, wide,
                   gbd_wait_spins());
    }
    if (e == cudaSuccess) {
        sweep_finalize_kernel<<<(P->n_inst + 127) / 128, 128, 0, s>>>(
            reinterpret_cast<const double*>(w + P->off_moments), P->n_inst, P->n_blocks,
            P->regions.n, scores);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
    return GBD_OK;
}

static void sweep_layout(gbd_sweep_plan* P, int nx, int ny) {
    size_t off = 0;
    P->off_counter = off;
    off += 256;
    P->off_inst = off;
    off = align256(off + sizeof(gbd_instance_dev) * P->n_inst);
    P->off_itiles = off;
    off = align256(off + sizeof(int2) * P->n_inst);
    P->off_rbase = off;
    off = align256(off + sizeof(int) * P->rbase.size());
    P->off_rows = off;
    off = align256(off + sizeof(int) * P->rows.size());
    P->off_items = off;
    off = align256(off + sizeof(int2) * P->items.size());
    P->off_airy = off;
    off = align256(off + sizeof(double2) * (size_t)nx * ny);
    P->off_moments = off;
    off = align256(off + sizeof(double) * (1 + 4 * P->regions.n) * (size_t)P->n_inst * P->n_blocks);
    P->off_coef = off;
    off = align256(off + (size_t)P->total_tiles * gbd::kMixedTileBytes);
    P->bytes = off;
}

// Plan of a sweep through the thin-lens system `tp` or, when `mp` is not null, through
// the mirror sequence `mp`; lam_fnum = lambda F# sets the Airy pattern's scale.
static gbd_status sweep_create(const gbd_trace_params& tp, const gbd_mirror_params* mp,
                               double wavelength, double diameter, double lam_fnum,
                               const int32_t* n_across, const double* overlap_factor,
                               const double* waist_ratio, int32_t n_instances,
                               const gbd_detector* detector, const gbd_shape* shape,
                               gbd_sweep_plan** plan) {
    // real-ray traced beamlets carry a uv term (the mirrors' small astigmatism): mirror
    // sweeps default to the row pairs, which carry it along the row (the App. B telescope's
    // 1024-instance sweep: 349 ms; scores within 9e-5 of the oracle's where the two paths
    // differ most); the row triples with per-column row factors take 340 ms but sit up to
    // 2.2e-4 from the oracle there (643 ms when they evaluated these fields directly)
    gbd_status st = gbd_check_detector(detector);
    if (st != GBD_OK) return st;
    if (!(isfinite(diameter) && diameter > 0.0))
        return gbd_set_error(GBD_EINVAL, "diameter must be finite and > 0");
    if (n_instances < 1 || n_instances > (1 << 20))
        return gbd_set_error(GBD_EINVAL, "n_instances must be in [1, 2^20]");
    if (!n_across || !overlap_factor || !waist_ratio)
        return gbd_set_error(GBD_EINVAL, "instance arrays are NULL");
    // default: row triples on 8 columns (or row pairs on 4, whichever fits the width)
    const int cb = shape ? shape->cols_per_thread : gbd_auto_cols(detector->nx, 4);
    const int rb = shape ? shape->rows_per_thread : (cb == 8 && !mp ? 3 : 2);
    const int scheme = shape ? shape->scheme : GBD_SCHEME_ROW_PAIR;
    if (!find_sweep_shape(rb, cb, scheme))
        return gbd_set_error(GBD_EINVAL, "unsupported sweep shape");
    gbd_sweep_plan* P = new gbd_sweep_plan();
    P->tp = tp;
    if (mp) {
        P->mirrors = true;
        P->mp = *mp;
    }
    P->pp = gbd_make_project_params(wavelength, detector);
    P->lam_fnum = lam_fnum;
    P->r3 = 10.173468135062722 * P->lam_fnum / M_PI;  // third zero of J1
    P->regions.n = 1;
    P->regions.lo[0] = 0.0;
    P->regions.hi[0] = 10.173468135062722 / M_PI;
    P->n_inst = n_instances;
    P->rb = rb;
    P->cb = cb;
    P->scheme = scheme;
    P->tiles_x = (detector->nx + 32 * cb - 1) / (32 * cb);
    P->tiles_y = (detector->ny + 8 * rb - 1) / (8 * rb);
    P->n_blocks = P->tiles_x * P->tiles_y;
    P->max_n = 0;
    int64_t tile = 0;
    P->total_beamlets = 0;
    for (int k = 0; k < n_instances; ++k) {
        gbd_pupil pu{diameter, n_across[k], 0};
        const int32_t nb = gbd_beamlet_count(&pu);
        if (nb < 1 || !(overlap_factor[k] > 0.0) || !(waist_ratio[k] > 0.0) ||
            !isfinite(overlap_factor[k]) || !isfinite(waist_ratio[k])) {
            delete P;
            return gbd_set_error(GBD_EINVAL, "instance with invalid n_across / OF / WR");
        }
        const int nt = (nb + gbd::kTile - 1) / gbd::kTile;
        // first beamlet of each grid row: rows are contiguous runs of centres with
        // (2i-(N-1))^2 + (2j-(N-1))^2 <= N^2
        {
            const long long N = n_across[k];
            P->rbase.push_back((int)P->rows.size());
            int acc = 0;
            for (long long j = 0; j < N; ++j) {
                P->rows.push_back(acc);
                const long long b = 2 * j - (N - 1), r2 = N * N - b * b;
                for (long long a = -(N - 1); a <= N - 1; a += 2)
                    if (a * a <= r2) ++acc;
            }
            if (acc != nb) {
                delete P;
                return gbd_set_error(GBD_EINVAL, "internal: row table disagrees with the count");
            }
        }
        gbd_instance_dev I;
        I.n_across = n_across[k];
        I.reserved = nb;
        I.offset = tile * gbd::kTile;
        I.overlap_factor = overlap_factor[k];
        I.waist_ratio = waist_ratio[k];
        I.grid = gbd_make_grid(diameter, wavelength, n_across[k], overlap_factor[k],
                               waist_ratio[k]);
        P->inst.push_back(I);
        P->inst_tiles.push_back(make_int2((int)tile, nt));
        tile += nt;
        P->total_beamlets += nb;
        P->max_n = std::max(P->max_n, (int)n_across[k]);
    }
    if (tile > INT32_MAX / 2) {
        delete P;
        return gbd_set_error(GBD_EINVAL, "sweep too large");
    }
    P->total_tiles = tile;
    P->evals = (double)P->total_beamlets * detector->nx * detector->ny;
    // longest first: instances with more beamlet tiles run first
    std::vector<int> order(n_instances);
    for (int k = 0; k < n_instances; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return P->inst_tiles[a].y > P->inst_tiles[b].y; });
    for (int k : order)
        for (int t = 0; t < P->n_blocks; ++t) P->items.push_back(make_int2(k, t));
    P->n_items = (int)P->items.size();
    sweep_layout(P, detector->nx, detector->ny);
    *plan = P;
    return GBD_OK;
}

extern "C" {

gbd_status gbd_sweep_plan_create(const gbd_system* system, double diameter, const int32_t* n_across,
                                 const double* overlap_factor, const double* waist_ratio,
                                 int32_t n_instances, const gbd_detector* detector,
                                 const gbd_shape* shape, gbd_sweep_plan** plan) {
    GBD_NVTX_RANGE("gbd_sweep_plan_create");
    if (!plan) return gbd_set_error(GBD_EINVAL, "plan is NULL");
    *plan = nullptr;
    gbd_status st = gbd_check_system(system);
    if (st != GBD_OK) return st;
    if (isinf(system->focal_length))
        return gbd_set_error(GBD_EINVAL, "the Airy score needs a lens (finite focal length)");
    if (!(isfinite(diameter) && diameter > 0.0))
        return gbd_set_error(GBD_EINVAL, "diameter must be finite and > 0");
    return sweep_create(gbd_make_trace_params(system, diameter), nullptr, system->wavelength,
                        diameter, system->wavelength * fabs(system->focal_length) / diameter,
                        n_across, overlap_factor, waist_ratio, n_instances, detector, shape, plan);
}

gbd_status gbd_sweep_plan_create_mirrors(const gbd_mirror_system* system, double diameter,
                                         double f_number, const int32_t* n_across,
                                         const double* overlap_factor, const double* waist_ratio,
                                         int32_t n_instances, const gbd_detector* detector,
                                         const gbd_shape* shape, gbd_sweep_plan** plan) {
    GBD_NVTX_RANGE("gbd_sweep_plan_create_mirrors");
    if (!plan) return gbd_set_error(GBD_EINVAL, "plan is NULL");
    *plan = nullptr;
    if (!(isfinite(diameter) && diameter > 0.0))
        return gbd_set_error(GBD_EINVAL, "diameter must be finite and > 0");
    if (!(isfinite(f_number) && f_number > 0.0))
        return gbd_set_error(GBD_EINVAL, "f_number must be finite and > 0");
    gbd_mirror_params mp;
    gbd_status st = gbd_make_mirror_params(system, diameter, &mp);
    if (st != GBD_OK) return st;
    gbd_trace_params tp;
    memset(&tp, 0, sizeof(tp));
    tp.wavelength = system->wavelength;
    tp.diameter = diameter;
    tp.zdeg = -1;
    return sweep_create(tp, &mp, system->wavelength, diameter, system->wavelength * f_number,
                        n_across, overlap_factor, waist_ratio, n_instances, detector, shape, plan);
}

size_t gbd_sweep_workspace_bytes(const gbd_sweep_plan* plan) { return plan ? plan->bytes : 0; }

gbd_status gbd_sweep_set_zones(gbd_sweep_plan* P, int32_t n_zones, const double* lo,
                               const double* hi) {
    if (!P) return gbd_set_error(GBD_EINVAL, "plan is NULL");
    if (P->ws) return gbd_set_error(GBD_EINVAL, "set zones before gbd_sweep_bind");
    if (n_zones < 0 || n_zones > kMaxRegions - 1)
        return gbd_set_error(GBD_EINVAL, "n_zones must be in [0, 7]");
    if (n_zones > 0 && (!lo || !hi)) return gbd_set_error(GBD_EINVAL, "zone bounds are NULL");
    for (int z = 0; z < n_zones; ++z)
        if (!(lo[z] >= 0.0) || !(hi[z] > lo[z]) || !isfinite(hi[z]))
            return gbd_set_error(GBD_EINVAL, "zone bounds must satisfy 0 <= lo < hi < inf");
    P->regions.n = 1 + n_zones;
    for (int z = 0; z < n_zones; ++z) {
        P->regions.lo[1 + z] = lo[z];
        P->regions.hi[1 + z] = hi[z];
    }
    sweep_layout(P, P->pp.nx, P->pp.ny);
    return GBD_OK;
}

gbd_status gbd_sweep_info(const gbd_sweep_plan* plan, double* evals, int64_t* beamlets,
                          int32_t* items) {
    if (!plan) return gbd_set_error(GBD_EINVAL, "plan is NULL");
    if (evals) *evals = plan->evals;
    if (beamlets) *beamlets = plan->total_beamlets;
    if (items) *items = plan->n_items;
    return GBD_OK;
}

gbd_status gbd_sweep_bind(gbd_sweep_plan* P, void* workspace, size_t bytes, void* stream) {
    GBD_NVTX_RANGE("gbd_sweep_bind");
    if (!P) return gbd_set_error(GBD_EINVAL, "plan is NULL");
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return gbd_set_error(GBD_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    if (bytes < P->bytes) return gbd_set_error(GBD_ENOMEM, "sweep workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (P->graph) {
        cudaGraphExecDestroy(P->graph);
        P->graph = nullptr;
    }
    P->ws = static_cast<char*>(workspace);
    cudaGetDevice(&P->device);
    char* w = P->ws;
    cudaError_t e = cudaMemcpyAsync(w + P->off_inst, P->inst.data(),
                                    sizeof(gbd_instance_dev) * P->inst.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + P->off_itiles, P->inst_tiles.data(),
                            sizeof(int2) * P->inst_tiles.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + P->off_items, P->items.data(), sizeof(int2) * P->items.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + P->off_rbase, P->rbase.data(), sizeof(int) * P->rbase.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + P->off_rows, P->rows.data(), sizeof(int) * P->rows.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const int npix = P->pp.nx * P->pp.ny;
        airy_table_kernel<<<(npix + 255) / 256, 256, 0, s>>>(
            P->pp.nx, P->pp.ny, P->pp.px, P->pp.py, P->lam_fnum, P->regions,
            reinterpret_cast<double2*>(w + P->off_airy));
        e = cudaGetLastError();
    }
    // the host tables are read by the copies above: finish before returning
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
    return GBD_OK;
}

gbd_status gbd_sweep_run(gbd_sweep_plan* P, double* scores, void* stream) {
    GBD_NVTX_RANGE("gbd_sweep_run");
    if (!P || !P->ws) return gbd_set_error(GBD_EINVAL, "plan is NULL or not bound");
    if (!scores) return gbd_set_error(GBD_EINVAL, "scores is NULL");
    return sweep_enqueue(P, scores, static_cast<cudaStream_t>(stream));
}

gbd_status gbd_sweep_run_graph(gbd_sweep_plan* P, double* scores, void* stream) {
    GBD_NVTX_RANGE("gbd_sweep_run_graph");
    if (!P || !P->ws) return gbd_set_error(GBD_EINVAL, "plan is NULL or not bound");
    if (!scores) return gbd_set_error(GBD_EINVAL, "scores is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
        return gbd_set_error(GBD_EINVAL, "graph capture needs a created (non-default) stream");
    // the captured kernels hold the wait limit by value: a new limit needs a new capture
    const uint32_t spins = gbd_wait_spins();
    int dev = -1;
    cudaGetDevice(&dev);
    if (!P->graph || P->graph_scores != scores || P->graph_stream != s || P->graph_spins != spins ||
        P->graph_device != dev) {
        if (P->graph) {
            cudaGraphExecDestroy(P->graph);
            P->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
        gbd_status st = sweep_enqueue(P, scores, s);
        e = cudaStreamEndCapture(s, &g);
        if (st != GBD_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
        e = cudaGraphInstantiate(&P->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            P->graph = nullptr;
            return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
        }
        P->graph_scores = scores;
        P->graph_stream = s;
        P->graph_spins = spins;
        P->graph_device = dev;
    }
    cudaError_t e = cudaGraphLaunch(P->graph, s);
    if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
    return GBD_OK;
}

void gbd_sweep_plan_destroy(gbd_sweep_plan* P) {
    if (!P) return;
    if (P->graph) cudaGraphExecDestroy(P->graph);
    delete P;
}

}  // extern "C"

extern "C" gbd_status gbd_sweep_autotune(const gbd_system* system, double diameter,
                                         const int32_t* n_across, const double* overlap_factor,
                                         const double* waist_ratio, int32_t n_instances,
                                         const gbd_detector* detector, void* workspace,
                                         size_t bytes, double* scores, void* stream,
                                         gbd_shape* best) {
    if (!best) return gbd_set_error(GBD_EINVAL, "best is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return gbd_set_error(GBD_ECUDA, "autotune events");
    gbd_shape win{0, 0, 1, 1e30f, 0};
    gbd_status st = GBD_OK;
    for (const auto& sh : kSweepShapes) {
        gbd_shape cand{sh.rb, sh.cb, 1, 0.f, sh.scheme};
        gbd_sweep_plan* P = nullptr;
        st = gbd_sweep_plan_create(system, diameter, n_across, overlap_factor, waist_ratio,
                                   n_instances, detector, &cand, &P);
        if (st != GBD_OK) break;
        if (P->bytes > bytes) {
            gbd_sweep_plan_destroy(P);
            continue;
        }
        st = gbd_sweep_bind(P, workspace, bytes, stream);
        float ms = 1e30f;
        for (int rep = 0; st == GBD_OK && rep < 2; ++rep) {
            cudaEventRecord(e0, s);
            st = gbd_sweep_run(P, scores, stream);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = gbd_set_error(GBD_ECUDA, "autotune");
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = t;
        }
        gbd_sweep_plan_destroy(P);
        if (st != GBD_OK) break;
        if (ms < win.ms) {
            win = cand;
            win.ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GBD_OK) return st;
    if (win.rows_per_thread == 0) return gbd_set_error(GBD_ENOMEM, "no shape fits the workspace");
    *best = win;
    return GBD_OK;
}
