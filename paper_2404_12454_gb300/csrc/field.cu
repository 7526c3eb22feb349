// Per-(beamlet, pixel) evaluation and coherent sum (Eq. sum_gaussian evaluated with the
// plane form of Eq. collins_factored): the hot path.
//
// A CTA owns a block of pixels and a contiguous range of beamlet tiles (a "split").  The
// projected beamlet records are streamed through shared memory in 64-beamlet tiles by
// the TMA bulk-copy engine (4-stage mbarrier pipeline, one elected producer thread); each
// thread keeps RB x CB pixels in registers and evaluates every beamlet of the tile on
// them.  Splits write partial fields (the mixed kernels round their compensated (hi, lo)
// sums to FP32 pairs, the FP64 kernels write FP64), summed in a fixed order in FP64 by a
// second kernel that
// also applies the per-pixel carrier of a tilted plane.
//
// Mixed path, per (beamlet, pixel): 4 FFMA for the quadratic form (row terms shared across
// the thread's columns; phase coefficients in radians), ex2 / sin / cos on the MUFU pipe,
// 2 FFMA to accumulate.  If the projection found a beamlet whose phase can exceed 128 rad
// on the detector, the instantiation that reduces every phase exactly runs instead.  The sum runs in FP32 over each 64-beamlet tile and is folded into a
// (hi, lo) pair with TwoSum between tiles.
#include <math.h>

#include "field_core.cuh"
#include "gbd_internal.cuh"

namespace {

using gbd::kStages;
using gbd::kThreads;
using gbd::kWarps;

__device__ unsigned int g_field_status = 0;

__device__ __forceinline__ void record_timeout() { atomicOr(&g_field_status, gbd::kStatusTimeout); }

// WIDE selects the instantiation with per-pixel phase reduction, PAIR (RB = 2) the row-pair
// evaluation.  Several instantiations are launched for one field; each returns at once
// unless the projection's flag word, masked by `mask`, equals `want` and (if `anyof` is
// not 0) shares a bit with `anyof`.
// WIDE: 0 narrow phases, 1 every phase reduced exactly, kWideByFlag either, per the
// flag word's wide bit (the direct steep fallback of the row-pair launches).
constexpr int kWideByFlag = 2;
template <int RB, int CB, int WIDE, bool PAIR, bool LOOP = false>
__global__ void __launch_bounds__(kThreads, 2)
    field_mixed_kernel(const float4* __restrict__ coef, int n_tiles, int tiles_per_split, int nx,
                       int ny, float2* __restrict__ partial, const unsigned* __restrict__ flags,
                       unsigned mask, unsigned want, unsigned anyof, uint32_t spins) {
    static_assert(!PAIR || RB == 2, "row pairs need two rows per thread");
    const unsigned fw = *flags;
    if ((fw & mask) != want || (anyof != 0u && (fw & anyof) == 0u)) return;
    constexpr int kTileF4 = gbd::kMixedFields * gbd::kTile;
    __shared__ __align__(128) float4 stage[kStages][kTileF4];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
    __shared__ int flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    gbd::init_stream_barriers(full, empty, tid);
    // split `split` of the beamlets into its partial field, the CTA's stream starting at its
    // g-th tile; false after a failed wait (the CTA then leaves)
    auto run = [&](int split, int g) -> bool {
        const int t0 = split * tiles_per_split;
        gbd::TileStream<float4, kTileF4> ts{stage, full, empty, coef + (size_t)t0 * kTileF4,
                                            min(n_tiles - t0, tiles_per_split), g,
                                            gbd::kMixedTileBytes, 0};
        bool ok = ts.start(tid, spins, &flag);

        const int col0 = blockIdx.x * (32 * CB) + lane;
        const int row0 = blockIdx.y * (8 * RB) + warp;
        float colf[CB], rowf[RB];
#pragma unroll
        for (int c = 0; c < CB; ++c) colf[c] = (float)(col0 + 32 * c);
#pragma unroll
        for (int r = 0; r < RB; ++r) rowf[r] = (float)(row0 + 8 * r);

        float2 acc[RB][CB], hi[RB][CB], lo[RB][CB];
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int c = 0; c < CB; ++c) acc[r][c] = hi[r][c] = lo[r][c] = make_float2(0.f, 0.f);

        int k = 0;
        for (; ok && k < ts.nt; ++k) {
            if (!ts.acquire(k, spins)) {
                ok = false;
                break;
            }
            if constexpr (PAIR) {
                gbd::mixed_tile_pair<CB, WIDE == 1>(ts.tile(k), colf, rowf[0], acc);
            } else if constexpr (WIDE == kWideByFlag) {  // the steep fallback: both in one
                if (fw & gbd::kFlagWide)
                    gbd::mixed_tile<RB, CB, true>(ts.tile(k), colf, rowf, acc);
                else
                    gbd::mixed_tile<RB, CB, false>(ts.tile(k), colf, rowf, acc);
            } else {
                gbd::mixed_tile<RB, CB, WIDE == 1>(ts.tile(k), colf, rowf, acc);
            }
            gbd::mixed_fold<RB, CB>(acc, hi, lo);
            if (!ts.release(k, lane, warp, spins)) {
                ok = false;
                ++k;
                break;
            }
        }
        if (!ok) {
            record_timeout();
            if (tid == 0) ts.drain(k, spins);
            return false;
        }
        const size_t npix = (size_t)nx * ny;
        float2* out = partial + (size_t)split * npix;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int row = row0 + 8 * r;
            if (row >= ny) continue;
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const int col = col0 + 32 * c;
                if (col >= nx) continue;
                out[(size_t)row * nx + col] = gbd::round_pair(hi[r][c], lo[r][c]);
            }
        }
        return true;
    };
    if constexpr (LOOP) {
        // a fallback launch (fallback_z): splits blockIdx.z, blockIdx.z + gridDim.z, ...
        const int nsplit = (n_tiles + tiles_per_split - 1) / tiles_per_split;
        int g = 0;  // tiles this CTA has streamed (keeps the barrier phases in step)
        for (int split = blockIdx.z; split < nsplit; split += gridDim.z) {
            if (!run(split, g)) return;
            g += min(n_tiles - split * tiles_per_split, tiles_per_split);
        }
    } else {
        run(blockIdx.z, 0);
    }
}

// Row pairs on 2 x CB pixels per thread with the compensation pairs in shared memory
// (wider blocks amortise the per-beamlet row terms over more columns).  Dynamic shared
// memory: the kStages record stages, then 2 CB x kThreads float4 (hi, lo) slots, then
// (narrow instantiation) each warp's row terms of the current tile, kPairRowF4 x kTile
// float4 per warp.
template <int CB, bool WIDE, bool CROSS = true, bool LOOP = false>
__global__ void __launch_bounds__(kThreads, 2)
    field_mixed_pair_smem_kernel(const float4* __restrict__ coef, int n_tiles, int tiles_per_split,
                                 int nx, int ny, float2* __restrict__ partial,
                                 const unsigned* __restrict__ flags, unsigned mask, unsigned want,
                                 unsigned anyof, uint32_t spins) {
    const unsigned fw = *flags;
    if ((fw & mask) != want || (anyof != 0u && (fw & anyof) == 0u)) return;
    constexpr int kTileF4 = gbd::kMixedFields * gbd::kTile;
    extern __shared__ __align__(128) float4 dyn4[];
    float4(*stage)[kTileF4] = reinterpret_cast<float4(*)[kTileF4]>(dyn4);
    float4* comp = dyn4 + kStages * kTileF4;
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
    __shared__ int flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4* ent = comp + 2 * CB * kThreads + warp * (gbd::kPairRowF4 * gbd::kTile);
    gbd::init_stream_barriers(full, empty, tid);
    // split `split` into its partial field (as field_mixed_kernel's)
    auto run = [&](int split, int g) -> bool {
        // each thread clears and later reads only its own compensation slots
#pragma unroll
        for (int m = 0; m < 2 * CB; ++m)
            comp[m * kThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int t0 = split * tiles_per_split;
        gbd::TileStream<float4, kTileF4> ts{stage, full, empty, coef + (size_t)t0 * kTileF4,
                                            min(n_tiles - t0, tiles_per_split), g,
                                            gbd::kMixedTileBytes, 0};
        bool ok = ts.start(tid, spins, &flag);

        const int col0 = blockIdx.x * (32 * CB) + lane;
        const int row0 = blockIdx.y * 16 + warp;
        float colf[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c) colf[c] = (float)(col0 + 32 * c);
        const float rowf = (float)row0;

        float2 acc[2][CB];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < CB; ++c) acc[r][c] = make_float2(0.f, 0.f);

        int k = 0;
        for (; ok && k < ts.nt; ++k) {
            if (!ts.acquire(k, spins)) {
                ok = false;
                break;
            }
            if constexpr (WIDE) {
                gbd::mixed_tile_pair<CB, WIDE>(ts.tile(k), colf, rowf, acc);
            } else {
                __syncwarp();  // every lane is done with the previous tile's row terms
                gbd::mixed_pair_rows<CROSS>(ts.tile(k), rowf, ent, lane);
                __syncwarp();
                gbd::mixed_tile_pair_rows<CB, CROSS>(ts.tile(k), ent, colf, acc);
            }
            gbd::mixed_fold_smem<2, CB>(acc, comp, tid);
            if (!ts.release(k, lane, warp, spins)) {
                ok = false;
                ++k;
                break;
            }
        }
        if (!ok) {
            record_timeout();
            if (tid == 0) ts.drain(k, spins);
            return false;
        }
        const size_t npix = (size_t)nx * ny;
        float2* out = partial + (size_t)split * npix;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int row = row0 + 8 * r;
            if (row >= ny) continue;
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const int col = col0 + 32 * c;
                if (col >= nx) continue;
                const float4 v = comp[(r * CB + c) * kThreads + tid];
                out[(size_t)row * nx + col] =
                    gbd::round_pair(make_float2(v.x, v.y), make_float2(v.z, v.w));
            }
        }
        return true;
    };
    if constexpr (LOOP) {
        // a fallback launch (fallback_z): splits blockIdx.z, blockIdx.z + gridDim.z, ...
        const int nsplit = (n_tiles + tiles_per_split - 1) / tiles_per_split;
        int g = 0;  // tiles this CTA has streamed (keeps the barrier phases in step)
        for (int split = blockIdx.z; split < nsplit; split += gridDim.z) {
            if (!run(split, g)) return;
            g += min(n_tiles - split * tiles_per_split, tiles_per_split);
        }
    } else {
        run(blockIdx.z, 0);
    }
}

// Split partials of pixel p summed in split order with Neumaier's compensation in FP32 (the
// partials were written by other CTAs: read through L2).
__device__ __forceinline__ void neumaier_add(float& sum, float& comp, float x) {
    const float t = __fadd_rn(sum, x);
    comp = __fadd_rn(comp, fabsf(sum) >= fabsf(x) ? __fadd_rn(__fsub_rn(sum, t), x)
                                                   : __fadd_rn(__fsub_rn(x, t), sum));
    sum = t;
}

}  // namespace

namespace gbd {
__device__ __forceinline__ float2 sum_partials(const float2* __restrict__ partial, size_t npix,
                                               size_t p, int splits) {
    float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;
    int s = 0;
    for (; s + 8 <= splits; s += 8) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(partial + (size_t)(s + u) * npix + p);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            neumaier_add(sr, cr, v[u].x);
            neumaier_add(si, ci, v[u].y);
        }
    }
    for (; s < splits; ++s) {
        const float2 v = __ldcg(partial + (size_t)s * npix + p);
        neumaier_add(sr, cr, v.x);
        neumaier_add(si, ci, v.y);
    }
    return make_float2(__fadd_rn(sr, cr), __fadd_rn(si, ci));
}

// The same sum for NP pixels at once (NP x 8 loads in flight instead of 8: the sum of a
// whole pixel block by one CTA is latency-bound otherwise); each pixel's additions are in
// the same order as sum_partials', so the results are the same bits.
template <int NP>
__device__ __forceinline__ void sum_partials_n(const float2* __restrict__ partial, size_t npix,
                                               const size_t (&p)[NP], int splits,
                                               float2 (&res)[NP]) {
    float sr[NP], si[NP], cr[NP], ci[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) sr[q] = si[q] = cr[q] = ci[q] = 0.f;
    int s = 0;
    for (; s + 8 <= splits; s += 8) {
        float2 v[NP][8];
#pragma unroll
        for (int q = 0; q < NP; ++q)
#pragma unroll
            for (int u = 0; u < 8; ++u) v[q][u] = __ldcg(partial + (size_t)(s + u) * npix + p[q]);
#pragma unroll
        for (int q = 0; q < NP; ++q)
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                neumaier_add(sr[q], cr[q], v[q][u].x);
                neumaier_add(si[q], ci[q], v[q][u].y);
            }
    }
    for (; s < splits; ++s)
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const float2 v = __ldcg(partial + (size_t)s * npix + p[q]);
            neumaier_add(sr[q], cr[q], v.x);
            neumaier_add(si[q], ci[q], v.y);
        }
#pragma unroll
    for (int q = 0; q < NP; ++q) res[q] = make_float2(__fadd_rn(sr[q], cr[q]), __fadd_rn(si[q], ci[q]));
}

// Slab pixel (row, col) of the summed field into the output window, carrier applied (its
// phase in turns reduced in FP64, the rotation in FP32).
__device__ __forceinline__ void reduce_store(const ReduceOut& ro, int nx, int row, int col,
                                             float2 v) {
    const int orow = row - ro.skip;
    if (orow < 0 || orow >= ro.out_rows) return;
    float re = v.x, im = v.y;
    if (ro.cx != 0.0 || ro.cy != 0.0) {
        const int j = row + ro.row0;
        const double turns = ro.cx * (col - nx / 2) + ro.cy * (j - ro.ny / 2);
        float sn, cs;
        sincospif(2.0f * (float)(turns - rint(turns)), &sn, &cs);
        const float r2 = re * cs - im * sn;
        im = re * sn + im * cs;
        re = r2;
    }
    static_cast<float2*>(ro.out)[(size_t)orow * nx + col] = make_float2(re, im);
}
}  // namespace gbd

namespace {

// Row triples or quadruples on RB x CB pixels per thread (rows 8 apart, columns 32
// apart): without a uv term mixed_tile_rows (or its packed form), with one (CROSS)
// mixed_tile_rows_cross with the per-column row factors.  The sums stay in FP32 registers
// over the whole split, so the launch requires short splits (at most kRowsMaxTiles tiles
// = 1,024 beamlets); the reduction sums the splits with compensation.  Dynamic shared
// memory: the kStages record stages, then each warp's row terms of the current tile.
//
// The grid runs the splits of a pixel block next to each other (blockIdx.x = split, y and z
// = the pixel block), so a block's split partials are written close together in time and
// stay in L2.  Each CTA writes its partial, then bumps the block's counter; the CTA that
// completes the block sums the block's partials in split order with Neumaier's compensation
// (the reduction kernel's arithmetic, so the bits are the same), applies the tilted plane's
// carrier and writes the field rows of the output window.  No CTA waits for another.
constexpr int kRowsMaxTiles = 16;
template <int RB, int CB, bool CROSS = false>
__global__ void __launch_bounds__(kThreads, 2)
    field_mixed_rows_kernel(const float4* __restrict__ coef, int n_tiles, int tiles_per_split,
                            int nx, int ny, float2* __restrict__ partial,
                            const unsigned* __restrict__ flags, unsigned mask, unsigned want,
                            uint32_t spins, unsigned* __restrict__ done,
                            gbd::ReduceOut ro) {
    const unsigned fw = *flags;
    if ((fw & mask) != want) return;
    constexpr int kTileF4 = gbd::kMixedFields * gbd::kTile;
    extern __shared__ __align__(128) float4 dyn4[];
    float4(*stage)[kTileF4] = reinterpret_cast<float4(*)[kTileF4]>(dyn4);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
    __shared__ int flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr bool kX2 = !CROSS && RB == 4 && CB == 8;  // the packed quadruples
    constexpr int kEntF4 = CROSS ? gbd::kRowsCrossF4<RB> : kX2 ? gbd::kRowsX2F4 : gbd::kRowsF4;
    float4* ent = dyn4 + kStages * kTileF4 + warp * (kEntF4 * gbd::kTile);
    const int split = blockIdx.x, bx = blockIdx.y, by = blockIdx.z;
    const int t0 = split * tiles_per_split;
    gbd::init_stream_barriers(full, empty, tid);
    gbd::TileStream<float4, kTileF4> ts{stage, full, empty, coef + (size_t)t0 * kTileF4,
                                        max(0, min(n_tiles - t0, tiles_per_split)), 0,
                                        gbd::kMixedTileBytes, 0};
    bool ok = ts.start(tid, spins, &flag);

    const int col0 = bx * (32 * CB) + lane;
    // the block's first row in slab coordinates: blocks sit at detector rows that are
    // multiples of 8 RB, so every pixel is computed by the same thread row as in the whole
    // field.  Slabs start at multiples of the launch's row-block height, which the blocks
    // without a uv term divide; the uv-term triples behind a 4 x 8 pick (24 rows against
    // a 32-row alignment) may start inside their first block and evaluate the rows before
    // the slab without storing them (kAnchor)
    constexpr bool kAnchor = CROSS;
    const int rb0 = by * (8 * RB) - (kAnchor ? ro.row0 % (8 * RB) : 0);
    const int row0 = rb0 + warp;
    float colf[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) colf[c] = (float)(col0 + 32 * c);
    const float rowf = (float)row0;

    float2 acc[RB][CB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c) acc[r][c] = make_float2(0.f, 0.f);

    int k = 0;
    for (; ok && k < ts.nt; ++k) {
        if (!ts.acquire(k, spins)) {
            ok = false;
            break;
        }
        __syncwarp();  // every lane is done with the previous tile's row terms
        if constexpr (CROSS)
            gbd::mixed_rows_cross_terms<RB>(ts.tile(k), rowf, ent, lane);
        else
            gbd::mixed_rows_terms<RB, kX2>(ts.tile(k), rowf, ent, lane);
        __syncwarp();
        // packed FP32x2 arithmetic where it pays: on airy_large the 4 x 8 shape (2 CTAs per
        // SM) ran 2.85 ms with it against 3.02 without; 4 x 4 (2.92 -> 3.00 ms) and 3 x 8
        // (2.99 -> 3.30 ms) are faster with scalar instructions
        if constexpr (CROSS)
            gbd::mixed_tile_rows_cross<RB, CB>(ent, colf, acc);
        else if constexpr (RB == 4 && CB == 8)
            gbd::mixed_tile_rows_x2<RB, CB>(ent, colf, acc);
        else
            gbd::mixed_tile_rows<RB, CB>(ent, colf, acc);
        if (!ts.release(k, lane, warp, spins)) {
            ok = false;
            ++k;
            break;
        }
    }
    if (!ok) {
        // the partial is still written (garbage) and counted, so the block completes
        record_timeout();
        if (tid == 0) ts.drain(k, spins);
    }
    const size_t npix = (size_t)nx * ny;
    float2* out = partial + (size_t)split * npix;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const int row = row0 + 8 * r;
        if ((kAnchor && row < 0) || row >= ny) continue;
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const int col = col0 + 32 * c;
            if (col >= nx) continue;
            out[(size_t)row * nx + col] = acc[r][c];
        }
    }
    // the last CTA of this pixel block to finish sums the block's partials
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned blk = (unsigned)(by * gridDim.y + bx);
        last = atomicAdd(&done[blk], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int splits = gridDim.x;
    // the thread's pixels 2 at a time, 16 loads in flight (off-detector ones read pixel 0
    // and are not stored; 4 at a time would cost the 4 x 4 shape its third CTA per SM)
    constexpr int kNP = 2;
    static_assert((RB * CB) % kNP == 0, "pixel groups");
#pragma unroll 1
    for (int m0 = 0; m0 < RB * CB; m0 += kNP) {
        size_t pq[kNP];
        float2 v[kNP];
#pragma unroll
        for (int q = 0; q < kNP; ++q) {
            const int row = row0 + 8 * ((m0 + q) / CB), col = col0 + 32 * ((m0 + q) % CB);
            pq[q] = (!kAnchor || row >= 0) && row < ny && col < nx ? (size_t)row * nx + col : 0;
        }
        gbd::sum_partials_n<kNP>(partial, npix, pq, splits, v);
#pragma unroll
        for (int q = 0; q < kNP; ++q) {
            const int row = row0 + 8 * ((m0 + q) / CB), col = col0 + 32 * ((m0 + q) % CB);
            if ((!kAnchor || row >= 0) && row < ny && col < nx)
                gbd::reduce_store(ro, nx, row, col, v[q]);
        }
    }
    // The block's partials are consumed: drop their L2 lines instead of letting them be
    // written back to HBM.  Only when every 128-byte line of the block's rows belongs to
    // this block (rows of a multiple of 16 pixels; the block spans 32 CB pixels = 2 CB lines).
    if ((nx & 15) == 0) {
        __syncthreads();  // every thread has read its pixels' partials
        const int r_lo = kAnchor ? max(rb0, 0) : rb0;
        const int rows_here = min(rb0 + 8 * RB, ny) - r_lo;
        const int lines_per_row = (min(32 * CB, nx - bx * (32 * CB)) * 8 + 127) / 128;
        const int per_split = rows_here * lines_per_row;
        const long long total = (long long)splits * per_split;
        for (long long q = tid; q < total; q += kThreads) {
            const int s = (int)(q / per_split), rem = (int)(q % per_split);
            const int row = r_lo + rem / lines_per_row, line = rem % lines_per_row;
            const float2* a = partial + (size_t)s * npix + (size_t)row * nx + bx * (32 * CB);
            gbd::discard_l2_line(reinterpret_cast<const char*>(a) + 128 * line);
        }
    }
}

// The flag bits that hand a field from the multi-row kernels to the row pairs.
constexpr unsigned kRowsNarrow = gbd::kFlagWide | gbd::kFlagSteep | gbd::kFlagColSteep |
                                 gbd::kFlagCross | gbd::kFlagSteepRows;
// The bits that hand it to the row pairs whether or not it has a uv term (the multi-row
// kernels store the field themselves when these are all clear).
constexpr unsigned kRowsTaken = kRowsNarrow & ~gbd::kFlagCross;

template <bool CROSS = false, int RB = 4, int CB = 4>
constexpr size_t rows_smem_bytes() {
    return (size_t)kStages * gbd::kMixedTileBytes +
           (size_t)kWarps *
               (CROSS ? gbd::kRowsCrossF4<RB>
                      : RB == 4 && CB == 8 ? gbd::kRowsX2F4 : gbd::kRowsF4) *
               gbd::kTile * sizeof(float4);
}

template <int CB>
constexpr size_t pair_smem_bytes() {
    return (size_t)kStages * gbd::kMixedTileBytes + (size_t)2 * CB * kThreads * sizeof(float4) +
           (size_t)kWarps * gbd::kPairRowF4 * gbd::kTile * sizeof(float4);
}

template <int RB, int CB>
__global__ void __launch_bounds__(kThreads)
    field_f64_kernel(const double2* __restrict__ coef, int n_tiles, int tiles_per_split, int nx,
                     int ny, double2* __restrict__ partial, uint32_t spins) {
    constexpr int kTileD2 = gbd::kF64Fields * gbd::kTile;
    extern __shared__ __align__(128) double2 dyn[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
    __shared__ int flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t0 = blockIdx.z * tiles_per_split;
    gbd::init_stream_barriers(full, empty, tid);
    gbd::TileStream<double2, kTileD2> ts{reinterpret_cast<double2(*)[kTileD2]>(dyn), full, empty,
                                         coef + (size_t)t0 * kTileD2,
                                         min(n_tiles - t0, tiles_per_split), 0,
                                         gbd::kF64TileBytes, 0};
    bool ok = ts.start(tid, spins, &flag);

    const int col0 = blockIdx.x * (32 * CB) + lane;
    const int row0 = blockIdx.y * (8 * RB) + warp;
    double acc_re[RB][CB], acc_im[RB][CB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c) acc_re[r][c] = acc_im[r][c] = 0.0;

    int k = 0;
    for (; ok && k < ts.nt; ++k) {
        if (!ts.acquire(k, spins)) {
            ok = false;
            break;
        }
        const double2* st = ts.tile(k);
#pragma unroll 1
        for (int b = 0; b < gbd::kTile; ++b) {
            // (i0, j0) (a0, p0) (a1u, p1u) (a1v, p1v) (auu, puu) (auv, puv) (avv, pvv)
            const double2 ij = st[b];
            const double2 c0 = st[gbd::kTile + b];
            const double2 cu = st[2 * gbd::kTile + b];
            const double2 cv = st[3 * gbd::kTile + b];
            const double2 cuu = st[4 * gbd::kTile + b];
            const double2 cuv = st[5 * gbd::kTile + b];
            const double2 cvv = st[6 * gbd::kTile + b];
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const double tv = (double)(row0 + 8 * r) - ij.y;
                const double ra = fma(tv, fma(cvv.x, tv, cv.x), c0.x);
                const double rp = fma(tv, fma(cvv.y, tv, cv.y), c0.y);
                const double sa = fma(cuv.x, tv, cu.x);
                const double sp = fma(cuv.y, tv, cu.y);
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    const double tu = (double)(col0 + 32 * c) - ij.x;
                    const double ea = fma(tu, fma(cuu.x, tu, sa), ra);
                    const double ep = fma(tu, fma(cuu.y, tu, sp), rp);
                    const double amp = exp2(ea);
                    double sn, cs;
                    sincospi(2.0 * (ep - rint(ep)), &sn, &cs);
                    acc_re[r][c] = fma(amp, cs, acc_re[r][c]);
                    acc_im[r][c] = fma(amp, sn, acc_im[r][c]);
                }
            }
        }
        if (!ts.release(k, lane, warp, spins)) {
            ok = false;
            ++k;
            break;
        }
    }
    if (!ok) {
        record_timeout();
        if (tid == 0) ts.drain(k, spins);
        return;
    }
    const size_t npix = (size_t)nx * ny;
    double2* out = partial + (size_t)blockIdx.z * npix;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const int row = row0 + 8 * r;
        if (row >= ny) continue;
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const int col = col0 + 32 * c;
            if (col >= nx) continue;
            out[(size_t)row * nx + col] = make_double2(acc_re[r][c], acc_im[r][c]);
        }
    }
}

// FP64 path on contiguous row segments.  Along a row the exponent is quadratic in the
// column, so E(u+1) = E(u) R(u) and R(u+1) = R(u) S with S = exp(2 c_uu) fixed per beamlet
// (record field 7): per (beamlet, row segment) the thread evaluates E and R once with
// exp2 + sincospi and then advances with two complex multiplies per pixel.  The products
// keep FP64 relative precision; a beamlet whose amplitude at the segment's first pixel
// is below 2^-1000 contributes zero to that segment (it cannot rise by 2^900 within the
// CB pixels of a segment sampled by the detector).
// A beamlet without a uv term (c_uv = 0, a block-uniform test) factorises on the segment:
// E(u, v) = X(u) Y(v) with X = exp(c_u t_u + c_uu t_u^2) advanced along the row as above
// and Y = exp(c_0 + c_v t_v + c_vv t_v^2) the same for every thread of a row band.  With
// RB > 1 rows per thread each warp evaluates Y once per tile for the (at most two) bands
// its lanes cover, into a shared-memory table (exp2 + sincospi per beamlet, band and row,
// shared by the band's lanes), and a lane then spends 4 + 4 + 4 RB FP64 operations per
// column of RB pixels and two exact evaluations (X, R) per beamlet and segment, instead of
// 10 RB operations and 2 RB evaluations.  Warps covering more bands (narrow detectors) and
// beamlets with a uv term take the per-row recurrence.
constexpr int kYBands = 2;  // row bands per warp table
template <int RB>
constexpr size_t f64_row_smem() {
    return (size_t)kStages * gbd::kF64TileBytes +
           (RB > 1 ? (size_t)(kThreads / 32) * kYBands * RB * gbd::kTile * sizeof(double2) : 0);
}
template <int RB, int CB>
__global__ void __launch_bounds__(kThreads)
    field_f64_row_kernel(const double2* __restrict__ coef, int n_tiles, int tiles_per_split,
                         int nx, int ny, double2* __restrict__ partial, uint32_t spins) {
    constexpr int kTileD2 = gbd::kF64Fields * gbd::kTile;
    extern __shared__ __align__(128) double2 dyn[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
    __shared__ int flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t0 = blockIdx.z * tiles_per_split;
    gbd::init_stream_barriers(full, empty, tid);
    gbd::TileStream<double2, kTileD2> ts{reinterpret_cast<double2(*)[kTileD2]>(dyn), full, empty,
                                         coef + (size_t)t0 * kTileD2,
                                         min(n_tiles - t0, tiles_per_split), 0,
                                         gbd::kF64TileBytes, 0};
    bool ok = ts.start(tid, spins, &flag);

    // thread -> segment of CB columns x RB rows, segments numbered row-band by row-band
    const int segs_x = (nx + CB - 1) / CB;
    const long long seg = (long long)blockIdx.x * kThreads + tid;
    const int col0 = (int)(seg % segs_x) * CB;
    const int row0 = (int)(seg / segs_x) * RB;  // rows row0 .. row0 + RB - 1
    // the warp's row bands and its table of Y (beamlets without a uv term)
    const long long wseg0 = (long long)blockIdx.x * kThreads + (tid & ~31);
    const int wband0 = (int)(wseg0 / segs_x);
    const int wbands = (int)((wseg0 + 31) / segs_x) - wband0 + 1;
    const bool wtable = RB > 1 && wbands <= kYBands;
    const int yband = (int)(seg / segs_x) - wband0;  // this lane's band in the table
    double2* ytab = dyn + kStages * kTileD2 + warp * (kYBands * RB * gbd::kTile);
    double acc_re[RB][CB], acc_im[RB][CB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c) acc_re[r][c] = acc_im[r][c] = 0.0;

    int k = 0;
    for (; ok && k < ts.nt; ++k) {
        if (!ts.acquire(k, spins)) {
            ok = false;
            break;
        }
        const double2* st = ts.tile(k);
        if (wtable) {
            __syncwarp();  // every lane is done with the previous tile's table
            for (int e = lane; e < wbands * RB * gbd::kTile; e += 32) {
                const int b = e % gbd::kTile, r = (e / gbd::kTile) % RB, q = e / (gbd::kTile * RB);
                const double2 cuv = st[5 * gbd::kTile + b];
                double2 y = make_double2(0.0, 0.0);
                if (cuv.x == 0.0 && cuv.y == 0.0) {
                    const double2 ij = st[b];
                    const double2 c0 = st[gbd::kTile + b];
                    const double2 cv = st[3 * gbd::kTile + b];
                    const double2 cvv = st[6 * gbd::kTile + b];
                    const double tv = (double)((wband0 + q) * RB + r) - ij.y;
                    const double ya = fma(tv, fma(cvv.x, tv, cv.x), c0.x);
                    const double yp = fma(tv, fma(cvv.y, tv, cv.y), c0.y);
                    const double amp = exp2(ya);
                    double sn, cs;
                    sincospi(2.0 * (yp - rint(yp)), &sn, &cs);
                    y = make_double2(amp * cs, amp * sn);
                }
                ytab[(q * RB + r) * gbd::kTile + b] = y;
            }
            __syncwarp();
        }
#pragma unroll 1
        for (int b = 0; b < gbd::kTile; ++b) {
            const double2 ij = st[b];
            const double2 c0 = st[gbd::kTile + b];
            const double2 cu = st[2 * gbd::kTile + b];
            const double2 cv = st[3 * gbd::kTile + b];
            const double2 cuu = st[4 * gbd::kTile + b];
            const double2 cuv = st[5 * gbd::kTile + b];
            const double2 cvv = st[6 * gbd::kTile + b];
            const double2 S = st[7 * gbd::kTile + b];
            const double tu = (double)col0 - ij.x;
            if (wtable && cuv.x == 0.0 && cuv.y == 0.0) {
                const double xa = tu * fma(cuu.x, tu, cu.x);
                if (!(xa > -1000.0)) continue;  // X below 2^-1000 on the whole segment
                const double xp = tu * fma(cuu.y, tu, cu.y);
                const double da = fma(cuu.x, 2.0 * tu + 1.0, cu.x);
                const double dp = fma(cuu.y, 2.0 * tu + 1.0, cu.y);
                double er, ei, rr, ri;
                {
                    const double amp = exp2(xa);
                    double sn, cs;
                    sincospi(2.0 * (xp - rint(xp)), &sn, &cs);
                    er = amp * cs;
                    ei = amp * sn;
                }
                {
                    const double amp = exp2(da);
                    double sn, cs;
                    sincospi(2.0 * (dp - rint(dp)), &sn, &cs);
                    rr = amp * cs;
                    ri = amp * sn;
                }
                double2 y[RB];
#pragma unroll
                for (int r = 0; r < RB; ++r) y[r] = ytab[(yband * RB + r) * gbd::kTile + b];
#pragma unroll
                for (int c = 0; c < CB; ++c) {
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        acc_re[r][c] = fma(er, y[r].x, fma(-ei, y[r].y, acc_re[r][c]));
                        acc_im[r][c] = fma(er, y[r].y, fma(ei, y[r].x, acc_im[r][c]));
                    }
                    const double nr = fma(er, rr, -ei * ri), ni = fma(er, ri, ei * rr);
                    er = nr;
                    ei = ni;
                    const double mr = fma(rr, S.x, -ri * S.y), mi = fma(rr, S.y, ri * S.x);
                    rr = mr;
                    ri = mi;
                }
                continue;
            }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const double tv = (double)(row0 + r) - ij.y;
                const double ra = fma(tv, fma(cvv.x, tv, cv.x), c0.x);
                const double rp = fma(tv, fma(cvv.y, tv, cv.y), c0.y);
                const double sa = fma(cuv.x, tv, cu.x);
                const double sp = fma(cuv.y, tv, cu.y);
                // exponent at the first pixel and its step to the next
                const double ea = fma(tu, fma(cuu.x, tu, sa), ra);
                const double ep = fma(tu, fma(cuu.y, tu, sp), rp);
                const double da = fma(cuu.x, 2.0 * tu + 1.0, sa);
                const double dp = fma(cuu.y, 2.0 * tu + 1.0, sp);
                double er = 0.0, ei = 0.0, rr, ri;
                if (ea > -1000.0) {
                    const double amp = exp2(ea);
                    double sn, cs;
                    sincospi(2.0 * (ep - rint(ep)), &sn, &cs);
                    er = amp * cs;
                    ei = amp * sn;
                }
                {
                    const double amp = exp2(da);
                    double sn, cs;
                    sincospi(2.0 * (dp - rint(dp)), &sn, &cs);
                    rr = amp * cs;
                    ri = amp * sn;
                }
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    acc_re[r][c] += er;
                    acc_im[r][c] += ei;
                    const double nr = fma(er, rr, -ei * ri), ni = fma(er, ri, ei * rr);
                    er = nr;
                    ei = ni;
                    const double mr = fma(rr, S.x, -ri * S.y), mi = fma(rr, S.y, ri * S.x);
                    rr = mr;
                    ri = mi;
                }
            }
        }
        if (!ts.release(k, lane, warp, spins)) {
            ok = false;
            ++k;
            break;
        }
    }
    if (!ok) {
        record_timeout();
        if (tid == 0) ts.drain(k, spins);
        return;
    }
    const size_t npix = (size_t)nx * ny;
    double2* out = partial + (size_t)blockIdx.z * npix;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const int row = row0 + r;
        if (row >= ny) continue;
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const int col = col0 + c;
            if (col >= nx) continue;
            out[(size_t)row * nx + col] = make_double2(acc_re[r][c], acc_im[r][c]);
        }
    }
}

// Fixed-order FP64 sum of the split partials (float2 from the mixed kernels, double2 from
// the FP64 ones), times the carrier exp(-ik z(s)) of each pixel (z = n.s is the axial
// offset of the tilted plane), written as complex64/128.
template <bool F64, typename P>
__global__ void __launch_bounds__(256) field_reduce_kernel(const P* __restrict__ partial,
                                                           int splits, int nx, int ny, int rows,
                                                           int row0, int skip, int out_rows,
                                                           double cx, double cy,
                                                           void* __restrict__ out) {
    const size_t npix = (size_t)nx * rows;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)nx * out_rows) return;
    const size_t p = q + (size_t)skip * nx;
    // split order, eight loads in flight per thread (the loop is latency-bound otherwise)
    double re = 0.0, im = 0.0;
    int s = 0;
    for (; s + 8 <= splits; s += 8) {
        P v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(partial + (size_t)(s + u) * npix + p);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            re += (double)v[u].x;
            im += (double)v[u].y;
        }
    }
    for (; s < splits; ++s) {
        const P v = __ldg(partial + (size_t)s * npix + p);
        re += (double)v.x;
        im += (double)v.y;
    }
    if (cx != 0.0 || cy != 0.0) {
        const int i = (int)(p % nx), j = (int)(p / nx) + row0;
        const double turns = cx * (i - nx / 2) + cy * (j - ny / 2);
        double sn, cs;
        sincospi(2.0 * (turns - rint(turns)), &sn, &cs);
        const double r2 = re * cs - im * sn;
        im = re * sn + im * cs;
        re = r2;
    }
    if (F64)
        static_cast<double2*>(out)[q] = make_double2(re, im);
    else
        static_cast<float2*>(out)[q] = make_float2((float)re, (float)im);
}

// The mixed path's reduction: GB300's FP64 pipe is too slow for an FP64 add per split and
// pixel (it made this kernel FP64-bound at ~1 TB/s), so the float2 partials are summed in
// FP32 with Neumaier's compensation, in split order; the carrier's phase in turns is
// reduced in FP64 (one multiply-add and a rounding) and rotated in FP32.  When the flag
// word shows that the multi-row kernel took the field (rows_mask: its hand-over bits all
// clear), that kernel has already summed and stored every pixel and this one returns.
__global__ void __launch_bounds__(256) field_reduce_mixed_kernel(const float2* __restrict__ partial,
                                                                 int splits,
                                                                 const unsigned* __restrict__ flags,
                                                                 unsigned rows_mask, int nx,
                                                                 int rows, gbd::ReduceOut ro) {
    if (rows_mask != 0u && flags && (*flags & rows_mask) == 0u) return;
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)nx * ro.out_rows) return;
    const size_t p = q + (size_t)ro.skip * nx;
    gbd::reduce_store(ro, nx, (int)(p / nx), (int)(p % nx),
                      gbd::sum_partials(partial, (size_t)nx * rows, p, splits));
}

template <int RB, int CB>
cudaError_t launch_mixed(const void* coeffs, int n_tiles, const gbd_project_params& p,
                         const gbd_field_launch& L, void* partial_v, const unsigned* flags,
                         uint32_t spins, const gbd::ReduceOut&, cudaStream_t s) {
    using gbd::kFlagWide;
    float2* partial = static_cast<float2*>(partial_v);
    dim3 grid((p.nx + 32 * CB - 1) / (32 * CB), (p.ny + 8 * RB - 1) / (8 * RB), L.splits);
    const float4* c = static_cast<const float4*>(coeffs);
    const int tps = L.tiles_per_split;
    field_mixed_kernel<RB, CB, false, false><<<grid, kThreads, 0, s>>>(
        c, n_tiles, tps, p.nx, p.ny, partial, flags, kFlagWide, 0u, 0u, spins);
    field_mixed_kernel<RB, CB, true, false><<<grid, kThreads, 0, s>>>(
        c, n_tiles, tps, p.nx, p.ny, partial, flags, kFlagWide, kFlagWide, 0u, spins);
    return cudaGetLastError();
}

// Grid depth of a fallback launch, which the flag word selects only for some fields and
// which otherwise returns at once: its CTAs take the splits in equal shares (the LOOP
// instantiations of field_mixed_kernel and field_mixed_pair_smem_kernel), about 8 CTAs per
// SM in all, so that an idle launch schedules far fewer CTAs.
unsigned fallback_z(int splits, unsigned blocks_xy) {
    const long want = (8L * gbd_sm_count() + blocks_xy - 1) / blocks_xy;
    const int z = (int)(want < 1 ? 1 : want < splits ? want : splits);
    const int per = (splits + z - 1) / z;
    return (unsigned)((splits + per - 1) / per);
}

// Row pairs, with the direct 2 x CB kernels as the fallback when the projection flags a
// beamlet too steep for the recurrence.
template <int CB>
cudaError_t launch_mixed_pair(const void* coeffs, int n_tiles, const gbd_project_params& p,
                              const gbd_field_launch& L, void* partial_v, const unsigned* flags,
                              uint32_t spins, const gbd::ReduceOut&, cudaStream_t s) {
    float2* partial = static_cast<float2*>(partial_v);
    using gbd::kFlagColSteep;
    using gbd::kFlagSteep;
    using gbd::kFlagWide;
    constexpr unsigned kBoth = kFlagWide | kFlagSteep, kAll = kBoth | kFlagColSteep;
    dim3 grid((p.nx + 32 * CB - 1) / (32 * CB), (p.ny + 15) / 16, L.splits);
    const dim3 grid_fb(grid.x, grid.y, fallback_z(L.splits, grid.x * grid.y));
    const float4* c = static_cast<const float4*>(coeffs);
    const int tps = L.tiles_per_split;
    (void)kBoth;
    // exactly one runs: narrow, then wide (or column-steep), then the steep fallback
    field_mixed_kernel<2, CB, 0, true><<<grid, kThreads, 0, s>>>(
        c, n_tiles, tps, p.nx, p.ny, partial, flags, kAll, 0u, 0u, spins);
    field_mixed_kernel<2, CB, 1, true, true><<<grid_fb, kThreads, 0, s>>>(
        c, n_tiles, tps, p.nx, p.ny, partial, flags, kFlagSteep, 0u, kFlagWide | kFlagColSteep,
        spins);
    field_mixed_kernel<2, CB, kWideByFlag, false, true><<<grid_fb, kThreads, 0, s>>>(
        c, n_tiles, tps, p.nx, p.ny, partial, flags, kFlagSteep, kFlagSteep, 0u, spins);
    return cudaGetLastError();
}

template <int RB, int CB>
cudaError_t launch_f64(const void* coeffs, int n_tiles, const gbd_project_params& p,
                       const gbd_field_launch& L, void* partial_v, const unsigned* /*wide*/,
                       uint32_t spins, const gbd::ReduceOut&, cudaStream_t s) {
    double2* partial = static_cast<double2*>(partial_v);
    const size_t smem = (size_t)kStages * gbd::kF64TileBytes;
    cudaError_t e = cudaFuncSetAttribute(field_f64_kernel<RB, CB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.nx + 32 * CB - 1) / (32 * CB), (p.ny + 8 * RB - 1) / (8 * RB), L.splits);
    field_f64_kernel<RB, CB><<<grid, kThreads, smem, s>>>(static_cast<const double2*>(coeffs),
                                                          n_tiles, L.tiles_per_split, p.nx, p.ny,
                                                          partial, spins);
    return cudaGetLastError();
}

template <int RB, int CB>
cudaError_t launch_f64_row(const void* coeffs, int n_tiles, const gbd_project_params& p,
                           const gbd_field_launch& L, void* partial_v, const unsigned* /*wide*/,
                           uint32_t spins, const gbd::ReduceOut&, cudaStream_t s) {
    double2* partial = static_cast<double2*>(partial_v);
    const size_t smem = f64_row_smem<RB>();
    cudaError_t e = cudaFuncSetAttribute(field_f64_row_kernel<RB, CB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long segs = (long long)((p.nx + CB - 1) / CB) * ((p.ny + RB - 1) / RB);
    dim3 grid((unsigned)((segs + kThreads - 1) / kThreads), 1, L.splits);
    field_f64_row_kernel<RB, CB><<<grid, kThreads, smem, s>>>(static_cast<const double2*>(coeffs),
                                                              n_tiles, L.tiles_per_split, p.nx,
                                                              p.ny, partial, spins);
    return cudaGetLastError();
}

// Row pairs on 2 x CB pixels with shared-memory compensation; the direct 2 x 4 kernels (on
// their own pixel grid, same splits) are the steep-beamlet fallback.
// With `after_triple` the row-triple (or quadruple) kernels have been launched first and
// take the fields without multi-row steepness, with or without a uv term; the narrow row
// pairs with the column factor's update (exact for T = 1 as well) then take the rest.
template <int CB>
cudaError_t launch_pair_set(const void* coeffs, int n_tiles, const gbd_project_params& p,
                            const gbd_field_launch& L, void* partial_v, const unsigned* flags,
                            uint32_t spins, cudaStream_t s, bool after_triple) {
    float2* partial = static_cast<float2*>(partial_v);
    using gbd::kFlagColSteep;
    using gbd::kFlagCross;
    using gbd::kFlagSteep;
    using gbd::kFlagWide;
    constexpr unsigned kBoth = kFlagWide | kFlagSteep, kAll = kBoth | kFlagColSteep;
    constexpr size_t smem = pair_smem_bytes<CB>();
    cudaError_t e = cudaSuccess;
    for (const void* fn : {(const void*)field_mixed_pair_smem_kernel<CB, false, false>,
                           (const void*)field_mixed_pair_smem_kernel<CB, false, true>,
                           (const void*)field_mixed_pair_smem_kernel<CB, false, true, true>,
                           (const void*)field_mixed_pair_smem_kernel<CB, true, true, true>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.nx + 32 * CB - 1) / (32 * CB), (p.ny + 15) / 16, L.splits);
    const dim3 grid_fb(grid.x, grid.y, fallback_z(L.splits, grid.x * grid.y));
    dim3 grid24((p.nx + 127) / 128, (p.ny + 15) / 16, 1);
    grid24.z = fallback_z(L.splits, grid24.x * grid24.y);
    const float4* c = static_cast<const float4*>(coeffs);
    const int tps = L.tiles_per_split;
    (void)kBoth;
    // exactly one runs: narrow without a uv term (unless the multi-row kernels ran), narrow
    // with one (behind the multi-row kernels a fallback: narrow and multi-row steep), then
    // wide (or column-steep), then the steep fallback
    if (!after_triple) {
        field_mixed_pair_smem_kernel<CB, false, false><<<grid, kThreads, smem, s>>>(
            c, n_tiles, tps, p.nx, p.ny, partial, flags, kAll | kFlagCross, 0u, 0u, spins);
        field_mixed_pair_smem_kernel<CB, false, true><<<grid, kThreads, smem, s>>>(
            c, n_tiles, tps, p.nx, p.ny, partial, flags, kAll, 0u, kFlagCross, spins);
    } else {
        field_mixed_pair_smem_kernel<CB, false, true, true><<<grid_fb, kThreads, smem, s>>>(
            c, n_tiles, tps, p.nx, p.ny, partial, flags, kAll, 0u, gbd::kFlagSteepRows, spins);
    }
    field_mixed_pair_smem_kernel<CB, true, true, true><<<grid_fb, kThreads, smem, s>>>(
        c, n_tiles, tps, p.nx, p.ny, partial, flags, kFlagSteep, 0u, kFlagWide | kFlagColSteep,
        spins);
    field_mixed_kernel<2, 4, kWideByFlag, false, true><<<grid24, kThreads, 0, s>>>(
        c, n_tiles, tps, p.nx, p.ny, partial, flags, kFlagSteep, kFlagSteep, 0u, spins);
    return cudaGetLastError();
}

template <int CB>
cudaError_t launch_mixed_pair_smem(const void* coeffs, int n_tiles, const gbd_project_params& p,
                                   const gbd_field_launch& L, void* partial, const unsigned* flags,
                                   uint32_t spins, const gbd::ReduceOut&, cudaStream_t s) {
    return launch_pair_set<CB>(coeffs, n_tiles, p, L, partial, flags, spins, s, false);
}

// Row triples or quadruples (RB x CB) when the splits are short enough for FP32 sums,
// with the 2 x CB row-pair set behind them for fields they cannot take; longer splits run
// the row-pair set alone.
template <int RB, int CB>
cudaError_t launch_mixed_rows(const void* coeffs, int n_tiles, const gbd_project_params& p,
                              const gbd_field_launch& L, void* partial, const unsigned* flags,
                              uint32_t spins, const gbd::ReduceOut& ro, cudaStream_t s) {
    // the row pairs behind: 8 columns per thread (the faster pairs) on detectors at least
    // 256 pixels wide, else the multi-row shape's own column count
    auto pairs = [&](bool after) {
        return p.nx >= 256 || CB == 8
                   ? launch_pair_set<8>(coeffs, n_tiles, p, L, partial, flags, spins, s, after)
                   : launch_pair_set<CB>(coeffs, n_tiles, p, L, partial, flags, spins, s, after);
    };
    if (L.tiles_per_split > kRowsMaxTiles) return pairs(false);
    // fields with a uv term on row triples behind the 4 x 8 quadruples (tilted Zernike
    // 1024^2: 4.60 ms against 4.70 ms on 4 x 8; the telescope's PSF 4.68 against 4.89)
    constexpr int RX = RB == 4 && CB == 8 ? 3 : RB;
    constexpr size_t smem = rows_smem_bytes<false, RB, CB>(),
                     smem_x = rows_smem_bytes<true, RX>();
    cudaError_t e = cudaFuncSetAttribute(field_mixed_rows_kernel<RB, CB, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(field_mixed_rows_kernel<RX, CB, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_x);
    if (e != cudaSuccess) return e;
    // splits fastest: a pixel block's splits run together
    // pixel blocks at detector rows that are multiples of 8 RB (p.ny: the slab's rows, its
    // first detector row ro.row0, a multiple of 8 RB for the kernel without a uv term; the
    // one with a uv term may start inside its first block)
    const int gx = (p.nx + 32 * CB - 1) / (32 * CB);
    const int off_x = ro.row0 % (8 * RX);
    dim3 grid(L.splits, gx, (p.ny + 8 * RB - 1) / (8 * RB));
    dim3 grid_x(L.splits, gx, (p.ny + off_x + 8 * RX - 1) / (8 * RX));
    // exactly one of the two runs (or neither): without a uv term, then with one
    field_mixed_rows_kernel<RB, CB, false><<<grid, kThreads, smem, s>>>(
        static_cast<const float4*>(coeffs), n_tiles, L.tiles_per_split, p.nx, p.ny,
        static_cast<float2*>(partial), flags, kRowsNarrow, 0u, spins, ro.done, ro);
    field_mixed_rows_kernel<RX, CB, true><<<grid_x, kThreads, smem_x, s>>>(
        static_cast<const float4*>(coeffs), n_tiles, L.tiles_per_split, p.nx, p.ny,
        static_cast<float2*>(partial), flags, kRowsNarrow, gbd::kFlagCross, spins, ro.done, ro);
    return pairs(true);
}

typedef cudaError_t (*launch_fn)(const void*, int, const gbd_project_params&,
                                 const gbd_field_launch&, void*, const unsigned*, uint32_t,
                                 const gbd::ReduceOut&, cudaStream_t);

struct ShapeEntry {
    int rb, cb, scheme;
    launch_fn fn;
    const void* kernel;
    size_t smem;  // dynamic shared memory of `kernel` (0: static only)
};

const ShapeEntry kMixedShapes[] = {
    {1, 4, GBD_SCHEME_DIRECT, launch_mixed<1, 4>, (const void*)field_mixed_kernel<1, 4, false, false>},
    {2, 2, GBD_SCHEME_DIRECT, launch_mixed<2, 2>, (const void*)field_mixed_kernel<2, 2, false, false>},
    {2, 4, GBD_SCHEME_DIRECT, launch_mixed<2, 4>, (const void*)field_mixed_kernel<2, 4, false, false>},
    {4, 2, GBD_SCHEME_DIRECT, launch_mixed<4, 2>, (const void*)field_mixed_kernel<4, 2, false, false>},
    {2, 2, GBD_SCHEME_ROW_PAIR, launch_mixed_pair<2>, (const void*)field_mixed_kernel<2, 2, false, true>},
    {2, 4, GBD_SCHEME_ROW_PAIR, launch_mixed_pair<4>, (const void*)field_mixed_kernel<2, 4, false, true>},
    {2, 8, GBD_SCHEME_ROW_PAIR, launch_mixed_pair_smem<8>,
     (const void*)field_mixed_pair_smem_kernel<8, false, false>, pair_smem_bytes<8>()},
    {3, 8, GBD_SCHEME_ROW_PAIR, launch_mixed_rows<3, 8>,
     (const void*)field_mixed_rows_kernel<3, 8>,
     rows_smem_bytes()},
    {4, 8, GBD_SCHEME_ROW_PAIR, launch_mixed_rows<4, 8>,
     (const void*)field_mixed_rows_kernel<4, 8>,
     rows_smem_bytes<false, 4, 8>()},
    {4, 4, GBD_SCHEME_ROW_PAIR, launch_mixed_rows<4, 4>,
     (const void*)field_mixed_rows_kernel<4, 4>,
     rows_smem_bytes()},
};
// (1,2), (2,2): every pixel evaluated directly (columns 32 apart); (1,8), (1,16), (2,8),
// (1,32), (4,8), (2,16), (8,4): contiguous row segments advanced by complex multiplies
// (with RB > 1 rows, the row factors of beamlets without a uv term from a warp table).
constexpr size_t kF64Smem = (size_t)kStages * gbd::kF64TileBytes;
const ShapeEntry kF64Shapes[] = {
    {1, 2, 0, launch_f64<1, 2>, (const void*)field_f64_kernel<1, 2>, kF64Smem},
    {2, 2, 0, launch_f64<2, 2>, (const void*)field_f64_kernel<2, 2>, kF64Smem},
    {1, 8, 0, launch_f64_row<1, 8>, (const void*)field_f64_row_kernel<1, 8>, kF64Smem},
    {2, 8, 0, launch_f64_row<2, 8>, (const void*)field_f64_row_kernel<2, 8>, f64_row_smem<2>()},
    {1, 16, 0, launch_f64_row<1, 16>, (const void*)field_f64_row_kernel<1, 16>, kF64Smem},
    {1, 32, 0, launch_f64_row<1, 32>, (const void*)field_f64_row_kernel<1, 32>, kF64Smem},
    {4, 8, 0, launch_f64_row<4, 8>, (const void*)field_f64_row_kernel<4, 8>, f64_row_smem<4>()},
    {2, 16, 0, launch_f64_row<2, 16>, (const void*)field_f64_row_kernel<2, 16>,
     f64_row_smem<2>()},
    {8, 4, 0, launch_f64_row<8, 4>, (const void*)field_f64_row_kernel<8, 4>, f64_row_smem<8>()},
};

const ShapeEntry* find_shape(int precision, int rb, int cb, int scheme) {
    if (precision == GBD_PREC_MIXED) {
        for (const auto& e : kMixedShapes)
            if (e.rb == rb && e.cb == cb && e.scheme == scheme) return &e;
    } else if (scheme == GBD_SCHEME_DIRECT) {
        for (const auto& e : kF64Shapes)
            if (e.rb == rb && e.cb == cb) return &e;
    }
    return nullptr;
}

}  // namespace

bool gbd_field_shape_supported(int precision, int rb, int cb, int scheme) {
    return find_shape(precision, rb, cb, scheme) != nullptr;
}

int gbd_field_occupancy(int precision, int rb, int cb, int scheme) {
    const ShapeEntry* e = find_shape(precision, rb, cb, scheme);
    if (!e) return 0;
    int blocks = 0;
    const size_t smem = e->smem;
    if (smem > 0)
        cudaFuncSetAttribute(e->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, e->kernel, kThreads, smem) !=
        cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t gbd_launch_field_kernel(int precision, const void* coeffs, int n_tiles,
                                    const gbd_project_params& p, const gbd_field_launch& L,
                                    void* partial, const unsigned* wide, uint32_t wait_spins,
                                    const gbd::ReduceOut& ro, cudaStream_t s) {
    const ShapeEntry* e = find_shape(precision, L.rows_per_thread, L.cols_per_thread, L.scheme);
    if (!e) return cudaErrorInvalidValue;
    // the kernels see the slab as a detector of p.rows rows (the records' centre rows are
    // relative to its first row); the partial fields are p.rows x nx
    gbd_project_params slab = p;
    slab.ny = p.rows;
    return e->fn(coeffs, n_tiles, slab, L, partial, wide, wait_spins, ro, s);
}

int gbd_field_row_block(int precision, const gbd_field_launch& L) {
    const int rb = L.rows_per_thread, cb = L.cols_per_thread;
    if (precision == GBD_PREC_F64) return cb >= 8 ? rb : 8 * rb;
    if (L.scheme == GBD_SCHEME_DIRECT) return 8 * rb;
    if (rb == 2) return 16;
    // row triples / quadruples with the 16-row pair set behind them (behind 4 x 8 the row
    // triples that take fields with a uv term place their 24-row blocks at detector rows,
    // whatever the slab's first row)
    return rb == 3 ? 48 : 32;
}

gbd::ReduceOut gbd_reduce_out(const gbd_project_params& p, void* out, unsigned* done,
                              int out_row0, int out_rows) {
    gbd::ReduceOut ro;
    ro.out = out;
    ro.done = done;
    ro.ny = p.ny;
    ro.row0 = p.row0;
    ro.skip = out_row0 - p.row0;
    ro.out_rows = out_rows;
    ro.cx = -p.n[0] * p.px / p.wavelength;
    ro.cy = -p.n[1] * p.py / p.wavelength;
    return ro;
}

cudaError_t gbd_launch_field_reduce(int precision, const gbd_project_params& p,
                                    const gbd_field_launch& L, const unsigned* flags,
                                    const void* partial, const gbd::ReduceOut& ro,
                                    cudaStream_t s) {
    // partial fields: rows p.row0 .. p.row0 + p.rows - 1; output: the window of ro
    const size_t nout = (size_t)p.nx * ro.out_rows;
    if (nout == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((nout + 255) / 256);
    if (precision == GBD_PREC_F64) {
        field_reduce_kernel<true, double2><<<blocks, 256, 0, s>>>(
            static_cast<const double2*>(partial), L.splits, p.nx, p.ny, p.rows, p.row0, ro.skip,
            ro.out_rows, ro.cx, ro.cy, ro.out);
    } else {
        // a multi-row launch whose kernels took the field has stored it already
        const bool rows = L.scheme == GBD_SCHEME_ROW_PAIR && L.rows_per_thread >= 3 &&
                          L.tiles_per_split <= kRowsMaxTiles;
        field_reduce_mixed_kernel<<<blocks, 256, 0, s>>>(static_cast<const float2*>(partial),
                                                         L.splits, flags,
                                                         rows ? kRowsTaken : 0u, p.nx, p.rows,
                                                         ro);
    }
    return cudaGetLastError();
}

// The status word: copied into pinned host memory on the caller's stream (gbd_sync), and
// cleared once it has been reported.
cudaError_t gbd_field_status_fetch(unsigned* host, cudaStream_t s) {
    return cudaMemcpyFromSymbolAsync(host, g_field_status, sizeof(unsigned), 0,
                                     cudaMemcpyDeviceToHost, s);
}
void gbd_field_status_clear() {
    const unsigned zero = 0;
    cudaMemcpyToSymbol(g_field_status, &zero, sizeof(zero));
}
