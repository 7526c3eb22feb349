// Shared building blocks of the field kernels (field.cu) and the persistent sweep kernel
// (sweep.cu): the TMA tile stream through shared memory and the mixed-precision
// per-(beamlet, pixel) evaluation of one 64-beamlet tile.
#pragma once

#include "gbd_internal.cuh"

namespace gbd {

constexpr int kStages = 4;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Warp-uniform bounded wait: every lane polls and the warp leaves together, either when
// all lanes see the phase complete or after `spins` polls.  A completed phase stays
// visible until this warp releases the stage, so the vote cannot flip back.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint32_t spins) {
    for (uint32_t it = 0; it < spins; ++it) {
        const bool d = mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, d)) return true;
    }
    return false;
}

// Barriers of a tile stream, initialised once per CTA by all threads together.
__device__ __forceinline__ void init_stream_barriers(uint64_t* full, uint64_t* empty, int tid) {
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kWarps);
        }
        mbar_fence_init();
    }
    __syncthreads();
}

// Stream of `nt` tiles of `bytes` bytes from global memory through kStages shared
// buffers.  Tile k of this stream is the g0 + k-th tile the CTA has streamed (a CTA
// that runs several streams in turn keeps counting, so barrier phases stay in step).
// Thread 0 is the producer; every warp consumes every tile.
template <typename T, int kElems>
struct TileStream {
    T (*stage)[kElems];
    uint64_t* full;
    uint64_t* empty;
    const T* src;
    int nt;
    int g0;
    uint32_t bytes;
    int issued;

    // Producer: once every warp has released the tile that last used the stage, copy
    // tile k into it.  Thread 0 only.
    __device__ bool issue(int k, uint32_t spins) {
        const int g = g0 + k, s = g % kStages;
        if (g >= kStages && !mbar_wait_bounded(&empty[s], ((g / kStages) - 1) & 1, spins))
            return false;
        mbar_arrive_expect_tx(&full[s], bytes);
        bulk_copy_g2s(stage[s], src + (size_t)k * kElems, bytes, &full[s]);
        return true;
    }
    // Prologue: thread 0 issues the first tiles; block-uniform result through `flag`.
    __device__ bool start(int tid, uint32_t spins, int* flag) {
        issued = 0;
        if (tid == 0) {
            bool ok = true;
            const int first = nt < kStages ? nt : kStages;
            for (; issued < first; ++issued)
                if (!issue(issued, spins)) {
                    ok = false;
                    break;
                }
            *flag = ok ? 1 : 0;
        }
        __syncthreads();
        const bool ok = *flag != 0;
        __syncthreads();
        return ok;
    }
    // Wait until tile k is in shared memory (warp-uniform result).
    __device__ bool acquire(int k, uint32_t spins) {
        const int g = g0 + k;
        return warp_wait(&full[g % kStages], (g / kStages) & 1, spins);
    }
    __device__ const T* tile(int k) const { return stage[(g0 + k) % kStages]; }
    // This warp is done with tile k; warp 0 then refills the stage with tile k + kStages.
    // Warp-uniform result.
    __device__ bool release(int k, int lane, int warp, uint32_t spins) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[(g0 + k) % kStages]);
        if (warp != 0 || k + kStages >= nt) return true;
        bool good = true;
        if (lane == 0) good = issue(k + kStages, spins);
        good = __shfl_sync(0xffffffffu, good, 0) != 0;
        if (good) ++issued;
        return good;
    }
    // After a failed wait: the producer waits for the copies it issued that nobody
    // consumed, so none lands in shared memory after the CTA has moved on or exited.
    // Uses at least the default limit: copies complete within microseconds.
    __device__ void drain(int consumed, uint32_t spins) {
        const uint32_t lim = spins > kDefaultWaitSpins ? spins : kDefaultWaitSpins;
        for (int k = consumed; k < issued; ++k) {
            const int g = g0 + k;
            mbar_wait_bounded(&full[g % kStages], (g / kStages) & 1, lim);
        }
    }
};

// Phase magnitude (radians) above which a beamlet's phase is range-reduced per pixel.
// Below it the MUFU sin/cos take the radians directly, saving four instructions.  A phase
// held in FP32 is off by about |x| 2^-24 however it is reduced; unreduced, the MUFU adds
// an error that also grows with |x| (3e-7 at pi, 1e-5 at 100 rad on GB300).  Measured with
// 3,228 beamlets 41 lambda F# wide on detectors whose phase bound runs from 100 to 250 rad,
// the field's relative L2 error against the oracle grows from 2.1e-6 to 4.1e-6 unreduced
// and stays 1.4-2.3e-6 reduced; at this bound it is 2.2e-6 (the benchmark workloads stay
// under 101 rad, so none of them pays for the reduction).
constexpr float kWidePhase = 128.0f;

// One 64-beamlet tile of mixed-precision evaluation on a thread's RB x CB pixels.
// Record fields: (i0, j0, a0, p0) (a1u, p1u, a1v, p1v) (auu, puu, auv, puv) (avv, pvv, T)
// with log2 |E| = a0 + a1u tu + a1v tv + auu tu^2 + auv tu tv + avv tv^2 and the phase in
// radians the same in p, tu = i - i0, tv = j - j0.  WIDE: some beamlet's phase may exceed
// kWidePhase on this detector, so every phase is reduced exactly to [-pi, pi] (in turns,
// where x - rint(x) is exact) before sin/cos.
template <int RB, int CB, bool WIDE>
__device__ __forceinline__ void mixed_tile(const float4* __restrict__ st, const float (&colf)[CB],
                                           const float (&rowf)[RB], float2 (&acc)[RB][CB]) {
    const float kTwoPi = 6.28318530717958647692f, kInvTwoPi = 0.15915494309189533577f;
#pragma unroll 1
    for (int b = 0; b < kTile; ++b) {
        const float4 q0 = st[b];
        const float4 q1 = st[kTile + b];
        const float4 q2 = st[2 * kTile + b];
        const float4 q3 = st[3 * kTile + b];
        float tu[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c) tu[c] = colf[c] - q0.x;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const float tv = rowf[r] - q0.y;
            const float ra = fmaf(tv, fmaf(q3.x, tv, q1.z), q0.z);
            const float rp = fmaf(tv, fmaf(q3.y, tv, q1.w), q0.w);
            const float sa = fmaf(q2.z, tv, q1.x);
            const float sp = fmaf(q2.w, tv, q1.y);
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const float ea = fmaf(tu[c], fmaf(q2.x, tu[c], sa), ra);
                float x = fmaf(tu[c], fmaf(q2.y, tu[c], sp), rp);
                if (WIDE) x = frac_turns(x * kInvTwoPi) * kTwoPi;
                const float amp = mufu_ex2(ea);
                acc[r][c].x = fmaf(amp, mufu_cos(x), acc[r][c].x);
                acc[r][c].y = fmaf(amp, mufu_sin(x), acc[r][c].y);
            }
        }
    }
}

// Row-pair variant of mixed_tile on rows v (evaluated directly) and v + 8 (derived): with
// ln E quadratic in the pixel, E(u, v + 8) = E(u, v) R(u) where the 8-row step factor
// R(u) = exp(8 (c_v + c_uv tu + c_vv (2 tv + 8))) is itself geometric along the thread's
// columns, R(u + 32) = R(u) T with T = exp(256 c_uv) from the record.  Per beamlet and
// thread: one exact R (ex2 + sin + cos; its phase, at most 64 rad unless the field is
// wide, reduced to [-pi, pi] in the WIDE instantiation), sin + cos
// for each first-row pixel, and (narrow phases) the first row's amplitude by a real
// recurrence: 4 ex2 + 2 (CB + 1) sin/cos for 2 CB pixels instead of 6 CB MUFU operations.
// The second row costs 2 FMUL + 4 FFMA per pixel (+ 4 for the next R, + 2 for the next
// amplitude).  Requires the projection's steep flag to be clear (every R within 2^+-64).
template <int CB, bool WIDE>
__device__ __forceinline__ void mixed_tile_pair(const float4* __restrict__ st,
                                                const float (&colf)[CB], float rowf,
                                                float2 (&acc)[2][CB]) {
    const float kTwoPi = 6.28318530717958647692f, kInvTwoPi = 0.15915494309189533577f;
#pragma unroll 1
    for (int b = 0; b < kTile; ++b) {
        const float4 q0 = st[b];
        const float4 q1 = st[kTile + b];
        const float4 q2 = st[2 * kTile + b];
        const float4 q3 = st[3 * kTile + b];
        float tu[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c) tu[c] = WIDE || c == 0 ? colf[c] - q0.x : 0.f;
        const float tv = rowf - q0.y;
        const float ra = fmaf(tv, fmaf(q3.x, tv, q1.z), q0.z);
        const float rp = fmaf(tv, fmaf(q3.y, tv, q1.w), q0.w);
        const float sa = fmaf(q2.z, tv, q1.x);
        const float sp = fmaf(q2.w, tv, q1.y);
        const float w = fmaf(2.0f, tv, 8.0f);
        const float ga = 8.0f * fmaf(q3.x, w, fmaf(q2.z, tu[0], q1.z));
        float gp = 8.0f * fmaf(q3.y, w, fmaf(q2.w, tu[0], q1.w));
        // narrow phases: the first row's phase at column c as x0 + c (d1 + c d2), the
        // quadratic in tu = tu0 + 32 c expanded about the thread's first column
        const float x0 = fmaf(tu[0], fmaf(q2.y, tu[0], sp), rp);
        const float d1 = 32.0f * fmaf(q2.y, tu[0] + tu[0], sp), d2 = 1024.0f * q2.y;
        // the projection holds |gp| to 64 rad unless the wide flag is set
        if (WIDE) gp = frac_turns(gp * kInvTwoPi) * kTwoPi;
        const float gm = mufu_ex2(ga);
        float rx = gm * mufu_cos(gp), ry = gm * mufu_sin(gp);
        // narrow phases: the first row's amplitude along the thread's columns by a real
        // recurrence, amp(c + 1) = amp(c) rho(c), rho(c + 1) = rho(c) sig with
        // log2 rho(0) = 32 (sa + a_uu (2 tu0 + 32)) and log2 sig = 2048 a_uu: three ex2
        // instead of CB (the launch requires the projection's column-steep flag clear).
        // The WIDE instantiation, which also serves column-steep fields, evaluates each.
        float amp = 0.f, rho = 0.f, sig = 0.f;
        if (!WIDE) {
            amp = mufu_ex2(fmaf(tu[0], fmaf(q2.x, tu[0], sa), ra));
            rho = mufu_ex2(32.0f * fmaf(q2.x, fmaf(2.0f, tu[0], 32.0f), sa));
            sig = mufu_ex2(2048.0f * q2.x);
        }
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            float x;
            if (WIDE) {
                x = fmaf(tu[c], fmaf(q2.y, tu[c], sp), rp);
                x = frac_turns(x * kInvTwoPi) * kTwoPi;
                amp = mufu_ex2(fmaf(tu[c], fmaf(q2.x, tu[c], sa), ra));
            } else {
                x = c == 0 ? x0 : fmaf((float)(c * c), d2, fmaf((float)c, d1, x0));
            }
            const float cs = mufu_cos(x), sn = mufu_sin(x);
            acc[0][c].x = fmaf(amp, cs, acc[0][c].x);
            acc[0][c].y = fmaf(amp, sn, acc[0][c].y);
            const float wx = amp * rx, wy = amp * ry;
            acc[1][c].x = fmaf(cs, wx, fmaf(-sn, wy, acc[1][c].x));
            acc[1][c].y = fmaf(cs, wy, fmaf(sn, wx, acc[1][c].y));
            if (c + 1 < CB) {
                const float nx = fmaf(rx, q3.z, -ry * q3.w);
                ry = fmaf(rx, q3.w, ry * q3.z);
                rx = nx;
                if (!WIDE) {
                    amp *= rho;
                    rho *= sig;
                }
            }
        }
    }
}

// Row terms of a tile for the narrow row-pair evaluation.  Within a warp every lane shares
// the first row v (the lanes differ only in their columns), so the parts of the
// per-beamlet setup that do not depend on the column are computed once per warp and tile:
// lane l takes beamlets l and l + 32 and stores, SoA over the tile's 64 beamlets,
//   ent[0][b] = (ra, rp, sa, sp): log2-amplitude / phase of the row at tu = 0 and their
//               tu-slopes (the quadratic form with tv = v - v_c substituted),
//   ent[1][b] = (32 sa + 1024 a_uu, 32 sp, 8 (a_v + a_vv (2 tv + 8)), 8 (p_v + p_vv (2 tv + 8))),
//   ent[2][b] = (64 a_uu, 64 p_uu, 8 a_uv, 8 p_uv),
// so that mixed_tile_pair_rows forms the first-row amplitude and phase, the amplitude's
// first ratio rho, the phase step d1 and the 8-row step factor's exponent with one or two
// FFMA each in the thread's first column tu0.  Without a uv term (CROSS = false, the
// projection's cross flag clear) the step factor R does not depend on the column and
// ent[1][b].zw holds R itself, formed here once per warp with its phase reduced exactly.
// kPairRowF4 float4 per beamlet and warp.
constexpr int kPairRowF4 = 3;
template <bool CROSS>
__device__ __forceinline__ void mixed_pair_rows(const float4* __restrict__ st, float rowf,
                                                float4* __restrict__ ent, int lane) {
#pragma unroll
    for (int h = 0; h < kTile / 32; ++h) {
        const int b = lane + 32 * h;
        const float4 q0 = st[b];
        const float4 q1 = st[kTile + b];
        const float4 q2 = st[2 * kTile + b];
        const float4 q3 = st[3 * kTile + b];
        const float tv = rowf - q0.y;
        const float ra = fmaf(tv, fmaf(q3.x, tv, q1.z), q0.z);
        const float rp = fmaf(tv, fmaf(q3.y, tv, q1.w), q0.w);
        const float sa = fmaf(q2.z, tv, q1.x);
        const float sp = fmaf(q2.w, tv, q1.y);
        const float w = fmaf(2.0f, tv, 8.0f);
        ent[b] = make_float4(ra, rp, sa, sp);
        const float ga = 8.0f * fmaf(q3.x, w, q1.z), gp = 8.0f * fmaf(q3.y, w, q1.w);
        if (CROSS) {
            ent[kTile + b] = make_float4(fmaf(1024.0f, q2.x, 32.0f * sa), 32.0f * sp, ga, gp);
        } else {
            const float gr = frac_turns(gp * 0.15915494309189533577f) * 6.28318530717958647692f;
            const float gm = mufu_ex2(ga);
            ent[kTile + b] = make_float4(fmaf(1024.0f, q2.x, 32.0f * sa), 32.0f * sp,
                                         gm * mufu_cos(gr), gm * mufu_sin(gr));
        }
        ent[2 * kTile + b] = make_float4(64.0f * q2.x, 64.0f * q2.y, 8.0f * q2.z, 8.0f * q2.w);
    }
}

// Row terms of a tile for the row triples and quadruples on fields without a uv term
// (a_uv = p_uv = 0 for every beamlet, the projection's cross flag clear; with one,
// mixed_rows_cross_terms adds the column factors to these).  The 8-row step factor
// R = exp(8 (c_v + c_vv (2 tv + 8))) then does not depend
// on the column, so it and its products S_2 = R (R K), S_3 = S_2 (R K^2)
// (K = exp(128 c_vv), the ratio of consecutive step factors) are the same for all lanes
// of the warp and are formed here, once per warp and beamlet, with their phases reduced
// exactly.  Lane l takes beamlets l and l + 32; kRowsF4 float4 per beamlet and warp:
//   ent[0][b] = (u_c, ra, rp, sa),  ent[1][b] = (sp, 32 sa + 1024 a_uu, 32 sp, sig),
//   ent[2][b] = (64 a_uu, 64 p_uu, R),  ent[3][b] = (S_2, S_3),
// with ra, rp, sa, sp as in mixed_pair_rows and sig = 2^(2048 a_uu).
constexpr int kRowsF4 = 4;
// The packed quadruples (mixed_tile_rows_x2) also take the pairs (-S_r.im, S_r.re) from
// the row terms: ent[4][b] = (-S_1.im, S_1.re, -S_2.im, S_2.re), ent[5][b] = (-S_3.im,
// S_3.re, 0, 0), formed once per warp instead of by every thread.
constexpr int kRowsX2F4 = 6;
// The row terms of stage beamlet b, written to ent[k * stride + i] (k = 0..3, and 4, 5
// with SWAP).
template <int RB, bool SWAP = false>
__device__ __forceinline__ void mixed_rows_term(const float4* __restrict__ st, int b, float rowf,
                                                float4* __restrict__ ent, int i, int stride) {
    const float kTwoPi = 6.28318530717958647692f, kInvTwoPi = 0.15915494309189533577f;
    const float4 q0 = st[b];
    const float4 q1 = st[kTile + b];
    const float4 q2 = st[2 * kTile + b];
    const float4 q3 = st[3 * kTile + b];
    const float tv = rowf - q0.y;
    const float ra = fmaf(tv, fmaf(q3.x, tv, q1.z), q0.z);
    const float rp = fmaf(tv, fmaf(q3.y, tv, q1.w), q0.w);
    const float sa = fmaf(q2.z, tv, q1.x);
    const float sp = fmaf(q2.w, tv, q1.y);
    const float w = fmaf(2.0f, tv, 8.0f);
    // R = 2^(8 (a_v + a_vv w)) e^(i 8 (p_v + p_vv w)), K likewise with 128 a_vv, 128 p_vv
    const float gp = frac_turns(8.0f * fmaf(q3.y, w, q1.w) * kInvTwoPi) * kTwoPi;
    const float gm = mufu_ex2(8.0f * fmaf(q3.x, w, q1.z));
    const float2 R = make_float2(gm * mufu_cos(gp), gm * mufu_sin(gp));
    const float kp = frac_turns(128.0f * q3.y * kInvTwoPi) * kTwoPi;
    const float km = mufu_ex2(128.0f * q3.x);
    const float2 K = make_float2(km * mufu_cos(kp), km * mufu_sin(kp));
    const float2 f2 = make_float2(fmaf(R.x, K.x, -R.y * K.y), fmaf(R.x, K.y, R.y * K.x));
    const float2 S2 = make_float2(fmaf(R.x, f2.x, -R.y * f2.y), fmaf(R.x, f2.y, R.y * f2.x));
    float2 S3 = make_float2(0.0f, 0.0f);
    if (RB > 3) {
        const float2 f3 = make_float2(fmaf(f2.x, K.x, -f2.y * K.y), fmaf(f2.x, K.y, f2.y * K.x));
        S3 = make_float2(fmaf(S2.x, f3.x, -S2.y * f3.y), fmaf(S2.x, f3.y, S2.y * f3.x));
    }
    ent[i] = make_float4(q0.x, ra, rp, sa);
    ent[stride + i] = make_float4(sp, fmaf(1024.0f, q2.x, 32.0f * sa), 32.0f * sp,
                                  mufu_ex2(2048.0f * q2.x));
    ent[2 * stride + i] = make_float4(64.0f * q2.x, 64.0f * q2.y, R.x, R.y);
    ent[3 * stride + i] = make_float4(S2.x, S2.y, S3.x, S3.y);
    if (SWAP) {
        ent[4 * stride + i] = make_float4(-R.y, R.x, -S2.y, S2.x);
        ent[5 * stride + i] = make_float4(-S3.y, S3.x, 0.0f, 0.0f);
    }
}

// All 64 beamlets of the tile: lane l takes beamlets l and l + 32.
template <int RB, bool SWAP = false>
__device__ __forceinline__ void mixed_rows_terms(const float4* __restrict__ st, float rowf,
                                                 float4* __restrict__ ent, int lane) {
#pragma unroll
    for (int h = 0; h < kTile / 32; ++h)
        mixed_rows_term<RB, SWAP>(st, lane + 32 * h, rowf, ent, lane + 32 * h, kTile);
}

// The narrow instantiation of mixed_tile_pair (same arithmetic, regrouped) on the row
// terms of mixed_pair_rows: per beamlet and thread only the column-dependent setup is
// left (about 27 instructions instead of 43 for the 2 x CB pixels).  CROSS = false is
// for fields without a uv term (the projection's cross flag clear): there every T is
// exactly 1, R(u + 32) = R(u) T is the identity, and its update is left out; R itself
// comes from the warp's row terms (about 19 instructions of setup).
template <int CB, bool CROSS>
__device__ __forceinline__ void mixed_tile_pair_rows(const float4* __restrict__ st,
                                                     const float4* __restrict__ ent,
                                                     const float (&colf)[CB],
                                                     float2 (&acc)[2][CB]) {
    const float* stf = reinterpret_cast<const float*>(st);
#pragma unroll 1
    for (int b = 0; b < kTile; ++b) {
        const float uc = stf[4 * b];                                               // q0.x
        const float2 quu = reinterpret_cast<const float2*>(st + 2 * kTile + b)[0];  // q2.xy
        const float2 T = reinterpret_cast<const float2*>(st + 3 * kTile + b)[1];    // q3.zw
        const float4 e0 = ent[b];
        const float4 e1 = ent[kTile + b];
        const float4 e2 = ent[2 * kTile + b];
        const float tu0 = colf[0] - uc;
        const float x0 = fmaf(tu0, fmaf(quu.y, tu0, e0.w), e0.y);
        const float d1 = fmaf(e2.y, tu0, e1.y);
        float rx, ry;
        if (CROSS) {
            const float ga = fmaf(e2.z, tu0, e1.z);
            const float gp = fmaf(e2.w, tu0, e1.w);  // within 64 rad: the field is not wide
            const float gm = mufu_ex2(ga);
            rx = gm * mufu_cos(gp);
            ry = gm * mufu_sin(gp);
        } else {  // the same R on every column, from the warp's row terms
            rx = e1.z;
            ry = e1.w;
        }
        float amp = mufu_ex2(fmaf(tu0, fmaf(quu.x, tu0, e0.z), e0.x));
        float rho = mufu_ex2(fmaf(e2.x, tu0, e1.x));
        const float sig = mufu_ex2(2048.0f * quu.x);
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            // first-row phase x0 + c d1 + 1024 c^2 p_uu about the thread's first column
            const float x = c == 0 ? x0 : fmaf((float)(1024 * c * c), quu.y, fmaf((float)c, d1, x0));
            const float cs = mufu_cos(x), sn = mufu_sin(x);
            acc[0][c].x = fmaf(amp, cs, acc[0][c].x);
            acc[0][c].y = fmaf(amp, sn, acc[0][c].y);
            const float wx = amp * rx, wy = amp * ry;
            acc[1][c].x = fmaf(cs, wx, fmaf(-sn, wy, acc[1][c].x));
            acc[1][c].y = fmaf(cs, wy, fmaf(sn, wx, acc[1][c].y));
            if (c + 1 < CB) {
                if (CROSS) {
                    const float nx = fmaf(rx, T.x, -ry * T.y);
                    ry = fmaf(rx, T.y, ry * T.x);
                    rx = nx;
                }
                amp *= rho;
                rho *= sig;
            }
        }
    }
}

// Row triples (RB = 3: rows v, v + 8, v + 16) and quadruples (RB = 4: also v + 24) for
// fields without a uv term, on the row terms of mixed_rows_terms (NB beamlets, SoA with
// stride NB): row 8 r below the first
// is the first times S_r (S_1 = R), the same for the whole row.  Per beamlet and thread
// only the first row's amplitude and phase polynomials in the thread's first column tu0
// are left (2 ex2 and 7 FMA-pipe instructions); per column the first row's value
// E0 = amp (cos, sin) and 4 FFMA per later row: 19 instructions for 3 pixels, 23 for 4,
// 16 sin/cos + 2 ex2 per 8 RB pixels.  The products a_uu tu0 and 1024 c^2 p_uu are formed
// as (64 a_uu)(tu0 / 64) and 16 c^2 (64 p_uu), the same values exactly.  Requires the
// steep and multi-row steep flags clear (every |log2 S_r| within 64).
template <int RB, int CB, int NB = kTile>
__device__ __forceinline__ void mixed_tile_rows(const float4* __restrict__ ent,
                                                const float (&colf)[CB],
                                                float2 (&acc)[RB][CB]) {
    static_assert(RB == 3 || RB == 4, "row triples or quadruples");
#pragma unroll 1
    for (int b = 0; b < NB; ++b) {
        const float4 e0 = ent[b];
        const float4 e1 = ent[NB + b];
        const float4 e2 = ent[2 * NB + b];
        const float4 e3 = ent[3 * NB + b];
        const float2 S[3] = {make_float2(e2.z, e2.w), make_float2(e3.x, e3.y),
                             make_float2(e3.z, e3.w)};
        const float tu0 = colf[0] - e0.x;
        const float t64 = tu0 * 0.015625f;
        const float x0 = fmaf(tu0, fmaf(e2.y, t64, e1.x), e0.z);
        const float d1 = fmaf(e2.y, tu0, e1.z);
        float amp = mufu_ex2(fmaf(tu0, fmaf(e2.x, t64, e0.w), e0.y));
        float rho = mufu_ex2(fmaf(e2.x, tu0, e1.y));
        const float sig = e1.w;
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const float x = c == 0 ? x0 : fmaf((float)(16 * c * c), e2.y, fmaf((float)c, d1, x0));
            // the first row's value E0 once, then E0 S_r into the later rows
            const float ex = amp * mufu_cos(x), ey = amp * mufu_sin(x);
            acc[0][c].x += ex;
            acc[0][c].y += ey;
#pragma unroll
            for (int r = 1; r < RB; ++r) {
                acc[r][c].x = fmaf(ex, S[r - 1].x, fmaf(-ey, S[r - 1].y, acc[r][c].x));
                acc[r][c].y = fmaf(ex, S[r - 1].y, fmaf(ey, S[r - 1].x, acc[r][c].y));
            }
            if (c + 1 < CB) {
                amp *= rho;
                rho *= sig;
            }
        }
    }
}

// mixed_tile_rows with the complex arithmetic in packed FP32x2 instructions (FFMA2, FMUL2,
// FADD2 on (re, im) pairs): E0 = amp (cos, sin) one FMUL2, the first row one FADD2, each
// later row two FFMA2 (E0.re (S.re, S.im) and E0.im (-S.im, S.re) onto (re, im)); the
// amplitude recurrence in two scalar FMULs (the FMA-lite pipe takes them).  The pairs
// (-S.im, S.re) come from the row terms (mixed_rows_term<RB, true>: ent[4], ent[5]), formed
// once per warp instead of by every thread (a negation and a move each).  Every lane rounds
// as the scalar FMA / FMUL / FADD, in the same order, so the sums are the same bits as
// mixed_tile_rows' (up to the compiler's choice of contracting the first row's add into an
// FMA there).  The packed operations all run on the FMA-heavy pipe, which then binds (ncu:
// math-pipe throttle the largest stall); moving a row back to scalar FFMA did not help
// (3.04 and 2.89 ms for one and two scalar rows against 2.85 ms), nor did forming E0 by
// scalar FMULs (2.78 ms against 2.74 ms).
template <int RB, int CB, int NB = kTile>
__device__ __forceinline__ void mixed_tile_rows_x2(const float4* __restrict__ ent,
                                                   const float (&colf)[CB],
                                                   float2 (&acc)[RB][CB]) {
    static_assert(RB == 3 || RB == 4, "row triples or quadruples");
#pragma unroll 1
    for (int b = 0; b < NB; ++b) {
        const float4 e0 = ent[b];
        const float4 e1 = ent[NB + b];
        const float4 e2 = ent[2 * NB + b];
        const float4 e3 = ent[3 * NB + b];
        const float4 e4 = ent[4 * NB + b];
        const float4 e5 = ent[5 * NB + b];
        const float2 S[3] = {make_float2(e2.z, e2.w), make_float2(e3.x, e3.y),
                             make_float2(e3.z, e3.w)};
        // (-S.im, S.re): multiplies E0.im (from the row terms)
        const float2 Sr[3] = {make_float2(e4.x, e4.y), make_float2(e4.z, e4.w),
                              make_float2(e5.x, e5.y)};
        const float tu0 = colf[0] - e0.x;
        const float t64 = tu0 * 0.015625f;
        const float x0 = fmaf(tu0, fmaf(e2.y, t64, e1.x), e0.z);
        const float d1 = fmaf(e2.y, tu0, e1.z);
        // the first row's amplitude at the thread's column and its ratio, advanced in scalar
        // FMULs (the FMA-lite pipe can take them; the packed form sits on the heavy pipe)
        float amp = mufu_ex2(fmaf(tu0, fmaf(e2.x, t64, e0.w), e0.y));
        float rho = mufu_ex2(fmaf(e2.x, tu0, e1.y));
        const float sig = e1.w;
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const float x = c == 0 ? x0 : fmaf((float)(16 * c * c), e2.y, fmaf((float)c, d1, x0));
            const float2 E0 = __fmul2_rn(make_float2(amp, amp), make_float2(mufu_cos(x), mufu_sin(x)));
            acc[0][c] = __fadd2_rn(acc[0][c], E0);
#pragma unroll
            for (int r = 1; r < RB; ++r) {
                acc[r][c] = __ffma2_rn(make_float2(E0.y, E0.y), Sr[r - 1], acc[r][c]);
                acc[r][c] = __ffma2_rn(make_float2(E0.x, E0.x), S[r - 1], acc[r][c]);
            }
            if (c + 1 < CB) {
                amp *= rho;
                rho *= sig;
            }
        }
    }
}

// Row terms of a tile for the row triples and quadruples on fields with a uv term.  The
// 8-row step factor at column offset tu from the beamlet's centre is then R W(tu) with
// W(tu) = exp(8 c_uv tu), so row 8 r below the first is the first times
// P_r(tu) = S_r W(tu)^r, S_r the column-free products of mixed_rows_term; along a thread's
// columns (32 apart) P_r steps by T^r, T = W(32) = exp(256 c_uv) (stored in the record).
// kRowsCrossF4<RB> float4 per beamlet and warp: the kRowsF4 of mixed_rows_term, with
//   ent[4][b] = (T.re, T^2.re, T.im, T^2.im)   (rows 1 and 2 step as one FP32x2 pair),
// and (8 a_uv, 8 p_uv) in the unused S_3 slot of ent[3][b] for the triples; the
// quadruples add ent[5][b] = (T^3, 8 a_uv, 8 p_uv).
template <int RB>
constexpr int kRowsCrossF4 = RB > 3 ? 6 : 5;
// The cross row terms of stage beamlet b, written to ent[k * stride + i].
template <int RB>
__device__ __forceinline__ void mixed_rows_cross_term(const float4* __restrict__ st, int b,
                                                      float rowf, float4* __restrict__ ent,
                                                      int i, int stride) {
    mixed_rows_term<RB>(st, b, rowf, ent, i, stride);
    const float4 q2 = st[2 * kTile + b];
    const float4 q3 = st[3 * kTile + b];
    const float2 T = make_float2(q3.z, q3.w);
    const float2 T2 = make_float2(fmaf(T.x, T.x, -T.y * T.y), 2.0f * T.x * T.y);
    ent[4 * stride + i] = make_float4(T.x, T2.x, T.y, T2.y);
    if (RB > 3) {
        const float2 T3 =
            make_float2(fmaf(T2.x, T.x, -T2.y * T.y), fmaf(T2.x, T.y, T2.y * T.x));
        ent[5 * stride + i] = make_float4(T3.x, T3.y, 8.0f * q2.z, 8.0f * q2.w);
    } else {
        const float4 e3 = ent[3 * stride + i];  // written above by this thread
        ent[3 * stride + i] = make_float4(e3.x, e3.y, 8.0f * q2.z, 8.0f * q2.w);
    }
}

// All 64 beamlets of the tile: lane l takes beamlets l and l + 32.
template <int RB>
__device__ __forceinline__ void mixed_rows_cross_terms(const float4* __restrict__ st, float rowf,
                                                       float4* __restrict__ ent, int lane) {
#pragma unroll
    for (int h = 0; h < kTile / 32; ++h)
        mixed_rows_cross_term<RB>(st, lane + 32 * h, rowf, ent, lane + 32 * h, kTile);
}

// mixed_tile_rows for fields with a uv term, on the cross row terms (NB beamlets, SoA with
// stride NB).
// Per beamlet and thread, besides the first row's polynomials: W0 = W(tu0) at the thread's
// first column (one ex2 and a sin/cos of a phase within 64 rad, reduced exactly first) and
// P_r = S_r W0^r by complex multiplies.  Per column: the first row's value E0 as in
// mixed_tile_rows, 4 FFMA per later row (E0 P_r), and the step P_r <- P_r T^r: rows 1 and 2
// as the FP32x2 pairs X = (P_1.re, P_2.re), Y = (P_1.im, P_2.im), X <- X (T.re, T^2.re) -
// Y (T.im, T^2.im), Y <- X (T.im, T^2.im) + Y (T.re, T^2.re) (4 packed instructions, no
// operand moves), row 3 (quadruples) in scalar.  Requires the same flags clear as
// mixed_tile_rows except the cross flag: the steep-rows bound covers |log2 P_r| with the
// uv term over the detector, the wide bound the step phase 8 (p_v + p_uv tu + ...).
template <int RB, int CB, int NB = kTile>
__device__ __forceinline__ void mixed_tile_rows_cross(const float4* __restrict__ ent,
                                                      const float (&colf)[CB],
                                                      float2 (&acc)[RB][CB]) {
    static_assert(RB == 3 || RB == 4, "row triples or quadruples");
    const float kTwoPi = 6.28318530717958647692f, kInvTwoPi = 0.15915494309189533577f;
#pragma unroll 1
    for (int b = 0; b < NB; ++b) {
        const float4 e0 = ent[b];
        const float4 e1 = ent[NB + b];
        const float4 e2 = ent[2 * NB + b];
        const float4 e3 = ent[3 * NB + b];
        const float4 e4 = ent[4 * NB + b];
        // (T^3, 8 a_uv, 8 p_uv); the triples keep the last two in e3.zw
        const float4 e5 = RB > 3 ? ent[5 * NB + b] : make_float4(0.0f, 0.0f, e3.z, e3.w);
        const float tu0 = colf[0] - e0.x;
        const float t64 = tu0 * 0.015625f;
        const float x0 = fmaf(tu0, fmaf(e2.y, t64, e1.x), e0.z);
        const float d1 = fmaf(e2.y, tu0, e1.z);
        float amp = mufu_ex2(fmaf(tu0, fmaf(e2.x, t64, e0.w), e0.y));
        float rho = mufu_ex2(fmaf(e2.x, tu0, e1.y));
        const float sig = e1.w;
        // W0 = 2^(8 a_uv tu0) e^(i 8 p_uv tu0) and P_r = S_r W0^r at the first column
        const float wp = frac_turns(e5.w * tu0 * kInvTwoPi) * kTwoPi;
        const float wm = mufu_ex2(e5.z * tu0);
        const float2 W = make_float2(wm * mufu_cos(wp), wm * mufu_sin(wp));
        const float2 W2 = make_float2(fmaf(W.x, W.x, -W.y * W.y), 2.0f * W.x * W.y);
        const float2 S1 = make_float2(e2.z, e2.w), S2 = make_float2(e3.x, e3.y);
        float2 X = make_float2(fmaf(S1.x, W.x, -S1.y * W.y), fmaf(S2.x, W2.x, -S2.y * W2.y));
        float2 Y = make_float2(fmaf(S1.x, W.y, S1.y * W.x), fmaf(S2.x, W2.y, S2.y * W2.x));
        float2 P3 = make_float2(0.0f, 0.0f);
        if (RB > 3) {
            const float2 W3 = make_float2(fmaf(W2.x, W.x, -W2.y * W.y), fmaf(W2.x, W.y, W2.y * W.x));
            P3 = make_float2(fmaf(e3.z, W3.x, -e3.w * W3.y), fmaf(e3.z, W3.y, e3.w * W3.x));
        }
        const float2 Tx = make_float2(e4.x, e4.y), Ty = make_float2(e4.z, e4.w);
        const float2 Tyn = make_float2(-e4.z, -e4.w);
        const float2 T3 = make_float2(e5.x, e5.y);
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const float x = c == 0 ? x0 : fmaf((float)(16 * c * c), e2.y, fmaf((float)c, d1, x0));
            const float ex = amp * mufu_cos(x), ey = amp * mufu_sin(x);
            acc[0][c].x += ex;
            acc[0][c].y += ey;
            acc[1][c].x = fmaf(ex, X.x, fmaf(-ey, Y.x, acc[1][c].x));
            acc[1][c].y = fmaf(ex, Y.x, fmaf(ey, X.x, acc[1][c].y));
            acc[2][c].x = fmaf(ex, X.y, fmaf(-ey, Y.y, acc[2][c].x));
            acc[2][c].y = fmaf(ex, Y.y, fmaf(ey, X.y, acc[2][c].y));
            if (RB > 3) {
                acc[RB - 1][c].x = fmaf(ex, P3.x, fmaf(-ey, P3.y, acc[RB - 1][c].x));
                acc[RB - 1][c].y = fmaf(ex, P3.y, fmaf(ey, P3.x, acc[RB - 1][c].y));
            }
            if (c + 1 < CB) {
                const float2 Xn = __ffma2_rn(Y, Tyn, __fmul2_rn(X, Tx));
                Y = __ffma2_rn(Y, Tx, __fmul2_rn(X, Ty));
                X = Xn;
                if (RB > 3) {
                    const float p3x = fmaf(P3.x, T3.x, -P3.y * T3.y);
                    P3.y = fmaf(P3.x, T3.y, P3.y * T3.x);
                    P3.x = p3x;
                }
                amp *= rho;
                rho *= sig;
            }
        }
    }
}

// A compensated (hi, lo) sum rounded once to FP32 (the split partial written to memory).
__device__ __forceinline__ float2 round_pair(float2 hi, float2 lo) {
    return make_float2((float)((double)hi.x + (double)lo.x), (float)((double)hi.y + (double)lo.y));
}

// Fold a tile's FP32 sums into compensated (hi, lo) pairs (TwoSum) and clear them.
template <int RB, int CB>
__device__ __forceinline__ void mixed_fold(float2 (&acc)[RB][CB], float2 (&hi)[RB][CB],
                                           float2 (&lo)[RB][CB]) {
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            float sx, ex, sy, ey;
            two_sum(hi[r][c].x, acc[r][c].x, sx, ex);
            two_sum(hi[r][c].y, acc[r][c].y, sy, ey);
            hi[r][c] = make_float2(sx, sy);
            lo[r][c].x += ex;
            lo[r][c].y += ey;
            acc[r][c] = make_float2(0.f, 0.f);
        }
}

// mixed_fold with the (hi, lo) pairs in shared memory: comp[(r * CB + c) * kThreads + tid]
// holds (hi.re, hi.im, lo.re, lo.im) of the thread's pixel (r, c); one 16-byte load and
// store per pixel and tile, conflict-free.  Frees 4 registers per pixel for larger blocks.
template <int RB, int CB>
__device__ __forceinline__ void mixed_fold_smem(float2 (&acc)[RB][CB], float4* __restrict__ comp,
                                                int tid) {
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            float4 v = comp[(r * CB + c) * kThreads + tid];
            float sx, ex, sy, ey;
            two_sum(v.x, acc[r][c].x, sx, ex);
            two_sum(v.y, acc[r][c].y, sy, ey);
            v.x = sx;
            v.y = sy;
            v.z += ex;
            v.w += ey;
            comp[(r * CB + c) * kThreads + tid] = v;
            acc[r][c] = make_float2(0.f, 0.f);
        }
}

}  // namespace gbd
