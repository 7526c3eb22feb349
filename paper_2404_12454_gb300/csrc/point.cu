// Point evaluation (the prior method of Sec. 2.2): every beamlet is propagated to every
// pixel separately.  In this paraxial setting the beamlet leaving the reference plane with
// complex curvature P, centroid rho_c, slope theta and path L is carried by free space to
// the pixel's own axial offset z:
//     P(z) = P (I + z P)^-1,   amplitude alpha / sqrtdet(I + z P),
//     phase -k [L + z (1 + |theta|^2/2) + theta.w + w^T P(z) w / 2],  w = delta - z theta,
// and evaluated at the pixel, with sqrtdet on the eigenvalue branch.  The plane rule
// (field.cu) keeps only the terms of second order in the pixel position; on an untilted
// plane (z = 0) both are the same.  Each evaluation costs a 2x2 complex inverse, three
// complex square roots and a complex exponential in FP64, which is why the plane rule is
// the paper's acceleration.  The common carrier exp(-ik z) is applied after the sum by
// the split reduction, as for the plane rule.
#include <math.h>

#include "field_core.cuh"
#include "gbd_internal.cuh"

using gbd::cd;
using gbd::kStages;
using gbd::kThreads;

namespace {

__device__ unsigned int g_point_status = 0;

// Packed beamlet for point evaluation, 8 double2 fields in the tiled layout:
// (rho) (theta) (L, 0) (alpha) (P00) (P01) (P10) (P11)
__global__ void __launch_bounds__(128) pack_point_kernel(const gbd_beamlet* __restrict__ b, int n,
                                                         int n_pad, double2* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_pad) return;
    double2 f[gbd::kF64Fields];
    for (int m = 0; m < gbd::kF64Fields; ++m) f[m] = make_double2(0.0, 0.0);
    if (t < n) {
        const gbd_beamlet& r = b[t];
        f[0] = make_double2(r.rho[0], r.rho[1]);
        f[1] = make_double2(r.theta[0], r.theta[1]);
        f[2] = make_double2(r.path, 0.0);
        f[3] = make_double2(r.amp[0], r.amp[1]);
        for (int q = 0; q < 4; ++q) f[4 + q] = make_double2(r.curv[2 * q], r.curv[2 * q + 1]);
    }
    double2* tile = out + (size_t)(t / gbd::kTile) * gbd::kF64Fields * gbd::kTile;
    const int l = t % gbd::kTile;
    for (int m = 0; m < gbd::kF64Fields; ++m) tile[m * gbd::kTile + l] = f[m];
}

__device__ __forceinline__ cd cexp_d(cd z) {
    double sn, cs;
    sincos(z.im, &sn, &cs);
    const double a = exp(z.re);
    return cd{a * cs, a * sn};
}

template <int CB>
__global__ void __launch_bounds__(kThreads)
    field_point_kernel(const double2* __restrict__ coef, int n_tiles, int tiles_per_split,
                       gbd_project_params G, double2* __restrict__ partial, uint32_t spins) {
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

    const int row = blockIdx.y * 8 + warp;
    const int col0 = blockIdx.x * (32 * CB) + lane;
    const double k = 2.0 * M_PI / G.wavelength;
    // lab offsets of this thread's pixels from the reference point
    double vx[CB], vy[CB], vz[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) {
        const double sx = (col0 + 32 * c - G.nx / 2) * G.px, sy = (row - G.ny / 2) * G.py;
        vx[c] = G.M[0] * sx + G.M[1] * sy;
        vy[c] = G.M[2] * sx + G.M[3] * sy;
        vz[c] = G.n[0] * sx + G.n[1] * sy;
    }
    double acc_re[CB], acc_im[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) acc_re[c] = acc_im[c] = 0.0;

    int kk = 0;
    for (; ok && kk < ts.nt; ++kk) {
        if (!ts.acquire(kk, spins)) {
            ok = false;
            break;
        }
        const double2* st = ts.tile(kk);
#pragma unroll 1
        for (int b = 0; b < gbd::kTile; ++b) {
            const double2 rho = st[b], th = st[gbd::kTile + b], Lr = st[2 * gbd::kTile + b];
            const double2 al = st[3 * gbd::kTile + b];
            if (al.x == 0.0 && al.y == 0.0) continue;  // padding
            const cd P00{st[4 * gbd::kTile + b].x, st[4 * gbd::kTile + b].y};
            const cd P01{st[5 * gbd::kTile + b].x, st[5 * gbd::kTile + b].y};
            const cd P10{st[6 * gbd::kTile + b].x, st[6 * gbd::kTile + b].y};
            const cd P11{st[7 * gbd::kTile + b].x, st[7 * gbd::kTile + b].y};
            const double th2 = th.x * th.x + th.y * th.y;
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const double z = vz[c];
                const double wx = vx[c] - rho.x - z * th.x, wy = vy[c] - rho.y - z * th.y;
                // Mz = I + z P, Pz = P Mz^-1
                const cd m00 = gbd::mk(1.0) + z * P00, m01 = z * P01, m10 = z * P10,
                         m11 = gbd::mk(1.0) + z * P11;
                const cd det = m00 * m11 - m01 * m10;
                const cd rd = gbd::cdiv(gbd::mk(1.0), det);
                const cd i00 = m11 * rd, i01 = gbd::mk(0.0) - m01 * rd, i10 = gbd::mk(0.0) - m10 * rd,
                         i11 = m00 * rd;
                const cd q00 = P00 * i00 + P01 * i10, q01 = P00 * i01 + P01 * i11;
                const cd q10 = P10 * i00 + P11 * i10, q11 = P10 * i01 + P11 * i11;
                const cd quad = wx * (wx * q00 + wy * q01) + wy * (wx * q10 + wy * q11);
                // sqrtdet(Mz) from the eigenvalues
                const cd ht = 0.5 * (m00 + m11);
                const cd disc = gbd::csqrt_p(ht * ht - det);
                const cd sd = gbd::csqrt_p(ht + disc) * gbd::csqrt_p(ht - disc);
                const cd amp = gbd::cdiv(cd{al.x, al.y}, sd);
                // -ik [L + z |theta|^2/2 + theta.w + quad/2] (the carrier z is applied later)
                const double path = Lr.x + 0.5 * z * th2 + th.x * wx + th.y * wy;
                const cd ex{0.5 * k * quad.im, -k * (path + 0.5 * quad.re)};
                const cd e = amp * cexp_d(ex);
                acc_re[c] += e.re;
                acc_im[c] += e.im;
            }
        }
        if (!ts.release(kk, lane, warp, spins)) {
            ok = false;
            ++kk;
            break;
        }
    }
    if (!ok) {
        atomicOr(&g_point_status, gbd::kStatusTimeout);
        if (tid == 0) ts.drain(kk, spins);
        return;
    }
    if (row >= G.ny) return;
    double2* out = partial + (size_t)blockIdx.z * G.nx * G.ny;
#pragma unroll
    for (int c = 0; c < CB; ++c) {
        const int col = col0 + 32 * c;
        if (col < G.nx) out[(size_t)row * G.nx + col] = make_double2(acc_re[c], acc_im[c]);
    }
}

constexpr int kPointCB = 2;

}  // namespace

long gbd_point_pixel_ctas(int nx, int ny) {
    return (long)((nx + 32 * kPointCB - 1) / (32 * kPointCB)) * ((ny + 7) / 8);
}

int gbd_point_occupancy() {
    const size_t smem = (size_t)kStages * gbd::kF64TileBytes;
    cudaFuncSetAttribute(field_point_kernel<kPointCB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, field_point_kernel<kPointCB>, kThreads,
                                                      smem) != cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

cudaError_t gbd_launch_point(const gbd_beamlet* b, int n, const gbd_project_params& p, void* coeffs,
                             int splits, int tiles_per_split, double2* partial, uint32_t spins,
                             cudaStream_t s) {
    const int n_pad = (n + gbd::kTile - 1) / gbd::kTile * gbd::kTile;
    pack_point_kernel<<<(n_pad + 127) / 128, 128, 0, s>>>(b, n, n_pad, static_cast<double2*>(coeffs));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)kStages * gbd::kF64TileBytes;
    e = cudaFuncSetAttribute(field_point_kernel<kPointCB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.nx + 32 * kPointCB - 1) / (32 * kPointCB), (p.ny + 7) / 8, splits);
    field_point_kernel<kPointCB><<<grid, kThreads, smem, s>>>(
        static_cast<const double2*>(coeffs), n_pad / gbd::kTile, tiles_per_split, p, partial, spins);
    return cudaGetLastError();
}

// The status word: copied into pinned host memory on the caller's stream (gbd_sync), and
// cleared once it has been reported.
cudaError_t gbd_point_status_fetch(unsigned* host, cudaStream_t s) {
    return cudaMemcpyFromSymbolAsync(host, g_point_status, sizeof(unsigned), 0,
                                     cudaMemcpyDeviceToHost, s);
}
void gbd_point_status_clear() {
    const unsigned zero = 0;
    cudaMemcpyToSymbol(g_point_status, &zero, sizeof(zero));
}
