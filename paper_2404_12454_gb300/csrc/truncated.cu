// Truncated beamlets at the aperture edge (the paper's Sec. 1 and Conclusion point to Worku
// & Gross's truncated Gaussian beamlets for hard edges; the plane-evaluation method takes any
// closed-form solution of the Collins integral, Eq. collins).
//
// The decomposition grid is extended to every centre within R + margin w0; beamlets within
// margin w0 of the edge have their input Gaussian cut by the aperture's tangent half-plane
// n.(r - r_j) <= d_j.  Integrated over that half-plane, the Collins integral of a Gaussian is
// the whole beamlet times 1/2 erfc(zeta), zeta affine in the position on an untilted plane,
// so each edge beamlet becomes (besides its Gaussian) one affine and one more quadratic form
// in pixel coordinates (project_edge_kernel), and per pixel
//     E 1/2 erfc(zeta) = e^Psi w(i zeta)          (Re zeta >= 0)
//                      = E - e^Psi w(-i zeta)     (Re zeta <  0),   Psi = ln E - zeta^2 + ln 1/2,
// with w(z) = e^(-z^2) erfc(-iz) the Faddeeva function, evaluated in the closed upper
// half-plane only.  w is Weideman's rational approximation (J.A.C. Weideman, "Computation of
// the complex error function", SIAM J. Numer. Anal. 31, 1994): with L = (N / sqrt 2)^(1/2),
// Z = (L + iz) / (L - iz),
//     w(z) ~ 2 sum_{n=1}^{N} a_n Z^(n-1) / (L - iz)^2 + 1 / (sqrt(pi) (L - iz)),
// a_n the Fourier coefficients of f(t) = e^(-t^2) (L^2 + t^2) in theta, t = L tan(theta/2),
// computed here on the host by a direct cosine sum over 2N sample angles.  N = 36 for the
// FP64 path (relative error 2e-14 against a reference Faddeeva function on the upper
// half-plane), N = 16 for the mixed path (4e-7).
//
// The interior beamlets run through gbd_field unchanged; the edge kernel adds the edge
// beamlets' sum onto its output.
#include <math.h>

#include <mutex>

#include "gbd_internal.cuh"

namespace {

template <int NW>
struct FaddeevaCoef {
    double L;
    double a[NW];  // a_1 .. a_N
};

template <int NW>
FaddeevaCoef<NW> weideman_coefficients() {
    FaddeevaCoef<NW> c;
    const int M = 2 * NW;
    const double L = sqrt(NW / sqrt(2.0));
    c.L = L;
    // f sampled at theta_k = k pi / M, k = -M+1 .. M-1 (f = 0 at k = -M); f is even in k,
    // so its Fourier coefficients are the cosine sums below, divided by 2M
    double f[2 * NW];
    for (int k = 0; k < M; ++k) {
        const double t = L * tan(0.5 * k * M_PI / M);
        f[k] = exp(-t * t) * (L * L + t * t);
    }
    for (int n = 1; n <= NW; ++n) {
        double s = f[0];
        for (int k = 1; k < M; ++k) s += 2.0 * f[k] * cos(M_PI * n * k / M);
        c.a[n - 1] = s / (2.0 * M);
    }
    return c;
}

template <typename T, int NW>
struct FaddeevaT {
    T L;
    T a[NW];
};

template <typename T, int NW>
const FaddeevaT<T, NW>& faddeeva_table() {
    static FaddeevaT<T, NW> t;
    static std::once_flag once;
    std::call_once(once, [] {
        const FaddeevaCoef<NW> c = weideman_coefficients<NW>();
        t.L = (T)c.L;
        for (int n = 0; n < NW; ++n) t.a[n] = (T)c.a[n];
    });
    return t;
}

// w(z) for Im z >= 0 (z = zr + i zi): q = 1/(L - iz), Z = (L + iz) q, w = (2 p(Z) q + 1/sqrt(pi)) q.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <typename T, int NW>
__device__ __forceinline__ void faddeeva(T zr, T zi, const FaddeevaT<T, NW>& F, T& wr, T& wi) {
    const T dr = F.L + zi, di = -zr;  // L - iz
    const T inv = recip(dr * dr + di * di);
    const T qr = dr * inv, qi = -di * inv;  // 1 / (L - iz)
    const T nr = F.L - zi, ni = zr;         // L + iz
    const T Zr = nr * qr - ni * qi, Zi = nr * qi + ni * qr;
    T pr = F.a[NW - 1], pi = (T)0;
#pragma unroll
    for (int n = NW - 2; n >= 0; --n) {
        const T tr = pr * Zr - pi * Zi + F.a[n];
        pi = pr * Zi + pi * Zr;
        pr = tr;
    }
    const T isqrtpi = (T)0.56418958354775628695;
    const T sr = (T)2 * (pr * qr - pi * qi) + isqrtpi, si = (T)2 * (pr * qi + pi * qr);
    wr = sr * qr - si * qi;
    wi = sr * qi + si * qr;
}

// cos and sin of 2 pi p: the turns reduced exactly to [-1/2, 1/2], then (FP32) the MUFU
// sin/cos of the radians in [-pi, pi] (absolute error ~1e-6, well inside the mixed path's
// tolerance for these edge terms).
__device__ __forceinline__ void cis_turns(float p, float& c, float& s) {
    __sincosf(6.28318530717958647692f * (p - rintf(p)), &s, &c);
}
__device__ __forceinline__ void cis_turns(double p, double& c, double& s) {
    sincospi(2.0 * (p - rint(p)), &s, &c);
}
__device__ __forceinline__ float pow2(float a) { return exp2f(a); }
__device__ __forceinline__ double pow2(double a) { return exp2(a); }

template <typename T>
struct Cplx {
    T x, y;
};

// One Taylor step of w from z to z + h (FP32 path): the derivatives at z follow from
// w' = -2 z w + 2 i / sqrt(pi) by w^(n+1) = -2 z w^(n) - 2 n w^(n-1); to 4th order the step
// keeps 4e-7 relative over a segment of 8 steps while |h| (2 |z|_1 + 3) <= 0.2 (checked
// against a reference Faddeeva function off the device).  The step and its scaled copies
// for the Horner evaluation, h/4, h/3, h/2, h, are formed once per run of steps.
struct TaylorStep {
    float r[4], i[4];
};
__device__ __forceinline__ TaylorStep taylor_step(float hr, float hi) {
    const float third = 0.333333343f;
    return {{0.25f * hr, third * hr, 0.5f * hr, hr}, {0.25f * hi, third * hi, 0.5f * hi, hi}};
}
__device__ __forceinline__ void faddeeva_step(float zr, float zi, const TaylorStep& h, float& wr,
                                              float& wi) {
    const float c = 1.12837916709551257390f;  // 2 / sqrt(pi)
    const float d1r = -2.0f * fmaf(zr, wr, -zi * wi), d1i = fmaf(-2.0f, fmaf(zr, wi, zi * wr), c);
    const float d2r = fmaf(-2.0f, wr, -2.0f * fmaf(zr, d1r, -zi * d1i));
    const float d2i = fmaf(-2.0f, wi, -2.0f * fmaf(zr, d1i, zi * d1r));
    const float d3r = fmaf(-4.0f, d1r, -2.0f * fmaf(zr, d2r, -zi * d2i));
    const float d3i = fmaf(-4.0f, d1i, -2.0f * fmaf(zr, d2i, zi * d2r));
    const float d4r = fmaf(-6.0f, d2r, -2.0f * fmaf(zr, d3r, -zi * d3i));
    const float d4i = fmaf(-6.0f, d2i, -2.0f * fmaf(zr, d3i, zi * d3r));
    // Horner in h: w + h (d1 + h/2 (d2 + h/3 (d3 + h/4 d4)))
    float ar = d4r, ai = d4i, tr;
    tr = fmaf(h.r[0], ar, fmaf(-h.i[0], ai, d3r));
    ai = fmaf(h.r[0], ai, fmaf(h.i[0], ar, d3i));
    ar = tr;
    tr = fmaf(h.r[1], ar, fmaf(-h.i[1], ai, d2r));
    ai = fmaf(h.r[1], ai, fmaf(h.i[1], ar, d2i));
    ar = tr;
    tr = fmaf(h.r[2], ar, fmaf(-h.i[2], ai, d1r));
    ai = fmaf(h.r[2], ai, fmaf(h.i[2], ar, d1i));
    ar = tr;
    tr = fmaf(h.r[3], ar, fmaf(-h.i[3], ai, wr));
    wi = fmaf(h.r[3], ai, fmaf(h.i[3], ar, wi));
    wr = tr;
}

// The edge beamlets' sum over split blockIdx.y (beamlets [y per_split, (y + 1) per_split))
// into that split's partial field.  A thread takes kEdgePix consecutive pixels of one row;
// the edge records are staged through shared memory (converted to T) 32 beamlets at a time.  Per beamlet the quadratic forms' row terms are formed once for
// the thread's row (then 2 FMA per form and pixel, zeta 1 FMA).  The Faddeeva argument
// (i zeta or -i zeta, whichever lies in the upper half-plane) is selected without a
// branch; STEP (the FP32 path): w is evaluated exactly at the segment's first pixel,
// where the sign of Re zeta changes, and where the step is too long for the Taylor step,
// and Taylor-stepped from the previous pixel otherwise.  The Gaussian term is evaluated
// only where Re zeta < 0 (neighbouring pixels mostly agree on the sign).
constexpr int kEdgeChunk = 32, kEdgePix = 8;
template <typename T, int NW, bool STEP>
__global__ void __launch_bounds__(256) field_edge_kernel(const double2* __restrict__ rec,
                                                         int n_edge, int per_split, int nx,
                                                         int ny, FaddeevaT<T, NW> F,
                                                         Cplx<T>* __restrict__ partial) {
    __shared__ __align__(16) T s[kEdgeChunk][2 * gbd::kEdgeFields];
    const int segs_x = (nx + kEdgePix - 1) / kEdgePix;
    const long long seg = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = seg < (long long)segs_x * ny;
    const int row = live ? (int)(seg / segs_x) : 0;
    const int col0 = live ? (int)(seg % segs_x) * kEdgePix : 0;
    T accr[kEdgePix], acci[kEdgePix];
#pragma unroll
    for (int c = 0; c < kEdgePix; ++c) accr[c] = acci[c] = (T)0;
    const int b_lo = blockIdx.y * per_split, b_hi = min(n_edge, b_lo + per_split);
    for (int b0 = b_lo; b0 < b_hi; b0 += kEdgeChunk) {
        __syncthreads();
        for (int q = threadIdx.x; q < kEdgeChunk * gbd::kEdgeFields; q += blockDim.x) {
            const int bb = b0 + q / gbd::kEdgeFields, f = q % gbd::kEdgeFields;
            const double2 v = bb < b_hi ? rec[(size_t)bb * gbd::kEdgeFields + f]
                                        : make_double2(0.0, 0.0);
            s[q / gbd::kEdgeFields][2 * f] = (T)v.x;
            s[q / gbd::kEdgeFields][2 * f + 1] = (T)v.y;
        }
        __syncthreads();
        const int nb = min(kEdgeChunk, b_hi - b0);
        for (int b = 0; b < nb; ++b) {
            const T* r = s[b];
            const T tu0 = (T)col0 - r[0], tv = (T)row - r[1];
            // row terms: form(tu) = A + tu (B + C tu)
            const T eA = fma(tv, fma(r[12], tv, r[6]), r[2]), eB = fma(r[10], tv, r[4]);
            const T pA = fma(tv, fma(r[13], tv, r[7]), r[3]), pB = fma(r[11], tv, r[5]);
            const T gA = fma(tv, fma(r[30], tv, r[24]), r[20]), gB = fma(r[28], tv, r[22]);
            const T qA = fma(tv, fma(r[31], tv, r[25]), r[21]), qB = fma(r[29], tv, r[23]);
            const T zr0 = fma(r[18], tv, r[14]), zi0 = fma(r[19], tv, r[15]);
            T wr = (T)0, wi = (T)0, xpr = (T)0, xpi = (T)0;
            bool pneg = false;
            // zeta steps by (r16, r17) from pixel to pixel, so its image x = -i zeta
            // (Re zeta < 0) or i zeta steps by +-(r17, -r16): the Taylor step is fixed by
            // the sign, which only changes at an exact evaluation
            TaylorStep hs{};
            const T mh = fabs(r[16]) + fabs(r[17]);  // |h|_1
#pragma unroll
            for (int c = 0; c < kEdgePix; ++c) {
                const T tu = tu0 + (T)c;
                const T zr = fma(r[16], tu, zr0), zi = fma(r[17], tu, zi0);
                const bool neg = zr < (T)0;
                // i zeta = (-zi, zr); -i zeta = (zi, -zr): the one in the upper half-plane
                const T xr = neg ? zi : -zi, xi = neg ? -zr : zr;
                bool exact = true;
                if constexpr (STEP) {
                    if (c > 0 && neg == pneg) {
                        const T zz = fabs(xpr) + fabs(xpi);
                        exact = !(mh * fma((T)2, zz, (T)3) <= (T)0.2);
                    }
                }
                if (exact) {
                    faddeeva<T, NW>(xr, xi, F, wr, wi);
                    if constexpr (STEP)
                        hs = taylor_step(neg ? r[17] : -r[17], neg ? -r[16] : r[16]);
                } else {
                    if constexpr (STEP) faddeeva_step(xpr, xpi, hs, wr, wi);
                }
                xpr = xr;
                xpi = xi;
                pneg = neg;
                const T ga = fma(tu, fma(r[26], tu, gB), gA);
                const T gp = fma(tu, fma(r[27], tu, qB), qA);
                T gc, gs;
                cis_turns(gp, gc, gs);
                const T gm = pow2(ga);
                T tr = gm * (gc * wr - gs * wi), ti = gm * (gc * wi + gs * wr);
                if (neg) {
                    // where Re zeta < 0 the cut field is E - e^Psi w(-i zeta)
                    const T ea = fma(tu, fma(r[8], tu, eB), eA);
                    const T ep = fma(tu, fma(r[9], tu, pB), pA);
                    T ec, es;
                    cis_turns(ep, ec, es);
                    const T em = pow2(ea);
                    tr = em * ec - tr;
                    ti = em * es - ti;
                }
                accr[c] += tr;
                acci[c] += ti;
            }
        }
    }
    if (!live) return;
    Cplx<T>* part = partial + (size_t)blockIdx.y * nx * ny + (size_t)row * nx + col0;
#pragma unroll
    for (int c = 0; c < kEdgePix; ++c) {
        if (col0 + c >= nx) break;
        part[c] = Cplx<T>{accr[c], acci[c]};
    }
}

// out += the splits' partial fields, added in split order.
template <typename T>
__global__ void __launch_bounds__(256) field_edge_reduce_kernel(const Cplx<T>* __restrict__ partial,
                                                                int splits, long long npix,
                                                                Cplx<T>* __restrict__ out) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    T sx = partial[p].x, sy = partial[p].y;
    for (int k = 1; k < splits; ++k) {
        sx += partial[(size_t)k * npix + p].x;
        sy += partial[(size_t)k * npix + p].y;
    }
    out[p].x += sx;
    out[p].y += sy;
}

// Beamlet splits of the edge kernel: about 8 CTAs per SM in all (each thread walks its
// split's beamlets serially), at least 64 beamlets per split.
int edge_splits(int n_edge, int nx, int ny) {
    const long long segs = (long long)((nx + kEdgePix - 1) / kEdgePix) * ny;
    const long long pix_ctas = (segs + 255) / 256;
    long long want = (8LL * 152 + pix_ctas - 1) / pix_ctas;
    const long long cap = (n_edge + 63) / 64;
    if (want > cap) want = cap;
    return want < 1 ? 1 : (int)want;
}

}  // namespace

size_t gbd_field_edge_partial_bytes(int precision, int n_edge, int nx, int ny) {
    if (n_edge <= 0) return 0;
    const size_t elem = precision == GBD_PREC_F64 ? sizeof(Cplx<double>) : sizeof(Cplx<float>);
    return (size_t)edge_splits(n_edge, nx, ny) * nx * ny * elem;
}

cudaError_t gbd_launch_field_edge(int precision, const double2* edge_records, int n_edge, int nx,
                                  int ny, void* out, void* partial, cudaStream_t s) {
    if (n_edge <= 0) return cudaSuccess;
    const int splits = edge_splits(n_edge, nx, ny);
    const int per = (n_edge + splits - 1) / splits;
    const int per_split = (per + kEdgeChunk - 1) / kEdgeChunk * kEdgeChunk;
    const long long segs = (long long)((nx + kEdgePix - 1) / kEdgePix) * ny;
    const dim3 grid((unsigned)((segs + 255) / 256), (unsigned)splits);
    const long long npix = (long long)nx * ny;
    const unsigned rblocks = (unsigned)((npix + 255) / 256);
    if (precision == GBD_PREC_F64) {
        field_edge_kernel<double, 36, false><<<grid, 256, 0, s>>>(
            edge_records, n_edge, per_split, nx, ny, faddeeva_table<double, 36>(),
            static_cast<Cplx<double>*>(partial));
        field_edge_reduce_kernel<double><<<rblocks, 256, 0, s>>>(
            static_cast<const Cplx<double>*>(partial), splits, npix, static_cast<Cplx<double>*>(out));
    } else {
        field_edge_kernel<float, 16, true><<<grid, 256, 0, s>>>(
            edge_records, n_edge, per_split, nx, ny, faddeeva_table<float, 16>(),
            static_cast<Cplx<float>*>(partial));
        field_edge_reduce_kernel<float><<<rblocks, 256, 0, s>>>(
            static_cast<const Cplx<float>*>(partial), splits, npix, static_cast<Cplx<float>*>(out));
    }
    return cudaGetLastError();
}
