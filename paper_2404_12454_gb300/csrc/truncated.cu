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

// The edge beamlets' sum added onto the field, kEdgePix consecutive pixels (row-major
// order) per thread; the edge records are staged through shared memory (converted to T) 32
// beamlets at a time, and each thread loads a record once for its pixels.  Per pixel the
// Faddeeva argument (i zeta or -i zeta) is selected without a branch; the Gaussian term
// is evaluated only where Re zeta < 0 (neighbouring pixels mostly agree on the sign).
constexpr int kEdgeChunk = 32, kEdgePix = 4;
template <typename T, int NW>
__global__ void __launch_bounds__(256) field_edge_kernel(const double2* __restrict__ rec,
                                                         int n_edge, int nx, int ny,
                                                         FaddeevaT<T, NW> F,
                                                         Cplx<T>* __restrict__ out) {
    __shared__ __align__(16) T s[kEdgeChunk][2 * gbd::kEdgeFields];
    const long long npix = (long long)nx * ny;
    const long long p0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * kEdgePix;
    T pu[kEdgePix], pv[kEdgePix], accr[kEdgePix], acci[kEdgePix];
#pragma unroll
    for (int c = 0; c < kEdgePix; ++c) {
        const long long p = min(p0 + c, npix - 1);
        pu[c] = (T)(p % nx);
        pv[c] = (T)(p / nx);
        accr[c] = acci[c] = (T)0;
    }
    for (int b0 = 0; b0 < n_edge; b0 += kEdgeChunk) {
        __syncthreads();
        for (int q = threadIdx.x; q < kEdgeChunk * gbd::kEdgeFields; q += blockDim.x) {
            const int bb = b0 + q / gbd::kEdgeFields, f = q % gbd::kEdgeFields;
            const double2 v = bb < n_edge ? rec[(size_t)bb * gbd::kEdgeFields + f]
                                          : make_double2(0.0, 0.0);
            s[q / gbd::kEdgeFields][2 * f] = (T)v.x;
            s[q / gbd::kEdgeFields][2 * f + 1] = (T)v.y;
        }
        __syncthreads();
        const int nb = min(kEdgeChunk, n_edge - b0);
        for (int b = 0; b < nb; ++b) {
            T r[2 * gbd::kEdgeFields];
#pragma unroll
            for (int m = 0; m < 2 * gbd::kEdgeFields; ++m) r[m] = s[b][m];
#pragma unroll
            for (int c = 0; c < kEdgePix; ++c) {
                const T tu = pu[c] - r[0], tv = pv[c] - r[1];
                const T tuu = tu * tu, tuv = tu * tv, tvv = tv * tv;
                const T zr = r[14] + r[16] * tu + r[18] * tv;
                const T zi = r[15] + r[17] * tu + r[19] * tv;
                const bool neg = zr < (T)0;
                // i zeta = (-zi, zr); -i zeta = (zi, -zr): the one in the upper half-plane
                T wr, wi;
                faddeeva<T, NW>(neg ? zi : -zi, neg ? -zr : zr, F, wr, wi);
                const T ga = r[20] + r[22] * tu + r[24] * tv + r[26] * tuu + r[28] * tuv + r[30] * tvv;
                const T gp = r[21] + r[23] * tu + r[25] * tv + r[27] * tuu + r[29] * tuv + r[31] * tvv;
                T gc, gs;
                cis_turns(gp, gc, gs);
                const T gm = pow2(ga);
                T tr = gm * (gc * wr - gs * wi), ti = gm * (gc * wi + gs * wr);
                if (neg) {
                    // where Re zeta < 0 the cut field is E - e^Psi w(-i zeta)
                    const T ea = r[2] + r[4] * tu + r[6] * tv + r[8] * tuu + r[10] * tuv +
                                 r[12] * tvv;
                    const T ep = r[3] + r[5] * tu + r[7] * tv + r[9] * tuu + r[11] * tuv +
                                 r[13] * tvv;
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
#pragma unroll
    for (int c = 0; c < kEdgePix; ++c) {
        if (p0 + c >= npix) break;
        Cplx<T> o = out[p0 + c];
        o.x += accr[c];
        o.y += acci[c];
        out[p0 + c] = o;
    }
}

}  // namespace

cudaError_t gbd_launch_field_edge(int precision, const double2* edge_records, int n_edge, int nx,
                                  int ny, void* out, cudaStream_t s) {
    if (n_edge <= 0) return cudaSuccess;
    const long long npix = (long long)nx * ny;
    const unsigned blocks = (unsigned)((npix + 256LL * kEdgePix - 1) / (256LL * kEdgePix));
    if (precision == GBD_PREC_F64)
        field_edge_kernel<double, 36><<<blocks, 256, 0, s>>>(
            edge_records, n_edge, nx, ny, faddeeva_table<double, 36>(),
            static_cast<Cplx<double>*>(out));
    else
        field_edge_kernel<float, 16><<<blocks, 256, 0, s>>>(
            edge_records, n_edge, nx, ny, faddeeva_table<float, 16>(),
            static_cast<Cplx<float>*>(out));
    return cudaGetLastError();
}
