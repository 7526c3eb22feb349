// Beamlet decomposition + differential ray trace (FP64), and the per-beamlet projection
// onto the detector plane that turns each beamlet into one complex quadratic form.
//
// Trace: Sec. 2.2 (steps 1 and 4: chief + parabasal rays, differential ABCD), Eq. OF,
// Eq. abcd_sys (thin lens then distance), Eq. gauss_prop (complex curvature law and the
// 1/sqrtdet amplitude, with the eigenvalue route of App. C for the branch).
// Projection: Eq. collins_factored with the chief-ray propagation of Eqs. ab_prop /
// cd_prop, extended to a plane tilted about the reference point by second-order
// expansion in the pixel position.
#include <math.h>

#include "field_core.cuh"
#include "gbd_internal.cuh"

static_assert(sizeof(gbd_beamlet) == 36 * sizeof(double), "gbd_beamlet is 36 doubles");

using gbd::cd;

namespace {

// --------------------------------------------------------------------- trace --

// Number of grid centres inside the pupil in row j of an N x N cell-centred grid:
// a = 2i - (N-1) runs over the integers of N-1's parity with a^2 <= N^2 - b^2.
__device__ __forceinline__ int row_extent(int j, int N) {
    long long b = 2LL * j - (N - 1);
    long long r2 = (long long)N * N - b * b;
    if (r2 < 0) return -1;
    long long a = (long long)sqrt((double)r2);
    while (a * a > r2) --a;
    while ((a + 1) * (a + 1) <= r2) ++a;
    if (((a - (N - 1)) & 1LL) != 0) --a;
    return (int)a;  // -1 when the row is empty
}

struct Ray {
    double x, y, tx, ty, path;
};

// OPD plate polynomial and its gradient at (x, y).
__device__ void plate_eval(const gbd_trace_params& P, double x, double y, double& W, double& gx,
                           double& gy) {
    const double inv_r = 1.0 / P.zern_radius;
    const double xi = x * inv_r, eta = y * inv_r;
    double xp[11], yp[11];
    xp[0] = yp[0] = 1.0;
    for (int q = 1; q <= P.zdeg; ++q) {
        xp[q] = xp[q - 1] * xi;
        yp[q] = yp[q - 1] * eta;
    }
    double w = 0.0, dx = 0.0, dy = 0.0;
    for (int g = 0; g <= P.zdeg; ++g) {
        for (int b = 0; b <= g; ++b) {
            const int a = g - b;
            const double c = P.zpoly[gbd::plate_index(a, b)];
            if (c == 0.0) continue;
            w += c * xp[a] * yp[b];
            if (a > 0) dx += c * a * xp[a - 1] * yp[b];
            if (b > 0) dy += c * b * xp[a] * yp[b - 1];
        }
    }
    W = w;
    gx = dx * inv_r;
    gy = dy * inv_r;
}

// [plate] -> thin lens -> free space d.  `path` is the optical path beyond the axis.
__device__ void propagate(const gbd_trace_params& P, Ray& r) {
    if (P.zdeg >= 0) {
        double W, gx, gy;
        plate_eval(P, r.x, r.y, W, gx, gy);
        r.path += W;
        r.tx += gx;
        r.ty += gy;
    }
    r.path -= 0.5 * (r.x * r.x + r.y * r.y) * P.inv_f;
    r.tx -= r.x * P.inv_f;
    r.ty -= r.y * P.inv_f;
    r.x += P.d * r.tx;
    r.y += P.d * r.ty;
    r.path += 0.5 * P.d * (r.tx * r.tx + r.ty * r.ty);
}

// Ray propagators: map a ray leaving the pupil plane at (x, y) with slopes (tx, ty) to its
// position, slopes and optical path (in excess of the axial ray's) on the reference plane.
struct LensTracer {
    const gbd_trace_params& P;
    __device__ void operator()(Ray& r) const { propagate(P, r); }
};

// Real rays through reflective conic surfaces.  Along the ray q(t) = q + t u (q from the
// vertex) the implicit surface F = c (x^2 + y^2) - 2 z + (1 + K) c z^2 is the quadratic
// a t^2 + b t + c0, and dF/dt = 2 a t + b = +-sqrt(b^2 - 4 a c0) at its two roots.  The
// sheet through the vertex has grad F ~ (0, 0, -2) there, so the wanted root is the one with
// dF/dt of sign s = -sign(u_z).  It is evaluated without cancellation: (-b + s r) / 2a when
// -b and s r agree in sign, else 2 c0 / (-b - s r), which stays finite as a -> 0 (nearly
// flat or parabolic surfaces).  Normals come from the implicit gradient.
struct MirrorTracer {
    const gbd_mirror_params& M;
    __device__ void operator()(Ray& r) const {
        const double nrm = rsqrt(1.0 + r.tx * r.tx + r.ty * r.ty);
        double ux = r.tx * nrm, uy = r.ty * nrm, uz = nrm;
        double px = r.x, py = r.y, pz = M.z_ep, path = 0.0;
        for (int k = 0; k < M.n; ++k) {
            const double c = M.c[k], e = (1.0 + M.K[k]) * c;
            const double qz = pz - M.z[k];
            const double a = c * (ux * ux + uy * uy) + e * uz * uz;
            const double b = 2.0 * (c * (px * ux + py * uy) - uz + e * qz * uz);
            const double c0 = c * (px * px + py * py) - 2.0 * qz + e * qz * qz;
            const double sr = copysign(sqrt(fmax(b * b - 4.0 * a * c0, 0.0)), -uz);
            const double t = (b * sr < 0.0) ? (sr - b) / (2.0 * a) : 2.0 * c0 / (-b - sr);
            px += t * ux;
            py += t * uy;
            pz += t * uz;
            path += t;
            double nx = 2.0 * c * px, ny = 2.0 * c * py, nz = -2.0 + 2.0 * e * (pz - M.z[k]);
            const double inv = rsqrt(nx * nx + ny * ny + nz * nz);
            nx *= inv;
            ny *= inv;
            nz *= inv;
            const double un = ux * nx + uy * ny + uz * nz;
            ux -= 2.0 * un * nx;
            uy -= 2.0 * un * ny;
            uz -= 2.0 * un * nz;
        }
        const double t = (M.z_img - pz) / uz;
        r.x = px + t * ux;
        r.y = py + t * uy;
        r.tx = ux / uz;
        r.ty = uy / uz;
        r.path = path + t - M.axial_path;
    }
};

template <class Tracer>
__device__ void trace_one(const Tracer& T, const gbd_grid& g, int N, int i, int j,
                          gbd_beamlet* out) {
    const double s = g.s, w0 = g.w0, weight = g.weight, h = g.h, dth = g.dth;
    const double p1 = g.p1;  // P1 = i * p1 * I
    const double cx = (i - 0.5 * (N - 1)) * s, cy = (j - 0.5 * (N - 1)) * s;

    Ray c{cx, cy, 0.0, 0.0, 0.0};
    T(c);
    Ray wx{cx + h, cy, 0.0, 0.0, 0.0}, wy{cx, cy + h, 0.0, 0.0, 0.0};
    Ray dx{cx, cy, dth, 0.0, 0.0}, dy{cx, cy, 0.0, dth, 0.0};
    T(wx);
    T(wy);
    T(dx);
    T(dy);
    // columns: derivative of (x, y, tx, ty) with respect to (x0, y0 | tx0, ty0); one
    // reciprocal per step (from the grid) instead of 16 FP64 divisions (within an ulp)
    const double ih = g.ih, idt = g.idt;
    double A[4] = {(wx.x - c.x) * ih, (wy.x - c.x) * ih, (wx.y - c.y) * ih, (wy.y - c.y) * ih};
    double C[4] = {(wx.tx - c.tx) * ih, (wy.tx - c.tx) * ih, (wx.ty - c.ty) * ih,
                   (wy.ty - c.ty) * ih};
    double B[4] = {(dx.x - c.x) * idt, (dy.x - c.x) * idt, (dx.y - c.y) * idt, (dy.y - c.y) * idt};
    double Dm[4] = {(dx.tx - c.tx) * idt, (dy.tx - c.tx) * idt, (dx.ty - c.ty) * idt,
                    (dy.ty - c.ty) * idt};

    // M = A + B P1, N = C + D P1 (P1 purely imaginary, isotropic)
    cd M[4], Nn[4];
    for (int q = 0; q < 4; ++q) {
        M[q] = cd{A[q], B[q] * p1};
        Nn[q] = cd{C[q], Dm[q] * p1};
    }
    const cd detM = M[0] * M[3] - M[1] * M[2];
    // M^-1 = adj(M) / det
    const cd rdet = gbd::cdiv(gbd::mk(1.0), detM);
    const cd Mi[4] = {M[3] * rdet, gbd::mk(0.0) - M[1] * rdet, gbd::mk(0.0) - M[2] * rdet,
                      M[0] * rdet};
    cd Pm[4];
    Pm[0] = Nn[0] * Mi[0] + Nn[1] * Mi[2];
    Pm[1] = Nn[0] * Mi[1] + Nn[1] * Mi[3];
    Pm[2] = Nn[2] * Mi[0] + Nn[3] * Mi[2];
    Pm[3] = Nn[2] * Mi[1] + Nn[3] * Mi[3];
    // sqrtdet(M): principal roots of the eigenvalues tr/2 +- sqrt(tr^2/4 - det)
    const cd half_tr = 0.5 * (M[0] + M[3]);
    const cd disc = gbd::csqrt_p(half_tr * half_tr - detM);
    const cd sd = gbd::csqrt_p(half_tr + disc) * gbd::csqrt_p(half_tr - disc);
    const cd amp = gbd::cdiv(gbd::mk(weight), sd);

    gbd_beamlet r;
    r.rho[0] = c.x;
    r.rho[1] = c.y;
    r.theta[0] = c.tx;
    r.theta[1] = c.ty;
    r.path = c.path;
    r.amp[0] = amp.re;
    r.amp[1] = amp.im;
    for (int q = 0; q < 4; ++q) {
        r.curv[2 * q] = Pm[q].re;
        r.curv[2 * q + 1] = Pm[q].im;
        r.abcd[q] = A[q];
        r.abcd[4 + q] = B[q];
        r.abcd[8 + q] = C[q];
        r.abcd[12 + q] = Dm[q];
    }
    r.center[0] = cx;
    r.center[1] = cy;
    r.weight = weight;
    r.waist = w0;
    r.edge_distance = 0.0;
    *out = r;
}

// grid: (row j, instance, segment of the row).  Each CTA finds its row's first record
// index by summing the closed-form extents of the rows before it, then its threads take
// the row's inside centres in turn with the row's other segments.
__global__ void __launch_bounds__(128) trace_kernel(gbd_trace_params P,
                                                    const gbd_instance_dev* __restrict__ inst,
                                                    gbd_beamlet* __restrict__ out) {
    int N = P.n_across;
    const gbd_grid* g = &P.grid;
    long long base = 0;
    if (inst != nullptr) {
        const gbd_instance_dev& I = inst[blockIdx.y];
        N = I.n_across;
        g = &I.grid;
        base = I.offset;
    }
    const int j = blockIdx.x;
    if (j >= N) return;
    __shared__ long long warp_sum[4];
    long long acc = 0;
    for (int q = threadIdx.x; q < j; q += blockDim.x) acc += row_extent(q, N) + 1;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    const long long row_off = warp_sum[0] + warp_sum[1] + warp_sum[2] + warp_sum[3];
    const int a = row_extent(j, N);
    if (a < 0) return;
    const int i_lo = ((N - 1) - a) / 2;
    // the row's beamlets are shared by the gridDim.z CTAs of the row (one per thread for
    // rows of up to 128 gridDim.z beamlets), which spreads long rows over more SMs
    for (int t = blockIdx.z * blockDim.x + threadIdx.x; t <= a; t += blockDim.x * gridDim.z)
        trace_one(LensTracer{P}, *g, N, i_lo + t, j, out + base + row_off + t);
}

// Pupil in front of a sequence of conic mirrors, CTAs per grid row as in trace_kernel.
__global__ void __launch_bounds__(128) trace_mirrors_kernel(gbd_mirror_params M,
                                                            gbd_beamlet* __restrict__ out) {
    const int N = M.n_across;
    const int j = blockIdx.x;
    if (j >= N) return;
    __shared__ long long warp_sum[4];
    long long acc = 0;
    for (int q = threadIdx.x; q < j; q += blockDim.x) acc += row_extent(q, N) + 1;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    const long long row_off = warp_sum[0] + warp_sum[1] + warp_sum[2] + warp_sum[3];
    const int a = row_extent(j, N);
    if (a < 0) return;
    const int i_lo = ((N - 1) - a) / 2;
    for (int t = blockIdx.z * blockDim.x + threadIdx.x; t <= a; t += blockDim.x * gridDim.z)
        trace_one(MirrorTracer{M}, M.grid, N, i_lo + t, j, out + row_off + t);
}

// Truncated decomposition (gbd_trace_truncated): the grid extended to every centre within
// R + margin w0, interior beamlets (q < inner) first, then edge beamlets, each in row-major
// grid order; q = a^2 + b^2 in half-pitch units (a = 2i - (N-1), b = 2j - (N-1)), kept when
// q <= outer.  grid: (row of the extended grid, pass 0 interior / 1 edge); 128 threads.
// Each CTA sums the counts of the rows before its own (O(rows^2) per CTA, tiny), then its
// threads rank the row's members by a block-wide ballot scan.
__device__ __forceinline__ int truncated_class(int i, int j, int N, double inner, double outer) {
    const double a = 2.0 * i - (N - 1), b = 2.0 * j - (N - 1);
    const double q = a * a + b * b;  // exact: integers below 2^26
    if (q > outer) return -1;
    return q < inner ? 0 : 1;
}

__global__ void __launch_bounds__(128) trace_truncated_kernel(gbd_trace_params P, int ext,
                                                              double inner, double outer,
                                                              long long n_interior,
                                                              gbd_beamlet* __restrict__ out) {
    const int N = P.n_across, W = N + 2 * ext;
    const int j = (int)blockIdx.x - ext, pass = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ long long warp_sum[4];
    __shared__ int warp_cnt[4];
    long long acc = 0;
    for (long long q = tid; q < (long long)(j + ext) * W; q += blockDim.x)
        acc += truncated_class((int)(q % W) - ext, (int)(q / W) - ext, N, inner, outer) == pass;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) warp_sum[warp] = acc;
    __syncthreads();
    long long base = warp_sum[0] + warp_sum[1] + warp_sum[2] + warp_sum[3] +
                     (pass ? n_interior : 0);
    const double R = 0.5 * P.diameter;
    for (int c0 = 0; c0 < W; c0 += blockDim.x) {
        const int i = c0 + tid - ext;
        const bool mine = c0 + tid < W && truncated_class(i, j, N, inner, outer) == pass;
        const unsigned bal = __ballot_sync(0xffffffffu, mine);
        __syncthreads();  // warp_cnt of the previous chunk has been read
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        int before = __popc(bal & ((1u << lane) - 1u));
        for (int w = 0; w < warp; ++w) before += warp_cnt[w];
        if (mine) {
            gbd_beamlet* o = out + base + before;
            trace_one(LensTracer{P}, P.grid, N, i, j, o);
            if (pass) o->edge_distance = R - sqrt(o->center[0] * o->center[0] +
                                                  o->center[1] * o->center[1]);
        }
        base += warp_cnt[0] + warp_cnt[1] + warp_cnt[2] + warp_cnt[3];
    }
}

// ---------------------------------------------------------------- projection --

struct Quad {
    double a[6];  // log2 amplitude: 0, u, v, uu, uv, vv
    double p[6];  // phase in turns
    double i0, j0;
    bool pad;
};

// Per-beamlet quadratic form of ln E in pixel units around the pixel (i0, j0) nearest
// to where the chief ray meets the detector, with the carrier -ik z(s) common to all
// beamlets left out (it is applied once per pixel after the sum).
__device__ Quad project_one(const gbd_beamlet& b, const gbd_project_params& G) {
    Quad q;
    if (b.amp[0] == 0.0 && b.amp[1] == 0.0) {
        q.pad = true;
        return q;
    }
    q.pad = false;
    const double k = 2.0 * M_PI * G.inv_wavelength;
    const double th0 = b.theta[0], th1 = b.theta[1];
    const double th2 = th0 * th0 + th1 * th1;
    const cd P00{b.curv[0], b.curv[1]}, P01{b.curv[2], b.curv[3]}, P10{b.curv[4], b.curv[5]},
        P11{b.curv[6], b.curv[7]};
    const cd S01 = 0.5 * (P01 + P10);  // symmetric part: w^T P w = w^T Psym w
    const cd trP = P00 + P11;
    // in-plane map from detector coordinates to the beamlet's transverse offset w
    const double g00 = G.M[0] - th0 * G.n[0], g01 = G.M[1] - th0 * G.n[1];
    const double g10 = G.M[2] - th1 * G.n[0], g11 = G.M[3] - th1 * G.n[1];
    const double dg = g00 * g11 - g01 * g10;
    double ic = 0.5 * G.nx, jc = 0.5 * G.ny;
    const int hx = G.nx / 2, hy = G.ny / 2;
    if (fabs(dg) > 1e-12) {
        const double idg = 1.0 / dg;
        const double sx = (g11 * b.rho[0] - g01 * b.rho[1]) * idg;
        const double sy = (-g10 * b.rho[0] + g00 * b.rho[1]) * idg;
        ic = sx * G.inv_px + hx;
        jc = sy * G.inv_py + hy;
    }
    double i0 = rint(ic), j0 = rint(jc);
    if (!(i0 >= 0.0)) i0 = 0.0;
    if (!(j0 >= 0.0)) j0 = 0.0;
    if (i0 > G.nx - 1) i0 = G.nx - 1;
    if (j0 > G.ny - 1) j0 = G.ny - 1;
    q.i0 = i0;
    q.j0 = j0;
    const double s0x = (i0 - hx) * G.px, s0y = (j0 - hy) * G.py;
    const double d0x = G.M[0] * s0x + G.M[1] * s0y - b.rho[0];
    const double d0y = G.M[2] * s0x + G.M[3] * s0y - b.rho[1];
    const double z0 = G.n[0] * s0x + G.n[1] * s0y;
    const double wx = d0x - z0 * th0, wy = d0y - z0 * th1;
    // columns of the maps scaled to one pixel
    const double gu0 = g00 * G.px, gu1 = g10 * G.px, gv0 = g01 * G.py, gv1 = g11 * G.py;
    const double mu0 = G.M[0] * G.px, mu1 = G.M[2] * G.px, mv0 = G.M[1] * G.py, mv1 = G.M[3] * G.py;
    const double nu = G.n[0] * G.px, nv = G.n[1] * G.py;
    // Psym w
    const cd Pw0 = P00 * gbd::mk(wx) + S01 * gbd::mk(wy);
    const cd Pw1 = S01 * gbd::mk(wx) + P11 * gbd::mk(wy);
    const cd wPw = gbd::mk(wx) * Pw0 + gbd::mk(wy) * Pw1;
    // complex "path" parts X (multiplied by -ik) and direct parts Y, per coefficient
    cd X[6], Y[6];
    X[0] = gbd::mk(b.path - 0.5 * z0 * th2 + th0 * d0x + th1 * d0y) + 0.5 * wPw;
    Y[0] = -0.5 * z0 * trP;
    X[1] = gbd::mk(-0.5 * th2 * nu + mu0 * th0 + mu1 * th1) + (gu0 * Pw0 + gu1 * Pw1);
    Y[1] = -0.5 * nu * trP;
    X[2] = gbd::mk(-0.5 * th2 * nv + mv0 * th0 + mv1 * th1) + (gv0 * Pw0 + gv1 * Pw1);
    Y[2] = -0.5 * nv * trP;
    // second order: (1/2) t^T C2 t with C2 = -ik Gp^T Psym Gp
    const cd Gu0 = gu0 * P00 + gu1 * S01, Gu1 = gu0 * S01 + gu1 * P11;  // Psym gu
    const cd Gv0 = gv0 * P00 + gv1 * S01, Gv1 = gv0 * S01 + gv1 * P11;  // Psym gv
    X[3] = 0.5 * (gu0 * Gu0 + gu1 * Gu1);
    X[4] = gv0 * Gu0 + gv1 * Gu1;
    X[5] = 0.5 * (gv0 * Gv0 + gv1 * Gv1);
    Y[3] = Y[4] = Y[5] = gbd::mk(0.0);
    const double log2e = 1.4426950408889634, inv_two_pi = 0.15915494309189533577;
    for (int m = 0; m < 6; ++m) {
        // c = Y - ik X:  Re c = Re Y + k Im X,  Im c = Im Y - k Re X
        q.a[m] = (Y[m].re + k * X[m].im) * log2e;
        q.p[m] = Y[m].im * inv_two_pi - X[m].re * G.inv_wavelength;
    }
    return q;
}

// The beamlet amplitude's log2 modulus and argument (turns) added to the constant term,
// then the constant phase reduced to [-1/2, 1/2) turns.  FP64 for the FP64 records.
__device__ __forceinline__ void add_amplitude_f64(Quad& q, const gbd_beamlet& b) {
    const double am = sqrt(fma(b.amp[0], b.amp[0], b.amp[1] * b.amp[1]));
    q.a[0] += log2(am);
    const double p0 = q.p[0] + atan2(b.amp[1], b.amp[0]) * 0.15915494309189533577;
    q.p[0] = p0 - rint(p0);
}

// The same for the mixed records, whose coefficients are FP32: the amplitude is scaled by
// its binary exponent (exact) and the mantissa's log2 and argument taken in FP32, which
// saves two FP64 library calls per beamlet; the sum and the reduction stay FP64.
__device__ __forceinline__ void add_amplitude_f32(Quad& q, const gbd_beamlet& b) {
    int e;
    frexp(fmax(fabs(b.amp[0]), fabs(b.amp[1])), &e);
    const float re = (float)ldexp(b.amp[0], -e), im = (float)ldexp(b.amp[1], -e);
    q.a[0] += (double)e + 0.5 * (double)log2f(fmaf(re, re, im * im));
    const double p0 = q.p[0] + (double)atan2f(im, re) * 0.15915494309189533577;
    q.p[0] = p0 - rint(p0);
}

// Mixed-precision record of beamlet `t` in the tiled layout (4 float4 fields per beamlet),
// phase coefficients in radians; the last field's spare pair holds T = exp(256 c_uv), the
// factor between the 8-row steps of columns 32 apart (row-pair kernels).  Returns the flag
// bits: kFlagWide if the beamlet's phase can exceed the wide-phase bound anywhere on the
// detector (|tu| <= U, |tv| <= V around its centre), kFlagSteep if its log2 amplitude can
// change by more than 64 over an 8-row step there (with T^3 included), where the row-pair
// recurrence could under- or overflow FP32, and kFlagColSteep if it can change by more
// than 64 along a thread's 8 columns (the amplitude recurrence's limit).
__device__ __forceinline__ unsigned write_mixed(float4* __restrict__ out, long long t, const Quad& q,
                                                const gbd_project_params& G) {
    float4 f0, f1, f2, f3;
    unsigned flags = 0;
    if (q.pad) {
        f0 = make_float4(0.f, 0.f, gbd::kPadLog2Amp, 0.f);
        f1 = f2 = f3 = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        const double tp = 2.0 * M_PI;
        double p[6];
        for (int m = 0; m < 6; ++m) p[m] = q.p[m] * tp;
        const double U = fmax(q.i0, G.nx - 1 - q.i0), V = fmax(q.j0, G.ny - 1 - q.j0);
        const double bound = fabs(p[0]) + fabs(p[1]) * U + fabs(p[2]) * V + fabs(p[3]) * U * U +
                             fabs(p[4]) * U * V + fabs(p[5]) * V * V;
        // the row-pair kernels' 8-row step phase 8 (p_v + p_uv tu + p_vv (2 tv + 8)) is
        // taken unreduced by the narrow instantiations, so it is held to 64 rad as well
        const double rowstep = 8.0 * (fabs(p[2]) + fabs(p[4]) * U + fabs(p[5]) * (2.0 * V + 8.0));
        if (!(bound <= (double)gbd::kWidePhase) || !(rowstep <= 64.0)) flags |= gbd::kFlagWide;
        // log2 amplitude change over 8 rows: 8 (a_v + a_uv tu + a_vv (2 tv + 8))
        const double step = 8.0 * (fabs(q.a[2]) + fabs(q.a[4]) * (U + 96.0) +
                                    fabs(q.a[5]) * (2.0 * V + 8.0)) + 768.0 * fabs(q.a[4]);
        if (!(step <= 64.0)) flags |= gbd::kFlagSteep;
        // the same over 24 rows (row triples and quadruples: the last row is the first
        // times the product of two or three step factors)
        const double step24 = 24.0 * (fabs(q.a[2]) + fabs(q.a[4]) * (U + 96.0) +
                                      fabs(q.a[5]) * (2.0 * V + 24.0)) + 2304.0 * fabs(q.a[4]);
        if (!(step24 <= 64.0)) flags |= gbd::kFlagSteepRows;
        // log2 amplitude change over one 32-column step: the narrow-phase row-pair kernels
        // carry the first row's amplitude along a thread's (up to 8) columns by a
        // recurrence, which needs the whole 224-pixel span within 2^64
        const double colstep = 32.0 * (fabs(q.a[1]) + fabs(q.a[4]) * V +
                                       fabs(q.a[3]) * (2.0 * U + 32.0));
        if (!(8.0 * colstep <= 64.0)) flags |= gbd::kFlagColSteep;
        // T in FP32 (it is stored as FP32), its phase reduced in FP64 first
        const float tm = exp2f((float)(256.0 * q.a[4]));
        const double tt = 256.0 * q.p[4];
        float sn, cs;
        sincospif((float)(2.0 * (tt - rint(tt))), &sn, &cs);
        f0 = make_float4((float)q.i0, (float)(q.j0 - G.row0), (float)q.a[0], (float)p[0]);
        f1 = make_float4((float)q.a[1], (float)p[1], (float)q.a[2], (float)p[2]);
        f2 = make_float4((float)q.a[3], (float)p[3], (float)q.a[4], (float)p[4]);
        f3 = make_float4((float)q.a[5], (float)p[5], tm * cs, tm * sn);
        // without a uv term (both coefficients exactly 0) T is exactly 1 and the 8-row step
        // factor the same on every column: the row-pair kernels skip T's update and the
        // row triples / quadruples form the factors once per warp
        if (!(f2.z == 0.0f && f2.w == 0.0f && f3.z == 1.0f && f3.w == 0.0f))
            flags |= gbd::kFlagCross;
    }
    float4* tile = out + (size_t)(t / gbd::kTile) * gbd::kMixedFields * gbd::kTile;
    const int l = (int)(t % gbd::kTile);
    tile[l] = f0;
    tile[gbd::kTile + l] = f1;
    tile[2 * gbd::kTile + l] = f2;
    tile[3 * gbd::kTile + l] = f3;
    return flags;
}

__global__ void __launch_bounds__(128) project_mixed_kernel(const gbd_beamlet* __restrict__ b, int n,
                                                            int n_pad, gbd_project_params G,
                                                            float4* __restrict__ out,
                                                            unsigned* __restrict__ wide) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_pad) return;
    Quad q;
    q.pad = true;
    if (t < n) {
        q = project_one(b[t], G);
        if (!q.pad) add_amplitude_f32(q, b[t]);
    }
    const unsigned f = write_mixed(out, t, q, G);
    if (f && wide) atomicOr(wide, f);
}

__global__ void __launch_bounds__(128) project_f64_kernel(const gbd_beamlet* __restrict__ b, int n,
                                                          int n_pad, gbd_project_params G,
                                                          double2* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_pad) return;
    double2 f[gbd::kF64Fields];
    Quad q;
    q.pad = true;
    if (t < n) {
        q = project_one(b[t], G);
        if (!q.pad) add_amplitude_f64(q, b[t]);
    }
    if (q.pad) {
        for (int m = 0; m < gbd::kF64Fields; ++m) f[m] = make_double2(0.0, 0.0);
        f[1].x = 2.0 * gbd::kPadLog2Amp;
    } else {
        f[0] = make_double2(q.i0, q.j0 - G.row0);
        for (int m = 0; m < 6; ++m) f[1 + m] = make_double2(q.a[m], q.p[m]);
        // S = E(u+2)E(u)/E(u+1)^2 = exp of twice the uu coefficient, for row recurrences
        const double sa = exp2(2.0 * q.a[3]);
        const double sp = 2.0 * q.p[3];
        double sn, cs;
        sincospi(2.0 * (sp - rint(sp)), &sn, &cs);
        f[7] = make_double2(sa * cs, sa * sn);
    }
    double2* tile = out + (size_t)(t / gbd::kTile) * gbd::kF64Fields * gbd::kTile;
    const int l = t % gbd::kTile;
    for (int m = 0; m < gbd::kF64Fields; ++m) tile[m * gbd::kTile + l] = f[m];
}

// Batched trace + projection for a parameter sweep, one thread per record.  Records of
// instance k start at inst[k].offset (a tile boundary); rows[rbase[k] + j] is the index,
// inside the instance, of the first beamlet of grid row j.  Records between an instance's
// last beamlet and the next tile boundary are written as padding.  MIRRORS: the rays go
// through the mirror sequence M instead of the thin-lens system P (each instance keeps its
// own pupil sampling, I.grid).
template <bool MIRRORS>
__global__ void __launch_bounds__(256)
    trace_project_kernel(gbd_trace_params P, gbd_mirror_params M,
                         const gbd_instance_dev* __restrict__ inst, int n_inst,
                         const int* __restrict__ rbase, const int* __restrict__ rows,
                         long long n_records, gbd_project_params G, float4* __restrict__ out,
                         unsigned* __restrict__ wide) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_records) return;
    int lo = 0, hi = n_inst - 1;  // last instance starting at or before t
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (inst[mid].offset <= t) lo = mid;
        else hi = mid - 1;
    }
    const gbd_instance_dev I = inst[lo];
    const long long u = t - I.offset;
    Quad q;
    q.pad = true;
    if (u < I.reserved) {
        const int N = I.n_across;
        const int* R = rows + rbase[lo];
        int a = 0, b = N - 1;  // last row whose first beamlet is at or before u
        while (a < b) {
            const int m = (a + b + 1) / 2;
            if (R[m] <= u) a = m;
            else b = m - 1;
        }
        const int i = ((N - 1) - row_extent(a, N)) / 2 + (int)(u - R[a]);
        gbd_beamlet bm;
        if (MIRRORS)
            trace_one(MirrorTracer{M}, I.grid, N, i, a, &bm);
        else
            trace_one(LensTracer{P}, I.grid, N, i, a, &bm);
        q = project_one(bm, G);
        if (!q.pad) add_amplitude_f32(q, bm);
    }
    const unsigned f = write_mixed(out, t, q, G);
    if (f && wide) atomicOr(wide, f);
}

// Edge records of a truncated decomposition (FP64, gbd::kEdgeFields double2 per beamlet,
// beamlet after beamlet), for an untilted detector:
//   [0] (i0, j0)  [1..6] the beamlet's Gaussian, (log2 |E|, phase in turns) coefficients of
//   1, tu, tv, tu^2, tu tv, tv^2 (as the FP64 records)  [7..9] zeta = z0 + zu tu + zv tv
//   [10..15] Psi = ln E - zeta^2 + ln(1/2) in the same form.
// The cut beamlet's field is E 1/2 erfc(zeta) = e^Psi w(i zeta) (Re zeta >= 0) or
// E - e^Psi w(-i zeta) (Re zeta < 0), w the Faddeeva function; with n = r_j / |r_j|,
// M = A + B P1, zeta = (n^T M^-1 (rho - rho_c) - d) sqrt(i k / (2 n^T M^-1 B n)) (the
// Collins integral over the half-plane n.(r - r_j) <= d of the input, principal root).
__global__ void __launch_bounds__(128) project_edge_kernel(const gbd_beamlet* __restrict__ b,
                                                           int n, gbd_project_params G,
                                                           double2* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const gbd_beamlet bm = b[t];
    double2* o = out + (size_t)t * gbd::kEdgeFields;
    Quad q = project_one(bm, G);
    if (q.pad) {
        for (int m = 0; m < gbd::kEdgeFields; ++m) o[m] = make_double2(0.0, 0.0);
        o[1].x = o[10].x = 2.0 * gbd::kPadLog2Amp;
        return;
    }
    add_amplitude_f64(q, bm);
    const double k = 2.0 * M_PI * G.inv_wavelength;
    const double w0 = bm.waist, p1 = -G.wavelength / (M_PI * w0 * w0);  // P1 = i p1 I
    // M = A + B P1 and its inverse; sigma = n^T M^-1 B n; u = n^T M^-1
    const double* A = bm.abcd;
    const double* B = bm.abcd + 4;
    const cd M00{A[0], B[0] * p1}, M01{A[1], B[1] * p1}, M10{A[2], B[2] * p1}, M11{A[3], B[3] * p1};
    const cd idet = gbd::cdiv(gbd::mk(1.0), M00 * M11 - M01 * M10);
    const cd Mi00 = M11 * idet, Mi01 = gbd::mk(0.0) - M01 * idet, Mi10 = gbd::mk(0.0) - M10 * idet,
             Mi11 = M00 * idet;
    const double rr = sqrt(bm.center[0] * bm.center[0] + bm.center[1] * bm.center[1]);
    const double nx = rr > 0.0 ? bm.center[0] / rr : 1.0, ny = rr > 0.0 ? bm.center[1] / rr : 0.0;
    const cd u0 = nx * Mi00 + ny * Mi10, u1 = nx * Mi01 + ny * Mi11;  // n^T M^-1
    const double Bn0 = B[0] * nx + B[1] * ny, Bn1 = B[2] * nx + B[3] * ny;
    const cd sigma = Bn0 * u0 + Bn1 * u1;
    const cd root = gbd::csqrt_p(gbd::cdiv(cd{0.0, 0.5 * k}, sigma));
    const int hx = G.nx / 2, hy = G.ny / 2;
    const double d0x = (q.i0 - hx) * G.px - bm.rho[0], d0y = (q.j0 - hy) * G.py - bm.rho[1];
    const cd z0 = (u0 * gbd::mk(d0x) + u1 * gbd::mk(d0y) - gbd::mk(bm.edge_distance)) * root;
    const cd zu = G.px * (u0 * root), zv = G.py * (u1 * root);
    const cd zz[6] = {z0 * z0, 2.0 * (z0 * zu), 2.0 * (z0 * zv), zu * zu, 2.0 * (zu * zv),
                      zv * zv};
    const double log2e = 1.4426950408889634, inv_two_pi = 0.15915494309189533577;
    o[0] = make_double2(q.i0, q.j0);
    for (int m = 0; m < 6; ++m) {
        o[1 + m] = make_double2(q.a[m], q.p[m]);
        double pa = q.a[m] - zz[m].re * log2e, pp = q.p[m] - zz[m].im * inv_two_pi;
        if (m == 0) {
            pa -= 1.0;  // the factor 1/2
            pp -= rint(pp);
        }
        o[10 + m] = make_double2(pa, pp);
    }
    o[7] = make_double2(z0.re, z0.im);
    o[8] = make_double2(zu.re, zu.im);
    o[9] = make_double2(zv.re, zv.im);
}

}  // namespace

cudaError_t gbd_launch_trace_truncated(const gbd_trace_params& p, int ext, double inner,
                                       double outer, long long n_interior, gbd_beamlet* out,
                                       cudaStream_t s) {
    const int W = p.n_across + 2 * ext;
    trace_truncated_kernel<<<dim3(W, 2), 128, 0, s>>>(p, ext, inner, outer, n_interior, out);
    return cudaGetLastError();
}

cudaError_t gbd_launch_project_edge(const gbd_beamlet* b, int n, const gbd_project_params& p,
                                    double2* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    project_edge_kernel<<<(n + 127) / 128, 128, 0, s>>>(b, n, p, out);
    return cudaGetLastError();
}

cudaError_t gbd_launch_trace_project(const gbd_trace_params& p, const gbd_mirror_params* m,
                                     int n_instances, const gbd_instance_dev* d_inst,
                                     const int* d_rbase, const int* d_rows, long long n_records,
                                     const gbd_project_params& g, float4* out, unsigned* wide,
                                     cudaStream_t s) {
    if (n_records <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n_records + 255) / 256);
    if (m)
        trace_project_kernel<true><<<blocks, 256, 0, s>>>(p, *m, d_inst, n_instances, d_rbase, d_rows,
                                                          n_records, g, out, wide);
    else
        trace_project_kernel<false><<<blocks, 256, 0, s>>>(p, gbd_mirror_params{}, d_inst,
                                                           n_instances, d_rbase, d_rows, n_records,
                                                           g, out, wide);
    return cudaGetLastError();
}

cudaError_t gbd_launch_trace(const gbd_trace_params& p, int n_instances, int max_n_across,
                             const gbd_instance_dev* d_inst, gbd_beamlet* out, cudaStream_t s) {
    dim3 grid(max_n_across, n_instances, (max_n_across + 127) / 128);
    trace_kernel<<<grid, 128, 0, s>>>(p, d_inst, out);
    return cudaGetLastError();
}

cudaError_t gbd_launch_trace_mirrors(const gbd_mirror_params& m, gbd_beamlet* out, cudaStream_t s) {
    trace_mirrors_kernel<<<dim3(m.n_across, 1, (m.n_across + 127) / 128), 128, 0, s>>>(m, out);
    return cudaGetLastError();
}

cudaError_t gbd_launch_project(const gbd_beamlet* b, int n, const gbd_project_params& p,
                               int precision, void* coeffs, unsigned* wide, cudaStream_t s) {
    const int n_pad = (n + gbd::kTile - 1) / gbd::kTile * gbd::kTile;
    if (n_pad == 0) return cudaSuccess;
    const int blocks = (n_pad + 127) / 128;
    if (precision == GBD_PREC_MIXED)
        project_mixed_kernel<<<blocks, 128, 0, s>>>(b, n, n_pad, p, static_cast<float4*>(coeffs), wide);
    else
        project_f64_kernel<<<blocks, 128, 0, s>>>(b, n, n_pad, p, static_cast<double2*>(coeffs));
    return cudaGetLastError();
}
