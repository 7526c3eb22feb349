/*
 * FP64 CPU oracle of plane-evaluation Gaussian beamlet decomposition (GBD).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline / reference leg may load or call this code.  It shares
 * no code, header, table or helper with the CUDA library, and the library never
 * calls it.  Plain, slow and direct: every quantity is computed from its definition
 * in the order the method states it, in double precision.
 *
 * Steps (paper sections and equations):
 *   1. Pupil grid and beamlet waist from the overlap factor          Eq. OF (Sec. 6)
 *   2. Input beamlet a_j exp(-|r-r_j|^2/w0^2); complex curvature
 *      P1 = -i lambda/(pi w0^2) I (Eq. complexq, taken with the sign that makes
 *      exp(-ik r^T P r/2) decay; Eq. sum_gaussian)
 *   3. Chief ray + 4 parabasal rays through [OPD plate] -> thin lens -> distance d;
 *      one-sided differences give the 4x4 differential ray-transfer matrix
 *      (Sec. 2.2 steps 1 and 4; Eq. abcd_sys)
 *   4. Gaussian solution of the Collins integral: P2 = (C + D P1)(A + B P1)^-1 and
 *      amplitude a_j / sqrtdet(A + B P1), the square root of the determinant taken as
 *      the product of the principal square roots of the two eigenvalues (the
 *      eigenvalue route the paper uses for the Gouy phase, App. C)   Eq. gauss_prop
 *   5. Field of one beamlet on the common evaluation plane: the aligned solution
 *      centred on the chief ray's landing point rho_c, times the misalignment phase
 *      carried by the chief ray's slope theta and excess path L (Eq. collins_factored
 *      with r2M = A r1M + B th1M, th2M = C r1M + D th1M from Eqs. ab_prop / cd_prop):
 *          E_j(rho) = alpha_j exp(-ik [L + theta.(rho-rho_c) + (rho-rho_c)^T P (rho-rho_c)/2])
 *      For a plane tilted about the reference point, the beamlet propagated by the
 *      axial offset z of each pixel, expanded to second order in the pixel position:
 *          ln E_j = ln alpha_j - z tr(P)/2
 *                   - ik [L + z (1 - |theta|^2/2) + theta.delta + w^T P w / 2],
 *          delta = X_xy - rho_c,  w = delta - z theta
 *   6. Coherent sum over beamlets                                    Eq. sum_gaussian
 *   7. Airy score (RMS of |E|/|E(0)| - |2 J1(x)/x| inside the third dark ring) and the
 *      annular-zone scores                                                        Sec. 6
 *   8. Real rays through reflective conics (the Ritchey-Chretien telescope), the same
 *      steps 3-4 on their differences                                             App. B
 *
 * The global axial phase exp(-ik d) is dropped: phases are relative to the axial path.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Beamlet record, 40 doubles. */
enum {
    REC_RJ = 0,      /* r_j (x, y): beamlet centre in the pupil, m              */
    REC_A = 2,       /* a_j: decomposition weight                               */
    REC_W0 = 3,      /* w0: input waist, m                                      */
    REC_ABCD = 4,    /* A, B, C, D: 4 row-major 2x2 blocks (16 doubles)         */
    REC_P = 20,      /* P2: 2x2 complex, row-major (re, im) pairs (8 doubles)   */
    REC_ALPHA = 28,  /* alpha_j = a_j / sqrtdet(A + B P1)  (re, im)             */
    REC_L = 30,      /* chief-ray excess optical path over the axial path, m    */
    REC_RHO = 31,    /* rho_c: chief-ray landing point on the reference plane  */
    REC_THETA = 33,  /* theta: chief-ray slope                                  */
    REC_SIZE = 40
};

int orc_record_size(void) { return REC_SIZE; }

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- pupil grid -- */

/* Cell-centred grid, x_i = (i - (N-1)/2) s with s = D/N; a centre is inside when
 * |r| <= D/2.  In units of s/2 the test is (2i-(N-1))^2 + (2j-(N-1))^2 <= N^2,
 * which is exact in integers. */
static int inside(int i, int j, int n) {
    long a = 2L * i - (n - 1), b = 2L * j - (n - 1);
    return a * a + b * b <= (long)n * n;
}

int orc_count(int n_across) {
    int c = 0;
    for (int j = 0; j < n_across; ++j)
        for (int i = 0; i < n_across; ++i) c += inside(i, j, n_across);
    return c;
}

/* ------------------------------------------------------------- Zernike plate -- */

static double factorial(int n) {
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

/* Noll's ordering: radial order n, azimuthal order m, and whether the mode is a
 * sine (odd j) or cosine (even j) term. */
void orc_noll(int j, int* n_out, int* m_out, int* is_sin) {
    int n = 0;
    while ((n + 1) * (n + 2) / 2 < j) ++n;
    int k = j - n * (n + 1) / 2 - 1; /* position inside the row, 0-based */
    int m = (n % 2 == 0) ? 2 * ((k + 1) / 2) : 2 * (k / 2) + 1;
    *n_out = n;
    *m_out = m;
    *is_sin = (m != 0) && (j % 2 == 1);
}

/* One RMS-normalised Noll Zernike mode on the disk of radius R, with its gradient.
 * Z = N_nm R_n^m(rho) {cos|sin}(m phi) written in Cartesian form:
 *   rho^(n-2s) cos(m phi) = u^((n-m)/2 - s) Re(w^m),  u = (x^2+y^2)/R^2,  w = (x+iy)/R
 * which is a polynomial in x and y, so the gradient has no singularity at r = 0. */
void orc_zernike(int j, double R, double x, double y, double* Z, double* dZdx, double* dZdy) {
    int n, m, is_sin;
    orc_noll(j, &n, &m, &is_sin);
    double norm = (m == 0) ? sqrt(n + 1.0) : sqrt(2.0 * (n + 1.0));
    double u = (x * x + y * y) / (R * R);
    double complex w = (x + I * y) / R;
    /* w^m and its derivative factor m w^(m-1) */
    double complex wm = 1.0, wm1 = 0.0;
    for (int k = 0; k < m; ++k) {
        wm1 = wm;
        wm *= w;
    }
    double complex dwm = (m > 0) ? m * wm1 : 0.0; /* d(w^m)/dw */
    double ang = is_sin ? cimag(wm) : creal(wm);
    /* d(w^m)/dx = dwm / R, d(w^m)/dy = i dwm / R */
    double dang_dx = is_sin ? cimag(dwm / R) : creal(dwm / R);
    double dang_dy = is_sin ? cimag(I * dwm / R) : creal(I * dwm / R);
    double rad = 0.0, drad_du = 0.0;
    for (int s = 0; s <= (n - m) / 2; ++s) {
        double c = ((s % 2) ? -1.0 : 1.0) * factorial(n - s) /
                   (factorial(s) * factorial((n + m) / 2 - s) * factorial((n - m) / 2 - s));
        int p = (n - m) / 2 - s; /* power of u */
        rad += c * pow(u, p);
        if (p > 0) drad_du += c * p * pow(u, p - 1);
    }
    double du_dx = 2.0 * x / (R * R), du_dy = 2.0 * y / (R * R);
    *Z = norm * rad * ang;
    *dZdx = norm * (drad_du * du_dx * ang + rad * dang_dx);
    *dZdy = norm * (drad_du * du_dy * ang + rad * dang_dy);
}

typedef struct {
    double wavelength, f, d;
    int n_zern;
    const int* noll;
    const double* zc;
    double zrad;
} orc_system;

/* OPD of the plate and its gradient at (x, y). */
static void plate(const orc_system* S, double x, double y, double* W, double* gx, double* gy) {
    *W = *gx = *gy = 0.0;
    for (int t = 0; t < S->n_zern; ++t) {
        double z, zx, zy;
        orc_zernike(S->noll[t], S->zrad, x, y, &z, &zx, &zy);
        *W += S->zc[t] * z;
        *gx += S->zc[t] * zx;
        *gy += S->zc[t] * zy;
    }
}

/* Trace one paraxial ray (position r, slope th) through plate -> lens -> distance.
 * opl accumulates the excess optical path over the axial path. */
static void trace_ray(const orc_system* S, double r[2], double th[2], double* opl) {
    if (S->n_zern > 0) {
        double W, gx, gy;
        plate(S, r[0], r[1], &W, &gx, &gy);
        *opl += W;
        th[0] += gx;
        th[1] += gy;
    }
    /* thin lens: transmits exp(+ik r^2/2f), i.e. path -r^2/2f; slope kicked by -r/f */
    *opl -= (r[0] * r[0] + r[1] * r[1]) / (2.0 * S->f);
    th[0] -= r[0] / S->f;
    th[1] -= r[1] / S->f;
    /* free space over axial distance d: path d sqrt(1+|th|^2) ~ d + d |th|^2 / 2 */
    r[0] += S->d * th[0];
    r[1] += S->d * th[1];
    *opl += S->d * (th[0] * th[0] + th[1] * th[1]) / 2.0;
}

/* ------------------------------------------------------------- 2x2 algebra -- */

typedef struct { double complex m[2][2]; } cmat2;

static cmat2 cmul(cmat2 a, cmat2 b) {
    cmat2 c;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) c.m[i][j] = a.m[i][0] * b.m[0][j] + a.m[i][1] * b.m[1][j];
    return c;
}

static double complex cdet(cmat2 a) { return a.m[0][0] * a.m[1][1] - a.m[0][1] * a.m[1][0]; }

static cmat2 cinv(cmat2 a) {
    double complex dt = cdet(a);
    cmat2 r;
    r.m[0][0] = a.m[1][1] / dt;
    r.m[0][1] = -a.m[0][1] / dt;
    r.m[1][0] = -a.m[1][0] / dt;
    r.m[1][1] = a.m[0][0] / dt;
    return r;
}

/* sqrt(det M) on the branch continuous from M = I: product of the principal square
 * roots of the eigenvalues tr/2 +- sqrt(tr^2/4 - det). */
double complex orc_sqrtdet(double complex m00, double complex m01, double complex m10,
                           double complex m11) {
    double complex tr = m00 + m11, dt = m00 * m11 - m01 * m10;
    double complex disc = csqrt(tr * tr / 4.0 - dt);
    double complex l1 = tr / 2.0 + disc, l2 = tr / 2.0 - disc;
    return csqrt(l1) * csqrt(l2);
}

/* exported for tests: writes (re, im) of sqrtdet of the 2x2 complex matrix m (row-major
 * re/im pairs) */
void orc_sqrtdet_v(const double* m, double* out) {
    double complex r = orc_sqrtdet(m[0] + I * m[1], m[2] + I * m[3], m[4] + I * m[5],
                                   m[6] + I * m[7]);
    out[0] = creal(r);
    out[1] = cimag(r);
}

/* ------------------------------------------------------------------- trace -- */

/* One beamlet centred at (rx, ry) in the pupil: chief ray, 4 parabasal rays, one-sided
 * differences for ABCD (Sec. 2.2), Eq. gauss_prop with the eigenvalue sqrtdet; fills one
 * record (zeroed first). */
static void trace_beamlet(const orc_system* S, double rx, double ry, double a, double w0,
                          double h, double dth, double complex p1, double* rec) {
    memset(rec, 0, sizeof(double) * REC_SIZE);
    /* chief ray */
    double rc[2] = {rx, ry}, tc[2] = {0.0, 0.0}, L = 0.0;
    trace_ray(S, rc, tc, &L);
    /* waist rays (position offsets) -> columns of A and C */
    double A[2][2], B[2][2], C[2][2], D[2][2];
    for (int k = 0; k < 2; ++k) {
        double r[2] = {rx + (k == 0 ? h : 0.0), ry + (k == 1 ? h : 0.0)};
        double t[2] = {0.0, 0.0}, o = 0.0;
        trace_ray(S, r, t, &o);
        for (int q = 0; q < 2; ++q) {
            A[q][k] = (r[q] - rc[q]) / h;
            C[q][k] = (t[q] - tc[q]) / h;
        }
    }
    /* divergence rays (slope offsets) -> columns of B and D */
    for (int k = 0; k < 2; ++k) {
        double r[2] = {rx, ry};
        double t[2] = {k == 0 ? dth : 0.0, k == 1 ? dth : 0.0}, o = 0.0;
        trace_ray(S, r, t, &o);
        for (int q = 0; q < 2; ++q) {
            B[q][k] = (r[q] - rc[q]) / dth;
            D[q][k] = (t[q] - tc[q]) / dth;
        }
    }
    /* Eq. gauss_prop: M = A + B P1, P2 = (C + D P1) M^-1, amplitude 1/sqrtdet(M) */
    cmat2 M, Nn;
    for (int q = 0; q < 2; ++q)
        for (int k = 0; k < 2; ++k) {
            M.m[q][k] = A[q][k] + B[q][k] * p1;
            Nn.m[q][k] = C[q][k] + D[q][k] * p1;
        }
    cmat2 P = cmul(Nn, cinv(M));
    double complex alpha = a / orc_sqrtdet(M.m[0][0], M.m[0][1], M.m[1][0], M.m[1][1]);

    rec[REC_RJ] = rx;
    rec[REC_RJ + 1] = ry;
    rec[REC_A] = a;
    rec[REC_W0] = w0;
    for (int q = 0; q < 2; ++q)
        for (int k = 0; k < 2; ++k) {
            rec[REC_ABCD + 0 + 2 * q + k] = A[q][k];
            rec[REC_ABCD + 4 + 2 * q + k] = B[q][k];
            rec[REC_ABCD + 8 + 2 * q + k] = C[q][k];
            rec[REC_ABCD + 12 + 2 * q + k] = D[q][k];
            rec[REC_P + 2 * (2 * q + k)] = creal(P.m[q][k]);
            rec[REC_P + 2 * (2 * q + k) + 1] = cimag(P.m[q][k]);
        }
    rec[REC_ALPHA] = creal(alpha);
    rec[REC_ALPHA + 1] = cimag(alpha);
    rec[REC_L] = L;
    rec[REC_RHO] = rc[0];
    rec[REC_RHO + 1] = rc[1];
    rec[REC_THETA] = tc[0];
    rec[REC_THETA + 1] = tc[1];
}

/* Builds the beamlet table.  Returns the number of beamlets, or -1 when capacity is
 * too small.  out: capacity x REC_SIZE doubles; beamlets in row-major grid order
 * (row j along y outer, column i along x inner). */
int orc_trace(double wavelength, double f, double d, int n_zern, const int* noll,
              const double* zc, double zrad, double diameter, int n_across,
              double overlap_factor, double waist_ratio, double* out, int capacity) {
    orc_system S = {wavelength, f, d, n_zern, noll, zc, zrad};
    const int N = n_across;
    const double s = diameter / N;
    /* Eq. OF: OF = N 2 w0 / W  ->  w0 = OF W / (2N) */
    const double w0 = overlap_factor * diameter / (2.0 * N);
    /* weight so that sum_j a_j exp(-|r-r_j|^2/w0^2) ~ 1 inside the aperture */
    const double a = s * s / (M_PI * w0 * w0);
    /* parabasal steps: waist rays offset by h, divergence rays tilted by alpha */
    const double h = waist_ratio * w0;
    const double dth = waist_ratio * wavelength / (M_PI * w0);
    /* input complex curvature P1 = -i lambda / (pi w0^2) I */
    const double complex p1 = -I * wavelength / (M_PI * w0 * w0);
    int nb = 0;
    for (int j = 0; j < N; ++j) {
        for (int i = 0; i < N; ++i) {
            if (!inside(i, j, N)) continue;
            if (nb >= capacity) return -1;
            double rx = (i - (N - 1) / 2.0) * s, ry = (j - (N - 1) / 2.0) * s;
            trace_beamlet(&S, rx, ry, a, w0, h, dth, p1, out + (size_t)nb * REC_SIZE);
            ++nb;
        }
    }
    return nb;
}

/* Truncated decomposition (Sec. 1 and the Conclusion: beamlets truncated at the aperture
 * edge, Worku & Gross).  The same grid and weights as orc_trace, extended to every centre
 * with |r_j| <= R + margin w0 (R = D/2).  A beamlet whose centre lies within margin w0 of the
 * edge (| R - |r_j| | <= margin w0) is an edge beamlet: its input Gaussian is cut by the
 * half-plane n.r <= R tangent to the aperture at the point nearest to it, n = r_j/|r_j|,
 * i.e. by n.(r - r_j) <= d_j with d_j = R - |r_j| (negative for centres outside).  The
 * others are interior beamlets, used untruncated.  In half-pitch units (a = 2i - (N-1),
 * b = 2j - (N-1)) R = N and w0 = OF: interior a^2 + b^2 < (N - margin OF)^2, kept
 * a^2 + b^2 <= (N + margin OF)^2.  out: interior beamlets first, then edge beamlets, each in
 * row-major grid order; dist[k] = d_k (edge) or +inf (interior); *n_edge = edge count.
 * Returns the number of beamlets, or -1 when capacity is too small. */
int orc_trace_truncated(double wavelength, double f, double d, int n_zern, const int* noll,
                        const double* zc, double zrad, double diameter, int n_across,
                        double overlap_factor, double waist_ratio, double margin, double* out,
                        double* dist, int capacity, int* n_edge) {
    orc_system S = {wavelength, f, d, n_zern, noll, zc, zrad};
    const int N = n_across;
    const double s = diameter / N, R = 0.5 * diameter;
    const double w0 = overlap_factor * diameter / (2.0 * N);
    const double a = s * s / (M_PI * w0 * w0);
    const double h = waist_ratio * w0;
    const double dth = waist_ratio * wavelength / (M_PI * w0);
    const double complex p1 = -I * wavelength / (M_PI * w0 * w0);
    const double outer = (N + margin * overlap_factor) * (N + margin * overlap_factor);
    const double inner_r = N - margin * overlap_factor;
    const double inner = inner_r > 0.0 ? inner_r * inner_r : -1.0;
    /* grid indices whose centre can lie within R + margin w0 */
    const int ext = (int)ceil(0.5 * margin * overlap_factor) + 1;
    int nb = 0, ne = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int j = -ext; j < N + ext; ++j) {
            for (int i = -ext; i < N + ext; ++i) {
                const double aa = 2.0 * i - (N - 1), bb = 2.0 * j - (N - 1);
                const double q = aa * aa + bb * bb;
                if (q > outer) continue;
                const int edge = !(q < inner);
                if (edge != pass) continue;
                if (nb >= capacity) return -1;
                double rx = (i - (N - 1) / 2.0) * s, ry = (j - (N - 1) / 2.0) * s;
                trace_beamlet(&S, rx, ry, a, w0, h, dth, p1, out + (size_t)nb * REC_SIZE);
                dist[nb] = edge ? R - sqrt(rx * rx + ry * ry) : INFINITY;
                ne += edge;
                ++nb;
            }
        }
    }
    *n_edge = ne;
    return nb;
}

/* ------------------------------------------------------------------- field -- */

/* Offset of detector point s from the reference point (0, 0, d) in the lab frame:
 * X - (0, 0, d) = Ry(rot_y) Rx(rot_x) (sx, sy, 0).  Kept relative to the reference point
 * so that the axial offset z = X_z - d carries no rounding from d itself. */
static void detector_offset(double rot_x, double rot_y, double sx, double sy, double V[3]) {
    double ca = cos(rot_x), sa = sin(rot_x), cb = cos(rot_y), sb = sin(rot_y);
    double Rx[3][3] = {{1, 0, 0}, {0, ca, -sa}, {0, sa, ca}};
    double Ry[3][3] = {{cb, 0, sb}, {0, 1, 0}, {-sb, 0, cb}};
    double R[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            R[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) R[i][j] += Ry[i][k] * Rx[k][j];
        }
    double v[3] = {sx, sy, 0.0};
    for (int i = 0; i < 3; ++i) V[i] = R[i][0] * v[0] + R[i][1] * v[1] + R[i][2] * v[2];
}

/* Field of one beamlet at the point V (offset from the reference point) (step 5). */
static double complex beamlet_at(const double* rec, double k, const double V[3]) {
    double complex P[2][2];
    for (int q = 0; q < 2; ++q)
        for (int c = 0; c < 2; ++c)
            P[q][c] = rec[REC_P + 2 * (2 * q + c)] + I * rec[REC_P + 2 * (2 * q + c) + 1];
    double complex alpha = rec[REC_ALPHA] + I * rec[REC_ALPHA + 1];
    const double* rho = rec + REC_RHO;
    const double* th = rec + REC_THETA;
    double L = rec[REC_L];
    double z = V[2];
    double delta[2] = {V[0] - rho[0], V[1] - rho[1]};
    double w[2] = {delta[0] - z * th[0], delta[1] - z * th[1]};
    double th2 = th[0] * th[0] + th[1] * th[1];
    double complex quad = 0.0;
    for (int q = 0; q < 2; ++q)
        for (int c = 0; c < 2; ++c) quad += w[q] * P[q][c] * w[c];
    double complex trP = P[0][0] + P[1][1];
    double path = L + z * (1.0 - th2 / 2.0) + th[0] * delta[0] + th[1] * delta[1];
    double complex lnE = -0.5 * z * trP - I * k * (path + 0.5 * quad);
    return alpha * cexp(lnE);
}

/* Coherent sum of n_b beamlets at the pixels (cols[a], rows[b]) of a detector with
 * nx x ny pixels of pitch (px, py); pixel (i, j) sits at s = ((i - nx/2) px, (j - ny/2) py)
 * with integer division.  out: n_rows x n_cols complex values, (re, im) interleaved,
 * row-major.  Neumaier-compensated sum in beamlet order. */
void orc_field(const double* beamlets, int n_b, double wavelength, double d, double rot_x,
               double rot_y, int nx, int ny, double px, double py, const int* cols, int n_cols,
               const int* rows, int n_rows, double* out) {
    const double k = 2.0 * M_PI / wavelength;
    const long total = (long)n_cols * n_rows;
#pragma omp parallel for schedule(dynamic, 16)
    for (long p = 0; p < total; ++p) {
        int b = (int)(p / n_cols), a = (int)(p % n_cols);
        double sx = (cols[a] - nx / 2) * px, sy = (rows[b] - ny / 2) * py;
        double V[3];
        detector_offset(rot_x, rot_y, sx, sy, V);
        double sr = 0.0, si = 0.0, cr = 0.0, ci = 0.0;
        for (int j = 0; j < n_b; ++j) {
            double complex e = beamlet_at(beamlets + (size_t)j * REC_SIZE, k, V);
            double er = creal(e), ei = cimag(e);
            double t = sr + er;
            cr += (fabs(sr) >= fabs(er)) ? (sr - t) + er : (er - t) + sr;
            sr = t;
            t = si + ei;
            ci += (fabs(si) >= fabs(ei)) ? (si - t) + ei : (ei - t) + si;
            si = t;
        }
        out[2 * p] = sr + cr;
        out[2 * p + 1] = si + ci;
    }
}

/* Exact paraxial propagation of each beamlet to the axial offset z of every pixel:
 * centroid rho_c + z theta, P(z) = P (I + z P)^-1, amplitude det(I + z P)^(-1/2)
 * (branch from the eigenvalues), phase L + z (1 + |theta|^2/2) + theta.(rho - rho_c(z)).
 * Used to measure the second-order tilted-plane rule's method error. */
void orc_field_exact(const double* beamlets, int n_b, double wavelength, double d, double rot_x,
                     double rot_y, int nx, int ny, double px, double py, const int* cols,
                     int n_cols, const int* rows, int n_rows, double* out) {
    const double k = 2.0 * M_PI / wavelength;
    const long total = (long)n_cols * n_rows;
#pragma omp parallel for schedule(dynamic, 16)
    for (long p = 0; p < total; ++p) {
        int b = (int)(p / n_cols), a = (int)(p % n_cols);
        double sx = (cols[a] - nx / 2) * px, sy = (rows[b] - ny / 2) * py;
        double X[3];
        detector_offset(rot_x, rot_y, sx, sy, X);
        double complex acc = 0.0;
        for (int j = 0; j < n_b; ++j) {
            const double* rec = beamlets + (size_t)j * REC_SIZE;
            cmat2 P;
            for (int q = 0; q < 2; ++q)
                for (int c = 0; c < 2; ++c)
                    P.m[q][c] = rec[REC_P + 2 * (2 * q + c)] + I * rec[REC_P + 2 * (2 * q + c) + 1];
            double complex alpha = rec[REC_ALPHA] + I * rec[REC_ALPHA + 1];
            const double* rho = rec + REC_RHO;
            const double* th = rec + REC_THETA;
            double z = X[2];
            cmat2 Mz;
            Mz.m[0][0] = 1.0 + z * P.m[0][0];
            Mz.m[0][1] = z * P.m[0][1];
            Mz.m[1][0] = z * P.m[1][0];
            Mz.m[1][1] = 1.0 + z * P.m[1][1];
            cmat2 Pz = cmul(P, cinv(Mz));
            double complex amp = alpha / orc_sqrtdet(Mz.m[0][0], Mz.m[0][1], Mz.m[1][0], Mz.m[1][1]);
            double th2 = th[0] * th[0] + th[1] * th[1];
            double w[2] = {X[0] - rho[0] - z * th[0], X[1] - rho[1] - z * th[1]};
            double complex quad = 0.0;
            for (int q = 0; q < 2; ++q)
                for (int c = 0; c < 2; ++c) quad += w[q] * Pz.m[q][c] * w[c];
            double path = rec[REC_L] + z * (1.0 + th2 / 2.0) + th[0] * w[0] + th[1] * w[1];
            acc += amp * cexp(-I * k * (path + 0.5 * quad));
        }
        out[2 * p] = creal(acc);
        out[2 * p + 1] = cimag(acc);
    }
}

/* ------------------------------------------------------------ Airy scoring -- */

/* Normalised Airy amplitude |2 J1(x)/x|, x = pi r / (lambda F#); 1 at r = 0. */
double orc_airy_amp(double r, double wavelength, double fnum) {
    double x = M_PI * r / (wavelength * fnum);
    if (x == 0.0) return 1.0;
    return fabs(2.0 * j1(x) / x);
}

/* RMS of |E|/|E(centre)| - A over the pixels with lo <= r / (lambda F#) < hi (an annular
 * zone, Sec. 6).  Same layout and normalisation as orc_airy_score. */
double orc_zone_score(const double* field, int nx, int ny, double px, double py,
                      double wavelength, double fnum, double lo, double hi) {
    const double* ec = field + 2 * ((size_t)(ny / 2) * nx + nx / 2);
    double e0 = hypot(ec[0], ec[1]);
    double acc = 0.0;
    long n = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double sx = (i - nx / 2) * px, sy = (j - ny / 2) * py;
            double r = hypot(sx, sy), u = r / (wavelength * fnum);
            if (u < lo || u >= hi) continue;
            const double* e = field + 2 * ((size_t)j * nx + i);
            double diff = hypot(e[0], e[1]) / e0 - orc_airy_amp(r, wavelength, fnum);
            acc += diff * diff;
            ++n;
        }
    return sqrt(acc / (double)n);
}

/* RMS of |E|/|E(centre)| - A over the pixels with r <= r3, r3 = j_{1,3} lambda F# / pi
 * (inside the third dark ring).  field: ny x nx complex (re, im interleaved); the
 * centre pixel is (nx/2, ny/2).  Untilted detector. */
double orc_airy_score(const double* field, int nx, int ny, double px, double py,
                      double wavelength, double fnum) {
    const double j13 = 10.173468135062722; /* third zero of J1 */
    const double r3 = j13 * wavelength * fnum / M_PI;
    const double* ec = field + 2 * ((size_t)(ny / 2) * nx + nx / 2);
    double e0 = hypot(ec[0], ec[1]);
    double acc = 0.0;
    long n = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double sx = (i - nx / 2) * px, sy = (j - ny / 2) * py;
            double r = hypot(sx, sy);
            if (r > r3) continue;
            const double* e = field + 2 * ((size_t)j * nx + i);
            double diff = hypot(e[0], e[1]) / e0 - orc_airy_amp(r, wavelength, fnum);
            acc += diff * diff;
            ++n;
        }
    return sqrt(acc / (double)n);
}

/* ----------------------------------------------------- two-mirror telescope -- */
/* Real-ray trace through reflective conic surfaces (the Ritchey-Chretien prescription of
 * App. B), for beamlets decomposed on an entrance-pupil plane in front of the first
 * mirror.  Light enters travelling +z.  Mirror k: vertex z_k (z_1 = 0, z_{k+1} = z_k + t_k
 * with t_k the signed distance listed after surface k), radius R_k with App. B's sign
 * (negative = concave, positive = convex towards the arriving light), conic K_k.  With
 * s_k = +-1 the direction of travel before mirror k, the lab-frame curvature is
 * c_k = s_k / R_k and the surface is the conic
 *     z - z_k = c r^2 / (1 + sqrt(1 - (1 + K) c^2 r^2)),   r^2 = x^2 + y^2.
 * Intersections: Newton's method on the sag (starting from the vertex plane).  Normals
 * from the sag's gradient.  Reflection u' = u - 2 (u.n) n.  Optical path = geometric
 * length (air).  The image plane is t_last after the last vertex. */

typedef struct {
    int n;
    double z[8], c[8], K[8];
    double z_ep, z_img;
} orc_mirrors;

static void mirrors_setup(int n, const double* radius, const double* conic, const double* dist,
                          double pupil_offset, orc_mirrors* M) {
    M->n = n;
    double z = 0.0, s = 1.0;
    for (int k = 0; k < n; ++k) {
        M->z[k] = z;
        M->c[k] = s / radius[k];
        M->K[k] = conic[k];
        z += dist[k];
        s = -s;
    }
    M->z_img = z;
    M->z_ep = -pupil_offset;
}

static double sag(double c, double K, double r2) {
    return c * r2 / (1.0 + sqrt(1.0 - (1.0 + K) * c * c * r2));
}

/* d(sag)/d(r2) */
static double dsag_dr2(double c, double K, double r2) {
    double q = sqrt(1.0 - (1.0 + K) * c * c * r2);
    double den = 1.0 + q;
    /* sag = c r2 / den;  dq/dr2 = -(1+K) c^2 / (2 q) */
    double dq = -(1.0 + K) * c * c / (2.0 * q);
    return c / den - c * r2 * dq / (den * den);
}

/* Traces one ray from (x0, y0, z_ep) with direction slopes (ax, ay) to the image plane:
 * position, slopes and geometric path length. */
static void mirror_ray(const orc_mirrors* M, double x0, double y0, double ax, double ay,
                       double out_xy[2], double out_th[2], double* path) {
    double p[3] = {x0, y0, M->z_ep};
    double nu = sqrt(1.0 + ax * ax + ay * ay);
    double u[3] = {ax / nu, ay / nu, 1.0 / nu};
    double L = 0.0;
    for (int k = 0; k < M->n; ++k) {
        /* Newton on g(t) = z(t) - z_k - sag(r2(t)), starting at the vertex plane */
        double t = (M->z[k] - p[2]) / u[2];
        for (int it = 0; it < 60; ++it) {
            double x = p[0] + t * u[0], y = p[1] + t * u[1], zz = p[2] + t * u[2];
            double r2 = x * x + y * y;
            double g = zz - M->z[k] - sag(M->c[k], M->K[k], r2);
            double dg = u[2] - dsag_dr2(M->c[k], M->K[k], r2) * 2.0 * (x * u[0] + y * u[1]);
            double step = g / dg;
            t -= step;
            if (fabs(step) < 1e-16 * (1.0 + fabs(t))) break;
        }
        for (int q = 0; q < 3; ++q) p[q] += t * u[q];
        L += t;
        /* surface normal from the gradient of z - sag(r2) */
        double r2 = p[0] * p[0] + p[1] * p[1];
        double ds = dsag_dr2(M->c[k], M->K[k], r2);
        double n[3] = {-2.0 * ds * p[0], -2.0 * ds * p[1], 1.0};
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int q = 0; q < 3; ++q) n[q] /= nn;
        double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
        for (int q = 0; q < 3; ++q) u[q] -= 2.0 * un * n[q];
    }
    double t = (M->z_img - p[2]) / u[2];
    for (int q = 0; q < 3; ++q) p[q] += t * u[q];
    L += t;
    out_xy[0] = p[0];
    out_xy[1] = p[1];
    out_th[0] = u[0] / u[2];
    out_th[1] = u[1] / u[2];
    *path = L;
}

/* exported for tests: one ray (x0, y0, slopes ax, ay) -> (x, y, theta_x, theta_y, path) */
void orc_mirror_ray(int n, const double* radius, const double* conic, const double* dist,
                    double pupil_offset, double x0, double y0, double ax, double ay, double* out) {
    orc_mirrors M;
    mirrors_setup(n, radius, conic, dist, pupil_offset, &M);
    mirror_ray(&M, x0, y0, ax, ay, out, out + 2, out + 4);
}

/* Beamlet table for a pupil of `diameter` in front of the mirrors (same record layout and
 * steps as orc_trace; the path is relative to the axial ray). */
int orc_trace_mirrors(double wavelength, int n, const double* radius, const double* conic,
                      const double* dist, double pupil_offset, double diameter, int n_across,
                      double overlap_factor, double waist_ratio, double* out, int capacity) {
    orc_mirrors Msys;
    mirrors_setup(n, radius, conic, dist, pupil_offset, &Msys);
    const int N = n_across;
    const double s = diameter / N;
    const double w0 = overlap_factor * diameter / (2.0 * N);
    const double a = s * s / (M_PI * w0 * w0);
    const double h = waist_ratio * w0;
    const double dth = waist_ratio * wavelength / (M_PI * w0);
    const double complex p1 = -I * wavelength / (M_PI * w0 * w0);
    double axy[2], ath[2], apath;
    mirror_ray(&Msys, 0.0, 0.0, 0.0, 0.0, axy, ath, &apath);
    int nb = 0;
    for (int j = 0; j < N; ++j) {
        for (int i = 0; i < N; ++i) {
            if (!inside(i, j, N)) continue;
            if (nb >= capacity) return -1;
            double* rec = out + (size_t)nb * REC_SIZE;
            memset(rec, 0, sizeof(double) * REC_SIZE);
            double rx = (i - (N - 1) / 2.0) * s, ry = (j - (N - 1) / 2.0) * s;
            double rc[2], tc[2], Lc;
            mirror_ray(&Msys, rx, ry, 0.0, 0.0, rc, tc, &Lc);
            double A[2][2], B[2][2], C[2][2], D[2][2];
            for (int k = 0; k < 2; ++k) {
                double r[2], t[2], o;
                mirror_ray(&Msys, rx + (k == 0 ? h : 0.0), ry + (k == 1 ? h : 0.0), 0.0, 0.0, r, t, &o);
                for (int q = 0; q < 2; ++q) {
                    A[q][k] = (r[q] - rc[q]) / h;
                    C[q][k] = (t[q] - tc[q]) / h;
                }
                mirror_ray(&Msys, rx, ry, k == 0 ? dth : 0.0, k == 1 ? dth : 0.0, r, t, &o);
                for (int q = 0; q < 2; ++q) {
                    B[q][k] = (r[q] - rc[q]) / dth;
                    D[q][k] = (t[q] - tc[q]) / dth;
                }
            }
            cmat2 Mm, Nn;
            for (int q = 0; q < 2; ++q)
                for (int k = 0; k < 2; ++k) {
                    Mm.m[q][k] = A[q][k] + B[q][k] * p1;
                    Nn.m[q][k] = C[q][k] + D[q][k] * p1;
                }
            cmat2 P = cmul(Nn, cinv(Mm));
            double complex alpha = a / orc_sqrtdet(Mm.m[0][0], Mm.m[0][1], Mm.m[1][0], Mm.m[1][1]);
            rec[REC_RJ] = rx;
            rec[REC_RJ + 1] = ry;
            rec[REC_A] = a;
            rec[REC_W0] = w0;
            for (int q = 0; q < 2; ++q)
                for (int k = 0; k < 2; ++k) {
                    rec[REC_ABCD + 0 + 2 * q + k] = A[q][k];
                    rec[REC_ABCD + 4 + 2 * q + k] = B[q][k];
                    rec[REC_ABCD + 8 + 2 * q + k] = C[q][k];
                    rec[REC_ABCD + 12 + 2 * q + k] = D[q][k];
                    rec[REC_P + 2 * (2 * q + k)] = creal(P.m[q][k]);
                    rec[REC_P + 2 * (2 * q + k) + 1] = cimag(P.m[q][k]);
                }
            rec[REC_ALPHA] = creal(alpha);
            rec[REC_ALPHA + 1] = cimag(alpha);
            rec[REC_L] = Lc - apath;
            rec[REC_RHO] = rc[0];
            rec[REC_RHO + 1] = rc[1];
            rec[REC_THETA] = tc[0];
            rec[REC_THETA + 1] = tc[1];
            ++nb;
        }
    }
    return nb;
}
