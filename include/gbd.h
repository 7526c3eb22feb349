/*
 * gbd.h -- C ABI of a GB300-native plane-evaluation Gaussian beamlet decomposition (GBD).
 *
 * Method (arXiv 2404.12454): a pupil wavefront is decomposed into Gaussian beamlets on a
 * square grid (Eq. sum_gaussian, Eq. OF); each beamlet is carried through a paraxial
 * system by a chief ray and four parabasal rays whose one-sided differences give a 4x4
 * differential ray-transfer matrix (Sec. 2.2); the Gaussian solution of the Collins
 * integral (Eq. gauss_prop) propagates its complex curvature and amplitude; and the
 * beamlet is evaluated on every pixel of a common evaluation plane at once (Sec. 3,
 * Eq. collins_factored) before the coherent sum over beamlets.
 *
 * Conventions shared by every call:
 *   - SI units (metres), angles in radians, time convention exp(-ik * optical path).
 *   - Phases are relative to the axial path: the constant exp(-ik d) is not applied.
 *   - Calls are asynchronous on the CUDA stream passed as `stream` (a cudaStream_t; NULL
 *     is the legacy default stream).  Pointers documented as "device" must be device
 *     memory of the current device; the library never frees or retains caller memory.
 *   - Argument errors are found on the host before any launch and return GBD_EINVAL;
 *     nothing is launched then.  CUDA errors return GBD_ECUDA.  A kernel that gives up
 *     a bounded wait records GBD_ETIMEOUT in a per-device status word read by
 *     gbd_sync().  gbd_last_error() gives a message for the calling thread.
 *   - No call allocates device memory (gbd_probe_peaks excepted, which is a
 *     measurement tool); scratch memory is a caller-provided workspace whose size a
 *     *_workspace_bytes query returns.
 *   - All entry points are safe to call from several host threads on different streams.
 */
#ifndef GBD_H
#define GBD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBD_OK = 0,
    GBD_EINVAL = 1,       /* bad argument (detected on the host, nothing launched) */
    GBD_ECUDA = 2,        /* CUDA runtime error                                    */
    GBD_ENOMEM = 3,       /* workspace or capacity too small / host allocation     */
    GBD_ETIMEOUT = 4,     /* a device wait gave up (see gbd_sync)                  */
    GBD_EUNSUPPORTED = 5  /* device is not sm_103 / feature unavailable            */
} gbd_status;

enum { GBD_PREC_F64 = 0, GBD_PREC_MIXED = 1 };

#define GBD_MAX_ZERN 64   /* Zernike terms in an OPD plate                       */
#define GBD_MAX_NOLL 66   /* highest Noll index (radial order <= 10)             */

/* Paraxial system: [OPD plate] -> thin lens -> free space to the reference plane.
 * The plate is a thin phase screen at the pupil with optical path
 * W(x, y) = sum_t zern_coef[t] * Z_{noll[t]}(x / zern_radius, y / zern_radius), Noll-ordered,
 * RMS-normalised Zernike polynomials (Sec. 4.3 uses Noll modes).  The lens of focal
 * length f transmits exp(+ik r^2 / 2f) (use +INFINITY for no lens, Eq. abcd_sys). */
typedef struct {
    double wavelength;    /* m                                         */
    double focal_length;  /* m, +INFINITY = no lens                    */
    double distance;      /* m, lens (pupil) to the reference plane    */
    double zern_radius;   /* m, normalisation radius of the plate       */
    int32_t n_zern;       /* 0 .. GBD_MAX_ZERN                          */
    int32_t noll[GBD_MAX_ZERN];       /* 1 .. GBD_MAX_NOLL             */
    double zern_coef[GBD_MAX_ZERN];   /* m of optical path             */
} gbd_system;

/* Uniform circular pupil of `diameter` sampled by `n_across` beamlets across: centres
 * x_i = (i - (N-1)/2) s, s = D/N, kept when |r| <= D/2 (Eq. OF, Sec. 6). */
typedef struct {
    double diameter;      /* m                        */
    int32_t n_across;     /* 1 .. 4096                */
    int32_t reserved;
} gbd_pupil;

/* Detector plane through the reference point (0, 0, d), rotated by R = Ry(rot_y) Rx(rot_x).
 * Pixel (i, j) (column i, row j) sits at s = ((i - nx/2) pitch_x, (j - ny/2) pitch_y)
 * (integer division), lab point (0, 0, d) + R (s, 0).  A field is stored row-major
 * [ny][nx].  The second-order tilted-plane rule applies (see gbd_field). */
typedef struct {
    double pitch_x, pitch_y;   /* m, > 0               */
    double rot_x, rot_y;       /* rad, |.| < 1.2       */
    int32_t nx, ny;            /* 1 .. 16384 each      */
} gbd_detector;

/* One traced beamlet (FP64, 36 doubles = 288 bytes), written by gbd_trace and
 * gbd_trace_mirrors. */
typedef struct {
    double rho[2];      /* chief-ray landing point on the reference plane, m            */
    double theta[2];    /* chief-ray slope                                             */
    double path;        /* chief-ray optical path in excess of the axial path, m       */
    double amp[2];      /* a_j / sqrtdet(A + B P1), complex (re, im)                    */
    double curv[8];     /* P2 = (C + D P1)(A + B P1)^-1, 2x2 complex row-major (re, im) */
    double abcd[16];    /* A, B, C, D 2x2 blocks, each row-major                        */
    double center[2];   /* beamlet centre r_j in the pupil, m                           */
    double weight;      /* a_j = s^2 / (pi w0^2)                                        */
    double waist;       /* w0 = OF D / (2N), m                                          */
    double edge_distance; /* 0; for an edge beamlet of gbd_trace_truncated, the signed
                             distance d_j = R - |r_j| from its centre to the aperture edge */
} gbd_beamlet;

/* Message describing the last failure on this thread ("" when none). */
const char* gbd_last_error(void);

/* Library version string. */
const char* gbd_version(void);

/* Number of beamlets gbd_trace produces for `pupil` (host only, no GPU work), or -1 for
 * an invalid pupil.  Exact integer inside-test (2i-(N-1))^2 + (2j-(N-1))^2 <= N^2. */
int32_t gbd_beamlet_count(const gbd_pupil* pupil);

/* Synchronises `stream` and returns GBD_ETIMEOUT if any kernel of this library gave up a
 * bounded wait on the current device since the last gbd_sync (the word is then cleared),
 * GBD_ECUDA on a CUDA error, else GBD_OK.
 * gbd_sync is the only way to observe GBD_ETIMEOUT.  The status word is one per device,
 * not per stream or call: a timeout of a kernel on one stream is reported by whichever
 * gbd_sync on that device reads the word next, and a caller that synchronises by other
 * means (cudaStreamSynchronize, torch) never sees it.  After a timeout the outputs of the
 * calls since the previous gbd_sync are undefined; call gbd_sync after each batch of work
 * whose results are used. */
gbd_status gbd_sync(void* stream);

/* Test hook: sets the iteration limit of every device-side bounded wait on the current
 * device (0 restores the default of about a second).  A limit of 1 makes waits that are
 * not already satisfied give up at once, so tests can exercise GBD_ETIMEOUT. */
gbd_status gbd_set_wait_limit(uint32_t spins);

/* ---------------------------------------------------------------- gbd_trace -------
 * Decomposes the pupil and traces every beamlet (Sec. 2.2 steps 1 and 4, Eq. gauss_prop,
 * Eq. OF).  For each grid centre r_j inside the pupil, in row-major grid order:
 *   w0 = overlap_factor * D / (2N),  a_j = s^2 / (pi w0^2),  P1 = -i lambda/(pi w0^2) I;
 *   chief ray (r_j, 0); waist rays (r_j + h e_x|e_y, 0) with h = waist_ratio * w0;
 *   divergence rays (r_j, a e_x|e_y) with a = waist_ratio * lambda / (pi w0);
 *   each ray: plate (path += W, slope += grad W), lens (path -= r^2/2f, slope -= r/f),
 *   distance d (r += d slope, path += d |slope|^2 / 2);
 *   A, C columns = (waist ray - chief) / h,  B, D columns = (divergence ray - chief) / a;
 *   P2 = (C + D P1)(A + B P1)^-1, amp = a_j / sqrtdet(A + B P1) with sqrtdet the product
 *   of the principal square roots of the eigenvalues of A + B P1.
 * out: device array of `capacity` records; gbd_beamlet_count(pupil) of them are written.
 * Errors: GBD_EINVAL for non-finite / non-positive wavelength, distance or diameter,
 * overlap_factor or waist_ratio <= 0, bad Noll indices; GBD_ENOMEM if capacity is too
 * small.  FP64 throughout. */
gbd_status gbd_trace(const gbd_system* system, const gbd_pupil* pupil, double overlap_factor,
                     double waist_ratio, gbd_beamlet* out, int32_t capacity, void* stream);

/* ---------------------------------------------------------------- mirrors ---------
 * Real-ray trace through reflective conic surfaces (the Ritchey-Chretien telescope of
 * App. B), for the same decomposition as gbd_trace.  Light enters travelling +z; the
 * entrance pupil (where beamlets are decomposed and rays start, slopes 0 or the
 * divergence rays' a) is a plane pupil_offset before the first vertex.  Surface k has
 * vertex z_k (z_1 = 0, z_{k+1} = z_k + spacing[k]; the image / reference plane is
 * spacing[n-1] after the last vertex), radius with App. B's sign (negative = concave,
 * positive = convex towards the arriving light) and conic constant; its lab-frame
 * curvature is s_k / radius[k] with s_k = +-1 the direction of travel before it.  Rays are
 * traced exactly (intersection, reflection about the surface normal, geometric path);
 * path is the excess over the axial ray from the pupil plane to the reference plane.
 * No obscuration or vignetting is modelled (the paper removes the secondary's).
 * Errors: GBD_EINVAL for n_mirrors outside [1, GBD_MAX_MIRRORS], zero or non-finite
 * radius/spacing, non-finite conic, pupil_offset <= 0. */
#define GBD_MAX_MIRRORS 4
typedef struct {
    double wavelength;                 /* m                                        */
    double pupil_offset;               /* m, > 0                                   */
    int32_t n_mirrors;
    int32_t reserved;
    double radius[GBD_MAX_MIRRORS];    /* m, App. B sign convention                */
    double conic[GBD_MAX_MIRRORS];
    double spacing[GBD_MAX_MIRRORS];   /* m, signed axial distance to the next one */
} gbd_mirror_system;

gbd_status gbd_trace_mirrors(const gbd_mirror_system* system, const gbd_pupil* pupil,
                             double overlap_factor, double waist_ratio, gbd_beamlet* out,
                             int32_t capacity, void* stream);

/* ---------------------------------------------------------------- gbd_field -------
 * Coherent sum over beamlets of each beamlet's field on every detector pixel (Eq.
 * sum_gaussian, Eq. collins_factored with the chief-ray slope term, Eqs. ab_prop/cd_prop):
 *   E(s) = sum_j amp_j exp(-z tr(P)/2 - ik [path + z (1 - |theta|^2/2) + theta.delta
 *                                            + w^T P w / 2]),
 *   delta = X_xy(s) - rho_c,  z = X_z(s) - d,  w = delta - z theta,
 * i.e. each beamlet propagated paraxially by the pixel's axial offset z and expanded to
 * second order in s (exact for an untilted plane, z = 0).
 * precision GBD_PREC_F64: FP64 throughout, field_out is complex128 [ny][nx].
 * precision GBD_PREC_MIXED: per-beamlet projection in FP64 (constant phase reduced mod
 *   one turn), per-pixel quadratic form in FP32, exp2/sin/cos on the MUFU pipe (phases
 *   reduced exactly first when some beamlet's phase can exceed 128 rad on the detector).
 *   With the row-pair scheme (see gbd_shape) only one row of each pair 8 apart is
 *   evaluated so; the row 8 below is that value times the beamlet's exact 8-row step
 *   factor (an FP32 complex multiply); with row quadruples (the default) or triples also
 *   the rows 16 and 24 (16) below, by the next step factors (with a uv term: times the
 *   column's power W^r of the uv factor, stepped along the row; on row triples behind
 *   a 4x8 pick).  The sum runs in FP32 64-beamlet chunks combined with compensated (TwoSum)
 *   accumulation (row triples and quadruples: in FP32 over the whole beamlet split, which
 *   then holds at most 1,024 beamlets); beamlet
 *   splits are rounded once to FP32 and summed in split order with Neumaier's
 *   compensation; field_out is complex64.
 * workspace: device scratch of at least gbd_field_workspace_bytes(...) bytes, 256-byte
 *   aligned.  Contents on entry are ignored.
 * n_beamlets may be 0 (the field is then zero).
 * Errors: GBD_EINVAL (bad detector, precision, null pointers, misaligned workspace),
 * GBD_ENOMEM (workspace too small). */
size_t gbd_field_workspace_bytes(int32_t n_beamlets, const gbd_detector* detector,
                                 int32_t precision);
gbd_status gbd_field(const gbd_beamlet* beamlets, int32_t n_beamlets, double wavelength,
                     const gbd_detector* detector, int32_t precision, void* workspace,
                     size_t workspace_bytes, void* field_out, void* stream);

/* ------------------------------------------------------- truncated beamlets ------
 * Beamlets truncated at the aperture edge (Sec. 1 and the Conclusion: Worku & Gross's
 * truncated Gaussian beamlets represent hard edges better; the plane method applies to any
 * closed-form solution of the Collins integral, Eq. collins).
 * Decomposition (gbd_trace_truncated): the gbd_trace grid (same spacing s, waist w0, weights)
 *   extended to every centre with |r_j| <= R + margin w0 (R = D/2).  Centres more than
 *   margin w0 inside the edge give whole beamlets; the others are edge beamlets, whose input
 *   Gaussian is cut by the aperture's tangent half-plane n.(r - r_j) <= d_j, n = r_j/|r_j|,
 *   d_j = R - |r_j| (negative outside).  In half-pitch units (a = 2i - (N-1), b = 2j - (N-1))
 *   a centre is kept when a^2 + b^2 <= (N + margin OF)^2 and whole when a^2 + b^2 <
 *   (N - margin OF)^2.  out: the whole beamlets first, then the edge beamlets, each in
 *   row-major grid order (the grid's row j along y outer); an edge beamlet's edge_distance
 *   is d_j.  *n_edge (host, may be NULL) receives the edge count.
 * gbd_truncated_count: the number of beamlets (and in *n_edge the edge ones), or -1 for bad
 *   arguments (host only).
 * gbd_field_truncated: the field of such a table on an UNTILTED detector: the first
 *   n_beamlets - n_edge records as gbd_field, plus for each edge beamlet its Gaussian times
 *       1/2 erfc(zeta),  zeta = (n^T M^-1 (rho - rho_c) - d) sqrt(i k / (2 n^T M^-1 B n)),
 *   M = A + B P1 (the Collins integral of the cut Gaussian over its half-plane; principal
 *   root), evaluated through the Faddeeva function (Weideman's rational approximation:
 *   36 terms in FP64, 16 in the mixed path's FP32, where along a row it is Taylor-stepped
 *   to 4th order from pixel to pixel while the step is short).  The edge beamlets are split
 *   over CTAs into partial fields added in split order (deterministic).  workspace: at
 *   least gbd_field_truncated_workspace_bytes(...) bytes, 256-byte aligned (the edge
 *   records, then the larger of gbd_field's workspace and the edge partial fields).
 * Errors: GBD_EINVAL (bad arguments, margin outside [0, 10], n_edge outside
 *   [0, n_beamlets]), GBD_ENOMEM (capacity or workspace too small), GBD_EUNSUPPORTED (a
 *   tilted detector). */
int32_t gbd_truncated_count(const gbd_pupil* pupil, double overlap_factor, double margin,
                            int32_t* n_edge);
gbd_status gbd_trace_truncated(const gbd_system* system, const gbd_pupil* pupil,
                               double overlap_factor, double waist_ratio, double margin,
                               gbd_beamlet* out, int32_t capacity, int32_t* n_edge,
                               void* stream);
size_t gbd_field_truncated_workspace_bytes(int32_t n_beamlets, int32_t n_edge,
                                           const gbd_detector* detector, int32_t precision);
gbd_status gbd_field_truncated(const gbd_beamlet* beamlets, int32_t n_beamlets, int32_t n_edge,
                               double wavelength, const gbd_detector* detector, int32_t precision,
                               void* workspace, size_t workspace_bytes, void* field_out,
                               void* stream);

/* ------------------------------------------------------------ gbd_field_rows ------
 * The same field (Eq. sum_gaussian with the plane form of Eq. collins_factored, as
 * gbd_field) on detector rows [row_begin, row_end) only: a slab of the detector, for
 * spreading one field over several GPUs by pixels.  The beamlet table is the whole table
 * (every slab sums every beamlet); the plane-evaluation method is pixel-parallel (Sec. 5),
 * so slabs need no exchange but the final gather.
 *   detector: the WHOLE detector (pixel (i, j) is s = ((i - nx/2) px, (j - ny/2) py) as in
 *     gbd_field); 0 <= row_begin <= row_end <= ny.
 *   field_out: (row_end - row_begin) x nx complex64 (MIXED) or complex128 (F64), row-major,
 *     row 0 = detector row row_begin; device memory owned by the caller.
 *   workspace: at least gbd_field_rows_workspace_bytes(...) bytes, 256-byte aligned (the
 *     split partial fields cover only the slab, rounded down at its start to the launch's
 *     row-block height of at most 48 rows).
 * The launch (shape, splits) and the projection's kernel selection are those gbd_field
 * takes on the whole detector, and every pixel of the slab is computed by the same thread
 * row block, so the slab equals the same rows of gbd_field's output bit for bit, for any
 * row range.  An empty range writes nothing.  Errors as gbd_field, plus GBD_EINVAL for a
 * row range outside the detector. */
size_t gbd_field_rows_workspace_bytes(int32_t n_beamlets, const gbd_detector* detector,
                                      int32_t row_begin, int32_t row_end, int32_t precision);
gbd_status gbd_field_rows(const gbd_beamlet* beamlets, int32_t n_beamlets, double wavelength,
                          const gbd_detector* detector, int32_t row_begin, int32_t row_end,
                          int32_t precision, void* workspace, size_t workspace_bytes,
                          void* field_out, void* stream);

/* Per-beamlet projection alone (the first half of gbd_field), for inspection: writes the
 * quadratic-form record of every beamlet to `coeffs` (device).
 *   MIXED: 16 floats per beamlet in the tiled layout gbd_field uses
 *          [tile = b / 64][field f = 0..3][b % 64][4 floats];
 *          values (i0, j0, a0, p0 | a1u, p1u, a1v, p1v | auu, puu, auv, puv | avv, pvv, Tr, Ti)
 *          with log2 |E_j(i, j)| = a0 + a1u tu + a1v tv + auu tu^2 + auv tu tv + avv tv^2 and
 *          the phase in radians p0 + ... likewise (p0 in [-pi, pi)), tu = i - i0, tv = j - j0
 *          (pixel units), excluding the common carrier exp(-ik z(s)); T = Tr + i Ti =
 *          exp(256 (auv ln 2 + i puv)), the row-pair scheme's column factor.
 *          wide_flag (device, may be NULL; zero it first) is OR-ed with bit 0 if some
 *          beamlet's phase can exceed 128 rad on the detector (gbd_field then reduces every
 *          per-pixel phase exactly before sin/cos), bit 1 if some beamlet's log2
 *          amplitude can change by more than 64 over 8 rows (the row-pair scheme then falls
 *          back to direct evaluation), bit 2 if it can change by more than 64 over 8
 *          columns 32 apart (the row-pair scheme then evaluates each amplitude instead of
 *          carrying it along the row), bit 3 if some beamlet has a uv term (auv or puv not
 *          zero; without one T is exactly 1, the row-pair kernels leave out its update and
 *          the row triples and quadruples take the column-free step factors, with one
 *          their per-column factors) and bit 4 if its log2 amplitude can change by more
 *          than 64 over 24 rows (the row triples and quadruples then hand the field to the
 *          row pairs).
 *   F64:   16 doubles per beamlet [tile][field f = 0..7][b % 64][2 doubles], same order, the
 *          phase in turns (phase / 2 pi), field 7 = S = exp of twice the uu coefficient as
 *          a complex number (re, im), the second ratio of a row recurrence; wide_flag is
 *          not used.
 * coeffs must hold gbd_project_bytes(n, precision) bytes. */
size_t gbd_project_bytes(int32_t n_beamlets, int32_t precision);
gbd_status gbd_project(const gbd_beamlet* beamlets, int32_t n_beamlets, double wavelength,
                       const gbd_detector* detector, int32_t precision, void* coeffs,
                       uint32_t* wide_flag, void* stream);

/* ---------------------------------------------------------------- point evaluation --
 * The prior method the plane rule accelerates (Sec. 2.2): each beamlet propagated to each
 * pixel on its own.  Here the beamlet is carried paraxially from the reference plane to
 * the pixel's axial offset z: P(z) = P (I + z P)^-1, amplitude amp / sqrtdet(I + z P)
 * (eigenvalue branch), centroid rho + z theta, path + z (1 + |theta|^2 / 2), and evaluated
 * at the pixel; FP64, complex128 [ny][nx] output.  On an untilted plane it equals
 * gbd_field; on a tilted plane their difference is the plane rule's method error.
 * workspace >= gbd_field_point_workspace_bytes, 256-byte aligned. */
size_t gbd_field_point_workspace_bytes(int32_t n_beamlets, const gbd_detector* detector);
gbd_status gbd_field_point(const gbd_beamlet* beamlets, int32_t n_beamlets, double wavelength,
                           const gbd_detector* detector, void* workspace, size_t workspace_bytes,
                           void* field_out, void* stream);

/* ---------------------------------------------------------------- tuning ----------
 * Launch shape of the field kernels: pixels per thread (rows x cols), beamlet splits and
 * (mixed) evaluation scheme.  Unless a shape was set for the current device with
 * gbd_field_set_shape (NULL restores this default), gbd_field uses 8, 4 or 2 columns per
 * thread, whichever covers the detector's width at the least estimated cost (8 for widths
 * that are multiples of 256), as row quadruples (4x8) or row pairs (2x4, 2x2), or row
 * segments (F64: 1x32 on detectors 256 or more pixels wide, else 1x16), with splits from a built-in heuristic; gbd_autotune_field times the
 * candidate shapes on the given problem (synchronously, with CUDA events) and keeps the
 * fastest. */
typedef struct {
    int32_t rows_per_thread;   /* mixed: 1x4, 2x2, 2x4, 4x2 (columns 32 apart);   */
    int32_t cols_per_thread;   /* F64: 1x2, 2x2 (direct), 1x8, 2x8, 1x16, 1x32   */
                               /* (contiguous row segments, complex recurrence),  */
                               /* 2x16, 4x8, 8x4 (row bands: no-uv beamlets as    */
                               /* X(u) Y(v), Y from a per-warp table)             */
    int32_t splits;            /* beamlet splits (0 = heuristic)             */
    float   ms;                /* measured time of the shape (autotune)      */
    int32_t scheme;            /* mixed only: GBD_SCHEME_DIRECT, or           */
                               /* GBD_SCHEME_ROW_PAIR (2x2, 2x4, 2x8: the     */
                               /* second row from the first by a complex      */
                               /* factor; 3x8, 4x8, 4x4: row triples and      */
                               /* quadruples, for splits of at most 16 tiles  */
                               /* and fields whose 24-row amplitude step      */
                               /* stays within 2^64, the 2 x cols row pairs   */
                               /* otherwise)                                  */
} gbd_shape;

#define GBD_SCHEME_DIRECT 0
#define GBD_SCHEME_ROW_PAIR 1
gbd_status gbd_field_set_shape(int32_t precision, const gbd_shape* shape);
gbd_status gbd_field_get_shape(int32_t precision, int32_t n_beamlets,
                               const gbd_detector* detector, gbd_shape* out);
gbd_status gbd_autotune_field(const gbd_beamlet* beamlets, int32_t n_beamlets,
                              double wavelength, const gbd_detector* detector,
                              int32_t precision, void* workspace, size_t workspace_bytes,
                              void* field_out, void* stream, gbd_shape* best);

/* ---------------------------------------------------------------- no allocation ---
 * gbd_field without a workspace, for callers that must not allocate device memory: a
 * plugin inside a host application that owns every device allocation, or a real-time
 * loop whose memory is fixed at start-up, can neither call cudaMalloc nor pass scratch.
 * (No counterpart in the paper: this is a property of the library, not of the method.)
 * The scratch is one static device array of GBD_NOALLOC_SCRATCH_BYTES (32 MiB) inside
 * the library; every GPU that loads the library holds it until the process exits.
 *   - Same arguments and results as gbd_field, without workspace/workspace_bytes; the
 *     caller still owns beamlets and field_out.
 *   - The first call on a device looks the array's device address up (with that device
 *     current); make that first call before any stream capture.
 *   - A problem whose projected beamlet records plus one partial field of nx x ny pixels
 *     exceeds the array is rejected with GBD_EINVAL before any launch (beamlet splits are
 *     lowered to fit first; records take 64 B (mixed) / 128 B (FP64) per beamlet rounded
 *     up to 64 beamlets, a partial field 8 B (mixed) / 16 B (FP64) per pixel).
 *   - All calls share the array and each overwrites every byte it later reads, so nothing
 *     carries over from the previous call; calls that overlap on the GPU (for example
 *     on two streams of one device) race on it and must be serialised.  Each device
 *     has its own copy.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine. */
#define GBD_NOALLOC_SCRATCH_BYTES (32u << 20)
gbd_status gbd_field_noalloc(const gbd_beamlet* beamlets, int32_t n_beamlets, double wavelength,
                             const gbd_detector* detector, int32_t precision, void* field_out,
                             void* stream);

/* ---------------------------------------------------------------- host PSF --------
 * Trace + field + copy to the host in one call, for callers that want the field in host
 * memory: workspace (device, 256-byte aligned, >= gbd_psf_workspace_bytes) holds the
 * beamlet table, the device field and the field scratch; host_field_out (complex64 or
 * complex128 [ny][nx], pinned for a truly asynchronous copy) is valid after gbd_sync. */
size_t gbd_psf_workspace_bytes(const gbd_pupil* pupil, const gbd_detector* detector,
                               int32_t precision);
gbd_status gbd_psf(const gbd_system* system, const gbd_pupil* pupil, double overlap_factor,
                   double waist_ratio, const gbd_detector* detector, int32_t precision,
                   void* workspace, size_t workspace_bytes, void* host_field_out, void* stream);

/* ---------------------------------------------------------------- timing ----------
 * Measurement hooks.  While enabled, every launch of the traces, the per-beamlet
 * projection, the field kernels and the split reduction is bracketed by CUDA events on its
 * stream.  gbd_timing_read synchronises those events, returns per kind the summed
 * milliseconds and launch counts (index 0 mixed field kernel, 1 FP64 field kernel,
 * 2 projection, 3 reduction, 4 point evaluation, 5 trace (gbd_trace, gbd_trace_mirrors);
 * arrays of 6) and forgets them. */
gbd_status gbd_timing_enable(int32_t on);
gbd_status gbd_timing_read(double* total_ms, int64_t* launches);

/* ---------------------------------------------------------------- gbd_sweep -------
 * Batched parameter sweep (Sec. 6, Fig. optimal_param_search): n instances that share the
 * optics (system, pupil diameter) and an untilted detector but each have their own
 * beamlets across, overlap factor and waist ratio, evaluated in mixed precision and scored
 * by the RMS of |E|/|E(centre)| - |2 J1(x)/x| (x = pi r / (lambda F#), F# = f / D) over
 * the pixels with r <= j_{1,3} lambda F# / pi (inside the third dark ring); the centre is
 * pixel (nx/2, ny/2).
 * gbd_sweep_plan_create: host only; validates, lays out the tables and the work list
 *   ((instance, pixel block) items, instances with the most beamlet tiles first) and the
 *   workspace.  shape = NULL picks 8 or 4 columns per thread, whichever covers the
 *   detector's width at the lower estimated cost (8 for widths that are multiples of
 *   256): row triples (3x8; 256 x 24-pixel items; the sums folded every 16 tiles into a
 *   compensated pair with its low part in BF16; fields with a uv term with per-column
 *   row factors, folded every tile; fields too steep for the recurrence evaluated
 *   directly on the same items) or row pairs (2x4); a shape's scheme field selects direct
 *   or row-recurrence evaluation.
 * gbd_sweep_bind: records the caller's device workspace (>= gbd_sweep_workspace_bytes,
 *   256-byte aligned; it must outlive the plan's runs), uploads the tables and the Airy
 *   table; synchronises `stream`.
 * gbd_sweep_run: batched trace + projection, the persistent field + score kernel and the
 *   finalize, asynchronous on `stream`; scores = device double[n_instances].  The score
 *   of every instance is deterministic (fixed summation order).
 * gbd_sweep_run_graph: the same work captured once into a CUDA graph (on the first call
 *   for a given scores pointer and stream) and replayed; `stream` must be a created
 *   stream, not the legacy default stream.
 * gbd_sweep_autotune: times every supported shape on the given instances (synchronous)
 *   and returns the fastest; the workspace must hold the largest plan.
 * gbd_sweep_set_zones: optional annular zones lo[z] <= r / (lambda F#) < hi[z] (Sec. 6 uses
 *   0-5, 5-10, 10-15 lambda/D), at most 7, before gbd_sweep_bind; the scores array then
 *   holds 1 + n_zones doubles per instance: the score above, then the same RMS over
 *   each zone (same |E(centre)| normalisation).
 * gbd_sweep_info: total beamlet-pixel evaluations, beamlets and work items of a plan. */
typedef struct gbd_sweep_plan gbd_sweep_plan;
gbd_status gbd_sweep_plan_create(const gbd_system* system, double diameter, const int32_t* n_across,
                                 const double* overlap_factor, const double* waist_ratio,
                                 int32_t n_instances, const gbd_detector* detector,
                                 const gbd_shape* shape, gbd_sweep_plan** plan);
/* The same sweep with every instance's beamlets traced by real rays through a sequence of
 * conic mirrors (as gbd_trace_mirrors, App. B's telescope; Sec. 6 searches the parameters
 * on such a traced system).  diameter: the pupil's; f_number: the system's focal ratio,
 * which sets the Airy pattern of the score (x = pi r / (lambda f_number)); the detector is
 * centred on the mirror sequence's image plane.  Everything else as gbd_sweep_plan_create;
 * the plan is used with the same calls.  Errors: GBD_EINVAL for a bad mirror sequence (as
 * gbd_trace_mirrors), f_number <= 0 or bad instances. */
/* With shape = NULL a mirror sweep runs the row pairs (2 x 8 or 2 x 4): real-ray beamlets
 * carry a uv term, which the row triples take with per-column row factors, 2.5 % faster
 * but with scores further from the oracle's (up to 2.2e-4 relative at 256 across against
 * 9e-5 for the pairs). */
gbd_status gbd_sweep_plan_create_mirrors(const gbd_mirror_system* system, double diameter,
                                         double f_number, const int32_t* n_across,
                                         const double* overlap_factor, const double* waist_ratio,
                                         int32_t n_instances, const gbd_detector* detector,
                                         const gbd_shape* shape, gbd_sweep_plan** plan);
size_t gbd_sweep_workspace_bytes(const gbd_sweep_plan* plan);
gbd_status gbd_sweep_set_zones(gbd_sweep_plan* plan, int32_t n_zones, const double* lo,
                               const double* hi);
gbd_status gbd_sweep_info(const gbd_sweep_plan* plan, double* evals, int64_t* beamlets,
                          int32_t* items);
gbd_status gbd_sweep_bind(gbd_sweep_plan* plan, void* workspace, size_t bytes, void* stream);
gbd_status gbd_sweep_run(gbd_sweep_plan* plan, double* scores, void* stream);
gbd_status gbd_sweep_run_graph(gbd_sweep_plan* plan, double* scores, void* stream);
gbd_status gbd_sweep_autotune(const gbd_system* system, double diameter, const int32_t* n_across,
                              const double* overlap_factor, const double* waist_ratio,
                              int32_t n_instances, const gbd_detector* detector, void* workspace,
                              size_t bytes, double* scores, void* stream, gbd_shape* best);
void gbd_sweep_plan_destroy(gbd_sweep_plan* plan);

/* ---------------------------------------------------------------- MLP surrogate ---
 * Not in the paper: a small network that learns log10 of the sweep's Airy score from
 * (overlap factor, waist ratio, log2 beamlets across), standardised by the caller, so
 * that a search verifies only the parameter sets it predicts to be best.
 * Architecture: 3 -> 128 -> 128 -> 128 -> 128 -> 1, GELU x Phi(x) after each hidden layer
 * (Phi, the normal CDF, by Abramowitz & Stegun 7.1.26: absolute error <= 1.5e-7), linear
 * output.  GBD_MLP_PARAMS floats in the order
 * W1[128][3] b1[128] W2[128][128] b2[128] W3 b3 W4 b4 W5[1][128] b5[1] (W[out][in]).
 * Compute: BF16 weights (round to nearest even from the FP32 master copy), FP32
 * activations and accumulation; the 128 x 128 layers on the tensor cores with the FP32
 * operands split into BF16 parts (forward pass: three, FP32-accurate; training: two,
 * 2^-18 relative); loss = mean over the batch of (y - target)^2; Adam with bias correction
 * on the FP32 master weights.  All reductions have an order fixed by the batch size, so
 * results are deterministic.  x is float[batch][3], target/y float[batch], all device;
 * weights 16-byte aligned, workspaces 256-byte aligned (EINVAL otherwise); batch 1 .. 2^20
 * for training, 1 .. 2^24 for the forward pass.
 * gbd_mlp_pack:       weights (uint16 BF16 bits) = round(master).
 * gbd_mlp_forward:    y = MLP(x); no workspace.
 * gbd_mlp_grad:       grad = dLoss/dparams (float[GBD_MLP_PARAMS]) and *loss (device float,
 *                     may be NULL) at the BF16 weights; workspace >= gbd_mlp_workspace_bytes
 *                     (about 4 KB per sample: the layers' activations and errors in BF16
 *                     parts, a_4 and dL/dz_1 in FP32, y and dL/dy; a 106 KB weight image).
 * gbd_mlp_adam:       one Adam step (step counts from 1) on master/m/v, then repacks.
 * gbd_mlp_train:      `steps` full-batch steps (gradient, then Adam), step numbers
 *                     first_step, first_step + 1, ...; *loss (may be NULL) = the loss of
 *                     the last step, at the weights before its update.  One cooperative
 *                     launch runs all steps (every CTA resident; grid barriers between the
 *                     sample-parallel and the parameter-parallel phase of each step, bounded
 *                     waits: GBD_ETIMEOUT from gbd_sync); nothing is synchronised.
 *                     gbd_mlp_grad is the same launch with one step and no update.
 * gbd_mlp_train_step: gbd_mlp_train with steps = 1. */
#define GBD_MLP_PARAMS 50177
size_t gbd_mlp_workspace_bytes(int32_t batch);
gbd_status gbd_mlp_pack(const float* master, uint16_t* weights, void* stream);
gbd_status gbd_mlp_forward(const uint16_t* weights, const float* x, int32_t batch, float* y,
                           void* stream);
gbd_status gbd_mlp_grad(const uint16_t* weights, const float* x, const float* target,
                        int32_t batch, float* grad, float* loss, void* workspace, size_t bytes,
                        void* stream);
gbd_status gbd_mlp_adam(float* master, uint16_t* weights, float* m, float* v, const float* grad,
                        float lr, float beta1, float beta2, float eps, int32_t step, void* stream);
gbd_status gbd_mlp_train(float* master, uint16_t* weights, float* m, float* v, const float* x,
                         const float* target, int32_t batch, float lr, float beta1, float beta2,
                         float eps, int32_t first_step, int32_t steps, float* loss,
                         void* workspace, size_t bytes, void* stream);
gbd_status gbd_mlp_train_step(float* master, uint16_t* weights, float* m, float* v,
                              const float* x, const float* target, int32_t batch, float lr,
                              float beta1, float beta2, float eps, int32_t step, float* loss,
                              void* workspace, size_t bytes, void* stream);

/* ---------------------------------------------------------------- probes ----------
 * Throughput microbenchmarks of the pipes the field kernels are bound by, on the current
 * device (synchronous): MUFU ex2 / sin / cos results per second, FP32 FMA per second and
 * FP64 FMA per second.  out[5] = {ex2, sin, cos, ffma, dfma} in operations/s. */
gbd_status gbd_probe_peaks(double* out);

#ifdef __cplusplus
}
#endif
#endif /* GBD_H */
