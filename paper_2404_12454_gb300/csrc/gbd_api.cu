// C ABI of the GBD library: argument validation, host-side set-up of the kernels'
// parameters, launch-shape selection and the workspace layout.  All numerical work of
// the method runs in the kernels of trace.cu, field.cu and sweep.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "gbd.h"
#include "gbd_internal.cuh"

namespace {

thread_local char g_err[512] = "";

gbd_status fail(gbd_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

gbd_status cuda_fail(cudaError_t e, const char* where) {
    return fail(GBD_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

std::mutex g_mu;
std::map<int, uint32_t> g_wait_spins;                 // per device
std::map<std::pair<int, int>, gbd_shape> g_shapes;     // (device, precision) -> shape
std::map<int, int> g_sm_count;

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

uint32_t wait_spins() {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_wait_spins.find(current_device());
    return it == g_wait_spins.end() ? gbd::kDefaultWaitSpins : it->second;
}

int sm_count() {
    int dev = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_sm_count.find(dev);
    if (it != g_sm_count.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 1;
    g_sm_count[dev] = n;
    return n;
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// ------------------------------------------------------------- kernel timing --
// While enabled, launches of the measured kernels are bracketed by CUDA events on their
// own stream; gbd_timing_read synchronises the events and sums the durations.
enum {
    kTimeMixed = 0,
    kTimeF64 = 1,
    kTimeProject = 2,
    kTimeReduce = 3,
    kTimePoint = 4,
    kTimeTrace = 5,
    kTimeKinds = 6
};
struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
};
bool g_timing = false;
std::vector<TimedLaunch> g_timed;

struct TimingScope {
    TimedLaunch t{-1, nullptr, nullptr};
    cudaStream_t s;
    TimingScope(int kind, cudaStream_t st) : s(st) {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_timing) return;
        if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) return;
        t.kind = kind;
        cudaEventRecord(t.a, s);
    }
    ~TimingScope() {
        if (t.kind < 0) return;
        cudaEventRecord(t.b, s);
        std::lock_guard<std::mutex> lk(g_mu);
        g_timed.push_back(t);
    }
};

// ------------------------------------------------------------------ Zernike --

// Noll index -> radial order n, azimuthal order |m|, sine term?
void noll_nm(int j, int& n, int& m, bool& is_sin) {
    n = (int)floor((sqrt(8.0 * j - 7.0) - 1.0) / 2.0);
    while ((n + 1) * (n + 2) / 2 < j) ++n;  // guard the floor against rounding
    while (n > 0 && n * (n + 1) / 2 >= j) --n;
    const int p = j - n * (n + 1) / 2;  // 1-based position inside order n
    m = (n % 2 == 0) ? 2 * (p / 2) : 2 * ((p - 1) / 2) + 1;
    is_sin = (m != 0) && (j % 2 == 1);
}

double binom(int a, int b) {
    double r = 1.0;
    for (int q = 1; q <= b; ++q) r = r * (a - b + q) / q;
    return r;
}

double fact(int a) {
    double r = 1.0;
    for (int q = 2; q <= a; ++q) r *= q;
    return r;
}

// Adds coef * Z_j(xi, eta) to the degree-ordered monomial table.
void add_zernike(int j, double coef, double* table, int& max_deg) {
    int n, m;
    bool is_sin;
    noll_nm(j, n, m, is_sin);
    const double norm = (m == 0) ? sqrt(n + 1.0) : sqrt(2.0 * (n + 1.0));
    for (int s = 0; s <= (n - m) / 2; ++s) {
        const double cs = ((s & 1) ? -1.0 : 1.0) * fact(n - s) /
                          (fact(s) * fact((n + m) / 2 - s) * fact((n - m) / 2 - s));
        const int p = (n - m) / 2 - s;  // power of rho^2
        for (int a = 0; a <= p; ++a) {
            const double ca = binom(p, a);  // xi^(2a) eta^(2(p-a))
            for (int b = 0; b <= m; ++b) {
                // (xi + i eta)^m term: C(m,b) xi^(m-b) (i eta)^b
                const bool odd = (b & 1) != 0;
                if (odd != is_sin) continue;  // real part: even b; imaginary part: odd b
                const int quarter = is_sin ? (b - 1) / 2 : b / 2;
                const double sign = (quarter & 1) ? -1.0 : 1.0;
                const int ex = 2 * a + (m - b), ey = 2 * (p - a) + b;
                table[gbd::plate_index(ex, ey)] += coef * norm * cs * ca * binom(m, b) * sign;
                max_deg = std::max(max_deg, ex + ey);
            }
        }
    }
}

gbd_status check_system(const gbd_system* S) {
    if (!S) return fail(GBD_EINVAL, "system is NULL");
    if (!finite_pos(S->wavelength)) return fail(GBD_EINVAL, "wavelength must be finite and > 0");
    if (!(isfinite(S->distance) && S->distance >= 0.0))
        return fail(GBD_EINVAL, "distance must be finite and >= 0");
    if (S->focal_length == 0.0 || isnan(S->focal_length) || S->focal_length == -INFINITY)
        return fail(GBD_EINVAL, "focal_length must be non-zero (use +INFINITY for no lens)");
    if (S->n_zern < 0 || S->n_zern > GBD_MAX_ZERN)
        return fail(GBD_EINVAL, "n_zern must be in [0, %d]", GBD_MAX_ZERN);
    if (S->n_zern > 0 && !finite_pos(S->zern_radius))
        return fail(GBD_EINVAL, "zern_radius must be finite and > 0");
    for (int t = 0; t < S->n_zern; ++t) {
        if (S->noll[t] < 1 || S->noll[t] > GBD_MAX_NOLL)
            return fail(GBD_EINVAL, "noll[%d] = %d outside [1, %d]", t, S->noll[t], GBD_MAX_NOLL);
        if (!isfinite(S->zern_coef[t])) return fail(GBD_EINVAL, "zern_coef[%d] not finite", t);
    }
    return GBD_OK;
}

gbd_status check_pupil(const gbd_pupil* P) {
    if (!P) return fail(GBD_EINVAL, "pupil is NULL");
    if (!finite_pos(P->diameter)) return fail(GBD_EINVAL, "pupil diameter must be finite and > 0");
    if (P->n_across < 1 || P->n_across > 4096)
        return fail(GBD_EINVAL, "n_across must be in [1, 4096]");
    return GBD_OK;
}

gbd_status check_detector(const gbd_detector* D) {
    if (!D) return fail(GBD_EINVAL, "detector is NULL");
    if (D->nx < 1 || D->ny < 1 || D->nx > 16384 || D->ny > 16384)
        return fail(GBD_EINVAL, "detector size must be in [1, 16384] on each axis");
    if (!finite_pos(D->pitch_x) || !finite_pos(D->pitch_y))
        return fail(GBD_EINVAL, "pixel pitch must be finite and > 0");
    if (!(fabs(D->rot_x) < 1.2) || !(fabs(D->rot_y) < 1.2))
        return fail(GBD_EINVAL, "detector rotations must satisfy |rot| < 1.2 rad");
    return GBD_OK;
}

gbd_project_params project_params(double wavelength, const gbd_detector* D) {
    gbd_project_params p;
    const double ca = cos(D->rot_x), sa = sin(D->rot_x), cb = cos(D->rot_y), sb = sin(D->rot_y);
    // R = Ry(b) Rx(a); columns 0 and 1 map detector (s_x, s_y) into the lab frame
    p.M[0] = cb;
    p.M[1] = sb * sa;
    p.M[2] = 0.0;
    p.M[3] = ca;
    p.n[0] = -sb;
    p.n[1] = cb * sa;
    p.wavelength = wavelength;
    p.px = D->pitch_x;
    p.py = D->pitch_y;
    p.nx = D->nx;
    p.ny = D->ny;
    p.inv_wavelength = 1.0 / wavelength;
    p.inv_px = 1.0 / D->pitch_x;
    p.inv_py = 1.0 / D->pitch_y;
    p.row0 = 0;
    p.rows = D->ny;
    return p;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int n_tiles_of(int n) { return (n + gbd::kTile - 1) / gbd::kTile; }

size_t tile_bytes(int precision) {
    return precision == GBD_PREC_MIXED ? gbd::kMixedTileBytes : gbd::kF64TileBytes;
}

gbd_shape default_shape(int precision) {
    gbd_shape s;
    s.rows_per_thread = precision == GBD_PREC_MIXED ? 4 : 1;
    s.cols_per_thread = precision == GBD_PREC_MIXED ? 8 : 16;
    s.splits = 0;
    s.ms = 0.f;
    s.scheme = precision == GBD_PREC_MIXED ? GBD_SCHEME_ROW_PAIR : GBD_SCHEME_DIRECT;
    return s;
}

// Columns per thread of the default mixed shape for a detector nx pixels wide: a thread
// block covers 32 cb columns, so narrow or ragged detectors waste part of a 2 x 8 block;
// the pick minimises (columns covered / nx) x the shape's relative cost per pixel
// (measured on GB300: 2 x 8 row pairs 1, 2 x 4 about 1.2, 2 x 2 about 1.45).
int auto_cols(int nx, int min_cols = 2) {
    static const int kCols[3] = {8, 4, 2};
    static const double kCost[3] = {1.0, 1.2, 1.45};
    int best = 8;
    double best_cost = 1e300;
    for (int k = 0; k < 3 && kCols[k] >= min_cols; ++k) {
        const long span = 32L * kCols[k];
        const double cover = (double)((nx + span - 1) / span * span) / nx;
        if (cover * kCost[k] < best_cost) {
            best_cost = cover * kCost[k];
            best = kCols[k];
        }
    }
    return best;
}

// The shape set for this device and precision, else the default (for the mixed path with
// its columns per thread fitted to the detector's width: row quadruples on 8 columns, which
// run the 2 x 8 row pairs themselves for the fields they cannot take, else row pairs).
gbd_shape stored_shape(int precision, const gbd_detector* D) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_shapes.find({current_device(), precision});
        if (it != g_shapes.end()) return it->second;
    }
    gbd_shape s = default_shape(precision);
    if (precision == GBD_PREC_MIXED && D) {
        // 8 columns: the row quadruples in packed FP32x2 (airy_large 2.85 ms against 2.99
        // for the row triples); fields with a uv term fall back to the row pairs either way
        s.cols_per_thread = auto_cols(D->nx);
        s.rows_per_thread = s.cols_per_thread == 8 ? 4 : 2;
    }
    // FP64: 1 x 32 row segments on detectors 256 pixels wide or more (airy_large 335 ms
    // against 405 ms for 1 x 16; on fields with a uv term the fastest shape too); the
    // row-band shapes (8 x 4: 202 ms without a uv term, 2.6x slower with one) are left to
    // the autotuner, which sees the beamlets
    if (precision == GBD_PREC_F64 && D && D->nx >= 256) s.cols_per_thread = 32;
    return s;
}

// Beamlet splits: enough CTAs for about 16 waves of resident CTAs, so that the last,
// partly filled wave costs little (measured on GB300: 16 waves beat 4 by ~5 % on the
// 512^2-pixel, 51k-beamlet field), without splitting a beamlet range below 8 tiles.
// CTAs per beamlet split: pixel blocks of 32 cb x 8 rb (columns 32 apart), or for the FP64
// row-segment shapes (cb >= 8) 256 segments of cb x rb pixels.
long pixel_ctas(int precision, int rb, int cb, const gbd_detector* D) {
    if (precision == GBD_PREC_F64 && cb >= 8) {
        const long segs = (long)((D->nx + cb - 1) / cb) * ((D->ny + rb - 1) / rb);
        return (segs + 255) / 256;
    }
    return (long)((D->nx + 32 * cb - 1) / (32 * cb)) * ((D->ny + 8 * rb - 1) / (8 * rb));
}

// Resident CTAs per SM of a field kernel shape, queried once per device and shape.
int cached_occupancy(int precision, int rb, int cb, int scheme) {
    static std::map<std::array<int, 5>, int> cache;
    const std::array<int, 5> key = {current_device(), precision, rb, cb, scheme};
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    const int occ = std::max(1, gbd_field_occupancy(precision, rb, cb, scheme));
    std::lock_guard<std::mutex> lk(g_mu);
    cache[key] = occ;
    return occ;
}

int heuristic_splits(int precision, int rb, int cb, int scheme, int n_tiles,
                     const gbd_detector* D) {
    const long pix_ctas = pixel_ctas(precision, rb, cb, D);
    const int occ = cached_occupancy(precision, rb, cb, scheme);
    const long slots = (long)occ * sm_count();
    long s = (16 * slots + pix_ctas - 1) / pix_ctas;
    s = std::min<long>(s, std::max(1, n_tiles / 8));
    s = std::max<long>(1, std::min<long>(s, 64));
    const int tps = (n_tiles + (int)s - 1) / (int)s;
    return (n_tiles + tps - 1) / tps;
}

gbd_field_launch resolve_launch(int precision, const gbd_shape& sh, int n_tiles,
                                const gbd_detector* D) {
    gbd_field_launch L;
    L.rows_per_thread = sh.rows_per_thread;
    L.cols_per_thread = sh.cols_per_thread;
    L.scheme = sh.scheme;
    int s = sh.splits > 0 ? std::min(sh.splits, n_tiles)
                          : heuristic_splits(precision, sh.rows_per_thread, sh.cols_per_thread,
                                             sh.scheme, n_tiles, D);
    s = std::max(1, s);
    L.tiles_per_split = (n_tiles + s - 1) / s;
    L.splits = (n_tiles + L.tiles_per_split - 1) / L.tiles_per_split;
    return L;
}

// Workspace: [flag word | projected records | split partial fields], 256-byte aligned parts.
constexpr size_t kFlagBytes = 256;

// First row of the slab the kernels evaluate for output rows [row_begin, row_end): row_begin
// rounded down to the launch's row-block height, so that every pixel is computed by the
// same thread row block (and the same recurrence chain) as on the whole detector.
int slab_row0(int precision, const gbd_field_launch& L, int row_begin) {
    const int h = gbd_field_row_block(precision, L);
    return row_begin - row_begin % h;
}

// Completion counters of the multi-row kernel's pixel blocks (32 CB x 8 RB pixels; sized
// for the smallest block, 32 x 8, and one more block row: a slab may start inside its
// first block).
size_t counter_bytes(int nx, int rows) {
    return align256((size_t)((nx + 31) / 32) * ((rows + 7) / 8 + 1) * sizeof(unsigned));
}

size_t workspace_for(int precision, int n, const gbd_detector* D, const gbd_field_launch& L,
                     int row_begin = 0, int row_end = -1) {
    if (n <= 0) return 0;
    if (row_end < 0) row_end = D->ny;
    const int rows = row_end - slab_row0(precision, L, row_begin);
    const size_t coeff = align256((size_t)n_tiles_of(n) * tile_bytes(precision));
    const size_t elem = precision == GBD_PREC_MIXED ? sizeof(float2) : sizeof(double2);
    const size_t part = align256((size_t)L.splits * D->nx * rows * elem);
    return kFlagBytes + counter_bytes(D->nx, rows) + coeff + part;
}

// The field on detector rows [row_begin, row_end) (the whole detector: 0, ny).  The launch
// (shape, splits) and the projection's flags are those of the whole detector, so a row
// range gives the same bits as the same rows of the whole field.
gbd_status run_field(const gbd_beamlet* beamlets, int32_t n, double wavelength,
                     const gbd_detector* D, int32_t precision, void* ws, size_t ws_bytes, void* out,
                     cudaStream_t stream, const gbd_shape& sh, int row_begin = 0,
                     int row_end = -1) {
    if (row_end < 0) row_end = D->ny;
    gbd_project_params pp = project_params(wavelength, D);
    const size_t npix = (size_t)D->nx * (row_end - row_begin);
    if (n == 0 || npix == 0) {
        const size_t elem = precision == GBD_PREC_F64 ? 16 : 8;
        cudaError_t e = npix ? cudaMemsetAsync(out, 0, npix * elem, stream) : cudaSuccess;
        return e == cudaSuccess ? GBD_OK : cuda_fail(e, "gbd_field memset");
    }
    const int nt = n_tiles_of(n);
    const gbd_field_launch L = resolve_launch(precision, sh, nt, D);
    pp.row0 = slab_row0(precision, L, row_begin);
    pp.rows = row_end - pp.row0;
    const size_t need = workspace_for(precision, n, D, L, row_begin, row_end);
    if (ws_bytes < need)
        return fail(GBD_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes,
                    need);
    // [flag word | pixel-block counters | projected records | split partials]
    char* base = static_cast<char*>(ws);
    unsigned* wide = reinterpret_cast<unsigned*>(base);
    const size_t cnt = counter_bytes(D->nx, pp.rows);
    unsigned* done = reinterpret_cast<unsigned*>(base + kFlagBytes);
    void* coeffs = base + kFlagBytes + cnt;
    void* partial = base + kFlagBytes + cnt + align256((size_t)nt * tile_bytes(precision));
    cudaError_t e = cudaMemsetAsync(wide, 0, kFlagBytes + cnt, stream);
    if (e != cudaSuccess) return cuda_fail(e, "gbd_field flag reset");
    const gbd::ReduceOut ro = gbd_reduce_out(pp, out, done, row_begin, row_end - row_begin);
    {
        TimingScope ts(kTimeProject, stream);
        e = gbd_launch_project(beamlets, n, pp, precision, coeffs, wide, stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gbd_field projection launch");
    {
        TimingScope ts(precision == GBD_PREC_MIXED ? kTimeMixed : kTimeF64, stream);
        e = gbd_launch_field_kernel(precision, coeffs, nt, pp, L, partial, wide, wait_spins(),
                                    ro, stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gbd_field launch");
    {
        TimingScope ts(kTimeReduce, stream);
        e = gbd_launch_field_reduce(precision, pp, L, wide, partial, ro, stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gbd_field reduce launch");
    return GBD_OK;
}

gbd_status check_field_args(const gbd_beamlet* beamlets, int32_t n, double wavelength,
                            const gbd_detector* D, int32_t precision, void* ws, void* out) {
    gbd_status st = check_detector(D);
    if (st != GBD_OK) return st;
    if (precision != GBD_PREC_F64 && precision != GBD_PREC_MIXED)
        return fail(GBD_EINVAL, "precision must be GBD_PREC_F64 or GBD_PREC_MIXED");
    if (!finite_pos(wavelength)) return fail(GBD_EINVAL, "wavelength must be finite and > 0");
    if (n < 0) return fail(GBD_EINVAL, "n_beamlets must be >= 0");
    if (!out) return fail(GBD_EINVAL, "field_out is NULL");
    if (n > 0 && (!beamlets || !ws)) return fail(GBD_EINVAL, "beamlets/workspace is NULL");
    if (n > 0 && (reinterpret_cast<uintptr_t>(ws) & 255u))
        return fail(GBD_EINVAL, "workspace must be 256-byte aligned");
    if ((reinterpret_cast<uintptr_t>(out) & 15u) != 0)
        return fail(GBD_EINVAL, "field_out must be 16-byte aligned");
    return GBD_OK;
}

}  // namespace

gbd_status gbd_set_error(gbd_status st, const char* msg) { return fail(st, "%s", msg); }

gbd_status gbd_check_system(const gbd_system* s) { return check_system(s); }
gbd_status gbd_check_detector(const gbd_detector* d) { return check_detector(d); }
gbd_project_params gbd_make_project_params(double wavelength, const gbd_detector* d) {
    return project_params(wavelength, d);
}
int gbd_sm_count() { return sm_count(); }
int gbd_auto_cols(int nx, int min_cols) { return auto_cols(nx, min_cols); }
uint32_t gbd_wait_spins() { return wait_spins(); }

// Kernel parameters of the shared optics of a trace (the pupil sampling is set by the
// caller): lens, distance and the Zernike plate expanded into monomials of x/R, y/R.
gbd_trace_params gbd_make_trace_params(const gbd_system* system, double diameter) {
    gbd_trace_params p;
    memset(&p, 0, sizeof(p));
    p.wavelength = system->wavelength;
    p.inv_f = isinf(system->focal_length) ? 0.0 : 1.0 / system->focal_length;
    p.d = system->distance;
    p.zern_radius = system->n_zern > 0 ? system->zern_radius : 1.0;
    p.diameter = diameter;
    int deg = -1;
    for (int t = 0; t < system->n_zern; ++t)
        add_zernike(system->noll[t], system->zern_coef[t], p.zpoly, deg);
    p.zdeg = system->n_zern > 0 ? deg : -1;
    return p;
}

// gbd_field on a fixed scratch buffer of known size: the beamlet splits are lowered until
// the projected records and the split partial fields fit; sizes that do not fit even
// with one split are rejected before anything is launched.
gbd_status gbd_field_fixed_scratch(const gbd_beamlet* beamlets, int32_t n, double wavelength,
                                   const gbd_detector* detector, int32_t precision,
                                   void* scratch, size_t scratch_bytes, void* out,
                                   cudaStream_t stream) {
    GBD_NVTX_RANGE("gbd_field_fixed_scratch");
    gbd_status st = check_field_args(beamlets, n, wavelength, detector, precision, scratch, out);
    if (st != GBD_OK) return st;
    gbd_shape sh = stored_shape(precision, detector);
    if (n > 0) {
        const int nt = n_tiles_of(n);
        gbd_field_launch L = resolve_launch(precision, sh, nt, detector);
        sh.splits = L.splits;
        while (sh.splits > 1 && workspace_for(precision, n, detector, L) > scratch_bytes) {
            --sh.splits;
            L = resolve_launch(precision, sh, nt, detector);
        }
        const size_t need = workspace_for(precision, n, detector, L);
        if (need > scratch_bytes)
            return fail(GBD_EINVAL,
                        "problem needs %zu bytes of scratch (beamlet records + one partial field "
                        "of %d x %d pixels), more than the fixed %zu bytes",
                        need, detector->nx, detector->ny, scratch_bytes);
    }
    return run_field(beamlets, n, wavelength, detector, precision, scratch, scratch_bytes, out,
                     stream, sh);
}

// The truncated decomposition's grid classes in half-pitch units (a = 2i - (N-1),
// b = 2j - (N-1); R = N, w0 = OF): kept when a^2 + b^2 <= outer = (N + margin OF)^2,
// interior when a^2 + b^2 < inner = (N - margin OF)^2.
struct TruncatedGrid {
    int ext;
    double inner, outer;
    int32_t total, edge;
};

gbd_status truncated_grid(const gbd_pupil* pupil, double overlap_factor, double margin,
                          TruncatedGrid* g) {
    gbd_status st = check_pupil(pupil);
    if (st != GBD_OK) return st;
    if (!finite_pos(overlap_factor)) return fail(GBD_EINVAL, "overlap_factor must be > 0");
    if (!(margin >= 0.0 && margin <= 10.0)) return fail(GBD_EINVAL, "margin must be in [0, 10]");
    const int N = pupil->n_across;
    const double mo = margin * overlap_factor;
    const double ro = N + mo, ri = N - mo;
    g->outer = ro * ro;
    g->inner = ri > 0.0 ? ri * ri : -1.0;
    g->ext = (int)ceil(0.5 * mo) + 1;
    long long total = 0, edge = 0;
    for (int j = -g->ext; j < N + g->ext; ++j)
        for (int i = -g->ext; i < N + g->ext; ++i) {
            const double a = 2.0 * i - (N - 1), b = 2.0 * j - (N - 1);
            const double q = a * a + b * b;
            if (q > g->outer) continue;
            ++total;
            edge += !(q < g->inner);
        }
    if (total > INT32_MAX) return fail(GBD_EINVAL, "too many beamlets");
    g->total = (int32_t)total;
    g->edge = (int32_t)edge;
    return GBD_OK;
}

// Kernel parameters of a mirror sequence (lab-frame vertices and curvatures, the pupil
// plane and the axial path); the pupil sampling is set by the caller.
gbd_status gbd_make_mirror_params(const gbd_mirror_system* system, double diameter,
                                  gbd_mirror_params* out) {
    if (!system) return fail(GBD_EINVAL, "system is NULL");
    if (!finite_pos(system->wavelength)) return fail(GBD_EINVAL, "wavelength must be finite and > 0");
    if (!finite_pos(system->pupil_offset)) return fail(GBD_EINVAL, "pupil_offset must be > 0");
    const int n = system->n_mirrors;
    if (n < 1 || n > GBD_MAX_MIRRORS)
        return fail(GBD_EINVAL, "n_mirrors must be in [1, %d]", GBD_MAX_MIRRORS);
    for (int k = 0; k < n; ++k)
        if (!isfinite(system->radius[k]) || system->radius[k] == 0.0 ||
            !isfinite(system->spacing[k]) || system->spacing[k] == 0.0 ||
            !isfinite(system->conic[k]))
            return fail(GBD_EINVAL, "mirror %d: radius and spacing must be finite and non-zero", k);
    gbd_mirror_params& m = *out;
    memset(&m, 0, sizeof(m));
    m.n = n;
    double z = 0.0, dir = 1.0, axial = system->pupil_offset;
    for (int k = 0; k < n; ++k) {
        m.z[k] = z;
        m.c[k] = dir / system->radius[k];
        m.K[k] = system->conic[k];
        z += system->spacing[k];
        axial += fabs(system->spacing[k]);
        dir = -dir;
    }
    m.z_img = z;
    m.z_ep = -system->pupil_offset;
    m.axial_path = axial;
    m.wavelength = system->wavelength;
    m.diameter = diameter;
    return GBD_OK;
}

extern "C" {

const char* gbd_last_error(void) { return g_err; }

const char* gbd_version(void) { return "gbd-gb300 0.1 (sm_103a)"; }

int32_t gbd_beamlet_count(const gbd_pupil* pupil) {
    if (check_pupil(pupil) != GBD_OK) return -1;
    const long long N = pupil->n_across;
    long long count = 0;
    for (long long j = 0; j < N; ++j) {
        const long long b = 2 * j - (N - 1);
        const long long r2 = N * N - b * b;
        // the values a = 2i - (N-1), i = 0 .. N-1, with a^2 <= r2, i.e. |a| <= m = isqrt(r2):
        // i from ceil((N-1-m)/2) to floor((N-1+m)/2), within [0, N-1]
        long long m = (long long)sqrt((double)r2);
        while (m * m > r2) --m;
        while ((m + 1) * (m + 1) <= r2) ++m;
        const long long lo = N - 1 - m <= 0 ? 0 : (N - m) / 2;
        const long long hi = std::min(N - 1, (N - 1 + m) / 2);
        if (hi >= lo) count += hi - lo + 1;
    }
    return (int32_t)count;
}

gbd_status gbd_sync(void* stream) {
    // the four translation units' status words are copied into pinned host memory behind
    // the stream's work, so one synchronisation covers the work and the status
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    thread_local unsigned* h = nullptr;
    if (!h && cudaMallocHost(reinterpret_cast<void**>(&h), 4 * sizeof(unsigned)) != cudaSuccess) {
        h = nullptr;
        return cuda_fail(cudaGetLastError(), "gbd_sync status buffer");
    }
    cudaError_t e = gbd_field_status_fetch(h, s);
    if (e == cudaSuccess) e = gbd_sweep_status_fetch(h + 1, s);
    if (e == cudaSuccess) e = gbd_point_status_fetch(h + 2, s);
    if (e == cudaSuccess) e = gbd_mlp_status_fetch(h + 3, s);
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) return cuda_fail(e, "gbd_sync");
    if (h[0]) gbd_field_status_clear();
    if (h[1]) gbd_sweep_status_clear();
    if (h[2]) gbd_point_status_clear();
    if (h[3]) gbd_mlp_status_clear();
    if ((h[0] | h[1] | h[2] | h[3]) & gbd::kStatusTimeout)
        return fail(GBD_ETIMEOUT, "a device wait gave up (timeout)");
    return GBD_OK;
}

gbd_status gbd_set_wait_limit(uint32_t spins) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_wait_spins[current_device()] = spins == 0 ? gbd::kDefaultWaitSpins : spins;
    return GBD_OK;
}

gbd_status gbd_trace(const gbd_system* system, const gbd_pupil* pupil, double overlap_factor,
                     double waist_ratio, gbd_beamlet* out, int32_t capacity, void* stream) {
    GBD_NVTX_RANGE("gbd_trace");
    gbd_status st = check_system(system);
    if (st != GBD_OK) return st;
    if ((st = check_pupil(pupil)) != GBD_OK) return st;
    if (!finite_pos(overlap_factor)) return fail(GBD_EINVAL, "overlap_factor must be > 0");
    if (!finite_pos(waist_ratio)) return fail(GBD_EINVAL, "waist_ratio must be > 0");
    const int32_t n = gbd_beamlet_count(pupil);
    if (capacity < n) return fail(GBD_ENOMEM, "capacity %d < %d beamlets", capacity, n);
    if (n > 0 && !out) return fail(GBD_EINVAL, "out is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 15u) return fail(GBD_EINVAL, "out must be 16-byte aligned");
    gbd_trace_params p = gbd_make_trace_params(system, pupil->diameter);
    p.overlap_factor = overlap_factor;
    p.waist_ratio = waist_ratio;
    p.n_across = pupil->n_across;
    p.grid = gbd_make_grid(pupil->diameter, system->wavelength, pupil->n_across, overlap_factor,
                           waist_ratio);
    cudaError_t e;
    {
        TimingScope ts(kTimeTrace, static_cast<cudaStream_t>(stream));
        e = gbd_launch_trace(p, 1, pupil->n_across, nullptr, out, static_cast<cudaStream_t>(stream));
    }
    if (e != cudaSuccess) return cuda_fail(e, "gbd_trace launch");
    return GBD_OK;
}

gbd_status gbd_trace_mirrors(const gbd_mirror_system* system, const gbd_pupil* pupil,
                             double overlap_factor, double waist_ratio, gbd_beamlet* out,
                             int32_t capacity, void* stream) {
    GBD_NVTX_RANGE("gbd_trace_mirrors");
    if (!system) return fail(GBD_EINVAL, "system is NULL");
    gbd_status st = check_pupil(pupil);
    if (st != GBD_OK) return st;
    gbd_mirror_params m;
    if ((st = gbd_make_mirror_params(system, pupil->diameter, &m)) != GBD_OK) return st;
    if (!finite_pos(overlap_factor)) return fail(GBD_EINVAL, "overlap_factor must be > 0");
    if (!finite_pos(waist_ratio)) return fail(GBD_EINVAL, "waist_ratio must be > 0");
    const int32_t nb = gbd_beamlet_count(pupil);
    if (capacity < nb) return fail(GBD_ENOMEM, "capacity %d < %d beamlets", capacity, nb);
    if (nb > 0 && !out) return fail(GBD_EINVAL, "out is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 15u) return fail(GBD_EINVAL, "out must be 16-byte aligned");
    m.n_across = pupil->n_across;
    m.overlap_factor = overlap_factor;
    m.waist_ratio = waist_ratio;
    m.grid = gbd_make_grid(pupil->diameter, system->wavelength, pupil->n_across, overlap_factor,
                           waist_ratio);
    cudaError_t e;
    {
        TimingScope ts(kTimeTrace, static_cast<cudaStream_t>(stream));
        e = gbd_launch_trace_mirrors(m, out, static_cast<cudaStream_t>(stream));
    }
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "gbd_trace_mirrors launch");
}

size_t gbd_project_bytes(int32_t n_beamlets, int32_t precision) {
    if (n_beamlets <= 0) return 0;
    return (size_t)n_tiles_of(n_beamlets) *
           (precision == GBD_PREC_MIXED ? gbd::kMixedTileBytes : gbd::kF64TileBytes);
}

gbd_status gbd_project(const gbd_beamlet* beamlets, int32_t n_beamlets, double wavelength,
                       const gbd_detector* detector, int32_t precision, void* coeffs,
                       uint32_t* wide_flag, void* stream) {
    GBD_NVTX_RANGE("gbd_project");
    gbd_status st = check_field_args(beamlets, n_beamlets, wavelength, detector, precision,
                                     coeffs, coeffs ? coeffs : (void*)16);
    if (st != GBD_OK) return st;
    if (n_beamlets == 0) return GBD_OK;
    cudaError_t e = gbd_launch_project(beamlets, n_beamlets, project_params(wavelength, detector),
                                       precision, coeffs, wide_flag, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "gbd_project launch");
}

size_t gbd_field_workspace_bytes(int32_t n_beamlets, const gbd_detector* detector,
                                 int32_t precision) {
    if (check_detector(detector) != GBD_OK || n_beamlets <= 0) return 0;
    if (precision != GBD_PREC_F64 && precision != GBD_PREC_MIXED) return 0;
    const gbd_field_launch L =
        resolve_launch(precision, stored_shape(precision, detector), n_tiles_of(n_beamlets),
                       detector);
    return workspace_for(precision, n_beamlets, detector, L);
}

gbd_status gbd_field(const gbd_beamlet* beamlets, int32_t n_beamlets, double wavelength,
                     const gbd_detector* detector, int32_t precision, void* workspace,
                     size_t workspace_bytes, void* field_out, void* stream) {
    GBD_NVTX_RANGE("gbd_field");
    gbd_status st = check_field_args(beamlets, n_beamlets, wavelength, detector, precision,
                                     workspace, field_out);
    if (st != GBD_OK) return st;
    return run_field(beamlets, n_beamlets, wavelength, detector, precision, workspace,
                     workspace_bytes, field_out, static_cast<cudaStream_t>(stream),
                     stored_shape(precision, detector));
}

size_t gbd_field_rows_workspace_bytes(int32_t n_beamlets, const gbd_detector* detector,
                                      int32_t row_begin, int32_t row_end, int32_t precision) {
    if (check_detector(detector) != GBD_OK || n_beamlets <= 0) return 0;
    if (precision != GBD_PREC_F64 && precision != GBD_PREC_MIXED) return 0;
    if (row_begin < 0 || row_end > detector->ny || row_begin >= row_end) return 0;
    const gbd_field_launch L =
        resolve_launch(precision, stored_shape(precision, detector), n_tiles_of(n_beamlets),
                       detector);
    return workspace_for(precision, n_beamlets, detector, L, row_begin, row_end);
}

gbd_status gbd_field_rows(const gbd_beamlet* beamlets, int32_t n_beamlets, double wavelength,
                          const gbd_detector* detector, int32_t row_begin, int32_t row_end,
                          int32_t precision, void* workspace, size_t workspace_bytes,
                          void* field_out, void* stream) {
    GBD_NVTX_RANGE("gbd_field_rows");
    // an empty range writes nothing, so its output pointer may be NULL
    gbd_status st = check_field_args(beamlets, n_beamlets, wavelength, detector, precision,
                                     workspace,
                                     row_begin == row_end && !field_out ? (void*)16 : field_out);
    if (st != GBD_OK) return st;
    if (row_begin < 0 || row_end > detector->ny || row_begin > row_end)
        return fail(GBD_EINVAL, "row range [%d, %d) is not inside [0, %d)", row_begin, row_end,
                    detector->ny);
    return run_field(beamlets, n_beamlets, wavelength, detector, precision, workspace,
                     workspace_bytes, field_out, static_cast<cudaStream_t>(stream),
                     stored_shape(precision, detector), row_begin, row_end);
}

int32_t gbd_truncated_count(const gbd_pupil* pupil, double overlap_factor, double margin,
                            int32_t* n_edge) {
    TruncatedGrid g;
    if (truncated_grid(pupil, overlap_factor, margin, &g) != GBD_OK) return -1;
    if (n_edge) *n_edge = g.edge;
    return g.total;
}

gbd_status gbd_trace_truncated(const gbd_system* system, const gbd_pupil* pupil,
                               double overlap_factor, double waist_ratio, double margin,
                               gbd_beamlet* out, int32_t capacity, int32_t* n_edge,
                               void* stream) {
    GBD_NVTX_RANGE("gbd_trace_truncated");
    gbd_status st = check_system(system);
    if (st != GBD_OK) return st;
    TruncatedGrid g;
    if ((st = truncated_grid(pupil, overlap_factor, margin, &g)) != GBD_OK) return st;
    if (!finite_pos(waist_ratio)) return fail(GBD_EINVAL, "waist_ratio must be > 0");
    if (capacity < g.total) return fail(GBD_ENOMEM, "capacity %d < %d beamlets", capacity, g.total);
    if (g.total > 0 && !out) return fail(GBD_EINVAL, "out is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 15u) return fail(GBD_EINVAL, "out must be 16-byte aligned");
    if (n_edge) *n_edge = g.edge;
    gbd_trace_params p = gbd_make_trace_params(system, pupil->diameter);
    p.overlap_factor = overlap_factor;
    p.waist_ratio = waist_ratio;
    p.n_across = pupil->n_across;
    p.grid = gbd_make_grid(pupil->diameter, system->wavelength, pupil->n_across, overlap_factor,
                           waist_ratio);
    cudaError_t e;
    {
        TimingScope ts(kTimeTrace, static_cast<cudaStream_t>(stream));
        e = gbd_launch_trace_truncated(p, g.ext, g.inner, g.outer, g.total - g.edge, out,
                                       static_cast<cudaStream_t>(stream));
    }
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "gbd_trace_truncated launch");
}

size_t gbd_field_truncated_workspace_bytes(int32_t n_beamlets, int32_t n_edge,
                                           const gbd_detector* detector, int32_t precision) {
    if (check_detector(detector) != GBD_OK || n_beamlets < 0 || n_edge < 0 || n_edge > n_beamlets)
        return 0;
    if (precision != GBD_PREC_F64 && precision != GBD_PREC_MIXED) return 0;
    const size_t edge = align256((size_t)n_edge * gbd::kEdgeFields * sizeof(double2));
    // after the whole beamlets' field, its scratch holds the edge splits' partial fields
    return edge + std::max(gbd_field_workspace_bytes(n_beamlets - n_edge, detector, precision),
                           gbd_field_edge_partial_bytes(precision, n_edge, detector->nx,
                                                        detector->ny));
}

gbd_status gbd_field_truncated(const gbd_beamlet* beamlets, int32_t n_beamlets, int32_t n_edge,
                               double wavelength, const gbd_detector* detector, int32_t precision,
                               void* workspace, size_t workspace_bytes, void* field_out,
                               void* stream) {
    GBD_NVTX_RANGE("gbd_field_truncated");
    gbd_status st = check_field_args(beamlets, n_beamlets, wavelength, detector, precision,
                                     workspace, field_out);
    if (st != GBD_OK) return st;
    if (n_edge < 0 || n_edge > n_beamlets)
        return fail(GBD_EINVAL, "n_edge must be in [0, n_beamlets]");
    if (detector->rot_x != 0.0 || detector->rot_y != 0.0)
        return fail(GBD_EUNSUPPORTED, "truncated beamlets are evaluated on untilted planes");
    const size_t edge = align256((size_t)n_edge * gbd::kEdgeFields * sizeof(double2));
    if (workspace_bytes < edge + gbd_field_edge_partial_bytes(precision, n_edge, detector->nx,
                                                             detector->ny))
        return fail(GBD_ENOMEM, "workspace too small for the edge records and partial fields");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(workspace);
    st = run_field(beamlets, n_beamlets - n_edge, wavelength, detector, precision, base + edge,
                   workspace_bytes - edge, field_out, s, stored_shape(precision, detector));
    if (st != GBD_OK || n_edge == 0) return st;
    const gbd_project_params pp = project_params(wavelength, detector);
    double2* rec = reinterpret_cast<double2*>(base);
    cudaError_t e = gbd_launch_project_edge(beamlets + (n_beamlets - n_edge), n_edge, pp, rec, s);
    if (e == cudaSuccess)
        e = gbd_launch_field_edge(precision, rec, n_edge, detector->nx, detector->ny, field_out,
                                  base + edge, s);
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "gbd_field_truncated launch");
}

gbd_status gbd_field_set_shape(int32_t precision, const gbd_shape* shape) {
    if (precision != GBD_PREC_F64 && precision != GBD_PREC_MIXED)
        return fail(GBD_EINVAL, "precision must be GBD_PREC_F64 or GBD_PREC_MIXED");
    if (!shape) {  // back to the default (fitted to each detector)
        std::lock_guard<std::mutex> lk(g_mu);
        g_shapes.erase({current_device(), precision});
        return GBD_OK;
    }
    gbd_shape s = *shape;
    if (!gbd_field_shape_supported(precision, s.rows_per_thread, s.cols_per_thread, s.scheme))
        return fail(GBD_EINVAL, "unsupported shape %dx%d (scheme %d)", s.rows_per_thread,
                    s.cols_per_thread, s.scheme);
    if (s.splits < 0 || s.splits > 1024) return fail(GBD_EINVAL, "splits must be in [0, 1024]");
    std::lock_guard<std::mutex> lk(g_mu);
    g_shapes[{current_device(), precision}] = s;
    return GBD_OK;
}

gbd_status gbd_field_get_shape(int32_t precision, int32_t n_beamlets, const gbd_detector* detector,
                               gbd_shape* out) {
    if (!out) return fail(GBD_EINVAL, "out is NULL");
    gbd_status st = check_detector(detector);
    if (st != GBD_OK) return st;
    if (precision != GBD_PREC_F64 && precision != GBD_PREC_MIXED)
        return fail(GBD_EINVAL, "precision must be GBD_PREC_F64 or GBD_PREC_MIXED");
    gbd_shape s = stored_shape(precision, detector);
    if (n_beamlets > 0) {
        gbd_field_launch L = resolve_launch(precision, s, n_tiles_of(n_beamlets), detector);
        s.splits = L.splits;
    }
    *out = s;
    return GBD_OK;
}

gbd_status gbd_autotune_field(const gbd_beamlet* beamlets, int32_t n_beamlets, double wavelength,
                              const gbd_detector* detector, int32_t precision, void* workspace,
                              size_t workspace_bytes, void* field_out, void* stream,
                              gbd_shape* best) {
    GBD_NVTX_RANGE("gbd_autotune_field");
    gbd_status st = check_field_args(beamlets, n_beamlets, wavelength, detector, precision,
                                     workspace, field_out);
    if (st != GBD_OK) return st;
    if (n_beamlets == 0) return fail(GBD_EINVAL, "autotune needs at least one beamlet");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    static const int kMixed[][3] = {{1, 4, GBD_SCHEME_DIRECT},   {2, 2, GBD_SCHEME_DIRECT},
                                    {2, 4, GBD_SCHEME_DIRECT},   {4, 2, GBD_SCHEME_DIRECT},
                                    {2, 2, GBD_SCHEME_ROW_PAIR}, {2, 4, GBD_SCHEME_ROW_PAIR},
                                    {2, 8, GBD_SCHEME_ROW_PAIR}, {3, 8, GBD_SCHEME_ROW_PAIR},
                                    {4, 8, GBD_SCHEME_ROW_PAIR}, {4, 4, GBD_SCHEME_ROW_PAIR}};
    static const int kF64[][3] = {{1, 2, 0}, {2, 2, 0}, {1, 8, 0},  {2, 8, 0},
                                  {1, 16, 0}, {1, 32, 0}, {4, 8, 0}, {2, 16, 0}, {8, 4, 0}};
    std::vector<std::array<int, 3>> shapes;
    if (precision == GBD_PREC_MIXED)
        for (auto& v : kMixed) shapes.push_back({v[0], v[1], v[2]});
    else
        for (auto& v : kF64) shapes.push_back({v[0], v[1], v[2]});
    const int nt = n_tiles_of(n_beamlets);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "autotune events");
    gbd_shape win{0, 0, 0, 1e30f, 0};
    for (auto& rc : shapes) {
        gbd_shape cand{rc[0], rc[1], 0, 0.f, rc[2]};
        const int base = resolve_launch(precision, cand, nt, detector).splits;
        std::vector<int> splits = {std::max(1, base / 2), base, std::min(nt, base * 3 / 2),
                                   std::min(nt, base * 2), std::min(nt, base * 5 / 2)};
        std::sort(splits.begin(), splits.end());
        splits.erase(std::unique(splits.begin(), splits.end()), splits.end());
        for (int sp : splits) {
            cand.splits = sp;
            const gbd_field_launch L = resolve_launch(precision, cand, nt, detector);
            if (workspace_for(precision, n_beamlets, detector, L) > workspace_bytes) continue;
            float best_ms = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                st = run_field(beamlets, n_beamlets, wavelength, detector, precision, workspace,
                               workspace_bytes, field_out, s, cand);
                cudaEventRecord(e1, s);
                if (st != GBD_OK) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) best_ms = std::min(best_ms, ms);
            }
            if (st != GBD_OK) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st;
            }
            if (best_ms < win.ms) {
                win = cand;
                win.ms = best_ms;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (win.rows_per_thread == 0) return fail(GBD_ENOMEM, "no candidate shape fits the workspace");
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_shapes[{current_device(), precision}] = win;
    }
    if (best) *best = win;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "autotune");
}

gbd_status gbd_timing_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_timing = on != 0;
    return GBD_OK;
}

gbd_status gbd_timing_read(double* total_ms, int64_t* launches) {
    if (!total_ms || !launches) return fail(GBD_EINVAL, "outputs are NULL");
    std::vector<TimedLaunch> v;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        v.swap(g_timed);
    }
    for (int k = 0; k < kTimeKinds; ++k) {
        total_ms[k] = 0.0;
        launches[k] = 0;
    }
    cudaError_t err = cudaSuccess;
    for (auto& t : v) {
        cudaError_t e = cudaEventSynchronize(t.b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
        if (e == cudaSuccess) {
            total_ms[t.kind] += ms;
            launches[t.kind] += 1;
        } else {
            err = e;
        }
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    return err == cudaSuccess ? GBD_OK : cuda_fail(err, "gbd_timing_read");
}

size_t gbd_psf_workspace_bytes(const gbd_pupil* pupil, const gbd_detector* detector,
                               int32_t precision) {
    if (check_pupil(pupil) != GBD_OK || check_detector(detector) != GBD_OK) return 0;
    if (precision != GBD_PREC_F64 && precision != GBD_PREC_MIXED) return 0;
    const int32_t n = gbd_beamlet_count(pupil);
    const size_t elem = precision == GBD_PREC_F64 ? 16 : 8;
    return align256((size_t)std::max(n, 1) * sizeof(gbd_beamlet)) +
           align256((size_t)detector->nx * detector->ny * elem) +
           gbd_field_workspace_bytes(n, detector, precision);
}

gbd_status gbd_psf(const gbd_system* system, const gbd_pupil* pupil, double overlap_factor,
                   double waist_ratio, const gbd_detector* detector, int32_t precision,
                   void* workspace, size_t workspace_bytes, void* host_field_out, void* stream) {
    GBD_NVTX_RANGE("gbd_psf");
    gbd_status st = check_detector(detector);
    if (st != GBD_OK) return st;
    if ((st = check_pupil(pupil)) != GBD_OK) return st;
    if (precision != GBD_PREC_F64 && precision != GBD_PREC_MIXED)
        return fail(GBD_EINVAL, "precision must be GBD_PREC_F64 or GBD_PREC_MIXED");
    if (!host_field_out || !workspace) return fail(GBD_EINVAL, "NULL buffer");
    if (reinterpret_cast<uintptr_t>(workspace) & 255u)
        return fail(GBD_EINVAL, "workspace must be 256-byte aligned");
    const size_t need = gbd_psf_workspace_bytes(pupil, detector, precision);
    if (workspace_bytes < need)
        return fail(GBD_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed",
                    workspace_bytes, need);
    const int32_t n = gbd_beamlet_count(pupil);
    const size_t elem = precision == GBD_PREC_F64 ? 16 : 8;
    const size_t field_bytes = (size_t)detector->nx * detector->ny * elem;
    char* base = static_cast<char*>(workspace);
    gbd_beamlet* beamlets = reinterpret_cast<gbd_beamlet*>(base);
    char* dfield = base + align256((size_t)std::max(n, 1) * sizeof(gbd_beamlet));
    char* fws = dfield + align256(field_bytes);
    st = gbd_trace(system, pupil, overlap_factor, waist_ratio, beamlets, n, stream);
    if (st != GBD_OK) return st;
    st = gbd_field(beamlets, n, system->wavelength, detector, precision, fws,
                   workspace_bytes - (size_t)(fws - base), dfield, stream);
    if (st != GBD_OK) return st;
    cudaError_t e = cudaMemcpyAsync(host_field_out, dfield, field_bytes, cudaMemcpyDeviceToHost,
                                    static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "gbd_psf copy to host");
}

// Point evaluation: workspace [packed beamlet tiles | split partial fields].
static int point_splits(int n_tiles, const gbd_detector* D) {
    const long pix = gbd_point_pixel_ctas(D->nx, D->ny);
    const long slots = (long)gbd_point_occupancy() * sm_count();
    long s = (16 * slots + pix - 1) / pix;
    s = std::min<long>(s, std::max(1, n_tiles / 4));
    s = std::max<long>(1, std::min<long>(s, 64));
    const int tps = (n_tiles + (int)s - 1) / (int)s;
    return (n_tiles + tps - 1) / tps;
}

size_t gbd_field_point_workspace_bytes(int32_t n_beamlets, const gbd_detector* detector) {
    if (check_detector(detector) != GBD_OK || n_beamlets <= 0) return 0;
    const int nt = n_tiles_of(n_beamlets);
    const int sp = point_splits(nt, detector);
    return align256((size_t)nt * gbd::kF64TileBytes) +
           align256((size_t)sp * detector->nx * detector->ny * sizeof(double2));
}

gbd_status gbd_field_point(const gbd_beamlet* beamlets, int32_t n_beamlets, double wavelength,
                           const gbd_detector* detector, void* workspace, size_t workspace_bytes,
                           void* field_out, void* stream) {
    GBD_NVTX_RANGE("gbd_field_point");
    gbd_status st = check_field_args(beamlets, n_beamlets, wavelength, detector, GBD_PREC_F64,
                                     workspace, field_out);
    if (st != GBD_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const gbd_project_params pp = project_params(wavelength, detector);
    if (n_beamlets == 0) {
        cudaError_t e = cudaMemsetAsync(field_out, 0, (size_t)detector->nx * detector->ny * 16, s);
        return e == cudaSuccess ? GBD_OK : cuda_fail(e, "gbd_field_point memset");
    }
    const int nt = n_tiles_of(n_beamlets);
    const int sp = point_splits(nt, detector);
    const int tps = (nt + sp - 1) / sp;
    const size_t need = gbd_field_point_workspace_bytes(n_beamlets, detector);
    if (workspace_bytes < need)
        return fail(GBD_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed",
                    workspace_bytes, need);
    char* base = static_cast<char*>(workspace);
    double2* partial = reinterpret_cast<double2*>(base + align256((size_t)nt * gbd::kF64TileBytes));
    cudaError_t e;
    {
        TimingScope ts(kTimePoint, s);
        e = gbd_launch_point(beamlets, n_beamlets, pp, base, sp, tps, partial, wait_spins(), s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gbd_field_point launch");
    gbd_field_launch PL;
    PL.rows_per_thread = 1;
    PL.cols_per_thread = 1;
    PL.splits = sp;
    PL.tiles_per_split = tps;
    PL.scheme = GBD_SCHEME_DIRECT;
    e = gbd_launch_field_reduce(GBD_PREC_F64, pp, PL, nullptr, partial,
                                gbd_reduce_out(pp, field_out, nullptr, 0, detector->ny), s);
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "gbd_field_point reduce");
}

gbd_status gbd_probe_peaks(double* out) {
    if (!out) return fail(GBD_EINVAL, "out is NULL");
    cudaError_t e = gbd_run_probes(out);
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "gbd_probe_peaks");
}

}  // extern "C"
