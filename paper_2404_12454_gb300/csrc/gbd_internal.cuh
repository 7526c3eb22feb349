// Internal device helpers of the GBD library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "gbd.h"

namespace gbd {

// Named NVTX range over the host side of an API call, so that profiler timelines group
// each call's launches under its name (header-only NVTX v3: without an attached tool a
// push/pop pair costs a few nanoseconds).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define GBD_NVTX_RANGE(name) ::gbd::NvtxRange gbd_nvtx_range_(name)

// Beamlets per shared-memory tile of the field kernels.  A mixed-precision tile is
// 64 x 16 floats = 4 KB, an FP64 tile 64 x 16 doubles = 8 KB; both are one contiguous
// bulk copy.
constexpr int kTile = 64;
constexpr int kMixedFields = 4;   // float4 fields per beamlet
constexpr int kF64Fields = 8;     // double2 fields per beamlet
constexpr int kEdgeFields = 16;   // double2 fields per edge record (truncated beamlets)
constexpr uint32_t kMixedTileBytes = kTile * kMixedFields * 16;
constexpr uint32_t kF64TileBytes = kTile * kF64Fields * 16;
constexpr float kPadLog2Amp = -1000.0f;  // exp2 of this is 0: padding beamlets vanish

// Default iteration limit of the bounded mbarrier waits (about a second of spinning).
constexpr uint32_t kDefaultWaitSpins = 1u << 24;

// Status bits recorded in a translation unit's device status word.
constexpr unsigned kStatusTimeout = 1u;
// Bits of the projection's flag word (mixed records).
constexpr unsigned kFlagWide = 1u;   // some phase may exceed kWidePhase on the detector
constexpr unsigned kFlagSteep = 2u;  // the row-pair recurrence could leave FP32 range
constexpr unsigned kFlagColSteep = 4u;  // so could an amplitude recurrence along a row
constexpr unsigned kFlagCross = 8u;     // some beamlet has a uv term (column factor T != 1)
constexpr unsigned kFlagSteepRows = 16u;  // a 16- or 24-row step (row triples, quadruples)
                                          // could leave FP32 range

// ----------------------------------------------------------------- PTX wrappers --

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Drops the 128-byte L2 line at `p` (128-byte aligned) without writing it back: its
// contents become undefined.  For scratch data that has been consumed.
__device__ __forceinline__ void discard_l2_line(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Bounded wait on an mbarrier phase: false after `spins` unsuccessful polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t spins) {
    for (uint32_t it = 0; it < spins; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 1-D bulk copy global -> shared (TMA engine), completion signalled on `bar` as
// transaction bytes.  Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// MUFU (XU pipe) approximations, PTX-ISA documented forms.
__device__ __forceinline__ float mufu_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_sin(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_cos(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x - nearest integer, exact for |x| < 2^22, on the FMA pipe: adding and removing
// 1.5 * 2^23 rounds to an integer in the current (round-to-nearest-even) mode.
__device__ __forceinline__ float frac_turns(float x) {
    const float magic = 12582912.0f;
    float n = __fsub_rn(__fadd_rn(x, magic), magic);
    return __fsub_rn(x, n);
}

// Error-free transformation a + b = s + e (Knuth's TwoSum), FP32.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// ------------------------------------------------------------- FP64 complex --

struct cd {
    double re, im;
};
__host__ __device__ __forceinline__ cd mk(double r, double i = 0.0) { return cd{r, i}; }
__host__ __device__ __forceinline__ cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cd operator*(cd a, cd b) {
    return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cd cdiv(cd a, cd b) {
    // Smith's algorithm, one reciprocal of the denominator (FP64 division is slow on GB300)
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, inv = 1.0 / (b.re + b.im * r);
        return cd{(a.re + a.im * r) * inv, (a.im - a.re * r) * inv};
    } else {
        const double r = b.re / b.im, inv = 1.0 / (b.re * r + b.im);
        return cd{(a.re * r + a.im) * inv, (a.im * r - a.re) * inv};
    }
}
// Principal square root, branch cut on the negative real axis (sign of im kept).  The
// modulus is formed directly: the arguments here (entries of A + B P1 and their
// determinants) stay far from FP64 overflow and underflow, so hypot's scaling is not needed.
__host__ __device__ __forceinline__ cd csqrt_p(cd z) {
    double r = sqrt(fma(z.re, z.re, z.im * z.im));
    if (r == 0.0) return cd{0.0, z.im};
    if (z.re >= 0.0) {
        double t = sqrt(0.5 * (r + z.re));
        return cd{t, z.im / (2.0 * t)};
    }
    double t = sqrt(0.5 * (r - z.re));
    return cd{fabs(z.im) / (2.0 * t), copysign(t, z.im)};
}

}  // namespace gbd

// ----------------------------------------------------- cross-unit host entries --
// Implemented in the kernel translation units, called by the C ABI layer.

// Decomposition constants of one pupil sampling (Eq. OF): spacing s = D/N, waist
// w0 = OF D/(2N), weight s^2/(pi w0^2), parabasal steps h = WR w0 and
// dth = WR lambda/(pi w0) with their reciprocals, P1 = i p1 I with p1 = -lambda/(pi w0^2).
// Computed once per pupil on the host (IEEE FP64, as on the device).
struct gbd_grid {
    double s, w0, weight, h, dth, p1, ih, idt;
};
inline gbd_grid gbd_make_grid(double D, double lambda, int N, double OF, double WR) {
    gbd_grid g;
    g.s = D / N;
    g.w0 = OF * D / (2.0 * N);
    const double ipw = 1.0 / (M_PI * g.w0);
    g.weight = g.s * g.s * ipw / g.w0;
    g.h = WR * g.w0;
    g.dth = WR * lambda * ipw;
    g.p1 = -lambda * ipw / g.w0;
    g.ih = 1.0 / g.h;
    g.idt = 1.0 / g.dth;
    return g;
}

struct gbd_trace_params {
    double wavelength, inv_f, d, zern_radius;
    double diameter, overlap_factor, waist_ratio;
    int32_t n_across;
    int32_t zdeg;                 // degree of the plate polynomial (-1 = no plate)
    double zpoly[66];             // W(x/R, y/R) = sum zpoly[idx(a,b)] (x/R)^a (y/R)^b
    gbd_grid grid;                // of the single pupil traced without an instance table
};

// Sequence of reflective conics (lab-frame curvatures, vertices) for real-ray traces.
struct gbd_mirror_params {
    int32_t n;
    int32_t n_across;
    double z[GBD_MAX_MIRRORS], c[GBD_MAX_MIRRORS], K[GBD_MAX_MIRRORS];
    double z_ep, z_img, axial_path;
    double wavelength, diameter, overlap_factor, waist_ratio;
    gbd_grid grid;
};

struct gbd_project_params {
    double wavelength;
    double M[4];       // detector (s_x, s_y) -> lab (x, y), row-major
    double n[2];       // detector (s_x, s_y) -> lab axial offset z
    double px, py;
    int32_t nx, ny;
    double inv_wavelength, inv_px, inv_py;  // reciprocals (FP64 division is slow here)
    // Row slab evaluated by the field kernels: detector rows row0 .. row0 + rows - 1.  The
    // projection stores each beamlet's centre row relative to row0 (j0 - row0), so the
    // kernels index the slab's rows from 0 with the same integer offsets tv as on the whole
    // detector; everything else (flags, bounds) refers to the whole nx x ny detector.
    int32_t row0, rows;
};

struct gbd_field_launch {
    int rows_per_thread, cols_per_thread, splits, tiles_per_split, scheme;
};

namespace gbd {
// Where the summed split partials go: the output window (rows skip .. skip + out_rows - 1 of
// the evaluated slab, the slab starting at detector row row0 of ny) with the tilted plane's
// carrier exp(2 pi i (cx (i - nx/2) + cy (j - ny/2))) applied, and the per-pixel-block
// completion counters of the multi-row kernel (zeroed before each field).
struct ReduceOut {
    void* out;
    unsigned* done;
    int ny, row0, skip, out_rows;
    double cx, cy;
};
}  // namespace gbd

namespace gbd {
// Index of the monomial xi^a eta^b in a degree-ordered table: degree g = a + b occupies
// entries g(g+1)/2 .. g(g+1)/2 + g.  Degree <= 10 needs 66 entries.
__host__ __device__ __forceinline__ int plate_index(int a, int b) {
    int g = a + b;
    return g * (g + 1) / 2 + b;
}
}  // namespace gbd

// One instance of a batched trace: its own pupil sampling, written from record `offset`
// (`reserved` carries the instance's beamlet count for the batched projection).
struct gbd_instance_dev {
    int32_t n_across;
    int32_t reserved;
    int64_t offset;
    double overlap_factor, waist_ratio;
    gbd_grid grid;
};

// Traces one pupil (d_inst == nullptr: the sampling in p) or n_instances pupils sharing
// the optics in p, each from its own record offset.
cudaError_t gbd_launch_trace(const gbd_trace_params& p, int n_instances, int max_n_across,
                             const gbd_instance_dev* d_inst, gbd_beamlet* out, cudaStream_t s);
// Batched trace + mixed projection straight into the tiled records (sweep set-up).
// One thread per record; d_rows[d_rbase[k] + j] = first beamlet index of row j of
// instance k (inside the instance).
// Batched trace + projection of a sweep's instances: through the thin-lens system `p`,
// or, when `m` is not null, through its mirror sequence (real rays).
cudaError_t gbd_launch_trace_project(const gbd_trace_params& p, const gbd_mirror_params* m,
                                     int n_instances, const gbd_instance_dev* d_inst,
                                     const int* d_rbase, const int* d_rows, long long n_records,
                                     const gbd_project_params& g, float4* out, unsigned* wide,
                                     cudaStream_t s);
// `wide` (mixed only, may be null): set to 1 when some beamlet's phase may exceed the
// wide-phase bound on this detector; the caller zeroes it first.
cudaError_t gbd_launch_project(const gbd_beamlet* b, int n, const gbd_project_params& p,
                               int precision, void* coeffs, unsigned* wide, cudaStream_t s);
cudaError_t gbd_launch_trace_mirrors(const gbd_mirror_params& m, gbd_beamlet* out, cudaStream_t s);
// ro: where a kernel that sums the splits itself (the multi-row kernels) stores the field.
cudaError_t gbd_launch_field_kernel(int precision, const void* coeffs, int n_tiles,
                                    const gbd_project_params& p, const gbd_field_launch& L,
                                    void* partial, const unsigned* wide, uint32_t wait_spins,
                                    const gbd::ReduceOut& ro, cudaStream_t s);
// partial: float2 per pixel and split for GBD_PREC_MIXED, double2 for GBD_PREC_F64, over
// the slab p.row0 .. p.row0 + p.rows - 1; writes detector rows out_row0 .. + out_rows - 1
// (inside the slab) to `out`, row-major from out_row0
// Output window of a field: detector rows out_row0 .. out_row0 + out_rows - 1 (inside the
// evaluated slab p.row0 .. p.row0 + p.rows - 1) into `out`; `done`: the multi-row kernel's
// per-pixel-block counters (zeroed before the launch; at least ceil(nx/32) ceil(rows/8)).
gbd::ReduceOut gbd_reduce_out(const gbd_project_params& p, void* out, unsigned* done,
                              int out_row0, int out_rows);
// Sums the split partials into the output window, unless the flag word (may be null) shows
// that the launch's multi-row kernel took the field and stored it itself.
cudaError_t gbd_launch_field_reduce(int precision, const gbd_project_params& p,
                                    const gbd_field_launch& L, const unsigned* flags,
                                    const void* partial, const gbd::ReduceOut& ro,
                                    cudaStream_t s);
// Truncated decomposition: trace of the extended grid (interior beamlets first), and the
// edge records of its last n beamlets (see project_edge_kernel).
cudaError_t gbd_launch_trace_truncated(const gbd_trace_params& p, int ext, double inner,
                                       double outer, long long n_interior, gbd_beamlet* out,
                                       cudaStream_t s);
cudaError_t gbd_launch_project_edge(const gbd_beamlet* b, int n, const gbd_project_params& p,
                                    double2* out, cudaStream_t s);
// Partial fields of the edge kernel's beamlet splits (bytes, reusable scratch).
size_t gbd_field_edge_partial_bytes(int precision, int n_edge, int nx, int ny);
// Adds the edge beamlets' sum onto a field of nx x ny pixels (complex64 / complex128),
// through per-split partial fields in `partial` (gbd_field_edge_partial_bytes).
cudaError_t gbd_launch_field_edge(int precision, const double2* edge_records, int n_edge, int nx,
                                  int ny, void* out, void* partial, cudaStream_t s);
// Height of the pixel-row blocks of every kernel a launch runs: a slab that starts on a
// multiple of it is split into the same thread row blocks as the whole detector.
int gbd_field_row_block(int precision, const gbd_field_launch& L);
int gbd_field_occupancy(int precision, int rb, int cb, int scheme);
// Columns per thread (8, 4 or 2, at least min_cols) of the row-pair shape that covers a
// detector nx pixels wide at the least estimated cost.
int gbd_auto_cols(int nx, int min_cols);
gbd_status gbd_set_error(gbd_status st, const char* msg);  // sets gbd_last_error()
gbd_status gbd_check_system(const gbd_system* s);
// Mirror-sequence kernel parameters (validated; GBD_EINVAL with gbd_last_error set)
gbd_status gbd_make_mirror_params(const gbd_mirror_system* system, double diameter,
                                  gbd_mirror_params* out);
gbd_status gbd_check_detector(const gbd_detector* d);
gbd_project_params gbd_make_project_params(double wavelength, const gbd_detector* d);
gbd_trace_params gbd_make_trace_params(const gbd_system* system, double diameter);
int gbd_sm_count();
uint32_t gbd_wait_spins();
cudaError_t gbd_sweep_status_fetch(unsigned* host, cudaStream_t s);
void gbd_sweep_status_clear();
cudaError_t gbd_point_status_fetch(unsigned* host, cudaStream_t s);
void gbd_point_status_clear();
cudaError_t gbd_mlp_status_fetch(unsigned* host, cudaStream_t s);
void gbd_mlp_status_clear();
long gbd_point_pixel_ctas(int nx, int ny);
int gbd_point_occupancy();
// Point evaluation: packs the beamlets into `coeffs` (FP64 tiles) and launches the
// per-(beamlet, pixel) propagation kernel writing split partial fields.
cudaError_t gbd_launch_point(const gbd_beamlet* b, int n, const gbd_project_params& p, void* coeffs,
                             int splits, int tiles_per_split, double2* partial, uint32_t spins,
                             cudaStream_t s);
gbd_status gbd_field_fixed_scratch(const gbd_beamlet* beamlets, int32_t n, double wavelength,
                                   const gbd_detector* detector, int32_t precision,
                                   void* scratch, size_t scratch_bytes, void* out,
                                   cudaStream_t stream);
bool gbd_field_shape_supported(int precision, int rb, int cb, int scheme);
cudaError_t gbd_field_status_fetch(unsigned* host, cudaStream_t s);
void gbd_field_status_clear();
cudaError_t gbd_run_probes(double* out);
