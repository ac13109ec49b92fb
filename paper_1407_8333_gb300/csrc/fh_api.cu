// C ABI of libfh: plans, host-side validation, and the stream-ordered entry
// points fh_correct_doppler / fh_transform / fh_select_candidates.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <future>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

#include <unistd.h>

#include "fh_internal.h"

namespace fh {

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char *what)
{
    return set_error(FH_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace fh

using namespace fh;

namespace {

struct DeviceGuard {
    int prev = -1, want = -1;
    explicit DeviceGuard(int dev) : want(dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

namespace fh {

int device_error_code(int32_t bits)
{
    if (bits & (kErrCsr | kErrUnsorted))
        return set_error(FH_ERR_UNSORTED, "device inputs: offsets not a valid CSR, t_fft not "
                                          "increasing or freq not ascending within an FFT");
    if (bits & kErrInvalid)
        return set_error(FH_ERR_INVALID_ARG, "device inputs: non-finite or out-of-range value");
    if (bits & kErrRange)
        return set_error(FH_ERR_RANGE, "a fixed-point position or shift exceeds 2^28 cells");
    return FH_OK;
}


int max_optin_smem(int device)
{
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    return v > 0 ? v : 48 * 1024;
}

// the error word (bytes 0..3) and the largest |D| (bytes 16..23) of a plan,
// one allocation cleared by one memset per call
constexpr size_t kErrWordsBytes = 32;

// Device address of a page-locked (pinned or registered, mapped) host array,
// which kernels can read in place; nullptr for pageable or unknown memory.
const void *pinned_device_address(const void *h)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer != nullptr) ? a.devicePointer : nullptr;
}

// largest multiple-of-32 tile width whose counters fit the per-block limit
int32_t default_tile(const fh_plan_desc &d, int device, int32_t mode, int32_t nwarps, int32_t guard)
{
    const size_t lim = (size_t)max_optin_smem(device);
    int32_t w = 32;
    for (int32_t t = 32; t <= 8192; t += 32) {
        if (transform_smem_bytes(t, d.k_over, mode, nwarps, guard) > lim) break;
        w = t;
    }
    if (w > d.n_f0) w = d.n_f0;
    return w;
}

unsigned long long default_drift(const fh_plan_desc &d)
{
    const double cells = 0.5 * d.k_over + 0.25;
    return (unsigned long long)(cells * 4294967296.0);
}

int32_t default_guard(const fh_plan_desc &d) { return guard_for(default_drift(d)); }

// the largest |D_i| in 32.32 cells per row, from host-memory FFT times
unsigned long long host_drift(const fh_plan_desc &d, double kt, const double *t, int32_t n_fft)
{
    double m = 0.0;
    for (int32_t i = 0; i < n_fft; ++i) {
        const double x = std::fabs(d.fdot_step * ((t[i] - d.t_ref) * kt));
        if (x > m && x < 1e9) m = x;  // non-finite or absurd times are left to the checks
    }
    return (unsigned long long)(m * 4294967296.0) + 4;
}

int32_t host_guard(const fh_plan_desc &d, double kt, const double *t, int32_t n_fft)
{
    return guard_for(host_drift(d, kt, t, n_fft));
}

int32_t pair_delta(const fh_plan_desc &d) { return 2 * d.k_over + 4; }

bool pairs_apply(const fh_plan_desc &d, int device, int32_t n_fft, int32_t n_dir,
                 unsigned long long drift)
{
    if (n_dir < 2 || n_fft <= 0 || n_fft >= 65536 ||
        (int64_t)d.k_over * n_fft >= ((int64_t)1 << 25))
        return false;
    const int32_t g = guard_for(drift) + pair_delta(d);
    return transform_smem_bytes(256, d.k_over, FH_MODE_START, 32, g) <=
           (size_t)max_optin_smem(device);
}

bool rows_apply(const fh_plan_desc &d, int device, int32_t n_fft, int32_t n_dir,
                unsigned long long drift)
{
    if (n_dir != 1 || d.n_fdot <= kRows || n_fft <= 0 || n_fft >= 65536 ||
        (int64_t)d.k_over * n_fft >= ((int64_t)1 << 25))
        return false;
    const int32_t g = guard_for(drift, 2 * kRows - 1);
    return transform_smem_bytes(256, d.k_over, FH_MODE_START, 32, g) <=
           (size_t)max_optin_smem(device);
}

int validate_desc(const fh_plan_desc &d)
{
    auto bad = [](const char *m) { return set_error(FH_ERR_INVALID_ARG, "plan: %s", m); };
    if (!(std::isfinite(d.t_fft) && d.t_fft > 0.0)) return bad("t_fft must be finite and > 0");
    if (d.k_over < 1 || d.k_over > (1 << 16)) return bad("k_over must be in [1, 65536]");
    const double kt = (double)d.k_over * d.t_fft;
    if (std::fma((double)d.k_over, d.t_fft, -kt) != 0.0)
        return bad("k_over * t_fft must be exactly representable in binary64");
    if (!std::isfinite(d.f0_min)) return bad("f0_min must be finite");
    if (d.n_f0 < 1) return bad("n_f0 must be >= 1");
    if ((int64_t)d.n_f0 + d.k_over >= kFixedLimit)
        return set_error(FH_ERR_RANGE, "plan: n_f0 + k_over must stay below 2^28");
    if (!std::isfinite(d.fdot_min) || !std::isfinite(d.fdot_step))
        return bad("fdot_min and fdot_step must be finite");
    if (d.n_fdot < 1 || d.n_fdot > (1 << 20)) return bad("n_fdot must be in [1, 2^20]");
    if (!std::isfinite(d.t_ref)) return bad("t_ref must be finite");
    if (d.subband_cells < 1) return bad("subband_cells must be >= 1");
    if (d.top_k < 1 || d.top_k > 64) return bad("top_k must be in [1, 64]");
    if (d.excl_cells < 0 || d.sep_cells < 0) return bad("excl_cells and sep_cells must be >= 0");
    if (!(d.p0 > 0.0 && d.p0 < 1.0)) return bad("p0 must be in (0, 1)");
    if (d.max_fft < 1 || d.max_fft > (1 << 26)) return bad("max_fft must be in [1, 2^26]");
    if (d.max_dir < 1 || d.max_dir > 65535) return bad("max_dir must be in [1, 65535]");
    if (d.max_peaks < 1 || d.max_peaks >= ((int64_t)1 << 31))
        return bad("max_peaks must be in [1, 2^31)");
    if (d.mode < FH_MODE_AUTO || d.mode > FH_MODE_START) return bad("unknown mode");
    if (d.schedule < FH_SCHED_BATCHED || d.schedule > FH_SCHED_PLAIN)
        return bad("unknown schedule");
    if (d.tile_cells != 0 && d.tile_cells < 32) return bad("tile_cells must be 0 or >= 32");
    if (d.block_warps != 0 && (d.block_warps < 4 || d.block_warps > 32))
        return bad("block_warps must be 0 or in [4, 32]");
    return FH_OK;
}

}  // namespace fh

namespace {

struct Sizes {
    int64_t t, offsets, tables, freq, v, sky, A, profile, cand;
    int64_t total() const
    {
        return t + 2 * offsets + 2 * tables + freq + v + sky + A + profile + cand + 256;
    }
};

Sizes plan_sizes(const fh_plan_desc &d)
{
    const int64_t n_sb = (d.n_f0 + d.subband_cells - 1) / d.subband_cells;
    Sizes s;
    s.t = 8 * (int64_t)d.max_fft;
    s.offsets = 8 * ((int64_t)d.max_fft + 1);
    s.tables = 8 * (int64_t)d.max_fft;
    s.freq = 8 * d.max_peaks;
    s.v = 24 * (int64_t)d.max_fft;
    s.sky = 24 * (int64_t)d.max_dir;
    s.A = 8 * (int64_t)d.max_dir * d.max_peaks;
    s.profile = 8 * (int64_t)d.max_dir * d.n_f0;
    s.cand = (int64_t)sizeof(fh_candidate) * d.max_dir * n_sb * d.top_k;
    return s;
}

}  // namespace

constexpr int64_t kTimingSlots = 256;

struct fh_plan_s {
    fh_plan_desc d{};
    int device = 0;
    int n_sm = 0;
    double kt = 0.0;
    int32_t n_sb = 0;
    int32_t mode = FH_MODE_START;
    int32_t tile_cells = 0;
    int32_t block_warps = 32;
    double *t = nullptr, *freq = nullptr, *v = nullptr, *sky = nullptr;
    int64_t *offsets = nullptr, *S0 = nullptr, *D = nullptr, *A = nullptr;
    int64_t *offsets_raw = nullptr;  // host offsets as copied, for the device checks
    int32_t input_checks = FH_CHECKS_HOST;
    uint64_t *profile = nullptr;
    fh_candidate *cand = nullptr;
    int32_t *err = nullptr;
    int32_t *h_err = nullptr;  // pinned
    unsigned long long *dmax = nullptr;  // largest |D_i| of the current peakmap (in err's block)
    int32_t *dense = nullptr;            // set by the window pre-pass: an FFT with two peaks
                                         // in one cell (in err's block)
    int32_t *unit_delta = nullptr;       // per direction pair of a group: the largest distance
                                         // between a peak's two cells (window pre-pass)
    unsigned int *sched = nullptr;       // the batched transform's item counter (2 words,
                                         // zero between launches)
    uint32_t *win = nullptr;             // peak windows of the directions being transformed
    size_t win_bytes = 0;
    int32_t guard = 0;                   // guard cells for the transform's fast path (32 rows)
    unsigned long long drift = 0;        // bound of max |D_i| the guards are sized for
    int32_t pair_pref = 0;               // 0: pairs (of directions, or of one direction's row
                                         // halves) where they apply; 1: never
    int32_t item_counter = 1;            // batched transform: items from the counter (1) or
                                         // every grid-th item per block (0)
    int32_t n_fft = -1;
    int64_t n_peaks = 0;
    int32_t n_dir = 0;
    int64_t launches = 0;
    size_t prepared_smem[3] = {0, 0, 0};
    // adaptive weights (Eq. ncountadap), set by fh_set_weights until the next
    // fh_correct_doppler: W [max_dir][max_fft] and per-direction sums S1, S2
    int32_t *wq = nullptr;
    int64_t *ws = nullptr;       // [2][max_dir]: S1 then S2
    bool weighted = false;
    int64_t w_bound = 0;         // largest count bound over the directions (fh_set_weights)
    // optional kernel timing: per direction group of fh_transform, events before
    // the window pre-pass, between it and the transform, after the transform
    int32_t timing = 0;
    std::vector<cudaEvent_t> tev;  // 3 x kTimingSlots
    int64_t tev_next = 0;          // groups recorded since timing was switched on

    void release()
    {
        for (cudaEvent_t ev : tev) cudaEventDestroy(ev);
        tev.clear();
        void *bufs[] = {t,    freq, v,   sky,  offsets, offsets_raw, S0, D,
                        A,    profile, cand, err, win,  wq,  ws, unit_delta, sched};  // dmax: in err's block
        for (void *b : bufs)
            if (b) cudaFree(b);
        if (h_err) cudaFreeHost(h_err);
        t = freq = v = sky = nullptr;
        offsets = S0 = D = A = offsets_raw = nullptr;
        profile = nullptr;
        cand = nullptr;
        err = h_err = nullptr;
        dmax = nullptr;
        win = nullptr;
        win_bytes = 0;
        wq = nullptr;
        unit_delta = nullptr;
        sched = nullptr;
        ws = nullptr;
    }
};

namespace {

int prepare_transform(fh_plan p, int32_t mode, size_t smem)
{
    if (p->prepared_smem[mode] >= smem) return FH_OK;
    cudaError_t e = transform_prepare(mode, smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(transform)");
    p->prepared_smem[mode] = smem;
    return FH_OK;
}

int check_dirs(fh_plan p, int32_t dir_begin, int32_t n_dir)
{
    if (p->n_fft < 0)
        return set_error(FH_ERR_INVALID_ARG, "fh_correct_doppler has not been called on this plan");
    if (dir_begin < 0 || n_dir < 1 || (int64_t)dir_begin + n_dir > p->n_dir)
        return set_error(FH_ERR_INVALID_ARG, "directions [%d, %d) outside [0, %d)", dir_begin,
                         dir_begin + n_dir, p->n_dir);
    return FH_OK;
}

}  // namespace

namespace fh {

int validate_host_inputs(const fh_plan_desc &d, double kt, const fh_peakmap *pm, const double *v,
                         const double *sky, int32_t n_dir)
{
    const int32_t n = pm->n_fft;
    if (n > 0 && (!pm->t_fft || !v)) return set_error(FH_ERR_INVALID_ARG, "null t_fft or v");
    if (!pm->offsets) return set_error(FH_ERR_INVALID_ARG, "null offsets");
    if (pm->n_peaks > 0 && !pm->freq) return set_error(FH_ERR_INVALID_ARG, "null freq");
    if (pm->offsets[0] != 0) return set_error(FH_ERR_UNSORTED, "offsets[0] must be 0");
    for (int32_t i = 0; i < n; ++i) {
        if (pm->offsets[i + 1] < pm->offsets[i])
            return set_error(FH_ERR_UNSORTED, "offsets decrease at FFT %d", i);
        if (!std::isfinite(pm->t_fft[i]))
            return set_error(FH_ERR_INVALID_ARG, "t_fft[%d] not finite", i);
        if (i > 0 && !(pm->t_fft[i] > pm->t_fft[i - 1]))
            return set_error(FH_ERR_UNSORTED, "t_fft not strictly increasing at %d", i);
    }
    if (pm->offsets[n] != pm->n_peaks)
        return set_error(FH_ERR_UNSORTED, "offsets[n_fft] = %lld != n_peaks = %lld",
                         (long long)pm->offsets[n], (long long)pm->n_peaks);
    // Screening pass without branches (positive finite doubles order like their
    // bit patterns, read as unsigned integers); the detailed pass that names the
    // first bad peak runs only when the screen fails.  With every FFT's
    // frequencies ascending, the band's range comes from first and last peaks.
    {
        const uint64_t *fb = reinterpret_cast<const uint64_t *>(pm->freq);
        // bits - 1 of a positive finite double lies in [0, bits(DBL_MAX) - 1]; zero,
        // negatives, infinities and NaNs fall outside
        const uint64_t kPosFiniteMax = 0x7FEFFFFFFFFFFFFEull;
        auto screen = [&](int32_t i0, int32_t i1) {
            uint64_t bad = 0;
            for (int32_t i = i0; i < i1; ++i) {
                const int64_t a = pm->offsets[i], b = pm->offsets[i + 1];
                if (a >= b) continue;
                bad |= (uint64_t)((fb[a] - 1) > kPosFiniteMax);
                for (int64_t q = a + 1; q < b; ++q)
                    bad |= (uint64_t)((fb[q] - 1) > kPosFiniteMax) | (uint64_t)(fb[q] <= fb[q - 1]);
            }
            return bad;
        };
        // large peakmaps: FFT ranges on up to 8 threads
        const int parts =
            (int)std::min<int64_t>(8, std::max<int64_t>(1, pm->n_peaks / ((int64_t)1 << 18)));
        uint64_t bad = 0;
        if (parts > 1 && n >= parts) {
            std::vector<std::future<uint64_t>> fut;
            for (int k = 1; k < parts; ++k)
                fut.push_back(std::async(std::launch::async, screen,
                                         (int32_t)((int64_t)n * k / parts),
                                         (int32_t)((int64_t)n * (k + 1) / parts)));
            bad = screen(0, (int32_t)((int64_t)n / parts));
            for (auto &f : fut) bad |= f.get();
        } else {
            bad = screen(0, n);
        }
        if (bad) {
            for (int32_t i = 0; i < n; ++i) {
                for (int64_t q = pm->offsets[i]; q < pm->offsets[i + 1]; ++q) {
                    const double f = pm->freq[q];
                    if (!(std::isfinite(f) && f > 0.0))
                        return set_error(FH_ERR_INVALID_ARG, "freq[%lld] must be finite and > 0",
                                         (long long)q);
                    if (q > pm->offsets[i] && !(f > pm->freq[q - 1]))
                        return set_error(FH_ERR_UNSORTED, "freq not ascending within FFT %d", i);
                }
            }
        }
    }
    double fmin = INFINITY, fmax = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        const int64_t a = pm->offsets[i], b = pm->offsets[i + 1];
        if (a < b) {
            fmin = std::min(fmin, pm->freq[a]);
            fmax = std::max(fmax, pm->freq[b - 1]);
        }
    }
    double vmax = 0.0, nmax = 0.0, tmax = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        const double *x = v + 3 * (int64_t)i;
        if (!(std::isfinite(x[0]) && std::isfinite(x[1]) && std::isfinite(x[2])))
            return set_error(FH_ERR_INVALID_ARG, "v_over_c[%d] not finite", i);
        vmax = std::max(vmax, std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
        tmax = std::max(tmax, std::fabs(pm->t_fft[i] - d.t_ref));
    }
    for (int32_t k = 0; k < n_dir; ++k) {
        const double *x = sky + 3 * (int64_t)k;
        if (!(std::isfinite(x[0]) && std::isfinite(x[1]) && std::isfinite(x[2])))
            return set_error(FH_ERR_INVALID_ARG, "sky_n[%d] not finite", k);
        const double nn = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (nn > 1.000001) return set_error(FH_ERR_INVALID_ARG, "sky_n[%d] longer than 1", k);
        nmax = std::max(nmax, nn);
    }
    const double vn = vmax * nmax;
    if (!(vn < 0.1)) return set_error(FH_ERR_INVALID_ARG, "|v.n| must stay below 0.1 (units of c)");
    const double lim = (double)kFixedLimit * 0.999;
    if (pm->n_peaks > 0) {
        const double ulo = fmin / (1.0 + vn), uhi = fmax / (1.0 - vn);
        const double x = std::max(std::fabs((ulo - d.f0_min) * kt), std::fabs((uhi - d.f0_min) * kt));
        if (!(x + d.k_over + 2.0 < lim))
            return set_error(FH_ERR_RANGE, "peak positions exceed 2^28 cells from f0_min");
    }
    const double flast = d.fdot_min + (double)(d.n_fdot - 1) * d.fdot_step;
    const double fabsmax = std::max(std::fabs(d.fdot_min), std::fabs(flast));
    if (!(fabsmax * tmax * kt < lim))
        return set_error(FH_ERR_RANGE, "spin-down shifts exceed 2^28 cells");
    return FH_OK;
}

}  // namespace fh

extern "C" {

const char *fh_last_error(void) { return g_err; }

const char *fh_version(void) { return "fh-gb300 0.1 (sm_103a)"; }

int64_t fh_plan_device_bytes(const fh_plan_desc *desc)
{
    if (!desc || validate_desc(*desc) != FH_OK) return 0;
    return plan_sizes(*desc).total();
}

int fh_create_plan(const fh_plan_desc *desc, fh_plan *out)
{
    if (!desc || !out) return set_error(FH_ERR_INVALID_ARG, "null desc or out");
    *out = nullptr;
    int rc = validate_desc(*desc);
    if (rc) return rc;
    fh_plan p = new (std::nothrow) fh_plan_s;
    if (!p) return set_error(FH_ERR_NOMEM, "host allocation failed");
    p->d = *desc;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_error(e, "cudaGetDevice");
    }
    cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device);
    p->kt = (double)desc->k_over * desc->t_fft;
    p->n_sb = (desc->n_f0 + desc->subband_cells - 1) / desc->subband_cells;
    p->mode = desc->mode == FH_MODE_AUTO ? FH_MODE_START : desc->mode;
    p->block_warps = desc->block_warps ? desc->block_warps : 32;
    p->drift = default_drift(*desc);
    p->guard = default_guard(*desc);
    p->tile_cells = desc->tile_cells ? std::min(desc->tile_cells, desc->n_f0)
                                     : default_tile(*desc, p->device, p->mode, p->block_warps,
                                                    p->guard);
    if (transform_smem_bytes(p->tile_cells, desc->k_over, p->mode, p->block_warps, p->guard) >
        (size_t)max_optin_smem(p->device)) {
        delete p;
        return set_error(FH_ERR_INVALID_ARG, "tile_cells too wide for shared memory");
    }
    const Sizes s = plan_sizes(*desc);
    struct {
        void **ptr;
        int64_t bytes;
    } allocs[] = {{(void **)&p->t, s.t},           {(void **)&p->offsets, s.offsets},
                  {(void **)&p->offsets_raw, s.offsets},
                  {(void **)&p->S0, s.tables},     {(void **)&p->D, s.tables},
                  {(void **)&p->freq, s.freq},     {(void **)&p->v, s.v},
                  {(void **)&p->sky, s.sky},       {(void **)&p->A, s.A},
                  {(void **)&p->profile, s.profile}, {(void **)&p->cand, s.cand},
                  {(void **)&p->err, kErrWordsBytes},
                  {(void **)&p->unit_delta, 4 * ((int64_t)desc->max_dir / 2 + 1)},
                  {(void **)&p->sched, 16}};
    for (auto &a : allocs) {
        e = cudaMalloc(a.ptr, (size_t)std::max<int64_t>(a.bytes, 16));
        if (e != cudaSuccess) {
            cudaGetLastError();
            p->release();
            delete p;
            return set_error(FH_ERR_NOMEM, "cudaMalloc of %lld bytes failed: %s",
                             (long long)a.bytes, cudaGetErrorString(e));
        }
    }
    // the largest |D| lives in the error word's allocation, 16 bytes in, and
    // the window pre-pass's dense-FFT flag 24 bytes in
    p->dmax = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(p->err) + 16);
    p->dense = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(p->err) + 24);
    e = cudaMallocHost(&p->h_err, 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        p->release();
        delete p;
        return set_error(FH_ERR_NOMEM, "cudaMallocHost failed");
    }
    cudaMemset(p->err, 0, kErrWordsBytes);
    cudaMemset(p->sched, 0, 16);
    *out = p;
    return FH_OK;
}

int fh_destroy_plan(fh_plan p)
{
    if (!p) return FH_OK;
    {
        DeviceGuard g(p->device);
        cudaDeviceSynchronize();
        p->release();
    }
    delete p;
    return FH_OK;
}

int64_t fh_plan_launches(fh_plan p) { return p ? p->launches : -1; }

int fh_plan_set_input_checks(fh_plan p, int32_t where)
{
    if (!p) return set_error(FH_ERR_INVALID_ARG, "null plan");
    if (where != FH_CHECKS_HOST && where != FH_CHECKS_DEVICE)
        return set_error(FH_ERR_INVALID_ARG, "checks must be FH_CHECKS_HOST or FH_CHECKS_DEVICE");
    p->input_checks = where;
    return FH_OK;
}

int fh_refine(fh_plan p, const fh_peakmap *pm, const double *v_over_c, const int32_t *cand_cell,
              const int32_t *cand_row, int32_t n_cand, const double *sky_ref, int32_t n_ref,
              int32_t k_fdot, fh_candidate *out, int64_t capacity, void *stream)
{
    if (!p || !pm || !v_over_c || (n_cand > 0 && (!cand_cell || !cand_row || !sky_ref || !out)))
        return set_error(FH_ERR_INVALID_ARG, "null plan, peakmap, velocity or candidate array");
    if (pm->mem_kind != FH_MEM_HOST)
        return set_error(FH_ERR_INVALID_ARG, "fh_refine takes host-memory inputs");
    if (n_cand < 0 || n_ref < 1 || n_ref > 65535 || k_fdot < 1 || k_fdot > 64)
        return set_error(FH_ERR_INVALID_ARG, "need n_cand >= 0, n_ref in [1, 65535], "
                                             "k_fdot in [1, 64]");
    if ((int64_t)n_cand * n_ref > 1000000000)
        return set_error(FH_ERR_INVALID_ARG, "n_cand x n_ref too large");
    if (pm->n_fft < 0 || pm->n_peaks < 0 || pm->n_peaks >= ((int64_t)1 << 31) || !pm->offsets ||
        (pm->n_fft > 0 && !pm->t_fft) || (pm->n_peaks > 0 && !pm->freq))
        return set_error(FH_ERR_INVALID_ARG, "bad peakmap (n_fft >= 0, n_peaks in [0, 2^31))");
    if (capacity < n_cand)
        return set_error(FH_ERR_CAPACITY, "need %d refined candidate slots, capacity %lld", n_cand,
                         (long long)capacity);
    if (n_cand == 0) return FH_OK;
    DeviceGuard g(p->device);
    return refine_impl(p->d, p->n_sm, pm, v_over_c, cand_cell, cand_row, n_cand, sky_ref, n_ref,
                       k_fdot, out, p->input_checks == FH_CHECKS_HOST, as_stream(stream));
}

int fh_set_weights(fh_plan p, const double *w, int32_t n_dir, int32_t frac_bits, void *stream)
{
    if (!p) return set_error(FH_ERR_INVALID_ARG, "null plan");
    if (p->n_fft < 0)
        return set_error(FH_ERR_INVALID_ARG, "fh_correct_doppler has not been called on this plan");
    if (!w) {
        p->weighted = false;
        return FH_OK;
    }
    if (n_dir != p->n_dir)
        return set_error(FH_ERR_INVALID_ARG, "weights for %d directions, the plan holds %d", n_dir,
                         p->n_dir);
    if (frac_bits < 0 || frac_bits > 24)
        return set_error(FH_ERR_INVALID_ARG, "frac_bits must be in [0, 24]");
    const int32_t n = p->n_fft;
    const fh_plan_desc &d = p->d;
    // quantise on the host: W = rint(w 2^F) (binary64, ties to even; the product
    // by a power of two is exact), every weight finite and >= 0, and each
    // direction's sum below 2^30 (a cell of a bin-grid peakmap takes at most
    // two stripes of one FFT); then the exact count bound of this peakmap,
    // sum_i W_i c_i with c_i the most stripes of FFT i on one cell (from the
    // positions), must stay below 2^31
    const double scale = std::ldexp(1.0, frac_bits);
    std::vector<int32_t> W((size_t)n_dir * (size_t)std::max(1, n));
    std::vector<int64_t> sums(2 * (size_t)d.max_dir, 0);
    int64_t smax = 0;
    for (int32_t k = 0; k < n_dir; ++k) {
        int64_t s1 = 0, s2 = 0;
        for (int32_t i = 0; i < n; ++i) {
            const double x = w[(int64_t)k * n + i];
            if (!(std::isfinite(x) && x >= 0.0))
                return set_error(FH_ERR_INVALID_ARG, "weight [%d][%d] must be finite and >= 0", k,
                                 i);
            const double q = std::nearbyint(x * scale);
            if (!(q < 1073741824.0))
                return set_error(FH_ERR_RANGE, "weight [%d][%d] is 2^30 or more after scaling", k,
                                 i);
            const int64_t qi = (int64_t)q;
            s1 += qi;
            if (s1 >= ((int64_t)1 << 30))
                return set_error(FH_ERR_RANGE, "direction %d: weights sum to 2^30 or more", k);
            s2 += qi * qi;
            W[(size_t)k * n + i] = (int32_t)qi;
        }
        sums[k] = s1;
        sums[d.max_dir + k] = s2;
        smax = std::max(smax, s1);
    }
    DeviceGuard g(p->device);
    cudaError_t e = cudaSuccess;
    if (!p->wq) {
        e = cudaMalloc(&p->wq, sizeof(int32_t) * (size_t)d.max_dir * (size_t)std::max(1, d.max_fft));
        // S1, S2 and the count bound per direction
        if (e == cudaSuccess) e = cudaMalloc(&p->ws, sizeof(int64_t) * 3 * (size_t)d.max_dir);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(FH_ERR_NOMEM, "cudaMalloc (weights) failed");
        }
    }
    cudaStream_t s = as_stream(stream);
    // pageable sources: each copy has taken its data when it returns
    if (n > 0)
        e = cudaMemcpyAsync(p->wq, W.data(), sizeof(int32_t) * W.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->ws, sums.data(), sizeof(int64_t) * sums.size(),
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(weights)");
    // the count bound of every direction from its positions (synchronises)
    unsigned long long *bound = reinterpret_cast<unsigned long long *>(p->ws + 2 * d.max_dir);
    e = cudaMemsetAsync(bound, 0, sizeof(unsigned long long) * (size_t)n_dir, s);
    if (e == cudaSuccess)
        e = launch_weight_bound(p->A, p->offsets, p->wq, n, n_dir, p->n_peaks, d.k_over, bound, s);
    std::vector<unsigned long long> hb((size_t)std::max(1, n_dir), 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb.data(), bound, sizeof(unsigned long long) * (size_t)n_dir,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->h_err, p->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "weight count bound");
    // an input rejected by the device checks is reported as such (its
    // positions are not trusted, so neither is their bound)
    int rc = device_error_code(*p->h_err);
    if (rc) return rc;
    unsigned long long bmax = 0;
    for (int32_t k = 0; k < n_dir; ++k) {
        if (hb[k] >= (1ull << 31))
            return set_error(FH_ERR_RANGE,
                             "direction %d: weighted counts could reach 2^31 (bound %llu: "
                             "dense peaks of one FFT under large weights)", k, hb[k]);
        bmax = std::max(bmax, hb[k]);
    }
    (void)smax;
    p->weighted = true;
    p->w_bound = (int64_t)bmax;
    return FH_OK;
}

int fh_plan_set_timing(fh_plan p, int32_t on)
{
    if (!p) return set_error(FH_ERR_INVALID_ARG, "null plan");
    DeviceGuard g(p->device);
    if (on && p->tev.empty()) {
        p->tev.resize(3 * (size_t)kTimingSlots, nullptr);
        for (auto &ev : p->tev) {
            const cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) {
                for (cudaEvent_t x : p->tev)
                    if (x) cudaEventDestroy(x);
                p->tev.clear();
                return cuda_error(e, "cudaEventCreate");
            }
        }
    }
    p->timing = on ? 1 : 0;
    p->tev_next = 0;
    return FH_OK;
}

int fh_plan_kernel_times(fh_plan p, int64_t *n_groups, double *windows_ms, double *transform_ms)
{
    if (!p || !n_groups || !windows_ms || !transform_ms)
        return set_error(FH_ERR_INVALID_ARG, "null plan or output");
    DeviceGuard g(p->device);
    const int64_t n = std::min(p->tev_next, kTimingSlots);
    double w = 0.0, t = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t slot = (p->tev_next - n + k) % kTimingSlots;
        cudaEvent_t *ev = &p->tev[3 * (size_t)slot];
        cudaError_t e = cudaEventSynchronize(ev[2]);
        float a = 0.f, b = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[1], ev[2]);
        if (e != cudaSuccess) return cuda_error(e, "kernel timing events");
        w += a;
        t += b;
    }
    *n_groups = n;
    *windows_ms = w;
    *transform_ms = t;
    return FH_OK;
}

int fh_correct_doppler(fh_plan p, const fh_peakmap *pm, const double *v_over_c,
                       const double *sky_n, int32_t n_dir, double *out_r, int64_t *out_A,
                       void *stream)
{
    if (!p || !pm || !sky_n) return set_error(FH_ERR_INVALID_ARG, "null plan, peakmap or sky_n");
    if (pm->mem_kind != FH_MEM_HOST && pm->mem_kind != FH_MEM_DEVICE)
        return set_error(FH_ERR_INVALID_ARG, "unknown mem_kind");
    if (pm->n_fft < 0 || pm->n_fft > p->d.max_fft)
        return set_error(FH_ERR_INVALID_ARG, "n_fft %d outside [0, max_fft=%d]", pm->n_fft,
                         p->d.max_fft);
    if (pm->n_peaks < 0 || pm->n_peaks > p->d.max_peaks)
        return set_error(FH_ERR_INVALID_ARG, "n_peaks outside [0, max_peaks]");
    if (n_dir < 1 || n_dir > p->d.max_dir)
        return set_error(FH_ERR_INVALID_ARG, "n_dir %d outside [1, max_dir=%d]", n_dir,
                         p->d.max_dir);
    if (pm->n_fft > 0 && !v_over_c) return set_error(FH_ERR_INVALID_ARG, "null v_over_c");
    DeviceGuard g(p->device);
    cudaStream_t s = as_stream(stream);
    const int32_t n = pm->n_fft;
    const int64_t np = pm->n_peaks;
    const double *t_src, *f_src, *v_src, *sky_src;
    const int64_t *offs_in_place = nullptr;  // page-locked host offsets read in place
    const bool host_checks = p->input_checks == FH_CHECKS_HOST;
    p->weighted = false;  // a new peakmap starts with unit weights
    // the error word and the largest |D| share one allocation: one memset
    cudaError_t e = cudaMemsetAsync(p->err, 0, kErrWordsBytes, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
    if (pm->mem_kind == FH_MEM_HOST) {
        if (!pm->offsets || (n > 0 && !pm->t_fft) || (np > 0 && !pm->freq))
            return set_error(FH_ERR_INVALID_ARG, "null peakmap array");
        // With one direction every input array is read once, so page-locked
        // arrays are read in place by the kernels over the host link (no copy
        // in front of them); pageable arrays, and every array when several
        // directions would re-read it, are copied into the plan's buffers.
        const bool in_place = n_dir == 1;
        auto mapped = [&](const void *h, size_t bytes) -> const void * {
            return (in_place && bytes > 0) ? pinned_device_address(h) : nullptr;
        };
        const void *off_m = mapped(pm->offsets, 8 * ((size_t)n + 1));
        const void *t_m = mapped(pm->t_fft, 8 * (size_t)n);
        const void *f_m = mapped(pm->freq, 8 * (size_t)np);
        const void *v_m = mapped(v_over_c, 24 * (size_t)n);
        const void *sky_m = mapped(sky_n, 24 * (size_t)n_dir);
        // the copies are enqueued first, so that the host checks below run while
        // the inputs move; a failed check leaves the plan without a peakmap
        struct {
            void *dst;
            const void *src;
            size_t bytes;
        } cp[] = {{host_checks ? p->offsets : p->offsets_raw, pm->offsets,
                   off_m ? 0 : 8 * ((size_t)n + 1)},
                  {p->t, pm->t_fft, t_m ? 0 : 8 * (size_t)n},
                  {p->freq, pm->freq, f_m ? 0 : 8 * (size_t)np},
                  {p->v, v_over_c, v_m ? 0 : 24 * (size_t)n},
                  {p->sky, sky_n, sky_m ? 0 : 24 * (size_t)n_dir}};
        p->n_fft = -1;
        for (auto &c : cp) {
            if (c.bytes == 0) continue;
            e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(H2D inputs)");
        }
        if (host_checks) {
            int rc = validate_host_inputs(p->d, p->kt, pm, v_over_c, sky_n, n_dir);
            if (rc) return rc;
        }
        // the guard from the FFT times (the device checks of FH_CHECKS_DEVICE see the
        // rest); one that would not leave room for a tile falls back to the plan's
        // default, and the transform then takes its clamped walk if the drift is larger
        unsigned long long dr = std::max(default_drift(p->d), host_drift(p->d, p->kt, pm->t_fft, n));
        if (transform_smem_bytes(64, p->d.k_over, p->mode, p->block_warps, guard_for(dr)) >
            (size_t)max_optin_smem(p->device))
            dr = default_drift(p->d);
        p->drift = dr;
        p->guard = guard_for(dr);
        t_src = t_m ? static_cast<const double *>(t_m) : p->t;
        f_src = f_m ? static_cast<const double *>(f_m) : p->freq;
        v_src = v_m ? static_cast<const double *>(v_m) : p->v;
        sky_src = sky_m ? static_cast<const double *>(sky_m) : p->sky;
        offs_in_place = static_cast<const int64_t *>(off_m);
    } else {
        if (!pm->offsets || (n > 0 && !pm->t_fft) || (np > 0 && !pm->freq))
            return set_error(FH_ERR_INVALID_ARG, "null device peakmap array");
        // the FFT times are not seen on the host: the guards of the grid's own drift
        p->drift = default_drift(p->d);
        p->guard = default_guard(p->d);
        t_src = pm->t_fft;
        f_src = pm->freq;
        v_src = v_over_c;
        sky_src = sky_n;
    }
    const fh_plan_desc &d = p->d;
    // device checks: for device inputs, and for host inputs under FH_CHECKS_DEVICE
    const bool on_device = pm->mem_kind == FH_MEM_DEVICE || !host_checks;
    PrepArgs pa{};
    pa.offsets_in = pm->mem_kind == FH_MEM_DEVICE
                        ? pm->offsets
                        : (offs_in_place ? offs_in_place
                                         : (host_checks ? nullptr : p->offsets_raw));
    pa.offsets_out = p->offsets;
    pa.t = t_src;
    pa.v = v_src;
    pa.sky = sky_src;
    pa.n_fft = n;
    pa.n_dir = n_dir;
    pa.n_fdot = d.n_fdot;
    pa.validate = on_device ? 1 : 0;
    pa.n_peaks = np;
    pa.t_ref = d.t_ref;
    pa.kt = p->kt;
    pa.fdot_min = d.fdot_min;
    pa.fdot_step = d.fdot_step;
    pa.S0 = p->S0;
    pa.D = p->D;
    pa.dmax = p->dmax;
    pa.err = p->err;
    // a1 - a3 in one launch (the CSR pass, the shift tables and the positions of
    // every direction run side by side)
    e = launch_correct(pa, f_src, d.f0_min, d.k_over, p->A, out_r, s);
    if (e != cudaSuccess) return cuda_error(e, "correction launch");
    p->launches += (n > 0 || pa.offsets_in || pa.validate) ? 1 : 0;
    if (out_A && np > 0) {
        e = cudaMemcpyAsync(out_A, p->A, 8 * (size_t)np * n_dir, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(out_A)");
    }
    p->n_fft = n;
    p->n_peaks = np;
    p->n_dir = n_dir;
    return FH_OK;
}

// What an item of n_dir directions of the plan's current peakmap pairs in
// the shared counter words (pref 0: where it applies; 1: never): 0 nothing,
// 1 two directions, 2 (one direction) two 32-row halves of a 64-row slab.
enum : int32_t { kPairNone = 0, kPairDirs = 1, kPairRows = 2 };
static int32_t plan_pairs(fh_plan p, int32_t n_dir, int32_t pref)
{
    if (pref == 1 || p->mode != FH_MODE_START || p->weighted) return kPairNone;
    if (pairs_apply(p->d, p->device, p->n_fft, n_dir, p->drift)) return kPairDirs;
    if (rows_apply(p->d, p->device, p->n_fft, n_dir, p->drift)) return kPairRows;
    return kPairNone;
}

static int32_t plan_guard(fh_plan p, int32_t kind)
{
    return kind == kPairDirs   ? p->guard + pair_delta(p->d)
           : kind == kPairRows ? std::max(p->guard, guard_for(p->drift, 2 * kRows - 1))
                               : p->guard;
}

static int run_transform(fh_plan p, int32_t dir_begin, int32_t n_dir, int32_t *out_maps,
                         int32_t tile, int32_t nwarps, int32_t schedule, cudaStream_t s,
                         int32_t pair_pref, int32_t item_counter)
{
    const fh_plan_desc &d = p->d;
    // keep the tile's counters within shared memory with this plan's guard cells
    const int32_t kind = schedule != FH_SCHED_PLAIN ? plan_pairs(p, n_dir, pair_pref) : kPairNone;
    const bool pairs = kind == kPairDirs;
    const int32_t guard = plan_guard(p, kind);
    const int32_t wmax = default_tile(d, p->device, p->mode, nwarps, guard);
    if (tile > wmax) tile = wmax;
    const size_t smem = transform_smem_bytes(tile, d.k_over, p->mode, nwarps, guard);
    int rc = prepare_transform(p, p->mode, smem);
    if (rc) return rc;
    // the window pre-pass clears each direction's profile before the transform
    // merges into it; without FFTs there is no pre-pass, so clear it here
    cudaError_t e = cudaSuccess;
    if (p->n_fft <= 0)
        e = cudaMemsetAsync(p->profile + (int64_t)dir_begin * d.n_f0, 0,
                            sizeof(uint64_t) * (size_t)n_dir * d.n_f0, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(profile)");
    TransformJob job{};
    job.A = p->A;
    job.offsets = p->offsets;
    job.S0 = p->S0;
    job.D = p->D;
    job.profile = p->profile;
    job.dmax = p->dmax;
    job.err = p->err;
    job.weights = p->weighted ? p->wq : nullptr;
    job.count_bound = p->weighted ? p->w_bound : p->n_peaks;
    job.n_peaks = p->n_peaks;
    job.n_fft = p->n_fft;
    job.n_f0 = d.n_f0;
    job.n_fdot = d.n_fdot;
    job.k_over = d.k_over;
    job.tile_cells = tile;
    job.dir_pairs = pairs ? 1 : 0;
    job.row_pairs = kind == kPairRows ? 1 : 0;
    job.dense = p->dense;
    job.unit_delta = p->unit_delta;
    job.delta_alloc = pair_delta(d);
    const int32_t slab_rows = kind == kPairRows ? 2 * kRows : kRows;
    job.n_slabs = (d.n_fdot + slab_rows - 1) / slab_rows;
    job.n_tiles = (d.n_f0 + tile - 1) / tile;
    const int64_t per_dir = (int64_t)job.n_slabs * job.n_tiles;
    int bps = transform_blocks_per_sm(p->mode, nwarps, smem);
    if (bps < 1) return set_error(FH_ERR_CUDA, "transform kernel cannot be resident");
    // peak windows of a group of directions (bounded table), then the transform;
    // with direction pairs the table and the work items are per pair, and a group
    // holds whole pairs
    const size_t per_dir_win = sizeof(uint32_t) * (size_t)per_dir * (size_t)std::max(1, p->n_fft);
    const size_t win_cap = std::max(per_dir_win, (size_t)1 << 32);
    const int32_t per_unit = pairs ? 2 : 1;
    // (the windows grid has one block row per unit: at most 65535)
    const size_t zcap = 65535;
    int32_t group = schedule == FH_SCHED_PLAIN
                        ? 1
                        : (int32_t)std::max<size_t>(1, std::min<size_t>(
                              std::min<size_t>((size_t)n_dir, zcap),
                              per_unit * (win_cap / per_dir_win)));
    if (pairs && group < n_dir) group = std::max(2, group & ~1);
    const size_t need = per_dir_win * (size_t)((group + per_unit - 1) / per_unit);
    if (need > p->win_bytes) {
        if (p->win) cudaFree(p->win);
        p->win = nullptr;
        p->win_bytes = 0;
        e = cudaMalloc(&p->win, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(FH_ERR_NOMEM, "cudaMalloc of %zu bytes (peak windows) failed", need);
        }
        p->win_bytes = need;
    }
    JobTable tbl{};
    tbl.n_jobs = 1;
    for (int32_t g0 = 0; g0 < n_dir; g0 += group) {
        const int32_t gn = std::min(group, n_dir - g0);
        job.dir_begin = dir_begin + g0;
        job.n_dir = gn;
        job.maps = out_maps ? out_maps + (int64_t)g0 * d.n_fdot * d.n_f0 : nullptr;
        job.item_begin = 0;
        job.n_items = per_dir * ((gn + per_unit - 1) / per_unit);
        job.windows = p->win;
        if (pairs) {
            e = cudaMemsetAsync(p->unit_delta, 0, sizeof(int32_t) * (size_t)((gn + 1) / 2), s);
            if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(pair distances)");
        }
        cudaEvent_t *ev = nullptr;
        if (p->timing && !p->tev.empty()) {
            ev = &p->tev[3 * (size_t)(p->tev_next % kTimingSlots)];
            ++p->tev_next;
            cudaEventRecord(ev[0], s);
        }
        e = launch_windows(job, p->win, s);
        if (e != cudaSuccess) return cuda_error(e, "windows launch");
        ++p->launches;
        if (ev) cudaEventRecord(ev[1], s);
        tbl.job[0] = job;
        if (schedule == FH_SCHED_PLAIN) {
            // one sky direction per launch, one block per work item
            e = launch_transform(p->mode, tbl, job.n_items, (int32_t)job.n_items, nwarps, smem,
                                 guard, s);
        } else {
            const int64_t cap = (int64_t)p->n_sm * bps;
            const int32_t grid = (int32_t)std::min<int64_t>(job.n_items, cap);
            e = launch_transform(p->mode, tbl, job.n_items, grid, nwarps, smem, guard, s,
                                 item_counter ? p->sched : nullptr);
        }
        if (e != cudaSuccess) return cuda_error(e, "transform launch");
        ++p->launches;
        if (ev) cudaEventRecord(ev[2], s);
    }
    return FH_OK;
}

int fh_transform(fh_plan p, int32_t dir_begin, int32_t n_dir, int32_t *out_maps, void *stream)
{
    if (!p) return set_error(FH_ERR_INVALID_ARG, "null plan");
    int rc = check_dirs(p, dir_begin, n_dir);
    if (rc) return rc;
    DeviceGuard g(p->device);
    return run_transform(p, dir_begin, n_dir, out_maps, p->tile_cells, p->block_warps,
                         p->d.schedule, as_stream(stream), p->pair_pref, p->item_counter);
}

int fh_copy_profile(fh_plan p, int32_t dir_begin, int32_t n_dir, uint64_t *out, void *stream)
{
    if (!p || !out) return set_error(FH_ERR_INVALID_ARG, "null plan or out");
    int rc = check_dirs(p, dir_begin, n_dir);
    if (rc) return rc;
    DeviceGuard g(p->device);
    cudaError_t e = cudaMemcpyAsync(out, p->profile + (int64_t)dir_begin * p->d.n_f0,
                                    sizeof(uint64_t) * (size_t)n_dir * p->d.n_f0,
                                    cudaMemcpyDeviceToDevice, as_stream(stream));
    return e == cudaSuccess ? FH_OK : cuda_error(e, "cudaMemcpyAsync(profile)");
}

int fh_sync(fh_plan p, void *stream)
{
    if (!p) return set_error(FH_ERR_INVALID_ARG, "null plan");
    DeviceGuard g(p->device);
    cudaStream_t s = as_stream(stream);
    cudaError_t e = cudaMemcpyAsync(p->h_err, p->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "fh_sync");
    return device_error_code(*p->h_err);
}

int fh_select_candidates(fh_plan p, int32_t dir_begin, int32_t n_dir, fh_candidate *out,
                         int64_t capacity, int64_t *n_out, int32_t out_mem_kind, void *stream)
{
    if (!p || !n_out) return set_error(FH_ERR_INVALID_ARG, "null plan or n_out");
    int rc = check_dirs(p, dir_begin, n_dir);
    if (rc) return rc;
    if (out_mem_kind != FH_MEM_HOST && out_mem_kind != FH_MEM_DEVICE)
        return set_error(FH_ERR_INVALID_ARG, "unknown out_mem_kind");
    const fh_plan_desc &d = p->d;
    const int64_t need = (int64_t)n_dir * p->n_sb * d.top_k;
    *n_out = need;
    if (capacity < need || !out)
        return set_error(FH_ERR_CAPACITY, "need %lld candidate slots, capacity %lld",
                         (long long)need, (long long)capacity);
    DeviceGuard g(p->device);
    cudaStream_t s = as_stream(stream);
    SelectArgs a{};
    a.profile = p->profile;
    a.out = out_mem_kind == FH_MEM_DEVICE ? out : p->cand;
    a.n_f0 = d.n_f0;
    a.subband_cells = d.subband_cells;
    a.top_k = d.top_k;
    a.excl = d.excl_cells;
    a.sep = d.sep_cells;
    a.n_thr = d.n_thr;
    a.n_sb = p->n_sb;
    a.dir_begin = dir_begin;
    a.n_dir = n_dir;
    a.n_fft = p->n_fft;
    a.f0_min = d.f0_min;
    a.kt = p->kt;
    a.fdot_min = d.fdot_min;
    a.fdot_step = d.fdot_step;
    a.p0 = d.p0;
    a.s1 = p->weighted ? p->ws : nullptr;
    a.s2 = p->weighted ? p->ws + d.max_dir : nullptr;
    cudaError_t e = launch_select(a, s);
    if (e != cudaSuccess) return cuda_error(e, "select launch");
    ++p->launches;
    if (out_mem_kind == FH_MEM_DEVICE) return FH_OK;
    e = cudaMemcpyAsync(out, p->cand, sizeof(fh_candidate) * (size_t)need,
                        cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(candidates)");
    return fh_sync(p, stream);
}

}  // extern "C"

namespace {

// Autotuner results: (tile width, block warps, direction pairs) per grid shape,
// kept in memory for the process and, when FH_AUTOTUNE_CACHE names a file, in
// that JSON file (one entry per line, rewritten atomically by rename) so that
// later processes on the same GPU model reuse them.
struct TuneChoice {
    int32_t tile = 0, warps = 0, pairs = 0, counter = 1;
    double ms = 0.0;
};
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;
bool g_tune_loaded = false;

const char *tune_path() { return std::getenv("FH_AUTOTUNE_CACHE"); }

void tune_load_locked()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = tune_path();
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (std::fgets(line, sizeof line, f)) {
        const char *k = std::strstr(line, "\"key\": \"");
        if (!k) continue;
        k += 8;
        const char *ke = std::strchr(k, '"');
        if (!ke) continue;
        TuneChoice c;
        const char *t = std::strstr(ke, "\"tile_cells\": ");
        const char *w = std::strstr(ke, "\"block_warps\": ");
        const char *r = std::strstr(ke, "\"dir_pairs\": ");
        const char *m = std::strstr(ke, "\"ms\": ");
        const char *ic = std::strstr(ke, "\"item_counter\": ");
        if (!t || !w || !r || std::sscanf(t + 14, "%d", &c.tile) != 1 ||
            std::sscanf(w + 15, "%d", &c.warps) != 1 || std::sscanf(r + 13, "%d", &c.pairs) != 1)
            continue;
        if (m) std::sscanf(m + 6, "%lf", &c.ms);
        if (ic && std::sscanf(ic + 16, "%d", &c.counter) != 1) continue;
        if (c.tile < 32 || (c.warps != 16 && c.warps != 20 && c.warps != 24 && c.warps != 32) ||
            (c.pairs != 0 && c.pairs != 1) || (c.counter != 0 && c.counter != 1))
            continue;  // not one of ours: ignored
        g_tune[std::string(k, ke)] = c;
    }
    std::fclose(f);
}

void tune_store_locked()
{
    const char *path = tune_path();
    if (!path || !*path) return;
    const std::string tmp = std::string(path) + ".tmp." + std::to_string((long long)getpid());
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\"version\": 1, \"entries\": [\n");
    size_t k = 0;
    for (const auto &e : g_tune) {
        std::fprintf(f,
                     "{\"key\": \"%s\", \"tile_cells\": %d, \"block_warps\": %d, "
                     "\"dir_pairs\": %d, \"item_counter\": %d, \"ms\": %.6f}%s\n",
                     e.first.c_str(), e.second.tile, e.second.warps, e.second.pairs,
                     e.second.counter, e.second.ms, ++k < g_tune.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    const bool ok = std::fclose(f) == 0;
    if (ok) std::rename(tmp.c_str(), path);
    else std::remove(tmp.c_str());
}

}  // namespace

extern "C" {

int fh_autotune(fh_plan p, int32_t dir_begin, int32_t n_dir, int32_t *tile_cells,
                int32_t *block_warps, void *stream)
{
    if (!p) return set_error(FH_ERR_INVALID_ARG, "null plan");
    int rc = check_dirs(p, dir_begin, n_dir);
    if (rc) return rc;
    DeviceGuard g(p->device);
    cudaStream_t s = as_stream(stream);
    const fh_plan_desc &d = p->d;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) {
        cudaGetLastError();
        std::strcpy(prop.name, "gpu");
    }
    for (char *c = prop.name; *c; ++c)
        if (*c == '"' || *c == '\\' || *c == ' ') *c = '_';
    // the grid shape: (n_f0, n_fdot, K, T_FFT, N_t, n_dir), with the counting
    // mode, the weighting and the GPU model
    char key[512];
    std::snprintf(key, sizeof key, "%s|mode%d|w%d|n_f0=%d|n_fdot=%d|K=%d|T=%.17g|n_fft=%d|n_dir=%d",
                  prop.name, p->mode, p->weighted ? 1 : 0, d.n_f0, d.n_fdot, d.k_over, d.t_fft,
                  p->n_fft, n_dir);
    auto apply = [&](const TuneChoice &c) {
        p->tile_cells = c.tile;
        p->block_warps = c.warps;
        p->pair_pref = c.pairs ? 0 : 1;
        p->item_counter = c.counter;
        if (tile_cells) *tile_cells = p->tile_cells;
        if (block_warps) *block_warps = p->block_warps;
    };
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            apply(it->second);
            return FH_OK;
        }
    }
    // candidates: pairs (of directions, or of a single direction's row halves;
    // where they apply) or not, block warps, tile widths up to the widest that
    // fits with that choice's guard cells
    const int lim = max_optin_smem(p->device);
    std::vector<TuneChoice> cands;
    const int32_t nt = std::min<int32_t>(n_dir, 8);
    const int32_t pair_kind = plan_pairs(p, nt, 0);
    const bool pairs_ok = pair_kind != kPairNone;
    for (int pr : {1, 0}) {
        if (pr && !pairs_ok) continue;
        const int32_t guard = plan_guard(p, pr ? pair_kind : kPairNone);
        for (int nw : {24, 20, 32, 16}) {
            // DIFF kernels: 512 / 1024 threads
            if ((nw == 24 || nw == 20) && p->mode == FH_MODE_DIFF) continue;
            const int32_t wmax = default_tile(d, p->device, p->mode, nw, guard);
            for (int32_t w : {wmax, 1280, 1024, 768}) {
                if (w > wmax || w > d.n_f0) continue;
                if (transform_smem_bytes(w, d.k_over, p->mode, nw, guard) > (size_t)lim) continue;
                bool dup = false;
                for (const auto &c : cands) dup = dup || (c.tile == w && c.warps == nw && c.pairs == pr);
                if (!dup) cands.push_back({w, nw, pr, 1, 0.0});
            }
        }
    }
    if (cands.empty()) cands.push_back({p->tile_cells, p->block_warps, 0, 1, 0.0});
    // timed on at most 8 of the directions (one window group): the per-item
    // work, and so the best tile, does not depend on how many there are
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    TuneChoice pick = cands[0];
    auto time_choice = [&](TuneChoice &c) {
        const int32_t pref = c.pairs ? 0 : 1;
        rc = run_transform(p, dir_begin, nt, nullptr, c.tile, c.warps, FH_SCHED_BATCHED, s, pref,
                           c.counter);
        if (rc) return;
        float ms = 0.f;
        for (int reps = 1; reps <= 4 && rc == FH_OK; reps *= 4) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && rc == FH_OK; ++r)
                rc = run_transform(p, dir_begin, nt, nullptr, c.tile, c.warps, FH_SCHED_BATCHED,
                                   s, pref, c.counter);
            cudaEventRecord(e1, s);
            if (rc) break;
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)reps;
            if (ms > 5.0f) break;  // long enough to time once
        }
        c.ms = ms;
        if (rc == FH_OK && ms < best) {
            best = ms;
            pick = c;
        }
    };
    for (auto &c : cands) {
        time_choice(c);
        if (rc) break;
    }
    // the item schedule of the fastest shape: the counter, or every grid-th item
    // per block (no counter round trip per item; better balanced only when the
    // items cost alike)
    if (rc == FH_OK) {
        TuneChoice c = pick;
        c.counter = 0;
        time_choice(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    apply(pick);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = pick;
        tune_store_locked();
    }
    return FH_OK;
}

int fh_bench_fp64(int32_t iters, double *ops_per_s, double *ms, void *stream)
{
    if (!ops_per_s || iters < 1) return set_error(FH_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = as_stream(stream);
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    double *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(double));
    if (e != cudaSuccess) return set_error(FH_ERR_NOMEM, "cudaMalloc(sink)");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = n_sm * 4;  // 4 blocks of 512 threads per SM
    e = launch_fp64_bench(std::max(1, iters / 8), grid, sink, s);  // warm-up
    cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_fp64_bench(iters, grid, sink, s);
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_error(e, "fp64 bench");
    *ops_per_s = (double)grid * 512.0 * 16.0 * (double)iters / ((double)t * 1e-3);
    if (ms) *ms = t;
    return FH_OK;
}

int fh_bench_smem_atomics(int32_t variant, int32_t iters, double *atomics_per_s, double *ms,
                          void *stream)
{
    if (!atomics_per_s || iters < 1 || variant < 0 || variant > 1)
        return set_error(FH_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = as_stream(stream);
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    unsigned long long *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(unsigned long long));
    if (e != cudaSuccess) return set_error(FH_ERR_NOMEM, "cudaMalloc(sink)");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = n_sm * 2;
    e = launch_smem_atomic_bench(variant, std::max(1, iters / 8), grid, sink, s);  // warm-up
    cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_smem_atomic_bench(variant, iters, grid, sink, s);
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_error(e, "smem atomic bench");
    *atomics_per_s = (double)grid * 1024.0 * 8.0 * (double)iters / ((double)t * 1e-3);
    if (ms) *ms = t;
    return FH_OK;
}

}  // extern "C"
