// fh_search_static: the whole hot path for one sky direction without any
// device allocation.
//
// Some callers cannot allocate device memory while they run: an application
// that reserves all of the GPU's memory up front for its own pool (so a
// cudaMalloc from a library would fail or would have to be carved out of
// their budget), or one that must not take the implicit device-wide
// synchronisation a cudaMalloc/cudaFree can cause in the middle of a latency
// sensitive loop.  For them this entry point keeps its working memory -- the
// sanitised CSR offsets, the spin-down shift tables, the fixed-point peak
// positions, the per-cell profile and an error word -- in one file-scope
// __device__ array of fixed size.  Every GPU that loads this part of the
// library holds that array until the process exits.
//
// The array's host-side name is only a handle: host code never passes it to a
// kernel.  The device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached for the life of
// the process (the primary context is assumed to live as long).  This file
// has no kernels, so it is a module of its own: under lazy module loading the
// first lookup on a device is when the driver loads it and commits the array's
// device memory; later calls take none.
#include <cstring>
#include <mutex>

#include "fh_internal.h"

using namespace fh;

namespace {

constexpr int64_t kStaticMaxPeaks = int64_t(1) << 21;  // 2,097,152 peaks
constexpr int32_t kStaticMaxFft = 1 << 16;              // 65,536 FFTs
constexpr int32_t kStaticMaxCells = 1 << 18;            // 262,144 frequency cells

constexpr size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t kOffOffsets = 0;
constexpr size_t kOffS0 = kOffOffsets + round256(8 * ((size_t)kStaticMaxFft + 1));
constexpr size_t kOffD = kOffS0 + round256(8 * (size_t)kStaticMaxFft);
constexpr size_t kOffA = kOffD + round256(8 * (size_t)kStaticMaxFft);
constexpr size_t kOffProfile = kOffA + round256(8 * (size_t)kStaticMaxPeaks);
constexpr size_t kOffErr = kOffProfile + round256(8 * (size_t)kStaticMaxCells);
constexpr size_t kOffDmax = kOffErr + 256;
constexpr size_t kScratchBytes = kOffDmax + 256;

static __device__ __align__(256) unsigned char g_fh_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int scratch_for_current_device(unsigned char **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(FH_ERR_INVALID_ARG, "device index %d", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fh_static_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return FH_OK;
}

}  // namespace

extern "C" {

int fh_search_static(const fh_plan_desc *desc, const fh_peakmap *pm, const double *v_over_c,
                     const double *sky_n, fh_candidate *out, int64_t capacity, int64_t *n_out,
                     int32_t *device_status, void *stream)
{
    if (!desc || !pm || !sky_n || !out || !n_out)
        return set_error(FH_ERR_INVALID_ARG, "null desc, peakmap, sky_n, out or n_out");
    fh_plan_desc d = *desc;
    d.max_fft = pm->n_fft > 0 ? pm->n_fft : 1;
    d.max_dir = 1;
    d.max_peaks = pm->n_peaks > 0 ? pm->n_peaks : 1;
    int rc = validate_desc(d);
    if (rc) return rc;
    if (pm->mem_kind != FH_MEM_DEVICE)
        return set_error(FH_ERR_INVALID_ARG, "fh_search_static takes device-memory inputs");
    if (pm->n_fft < 0 || pm->n_peaks < 0)
        return set_error(FH_ERR_INVALID_ARG, "negative n_fft or n_peaks");
    if (pm->n_fft > kStaticMaxFft || pm->n_peaks > kStaticMaxPeaks || d.n_f0 > kStaticMaxCells)
        return set_error(FH_ERR_TOO_LARGE,
                         "fh_search_static handles at most %d FFTs, %lld peaks and %d frequency "
                         "cells (got %d, %lld, %d)",
                         kStaticMaxFft, (long long)kStaticMaxPeaks, kStaticMaxCells, pm->n_fft,
                         (long long)pm->n_peaks, d.n_f0);
    if (!pm->offsets || (pm->n_fft > 0 && (!pm->t_fft || !v_over_c)) ||
        (pm->n_peaks > 0 && !pm->freq))
        return set_error(FH_ERR_INVALID_ARG, "null device peakmap array");
    const int32_t n_sb = (d.n_f0 + d.subband_cells - 1) / d.subband_cells;
    const int64_t need = (int64_t)n_sb * d.top_k;
    *n_out = need;
    if (capacity < need)
        return set_error(FH_ERR_CAPACITY, "need %lld candidate slots, capacity %lld",
                         (long long)need, (long long)capacity);

    unsigned char *base = nullptr;
    rc = scratch_for_current_device(&base);
    if (rc) return rc;
    int64_t *offsets = reinterpret_cast<int64_t *>(base + kOffOffsets);
    int64_t *S0 = reinterpret_cast<int64_t *>(base + kOffS0);
    int64_t *D = reinterpret_cast<int64_t *>(base + kOffD);
    int64_t *A = reinterpret_cast<int64_t *>(base + kOffA);
    uint64_t *profile = reinterpret_cast<uint64_t *>(base + kOffProfile);
    int32_t *err = reinterpret_cast<int32_t *>(base + kOffErr);
    unsigned long long *dmax = reinterpret_cast<unsigned long long *>(base + kOffDmax);

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int32_t n = pm->n_fft;
    const int64_t np = pm->n_peaks;
    const double kt = (double)d.k_over * d.t_fft;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);

    // the array keeps the previous call's contents: clear what must start at zero
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(profile, 0, sizeof(uint64_t) * (size_t)d.n_f0, s);
    PrepArgs pa{};
    pa.offsets_in = pm->offsets;
    pa.offsets_out = offsets;
    pa.t = pm->t_fft;
    pa.v = v_over_c;
    pa.sky = sky_n;
    pa.n_fft = n;
    pa.n_dir = 1;
    pa.n_fdot = d.n_fdot;
    pa.validate = 1;
    pa.n_peaks = np;
    pa.t_ref = d.t_ref;
    pa.kt = kt;
    pa.fdot_min = d.fdot_min;
    pa.fdot_step = d.fdot_step;
    pa.S0 = S0;
    pa.D = D;
    pa.dmax = dmax;
    pa.err = err;
    if (e == cudaSuccess) e = launch_correct(pa, pm->freq, d.f0_min, d.k_over, A, nullptr, s);
    if (e != cudaSuccess) return cuda_error(e, "fh_search_static set-up");

    const int32_t mode = d.mode == FH_MODE_DIFF ? FH_MODE_DIFF : FH_MODE_START;
    const int32_t nwarps = d.block_warps ? d.block_warps : 32;
    const int32_t guard = default_guard(d);
    int32_t tile = d.tile_cells ? (d.tile_cells < d.n_f0 ? d.tile_cells : d.n_f0)
                                : default_tile(d, dev, mode, nwarps, guard);
    const size_t smem = transform_smem_bytes(tile, d.k_over, mode, nwarps, guard);
    if (smem > (size_t)max_optin_smem(dev))
        return set_error(FH_ERR_INVALID_ARG, "tile_cells too wide for shared memory");
    e = transform_prepare(mode, smem);
    if (e != cudaSuccess) return cuda_error(e, "transform_prepare");
    JobTable tbl{};
    tbl.n_jobs = 1;
    TransformJob &job = tbl.job[0];
    job.A = A;
    job.offsets = offsets;
    job.S0 = S0;
    job.D = D;
    job.profile = profile;
    job.maps = nullptr;
    job.windows = nullptr;  // no window table in the fixed scratch: binary search
    job.dmax = dmax;
    job.err = err;
    job.weights = nullptr;
    job.count_bound = np;
    job.n_peaks = np;
    job.item_begin = 0;
    job.n_fft = n;
    job.n_f0 = d.n_f0;
    job.n_fdot = d.n_fdot;
    job.k_over = d.k_over;
    job.tile_cells = tile;
    job.n_slabs = (d.n_fdot + kRows - 1) / kRows;
    job.n_tiles = (d.n_f0 + tile - 1) / tile;
    job.dir_begin = 0;
    job.n_dir = 1;
    job.n_items = (int64_t)job.n_slabs * job.n_tiles;
    const int bps = transform_blocks_per_sm(mode, nwarps, smem);
    if (bps < 1) return set_error(FH_ERR_CUDA, "transform kernel cannot be resident");
    const int64_t cap = (int64_t)n_sm * bps;
    const int32_t grid = (int32_t)(job.n_items < cap ? job.n_items : cap);
    e = launch_transform(mode, tbl, job.n_items, grid, nwarps, smem, guard, s);
    if (e != cudaSuccess) return cuda_error(e, "transform launch");

    SelectArgs a{};
    a.profile = profile;
    a.out = out;
    a.n_f0 = d.n_f0;
    a.subband_cells = d.subband_cells;
    a.top_k = d.top_k;
    a.excl = d.excl_cells;
    a.sep = d.sep_cells;
    a.n_thr = d.n_thr;
    a.n_sb = n_sb;
    a.dir_begin = 0;
    a.n_dir = 1;
    a.n_fft = n;
    a.f0_min = d.f0_min;
    a.kt = kt;
    a.fdot_min = d.fdot_min;
    a.fdot_step = d.fdot_step;
    a.p0 = d.p0;
    e = launch_select(a, s);
    if (e == cudaSuccess && device_status)
        e = cudaMemcpyAsync(device_status, err, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "fh_search_static select");
    return FH_OK;
}

}  // extern "C"
