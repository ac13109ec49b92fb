// Internal declarations of libfh (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "fh.h"

namespace fh {

// Spin-down rows per slab: one row per lane of a warp.  The transform's
// shared-memory histogram is laid out [cell][row] with a row stride of 32
// words, so lane l (row l) always hits bank l and the +1 atomics of one warp
// instruction never conflict, wherever the 32 stripes start.
constexpr int kRows = 32;
constexpr int kMaxBatchJobs = 12;
constexpr int64_t kFixedLimit = int64_t(1) << 28;  // |cells| bound for 32.32 fixed point

// error bits written by the device-side input checks
enum : int32_t { kErrUnsorted = 1, kErrRange = 2, kErrInvalid = 4, kErrCsr = 8 };

// One direction set of one plan, as the transform kernel sees it.
struct TransformJob {
    const int64_t *A;        // positions, [dir][n_peaks] (absolute directions)
    const int64_t *offsets;  // n_fft + 1, valid CSR
    const int64_t *S0;       // n_fft
    const int64_t *D;        // n_fft
    uint64_t *profile;       // [dir][n_f0] (absolute directions)
    int32_t *maps;           // nullable, [dir - dir_begin][n_fdot][n_f0]
    int64_t n_peaks;
    int64_t item_begin;      // first work item of this job in the launch
    int64_t n_items;         // n_dir * n_slabs * n_tiles
    int32_t n_fft, n_f0, n_fdot, k_over;
    int32_t tile_cells;      // W
    int32_t n_slabs, n_tiles;
    int32_t dir_begin, n_dir;
};

struct JobTable {
    int32_t n_jobs;
    TransformJob job[kMaxBatchJobs];
};

struct SelectArgs {
    const uint64_t *profile; // [dir][n_f0]
    fh_candidate *out;       // [dir - dir_begin][n_sb][top_k]
    int32_t n_f0, subband_cells, top_k, excl, sep, n_thr, n_sb;
    int32_t dir_begin, n_dir, n_fft;
    double f0_min, kt, fdot_min, fdot_step, p0;
};

// ---- launchers (fh_kernels.cu); all return cudaGetLastError() ----
cudaError_t launch_shift_tables(const double *t, int32_t n_fft, double t_ref, double kt,
                                double fdot_min, double fdot_step, int32_t n_fdot,
                                int64_t *S0, int64_t *D, int32_t *err, cudaStream_t s);
cudaError_t launch_positions(const double *freq, const int64_t *offsets, const double *v,
                             const double *sky, int32_t n_fft, int64_t n_peaks, int32_t n_dir,
                             double f0_min, double kt, int32_t k_over, int64_t *A,
                             double *out_r, int32_t *err, cudaStream_t s);
cudaError_t launch_sanitize_offsets(const int64_t *in, int32_t n_fft, int64_t n_peaks,
                                    int64_t *out, int32_t *err, cudaStream_t s);
cudaError_t launch_validate_device_inputs(const double *t, const double *freq,
                                          const int64_t *offsets, const double *v,
                                          const double *sky, int32_t n_fft, int32_t n_dir,
                                          int32_t *err, cudaStream_t s);
// smem bytes the transform needs for tile width W (and mode)
size_t transform_smem_bytes(int32_t tile_cells, int32_t k_over, int32_t mode, int32_t nwarps);
cudaError_t transform_prepare(int32_t mode, size_t smem);  // opt-in dynamic smem
cudaError_t launch_transform(int32_t mode, const JobTable &tbl, int64_t total_items,
                             int32_t grid, int32_t nwarps, size_t smem, cudaStream_t s);
int transform_blocks_per_sm(int32_t mode, int32_t nwarps, size_t smem);
cudaError_t launch_select(const SelectArgs &a, cudaStream_t s);
cudaError_t launch_smem_atomic_bench(int32_t variant, int32_t iters, int32_t grid,
                                     unsigned long long *sink, cudaStream_t s);

// ---- host helpers (fh_api.cu) ----
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
int max_optin_smem(int device);
int32_t default_tile(const fh_plan_desc &d, int device, int32_t mode, int32_t nwarps);
int validate_desc(const fh_plan_desc &d);
// host-memory inputs: CSR, ordering, finiteness and the 32.32 fixed-point range
int validate_host_inputs(const fh_plan_desc &d, double kt, const fh_peakmap *pm, const double *v,
                         const double *sky, int32_t n_dir);

}  // namespace fh
