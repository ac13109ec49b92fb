// Internal declarations of libfh (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fh.h"

namespace fh {

// Spin-down rows per slab: one row per lane of a warp.  The transform's
// shared-memory histogram is laid out [cell][row] with a row stride of 32
// words, so lane l (row l) always hits bank l and the +1 atomics of one warp
// instruction never conflict, wherever the 32 stripes start.
constexpr int kRows = 32;
constexpr int kMaxBatchJobs = 12;
constexpr int64_t kFixedLimit = int64_t(1) << 28;  // |cells| bound for 32.32 fixed point
// window table entry of an FFT whose window start or count does not fit 16 bits:
// the transform looks that window up by binary search instead
constexpr uint32_t kWinLookup = 0xFFFFFFFFu;

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
    const unsigned long long *dmax;  // max_i |D_i| (32.32 cells per row), from a3
    const int32_t *err;      // the job's device error word: the unclamped walk, which
                             // trusts the peak windows (sorted positions), runs only
                             // while it is 0
    const int32_t *weights;  // nullable (plain map): adaptive integer weights, [dir][n_fft]
                             // (absolute directions); each update adds its FFT's weight
    int64_t count_bound;     // no count of the job's maps exceeds it
    const uint32_t *windows; // nullable: precomputed peak windows per
                             // [dir - dir_begin][slab][tile][fft], each the first peak
                             // relative to the FFT's first (low 16 bits) and the count
                             // (high 16 bits), or kWinLookup: looked up (binary search)
    int32_t *dense;          // nullable: set by the window pre-pass when some FFT has two
                             // peaks within one cell (the packed counters then do not
                             // apply: each direction of a pair is walked on its own)
    int32_t dir_pairs;       // 1: items cover directions 2u and 2u + 1 with two 16-bit
                             // counts per shared word (plain START map, every job of a
                             // launch alike); the window table is per pair
    int32_t *unit_delta;     // (dir_pairs) per pair, the largest cell distance between a
                             // peak's two positions (+2), from the window pre-pass
    int32_t delta_alloc;     // (dir_pairs) the part of the guard that holds that distance;
                             // a pair beyond it takes the clamped walk
    int32_t row_pairs;       // 1 (plain START map of one direction, not with dir_pairs):
                             // slabs of 64 rows, rows j0 + r and j0 + 32 + r in the low and
                             // high halves of one shared word; the window table is per
                             // 64-row slab and the guard holds 63 rows of drift
    int64_t n_peaks;
    int64_t item_begin;      // first work item of this job in the launch
    int64_t n_items;         // units * n_slabs * n_tiles
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
    const int64_t *s1, *s2;  // nullable (plain map): per absolute direction, sums of the
                             // adaptive weights and of their squares
};

// ---- launchers (fh_kernels.cu); all return cudaGetLastError() ----
// Per-call set-up in one block: (a) if offsets_in is given, the sanitised
// CSR copy of it (clamped to [0, n_peaks], non-decreasing, first 0, last
// n_peaks; kErrCsr if anything changed); (b) the spin-down shift tables S0, D
// of every FFT and the largest |D| (atomicMax into *dmax, which starts at 0);
// (c) if validate: t finite and strictly increasing, |v| < 0.1 componentwise,
// sky components within 1.000001.
struct PrepArgs {
    const int64_t *offsets_in;  // device CSR to sanitise, or null (offsets_out already valid)
    int64_t *offsets_out;
    const double *t, *v, *sky;
    int32_t n_fft, n_dir, n_fdot, validate;
    int64_t n_peaks;
    double t_ref, kt, fdot_min, fdot_step;
    int64_t *S0, *D;
    unsigned long long *dmax;
    int32_t *err;
};
cudaError_t launch_prep(const PrepArgs &a, cudaStream_t s);
// a1 - a3 in one launch: prep's work (a.offsets_in sanitised into
// a.offsets_out, shift tables, checks) and the positions of every (direction,
// peak) of the peakmap described by a, frequencies freq
cudaError_t launch_correct(const PrepArgs &a, const double *freq, double f0_min,
                           int32_t k_over, int64_t *A, double *out_r, cudaStream_t s);

// fh_refine on the plan's grid d (host inputs, host output; synchronises)
int refine_impl(const fh_plan_desc &d, int n_sm, const fh_peakmap *pm, const double *v_over_c,
                const int32_t *cand_cell, const int32_t *cand_row, int32_t n_cand,
                const double *sky_ref, int32_t n_ref, int32_t k_fdot, fh_candidate *out,
                bool host_checks, cudaStream_t s);
// the error of a device error word (0: FH_OK)
int device_error_code(int32_t bits);
// positions of n_batch peakmaps (refinement): batch c has offsets
// offsets + c (n_fft + 1), source index src + c n_fft, sky + 3 c n_dir, its peak
// count n_peaks[c] (device) and its positions at A + a_base[c] (device),
// direction-major ([direction][peak] within each batch)
cudaError_t launch_positions_batched(const double *freq, const int64_t *offsets,
                                     const double *v, const double *sky, int32_t n_fft,
                                     int32_t n_dir, int32_t n_batch, const int64_t *a_base,
                                     const int64_t *n_peaks, double f0_min, double kt,
                                     int32_t k_over, int64_t *A, int32_t *err, bool validate,
                                     const int64_t *src, cudaStream_t s);
cudaError_t launch_validate_device_inputs(const double *t, const double *freq,
                                          const int64_t *offsets, const double *v,
                                          const double *sky, int32_t n_fft, int32_t n_dir,
                                          int32_t *err, cudaStream_t s);
// Guard cells kept below and above a tile so that, in the fast path, no
// update of a slab needs a bounds clamp: enough for a drift of span_rows (the
// slab's rows - 1) x max|D| cells.  guard_for(dmax, rows - 1) is what a job
// needs; a launch allocates one guard for all its jobs and jobs needing more
// take the clamped path.
__host__ __device__ int32_t guard_for(unsigned long long dmax, int32_t span_rows = kRows - 1);
// smem bytes the transform needs for tile width W (and mode)
size_t transform_smem_bytes(int32_t tile_cells, int32_t k_over, int32_t mode, int32_t nwarps,
                            int32_t guard);
cudaError_t transform_prepare(int32_t mode, size_t smem);  // opt-in dynamic smem
// sched: null (every block takes every grid-th item) or two device words that
// are zero at the launch (a counter handing out items after each block's
// first, and a count of finished blocks); the kernel's last block zeroes them
// again, so launches on one stream can share them (not concurrent launches).
cudaError_t launch_transform(int32_t mode, const JobTable &tbl, int64_t total_items,
                             int32_t grid, int32_t nwarps, size_t smem, int32_t guard,
                             cudaStream_t s, unsigned int *sched = nullptr);
int transform_blocks_per_sm(int32_t mode, int32_t nwarps, size_t smem);
// Peak windows of every (direction, slab, tile, FFT) of a job, written to
// job.windows (the job's other fields as for the transform).
cudaError_t launch_windows(const TransformJob &job, uint32_t *windows, cudaStream_t s);
cudaError_t launch_select(const SelectArgs &a, cudaStream_t s);
// Adaptive map's count bound: bound[d] += sum_i W[d][i] c_{d,i}, c_{d,i} = the
// most positions of FFT i (direction d) inside a half-open window of K cells
// (bound: n_dir words, zeroed by the caller).
cudaError_t launch_weight_bound(const int64_t *A, const int64_t *offsets, const int32_t *W,
                                int32_t n_fft, int32_t n_dir, int64_t n_peaks, int32_t k_over,
                                unsigned long long *bound, cudaStream_t s);
// binary64 multiply + add chains, grid blocks of 512 threads, 16 operations
// per thread per iteration
cudaError_t launch_fp64_bench(int32_t iters, int32_t grid, double *sink, cudaStream_t s);
cudaError_t launch_smem_atomic_bench(int32_t variant, int32_t iters, int32_t grid,
                                     unsigned long long *sink, cudaStream_t s);

// Exclusive scan of n int32 counts into int64 (one block): pref[0 .. n] (may be
// null) and strided[r] = pref[r * stride] for r = 0 .. n / stride (may be null).
cudaError_t launch_exclusive_scan(const int32_t *cnt, int64_t n, int64_t *pref, int32_t stride,
                                  int64_t *strided, cudaStream_t s);

// Device buffers of one call, taken stream-ordered (cudaMallocAsync) and
// returned stream-ordered when the object goes out of scope.
struct Scratch {
    cudaStream_t s;
    std::vector<void *> bufs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    template <typename T>
    cudaError_t get(T **p, size_t n)
    {
        void *q = nullptr;
        const cudaError_t e = cudaMallocAsync(&q, (n ? n : 1) * sizeof(T), s);
        if (e == cudaSuccess) bufs.push_back(q);
        *p = static_cast<T *>(q);
        return e;
    }
    ~Scratch()
    {
        for (void *b : bufs) cudaFreeAsync(b, s);
    }
};

// ---- host helpers (fh_api.cu) ----
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
int max_optin_smem(int device);
int32_t default_tile(const fh_plan_desc &d, int device, int32_t mode, int32_t nwarps,
                     int32_t guard);
// guard for a plan when the FFT times are not known on the host: the drift of
// a grid with fdot_step = 1/(T_FFT T_obs) over +-T_obs/2 is K/2 cells per row
int32_t default_guard(const fh_plan_desc &d);
// guard for FFT start times held in host memory (exact drift of the grid)
int32_t host_guard(const fh_plan_desc &d, double kt, const double *t, int32_t n_fft);
// the drift bounds behind those guards: max |D_i| in 32.32 cells per row
unsigned long long default_drift(const fh_plan_desc &d);
unsigned long long host_drift(const fh_plan_desc &d, double kt, const double *t, int32_t n_fft);
// Whether a plain START map of n_dir directions may pair them (two 16-bit
// counts per shared word): its stripe-start counts fit 16 bits by its size
// (n_fft < 2^16; the window pre-pass checks the peaks' spacing), its counts
// keep the reduction key below 2^31 (K n_fft < 2^25) and a tile fits with the
// guard of drift bound `drift` plus the pair allowance pair_delta(d).
bool pairs_apply(const fh_plan_desc &d, int device, int32_t n_fft, int32_t n_dir,
                 unsigned long long drift);
// Whether one direction (n_dir == 1) of a plain START map may pair the two
// 32-row halves of 64-row slabs in the counters' 16-bit halves: the same
// 16-bit and key conditions as for direction pairs, and a tile fits with the
// guard of 63 rows of drift.
bool rows_apply(const fh_plan_desc &d, int device, int32_t n_fft, int32_t n_dir,
                unsigned long long drift);
// Cells of guard kept for the distance between a peak's positions in the two
// directions of a pair: neighbouring directions of a sky grid at the Doppler
// resolution differ by about one input bin (K cells); 2 K + 4 leaves room.
int32_t pair_delta(const fh_plan_desc &d);
int validate_desc(const fh_plan_desc &d);
// host-memory inputs: CSR, ordering, finiteness and the 32.32 fixed-point range
int validate_host_inputs(const fh_plan_desc &d, double kt, const fh_peakmap *pm, const double *v,
                         const double *sky, int32_t n_dir);

}  // namespace fh
