/*
 * fh.h -- C ABI of the GB300 frequency-Hough (FH) library (libfh.so).
 *
 * The FH transform (Astone et al., arXiv:1407.8333, Sec. VI) maps a
 * time-frequency peakmap, Doppler-corrected for one sky direction, into the
 * source frequency / spin-down plane: each peak (t_i, f) becomes a stripe of
 * the line f0 = f - fdot (t_i - t0) (Eq. uno), one input bin wide (Eq. due),
 * on a frequency axis over-resolved by K (Eq. freqres), and every cell the
 * stripe touches gains one count (Eq. ncount).  Candidates are then taken per
 * frequency sub-band over all spin-down rows (Sec. VIII).
 *
 * Numerical definition (bit-exact contract; all floating point is IEEE-754
 * binary64, round-to-nearest-even, one rounding per operation, no fused
 * multiply-add):
 *   a1  r[d][i] = 1 / (1 + ((v_x n_x + v_y n_y) + v_z n_z))          (Eq. fdopp)
 *   a2  A[d][p] = floor(((f_p r[d][i] - f0_min) * KT + (0.5 - 0.5 K)) * 2^32)
 *       with KT = K * T_FFT; a stripe covers the K cells whose centres lie in
 *       (x - K/2, x + K/2], x = the corrected frequency in cell units.
 *   a3  c_i = (t_i - t_ref) * KT;  S0[i] = floor((fdot_min c_i) 2^32);
 *       D[i] = floor((fdot_step c_i) 2^32)                    (Eqs. uno, sdstep)
 *   a4  s = floor((A[d][p] - (S0[i] + j D[i])) / 2^32): first cell of the
 *       stripe of peak p on spin-down row j; cells [s, s + K) clipped to
 *       [0, n_f0) each get +1
 *   a5  count[d][j][b] = number of (peak) stripes covering cell b on row j
 *   a6  profile[b] = max_j count[j][b] (smallest such j); per sub-band of
 *       subband_cells cells, up to top_k greedy picks by (count desc, row asc,
 *       cell asc), each outside +-excl_cells of earlier picks, stopping at a
 *       count < n_thr or a pick closer than sep_cells to an earlier one.
 * Cell b covers [f0_min + b/KT, f0_min + (b + 1)/KT); row j has
 * fdot_j = fdot_min + j * fdot_step.
 *
 * Conventions.  Every function returns an int status (FH_OK or a negative
 * FH_ERR_*) and never aborts; fh_last_error() gives a thread-local message.
 * Streams are cudaStream_t values passed as void* (NULL = the legacy default
 * stream).  Pointers marked "device" must be device (or managed) memory of
 * the current device; "host" pointers are ordinary host memory.  Calls are
 * stream-ordered: unless a function says it synchronises, it only enqueues
 * work, and device buffers the caller passed must stay valid until that work
 * completes.  The caller owns every buffer it passes; the library owns the
 * plan's internal buffers.  A plan is used by one host thread at a time, and
 * its work on one stream at a time (its buffers, the transform's item counter
 * among them, are shared by every call on the plan); a server is thread-safe.
 */
#ifndef FH_H
#define FH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
enum {
    FH_OK = 0,
    FH_ERR_INVALID_ARG = -1, /* null handle/pointer, bad size, non-finite value  */
    FH_ERR_UNSORTED = -2,    /* t_fft not increasing, freq not ascending in an FFT,
                                offsets not a valid CSR                          */
    FH_ERR_RANGE = -3,       /* a fixed-point quantity would leave +-2^60        */
    FH_ERR_NOMEM = -4,       /* device allocation failed                         */
    FH_ERR_TOO_LARGE = -5,   /* job can never fit the server's memory budget     */
    FH_ERR_CUDA = -6,        /* a CUDA runtime call failed                       */
    FH_ERR_TIMEOUT = -7,     /* a bounded wait ran out                           */
    FH_ERR_NOT_READY = -8,   /* fh_poll: the job has not finished                */
    FH_ERR_CANCELLED = -9,   /* the job was cancelled                            */
    FH_ERR_BAD_HANDLE = -10, /* unknown job id / destroyed server                */
    FH_ERR_CAPACITY = -11    /* output buffer smaller than *n_out                */
};

/* where the arrays of an input live */
enum { FH_MEM_HOST = 0, FH_MEM_DEVICE = 1 };

/* counting kernels (fh_plan_desc.mode) -- both give the same integers */
enum {
    FH_MODE_AUTO = 0,  /* library default (FH_MODE_START)                       */
    FH_MODE_DIFF = 1,  /* +1 at the stripe start, -1 after its end, prefix sum  */
    FH_MODE_START = 2  /* +1 at the stripe start only, sum over a K-cell window */
};

/* how fh_transform schedules a set of directions (fh_plan_desc.schedule) */
enum {
    FH_SCHED_BATCHED = 0, /* one persistent launch over all directions' tiles    */
    FH_SCHED_PLAIN = 1    /* one launch per sky direction                         */
};

typedef struct fh_plan_s *fh_plan;     /* opaque, owned by the library */
typedef struct fh_server_s *fh_server; /* opaque, owned by the library */
typedef int64_t fh_job_id;

/* Peakmap (Sec. V): the peaks of every FFT, CSR by FFT, FFTs in time order. */
typedef struct {
    int32_t n_fft;          /* number of FFTs (>= 0)                              */
    int64_t n_peaks;        /* total number of peaks = offsets[n_fft]             */
    const double *t_fft;    /* n_fft FFT start times [s], strictly increasing     */
    const int64_t *offsets; /* n_fft + 1; peaks of FFT i are [offsets[i], offsets[i+1]);
                               offsets[0] = 0, non-decreasing                     */
    const double *freq;     /* n_peaks frequencies [Hz] > 0, strictly ascending
                               within each FFT                                    */
    int32_t mem_kind;       /* FH_MEM_HOST or FH_MEM_DEVICE, for all three arrays
                               and for the velocity and sky arrays of
                               fh_correct_doppler                                 */
} fh_peakmap;

/* Plan: grids of Sec. VII and the selection rule of Sec. VIII. */
typedef struct {
    double t_fft;            /* T_FFT [s] > 0                                     */
    int32_t k_over;          /* frequency over-resolution K >= 1 (Eq. freqres)     */
    double f0_min;           /* lower edge of map cell 0 [Hz]                     */
    int32_t n_f0;            /* number of over-resolved frequency cells >= 1      */
    double fdot_min;         /* spin-down of row 0 [Hz/s]                         */
    double fdot_step;        /* spin-down step [Hz/s] (Eq. sdstep)                */
    int32_t n_fdot;          /* number of spin-down rows >= 1                     */
    double t_ref;            /* reference time t0 [s] (middle of the run, Sec. VI) */
    int32_t subband_cells;   /* sub-band width in cells >= 1                      */
    int32_t top_k;           /* picks per sub-band, 1 .. 64                        */
    int32_t excl_cells;      /* exclusion half-width around a pick, cells >= 0    */
    int32_t sep_cells;       /* minimum distance to earlier picks, cells >= 0     */
    int32_t n_thr;           /* minimum count of a pick                           */
    double p0;               /* peak probability for the critical ratio (Eq. cr), in (0,1) */
    int32_t max_fft;         /* capacity: FFTs per peakmap                        */
    int32_t max_dir;         /* capacity: directions per fh_correct_doppler call,
                                1 .. 65535                                        */
    int64_t max_peaks;       /* capacity: peaks per peakmap (< 2^31)              */
    int32_t mode;            /* FH_MODE_*                                          */
    int32_t schedule;        /* FH_SCHED_*                                         */
    int32_t tile_cells;      /* f0 tile width in cells; 0 = library default        */
    int32_t block_warps;     /* warps per transform block (4..32); 0 = default     */
} fh_plan_desc;

/* One candidate slot.  Empty slots have row = cell = count = -1 and zero
 * f0/fdot/cr; dir, subband and rank are always set. */
typedef struct {
    int32_t dir;      /* absolute direction index of the fh_correct_doppler call */
    int32_t subband;  /* sub-band index q: cells [q W, q W + W)                  */
    int32_t rank;     /* 0 .. top_k - 1 within the sub-band                       */
    int32_t row;      /* spin-down row j                                          */
    int32_t cell;     /* frequency cell b                                         */
    int32_t count;    /* number count n (Eq. ncount; weighted, in units of 2^-F,
                         after fh_set_weights)                                   */
    double f0;        /* f0_min + (b + 0.5) / KT [Hz], cell centre                */
    double fdot;      /* fdot_min + j * fdot_step [Hz/s]                          */
    double cr;        /* (n - N p0) / sqrt(N p0 (1 - p0)), N = n_fft (Eq. cr);
                         adaptive map: see fh_set_weights                        */
} fh_candidate;

/* ---- plan -------------------------------------------------------------- */

/* Validate desc, allocate the plan's device buffers (sized by the max_*
 * capacities) on the current device.  Errors: FH_ERR_INVALID_ARG,
 * FH_ERR_RANGE (grid does not fit 32.32 fixed point), FH_ERR_NOMEM. */
int fh_create_plan(const fh_plan_desc *desc, fh_plan *out);

/* Synchronise the device and free the plan.  NULL is accepted. */
int fh_destroy_plan(fh_plan plan);

/* Bytes of device memory a plan with this desc allocates (0 if invalid). */
int64_t fh_plan_device_bytes(const fh_plan_desc *desc);

/* Steps a1-a3 (Sec. VI, Eq. fdopp): Doppler factor of every (direction,
 * FFT), fixed-point corrected position of every (direction, peak) and the
 * spin-down shift tables, into the plan's buffers.  These directions are the
 * ones fh_transform and fh_select_candidates refer to by index.
 *   pm        peakmap; host arrays are validated on the host (or, after
 *             fh_plan_set_input_checks(FH_CHECKS_DEVICE), by the kernels) and
 *             copied -- except that with n_dir == 1, page-locked (pinned or
 *             registered) host arrays are read in place by the enqueued kernels
 *             over the host link, so they must stay valid and unchanged until
 *             the next synchronising call, as for any asynchronous copy;
 *             device arrays are read in place by the enqueued kernels and
 *             validated on the device (a failure is reported by the next
 *             fh_sync / host-output fh_select_candidates as FH_ERR_UNSORTED or
 *             FH_ERR_INVALID_ARG; the offsets the kernels use are clamped to a
 *             valid CSR first, so bad device input never reads out of bounds)
 *   v_over_c  n_fft x 3 detector velocities in units of c (same memory kind)
 *   sky_n     n_dir x 3 sky unit vectors, same frame (same memory kind)
 *   n_dir     1 .. max_dir
 *   out_r     nullable device n_dir x n_fft: copy of the Doppler factors
 *   out_A     nullable device n_dir x n_peaks: copy of the positions A
 * Host-input errors: FH_ERR_INVALID_ARG, FH_ERR_UNSORTED, FH_ERR_RANGE; after
 * one the plan holds no peakmap (fh_transform refuses until the next
 * successful call), since its device copies of the inputs were already being
 * overwritten. */
int fh_correct_doppler(fh_plan plan, const fh_peakmap *pm, const double *v_over_c,
                       const double *sky_n, int32_t n_dir, double *out_r,
                       int64_t *out_A, void *stream);

/* Steps a4-a5 and the profile half of a6 (Eqs. due, ncount) for directions
 * [dir_begin, dir_begin + n_dir) of the last fh_correct_doppler call.
 *   out_maps  nullable device int32 n_dir x n_fdot x n_f0 (row-major): the
 *             number counts; NULL = candidates only (the map stays on chip)
 * The per-cell profile is kept in the plan for fh_select_candidates. */
int fh_transform(fh_plan plan, int32_t dir_begin, int32_t n_dir, int32_t *out_maps,
                 void *stream);

/* Adaptive map (Eq. ncountadap: n = sum_i w_i n_i) for the directions of the
 * last fh_correct_doppler call.
 *   w          HOST n_dir x n_fft weights (direction-major), finite and >= 0;
 *              NULL returns the plan to the plain map
 *   n_dir      must equal the n_dir of that call
 *   frac_bits  F in [0, 24]: the weights are quantised to integers
 *              W = rint(w 2^F) (binary64, ties to even), so that maps stay
 *              exact integers; each direction's W must sum below 2^30
 * Until the next fh_correct_doppler (which returns the plan to unit
 * weights), fh_transform adds W_i for every stripe of FFT i instead of 1:
 * maps, profiles, candidate counts and n_thr are in units of 2^-F, and the
 * critical ratio becomes (n - S1 p0) / sqrt((S2 p0)(1 - p0)), S1 and S2 the
 * direction's sums of W and of W^2 (for unit weights S1 = S2 = N: Eq. cr).
 * The weights are checked and quantised on the host and copied to the
 * device on stream; then the call computes, on the device, a bound of every
 * count of each direction, sum_i W_i c_i with c_i the most positions of FFT i
 * inside a half-open window of K cells (two stripes of one FFT share a cell
 * only if their positions are less than K cells apart), and synchronises the
 * stream to check it.  Errors: FH_ERR_INVALID_ARG (bad weight, wrong n_dir,
 * no peakmap), FH_ERR_RANGE (a weight or a direction's sum reaching 2^30, or
 * a direction's count bound reaching 2^31: dense off-grid peaks of one FFT
 * under large weights), or the error of the last correction's device-side
 * input checks (its positions are then not trusted). */
int fh_set_weights(fh_plan plan, const double *w, int32_t n_dir, int32_t frac_bits,
                   void *stream);

/* Copy the profile of directions [dir_begin, dir_begin + n_dir) into
 * out (device, n_dir x n_f0 uint64): key = (count << 32) | (0xFFFFFFFF - row). */
int fh_copy_profile(fh_plan plan, int32_t dir_begin, int32_t n_dir, uint64_t *out,
                    void *stream);

/* Step a6 (Sec. VIII; Eq. cr): candidate slots of directions
 * [dir_begin, dir_begin + n_dir), n_dir x n_sb x top_k records, n_sb =
 * ceil(n_f0 / subband_cells), direction-major.  *n_out receives that count;
 * if capacity < *n_out nothing is written and FH_ERR_CAPACITY is returned.
 * out_mem_kind FH_MEM_HOST: copies to host memory and synchronises the stream
 * (and reports device-side input validation failures); FH_MEM_DEVICE:
 * enqueues a device copy. */
int fh_select_candidates(fh_plan plan, int32_t dir_begin, int32_t n_dir, fh_candidate *out,
                         int64_t capacity, int64_t *n_out, int32_t out_mem_kind,
                         void *stream);

/* CUDA graphs.  Once a plan has run a step of a given shape (directions,
 * tile, schedule) -- which sizes its window table and sets its kernels'
 * shared-memory limits -- fh_correct_doppler on DEVICE inputs, fh_transform and
 * fh_select_candidates into DEVICE memory enqueue only kernels, memsets and
 * device-to-device copies on the given stream, and none of them synchronises.
 * Such a step can be captured into a CUDA graph and replayed; a replay reads
 * the device inputs at the addresses given at capture time (update their
 * contents in place), and fh_sync after it reports the device-side input
 * checks as usual.  (Host inputs and host candidate output synchronise and
 * cannot be captured.) */

/* Synchronise the stream and report device-side input validation (FH_OK,
 * FH_ERR_UNSORTED, FH_ERR_INVALID_ARG) since the last fh_correct_doppler. */
int fh_sync(fh_plan plan, void *stream);

/* Time fh_transform over its launch shapes on the current directions (at most
 * 8 of them: the per-item work does not depend on the count) and keep the
 * fastest in the plan; returns its tile width and block warps.  The shapes
 * are: pairs on or off (where the plain START map allows them: two
 * directions with one 16-bit count each per shared word, or for a single
 * direction the two 32-row halves of 64-row slabs), block warps (16, 20, 24,
 * 32) and tile widths up to the widest that fits shared memory with the
 * guard cells of that choice; then, for the fastest of them, the item
 * schedule (blocks taking their next item from a device counter, or every
 * grid-th item).  The shape is chosen for the plan as it stands, weights
 * included: after fh_set_weights, tune again for the weighted map (which
 * pairs nothing).  Synchronises.  Results are cached per process by grid
 * shape (GPU model, counting mode, weighting, n_f0, n_fdot, K, T_FFT, N_t,
 * n_dir); when the environment variable FH_AUTOTUNE_CACHE names a file, they
 * are also read from and written to it (JSON, one entry per line), so later
 * processes reuse them without timing. */
int fh_autotune(fh_plan plan, int32_t dir_begin, int32_t n_dir, int32_t *tile_cells,
                int32_t *block_warps, void *stream);

/* Number of transform/select kernel launches the last fh_transform /
 * fh_select_candidates / fh_correct_doppler calls enqueued (cumulative since
 * plan creation). */
int64_t fh_plan_launches(fh_plan plan);

/* Kernel timing (measurement aid, off by default).  With timing on, every
 * fh_transform records CUDA events on its stream around each direction
 * group's window pre-pass and transform kernel (the last 256 groups are
 * kept); switching it on (again) forgets earlier records.  Do not switch it
 * on for a step that is being captured into a CUDA graph. */
int fh_plan_set_timing(fh_plan plan, int32_t on);

/* Sums, over the recorded groups, of the window pre-pass and transform kernel
 * durations in milliseconds (waits for the last recorded group to finish);
 * *n_groups receives the number of groups summed. */
int fh_plan_kernel_times(fh_plan plan, int64_t *n_groups, double *windows_ms,
                         double *transform_ms);

/* Where fh_correct_doppler checks HOST inputs.  FH_CHECKS_HOST (the default):
 * on the host, before anything is launched; a failed check returns its error
 * from fh_correct_doppler and leaves the plan without a peakmap.
 * FH_CHECKS_DEVICE: the inputs are copied and checked by the kernels, exactly
 * as device inputs are (CSR, ordering, finiteness, fixed-point range), so the
 * call returns as soon as the work is enqueued; a failure is reported, as for
 * device inputs, by the next fh_sync or host-output fh_select_candidates, and
 * no input can make a kernel leave its buffers. */
enum { FH_CHECKS_HOST = 0, FH_CHECKS_DEVICE = 1 };
int fh_plan_set_input_checks(fh_plan plan, int32_t where);

/* ---- peakmap construction and cleaning ------------------------------------ */
/* A binned peakmap: offsets (n_fft + 1, int64, a CSR by FFT, offsets[0] = 0) and
 * the band-relative bin index of every peak (int32, ascending within an FFT);
 * bin b is frequency (k0 + b) / t_fft.  The optional freq outputs hold exactly
 * that (binary64), ready for fh_correct_doppler.  All arrays are DEVICE memory
 * of the current device; each call takes its scratch stream-ordered, runs on
 * `stream` and synchronises it (the counts come back to the host).  Output
 * lists hold `capacity` peaks; a larger result writes the first `capacity`,
 * sets *n_* to the full count and returns FH_ERR_CAPACITY.  Device-side
 * checks: offsets that are not a CSR of n_peaks, or bins outside the band,
 * give FH_ERR_INVALID_ARG (the kernels clamp every range, nothing is read out
 * of bounds). */

/* Peak selection (Sec. "Peakmap", Eq. pm).  s_p, s_ar: n_fft rows of n_bins
 * binary32 values (periodogram and average-spectrum estimate at the same
 * resolution), row pitch `pitch` elements.  R = s_p / s_ar, one IEEE binary32
 * division per bin; bin j of FFT i is a peak when R > theta and R is above
 * both R(j - 1) and R(j + 1) (so bins 0 and n_bins - 1, with one neighbour, are
 * never peaks).  Outputs offsets, bins, freq (nullable); *n_peaks (HOST).
 * n_fft <= 65535.  workspace: NULL (the call takes its scratch stream-ordered)
 * or DEVICE memory of at least fh_peakmap_select_workspace(n_fft, n_bins)
 * bytes, 256-byte aligned, not used by anything else until the call's work on
 * `stream` is done.  With n_peaks NULL the call is asynchronous (no
 * synchronisation; with a workspace nothing is allocated, so it can be
 * captured in a CUDA graph): the total is offsets[n_fft] on the device, and
 * peaks beyond `capacity` are counted there but not written. */
int fh_peakmap_select(const float *s_p, const float *s_ar, int32_t n_fft, int32_t n_bins,
                      int64_t pitch, float theta, int64_t k0, double t_fft, int64_t *offsets,
                      int32_t *bins, double *freq, int64_t capacity, int64_t *n_peaks,
                      void *workspace, int64_t workspace_bytes, void *stream);

/* Bytes of the selection's workspace (a bit per bin and a count per 4096-bin
 * segment); -1 for negative sizes. */
int64_t fh_peakmap_select_workspace(int32_t n_fft, int32_t n_bins);

/* Wandering-line veto (Sec. "Removal of spectral wandering lines").  The gross
 * histogram hist (DEVICE, n_th x n_fh int32, written) counts the peaks per
 * cell: time cell floor((t[i] - t0_h) / dt_h) of the FFT's start time,
 * frequency cell floor(((k0 + b) / t_fft - f0_h) / df_h) (binary64 operations
 * in this order); peaks off the grid are not counted.  Every peak of a cell
 * holding more than `threshold` peaks is removed; the others are written, in
 * order, to offsets_out / bins_out / freq_out (nullable); *n_out (HOST). */
int fh_peakmap_gross_veto(const double *t, const int64_t *offsets, const int32_t *bins,
                          int32_t n_fft, int64_t n_peaks, int64_t k0, double t_fft, double t0_h,
                          double dt_h, int32_t n_th, double f0_h, double df_h, int32_t n_fh,
                          int32_t threshold, int32_t *hist, int64_t *offsets_out,
                          int32_t *bins_out, double *freq_out, int64_t capacity, int64_t *n_out,
                          void *stream);

/* Constant-line veto by persistency (Sec. "Removal of spectral lines of
 * constant frequency"; App. "Robust statistic").  hist (DEVICE, n_bins int32,
 * written): the number of peaks in each bin over all FFTs.  stats (HOST, 3
 * doubles, written): m1 = median(hist) (the mean of the two middle values for
 * an even n_bins), m2 = median(|hist - m1|) / 0.6745, thr = m1 + k_sigma m2.
 * Every peak of a bin with hist > thr is removed; the rest is written as for
 * the gross veto. */
int fh_peakmap_persistency_veto(const int64_t *offsets, const int32_t *bins, int32_t n_fft,
                                int64_t n_peaks, int32_t n_bins, double k_sigma, int64_t k0,
                                double t_fft, int32_t *hist, double *stats,
                                int64_t *offsets_out, int32_t *bins_out, double *freq_out,
                                int64_t capacity, int64_t *n_out, void *stream);

/* ---- candidate clustering and coincidences --------------------------------- */
/* A candidate's parameters (sky position in ecliptic longitude and latitude,
 * radians; frequency, Hz; spin-down, Hz/s) and the widths of its coarse bins
 * in each (the longitude width depends on the latitude).  64 bytes. */
typedef struct fh_cand_params {
    double lam, beta, f, fdot;
    double dlam, dbeta, df, dfdot;
} fh_cand_params;

/* Clusters of one candidate set (Sec. "Candidate clustering and
 * coincidences", Eq. norm).  The distance of two candidates is
 * d = sqrt(((k_lam^2 + k_beta^2) + k_f^2) + k_fdot^2), k_x = |x2 - x1| /
 * ((dx1 + dx2) * 0.5) (binary64, in this order; a longitude difference above
 * pi is taken as 2 pi - it).  Candidates linked by chains of d <= d_max form a
 * cluster; label[i] (DEVICE, n int32, written) is the smallest index of i's
 * cluster; *n_clusters (HOST).  cands: DEVICE, n records, values finite and
 * widths > 0 (else FH_ERR_INVALID_ARG).  Synchronises the stream. */
int fh_cluster(const fh_cand_params *cands, int32_t n, double d_max, int32_t *label,
               int32_t *n_clusters, void *stream);

/* Coincident pairs of two candidate sets (Sec. "Candidate clustering and
 * coincidences"; App. "Theory of coincidences").  Frequencies are referred to
 * the common time t_c first, f + fdot (t_c - t_ref) (the set's own reference
 * time); candidate i of set 1 and j of set 2 coincide when k_lam <= win[0],
 * k_beta <= win[1], k_f <= win[2] and k_fdot <= win[3] (k as for fh_cluster;
 * win HOST, 4 windows in bins, the sum of the two sets' half-windows).
 * pairs (DEVICE, 2 x capacity int32, written): (i, j) in (i, j) order;
 * *n_pairs (HOST) the count (more than capacity: FH_ERR_CAPACITY, the list is
 * then incomplete); n_match1 / n_match2 (DEVICE, nullable) the number of
 * partners of each candidate.  Synchronises the stream. */
int fh_coincidences(const fh_cand_params *c1, int32_t n1, double t_ref1,
                    const fh_cand_params *c2, int32_t n2, double t_ref2, double t_c,
                    const double *win, int32_t *pairs, int64_t capacity, int64_t *n_pairs,
                    int32_t *n_match1, int32_t *n_match2, void *stream);

/* Coincidences among clusters (Sec. "Candidate clustering and coincidences"):
 * two clusters coincide when at least one pair of their members does; each
 * coincident pair of clusters keeps only its nearest coincident pair, the
 * smallest distance of Eq. norm at the common time t_c (ties: the smallest
 * (i, j)).  label1 / label2 (DEVICE): the clusters of fh_cluster; pairs
 * (DEVICE, 2 x n_pairs int32): coincident pairs in strictly increasing (i, j)
 * order, as fh_coincidences writes them (checked).  out (DEVICE, 4 x capacity
 * int32): cluster 1, cluster 2, i, j of each kept pair, in (i, j) order;
 * out_d (DEVICE, nullable): its distance; *n_out (HOST).  Synchronises. */
int fh_cluster_coincidences(const fh_cand_params *c1, int32_t n1, double t_ref1,
                            const int32_t *label1, const fh_cand_params *c2, int32_t n2,
                            double t_ref2, const int32_t *label2, double t_c,
                            const int32_t *pairs, int64_t n_pairs, int32_t *out, double *out_d,
                            int64_t capacity, int64_t *n_out, void *stream);

/* ---- refined grid around coarse candidates -------------------------------- */

/* Refined-grid search (Sec. "Refined Grid in the parameter space"): one
 * refined candidate per coarse candidate (cand_cell[c], cand_row[c] of the
 * plan's grid).  The transform runs again on the same K-over-resolved cells,
 * +-1 coarse bin around the candidate (cells b_c - K .. b_c + K), on a
 * spin-down step refined by k_fdot with 2 k_fdot rows below the coarse value
 * and 2 k_fdot - 1 above (refined row 0 lies on coarse row j_c - 2: shift
 * S0_i + (j_c - 2) D_i, refined step D'_i = floor((fdot_step / k_fdot) c_i
 * 2^32)), and on the n_ref refined sky directions sky_ref[c] of each
 * candidate.  The refined candidate is the largest count over all refined
 * directions, rows and cells (ties: smallest direction, then row, then cell).
 *   plan      the coarse grid and selection parameters (its buffers are not
 *             used, and its peakmap is not changed)
 *   pm, v_over_c  HOST peakmap (n_peaks < 2^31) and velocities, checked as by
 *             fh_correct_doppler; the refined maps are plain (unweighted) counts
 *   sky_ref   HOST n_cand x n_ref x 3 unit vectors
 *   k_fdot    1 .. 64
 *   out       HOST n_cand slots: dir = refined direction index, subband = c,
 *             rank = 0, row = refined row, cell = cell of the plan's grid,
 *             count, f0 = f0_min + (cell + 0.5) / KT, fdot = (fdot_min +
 *             (j_c - 2) fdot_step) + row (fdot_step / k_fdot), cr (Eq. cr)
 * Synchronises the stream; device memory is taken and returned stream-ordered.
 * Errors: FH_ERR_INVALID_ARG, FH_ERR_UNSORTED, FH_ERR_RANGE, FH_ERR_CAPACITY
 * (capacity < n_cand). */
int fh_refine(fh_plan plan, const fh_peakmap *pm, const double *v_over_c,
              const int32_t *cand_cell, const int32_t *cand_row, int32_t n_cand,
              const double *sky_ref, int32_t n_ref, int32_t k_fdot, fh_candidate *out,
              int64_t capacity, void *stream);

/* ---- allocation-free search (one direction) ------------------------------ */

/* fh_search_static: steps a1-a6 for ONE sky direction, like fh_correct_doppler
 * + fh_transform + fh_select_candidates on a plan, but without allocating any
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate while they run -- an application that has
 * reserved the GPU's memory for its own pool, or a loop that must not take the
 * device-wide synchronisation a cudaMalloc/cudaFree can cause.  Its working
 * memory (CSR copy, shift tables, positions, profile, error and drift words;
 * 20,448,000 bytes, 19.5 MiB) is one fixed-size __device__ array in the
 * library, held by every GPU that loads this part of the library until the
 * process exits.
 *   desc          grids and selection as for fh_create_plan (max_* ignored)
 *   pm            peakmap in DEVICE memory; at most 65,536 FFTs and 2,097,152
 *                 peaks; desc->n_f0 at most 262,144 cells -- larger inputs are
 *                 rejected with FH_ERR_TOO_LARGE before anything is enqueued
 *   v_over_c      device, pm->n_fft x 3; sky_n device, 1 x 3
 *   out           device, n_sb x top_k candidate slots (capacity >= *n_out)
 *   device_status nullable device int32: receives the device-side input
 *                 checks (0 = inputs valid) when the enqueued work completes
 * The first call on each device looks up the array's device address (with that
 * device current) and caches it for the life of the process, which assumes the
 * device's primary context lives as long: after cudaDeviceReset the cached
 * address is stale.  Under the CUDA runtime's default lazy module loading that
 * first lookup is also when the driver loads the array, taking its 19.5 MiB of
 * device memory then: make the first call before reserving the rest of the
 * GPU for a pool of your own, and before any stream capture.  Every later call
 * takes no device memory.  Every call reuses the same array, so calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race: serialise them, e.g. on one stream.  Calls only enqueue work; nothing
 * is allocated, nothing is freed. */
int fh_search_static(const fh_plan_desc *desc, const fh_peakmap *pm, const double *v_over_c,
                     const double *sky_n, fh_candidate *out, int64_t capacity, int64_t *n_out,
                     int32_t *device_status, void *stream);

/* ---- serving (continuous batching) --------------------------------------- */

enum { FH_JOB_QUEUED = 0, FH_JOB_RUNNING = 1, FH_JOB_DONE = 2, FH_JOB_FAILED = 3,
       FH_JOB_CANCELLED = 4 };

/* One Hough job: a band x T_FFT x sky patch (configuration 4 of the paper's
 * workload mix), searched with the plain map.  All arrays are host memory;
 * fh_submit copies them before it returns, so the caller may free them at
 * once. */
typedef struct {
    fh_plan_desc plan;      /* grids and selection; max_* are ignored          */
    fh_peakmap peaks;       /* mem_kind must be FH_MEM_HOST                    */
    const double *v_over_c; /* peaks.n_fft x 3                                 */
    const double *sky_n;    /* n_dir x 3                                       */
    int32_t n_dir;          /* >= 1                                            */
} fh_job_desc;

typedef struct {
    double submit_s;        /* host clock (seconds since server start)          */
    double start_s;         /* admitted to the device                          */
    double done_s;          /* results in host memory                          */
    int64_t updates;        /* n_dir * n_fdot * n_peaks                        */
    int64_t device_bytes;   /* device memory the job held                      */
    int32_t batch;          /* index of the launch batch that ran it           */
    int32_t batch_jobs;     /* jobs in that batch                              */
} fh_job_stats;

/* Start a server on the current device: a scheduler thread admits queued jobs
 * while their device memory fits device_mem_budget, batches all jobs admitted
 * together into one launch sequence on one of max_inflight streams, and lets
 * batches overlap on the device. */
int fh_server_create(int64_t device_mem_budget, int32_t max_inflight, fh_server *out);

/* Cancel queued jobs, wait (bounded, 60 s) for running ones, free everything. */
int fh_server_destroy(fh_server server);

/* Validate and enqueue a job.  FH_ERR_TOO_LARGE if it can never fit the budget. */
int fh_submit(fh_server server, const fh_job_desc *job, fh_job_id *out);

/* Non-blocking.  *state = FH_JOB_*.  When DONE, copies the job's
 * n_dir x n_sb x top_k candidate slots to out (host) -- FH_ERR_CAPACITY and
 * *n_out as in fh_select_candidates; otherwise returns FH_ERR_NOT_READY
 * (queued/running), the job's error (failed) or FH_ERR_CANCELLED. */
int fh_poll(fh_server server, fh_job_id id, int32_t *state, fh_candidate *out,
            int64_t capacity, int64_t *n_out);

/* Timing record of a finished job. */
int fh_job_get_stats(fh_server server, fh_job_id id, fh_job_stats *out);

/* Cancel a queued job (running jobs complete). */
int fh_cancel(fh_server server, fh_job_id id);

/* Block until every submitted job is done/failed/cancelled or timeout_s
 * passes (FH_ERR_TIMEOUT; nothing is cancelled). */
int fh_server_drain(fh_server server, double timeout_s);

/* paused != 0: stop admitting queued jobs (running batches complete);
 * paused = 0: resume.  For maintenance and for tests of stuck queues. */
int fh_server_pause(fh_server server, int32_t paused);

/* ---- measurement ------------------------------------------------------- */

/* Shared-memory atomic throughput of this GPU: every SM runs blocks of 1024
 * threads doing int32 atomicAdd into shared memory, conflict-free (variant 0,
 * lane l -> bank l) or to random addresses (variant 1).  Synchronises.
 * *atomics_per_s = lane-atomics per second over the whole GPU. */
int fh_bench_smem_atomics(int32_t variant, int32_t iters, double *atomics_per_s,
                          double *ms, void *stream);

/* Binary64 throughput of this GPU: every SM runs blocks of 512 threads, each
 * with 8 independent chains of one IEEE multiply and one IEEE add per step
 * (round to nearest, never fused: the operations the Doppler correction and
 * positions use, Eq. fdopp).  Synchronises.  *ops_per_s = binary64
 * operations per second over the whole GPU. */
int fh_bench_fp64(int32_t iters, double *ops_per_s, double *ms, void *stream);

/* ---- misc -------------------------------------------------------------- */
const char *fh_last_error(void);
const char *fh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FH_H */
