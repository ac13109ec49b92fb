// fh_refine: the refined-grid frequency-Hough search around coarse candidates
// (Sec. "Refined Grid in the parameter space").
//
// For each coarse candidate (cell b_c, row j_c of the plan's grid) the
// transform runs again on a small grid: the same K-over-resolved cells, +-1
// coarse bin around the candidate (cells b_c - K .. b_c + K); a spin-down step
// refined by K_fdot, 2 K_fdot rows below the coarse value and 2 K_fdot - 1
// above (refined row 0 on coarse row j_c - 2: shift S0_i + (j_c - 2) D_i, step
// D'_i = floor((fdot_step / K_fdot) c_i 2^32)); and the caller's refined sky
// directions.  One refined candidate is kept per coarse one: the largest count
// over all refined directions, rows and cells (ties: smallest direction, then
// row, then cell).
//
// Per call: the coarse and refined shift tables (prep kernels); per
// (candidate, FFT) the contiguous range of peaks that can reach the refined
// band (a conservative frequency window, binary search); compact per-candidate
// position arrays for those peaks only; peak windows and one batched transform
// launch per group of candidates; a pick kernel per candidate.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fh_internal.h"

using namespace fh;

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct RangeArgs {
    const double *t, *freq, *v, *sky;  // sky: [cand][n_ref][3]
    const int64_t *offsets, *S0, *D, *Dr;
    const int32_t *cell, *row;
    int32_t n_fft, n_cand, k_over, n_rows, n_ref;
    double f0_min, kt;
    int64_t *start;   // [cand][fft]: first peak of the range
    int32_t *count;   // [cand][fft]: peaks in the range
    int64_t *S0r;     // [cand][fft]: refined row-0 shift, cell offset included
};

// Refined band of candidate c in refined cells [0, 2K + 1): a stripe starting at
// s touches it iff s in [1 - K, 2K].  With the refined shifts X_j = S0r + j D'
// (j < n_rows), positions A in [min_j X_j + (1 - K) 2^32, max_j X_j + (2K + 1)
// 2^32) can touch it; one extra cell on each side covers rounding.  A position
// is about ((f r - f0_min) KT + 0.5 - 0.5 K) 2^32 with r = 1 / (1 + v.n), so
// the frequencies f = u (1 + v.n) of the peaks that can take part lie between
// the extremes of that product over u in [u_lo, u_hi] and v.n between its
// least and largest value over the candidate's refined directions (a bilinear
// form: the extremes are at the corners).  The margin of a cell is far above
// the rounding of these products; the transform decides exactly.
__global__ void refine_ranges_kernel(const RangeArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= a.n_fft) return;
    const int K = a.k_over;
    const int64_t lo_cell = (int64_t)a.cell[c] - K;
    const int64_t s0r = a.S0[i] + (int64_t)(a.row[c] - 2) * a.D[i] + lo_cell * 4294967296LL;
    a.S0r[(int64_t)c * a.n_fft + i] = s0r;
    const int64_t last = (int64_t)(a.n_rows - 1) * a.Dr[i];
    const double xmin = ((double)s0r + (double)(last < 0 ? last : 0)) / 4294967296.0;
    const double xmax = ((double)s0r + (double)(last > 0 ? last : 0)) / 4294967296.0;
    const double c_off = 0.5 - 0.5 * (double)K;
    const double u_lo = a.f0_min + (xmin + (double)(1 - K) - 1.0 - c_off) / a.kt;
    const double u_hi = a.f0_min + (xmax + (double)(2 * K + 1) + 1.0 - c_off) / a.kt;
    const double vx = a.v[3 * (int64_t)i], vy = a.v[3 * (int64_t)i + 1],
                 vz = a.v[3 * (int64_t)i + 2];
    double vn_lo = 0.0, vn_hi = 0.0;
    const double *n = a.sky + 3 * (int64_t)c * a.n_ref;
    for (int d = 0; d < a.n_ref; ++d, n += 3) {
        const double vn = vx * n[0] + vy * n[1] + vz * n[2];
        vn_lo = d ? fmin(vn_lo, vn) : vn;
        vn_hi = d ? fmax(vn_hi, vn) : vn;
    }
    const double f_lo = fmin(fmin(u_lo * (1.0 + vn_lo), u_lo * (1.0 + vn_hi)),
                             fmin(u_hi * (1.0 + vn_lo), u_hi * (1.0 + vn_hi)));
    const double f_hi = fmax(fmax(u_lo * (1.0 + vn_lo), u_lo * (1.0 + vn_hi)),
                             fmax(u_hi * (1.0 + vn_lo), u_hi * (1.0 + vn_hi)));
    int64_t lo = a.offsets[i], hi = a.offsets[i + 1];
    int64_t b = hi;
    while (lo < b) {  // first peak with f >= f_lo
        const int64_t m = (lo + b) >> 1;
        if (a.freq[m] < f_lo) lo = m + 1; else b = m;
    }
    int64_t e = lo;
    b = hi;
    while (e < b) {  // first peak with f > f_hi
        const int64_t m = (e + b) >> 1;
        if (a.freq[m] <= f_hi) e = m + 1; else b = m;
    }
    a.start[(int64_t)c * a.n_fft + i] = lo;
    a.count[(int64_t)c * a.n_fft + i] = (int32_t)(e - lo);
}

struct PickArgs {
    const uint64_t *const *prof;  // [cand] -> [n_ref][n_f0r] profile keys
    const int32_t *cell, *row;
    int32_t n_cand, n_ref, n_f0r, k_over, n_fft;
    double f0_min, kt, fdot_min, fdot_step, fdot_step_ref, p0;
    fh_candidate *out;
};

// one warp per candidate: the best (count desc, direction asc, row asc, cell asc)
// over the candidate's refined profile
__global__ void refine_pick_kernel(const PickArgs a)
{
    const int c = blockIdx.x;
    const int lane = threadIdx.x;
    const uint64_t *pr = a.prof[c];
    int bc = -1, bd = 0x7fffffff, bj = 0x7fffffff, bb = 0x7fffffff;
    const int n = a.n_ref * a.n_f0r;
    for (int k = lane; k < n; k += 32) {
        const uint64_t key = pr[k];
        const int cnt = (int)(uint32_t)(key >> 32);
        const int j = (int)(0xFFFFFFFFu - (uint32_t)key);
        const int d = k / a.n_f0r, b = k - d * a.n_f0r;
        const bool better = cnt > bc || (cnt == bc && (d < bd || (d == bd && (j < bj ||
                                                                   (j == bj && b < bb)))));
        if (key != 0 && better) {
            bc = cnt;
            bd = d;
            bj = j;
            bb = b;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const int c2 = __shfl_down_sync(kFull, bc, o), d2 = __shfl_down_sync(kFull, bd, o);
        const int j2 = __shfl_down_sync(kFull, bj, o), b2 = __shfl_down_sync(kFull, bb, o);
        const bool better = c2 > bc || (c2 == bc && (d2 < bd || (d2 == bd && (j2 < bj ||
                                                                  (j2 == bj && b2 < bb)))));
        if (better) {
            bc = c2;
            bd = d2;
            bj = j2;
            bb = b2;
        }
    }
    if (lane != 0) return;
    fh_candidate r;
    r.subband = c;
    r.rank = 0;
    if (bc < 0) {
        r.dir = r.row = r.cell = r.count = -1;
        r.f0 = r.fdot = r.cr = 0.0;
    } else {
        const int cell = a.cell[c] - a.k_over + bb;
        r.dir = bd;
        r.row = bj;
        r.cell = cell;
        r.count = bc;
        r.f0 = __dadd_rn(a.f0_min, __ddiv_rn(__dadd_rn((double)cell, 0.5), a.kt));
        const double fdot_lo =
            __dadd_rn(a.fdot_min, __dmul_rn((double)(a.row[c] - 2), a.fdot_step));
        r.fdot = __dadd_rn(fdot_lo, __dmul_rn((double)bj, a.fdot_step_ref));
        const double np0 = __dmul_rn((double)a.n_fft, a.p0);
        const double sd = __dsqrt_rn(__dmul_rn(np0, __dsub_rn(1.0, a.p0)));
        r.cr = __ddiv_rn(__dsub_rn((double)bc, np0), sd);
    }
    a.out[c] = r;
}

}  // namespace

namespace fh {

int refine_impl(const fh_plan_desc &d, int n_sm, const fh_peakmap *pm,
                const double *v_over_c, const int32_t *cand_cell, const int32_t *cand_row,
                int32_t n_cand, const double *sky_ref, int32_t n_ref, int32_t k_fdot,
                fh_candidate *out, bool host_checks, cudaStream_t s)
{
    const double kt = (double)d.k_over * d.t_fft;
    const int32_t n = pm->n_fft;
    const int64_t np = pm->n_peaks;
    const int K = d.k_over;
    const int32_t n_f0r = 2 * K + 1;
    const int32_t n_rows = 4 * k_fdot;
    const double step_ref = d.fdot_step / (double)k_fdot;
    // the inputs are checked on the host, or (FH_CHECKS_DEVICE) by the kernels
    if (host_checks) {
        const int rc = validate_host_inputs(d, kt, pm, v_over_c, sky_ref, n_cand * n_ref);
        if (rc) return rc;
    }
    for (int32_t c = 0; c < n_cand; ++c)
        if ((int64_t)cand_cell[c] - K < -(int64_t(1) << 27) ||
            (int64_t)cand_cell[c] + K >= (int64_t(1) << 27) || cand_row[c] < -(1 << 27) ||
            cand_row[c] >= (1 << 27))
            return set_error(FH_ERR_RANGE, "candidate %d outside the plan's fixed-point range", c);

    Scratch sc(s);
    double *t = nullptr, *freq = nullptr, *v = nullptr, *sky = nullptr;
    int64_t *off = nullptr, *S0 = nullptr, *D = nullptr, *S0x = nullptr, *Dr = nullptr;
    int64_t *start = nullptr, *S0r = nullptr;
    int32_t *count = nullptr, *cc = nullptr, *cr = nullptr, *err = nullptr;
    unsigned long long *dmax = nullptr;
    cudaError_t e = cudaSuccess;
    e = sc.get(&t, (size_t)n);
    if (e == cudaSuccess) e = sc.get(&freq, (size_t)np);
    if (e == cudaSuccess) e = sc.get(&v, 3 * (size_t)n);
    if (e == cudaSuccess) e = sc.get(&sky, 3 * (size_t)n_cand * n_ref);
    if (e == cudaSuccess) e = sc.get(&off, (size_t)n + 1);
    int64_t *off_raw = nullptr;
    if (e == cudaSuccess && !host_checks) e = sc.get(&off_raw, (size_t)n + 1);
    if (e == cudaSuccess) e = sc.get(&S0, (size_t)n);
    if (e == cudaSuccess) e = sc.get(&D, (size_t)n);
    if (e == cudaSuccess) e = sc.get(&S0x, (size_t)n);
    if (e == cudaSuccess) e = sc.get(&Dr, (size_t)n);
    if (e == cudaSuccess) e = sc.get(&start, (size_t)n_cand * n);
    if (e == cudaSuccess) e = sc.get(&S0r, (size_t)n_cand * n);
    if (e == cudaSuccess) e = sc.get(&count, (size_t)n_cand * n);
    if (e == cudaSuccess) e = sc.get(&cc, (size_t)n_cand);
    if (e == cudaSuccess) e = sc.get(&cr, (size_t)n_cand);
    if (e == cudaSuccess) e = sc.get(&err, 4);
    if (e == cudaSuccess) e = sc.get(&dmax, 2);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync (refinement)");
    struct {
        void *dst;
        const void *src;
        size_t bytes;
    } cp[] = {{t, pm->t_fft, 8 * (size_t)n},
              {freq, pm->freq, 8 * (size_t)np},
              {v, v_over_c, 24 * (size_t)n},
              {sky, sky_ref, 24 * (size_t)n_cand * n_ref},
              {host_checks ? off : off_raw, pm->offsets, 8 * ((size_t)n + 1)},
              {cc, cand_cell, 4 * (size_t)n_cand},
              {cr, cand_row, 4 * (size_t)n_cand}};
    for (auto &x : cp)
        if (x.bytes && e == cudaSuccess)
            e = cudaMemcpyAsync(x.dst, x.src, x.bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dmax, 0, 16, s);
    // coarse shift tables, then the refined step D' (and its largest |D'|)
    PrepArgs pa{};
    pa.offsets_in = host_checks ? nullptr : off_raw;  // sanitised into off by the checks
    pa.offsets_out = off;
    pa.validate = host_checks ? 0 : 1;
    pa.t = t;
    pa.v = v;
    pa.sky = sky;
    pa.n_fft = n;
    pa.n_dir = n_cand * n_ref;
    pa.n_fdot = d.n_fdot;
    pa.n_peaks = np;
    pa.t_ref = d.t_ref;
    pa.kt = kt;
    pa.fdot_min = d.fdot_min;
    pa.fdot_step = d.fdot_step;
    pa.S0 = S0;
    pa.D = D;
    pa.dmax = dmax + 1;  // the coarse drift is not needed
    pa.err = err;
    if (e == cudaSuccess) e = launch_prep(pa, s);
    // device checks: every peak's frequency too (the positions below cover only
    // the peaks near each candidate, and the range searches need sorted FFTs)
    if (e == cudaSuccess && !host_checks)
        e = launch_validate_device_inputs(t, freq, off, v, sky, n, n_cand * n_ref, err, s);
    PrepArgs pr = pa;
    pr.offsets_in = nullptr;  // sanitised and checked by the first launch
    pr.validate = 0;
    pr.n_fdot = n_rows;
    pr.fdot_min = 0.0;
    pr.fdot_step = step_ref;
    pr.S0 = S0x;
    pr.D = Dr;
    pr.dmax = dmax;
    if (e == cudaSuccess) e = launch_prep(pr, s);
    // the peaks of every (candidate, FFT) that can reach the refined band
    RangeArgs ra{};
    ra.t = t;
    ra.freq = freq;
    ra.v = v;
    ra.sky = sky;
    ra.n_ref = n_ref;
    ra.offsets = off;
    ra.S0 = S0;
    ra.D = D;
    ra.Dr = Dr;
    ra.cell = cc;
    ra.row = cr;
    ra.n_fft = n;
    ra.n_cand = n_cand;
    ra.k_over = K;
    ra.n_rows = n_rows;
    ra.f0_min = d.f0_min;
    ra.kt = kt;
    ra.start = start;
    ra.count = count;
    ra.S0r = S0r;
    if (e == cudaSuccess && n > 0 && n_cand > 0) {
        dim3 grid((n + 255) / 256, n_cand);
        refine_ranges_kernel<<<grid, 256, 0, s>>>(ra);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_error(e, "refinement set-up");
    // per-candidate compact offsets (host prefix sums)
    std::vector<int32_t> h_count((size_t)n_cand * n);
    if (!h_count.empty())
        e = cudaMemcpyAsync(h_count.data(), count, 4 * h_count.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "refinement ranges");
    std::vector<int64_t> h_off((size_t)n_cand * (n + 1));
    std::vector<int64_t> n_sub(n_cand);
    for (int32_t c = 0; c < n_cand; ++c) {
        int64_t acc = 0;
        int64_t *o = &h_off[(size_t)c * (n + 1)];
        for (int32_t i = 0; i < n; ++i) {
            o[i] = acc;
            acc += h_count[(size_t)c * n + i];
        }
        o[n] = acc;
        n_sub[c] = acc;
    }
    int64_t *sub_off = nullptr;
    e = sc.get(&sub_off, h_off.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sub_off, h_off.data(), 8 * h_off.size(), cudaMemcpyHostToDevice, s);
    // positions, profiles and windows of every candidate
    // one allocation each for all candidates' positions and profiles
    std::vector<int64_t *> A(n_cand, nullptr);
    std::vector<uint64_t *> prof(n_cand, nullptr);
    const int32_t n_slabs = (n_rows + kRows - 1) / kRows;
    size_t a_total = 0;
    for (int32_t c = 0; c < n_cand; ++c)
        a_total += (size_t)n_ref * std::max<int64_t>(1, n_sub[c]);
    const size_t prof_each = (size_t)n_ref * n_f0r;
    int64_t *a_all = nullptr;
    uint64_t *prof_all = nullptr;
    if (e == cudaSuccess) e = sc.get(&a_all, a_total);
    if (e == cudaSuccess) e = sc.get(&prof_all, prof_each * n_cand);
    if (e == cudaSuccess) e = cudaMemsetAsync(prof_all, 0, 8 * prof_each * n_cand, s);
    size_t a_at = 0;
    for (int32_t c = 0; c < n_cand; ++c) {
        A[c] = a_all + a_at;
        a_at += (size_t)n_ref * std::max<int64_t>(1, n_sub[c]);
        prof[c] = prof_all + prof_each * c;
    }
    // every candidate's positions in one launch
    std::vector<int64_t> h_batch(2 * (size_t)n_cand);
    for (int32_t c = 0; c < n_cand; ++c) {
        h_batch[c] = A[c] - a_all;
        h_batch[n_cand + c] = n_sub[c];
    }
    int64_t *d_batch = nullptr;
    if (e == cudaSuccess) e = sc.get(&d_batch, h_batch.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_batch, h_batch.data(), 8 * h_batch.size(), cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess)
        e = launch_positions_batched(freq, sub_off, v, sky, n, n_ref, n_cand, d_batch,
                                     d_batch + n_cand, d.f0_min, kt, K, a_all, err, !host_checks,
                                     start, s);
    if (e != cudaSuccess) return cuda_error(e, "refinement positions");
    // the refined drift on the host, for the guard cells (as the device's D')
    double m = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        const double x = std::fabs(step_ref * ((pm->t_fft[i] - d.t_ref) * kt));
        if (x > m && x < 1e9) m = x;  // non-finite times are left to the checks
    }
    const int32_t guard = guard_for((unsigned long long)(m * 4294967296.0) + 4);
    const int nwarps = 16;
    const size_t smem = transform_smem_bytes(n_f0r, K, FH_MODE_START, nwarps, guard);
    e = transform_prepare(FH_MODE_START, smem);
    if (e != cudaSuccess) return cuda_error(e, "transform_prepare");
    const int bps = std::max(1, transform_blocks_per_sm(FH_MODE_START, nwarps, smem));
    for (int32_t g = 0; g < n_cand; g += kMaxBatchJobs) {
        JobTable tbl{};
        int64_t items = 0;
        for (int32_t c = g; c < std::min(n_cand, g + kMaxBatchJobs); ++c) {
            TransformJob &j = tbl.job[tbl.n_jobs++];
            j.A = A[c];
            j.offsets = sub_off + (size_t)c * (n + 1);
            j.S0 = S0r + (size_t)c * n;
            j.D = Dr;
            j.profile = prof[c];
            j.maps = nullptr;
            j.dmax = dmax;
            j.err = err;
            j.weights = nullptr;
            j.count_bound = n_sub[c];
            // no window table: a candidate's ranges hold a few peaks per FFT, so
            // the transform's own binary search per FFT costs less than a pre-pass
            j.windows = nullptr;
            j.n_peaks = n_sub[c];
            j.n_fft = n;
            j.n_f0 = n_f0r;
            j.n_fdot = n_rows;
            j.k_over = K;
            j.tile_cells = n_f0r;
            j.n_slabs = n_slabs;
            j.n_tiles = 1;
            j.dir_begin = 0;
            j.n_dir = n_ref;
            j.item_begin = items;
            j.n_items = (int64_t)n_slabs * n_ref;
            items += j.n_items;

        }
        const int32_t grid = (int32_t)std::min<int64_t>(items, (int64_t)n_sm * bps);
        e = launch_transform(FH_MODE_START, tbl, items, grid, nwarps, smem, guard, s);
        if (e != cudaSuccess) return cuda_error(e, "refinement transform");
    }
    // the pick of every candidate
    uint64_t **d_prof = nullptr;
    fh_candidate *d_out = nullptr;
    e = sc.get(&d_prof, (size_t)n_cand);
    if (e == cudaSuccess) e = sc.get(&d_out, (size_t)n_cand);
    if (e == cudaSuccess && n_cand > 0)
        e = cudaMemcpyAsync(d_prof, prof.data(), sizeof(uint64_t *) * (size_t)n_cand,
                            cudaMemcpyHostToDevice, s);
    PickArgs pk{};
    pk.prof = d_prof;
    pk.cell = cc;
    pk.row = cr;
    pk.n_cand = n_cand;
    pk.n_ref = n_ref;
    pk.n_f0r = n_f0r;
    pk.k_over = K;
    pk.n_fft = n;
    pk.f0_min = d.f0_min;
    pk.kt = kt;
    pk.fdot_min = d.fdot_min;
    pk.fdot_step = d.fdot_step;
    pk.fdot_step_ref = step_ref;
    pk.p0 = d.p0;
    pk.out = d_out;
    if (e == cudaSuccess && n_cand > 0) {
        refine_pick_kernel<<<n_cand, 32, 0, s>>>(pk);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n_cand > 0)
        e = cudaMemcpyAsync(out, d_out, sizeof(fh_candidate) * (size_t)n_cand,
                            cudaMemcpyDeviceToHost, s);
    int32_t h_err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "refinement pick");
    if (h_err) return device_error_code(h_err);
    return FH_OK;
}

}  // namespace fh
