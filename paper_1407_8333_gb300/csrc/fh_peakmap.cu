// Peakmap construction and cleaning on the GPU (the step before the transform).
//
//   fh_peakmap_select            Sec. "Peakmap", Eq. pm: R = S_P / S_AR bin by bin
//                                (binary32), peaks = bins above theta that are strict
//                                local maxima of R in their FFT
//   fh_peakmap_gross_veto        Sec. "Removal of spectral wandering lines": the
//                                "gross histogram" of a Delta t_H x Delta f_H grid;
//                                peaks in cells above the threshold are removed
//   fh_peakmap_persistency_veto  Sec. "Removal of spectral lines of constant
//                                frequency" with App. "Robust statistic": per-bin
//                                FFT counts, m1 = median, m2 = median(|x - m1|) /
//                                0.6745; bins above m1 + k m2 lose their peaks
//
// Selection streams the two spectra once (8 bytes per bin, the HBM-bound part):
// a block takes 4096 bins of one FFT, keeps R in shared memory with one halo
// bin on each side, and writes one selection bit per bin (a warp ballot per 32
// bins) and the segment's count; a single-block scan turns the counts into the
// CSR offsets and per-segment bases; a second pass expands the bits into bin
// indices.  Cleaning works on the peak lists: histograms by global atomics, a
// warp per FFT for the keep/drop pass (ballot ranks keep the order), the same
// scan for the new offsets.  The robust statistic needs only the histogram of
// the per-bin counts (values 0 .. n_fft), so its medians are order statistics
// found by one block scanning that histogram; every median is exact (integers
// and half-integers), and m2 and the threshold are single binary64 operations
// in the order written above.
#include <cmath>
#include <cstdint>
#include <vector>

#include "fh_internal.h"

namespace fh {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSegBins = 4096;    // bins of one FFT per selection block
constexpr int kSegThreads = 256;  // 16 bins per thread
constexpr int kSegWords = kSegBins / 32;
constexpr int kScanThreads = 1024;

// (k0 + b) / t_fft, the IEEE quotient.  When t_fft is a power of two the
// quotient is the exact product with inv = 1 / t_fft (also exact), and a
// binary64 multiply replaces the much slower division.
struct FreqOf {
    int64_t k0;
    double t_fft, inv;
    bool pow2;
    __device__ __forceinline__ double operator()(int32_t b) const
    {
        const double x = (double)(k0 + b);
        return pow2 ? __dmul_rn(x, inv) : __ddiv_rn(x, t_fft);
    }
};

FreqOf make_freq_of(int64_t k0, double t_fft)
{
    int ex = 0;
    const double m = std::frexp(t_fft, &ex);
    FreqOf f;
    f.k0 = k0;
    f.t_fft = t_fft;
    f.pow2 = m == 0.5 && ex > -1000 && ex < 1000;
    f.inv = f.pow2 ? std::ldexp(1.0, 1 - ex) : 0.0;
    return f;
}

// ---------------------------------------------------------------- selection
struct SelArgs {
    const float *s_p, *s_ar;
    int64_t pitch;
    int32_t n_fft, n_bins, n_seg, n_words;
    float theta;
    uint32_t *mask;     // [fft][word]
    int32_t *seg_count; // [fft][seg]
    int32_t *err;       // bulk-copy waits that ran out
};

__device__ __forceinline__ float ratio_at(const float *sp, const float *sa, int j, int n_bins)
{
    // bins outside the FFT are never compared (the flags of bins 0 and
    // n_bins - 1 are false), so any value serves there
    return (j >= 0 && j < n_bins) ? __fdiv_rn(__ldg(sp + j), __ldg(sa + j)) : 0.0f;
}

constexpr int kBulkPolls = 1 << 22;  // a bulk copy always completes; this only bounds the wait

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// The selection pass with the two spectrum rows of a tile brought into shared
// memory by bulk copies (cp.async.bulk, the 1-D form of the tensor memory
// accelerator) that complete on one mbarrier: 32 KB per block in flight at
// once, no registers held by loads.  Used when both spectra are 16-byte
// aligned, the pitch is a multiple of 4 floats and so is n_bins, so that every
// copy starts on a 16-byte boundary and moves a multiple of 16 bytes.  The
// ratios are formed in place; flags and counts as in select_mask_kernel.
__global__ void __launch_bounds__(kSegThreads) select_mask_bulk_kernel(const SelArgs a)
{
    __shared__ __align__(128) float p_s[kSegBins + 8];  // p_s[4 + k]: S_P, then R, of bin j0 + k
    __shared__ __align__(128) float q_s[kSegBins];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int32_t warp_cnt[kSegThreads / 32];
    const int row = blockIdx.y, seg = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j0 = seg * kSegBins;
    const int nb = min(kSegBins, a.n_bins - j0);
    const float *sp = a.s_p + (int64_t)row * a.pitch;
    const float *sa = a.s_ar + (int64_t)row * a.pitch;
    const uint32_t bar_a = (uint32_t)__cvta_generic_to_shared(&bar);
    if (tid == 0) {
        const uint32_t bytes = 4u * (uint32_t)nb;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a),
                     "r"(2u * bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"((uint32_t)__cvta_generic_to_shared(p_s + 4)),
            "l"(sp + j0), "r"(bytes), "r"(bar_a)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"((uint32_t)__cvta_generic_to_shared(q_s)),
            "l"(sa + j0), "r"(bytes), "r"(bar_a)
            : "memory");
    }
    // the halo bins (outside the copies)
    if (tid == 32) p_s[3] = ratio_at(sp, sa, j0 - 1, a.n_bins);
    if (tid == 64) p_s[4 + kSegBins] = ratio_at(sp, sa, j0 + kSegBins, a.n_bins);
    __syncthreads();  // the barrier is initialised before anyone waits on it
    bool done = false;
    for (int it = 0; it < kBulkPolls && !done; ++it) done = mbar_try_wait(bar_a, 0);
    if (!done) {
        // never expected: report, then still wait (bounded) for the block's own
        // copies before the shared memory is given up
        if (tid == 0) atomicOr(a.err, kErrRange);
        for (int it = 0; it < kBulkPolls && !done; ++it) done = mbar_try_wait(bar_a, 0);
    }
    for (int k = tid; k < nb; k += kSegThreads) p_s[4 + k] = __fdiv_rn(p_s[4 + k], q_s[k]);
    __syncthreads();
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < kSegWords / (kSegThreads / 32); ++k) {
        const int wl = k * (kSegThreads / 32) + warp;  // word of the segment
        const int loc = wl * 32 + lane;
        const int j = j0 + loc;
        const float r = p_s[4 + loc];
        const bool f = j >= 1 && j <= a.n_bins - 2 && r > a.theta && r > p_s[3 + loc] &&
                       r > p_s[5 + loc];
        const unsigned word = __ballot_sync(kFull, f);
        const int w = seg * kSegWords + wl;
        if (lane == 0 && w < a.n_words) a.mask[(int64_t)row * a.n_words + w] = word;
        cnt += __popc(word);
    }
    if (lane == 0) warp_cnt[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        int c = lane < kSegThreads / 32 ? warp_cnt[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if (lane == 0) a.seg_count[(int64_t)row * a.n_seg + seg] = c;
    }
}


// A block takes 4096 bins of one FFT.  Loads: 16 bins per thread, as four
// float4 per spectrum when the rows are 16-byte aligned (VEC), so that each
// SM keeps ~256 KB of loads in flight; the ratios go to shared memory with one
// halo bin on each side.  Flags: warp w takes words w, w + 8, ... (32 bins
// each), one ballot per word.
template <bool VEC>
__global__ void __launch_bounds__(kSegThreads) select_mask_kernel(const SelArgs a)
{
    __shared__ float r_s[kSegBins + 2];  // r_s[1 + k] = R(j0 + k); halos at 0 and kSegBins + 1
    __shared__ int32_t warp_cnt[kSegThreads / 32];
    const int row = blockIdx.y, seg = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j0 = seg * kSegBins;
    const float *sp = a.s_p + (int64_t)row * a.pitch;
    const float *sa = a.s_ar + (int64_t)row * a.pitch;
    if (VEC) {
        float4 p[4], q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = j0 + 4 * (k * kSegThreads + tid);
            if (j + 3 < a.n_bins) {
                p[k] = __ldg(reinterpret_cast<const float4 *>(sp + j));
                q[k] = __ldg(reinterpret_cast<const float4 *>(sa + j));
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int loc = 4 * (k * kSegThreads + tid);
            const int j = j0 + loc;
            if (j + 3 < a.n_bins) {
                r_s[1 + loc] = __fdiv_rn(p[k].x, q[k].x);
                r_s[2 + loc] = __fdiv_rn(p[k].y, q[k].y);
                r_s[3 + loc] = __fdiv_rn(p[k].z, q[k].z);
                r_s[4 + loc] = __fdiv_rn(p[k].w, q[k].w);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) r_s[1 + loc + e] = ratio_at(sp, sa, j + e, a.n_bins);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kSegBins / kSegThreads; ++k) {
            const int loc = k * kSegThreads + tid;
            r_s[1 + loc] = ratio_at(sp, sa, j0 + loc, a.n_bins);
        }
    }
    if (tid == 0) r_s[0] = ratio_at(sp, sa, j0 - 1, a.n_bins);
    if (tid == 1) r_s[kSegBins + 1] = ratio_at(sp, sa, j0 + kSegBins, a.n_bins);
    __syncthreads();
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < kSegWords / (kSegThreads / 32); ++k) {
        const int wl = k * (kSegThreads / 32) + warp;  // word of the segment
        const int loc = wl * 32 + lane;
        const int j = j0 + loc;
        const float r = r_s[1 + loc];
        const bool f = j >= 1 && j <= a.n_bins - 2 && r > a.theta && r > r_s[loc] &&
                       r > r_s[loc + 2];
        const unsigned word = __ballot_sync(kFull, f);
        const int w = seg * kSegWords + wl;
        if (lane == 0 && w < a.n_words) a.mask[(int64_t)row * a.n_words + w] = word;
        cnt += __popc(word);
    }
    if (lane == 0) warp_cnt[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        int c = lane < kSegThreads / 32 ? warp_cnt[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if (lane == 0) a.seg_count[(int64_t)row * a.n_seg + seg] = c;
    }
}

struct ExpandArgs {
    const uint32_t *mask;
    const int64_t *seg_base;  // [fft][seg] first output slot of the segment
    int32_t n_seg, n_words;
    int64_t capacity;
    FreqOf fq;
    int32_t *bins;
    double *freq;
};

// One block per (segment, FFT): 128 words, one per thread; a block scan of
// their counts ranks the segment's peaks, which are staged in shared memory in
// bin order and written as contiguous runs.
__global__ void __launch_bounds__(kSegWords) select_expand_kernel(const ExpandArgs a)
{
    __shared__ int32_t wsum[kSegWords / 32];
    __shared__ int32_t peaks_s[kSegBins / 2];  // strict maxima: at most every other bin
    const int row = blockIdx.y, seg = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int w = seg * kSegWords + tid;
    const uint32_t word = w < a.n_words ? a.mask[(int64_t)row * a.n_words + w] : 0u;
    const int c = __popc(word);
    int p = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, p, o);
        if (lane >= o) p += y;
    }
    if (lane == 31) wsum[warp] = p;
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int q = 0; q < kSegWords / 32; ++q) {
        before += q < warp ? wsum[q] : 0;
        total += wsum[q];
    }
    int pos = before + p - c;
    uint32_t m = word;
    while (m) {
        const int bit = __ffs(m) - 1;
        m &= m - 1;
        peaks_s[pos++] = w * 32 + bit;
    }
    __syncthreads();
    const int64_t base = a.seg_base[(int64_t)row * a.n_seg + seg];
    for (int k = tid; k < total; k += kSegWords) {
        const int64_t out = base + k;
        if (out < a.capacity) {
            const int32_t b = peaks_s[k];
            a.bins[out] = b;
            if (a.freq) a.freq[out] = a.fq(b);
        }
    }
}

// Exclusive scan of n int32 counts into int64: pref[0 .. n] (may be null) and
// strided[r] = pref[r * stride] for r = 0 .. n / stride (may be null).  One block.
__global__ void __launch_bounds__(kScanThreads)
scan_counts_kernel(const int32_t *cnt, int64_t n, int64_t *pref, int32_t stride, int64_t *strided)
{
    __shared__ int64_t part[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (n + kScanThreads - 1) / kScanThreads;
    const int64_t lo = min(n, (int64_t)tid * per), hi = min(n, lo + per);
    int64_t s = 0;
    for (int64_t k = lo; k < hi; ++k) s += cnt[k];
    int64_t p = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, p, o);
        if (lane >= o) p += y;
    }
    if (lane == 31) part[warp] = p;
    __syncthreads();
    int64_t before = 0;
    for (int q = 0; q < warp; ++q) before += part[q];
    int64_t run = before + p - s;
    for (int64_t k = lo; k < hi; ++k) {
        if (pref) pref[k] = run;
        if (strided && k % stride == 0) strided[k / stride] = run;
        run += cnt[k];
    }
    if (tid == kScanThreads - 1) {
        if (pref) pref[n] = run;
        if (strided) strided[n / stride] = run;
    }
}

// ---------------------------------------------------------------- cleaning
// The peak range of FFT i, clamped into [0, n_peaks] whatever the offsets hold;
// a CSR that is not one (o[0] != 0, o[n] != n_peaks or a decrease) is flagged.
__device__ __forceinline__ void peak_range(const int64_t *o, int i, int64_t n_peaks, int64_t &lo,
                                           int64_t &hi)
{
    lo = min(max(o[i], (int64_t)0), n_peaks);
    hi = min(max(o[i + 1], lo), n_peaks);
}

__global__ void check_csr_kernel(const int64_t *o, int32_t n_fft, int64_t n_peaks, int32_t *err)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n_fft; i += gridDim.x * blockDim.x) {
        bool bad = false;
        if (i == 0) bad = o[0] != 0;
        if (i == n_fft) bad = bad || o[n_fft] != n_peaks;
        if (i < n_fft) bad = bad || o[i] > o[i + 1];
        if (bad) atomicOr(err, kErrCsr);
    }
}

// floor(num / den) of the IEEE quotient: the product with inv = RN(1 / den)
// differs from the quotient by a few units of 2^-53 relative, so when it lies
// more than 1e-9 (relative, at least absolute) from an integer both have the
// same floor; otherwise the division decides.
__device__ __forceinline__ double floor_quot(double num, double den, double inv)
{
    const double q = __dmul_rn(num, inv);
    const double fq = floor(q);
    const double margin = 1e-9 * fmax(1.0, fabs(q));
    if (q - fq > margin && fq + 1.0 - q > margin) return fq;
    return floor(__ddiv_rn(num, den));
}

struct GrossCell {
    const double *t;
    FreqOf fq;
    double t0_h, dt_h, f0_h, df_h, inv_df;
    int32_t n_th, n_fh;
    // time cell of FFT i, or -1 off the grid
    __device__ __forceinline__ int64_t it_of(int i) const
    {
        const double x = floor(__ddiv_rn(__dsub_rn(__ldg(t + i), t0_h), dt_h));
        return (x >= 0.0 && x < (double)n_th) ? (int64_t)x : -1;
    }
    // gross cell of a peak of bin b in time cell it, or -1 off the grid
    __device__ __forceinline__ int32_t cell(int64_t it, int32_t b) const
    {
        if (it < 0) return -1;
        const double y = floor_quot(__dsub_rn(fq(b), f0_h), df_h, inv_df);
        return (y >= 0.0 && y < (double)n_fh) ? (int32_t)(it * n_fh + (int64_t)y) : -1;
    }
};

// warp per FFT: the gross cell of every peak (kept for the veto pass) and the
// histogram (warp-aggregated atomics)
__global__ void gross_hist_kernel(const int64_t *o, const int32_t *bins, int32_t n_fft,
                                  int64_t n_peaks, GrossCell g, int32_t *cell, int32_t *hist)
{
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_fft; i += nw) {
        int64_t lo, hi;
        peak_range(o, i, n_peaks, lo, hi);
        const int64_t it = g.it_of(i);
        for (int64_t q0 = lo; q0 < hi; q0 += 32) {
            const int64_t q = q0 + lane;
            const int32_t c = q < hi ? g.cell(it, __ldg(bins + q)) : -1;
            if (q < hi) cell[q] = c;
            // neighbouring peaks of an FFT mostly share a cell: one atomic per
            // distinct cell of the warp, adding its number of lanes
            const unsigned same = __match_any_sync(kFull, c);
            if (c >= 0 && lane == __ffs(same) - 1) atomicAdd(hist + c, __popc(same));
        }
    }
}

// warp per FFT: FFTs with a peak in each bin (bins outside [0, n_bins) are flagged)
__global__ void bin_hist_kernel(const int64_t *o, const int32_t *bins, int32_t n_fft,
                                int64_t n_peaks, int32_t n_bins, int32_t *hist, int32_t *err)
{
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_fft; i += nw) {
        int64_t lo, hi;
        peak_range(o, i, n_peaks, lo, hi);
        for (int64_t q = lo + lane; q < hi; q += 32) {
            const int32_t b = __ldg(bins + q);
            if (b >= 0 && b < n_bins)
                atomicAdd(hist + b, 1);
            else
                atomicOr(err, kErrInvalid);
        }
    }
}

// histogram of the per-bin counts: hc[v] = bins whose count is v (v <= vmax;
// larger counts, possible only for an invalid CSR, go to vmax and are flagged)
__global__ void count_hist_kernel(const int32_t *hist, int32_t n_bins, int32_t vmax, int32_t *hc,
                                  int32_t *err)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_bins; b += gridDim.x * blockDim.x) {
        int32_t v = hist[b];
        if (v < 0 || v > vmax) {
            atomicOr(err, kErrInvalid);
            v = v < 0 ? 0 : vmax;
        }
        atomicAdd(hc + v, 1);
    }
}

// the k-th smallest (0-based) of a multiset given by its value histogram
// h[0 .. nv): one block; every thread scans a contiguous run of values
__device__ int64_t kth_of_hist(const int32_t *h, int64_t nv, int64_t k, int64_t *part,
                               int64_t *result)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (nv + blockDim.x - 1) / blockDim.x;
    const int64_t lo = min(nv, (int64_t)tid * per), hi = min(nv, lo + per);
    int64_t s = 0;
    for (int64_t v = lo; v < hi; ++v) s += h[v];
    int64_t p = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, p, o);
        if (lane >= o) p += y;
    }
    if (lane == 31) part[warp] = p;
    if (tid == 0) *result = nv - 1;
    __syncthreads();
    int64_t run = p - s;
    for (int q = 0; q < warp; ++q) run += part[q];
    if (run <= k && k < run + s) {
        for (int64_t v = lo; v < hi; ++v) {
            run += h[v];
            if (k < run) {
                *result = v;
                break;
            }
        }
    }
    __syncthreads();
    const int64_t r = *result;
    __syncthreads();
    return r;
}

// App. "Robust statistic" on the per-bin counts, from their value histogram
// hc (vmax + 1 values) and n_bins values in all: m1 = median, m2 =
// median(|x - m1|) / 0.6745, thr = m1 + k m2.  The deviations are half-integers;
// hd (2 vmax + 1 entries, zeroed) receives their doubled values.  One block.
__global__ void __launch_bounds__(kScanThreads)
robust_stats_kernel(const int32_t *hc, int32_t vmax, int64_t n_bins, int32_t *hd, double k_sigma,
                    double *stats)
{
    __shared__ int64_t part[kScanThreads / 32];
    __shared__ int64_t res;
    const int64_t nv = (int64_t)vmax + 1;
    // median of an even count: the mean of the two middle values
    const int64_t ka = (n_bins - 1) / 2, kb = n_bins / 2;
    const int64_t va = kth_of_hist(hc, nv, ka, part, &res);
    const int64_t vb = kth_of_hist(hc, nv, kb, part, &res);
    const int64_t m1x2 = va + vb;  // 2 m1, an integer
    for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
        const int32_t c = hc[v];
        if (c) {
            const int64_t d = 2 * v - m1x2;
            atomicAdd(hd + (d < 0 ? -d : d), c);
        }
    }
    __syncthreads();
    const int64_t nd = 2 * nv + 1;
    const int64_t da = kth_of_hist(hd, nd, ka, part, &res);
    const int64_t db = kth_of_hist(hd, nd, kb, part, &res);
    if (threadIdx.x == 0) {
        const double m1 = __ddiv_rn((double)m1x2, 2.0);
        // median of |x - m1| = (da / 2 + db / 2) / 2, exact for these sizes
        const double med = __ddiv_rn((double)(da + db), 4.0);
        const double m2 = __ddiv_rn(med, 0.6745);
        stats[0] = m1;
        stats[1] = m2;
        stats[2] = __dadd_rn(m1, __dmul_rn(k_sigma, m2));
    }
}

// which peaks stay: the gross cell holds at most `thr` peaks (or is off the grid)
struct KeepGross {
    const int32_t *cell, *hist;
    int32_t thr;
    __device__ __forceinline__ bool operator()(int, int64_t q, int32_t) const
    {
        const int32_t c = cell[q];
        return c < 0 || hist[c] <= thr;
    }
};
// which peaks stay: the bin's count is not above the persistency threshold
struct KeepPersist {
    const int32_t *hist;
    const double *stats;
    int32_t n_bins;
    __device__ __forceinline__ bool operator()(int, int64_t, int32_t b) const
    {
        return b < 0 || b >= n_bins || !((double)hist[b] > stats[2]);
    }
};

// warp per FFT: kept peaks per FFT
template <class Keep>
__global__ void filter_count_kernel(const int64_t *o, const int32_t *bins, int32_t n_fft,
                                    int64_t n_peaks, Keep keep, int32_t *cnt)
{
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_fft; i += nw) {
        int64_t lo, hi;
        peak_range(o, i, n_peaks, lo, hi);
        int c = 0;
        for (int64_t q0 = lo; q0 < hi; q0 += 32) {
            const int64_t q = q0 + lane;
            const bool k = q < hi && keep(i, q, __ldg(bins + q));
            c += __popc(__ballot_sync(kFull, k));
        }
        if (lane == 0) cnt[i] = c;
    }
}

// warp per FFT: the kept peaks, in order, from the FFT's new offset
template <class Keep>
__global__ void filter_write_kernel(const int64_t *o, const int32_t *bins, int32_t n_fft,
                                    int64_t n_peaks, Keep keep, const int64_t *o_out,
                                    int64_t capacity, FreqOf fq, int32_t *bins_out,
                                    double *freq_out)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_fft; i += nw) {
        int64_t lo, hi;
        peak_range(o, i, n_peaks, lo, hi);
        int64_t pos = o_out[i];
        for (int64_t q0 = lo; q0 < hi; q0 += 32) {
            const int64_t q = q0 + lane;
            const int32_t b = q < hi ? __ldg(bins + q) : 0;
            const bool k = q < hi && keep(i, q, b);
            const unsigned m = __ballot_sync(kFull, k);
            const int64_t at = pos + __popc(m & lt);
            if (k && at < capacity) {
                bins_out[at] = b;
                if (freq_out) freq_out[at] = fq(b);
            }
            pos += __popc(m);
        }
    }
}

}  // namespace

cudaError_t launch_exclusive_scan(const int32_t *cnt, int64_t n, int64_t *pref, int32_t stride,
                                  int64_t *strided, cudaStream_t s)
{
    scan_counts_kernel<<<1, kScanThreads, 0, s>>>(cnt, n, pref, stride, strided);
    return cudaGetLastError();
}

namespace {

int warp_grid(int32_t n_fft)
{
    const int per_block = 8;  // warps of a 256-thread block
    return (int)std::min<int64_t>(((int64_t)n_fft + per_block - 1) / per_block, 65535);
}

// kept peaks -> new CSR and lists; *n_out and the device error word on the host
template <class Keep>
int run_filter(const int64_t *o, const int32_t *bins, int32_t n_fft, int64_t n_peaks, Keep keep,
               int64_t k0, double t_fft, int64_t *o_out, int32_t *bins_out, double *freq_out,
               int64_t capacity, int64_t *n_out, const int32_t *err, Scratch &sc, cudaStream_t s)
{
    int32_t *cnt = nullptr;
    cudaError_t e = sc.get(&cnt, (size_t)n_fft);
    const int grid = warp_grid(n_fft);
    if (e == cudaSuccess && n_fft > 0) {
        filter_count_kernel<<<grid, 256, 0, s>>>(o, bins, n_fft, n_peaks, keep, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        scan_counts_kernel<<<1, kScanThreads, 0, s>>>(cnt, n_fft, nullptr, 1, o_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n_fft > 0) {
        filter_write_kernel<<<grid, 256, 0, s>>>(o, bins, n_fft, n_peaks, keep, o_out, capacity,
                                                 make_freq_of(k0, t_fft), bins_out, freq_out);
        e = cudaGetLastError();
    }
    int64_t total = 0;
    int32_t h_err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, o_out + n_fft, sizeof(total), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "peakmap filter");
    if (h_err & kErrCsr) return set_error(FH_ERR_INVALID_ARG, "offsets are not a CSR of n_peaks");
    if (h_err & kErrInvalid)
        return set_error(FH_ERR_INVALID_ARG, "a bin index outside [0, n_bins)");
    *n_out = total;
    if (total > capacity)
        return set_error(FH_ERR_CAPACITY, "%lld peaks kept, capacity %lld", (long long)total,
                         (long long)capacity);
    return FH_OK;
}

int check_peakmap_args(const int64_t *o, const int32_t *bins, int32_t n_fft, int64_t n_peaks,
                       const int64_t *o_out, const int32_t *bins_out, int64_t capacity,
                       const int64_t *n_out)
{
    if (!o || !o_out || !n_out || (n_peaks > 0 && !bins) || (capacity > 0 && !bins_out))
        return set_error(FH_ERR_INVALID_ARG, "null offsets, bins or output");
    if (n_fft < 0 || n_peaks < 0 || n_peaks >= ((int64_t)1 << 40) || capacity < 0)
        return set_error(FH_ERR_INVALID_ARG, "need n_fft >= 0, n_peaks in [0, 2^40), capacity >= 0");
    return FH_OK;
}

}  // namespace
}  // namespace fh

using namespace fh;

extern "C" {

int64_t fh_peakmap_select_workspace(int32_t n_fft, int32_t n_bins)
{
    if (n_fft < 0 || n_bins < 0) return -1;
    const int64_t n_seg = (n_bins + kSegBins - 1) / kSegBins;
    const int64_t n_words = (n_bins + 31) / 32;
    auto up = [](int64_t b) { return (b + 255) / 256 * 256; };
    return up(4 * n_fft * n_words) + up(4 * n_fft * n_seg) + up(8 * (n_fft * n_seg + 1)) + 256;
}

int fh_peakmap_select(const float *s_p, const float *s_ar, int32_t n_fft, int32_t n_bins,
                      int64_t pitch, float theta, int64_t k0, double t_fft, int64_t *offsets,
                      int32_t *bins, double *freq, int64_t capacity, int64_t *n_peaks,
                      void *workspace, int64_t workspace_bytes, void *stream)
{
    if (!offsets || (n_fft > 0 && n_bins > 0 && (!s_p || !s_ar)) || (capacity > 0 && !bins))
        return set_error(FH_ERR_INVALID_ARG, "null spectrum, offsets, bins or n_peaks");
    if (n_fft < 0 || n_fft > 65535 * 1024 || n_bins < 0 || pitch < n_bins || capacity < 0)
        return set_error(FH_ERR_INVALID_ARG, "need n_fft >= 0, n_bins >= 0, pitch >= n_bins, "
                                             "capacity >= 0");
    if ((int64_t)n_fft * (n_bins / kSegBins + 1) > ((int64_t)1 << 31))
        return set_error(FH_ERR_INVALID_ARG, "spectra too large");
    if (!(t_fft > 0.0) || !std::isfinite(t_fft) || std::isnan(theta))
        return set_error(FH_ERR_INVALID_ARG, "need t_fft > 0 and a threshold");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int32_t n_seg = (n_bins + kSegBins - 1) / kSegBins;
    const int32_t n_words = (n_bins + 31) / 32;
    if (n_fft == 0 || n_seg == 0) {
        cudaError_t e = cudaMemsetAsync(offsets, 0, sizeof(int64_t) * (n_fft + 1), s);
        if (e == cudaSuccess && n_peaks) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync (peakmap)");
        if (n_peaks) *n_peaks = 0;
        return FH_OK;
    }
    if (n_fft > 65535) return set_error(FH_ERR_INVALID_ARG, "at most 65535 FFTs per call");
    Scratch sc(s);
    uint32_t *mask = nullptr;
    int32_t *seg_count = nullptr, *err = nullptr;
    int64_t *seg_base = nullptr;
    cudaError_t e = cudaSuccess;
    const int64_t need = fh_peakmap_select_workspace(n_fft, n_bins);
    if (workspace) {
        if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
            return set_error(FH_ERR_INVALID_ARG, "workspace of %lld bytes (256-byte aligned) "
                                                 "needed", (long long)need);
        char *w = static_cast<char *>(workspace);
        auto up = [](int64_t b) { return (b + 255) / 256 * 256; };
        mask = reinterpret_cast<uint32_t *>(w);
        seg_count = reinterpret_cast<int32_t *>(w + up(4 * (int64_t)n_fft * n_words));
        seg_base = reinterpret_cast<int64_t *>(w + up(4 * (int64_t)n_fft * n_words) +
                                               up(4 * (int64_t)n_fft * n_seg));
        err = reinterpret_cast<int32_t *>(w + need - 256);
    } else {
        e = sc.get(&mask, (size_t)n_fft * n_words);
        if (e == cudaSuccess) e = sc.get(&seg_count, (size_t)n_fft * n_seg);
        if (e == cudaSuccess) e = sc.get(&seg_base, (size_t)n_fft * n_seg + 1);
        if (e == cudaSuccess) e = sc.get(&err, 4);
        if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync (peakmap)");
    }
    SelArgs a{s_p, s_ar, pitch, n_fft, n_bins, n_seg, n_words, theta, mask, seg_count, err};
    const bool vec = ((reinterpret_cast<uintptr_t>(s_p) | reinterpret_cast<uintptr_t>(s_ar)) &
                      15u) == 0 && (pitch & 3) == 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync (peakmap)");
    if (vec && (n_bins & 3) == 0)
        select_mask_bulk_kernel<<<dim3(n_seg, n_fft), kSegThreads, 0, s>>>(a);
    else if (vec)
        select_mask_kernel<true><<<dim3(n_seg, n_fft), kSegThreads, 0, s>>>(a);
    else
        select_mask_kernel<false><<<dim3(n_seg, n_fft), kSegThreads, 0, s>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        scan_counts_kernel<<<1, kScanThreads, 0, s>>>(seg_count, (int64_t)n_fft * n_seg,
                                                      seg_base, n_seg, offsets);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ExpandArgs x{mask, seg_base, n_seg, n_words, capacity, make_freq_of(k0, t_fft), bins,
                     freq};
        select_expand_kernel<<<dim3(n_seg, n_fft), kSegWords, 0, s>>>(x);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_error(e, "peak selection");
    if (!n_peaks) return FH_OK;  // asynchronous: the total is offsets[n_fft]
    int64_t total = 0;
    int32_t h_err = 0;
    e = cudaMemcpyAsync(&total, offsets + n_fft, sizeof(total), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "peak selection");
    if (h_err) return set_error(FH_ERR_TIMEOUT, "peak selection: a bulk-copy wait ran out");
    *n_peaks = total;
    if (total > capacity)
        return set_error(FH_ERR_CAPACITY, "%lld peaks selected, capacity %lld", (long long)total,
                         (long long)capacity);
    return FH_OK;
}

int fh_peakmap_gross_veto(const double *t, const int64_t *offsets, const int32_t *bins,
                          int32_t n_fft, int64_t n_peaks, int64_t k0, double t_fft, double t0_h,
                          double dt_h, int32_t n_th, double f0_h, double df_h, int32_t n_fh,
                          int32_t threshold, int32_t *hist, int64_t *offsets_out,
                          int32_t *bins_out, double *freq_out, int64_t capacity, int64_t *n_out,
                          void *stream)
{
    int rc = check_peakmap_args(offsets, bins, n_fft, n_peaks, offsets_out, bins_out, capacity,
                                n_out);
    if (rc) return rc;
    if ((n_fft > 0 && !t) || !hist || n_th < 1 || n_fh < 1 ||
        (int64_t)n_th * n_fh > ((int64_t)1 << 31) || !(dt_h > 0.0) || !(df_h > 0.0) ||
        !(t_fft > 0.0) || !std::isfinite(t0_h) || !std::isfinite(f0_h) ||
        !std::isfinite(dt_h) || !std::isfinite(df_h) || !std::isfinite(t_fft))
        return set_error(FH_ERR_INVALID_ARG, "bad gross grid (n_th, n_fh >= 1, steps > 0)");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch sc(s);
    int32_t *err = nullptr;
    cudaError_t e = sc.get(&err, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * (size_t)n_th * n_fh, s);
    if (e == cudaSuccess) {
        check_csr_kernel<<<(n_fft + 256) / 256, 256, 0, s>>>(offsets, n_fft, n_peaks, err);
        e = cudaGetLastError();
    }
    GrossCell g{t, make_freq_of(k0, t_fft), t0_h, dt_h, f0_h, df_h, 1.0 / df_h, n_th, n_fh};
    int32_t *cell = nullptr;
    if (e == cudaSuccess) e = sc.get(&cell, (size_t)n_peaks);
    if (e == cudaSuccess && n_fft > 0) {
        gross_hist_kernel<<<warp_grid(n_fft), 256, 0, s>>>(offsets, bins, n_fft, n_peaks, g, cell,
                                                           hist);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_error(e, "gross histogram");
    return run_filter(offsets, bins, n_fft, n_peaks, KeepGross{cell, hist, threshold}, k0, t_fft,
                      offsets_out, bins_out, freq_out, capacity, n_out, err, sc, s);
}

int fh_peakmap_persistency_veto(const int64_t *offsets, const int32_t *bins, int32_t n_fft,
                                int64_t n_peaks, int32_t n_bins, double k_sigma, int64_t k0,
                                double t_fft, int32_t *hist, double *stats,
                                int64_t *offsets_out, int32_t *bins_out, double *freq_out,
                                int64_t capacity, int64_t *n_out, void *stream)
{
    int rc = check_peakmap_args(offsets, bins, n_fft, n_peaks, offsets_out, bins_out, capacity,
                                n_out);
    if (rc) return rc;
    if (!hist || !stats || n_bins < 1 || !std::isfinite(k_sigma) || !(t_fft > 0.0) ||
        !std::isfinite(t_fft))
        return set_error(FH_ERR_INVALID_ARG, "need n_bins >= 1, finite k_sigma, t_fft > 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch sc(s);
    int32_t *err = nullptr, *hc = nullptr, *hd = nullptr;
    double *d_stats = nullptr;
    // a bin's count is at most n_fft for a valid CSR; one more value catches the rest
    const int32_t vmax = n_fft + 1;
    cudaError_t e = sc.get(&err, 1);
    if (e == cudaSuccess) e = sc.get(&hc, (size_t)vmax + 1);
    if (e == cudaSuccess) e = sc.get(&hd, 2 * ((size_t)vmax + 1) + 1);
    if (e == cudaSuccess) e = sc.get(&d_stats, 3);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * (size_t)n_bins, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hc, 0, sizeof(int32_t) * ((size_t)vmax + 1), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(hd, 0, sizeof(int32_t) * (2 * ((size_t)vmax + 1) + 1), s);
    if (e == cudaSuccess) {
        check_csr_kernel<<<(n_fft + 256) / 256, 256, 0, s>>>(offsets, n_fft, n_peaks, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n_fft > 0) {
        bin_hist_kernel<<<warp_grid(n_fft), 256, 0, s>>>(offsets, bins, n_fft, n_peaks, n_bins,
                                                         hist, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int grid = (int)std::min<int64_t>(((int64_t)n_bins + 255) / 256, 4096);
        count_hist_kernel<<<grid, 256, 0, s>>>(hist, n_bins, vmax, hc, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        robust_stats_kernel<<<1, kScanThreads, 0, s>>>(hc, vmax, n_bins, hd, k_sigma, d_stats);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(stats, d_stats, 24, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_error(e, "persistency histogram");
    return run_filter(offsets, bins, n_fft, n_peaks, KeepPersist{hist, d_stats, n_bins}, k0,
                      t_fft, offsets_out, bins_out, freq_out, capacity, n_out, err, sc, s);
}

}  // extern "C"
