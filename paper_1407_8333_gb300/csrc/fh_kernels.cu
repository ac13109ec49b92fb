// Kernels of the frequency-Hough hot path (sm_103a).
//
//   correct_kernel       a1 - a3  one launch: CSR sanitising, per-FFT spin-down shift
//                                 (Eqs. uno, sdstep) and input checks, Doppler factor
//                                 and 32.32 fixed-point stripe start (Eq. fdopp;
//                                 Sec. VI; Eq. freqres) of every direction
//   prep_kernel          a3       the shift tables, CSR sanitising and checks alone
//   positions_kernel     a1 + a2  the positions alone, also of several peakmaps
//                                 (refined-grid search)
//   windows_kernel       a4       which peaks can reach each tile; clears the profile
//   transform_kernel     a4 + a5 + profile half of a6 (Eqs. due, ncount; Sec. VIII)
//   select_kernel        a6       per-sub-band greedy picks (Sec. VIII; Eq. cr)
//
// Floating point: every binary64 operation is an explicit round-to-nearest
// intrinsic (__dmul_rn, __dadd_rn, ...), so nothing is contracted into an FMA
// and the results are the IEEE values of the operations in the stated order.
// The final floor(x 2^32) of a peak position is taken exactly from the IEEE
// fields of x with integer operations.  After it the path is integer only.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <utility>

#include "fh_internal.h"

namespace fh {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kTwo32 = 4294967296.0;
constexpr int kPosFfts = 8;
constexpr int kPosThreads = 256;

// ---------------------------------------------------------------- a1 + a2
// several peakmaps in one launch (see positions_kernel); null a_base: one
struct PosBatch {
    const int64_t *a_base, *n_peaks;
};

// floor(x 2^32) for |x| < 2^28, exactly: x = m 2^(e - 1075) with m the
// significand (hidden bit included for normal numbers), so x 2^32 =
// m 2^(e - 1043), a left shift by at most 7 bits, or a right shift whose
// discarded bits round a negative value down.  Out-of-range inputs give some
// value; the caller flags them.
__device__ __forceinline__ int64_t floor_times_2p32(double x)
{
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (ex ? (uint64_t(1) << 52) : 0);
    const int sh = (ex ? ex : 1) - 1043;
    uint64_t q;
    bool frac;
    if (sh >= 0) {
        q = m << (sh < 10 ? sh : 10);
        frac = false;
    } else {
        const int rs = -sh;
        q = rs < 64 ? m >> rs : 0;
        frac = rs < 64 ? (m & ((uint64_t(1) << rs) - 1)) != 0 : m != 0;
    }
    return (bits >> 63) ? -(int64_t)q - (frac ? 1 : 0) : (int64_t)q;
}

// grid (ceil(n_fft / 8), n_dir): the block computes r = 1 / (1 + v.n) for 8
// FFTs of one direction, then the fixed-point position of each of their peaks
// (a contiguous CSR range, so loads and stores are coalesced).  With `src`,
// FFT i's peaks are read from freq[src[i] ...] (a sub-range of a larger
// peakmap) and written compactly by `offsets`.  With `validate`, the blocks of
// direction 0 also flag frequencies that are not finite and positive
// (kErrInvalid) or not strictly increasing within their FFT (kErrUnsorted).
// The body of one positions block: group `group` of 8 FFTs, direction d.
// With clamp_offsets the CSR entries are raw: each is clamped into
// [0, n_peaks] and made non-decreasing within the block, which keeps every
// access in bounds (a valid CSR is unchanged; an invalid one is flagged by the
// global CSR pass).
__device__ __forceinline__ void positions_block(
    const double *__restrict__ freq, const int64_t *__restrict__ offsets, bool clamp_offsets,
    const double *__restrict__ v, const double *__restrict__ sky, int32_t n_fft, int64_t n_peaks,
    double f0_min, double kt, double cshift, int64_t *__restrict__ A, double *__restrict__ out_r,
    int32_t *err, int32_t validate, const int64_t *__restrict__ src, int d, int group)
{
    __shared__ double r_s[kPosFfts];
    __shared__ int64_t off_s[kPosFfts + 1];
    __shared__ int64_t src_s[kPosFfts];  // where each FFT's peaks start in freq
    const int i0 = group * kPosFfts;
    const int nf = min(kPosFfts, n_fft - i0);
    if (threadIdx.x < nf) {
        const int i = i0 + threadIdx.x;
        const double px = __dmul_rn(v[3 * (int64_t)i + 0], sky[3 * (int64_t)d + 0]);
        const double py = __dmul_rn(v[3 * (int64_t)i + 1], sky[3 * (int64_t)d + 1]);
        const double pz = __dmul_rn(v[3 * (int64_t)i + 2], sky[3 * (int64_t)d + 2]);
        const double dot = __dadd_rn(__dadd_rn(px, py), pz);
        const double den = __dadd_rn(1.0, dot);
        const double r = __ddiv_rn(1.0, den);
        r_s[threadIdx.x] = r;
        if (out_r) out_r[(int64_t)d * n_fft + i] = r;
    }
    if (threadIdx.x <= nf) {
        int64_t o = offsets[i0 + threadIdx.x];
        if (clamp_offsets) o = o < 0 ? 0 : (o > n_peaks ? n_peaks : o);
        off_s[threadIdx.x] = o;
    }
    if (!clamp_offsets && threadIdx.x < nf)
        src_s[threadIdx.x] = src ? src[i0 + threadIdx.x] : offsets[i0 + threadIdx.x];
    __syncthreads();
    if (clamp_offsets) {
        if (threadIdx.x == 0)
            for (int k = 0; k <= nf; ++k) {
                if (k > 0 && off_s[k] < off_s[k - 1]) off_s[k] = off_s[k - 1];
                if (k < nf) src_s[k] = off_s[k];
            }
        __syncthreads();
    }
    const int64_t p_begin = off_s[0], p_end = off_s[nf];
    int64_t *__restrict__ Ad = A + (int64_t)d * n_peaks;
    const bool check = validate && d == 0;
    const int lane = threadIdx.x & 31;
    bool bad = false;
    int32_t ev = 0;
    // whole warps step together (the shuffle below needs all lanes)
    for (int64_t pw = p_begin + (threadIdx.x & ~31); pw < p_end; pw += blockDim.x) {
        const int64_t p = pw + lane;
        const bool in = p < p_end;
        int lo = 0, hi = nf;  // off_s[lo] <= p < off_s[hi]
        while (hi - lo > 1) {
            const int m = (lo + hi) >> 1;
            if (off_s[m] <= p) lo = m; else hi = m;
        }
        const int64_t fp = src_s[lo] + (p - off_s[lo]);
        const double f = in ? freq[fp] : 1.0;
        if (check) {
            // positive finite doubles order like their bit patterns
            const int64_t fb = __double_as_longlong(f);
            int64_t prev = __shfl_up_sync(kFull, fb, 1);
            if (lane == 0 && in && p > off_s[lo]) prev = __double_as_longlong(freq[fp - 1]);
            if (in) {
                if (!(fb > 0 && fb < 0x7FF0000000000000LL)) ev |= kErrInvalid;
                if (p > off_s[lo] && !(fb > prev)) ev |= kErrUnsorted;
            }
        }
        if (in) {
            const double u = __dmul_rn(f, r_s[lo]);
            const double x = __dsub_rn(u, f0_min);
            const double y = __dmul_rn(x, kt);
            const double a = __dadd_rn(y, cshift);
            // |a| < 2^28 exactly when the biased exponent is below 1023 + 28
            bad |= ((__double_as_longlong(a) >> 52) & 0x7FF) >= 1051;
            Ad[p] = floor_times_2p32(a);
        }
    }
    if (ev) atomicOr(err, ev);
    if (bad) atomicOr(err, kErrRange);
}

__global__ void __launch_bounds__(kPosThreads)
positions_kernel(const double *__restrict__ freq, const int64_t *__restrict__ offsets,
                 const double *__restrict__ v, const double *__restrict__ sky, int32_t n_fft,
                 int64_t n_peaks, double f0_min, double kt, double cshift,
                 int64_t *__restrict__ A, double *__restrict__ out_r, int32_t *err,
                 int32_t validate, const int64_t *__restrict__ src, PosBatch batch)
{
    // batches (refinement): block z is one peakmap of several, each with its own
    // offsets, source index, sky directions, output base and peak count
    if (batch.a_base) {
        const int c = blockIdx.z;
        offsets += (int64_t)c * (n_fft + 1);
        src += (int64_t)c * n_fft;
        sky += 3 * (int64_t)c * gridDim.y;
        A += batch.a_base[c];
        n_peaks = batch.n_peaks[c];
    }
    positions_block(freq, offsets, false, v, sky, n_fft, n_peaks, f0_min, kt, cshift, A, out_r,
                    err, validate, src, blockIdx.y, blockIdx.x);
}

// ---------------------------------------------------------------- a3 + per-call set-up
// The CSR pass (one block of any size): 4 consecutive entries per thread
// (4 x blockDim per pass), a running maximum inside the thread, a warp scan and
// one block step carry it across the pass; raw entries outside [0, n_peaks],
// a first entry other than 0, a last other than n_peaks or a decrease are
// flagged (kErrCsr).
__device__ __forceinline__ void csr_pass(const PrepArgs &a, int32_t &e)
{
    __shared__ int64_t wmax[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = a.n_fft;
    const int nt = blockDim.x;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base <= n; base += 4 * nt) {
        const int i0 = base + 4 * threadIdx.x;
        int64_t x[4];
        int64_t prev_raw = (i0 > 0 && i0 <= n) ? a.offsets_in[i0 - 1] : 0;
        int64_t run = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            int64_t y = 0;
            if (i <= n) {
                const int64_t raw = a.offsets_in[i];
                if (raw < 0 || raw > a.n_peaks) e |= kErrCsr;
                if (i == 0 && raw != 0) e |= kErrCsr;
                if (i == n && raw != a.n_peaks) e |= kErrCsr;
                if (i > 0 && raw < prev_raw) e |= kErrCsr;
                prev_raw = raw;
                y = raw < 0 ? 0 : (raw > a.n_peaks ? a.n_peaks : raw);
                if (i == 0) y = 0;
            }
            run = y > run ? y : run;
            x[j] = run;
        }
        // exclusive running maximum of the threads before this one
        int64_t inc = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o && y > inc) inc = y;
        }
        int64_t exc = __shfl_up_sync(kFull, inc, 1);
        if (lane == 0) exc = 0;
        if (lane == 31) wmax[warp] = inc;
        __syncthreads();
        int64_t pre = carry;
        for (int w = 0; w < warp; ++w) pre = wmax[w] > pre ? wmax[w] : pre;
        pre = exc > pre ? exc : pre;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            if (i <= n) a.offsets_out[i] = (i == n) ? a.n_peaks : (x[j] > pre ? x[j] : pre);
        }
        __syncthreads();
        if (threadIdx.x == nt - 1) carry = inc > pre ? inc : pre;
        __syncthreads();
    }
}

// Shift tables of FFT i (a3) and its checks; |D_i| into amax.
__device__ __forceinline__ void fft_tables(const PrepArgs &a, int i, int32_t &e,
                                           unsigned long long &amax)
{
    const double f_last = __dadd_rn(a.fdot_min, __dmul_rn((double)(a.n_fdot - 1), a.fdot_step));
    const double absmax = fabs(a.fdot_min) > fabs(f_last) ? fabs(a.fdot_min) : fabs(f_last);
    const double ti = a.t[i];
    const double dt = __dsub_rn(ti, a.t_ref);
    const double c = __dmul_rn(dt, a.kt);
    const double s0 = __dmul_rn(a.fdot_min, c);
    const double dd = __dmul_rn(a.fdot_step, c);
    if (!(fabs(c) * absmax < (double)kFixedLimit)) e |= kErrRange;
    a.S0[i] = (int64_t)floor(__dmul_rn(s0, kTwo32));
    const int64_t Di = (int64_t)floor(__dmul_rn(dd, kTwo32));
    a.D[i] = Di;
    const unsigned long long m = (unsigned long long)(Di < 0 ? -Di : Di);
    amax = m > amax ? m : amax;
    if (a.validate) {
        if (!isfinite(ti) || (i > 0 && !(ti > a.t[i - 1]))) e |= kErrUnsorted;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (!(fabs(a.v[3 * (int64_t)i + k]) < 0.1)) e |= kErrInvalid;
    }
}

__device__ __forceinline__ void sky_checks(const PrepArgs &a, int32_t &e)
{
    for (int d = threadIdx.x; d < a.n_dir; d += blockDim.x) {
        const double x = a.sky[3 * (int64_t)d], y = a.sky[3 * (int64_t)d + 1],
                     z = a.sky[3 * (int64_t)d + 2];
        if (!(fabs(x) <= 1.000001 && fabs(y) <= 1.000001 && fabs(z) <= 1.000001))
            e |= kErrInvalid;
    }
}

// the warp's largest |D| and error bits, one atomic each
__device__ __forceinline__ void flush_prep(const PrepArgs &a, int32_t e, unsigned long long amax)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_down_sync(kFull, amax, o);
        amax = y > amax ? y : amax;
    }
    if ((threadIdx.x & 31) == 0 && amax) atomicMax(a.dmax, amax);
    e = (int32_t)__reduce_or_sync(kFull, (unsigned)e);
    if ((threadIdx.x & 31) == 0 && e) atomicOr(a.err, e);
}

// grid 1 + ceil(n_fft / 1024), 1024 threads (see PrepArgs).  Block 0 sanitises
// the CSR and checks the sky directions; block b > 0 takes FFTs
// (b - 1) * 1024 ... b * 1024 - 1.
__global__ void __launch_bounds__(1024, 1) prep_kernel(const PrepArgs a)
{
    int32_t e = 0;
    unsigned long long amax = 0;
    if (blockIdx.x == 0) {
        if (a.offsets_in) csr_pass(a, e);
        if (a.validate) sky_checks(a, e);
    } else {
        const int i = (int)(blockIdx.x - 1) * 1024 + (int)threadIdx.x;
        if (i < a.n_fft) fft_tables(a, i, e, amax);
    }
    flush_prep(a, e, amax);
}

// a1 - a3 in one launch (fh_correct_doppler): grid (1 + ceil(n_fft / 8), n_dir),
// kPosThreads threads.  Block (0, 0) sanitises the CSR for the later kernels
// and checks the sky directions; block (x, d), x >= 1, computes the positions
// of FFTs 8 (x - 1) .. 8 (x - 1) + 7 for direction d (clamping the raw CSR
// entries it reads when they still need sanitising, so it does not wait for
// block (0, 0)), and the blocks of direction 0 also the shift tables and
// per-FFT checks of their FFTs.
__global__ void __launch_bounds__(kPosThreads)
correct_kernel(const PrepArgs a, const double *__restrict__ freq, double f0_min, double cshift,
               int64_t *__restrict__ A, double *__restrict__ out_r)
{
    int32_t e = 0;
    unsigned long long amax = 0;
    if (blockIdx.x == 0) {
        if (blockIdx.y != 0) return;
        if (a.offsets_in) csr_pass(a, e);
        if (a.validate) sky_checks(a, e);
        flush_prep(a, e, amax);
        return;
    }
    const int group = (int)blockIdx.x - 1, d = (int)blockIdx.y;
    if (d == 0) {
        const int i = group * kPosFfts + (int)threadIdx.x;
        if (threadIdx.x < kPosFfts && i < a.n_fft) fft_tables(a, i, e, amax);
        if (threadIdx.x < 32) flush_prep(a, e, amax);
    }
    const bool raw = a.offsets_in != nullptr;
    positions_block(freq, raw ? a.offsets_in : a.offsets_out, raw, a.v, a.sky, a.n_fft, a.n_peaks,
                    f0_min, a.kt, cshift, A, out_r, a.err, a.validate, nullptr, d, group);
}


// ---------------------------------------------------------------- device inputs
// Flags non-finite / unordered device inputs (the refined-grid search under
// device-side checks): one warp per FFT (its peaks are read coalesced and
// compared with their left neighbour, through an already sanitised CSR) and
// one thread per sky direction.
__global__ void validate_device_inputs_kernel(const double *__restrict__ t,
                                              const double *__restrict__ freq,
                                              const int64_t *__restrict__ offsets,
                                              const double *__restrict__ v,
                                              const double *__restrict__ sky, int32_t n_fft,
                                              int32_t n_dir, int32_t *err)
{
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int32_t e = 0;
    if (gw < n_fft) {
        const int i = gw;
        if (lane == 0) {
            if (!isfinite(t[i]) || (i > 0 && !(t[i] > t[i - 1]))) e |= kErrUnsorted;
            for (int c = 0; c < 3; ++c)
                if (!(fabs(v[3 * (int64_t)i + c]) < 0.1)) e |= kErrInvalid;
        }
        const int64_t o0 = offsets[i], o1 = offsets[i + 1];
        for (int64_t p = o0 + lane; p < o1; p += 32) {
            const double f = freq[p];
            if (!isfinite(f) || !(f > 0.0)) e |= kErrInvalid;
            if (p > o0 && !(f > freq[p - 1])) e |= kErrUnsorted;
        }
    }
    const int gt = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (gt < n_dir) {
        const double x = sky[3 * (int64_t)gt], y = sky[3 * (int64_t)gt + 1],
                     z = sky[3 * (int64_t)gt + 2];
        if (!(fabs(x) <= 1.000001 && fabs(y) <= 1.000001 && fabs(z) <= 1.000001))
            e |= kErrInvalid;
    }
    e = (int32_t)__reduce_or_sync(kFull, (unsigned)e);
    if (lane == 0 && e) atomicOr(err, e);
}

// ---------------------------------------------------------------- a4 + a5 + profile
// Peak window of FFT i on rows j0 .. j0 + R - 1 of a tile whose stripe starts
// L lie in [0, E), found by binary search over the FFT's ascending positions:
// the peaks with lo <= A < hi, lo = cb + min(0, (R-1) D), hi = cb + max(0,
// (R-1) D) + E 2^32, cb = S0 + j0 D + tile origin.  Outputs cb, D, the first
// peak q0 and the count n (0 for i >= n_fft).  Every index stays inside the
// FFT's CSR range for any input.  (Used where no window table was built.)
__device__ __forceinline__ void lookup_window(const int64_t *__restrict__ Ad,
                                              const int64_t *__restrict__ offs,
                                              const int64_t *__restrict__ S0,
                                              const int64_t *__restrict__ Dt, int n_fft, int i,
                                              int j0, int R, int64_t base_shift, int64_t e_fixed,
                                              int64_t &cb, int64_t &dv, int64_t &q0, int &n)
{
    const bool ok = i < n_fft;
    const int ii = ok ? i : 0;
    const int64_t o0 = ok ? __ldg(offs + ii) : 0;
    const int64_t o1 = ok ? __ldg(offs + ii + 1) : 0;
    dv = ok ? __ldg(Dt + ii) : 0;
    const int64_t s0 = ok ? __ldg(S0 + ii) : 0;
    cb = s0 + (int64_t)j0 * dv + base_shift;
    const int64_t span = (int64_t)(R - 1) * dv;
    const int64_t lo = cb + (span < 0 ? span : 0);
    const int64_t hi = cb + (span > 0 ? span : 0) + e_fixed;
    int64_t a = o0, b = o1;
    while (a < b) {
        const int64_t m = (a + b) >> 1;
        if (__ldg(Ad + m) < lo) a = m + 1; else b = m;
    }
    q0 = a;
    b = o1;
    while (a < b) {
        const int64_t m = (a + b) >> 1;
        if (__ldg(Ad + m) < hi) a = m + 1; else b = m;
    }
    n = (int)(a - q0);
}

// The transform's peak window of every (direction, slab, tile, FFT), to whole
// cells: the peaks whose cell floor(A / 2^32) lies in
// [floor(lo / 2^32), ceil(hi / 2^32)), where [lo, hi) is the hull of the
// positions whose stripe reaches the tile on some row of the slab.  The
// window is a superset of the peaks that reach the tile, by less than one cell
// on each side; those extra peaks reach only guard cells (the transform's
// guard keeps a margin of two cells), so they change no count.  For a pair of
// directions (PAIR) the entry is the union, as one index range, of the two
// directions' windows: with c_max(k) and c_min(k) the larger and the smaller
// of peak k's two cells (both non-decreasing in k, as each direction's cells
// are), the union of [lb_a(x), lb_a(y)) and [lb_b(x), lb_b(y)) is
// [lb_max(x), lb_min(y)), lb the first index whose cell is >= the bound -- so a
// pair costs two searches per entry, like one direction.  (Were one window
// empty, this range could also hold peaks whose two cells lie on both sides of
// the tile; the guard allowance for the pair distance makes that impossible
// on the paired walk, and the clamped walk takes any range.)
//
// A block takes 8 FFTs of one unit (a direction, or a pair of them): warp w
// copies FFT w's peak cells (for a pair: c_max and c_min) into shared memory
// once, between one sentinel on each side, four loads per lane in flight (an
// FFT with more than kPeaks - 2 peaks is read from global memory, with bounds
// checks, by the whole block).  Lane l of warp w then takes FFT l mod 8 and
// tiles 4 w + l / 8 + 32 m (M per pass, M = 1 .. 3 from the tile count, so
// that the per-slab work -- the 64-bit bounds, the branches -- is shared by M
// entries and the M searches of a slab are independent), and walks the slabs
// in order: the first slab's bounds come from a binary search, each later one
// from a step in the direction of its FFT's drift D (both bounds move
// monotonically with the slab, by 32 D; D does not depend on the direction).
// A warp's 32 entries of a slab are 4 tiles x 8 consecutive FFTs, i.e. four
// 32-byte runs of the [slab][tile][FFT] table, so each warp writes its own
// runs and the slab loop has no barrier.
// grid (ceil(n_fft / 8), units), 256 threads.
constexpr int kWinPad = 1;
constexpr int kWinMaxM = 3;
__device__ __forceinline__ int lower_bound_cell(const int32_t *a, int n, int x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (a[m] < x) lo = m + 1; else hi = m;
    }
    return lo;
}
__device__ __forceinline__ int global_cell(const int64_t *A, int k) { return (int)(A[k] >> 32); }
__device__ __forceinline__ int lower_bound_cell_g(const int64_t *A, int n, int x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (global_cell(A, m) < x) lo = m + 1; else hi = m;
    }
    return lo;
}
// first index >= q whose cell is >= x (a[n] is a sentinel): one predicated
// step, then a loop for the rare longer moves
__device__ __forceinline__ int step_up(const int32_t *a, int q, int x)
{
    q += a[q] < x;
    while (a[q] < x) ++q;
    return q;
}
// first index <= q whose cell is >= x, everything before it below x
// (a[-1] is a sentinel)
__device__ __forceinline__ int step_down(const int32_t *a, int q, int x)
{
    q -= a[q - 1] >= x;
    while (a[q - 1] >= x) --q;
    return q;
}

// cell of peak k for the lower (HI = false: the larger of a pair's two cells)
// or the upper (HI = true: the smaller) window bound; Ab = Aa for one direction
template <bool HI>
__device__ __forceinline__ int pair_cell_g(const int64_t *Aa, const int64_t *Ab, int k)
{
    const int ca = global_cell(Aa, k), cb = global_cell(Ab, k);
    return HI ? min(ca, cb) : max(ca, cb);
}
template <bool HI>
__device__ __forceinline__ int lower_bound_pair_g(const int64_t *Aa, const int64_t *Ab, int n,
                                                  int x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (pair_cell_g<HI>(Aa, Ab, m) < x) lo = m + 1; else hi = m;
    }
    return lo;
}

template <int M, bool PAIR>
__global__ void __launch_bounds__(256, 4)
windows_kernel(const TransformJob J, uint32_t *__restrict__ windows)
{
    constexpr int kTiles = 32 * M;  // tiles per pass
    constexpr int NR = PAIR ? 2 : 1;  // staged rows per FFT: c_max, c_min (PAIR)
    // staged peaks per FFT (the static shared memory holds 48 KB)
    constexpr int kPeaks = PAIR ? 736 : 1024;
    // rows padded by one word: lanes on different FFTs fall on different banks
    __shared__ int32_t cell_s[NR][8][kPeaks + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int unit = blockIdx.y;
    const int nd = PAIR ? min(2, J.n_dir - 2 * unit) : 1;  // directions of the unit
    const int d_first = J.dir_begin + (PAIR ? 2 * unit : unit);
    const int64_t *A0 = J.A + (int64_t)d_first * J.n_peaks;
    const int64_t *A1 = nd == 2 ? A0 + J.n_peaks : A0;  // the pair's second direction
    // the transform merges into each direction's profile by atomicMax from 0:
    // the blocks of the unit clear it here, a strided slice each
    for (int di = 0; di < nd; ++di) {
        uint64_t *pr = J.profile + (int64_t)(d_first + di) * J.n_f0;
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < J.n_f0;
             k += (int64_t)gridDim.x * blockDim.x)
            pr[k] = 0;
    }
    {
        // warp w stages FFT w of the block; with J.dense it also flags two
        // consecutive peaks whose cells (in either direction) differ by at most
        // 1 (positions less than one cell apart imply that), which the packed
        // transform's 16-bit counters cannot take
        const int is = blockIdx.x * 8 + warp;
        const bool ls = is < J.n_fft;
        const int64_t os = ls ? J.offsets[is] : 0;
        const int ns = ls ? (int)(J.offsets[is + 1] - os) : 0;
        const bool stage = ns + 2 * kWinPad <= kPeaks;
        bool close = false;
        if (stage || J.dense != nullptr) {
            const int64_t *Aa = A0 + os, *Ab = A1 + os;
            int32_t *c0 = &cell_s[0][warp][kWinPad];
            int32_t *c1 = &cell_s[NR - 1][warp][kWinPad];
            int carry_a = 0, carry_b = 0;
            for (int k0 = 0; k0 < ns; k0 += 128) {
                int ca[4], cb[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int k = k0 + 32 * r + lane;
                    ca[r] = k < ns ? global_cell(Aa, k) : 0;
                    cb[r] = (PAIR && k < ns) ? global_cell(Ab, k) : ca[r];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int k = k0 + 32 * r + lane;
                    if (stage && k < ns) {
                        c0[k] = max(ca[r], cb[r]);
                        if (PAIR) c1[k] = min(ca[r], cb[r]);
                    }
                    int pa = __shfl_up_sync(kFull, ca[r], 1);
                    if (lane == 0) pa = carry_a;
                    if (k > 0 && k < ns && (int64_t)ca[r] - (int64_t)pa <= 1) close = true;
                    carry_a = __shfl_sync(kFull, ca[r], 31);
                    if constexpr (PAIR) {
                        int pb = __shfl_up_sync(kFull, cb[r], 1);
                        if (lane == 0) pb = carry_b;
                        if (k > 0 && k < ns && (int64_t)cb[r] - (int64_t)pb <= 1) close = true;
                        carry_b = __shfl_sync(kFull, cb[r], 31);
                    }
                }
            }
            if (stage && lane < kWinPad) {
                c0[-1 - lane] = INT_MIN;
                c0[ns + lane] = INT_MAX;
                c1[-1 - lane] = INT_MIN;
                c1[ns + lane] = INT_MAX;
            }
            if (J.dense != nullptr && __any_sync(kFull, close) && lane == 0) atomicOr(J.dense, 1);
        }
        if (PAIR && nd == 2 && J.unit_delta != nullptr && lane == 0 && ns > 0) {
            // the pair's largest distance between a peak's two cells: the positions
            // differ by f (r_b - r_a) KT (+ rounding), linear in f, so it is largest
            // at the FFT's first or last peak (ascending frequencies); 2 cells of
            // rounding margin
            const int64_t *Aa = A0 + os, *Ab = A1 + os;
            const int64_t d0 = (int64_t)global_cell(Ab, 0) - global_cell(Aa, 0);
            const int64_t d1 = (int64_t)global_cell(Ab, ns - 1) - global_cell(Aa, ns - 1);
            const int64_t dm = max(d0 < 0 ? -d0 : d0, d1 < 0 ? -d1 : d1) + 2;
            atomicMax(J.unit_delta + unit, (int32_t)min(dm, (int64_t)INT_MAX));
        }
    }
    __syncthreads();
    // this lane's FFT and tiles
    const int f = lane & 7;
    const int tq = 4 * warp + (lane >> 3);
    const int i = blockIdx.x * 8 + f;
    const bool live = i < J.n_fft;
    const int64_t o0 = live ? J.offsets[i] : 0;
    const int n = live ? (int)(J.offsets[i + 1] - o0) : 0;
    const bool staged = n + 2 * kWinPad <= kPeaks;
    const int64_t dv = live ? J.D[i] : 0;
    const int64_t s0 = live ? J.S0[i] : 0;
    const int K = J.k_over, W = J.tile_cells;
    const int64_t nf = J.n_fft;
    const int64_t slab_stride = (int64_t)J.n_tiles * nf;
    uint32_t *out = windows + (int64_t)unit * J.n_slabs * slab_stride;
    const int32_t *cs_lo = &cell_s[0][f][kWinPad];       // lower bounds: c_max
    const int32_t *cs_hi = &cell_s[NR - 1][f][kWinPad];  // upper bounds: c_min
    const int64_t *Aa = A0 + o0, *Ab = A1 + o0;
    // every FFT of the block staged (the usual case): the slab loop reads shared
    // memory only; else the whole block takes the global-memory searches
    const bool all_staged = __syncthreads_and(staged ? 1 : 0) != 0;
    for (int t0 = 0; t0 < J.n_tiles; t0 += kTiles) {
        const int nt = min(kTiles, J.n_tiles - t0);
        // the lane's tiles: lower bound = Lc + b0 - K + 1, upper bound = Hc + b0 + Wt
        int blo[M], bhi[M], qa[M], qb[M];
        bool ok[M];
        uint32_t *dst[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int tt = tq + 32 * m;
            ok[m] = live && tt < nt;
            const int b0 = (t0 + tt) * W;
            blo[m] = b0 - K + 1;
            bhi[m] = b0 + min(W, J.n_f0 - b0);
            qa[m] = 0;
            qb[m] = 0;
            dst[m] = out + (int64_t)(t0 + tt) * nf + i;
        }
        // bounds of slab j0 = 32 s: floor((S0 + j0 D + min(0, (R-1) D)) / 2^32) and
        // ceil((S0 + j0 D + max(0, (R-1) D)) / 2^32) (+ the tile's terms), kept
        // as 64-bit sums that advance by 32 D per full slab
        const int RS = J.row_pairs ? 2 * kRows : kRows;  // rows per slab
        const int64_t span_full = (int64_t)(RS - 1) * dv;
        int64_t u = s0 + (span_full < 0 ? span_full : 0);
        int64_t w = s0 + (span_full > 0 ? span_full : 0);
        // One slab: its bounds, the searches (FIRST: binary; later slabs: steps
        // in the direction of D, UP for D >= 0, both bounds moving monotonically
        // with the slab), the entries.
        auto slab_pass = [&](auto first_tag, auto staged_tag, auto up_tag, const int slab) {
            constexpr bool FIRST = decltype(first_tag)::value;
            constexpr bool STG = decltype(staged_tag)::value;
            constexpr bool UP = decltype(up_tag)::value;
            if (slab == J.n_slabs - 1) {
                // the last slab may hold fewer rows
                const int R = J.n_fdot - slab * RS;
                const int64_t span = (int64_t)(R - 1) * dv;
                const int64_t jd = (int64_t)slab * RS * dv;
                u = s0 + jd + (span < 0 ? span : 0);
                w = s0 + jd + (span > 0 ? span : 0);
            }
            const int ul = (int)(u >> 32);
            const int wh = (int)(w >> 32) + ((uint32_t)w != 0u ? 1 : 0);
            if constexpr (STG) {
                // every lane searches (the sentinels bound the tiles past the last one)
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    if constexpr (FIRST) {
                        qa[m] = lower_bound_cell(cs_lo, n, ul + blo[m]);
                        qb[m] = lower_bound_cell(cs_hi, n, wh + bhi[m]);
                    } else if constexpr (UP) {
                        qa[m] = step_up(cs_lo, qa[m], ul + blo[m]);
                        qb[m] = step_up(cs_hi, qb[m], wh + bhi[m]);
                    } else {
                        qa[m] = step_down(cs_lo, qa[m], ul + blo[m]);
                        qb[m] = step_down(cs_hi, qb[m], wh + bhi[m]);
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    if (!ok[m]) continue;
                    const int xl = ul + blo[m], xh = wh + bhi[m];
                    int qa_m = qa[m], qb_m = qb[m];
                    if constexpr (FIRST) {
                        qa_m = lower_bound_pair_g<false>(Aa, Ab, n, xl);
                        qb_m = lower_bound_pair_g<true>(Aa, Ab, n, xh);
                    } else {
                        while (qa_m < n && pair_cell_g<false>(Aa, Ab, qa_m) < xl) ++qa_m;
                        while (qa_m > 0 && pair_cell_g<false>(Aa, Ab, qa_m - 1) >= xl) --qa_m;
                        while (qb_m < n && pair_cell_g<true>(Aa, Ab, qb_m) < xh) ++qb_m;
                        while (qb_m > 0 && pair_cell_g<true>(Aa, Ab, qb_m - 1) >= xh) --qb_m;
                    }
                    qa[m] = qa_m;
                    qb[m] = qb_m;
                }
            }
#pragma unroll
            for (int m = 0; m < M; ++m) {
                if (ok[m]) {
                    const int lo = qa[m], cnt = max(qa[m], qb[m]) - lo;
                    *dst[m] = (lo < 0xFFFF && cnt < 0xFFFF) ? (uint32_t)lo | ((uint32_t)cnt << 16)
                                                            : kWinLookup;
                }
                dst[m] += slab_stride;
            }
            u += RS * dv;
            w += RS * dv;
        };
        auto run = [&](auto staged_tag, auto up_tag) {
            slab_pass(std::true_type{}, staged_tag, up_tag, 0);
            for (int slab = 1; slab < J.n_slabs; ++slab)
                slab_pass(std::false_type{}, staged_tag, up_tag, slab);
        };
        if (!all_staged)
            run(std::false_type{}, std::true_type{});  // (both directions handled there)
        else if (dv >= 0)
            run(std::true_type{}, std::true_type{});
        else
            run(std::true_type{}, std::false_type{});
    }
}

// Cell of a 32.32 fixed-point position: its high word, read straight from
// the 64-bit register pair.
__device__ __forceinline__ uint32_t cell_of(int64_t X)
{
    uint32_t lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(X));
    return hi;
}

__host__ __device__ constexpr int ctz5(int x)
{
    return (x & 1) ? 0 : (x & 2) ? 1 : (x & 4) ? 2 : (x & 8) ? 3 : 4;
}

// DIFF mode (+1 at the first covered cell of the tile, -1 after the stripe)
// always clamps: the differential form itself cuts stripes at the tile edges.
template <int T>
__device__ __forceinline__ void diff_step(int32_t *H0, int lane, int64_t &X, const int64_t (&e)[5],
                                          int E, int Wt, int K, int32_t w)
{
    constexpr int gt = T ^ (T >> 1);
    const int row = lane ^ gt;
    const int L = (int)(X >> 32);
    const bool in = (unsigned)L < (unsigned)E;
    const int st = in ? max(L - K + 1, 0) : E;
    const int en = (in && L + 1 < Wt) ? L + 1 : E;
    atomicAdd(&H0[st * kRows + row], w);
    atomicAdd(&H0[en * kRows + row], -w);
    if constexpr (T < 31) {
        constexpr int b = ctz5(T + 1);
        if constexpr ((gt >> b) & 1) X -= e[b]; else X += e[b];
    }
}

// Step T of a peak's 32 row updates.  The lane visits row lane ^ g(T),
// g(T) = T ^ (T >> 1) (a Gray code; T, g(T), the bit b that flips next and its
// sign are compile-time constants): for every step the 32 lanes of a warp
// visit 32 different rows, i.e. 32 different banks of the [cell][row]
// counters, and from one step to the next the lane's row changes in bit b
// only, so X moves by e[b] = +-(D << b) (sign + when the lane's bit b is set,
// applied with the compile-time sign of the flip).
//   X      A - shift of the lane's current row - tile origin, 32.32 fixed point
//   rbase  shared address of (cell 0, row `lane`); cell 0 is 128-byte aligned
//   stride bytes per cell (128): a run-time value, or the constant where the
//          caller's kernel walks faster with it
// CLAMP = false: the caller guarantees every cell of the 32 rows lies inside
// the guard cells around the tile, so the atomic needs no bounds clamp.
// CLAMP = true: cells outside [0, E) go to the dump cell E (never read).
// Two peaks of one FFT per lane share the row walk, hence the step table e and
// each step's row offset.  Each update adds w, the FFT's weight (1 for the
// plain map; Eq. ncountadap for the adaptive one).
template <bool CLAMP, bool WEIGHTED, int T>
__device__ __forceinline__ void pair_step(uint32_t rbase, int64_t &X1, int64_t &X2,
                                          const int64_t (&e)[5], uint32_t stride, uint32_t E,
                                          uint32_t w)
{
    constexpr uint32_t gt = (uint32_t)(T ^ (T >> 1));
    const uint32_t rb = rbase ^ (gt << 2);
    uint32_t c1 = cell_of(X1);
    uint32_t c2 = cell_of(X2);
    if (CLAMP) {
        c1 = min(c1, E);
        c2 = min(c2, E);
    }
    const uint32_t a1 = c1 * stride + rb;
    const uint32_t a2 = c2 * stride + rb;
    if constexpr (WEIGHTED) {
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a1), "r"(w) : "memory");
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a2), "r"(w) : "memory");
    } else {
        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(a1) : "memory");
        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(a2) : "memory");
    }
    if constexpr (T < 31) {
        constexpr int b = ctz5(T + 1);
        if constexpr ((gt >> b) & 1) {
            X1 -= e[b];
            X2 -= e[b];
        } else {
            X1 += e[b];
            X2 += e[b];
        }
    }
}

template <bool CLAMP, bool WEIGHTED, int... Ts>
__device__ __forceinline__ void pair_steps(std::integer_sequence<int, Ts...>, uint32_t rbase,
                                           int64_t X1, int64_t X2, const int64_t (&e)[5],
                                           uint32_t stride, uint32_t E, uint32_t w)
{
    (pair_step<CLAMP, WEIGHTED, Ts>(rbase, X1, X2, e, stride, E, w), ...);
}

// x += y and x -= y on 64-bit positions as an explicit 32-bit carry chain
// (low words with carry out, high words with carry in).  The result is the
// same two's-complement sum; the paired walk ran faster with this form than
// with the compiler's own 64-bit add (by 1.8 % on the 900 Hz workload, 0.9 %
// on the 50 Hz one).
__device__ __forceinline__ void add_carry(int64_t &x, int64_t y)
{
    asm("{\n\t.reg .u32 xl, xh, yl, yh;\n\t"
        "mov.b64 {xl, xh}, %0;\n\tmov.b64 {yl, yh}, %1;\n\t"
        "add.cc.u32 xl, xl, yl;\n\taddc.u32 xh, xh, yh;\n\t"
        "mov.b64 %0, {xl, xh};\n\t}"
        : "+l"(x)
        : "l"(y));
}
__device__ __forceinline__ void sub_carry(int64_t &x, int64_t y)
{
    asm("{\n\t.reg .u32 xl, xh, yl, yh;\n\t"
        "mov.b64 {xl, xh}, %0;\n\tmov.b64 {yl, yh}, %1;\n\t"
        "sub.cc.u32 xl, xl, yl;\n\tsubc.u32 xh, xh, yh;\n\t"
        "mov.b64 %0, {xl, xh};\n\t}"
        : "+l"(x)
        : "l"(y));
}

// Step T of the paired walk (two directions of one pair, two 16-bit counters
// per word: the pair's first direction in the low half, its second in the
// high half): X1, X2 are the lane's two peaks in the first direction on row
// lane ^ g(T), Y1, Y2 the same peaks in the second.  A peak's shift tables do
// not depend on the direction (Eq. due), so all four share the row offset
// and the step; the low-half updates add 1, the high-half ones 2^16.  Every
// lane is still on its own bank.
template <bool CLAMP, int T>
__device__ __forceinline__ void quad_step(uint32_t rbase, int64_t &X1, int64_t &X2, int64_t &Y1,
                                          int64_t &Y2, const int64_t (&e)[5], uint32_t stride,
                                          uint32_t E)
{
    constexpr uint32_t gt = (uint32_t)(T ^ (T >> 1));
    const uint32_t rb = rbase ^ (gt << 2);
    uint32_t c1 = cell_of(X1), c2 = cell_of(X2), c3 = cell_of(Y1), c4 = cell_of(Y2);
    if (CLAMP) {
        c1 = min(c1, E);
        c2 = min(c2, E);
        c3 = min(c3, E);
        c4 = min(c4, E);
    }
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(c1 * stride + rb) : "memory");
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(c2 * stride + rb) : "memory");
    asm volatile("red.shared.add.u32 [%0], 65536;" ::"r"(c3 * stride + rb) : "memory");
    asm volatile("red.shared.add.u32 [%0], 65536;" ::"r"(c4 * stride + rb) : "memory");
    if constexpr (T < 31) {
        constexpr int b = ctz5(T + 1);
        if constexpr ((gt >> b) & 1) {
            sub_carry(X1, e[b]);
            sub_carry(X2, e[b]);
            sub_carry(Y1, e[b]);
            sub_carry(Y2, e[b]);
        } else {
            add_carry(X1, e[b]);
            add_carry(X2, e[b]);
            add_carry(Y1, e[b]);
            add_carry(Y2, e[b]);
        }
    }
}

template <bool CLAMP, int... Ts>
__device__ __forceinline__ void quad_steps(std::integer_sequence<int, Ts...>, uint32_t rbase,
                                           int64_t X1, int64_t X2, int64_t Y1, int64_t Y2,
                                           const int64_t (&e)[5], uint32_t stride, uint32_t E)
{
    (quad_step<CLAMP, Ts>(rbase, X1, X2, Y1, Y2, e, stride, E), ...);
}

// The first S Gray-code steps of the paired walk (unclamped), for a compacted
// last round (S < 32): a loop rather than unrolled steps, so that the paired
// kernel's registers stay within a 24-warp block.  Row lane ^ g(t) is reached
// from the start row lane by adding (lane - row) D.
__device__ __forceinline__ void quad_steps_short(int S, uint32_t rbase, uint32_t lane, int64_t X1,
                                                 int64_t X2, int64_t Y1, int64_t Y2, int64_t dv,
                                                 uint32_t stride)
{
#pragma unroll 1
    for (int t = 0; t < S; ++t) {
        const uint32_t gt = (uint32_t)(t ^ (t >> 1));
        const int64_t dl = (int64_t)((int)lane - (int)(lane ^ gt)) * dv;
        const uint32_t rb = rbase ^ (gt << 2);
        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(cell_of(X1 + dl) * stride + rb) : "memory");
        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(cell_of(X2 + dl) * stride + rb) : "memory");
        asm volatile("red.shared.add.u32 [%0], 65536;" ::"r"(cell_of(Y1 + dl) * stride + rb) : "memory");
        asm volatile("red.shared.add.u32 [%0], 65536;" ::"r"(cell_of(Y2 + dl) * stride + rb) : "memory");
    }
}

template <int... Ts>
__device__ __forceinline__ void diff_steps(std::integer_sequence<int, Ts...>, int32_t *H0, int lane,
                                           int64_t X, const int64_t (&e)[5], int E, int Wt, int K,
                                           int32_t w)
{
    (diff_step<Ts>(H0, lane, X, e, E, Wt, K, w), ...);
}

// One block per work item (unit = a direction or a pair of them, tile of W
// frequency cells, slab of spin-down rows; items tile by tile, a tile's slabs
// together); a persistent grid takes the items of all jobs, each block its
// first by block index and then (with a launch counter) whichever is next.
//
// Shared memory holds the tile's counters H[L][row], L = s - (b0 - K + 1) for
// a stripe starting at cell s (so L in [0, W + K - 1) covers every stripe that
// touches the tile), row stride 32 words: row r lives in bank r.
//
// Accumulate: each warp takes 32 FFTs at a time (lane <-> FFT) and reads, per
// FFT, the window of peaks that can reach the tile on some row of the slab
// (precomputed by windows_kernel, else a binary search).  The windowed peaks
// of the 32 FFTs are dealt out to the lanes in rounds of 32 slots (a warp scan
// of the per-FFT slot counts; each lane finds the FFT owning its slot from the
// round's start bits); START mode puts two peaks of one FFT in a slot.  For a
// single direction the next round's positions are loaded while the current
// round is added; every lane adds its peaks' row updates along the Gray-code
// row order (pair_step / quad_step / diff_step), so the 32 atomics of one warp
// instruction always go to 32 different banks.  A short last slab (R <= 16
// rows, unclamped walk) has a pass of its own in which every lane walks only
// the rows of its aligned block of 2^ceil(log2 R) lanes and the copies of a
// row are folded before the emit.
//
// PACK (START mode, plain map, several directions): an item covers two sky
// directions, d_a = 2u and d_b = 2u + 1 of the job, and each counter word holds
// two 16-bit counts of the same (cell, row), d_a's in the low half and d_b's in
// the high half.  The shift tables S0, D do not depend on the direction, so a
// dealt pair of peaks is walked in both directions with one step table (four
// atomics per step, quad_step); the item's windows are the union of the two
// directions' windows, and the guard cells hold in addition the largest cell
// distance between a peak's two positions (the window pre-pass measures it per
// pair; a pair beyond the job's allowance walks each direction on its own,
// clamped).  A
// stripe-start count stays below 2^16 when no FFT has two peaks within one cell
// (each FFT then starts at most one stripe per cell and row) and n_fft < 2^16;
// the window pre-pass flags the first condition per job (`dense`), and a
// flagged job walks each direction of a pair on its own with whole-word counts.
//
// Emit: warps take 16-cell groups along f0 (START, packed counts) or segments
// (DIFF, or counts too large to pack); lane l walks row l (of both directions
// of a pair): START sums a K-cell window of starts, DIFF takes a running sum
// with the other segments' totals as carry-in.  The count goes to the map
// (optional) and the warp's max over rows (smallest row on ties) to the
// direction's profile by a 64-bit atomicMax, which is order-independent.
template <int MODE, int MAXT, bool WEIGHTED, int PACK>
__global__ void __launch_bounds__(MAXT, 1)
transform_kernel(const __grid_constant__ JobTable tbl, int64_t total_items, int32_t hist_words,
                 int32_t guard, uint32_t cell_stride, unsigned int *__restrict__ sched)
{
    // PACK: 0 full-word counters; 1 direction pairs; 2 row pairs (one direction)
    static_assert(!PACK || (MODE == FH_MODE_START && !WEIGHTED), "packed counters: plain START");
    extern __shared__ __align__(16) int32_t smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    // counters: `guard` cells below the tile, the tile's W + K - 1 cells (plus
    // the dump cell), `guard` cells above; cell 0 sits at a 128-byte aligned
    // shared address (the allocation has 128 spare bytes), so a lane's row
    // offset is a single XOR
    const uint32_t sraw = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t hbase = (sraw + 127u) & ~127u;
    int32_t *const Hlo = smem_raw + ((hbase - sraw) >> 2);  // lowest guard cell
    int32_t *const H = Hlo + guard * kRows;                  // cell 0
    const uint32_t rbase = hbase + (uint32_t)guard * (kRows * 4u) + 4u * (uint32_t)lane;
    int32_t *const tab = Hlo + hist_words + warp * 32;  // per-warp owner table
    int32_t *const next_chunk = Hlo + hist_words + nwarps * 32 +
                                (MODE == FH_MODE_DIFF ? nwarps * 32 : 0);
    int32_t *const next_item = next_chunk + 1;  // the block's next item (sched)
    const unsigned lanemask_le = 0xffffffffu >> (31 - lane);
    const unsigned lanemask_lt = (1u << lane) - 1u;
    // Per job: the unclamped walk runs when the job's largest drift over a slab
    // stays inside the guards and no input check has failed.  Its windows then
    // hold sorted positions, so every row of every windowed peak lands in the
    // guard cells or the tile; after a failed check (unsorted or non-finite
    // input) the windows can hold anything and the clamped walk, which keeps
    // every update in [0, E], runs instead.  (PACK) direction pairs need the
    // job's allowance for the distance between a peak's two positions in the
    // guards too, and take the packed counters while the window pre-pass found
    // no FFT with two peaks in one cell.
    unsigned job_fast = 0;    // bit j: job j may take the unclamped walk
    unsigned job_packed = 0;  // bit j: job j's stripe-start counts fit 16 bits
    for (int j = 0; j < tbl.n_jobs; ++j) {
        const TransformJob &Jt = tbl.job[j];
        if (Jt.dmax != nullptr && Jt.err != nullptr && *Jt.err == 0 &&
            guard_for(*Jt.dmax, PACK == 2 && Jt.row_pairs ? 2 * kRows - 1 : kRows - 1) +
                    (PACK == 1 && Jt.dir_pairs ? Jt.delta_alloc : 0) <=
                guard)
            job_fast |= 1u << j;
        if (PACK && Jt.dense != nullptr && *Jt.dense == 0) job_packed |= 1u << j;
    }

    // Items: the first one per block by block index, then (sched) whichever
    // comes next from the launch's counter, so that blocks whose items were
    // cheaper take more of them; without a counter, every gridDim.x-th.  Thread
    // 0 asks the counter when its warp has no accumulation left to do (the
    // other warps may still be busy), and the answer is read after the emit.
    auto next_of = [&](int64_t it) -> int64_t {
        if (sched == nullptr) return it + gridDim.x;
        __syncthreads();
        return (int64_t)gridDim.x + *next_item;
    };
    for (int64_t item = blockIdx.x; item < total_items; item = next_of(item)) {
        int jb = 0;
        while (jb + 1 < tbl.n_jobs && item >= tbl.job[jb + 1].item_begin) ++jb;
        const TransformJob *J = &tbl.job[jb];
        const int64_t rem = item - J->item_begin;
        const int per_unit = J->n_slabs * J->n_tiles;
        const int unit = (int)(rem / per_unit);  // a direction, or (PACK) a pair of them
        const int r2 = (int)(rem - (int64_t)unit * per_unit);
        // items go tile by tile, a tile's slabs together: the blocks at work at one
        // time read the peaks of a few tiles' windows, which stay in L2 for all of
        // those tiles' slabs
        const int tile = r2 / J->n_slabs;
        const int slab = r2 - tile * J->n_slabs;
        const int K = J->k_over, W = J->tile_cells, n_f0 = J->n_f0, n_fdot = J->n_fdot;
        const int n_fft = J->n_fft;
        // (PACK) row pairs: one direction in slabs of 64 rows, rows j0 .. j0 + 31 in
        // the low halves and j0 + 32 .. j0 + 63 in the high halves of the counters
        const bool rowp = PACK == 2 && J->row_pairs;
        const int srows = rowp ? 2 * kRows : kRows;
        const int js = slab * srows;
        const int R_slab = min(srows, n_fdot - js);
        const int b0 = tile * W;
        const int Wt = min(W, n_f0 - b0);
        const int E = Wt + K - 1;
        const bool paired = PACK == 1 && J->dir_pairs;
        const int d_rel = paired ? 2 * unit : unit;  // d_a, relative to the job's first
        const bool has_b = paired && d_rel + 1 < J->n_dir;
        const int d_abs = J->dir_begin + d_rel;
        const int64_t *__restrict__ Ad = J->A + (int64_t)d_abs * J->n_peaks;
        const int64_t *__restrict__ Ad_b = has_b ? Ad + J->n_peaks : Ad;
        const int64_t *__restrict__ offs = J->offsets;
        const int64_t *__restrict__ S0 = J->S0;
        const int64_t *__restrict__ Dt = J->D;
        const uint32_t *__restrict__ wrow =
            J->windows ? J->windows + (((int64_t)unit * J->n_slabs + slab) * J->n_tiles + tile) *
                                          n_fft
                       : nullptr;
        const int32_t *__restrict__ wts =
            J->weights ? J->weights + (int64_t)d_abs * n_fft : nullptr;
        // a pair whose positions lie further apart than the job allows walks clamped
        const bool fast = MODE == FH_MODE_START && ((job_fast >> jb) & 1u) &&
                          (!has_b || J->unit_delta == nullptr ||
                           J->unit_delta[unit] <= J->delta_alloc);
        const int64_t base_shift = (int64_t)(b0 - K + 1) * 4294967296LL;
        const int64_t e_fixed = (int64_t)E * 4294967296LL;
        const int nchunks = (n_fft + 31) >> 5;

        // One pass over the tile: zero the counters, accumulate rows j0 .. j0 +
        // R - 1 of direction d_a + dsel (QUAD: of both directions of the pair, d_a
        // in the low halves, d_b in the high halves), emit.  The windows of a pair
        // (table or lookup) are the union of its two directions' windows, a
        // superset of either's.
        auto pass = [&](const int j0, const int R, auto quad_tag, const int dsel, auto short_tag) {
            // quad_tag: 0 one direction, 1 a pair of directions, 2 (ROWQ) the two
            // 32-row halves of a 64-row slab of one direction
            constexpr bool QUAD = decltype(quad_tag)::value != 0;
            constexpr bool ROWQ = decltype(quad_tag)::value == 2;
            constexpr bool SHORT = decltype(short_tag)::value;
            const bool row_ok = lane < R;
            const int64_t *__restrict__ Ap = dsel ? Ad_b : Ad;
            // SHORT: a pass of R <= 16 rows (a short last slab) on the unclamped
            // walk: every lane takes its own slot through the Srows =
            // 2^ceil(log2 R) rows of its aligned block of Srows lanes, counting
            // virtual row lane mod Srows in the lane's own bank (row lane ^ g(t));
            // the 32 / Srows copies of a row are summed before the emit.
            const int Srows = SHORT ? (R <= 1 ? 1 : R <= 2 ? 2 : R <= 4 ? 4 : R <= 8 ? 8 : 16) : 32;

            // zero the counters (with the guard cells in the fast path); reset the chunk counter
            {
                int4 *h4 = reinterpret_cast<int4 *>(fast ? Hlo : H);
                const int n4 = ((fast ? E + 2 * guard : E) * kRows) >> 2;
                for (int w = threadIdx.x; w < n4; w += blockDim.x) h4[w] = make_int4(0, 0, 0, 0);
                if (threadIdx.x == 0) *next_chunk = nwarps;
            }
            __syncthreads();

            // accumulate
            // chunks of 32 FFTs (lane <-> FFT): the first round one per warp, then
            // whoever is free
            for (int c = warp; c < nchunks;) {
                int64_t cb, dv, q0;
                int n;
                // the FFT's weight on this direction (adaptive map), 1 for the plain map
                int32_t wt = 1;
                if constexpr (WEIGHTED)
                    if (wts != nullptr && (c << 5) + lane < n_fft) wt = __ldg(wts + (c << 5) + lane);
                const int i_l = (c << 5) + lane;
                const uint32_t wv = (wrow != nullptr && i_l < n_fft) ? wrow[i_l] : kWinLookup;
                if (wrow != nullptr && wv != kWinLookup) {
                    // precomputed window: one coalesced load (start relative to the FFT's
                    // first peak, count); trusted on the unclamped walk (the input checks
                    // passed and the table was built from the sanitised CSR), else clamped
                    // into the FFT's CSR range
                    const int i = i_l;
                    const int64_t o0 = __ldg(offs + i);
                    dv = __ldg(Dt + i);
                    cb = __ldg(S0 + i) + (int64_t)j0 * dv + base_shift;
                    if (fast) {
                        q0 = o0 + (wv & 0xFFFFu);
                        n = (int)(wv >> 16);
                    } else {
                        const int64_t o1 = __ldg(offs + i + 1);
                        const int64_t a = min(o0 + (int64_t)(wv & 0xFFFFu), o1);
                        q0 = a;
                        n = (int)min((int64_t)(wv >> 16), o1 - a);
                    }
                } else if (wrow != nullptr && i_l >= n_fft) {
                    cb = 0;
                    dv = 0;
                    q0 = 0;
                    n = 0;
                } else {
                    int64_t cbs;
                    lookup_window(Ap, offs, S0, Dt, n_fft, (c << 5) + lane, js, R_slab, base_shift,
                                  e_fixed, cbs, dv, q0, n);
                    if (QUAD && !ROWQ) {
                        // the union (as one index range) with the other direction's window
                        int64_t cb2, dv2, q0b;
                        int nb;
                        lookup_window(Ad_b, offs, S0, Dt, n_fft, (c << 5) + lane, js, R_slab,
                                      base_shift, e_fixed, cb2, dv2, q0b, nb);
                        if (nb > 0) {
                            const int64_t hi = n > 0 ? max(q0 + n, q0b + nb) : q0b + nb;
                            q0 = n > 0 ? min(q0, q0b) : q0b;
                            n = (int)(hi - q0);
                        }
                    }
                    cb = cbs + (int64_t)(j0 - js) * dv;
                }
                // START mode deals the peaks out in pairs of one FFT (one slot = two
                // consecutive peaks of the window; an odd count leaves the last slot's
                // second peak empty), DIFF mode one peak per slot
                constexpr bool kPairs = MODE == FH_MODE_START;
                const int m = kPairs ? (n + 1) >> 1 : n;
                // exclusive scan of the per-FFT slot counts, owner table of non-empty FFTs
                int P = m;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, P, o);
                    if (lane >= o) P += y;
                }
                const int T = __shfl_sync(kFull, P, 31);
                P -= m;
                const bool has = m > 0;
                // the slot's first peak is kq + (pairs ? 2 : 1) g; the window ends at qe
                const int kq = (int)q0 - (kPairs ? 2 * P : P);
                const int qe = (int)q0 + n;
                const unsigned nonempty = __ballot_sync(kFull, has);
                if (has) tab[__popc(nonempty & lanemask_lt)] = lane;
                __syncwarp();

                // Slot g = base + lane of a round belongs to the non-empty FFT whose
                // range [P, P + m) holds it.  `before` counts the non-empty FFTs
                // starting below the base; bases are fetched in increasing order, 32
                // apart.  The slot's peaks are positions q0 + k, k = (pairs) 2 (g - P)
                // and 2 (g - P) + 1 (if below q0 + n), or (singles) g - P: the owner
                // publishes kq = q0 - 2 P (q0 - P) and its window end qe.
                int before = 0;
                // QUAD: b1, b2 are the same peaks' positions in direction d_b
                auto fetch = [&](int base, int64_t &a1, int64_t &a2, int64_t &b1, int64_t &b2,
                                 bool &two, int &owner) {
                    const unsigned rel = (unsigned)(P - base);
                    const unsigned bits =
                        __reduce_or_sync(kFull, (has && rel < 32u) ? (1u << rel) : 0u);
                    const int oc = before + __popc(bits & lanemask_le) - 1;
                    before += __popc(bits);
                    owner = tab[oc < 0 ? 0 : oc];
                    const int okq = __shfl_sync(kFull, kq, owner);
                    const int g = base + lane;
                    const bool live = g < T;
                    if (kPairs) {
                        const int oqe = __shfl_sync(kFull, qe, owner);
                        const int k = okq + 2 * g;
                        two = live && k + 1 < oqe;
                        a1 = live ? __ldg(Ap + k) : 0;
                        a2 = two ? __ldg(Ap + k + 1) : 0;
                        if constexpr (QUAD) {
                            // (row pairs: the same peaks 32 rows further, from a1, a2)
                            b1 = (live && !ROWQ) ? __ldg(Ad_b + k) : 0;
                            b2 = (two && !ROWQ) ? __ldg(Ad_b + k + 1) : 0;
                        }
                    } else {
                        two = false;
                        a1 = live ? __ldg(Ap + (okq + g)) : 0;
                        a2 = 0;
                    }
                };
                // X of the lane's row for the slot's peaks and their step table.  An
                // empty slot (g >= T) is parked in guard cell -1 with zero steps.  An
                // empty second peak walks with the first one's steps from a start
                // that keeps all the pass's rows in guard cells -guard .. -1 on the
                // unclamped walk (|31 D| is below guard - 1 cells there), and far below
                // cell 0 on the clamped walk (which sends it to the dump cell).  Never
                // read.  On the unclamped walk every windowed peak's rows stay inside
                // the guard cells: the window holds the peaks with A - cb in
                // [min(0, (R_slab-1) D), max(0, (R_slab-1) D) + E 2^32) (to one cell),
                // and |31 D| stays below guard - 2 cells; a pair's union window holds
                // peaks whose position in the other direction is that close, so each
                // position lies within the pair's distance of it, which the guard also
                // holds.  QUAD: Y1, Y2 are the same peaks in direction d_b.
                auto setup = [&](int g, int vlane, int64_t a1, int64_t a2, int64_t b1, int64_t b2,
                                 bool two, int owner, int64_t &X1, int64_t &X2, int64_t &Y1,
                                 int64_t &Y2, int64_t (&e)[5], int32_t &ow) {
                    if constexpr (WEIGHTED)
                        ow = __shfl_sync(kFull, wt, owner);
                    else
                        ow = 1;
                    const int64_t ocb = __shfl_sync(kFull, cb, owner);
                    const int64_t odv0 = __shfl_sync(kFull, dv, owner);
                    const bool live = g < T;
                    const int64_t odv = live ? odv0 : 0;
                    // e[b] = +-(D << b), + when bit b of the lane is set
                    const int64_t ndv = -odv;
#pragma unroll
                    for (int b = 0; b < 5; ++b)
                        e[b] = (((lane >> b) & 1) ? odv : ndv) * (int64_t)(1 << b);
                    // the start row: the lane's own, or its virtual row on a short pass
                    const int64_t lane_dv = (int64_t)vlane * odv;
                    X1 = live ? a1 - ocb - lane_dv : -(int64_t(1) << 32);
                    // (row pairs: row r + 32 of the same peak is 32 D further down)
                    const int64_t y_off = ROWQ ? odv * kRows : 0;
                    if constexpr (QUAD)
                        Y1 = live ? (ROWQ ? a1 : b1) - ocb - lane_dv - y_off : -(int64_t(1) << 32);
                    if (kPairs) {
                        const int64_t park =
                            fast ? (odv > 0 ? -(int64_t(1) << 32) : -((int64_t)guard << 32)) -
                                       lane_dv
                                 : -(int64_t(1) << 62);
                        X2 = two ? a2 - ocb - lane_dv : park;
                        if constexpr (QUAD)
                            Y2 = two ? (ROWQ ? a2 : b2) - ocb - lane_dv - y_off : park;
                    }
                };
                // the next round's peaks are loaded a round ahead, except on the paired
                // walk, whose registers hold four positions per slot already
                constexpr bool kAhead = !QUAD;
                int64_t a1_nx = 0, a2_nx = 0, b1_nx = 0, b2_nx = 0;
                bool two_nx = false;
                int own_nx = 0;
                if (kAhead && T > 0) fetch(0, a1_nx, a2_nx, b1_nx, b2_nx, two_nx, own_nx);
                for (int base = 0; base < T; base += 32) {
                    int64_t a1 = a1_nx, a2 = a2_nx, b1 = b1_nx, b2 = b2_nx;
                    bool two = two_nx;
                    int owner = own_nx;
                    if (!kAhead) fetch(base, a1, a2, b1, b2, two, owner);
                    else if (base + 32 < T)
                        fetch(base + 32, a1_nx, a2_nx, b1_nx, b2_nx, two_nx, own_nx);
                    // A last round of L <= 16 slots (unclamped START walk): S = the
                    // power of two >= L; slot q = lane mod S is walked by the 32 / S
                    // lanes lane = q + S p, lane p taking rows S p .. S p + S - 1 in
                    // S Gray-code steps (row = lane ^ g(t), t < S).  Every (slot, row)
                    // is added once, the 32 lanes stay on 32 banks, and the start
                    // X = A - cb - lane D and the step table are those of a full round.
                    // (A short pass walks Srows steps with one slot per lane instead.)
                    int S = Srows;
                    if (!SHORT && MODE == FH_MODE_START && fast && T - base <= 16) {
                        const int L = T - base;
                        S = L <= 1 ? 1 : (L <= 2 ? 2 : (L <= 4 ? 4 : (L <= 8 ? 8 : 16)));
                        const int src = lane & (S - 1);
                        a1 = __shfl_sync(kFull, a1, src);
                        a2 = __shfl_sync(kFull, a2, src);
                        if constexpr (QUAD) {
                            b1 = __shfl_sync(kFull, b1, src);
                            b2 = __shfl_sync(kFull, b2, src);
                        }
                        two = __shfl_sync(kFull, (int)two, src) != 0;
                        owner = __shfl_sync(kFull, owner, src);
                    }
                    int64_t X1, X2 = 0, Y1 = 0, Y2 = 0, e[5];
                    int32_t ow;
                    setup(SHORT ? base + lane : base + (lane & (S - 1)),
                          SHORT ? (lane & (Srows - 1)) : lane, a1, a2, b1, b2, two, owner, X1, X2,
                          Y1, Y2, e, ow);
                    if (MODE == FH_MODE_START) {
                        using std::make_integer_sequence;
                        // the cell stride as a compile-time constant in the
                        // direction-pair kernel (its walk ran 0.9 % faster so; the
                        // row-pair walk 3 % slower, which keeps the run-time value)
                        const uint32_t st = PACK == 1 ? kRows * 4u : cell_stride;
                        const uint32_t ee = (uint32_t)E, ww = (uint32_t)ow;
                        if constexpr (QUAD) {
                            // the same peaks in direction d_b, in the high halves
                            // (the paired walk runs unclamped only)
                            if (S == 32)
                                quad_steps<false>(make_integer_sequence<int, 32>{}, rbase, X1, X2,
                                                  Y1, Y2, e, st, ee);
                            else  // e[0] = +-D, + on odd lanes
                                quad_steps_short(S, rbase, (uint32_t)lane, X1, X2, Y1, Y2,
                                                 (lane & 1) ? e[0] : -e[0], st);
                        } else if (fast) {
                            switch (S) {
                            case 1:
                                pair_steps<false, WEIGHTED>(make_integer_sequence<int, 1>{}, rbase, X1, X2, e, st, ee, ww);
                                break;
                            case 2:
                                pair_steps<false, WEIGHTED>(make_integer_sequence<int, 2>{}, rbase, X1, X2, e, st, ee, ww);
                                break;
                            case 4:
                                pair_steps<false, WEIGHTED>(make_integer_sequence<int, 4>{}, rbase, X1, X2, e, st, ee, ww);
                                break;
                            case 8:
                                pair_steps<false, WEIGHTED>(make_integer_sequence<int, 8>{}, rbase, X1, X2, e, st, ee, ww);
                                break;
                            case 16:
                                pair_steps<false, WEIGHTED>(make_integer_sequence<int, 16>{}, rbase, X1, X2, e, st, ee, ww);
                                break;
                            default:
                                pair_steps<false, WEIGHTED>(make_integer_sequence<int, 32>{}, rbase, X1, X2, e, st, ee, ww);
                            }
                        } else
                            pair_steps<true, WEIGHTED>(make_integer_sequence<int, 32>{}, rbase, X1,
                                                       X2, e, st, ee, ww);
                    } else if (base + lane < T) {
                        diff_steps(std::make_integer_sequence<int, 32>{}, H, lane, X1, e, E, Wt, K,
                                   ow);
                    }
                }
                __syncwarp();
                int nc = 0;
                if (lane == 0) nc = atomicAdd(next_chunk, 1);
                c = __shfl_sync(kFull, nc, 0);
            }
            if (sched != nullptr && dsel == 0 && threadIdx.x == 0)
                *next_item = (int32_t)atomicAdd(sched, 1u);
            __syncthreads();
            if constexpr (SHORT) {
                // row r's count is the sum of its copies in banks r + Srows k (a
                // butterfly over the lane bits >= log2 Srows); cells 0 .. E (the
                // dump cell too, which the emit may read).  Packed words add half by
                // half: each half's sum is the count the direction would have in
                // one word.
                for (int cell = warp; cell <= E; cell += nwarps) {
                    int32_t v = H[cell * kRows + lane];
                    for (int o = 16; o >= Srows; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                    H[cell * kRows + lane] = v;
                }
                __syncthreads();
            }

            // emit counts, map and profile
            unsigned long long *prof = reinterpret_cast<unsigned long long *>(J->profile) +
                                       (int64_t)(d_abs + dsel) * n_f0 + b0;
            if constexpr (QUAD) {
                // Packed words: direction d_a's count of (cell, row lane) in the low
                // half, d_b's in the high half.  Per cell the lane forms both counts
                // (K-cell windows of starts) and one signed reduction per direction
                // gives the warp's (max count, smallest row), keyed 32 count + (31 -
                // lane); rows beyond the slab start their windows at -2^26 and never
                // win (counts stay below 2^25 on this path).
                // Row pairs: the high halves are rows j0 + 32 + lane of the same
                // direction, merged into its profile with the low halves' keys.
                unsigned long long *prof_b = ROWQ ? prof : prof + n_f0;
                const bool ok_a = lane < min(R, kRows);
                const bool ok_b = ROWQ ? lane < R - kRows : ok_a;
                int32_t *map_a = nullptr, *map_b = nullptr;
                if (J->maps != nullptr) {
                    int32_t *const m0 = J->maps + ((int64_t)d_rel * n_fdot + j0 + lane) * n_f0 + b0;
                    if (ok_a) map_a = m0;
                    if (ok_b) map_b = m0 + (ROWQ ? (int64_t)kRows * n_f0 : (int64_t)n_fdot * n_f0);
                }
                const int seg = (((Wt + nwarps - 1) / nwarps) + 15) & ~15;
                const int c0 = min(Wt, warp * seg);
                const int c1 = min(Wt, c0 + seg);
                const int c31 = 31 - lane;
                int wa = ok_a ? 0 : -(1 << 26);
                int wb = ok_b ? 0 : -(1 << 26);
                if (c0 < c1)
                    for (int L = c0; L < c0 + K; ++L) {
                        const uint32_t h = (uint32_t)H[L * kRows + lane];
                        wa += (int)(h & 0xFFFFu);
                        wb += (int)(h >> 16);
                    }
                const uint32_t key_lo = 0xFFFFFFFFu - (uint32_t)j0 - 31u;
                const uint32_t key_lo_b = ROWQ ? key_lo - (uint32_t)kRows : key_lo;
                auto key_of = [&](int v) {
                    return ((unsigned long long)(uint32_t)(v >> 5) << 32) |
                           (unsigned long long)(key_lo + (uint32_t)(v & 31));
                };
                auto key_of_b = [&](int v) {
                    return ((unsigned long long)(uint32_t)(v >> 5) << 32) |
                           (unsigned long long)(key_lo_b + (uint32_t)(v & 31));
                };
                // 16-byte stores only where both rows exist and are 16-byte aligned
                // (d_b's map starts n_fdot n_f0 words after d_a's)
                const bool vec_map = map_a != nullptr && map_b != nullptr &&
                                     (((uintptr_t)map_a & 15u) == 0) &&
                                     (((uintptr_t)map_b & 15u) == 0);
                auto run = [&](auto map_tag) {
                    constexpr bool kMap = decltype(map_tag)::value;
                    int c = c0;
                    for (; c + 16 <= c1; c += 16) {
                        const int32_t *h0 = H + c * kRows + lane;
                        const int32_t *h1 = h0 + K * kRows;
                        int myva = 0, myvb = 0;
                        int ca[kMap ? 16 : 1], cbn[kMap ? 16 : 1];
#pragma unroll
                        for (int m = 0; m < 16; ++m) {
                            const int na = wa, nb = wb;
                            const uint32_t x = (uint32_t)h1[m * kRows], y = (uint32_t)h0[m * kRows];
                            wa += (int)(x & 0xFFFFu) - (int)(y & 0xFFFFu);
                            wb += (int)(x >> 16) - (int)(y >> 16);
                            if constexpr (kMap) {
                                ca[m] = na;
                                cbn[m] = nb;
                            }
                            const int va = __reduce_max_sync(kFull, na * 32 + c31);
                            const int vb = __reduce_max_sync(kFull, nb * 32 + c31);
                            if (lane == m) {
                                myva = va;
                                myvb = vb;
                            }
                        }
                        if constexpr (kMap) {
                            if (vec_map) {
                                int4 *da = reinterpret_cast<int4 *>(map_a + c);
                                int4 *db = reinterpret_cast<int4 *>(map_b + c);
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    da[q] = make_int4(ca[4 * q], ca[4 * q + 1], ca[4 * q + 2], ca[4 * q + 3]);
                                    db[q] = make_int4(cbn[4 * q], cbn[4 * q + 1], cbn[4 * q + 2], cbn[4 * q + 3]);
                                }
                            } else {
#pragma unroll
                                for (int m = 0; m < 16; ++m) {
                                    if (map_a) map_a[c + m] = ca[m];
                                    if (map_b) map_b[c + m] = cbn[m];
                                }
                            }
                        }
                        if (lane < 16) {
                            if constexpr (ROWQ) {
                                const unsigned long long ka = key_of(myva), kb = key_of_b(myvb);
                                atomicMax(prof + c + lane, ka > kb ? ka : kb);
                            } else {
                                atomicMax(prof + c + lane, key_of(myva));
                                atomicMax(prof_b + c + lane, key_of(myvb));
                            }
                        }
                    }
                    for (; c < c1; ++c) {
                        const int na = wa, nb = wb;
                        // the segment's last step may read cell E (the dump cell); that value is unused
                        const uint32_t x = (uint32_t)H[(c + K) * kRows + lane];
                        const uint32_t y = (uint32_t)H[c * kRows + lane];
                        wa += (int)(x & 0xFFFFu) - (int)(y & 0xFFFFu);
                        wb += (int)(x >> 16) - (int)(y >> 16);
                        if (kMap && map_a) map_a[c] = na;
                        if (kMap && map_b) map_b[c] = nb;
                        const int va = __reduce_max_sync(kFull, na * 32 + c31);
                        const int vb = __reduce_max_sync(kFull, nb * 32 + c31);
                        if (lane == 0) {
                            if constexpr (ROWQ) {
                                const unsigned long long ka = key_of(va), kb = key_of_b(vb);
                                atomicMax(prof + c, ka > kb ? ka : kb);
                            } else {
                                atomicMax(prof + c, key_of(va));
                                atomicMax(prof_b + c, key_of(vb));
                            }
                        }
                    }
                };
                if (J->maps != nullptr)
                    run(std::true_type{});
                else
                    run(std::false_type{});
            } else {
                int32_t *maprow = nullptr;
                if (J->maps != nullptr && row_ok)
                    maprow = J->maps + ((int64_t)(d_rel + dsel) * n_fdot + j0 + lane) * n_f0 + b0;
                // Per cell the profile takes the warp's max over its rows, smallest row
                // on ties.  Counts below 2^26 fit one packed signed reduction
                // 32 count + (31 - lane); rows beyond the pass start their window at
                // -2^26, so they stay negative and never win.
                const bool packed = J->count_bound < (int64_t(1) << 26);
                const uint32_t key_lo = 0xFFFFFFFFu - (uint32_t)j0 - 31u;
                auto key_of = [&](int v) {
                    return ((unsigned long long)(uint32_t)(v >> 5) << 32) |
                           (unsigned long long)(key_lo + (uint32_t)(v & 31));
                };
                if (MODE == FH_MODE_START && packed) {
                    // a K-cell window slides along the warp's segment (count of cell c =
                    // sum of the starts in cells c .. c + K - 1), 16 cells per group:
                    // lane m keeps cell m's reduction and the group's 16 profile atomics
                    // go out together
                    const int seg = (((Wt + nwarps - 1) / nwarps) + 15) & ~15;
                    const int c0 = min(Wt, warp * seg);
                    const int c1 = min(Wt, c0 + seg);
                    const int c31 = 31 - lane;
                    int win = row_ok ? 0 : -(1 << 26);
                    if (c0 < c1)
                        for (int L = c0; L < c0 + K; ++L) win += H[L * kRows + lane];
                    // a lane's map row is written 16 cells (64 bytes) at a time, as four
                    // 16-byte stores where the row is 16-byte aligned (the group's cells
                    // start at a multiple of 16 of the tile), else one cell at a time
                    const bool vec_map = maprow != nullptr && (((uintptr_t)maprow & 15u) == 0);
                    auto run = [&](auto map_tag) {
                        constexpr bool kMap = decltype(map_tag)::value;
                        int c = c0;
                        for (; c + 16 <= c1; c += 16) {
                            const int32_t *h0 = H + c * kRows + lane;
                            const int32_t *h1 = h0 + K * kRows;
                            int myv = 0;
                            int cnts[kMap ? 16 : 1];
#pragma unroll
                            for (int m = 0; m < 16; ++m) {
                                const int cnt = win;
                                win += h1[m * kRows] - h0[m * kRows];
                                if constexpr (kMap) cnts[m] = cnt;
                                const int v = __reduce_max_sync(kFull, cnt * 32 + c31);
                                if (lane == m) myv = v;
                            }
                            if constexpr (kMap) {
                                if (vec_map) {
                                    int4 *d4 = reinterpret_cast<int4 *>(maprow + c);
#pragma unroll
                                    for (int q = 0; q < 4; ++q)
                                        d4[q] = make_int4(cnts[4 * q], cnts[4 * q + 1],
                                                          cnts[4 * q + 2], cnts[4 * q + 3]);
                                } else if (row_ok) {
#pragma unroll
                                    for (int m = 0; m < 16; ++m) maprow[c + m] = cnts[m];
                                }
                            }
                            if (lane < 16) atomicMax(prof + c + lane, key_of(myv));
                        }
                        for (; c < c1; ++c) {
                            const int cnt = win;
                            // the segment's last step may read cell E (the dump cell); that value is unused
                            win += H[(c + K) * kRows + lane] - H[c * kRows + lane];
                            if (kMap && row_ok) maprow[c] = cnt;
                            const int v = __reduce_max_sync(kFull, cnt * 32 + c31);
                            if (lane == 0) atomicMax(prof + c, key_of(v));
                        }
                    };
                    if (J->maps != nullptr)
                        run(std::true_type{});
                    else
                        run(std::false_type{});
                } else {
                    // generic path (DIFF mode, or counts too large to pack): one cell at a
                    // time, lane 0 takes the profile atomic
                    const int seg = (Wt + nwarps - 1) / nwarps;
                    const int c0 = min(Wt, warp * seg);
                    const int c1 = min(Wt, c0 + seg);
                    auto emit = [&](int c, int count) {
                        if (maprow) maprow[c] = count;
                        const int m = __reduce_max_sync(kFull, row_ok ? count : INT_MIN);
                        const unsigned rm =
                            __reduce_min_sync(kFull, (row_ok && count == m) ? (unsigned)lane : 32u);
                        const unsigned long long key =
                            ((unsigned long long)(unsigned)m << 32) |
                            (0xFFFFFFFFull - (unsigned long long)(unsigned)(j0 + rm));
                        if (lane == 0) atomicMax(prof + c, key);
                    };
                    if (MODE == FH_MODE_START) {
                        int win = 0;
                        if (c0 < c1)
                            for (int L = c0; L < c0 + K; ++L) win += H[L * kRows + lane];
                        for (int c = c0; c < c1; ++c) {
                            emit(c, win);
                            win += H[(c + K) * kRows + lane] - H[c * kRows + lane];
                        }
                    } else {
                        int32_t *segtot = Hlo + hist_words + nwarps * 32;
                        int tot = 0;
                        for (int c = c0; c < c1; ++c) tot += H[c * kRows + lane];
                        segtot[warp * 32 + lane] = tot;
                        __syncthreads();
                        int acc = 0;
                        for (int w = 0; w < warp; ++w) acc += segtot[w * 32 + lane];
                        for (int c = c0; c < c1; ++c) {
                            acc += H[c * kRows + lane];
                            emit(c, acc);
                        }
                    }
                }
            }
            __syncthreads();
        };

        const std::false_type nos{};
        if constexpr (PACK == 2) {
            if (rowp) {
                // a 64-row slab: both halves in one walk where the packed counters
                // apply, else its two 32-row halves one after the other
                if (R_slab > kRows && fast && ((job_packed >> jb) & 1u)) {
                    pass(js, R_slab, std::integral_constant<int, 2>{}, 0, nos);
                } else {
                    const int R0 = min(kRows, R_slab), R1 = R_slab - R0;
                    if (MODE == FH_MODE_START && fast && R0 <= 16)
                        pass(js, R0, std::false_type{}, 0, std::true_type{});
                    else
                        pass(js, R0, std::false_type{}, 0, nos);
                    if (R1 > 0) {
                        if (MODE == FH_MODE_START && fast && R1 <= 16)
                            pass(js + kRows, R1, std::false_type{}, 0, std::true_type{});
                        else
                            pass(js + kRows, R1, std::false_type{}, 0, nos);
                    }
                }
            } else {
                pass(js, R_slab, std::false_type{}, 0, nos);
            }
        } else if constexpr (PACK == 1) {
            if (has_b && fast && ((job_packed >> jb) & 1u)) {
                if (R_slab <= 16)
                    pass(js, R_slab, std::integral_constant<int, 1>{}, 0, std::true_type{});
                else
                    pass(js, R_slab, std::integral_constant<int, 1>{}, 0, nos);
            } else {
                // a single direction, a pair whose counts need whole words, or one
                // that takes the clamped walk: each direction on its own
                pass(js, R_slab, std::false_type{}, 0, nos);
                if (has_b) pass(js, R_slab, std::false_type{}, 1, nos);
            }
        } else if (MODE == FH_MODE_START && fast && R_slab <= 16) {
            pass(js, R_slab, std::false_type{}, 0, std::true_type{});
        } else {
            pass(js, R_slab, std::false_type{}, 0, nos);
        }
    }
    // the last block to finish returns the counter to zero for the next launch
    // on this stream (every block's last fetch precedes its count here)
    if (sched != nullptr && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(sched + 1, 1u) == gridDim.x - 1) {
            atomicExch(sched, 0u);
            atomicExch(sched + 1, 0u);
        }
    }
}

// ---------------------------------------------------------------- a6
// grid (n_sb, n_dir), 1024 threads: greedy picks of one sub-band of one direction.
// Order of the picks: profile key descending (count, then smaller row), then
// smaller cell.  A sub-band of up to kSelPer x 1024 cells is held in registers
// (kSelPer cells per thread); each pick zeroes the keys within `excl` cells of
// it, so later picks skip them.  Wider sub-bands rescan the profile per pick.
constexpr int kSelThreads = 1024;
constexpr int kSelPer = 8;

// best (key, cell) of the warp: max key, then min cell.  Keys are nonzero
// except for excluded / empty cells.
__device__ __forceinline__ void warp_best(unsigned long long &k, int &c)
{
    const unsigned h = (unsigned)(k >> 32), l = (unsigned)k;
    const unsigned mh = __reduce_max_sync(kFull, h);
    const unsigned ml = __reduce_max_sync(kFull, h == mh ? l : 0u);
    const unsigned mc = __reduce_min_sync(kFull, (h == mh && l == ml) ? (unsigned)c : 0x7FFFFFFFu);
    k = ((unsigned long long)mh << 32) | ml;
    c = (int)mc;
}

__global__ void __launch_bounds__(kSelThreads) select_kernel(const SelectArgs a)
{
    __shared__ int picks[64];
    __shared__ unsigned long long pkey[64];
    __shared__ unsigned long long wkey[kSelThreads / 32];
    __shared__ int wcell[kSelThreads / 32];
    __shared__ int npick, stop;
    const int q = blockIdx.x, d_rel = blockIdx.y;
    const int lo = q * a.subband_cells;
    const int hi = min(a.n_f0, lo + a.subband_cells);
    const int d_abs = a.dir_begin + d_rel;
    const unsigned long long *prof =
        reinterpret_cast<const unsigned long long *>(a.profile) + (int64_t)d_abs * a.n_f0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool in_regs = hi - lo <= kSelPer * kSelThreads;
    unsigned long long key[kSelPer];
#pragma unroll
    for (int j = 0; j < kSelPer; ++j) {
        const int b = lo + threadIdx.x + j * kSelThreads;
        key[j] = (in_regs && b < hi) ? prof[b] : 0ull;
    }
    if (threadIdx.x == 0) { npick = 0; stop = 0; }
    __syncthreads();
    for (int k = 0; k < a.top_k; ++k) {
        unsigned long long bk = 0ull;
        int bc = 0x7FFFFFFF;
        const int np = npick;
        if (in_regs) {
            // a thread's cells ascend with j: a strict > keeps the smaller cell on ties
#pragma unroll
            for (int j = 0; j < kSelPer; ++j)
                if (key[j] > bk) { bk = key[j]; bc = lo + threadIdx.x + j * kSelThreads; }
        } else {
            for (int b = lo + threadIdx.x; b < hi; b += blockDim.x) {
                bool ex = false;
                for (int m = 0; m < np; ++m) {
                    const int dd = b > picks[m] ? b - picks[m] : picks[m] - b;
                    if (dd <= a.excl) ex = true;
                }
                if (ex) continue;
                const unsigned long long kb = prof[b];
                if (kb > bk) { bk = kb; bc = b; }
            }
        }
        warp_best(bk, bc);
        if (lane == 0) { wkey[warp] = bk; wcell[warp] = bc; }
        __syncthreads();
        if (warp == 0) {
            bk = lane < nw ? wkey[lane] : 0ull;
            bc = lane < nw ? wcell[lane] : 0x7FFFFFFF;
            warp_best(bk, bc);
            if (lane == 0) {
                if (bk == 0ull) {
                    stop = 1;
                } else {
                    const int count = (int)(unsigned)(bk >> 32);
                    bool ok = count >= a.n_thr;
                    for (int m = 0; m < np && ok; ++m) {
                        const int dd = bc > picks[m] ? bc - picks[m] : picks[m] - bc;
                        if (dd < a.sep) ok = false;
                    }
                    if (!ok) {
                        stop = 1;
                    } else {
                        picks[np] = bc;
                        pkey[np] = bk;
                        npick = np + 1;
                    }
                }
            }
        }
        __syncthreads();
        if (stop) break;
        if (in_regs) {
            const int pc = picks[np];
#pragma unroll
            for (int j = 0; j < kSelPer; ++j) {
                const int b = lo + threadIdx.x + j * kSelThreads;
                const int dd = b > pc ? b - pc : pc - b;
                if (dd <= a.excl) key[j] = 0ull;
            }
        }
    }
    // CR (Eq. cr); adaptive map: mean S1 p0 and variance (S2 p0)(1 - p0) of the
    // weighted noise count, S1 / S2 = the direction's sums of W and W^2 (unit
    // weights give Eq. cr operation for operation)
    double np0, sd;
    if (a.s1 != nullptr) {
        np0 = __dmul_rn((double)a.s1[d_abs], a.p0);
        sd = __dsqrt_rn(__dmul_rn(__dmul_rn((double)a.s2[d_abs], a.p0), __dsub_rn(1.0, a.p0)));
    } else {
        np0 = __dmul_rn((double)a.n_fft, a.p0);
        sd = __dsqrt_rn(__dmul_rn(np0, __dsub_rn(1.0, a.p0)));
    }
    for (int k = threadIdx.x; k < a.top_k; k += blockDim.x) {
        fh_candidate c;
        c.dir = d_abs;
        c.subband = q;
        c.rank = k;
        if (k < npick) {
            const unsigned long long key = pkey[k];
            c.count = (int)(unsigned)(key >> 32);
            c.row = (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
            c.cell = picks[k];
            c.f0 = __dadd_rn(a.f0_min, __ddiv_rn(__dadd_rn((double)c.cell, 0.5), a.kt));
            c.fdot = __dadd_rn(a.fdot_min, __dmul_rn((double)c.row, a.fdot_step));
            c.cr = __ddiv_rn(__dsub_rn((double)c.count, np0), sd);
        } else {
            c.count = -1;
            c.row = -1;
            c.cell = -1;
            c.f0 = 0.0;
            c.fdot = 0.0;
            c.cr = 0.0;
        }
        a.out[((int64_t)d_rel * a.n_sb + q) * a.top_k + k] = c;
    }
}

// ---------------------------------------------------------------- adaptive count bound
// Eq. ncountadap adds W_i per stripe of FFT i, so a count is at most
// sum_i W_i c_i, c_i = the most stripes of FFT i on one cell.  Two stripes of
// FFT i share a cell on some row only if their positions differ by less than K
// cells (s_q - s_p <= K - 1 with s = floor((A - shift) / 2^32) forces
// A_q - A_p < K 2^32), so c_i <= the most positions of FFT i inside a
// half-open window of K cells, found here by two pointers over the FFT's
// ascending positions.  One thread per (direction, FFT); bound[d] receives
// sum_i W_{d,i} c_{d,i} (each product capped at 2^40, which already exceeds
// any admissible bound).  Every index stays inside the FFT's CSR range (a
// valid CSR); unsorted positions only loosen the bound, and such inputs are
// reported by the device checks.
__global__ void __launch_bounds__(256)
weight_bound_kernel(const int64_t *__restrict__ A, const int64_t *__restrict__ offsets,
                    const int32_t *__restrict__ W, int32_t n_fft, int64_t n_peaks,
                    int32_t k_over, unsigned long long *__restrict__ bound)
{
    const int d = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < n_fft) {
        const int64_t *Ad = A + (int64_t)d * n_peaks;
        const int64_t o0 = offsets[i], o1 = offsets[i + 1];
        const unsigned long long width = (unsigned long long)k_over << 32;
        int64_t q = o0, c = 0;
        for (int64_t p = o0; p < o1; ++p) {
            if (q < p + 1) q = p + 1;
            // positions within K cells of A_p (unsigned difference: a wrap from
            // unsorted input ends the window instead of overflowing)
            while (q < o1 && (unsigned long long)(Ad[q] - Ad[p]) < width) ++q;
            if (q - p > c) c = q - p;
        }
        const unsigned long long w = (unsigned long long)(uint32_t)W[(int64_t)d * n_fft + i];
        const unsigned long long cap = 1ull << 40;
        v = (c >= (int64_t)(cap >> 1) || w * (unsigned long long)c > cap) ? cap
                                                                          : w * (unsigned long long)c;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(bound + d, v);
}

// ---------------------------------------------------------------- measurement
// Shared-memory atomicAdd throughput.  Variant 0: lane l always hits bank l
// (8 independent words per thread, immediate offsets, no address math in the
// loop).  Variant 1: pseudo-random words of a 32 KB array.
__global__ void __launch_bounds__(1024, 1)
smem_atomic_bench_kernel(int32_t variant, int32_t iters, unsigned long long *sink)
{
    extern __shared__ __align__(16) int32_t s[];
    constexpr int kWords = 8192;
    for (int w = threadIdx.x; w < kWords; w += blockDim.x) s[w] = 0;
    __syncthreads();
    if (variant == 0) {
        int32_t *p = s + threadIdx.x;  // word w*32 + l, bank l
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 8; ++u) atomicAdd(p + u * 1024, 1);
        }
    } else {
        unsigned x = 2654435761u * (threadIdx.x + 1) + blockIdx.x;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                x = x * 1664525u + 1013904223u;
                atomicAdd(&s[x >> 19], 1);
            }
        }
    }
    __syncthreads();
    unsigned long long acc = 0;
    for (int w = threadIdx.x; w < kWords; w += blockDim.x) acc += (unsigned)s[w];
    atomicAdd(sink, acc);
}

// Binary64 throughput: every thread keeps 8 independent chains, each step one
// __dmul_rn and one __dadd_rn (never contracted into an FMA, like the
// positions' arithmetic); the sum of all chains goes to *sink so nothing is
// dead.  8 x 2 operations per thread per iteration.
__global__ void __launch_bounds__(512)
fp64_bench_kernel(int32_t iters, double a, double b, double *sink)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (double)(threadIdx.x + 37 * k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __dadd_rn(__dmul_rn(x[k], a), b);
    }
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc += x[k];
    if (acc == 12345.678) sink[0] = acc;  // almost never taken; keeps the chains live
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_prep(const PrepArgs &a, cudaStream_t s)
{
    if (a.n_fft <= 0 && !a.offsets_in && !(a.validate && a.n_dir > 0)) return cudaSuccess;
    const int blocks = 1 + (a.n_fft > 0 ? (a.n_fft + 1023) / 1024 : 0);
    prep_kernel<<<blocks, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_correct(const PrepArgs &a, const double *freq, double f0_min,
                           int32_t k_over, int64_t *A, double *out_r, cudaStream_t s)
{
    if (a.n_fft <= 0 && !a.offsets_in && !(a.validate && a.n_dir > 0)) return cudaSuccess;
    const double cshift = 0.5 - 0.5 * (double)k_over;
    const unsigned groups = (unsigned)((std::max(0, a.n_fft) + kPosFfts - 1) / kPosFfts);
    dim3 grid(1 + groups, std::max(1, a.n_dir));
    correct_kernel<<<grid, kPosThreads, 0, s>>>(a, freq, f0_min, cshift, A, out_r);
    return cudaGetLastError();
}

cudaError_t launch_positions_batched(const double *freq, const int64_t *offsets,
                                     const double *v, const double *sky, int32_t n_fft,
                                     int32_t n_dir, int32_t n_batch, const int64_t *a_base,
                                     const int64_t *n_peaks, double f0_min, double kt,
                                     int32_t k_over, int64_t *A, int32_t *err, bool validate,
                                     const int64_t *src, cudaStream_t s)
{
    if (n_fft <= 0 || n_dir <= 0 || n_batch <= 0) return cudaSuccess;
    const double cshift = 0.5 - 0.5 * (double)k_over;
    for (int32_t b0 = 0; b0 < n_batch; b0 += 65535) {
        const int32_t nb = std::min(65535, n_batch - b0);
        dim3 grid((n_fft + kPosFfts - 1) / kPosFfts, n_dir, nb);
        positions_kernel<<<grid, kPosThreads, 0, s>>>(
            freq, offsets + (int64_t)b0 * (n_fft + 1), v, sky + 3 * (int64_t)b0 * n_dir, n_fft,
            0, f0_min, kt, cshift, A, nullptr, err, validate ? 1 : 0, src + (int64_t)b0 * n_fft,
            PosBatch{a_base + b0, n_peaks + b0});
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_validate_device_inputs(const double *t, const double *freq,
                                          const int64_t *offsets, const double *v,
                                          const double *sky, int32_t n_fft, int32_t n_dir,
                                          int32_t *err, cudaStream_t s)
{
    // one warp per FFT; the first n_dir threads also check the sky vectors
    const int64_t threads = (int64_t)(n_fft > 0 ? n_fft : 0) * 32 > n_dir
                                ? (int64_t)n_fft * 32 : (int64_t)n_dir;
    if (threads <= 0) return cudaSuccess;
    validate_device_inputs_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        t, freq, offsets, v, sky, n_fft, n_dir, err);
    return cudaGetLastError();
}

__host__ __device__ int32_t guard_for(unsigned long long dmax, int32_t span_rows)
{
    // span_rows rows of drift, rounded up to whole cells, plus 2 cells of margin
    const unsigned long long drift = (unsigned long long)span_rows * dmax;
    return (int32_t)((drift + 0xFFFFFFFFull) >> 32) + 2;
}

size_t transform_smem_bytes(int32_t tile_cells, int32_t k_over, int32_t mode, int32_t nwarps,
                            int32_t guard)
{
    // counters of W + K - 1 cells, one dump cell and 2 x guard cells, per-warp
    // owner tables, (DIFF) per-warp segment totals, the chunk counter, and 128
    // bytes of alignment slack
    size_t words = (size_t)(tile_cells + k_over + 2 * guard) * kRows + (size_t)nwarps * 32;
    if (mode == FH_MODE_DIFF) words += (size_t)nwarps * 32;
    return (words + 4) * sizeof(int32_t) + 128;
}

// Kernel instantiation for a counting mode and block size: blocks of up to 512
// threads get up to 128 registers per thread, of up to 640 threads (START
// mode) 102, of up to 768 threads 80, of 1024 threads 64.
template <bool WEIGHTED, int PACK, typename F>
static auto with_transform_kernel_w(int32_t mode, int32_t nwarps, F &&f)
{
    if constexpr (!PACK) {
        if (mode == FH_MODE_DIFF)
            return nwarps > 16 ? f(transform_kernel<FH_MODE_DIFF, 1024, WEIGHTED, false>)
                               : f(transform_kernel<FH_MODE_DIFF, 512, WEIGHTED, false>);
    }
    return nwarps > 24   ? f(transform_kernel<FH_MODE_START, 1024, WEIGHTED, PACK>)
           : nwarps > 20 ? f(transform_kernel<FH_MODE_START, 768, WEIGHTED, PACK>)
           : nwarps > 16 ? f(transform_kernel<FH_MODE_START, 640, WEIGHTED, PACK>)
                         : f(transform_kernel<FH_MODE_START, 512, WEIGHTED, PACK>);
}
// weighted: instantiation that adds per-FFT weights (adaptive map); plain: +1;
// pack: direction pairs with two 16-bit counts per word (plain START map only)
template <typename F>
static auto with_transform_kernel(int32_t mode, int32_t nwarps, bool weighted, int pack, F &&f)
{
    if (pack == 1) return with_transform_kernel_w<false, 1>(FH_MODE_START, nwarps, f);
    if (pack == 2) return with_transform_kernel_w<false, 2>(FH_MODE_START, nwarps, f);
    return weighted ? with_transform_kernel_w<true, 0>(mode, nwarps, f)
                    : with_transform_kernel_w<false, 0>(mode, nwarps, f);
}

cudaError_t transform_prepare(int32_t mode, size_t smem)
{
    cudaError_t e = cudaSuccess;
    for (int nw : {16, 20, 24, 32})
        for (int v = 0; v < 4; ++v) {
            const bool wt = v == 1;
            const int pk = v >= 2 ? v - 1 : 0;
            if (pk && mode != FH_MODE_START) continue;
            const cudaError_t r = with_transform_kernel(mode, nw, wt, pk, [&](auto k) {
                return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem);
            });
            if (r != cudaSuccess) e = r;
        }
    return e;
}

int transform_blocks_per_sm(int32_t mode, int32_t nwarps, size_t smem)
{
    int n = 0;
    // (both instantiations are bounded to one block of nwarps warps per SM by
    // their launch bounds; shared memory decides the rest)
    const cudaError_t e = with_transform_kernel(mode, nwarps, false, 0, [&](auto k) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, nwarps * 32, smem);
    });
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_transform(int32_t mode, const JobTable &tbl, int64_t total_items,
                             int32_t grid, int32_t nwarps, size_t smem, int32_t guard,
                             cudaStream_t s, unsigned int *sched)
{
    if (total_items <= 0) return cudaSuccess;
    if (total_items >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
    // counters (+ dump cell) of the widest tile with its guard cells; owner tables follow
    int32_t hist_words = 0;
    for (int j = 0; j < tbl.n_jobs; ++j) {
        const int32_t w = (tbl.job[j].tile_cells + tbl.job[j].k_over + 2 * guard) * kRows;
        hist_words = w > hist_words ? w : hist_words;
    }
    // the launch's packing: every job with direction pairs (1), or with row pairs (2)
    bool weighted = false, dirs = mode == FH_MODE_START && tbl.n_jobs > 0, rows = dirs;
    for (int j = 0; j < tbl.n_jobs; ++j) {
        weighted = weighted || tbl.job[j].weights != nullptr;
        dirs = dirs && tbl.job[j].dir_pairs != 0;
        rows = rows && tbl.job[j].row_pairs != 0;
    }
    const int pack = dirs ? 1 : rows ? 2 : 0;
    if (weighted && pack) return cudaErrorInvalidValue;  // packed counters hold plain counts only
    with_transform_kernel(mode, nwarps, weighted, pack, [&](auto k) {
        k<<<grid, nwarps * 32, smem, s>>>(tbl, total_items, hist_words, guard, kRows * 4u, sched);
        return cudaSuccess;
    });
    return cudaGetLastError();
}

cudaError_t launch_windows(const TransformJob &job, uint32_t *windows, cudaStream_t s)
{
    if (job.n_fft <= 0 || job.n_dir <= 0) return cudaSuccess;
    dim3 grid((job.n_fft + 7) / 8, job.dir_pairs ? (job.n_dir + 1) / 2 : job.n_dir);
    // tiles per lane and pass: enough for all tiles in one pass, at most kWinMaxM
    const int m = std::min(kWinMaxM, std::max(1, (job.n_tiles + 31) / 32));
    auto go = [&](auto pair_tag) {
        constexpr bool P = decltype(pair_tag)::value;
        if (m == 1)
            windows_kernel<1, P><<<grid, 256, 0, s>>>(job, windows);
        else if (m == 2)
            windows_kernel<2, P><<<grid, 256, 0, s>>>(job, windows);
        else
            windows_kernel<3, P><<<grid, 256, 0, s>>>(job, windows);
    };
    if (job.dir_pairs)
        go(std::true_type{});
    else
        go(std::false_type{});
    return cudaGetLastError();
}

cudaError_t launch_select(const SelectArgs &a, cudaStream_t s)
{
    if (a.n_dir <= 0 || a.n_sb <= 0) return cudaSuccess;
    dim3 grid(a.n_sb, a.n_dir);
    select_kernel<<<grid, kSelThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_weight_bound(const int64_t *A, const int64_t *offsets, const int32_t *W,
                                int32_t n_fft, int32_t n_dir, int64_t n_peaks, int32_t k_over,
                                unsigned long long *bound, cudaStream_t s)
{
    if (n_fft <= 0 || n_dir <= 0) return cudaSuccess;
    dim3 grid((n_fft + 255) / 256, n_dir);
    weight_bound_kernel<<<grid, 256, 0, s>>>(A, offsets, W, n_fft, n_peaks, k_over, bound);
    return cudaGetLastError();
}

cudaError_t launch_fp64_bench(int32_t iters, int32_t grid, double *sink, cudaStream_t s)
{
    fp64_bench_kernel<<<grid, 512, 0, s>>>(iters, 0.999999, 1e-6, sink);
    return cudaGetLastError();
}

cudaError_t launch_smem_atomic_bench(int32_t variant, int32_t iters, int32_t grid,
                                     unsigned long long *sink, cudaStream_t s)
{
    const size_t smem = 8192 * sizeof(int32_t);
    smem_atomic_bench_kernel<<<grid, 1024, smem, s>>>(variant, iters, sink);
    return cudaGetLastError();
}

}  // namespace fh
