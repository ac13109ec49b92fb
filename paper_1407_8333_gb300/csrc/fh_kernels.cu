// Kernels of the frequency-Hough hot path (sm_103a).
//
//   positions_kernel     a1 + a2  Doppler factor and 32.32 fixed-point stripe start
//                                 (Eq. fdopp; Sec. VI; Eq. freqres)
//   shift_tables_kernel  a3       per-FFT spin-down shift (Eqs. uno, sdstep)
//   transform_kernel     a4 + a5 + profile half of a6 (Eqs. due, ncount; Sec. VIII)
//   select_kernel        a6       per-sub-band greedy picks (Sec. VIII; Eq. cr)
//
// Floating point: every binary64 operation is an explicit round-to-nearest
// intrinsic (__dmul_rn, __dadd_rn, ...), so nothing is contracted into an FMA
// and the results are the IEEE values of the operations in the stated order.
// After the fixed-point conversion the path is integer only.
#include <climits>
#include <cstdint>

#include "fh_internal.h"

namespace fh {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kTwo32 = 4294967296.0;
constexpr int kPosFfts = 64;
constexpr int kPosThreads = 256;

// ---------------------------------------------------------------- a1 + a2
// grid (ceil(n_fft / 64), n_dir): the block computes r = 1 / (1 + v.n) for 64
// FFTs of one direction, then the fixed-point position of each of their peaks
// (a contiguous CSR range, so loads and stores are coalesced).
__global__ void __launch_bounds__(kPosThreads)
positions_kernel(const double *__restrict__ freq, const int64_t *__restrict__ offsets,
                 const double *__restrict__ v, const double *__restrict__ sky, int32_t n_fft,
                 int64_t n_peaks, double f0_min, double kt, double cshift,
                 int64_t *__restrict__ A, double *__restrict__ out_r, int32_t *err)
{
    __shared__ double r_s[kPosFfts];
    __shared__ int64_t off_s[kPosFfts + 1];
    const int d = blockIdx.y;
    const int i0 = blockIdx.x * kPosFfts;
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
    if (threadIdx.x <= nf) off_s[threadIdx.x] = offsets[i0 + threadIdx.x];
    __syncthreads();
    const int64_t p_begin = off_s[0], p_end = off_s[nf];
    int64_t *__restrict__ Ad = A + (int64_t)d * n_peaks;
    bool bad = false;
    for (int64_t p = p_begin + threadIdx.x; p < p_end; p += blockDim.x) {
        int lo = 0, hi = nf;  // off_s[lo] <= p < off_s[hi]
        while (hi - lo > 1) {
            const int m = (lo + hi) >> 1;
            if (off_s[m] <= p) lo = m; else hi = m;
        }
        const double u = __dmul_rn(freq[p], r_s[lo]);
        const double x = __dsub_rn(u, f0_min);
        const double y = __dmul_rn(x, kt);
        const double a = __dadd_rn(y, cshift);
        bad |= !(fabs(a) < (double)kFixedLimit);
        Ad[p] = (int64_t)floor(__dmul_rn(a, kTwo32));
    }
    if (bad) atomicOr(err, kErrRange);
}

// ---------------------------------------------------------------- a3
__global__ void shift_tables_kernel(const double *__restrict__ t, int32_t n_fft, double t_ref,
                                    double kt, double fdot_min, double fdot_step,
                                    double fdot_absmax, int64_t *__restrict__ S0,
                                    int64_t *__restrict__ D, int32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_fft) return;
    const double dt = __dsub_rn(t[i], t_ref);
    const double c = __dmul_rn(dt, kt);
    const double s0 = __dmul_rn(fdot_min, c);
    const double dd = __dmul_rn(fdot_step, c);
    if (!(fabs(c) * fdot_absmax < (double)kFixedLimit)) atomicOr(err, kErrRange);
    S0[i] = (int64_t)floor(__dmul_rn(s0, kTwo32));
    D[i] = (int64_t)floor(__dmul_rn(dd, kTwo32));
}

// ---------------------------------------------------------------- device inputs
// One block: copy offsets[0..n_fft] into a valid CSR (clamped to [0, n_peaks],
// made non-decreasing by a running maximum, last entry = n_peaks) and flag
// any entry that had to change.  Later kernels index peaks only through the
// sanitised copy, so a bad device peakmap cannot make them read out of range.
__global__ void __launch_bounds__(1024)
sanitize_offsets_kernel(const int64_t *__restrict__ in, int32_t n_fft, int64_t n_peaks,
                        int64_t *__restrict__ out, int32_t *err)
{
    __shared__ int64_t wmax[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    bool bad = false;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base <= n_fft; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int64_t x = 0;
        if (i <= n_fft) {
            x = in[i];
            if (x < 0 || x > n_peaks) bad = true;
            if (i == 0 && x != 0) bad = true;
            if (i == n_fft && x != n_peaks) bad = true;
            if (i > 0 && x < in[i - 1]) bad = true;
            x = x < 0 ? 0 : (x > n_peaks ? n_peaks : x);
            if (i == 0) x = 0;
        }
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o && y > x) x = y;
        }
        if (lane == 31) wmax[warp] = x;
        __syncthreads();
        int64_t pre = carry;
        for (int w = 0; w < warp; ++w) pre = wmax[w] > pre ? wmax[w] : pre;
        if (pre > x) x = pre;
        if (i <= n_fft) out[i] = (i == n_fft) ? n_peaks : x;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = x;
        __syncthreads();
    }
    if (bad) atomicOr(err, kErrCsr);
}

// Flags non-finite / unordered device inputs (thread per FFT and per direction).
__global__ void validate_device_inputs_kernel(const double *__restrict__ t,
                                              const double *__restrict__ freq,
                                              const int64_t *__restrict__ offsets,
                                              const double *__restrict__ v,
                                              const double *__restrict__ sky, int32_t n_fft,
                                              int32_t n_dir, int32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t e = 0;
    if (i < n_fft) {
        if (!isfinite(t[i]) || (i > 0 && !(t[i] > t[i - 1]))) e |= kErrUnsorted;
        for (int c = 0; c < 3; ++c)
            if (!(fabs(v[3 * (int64_t)i + c]) < 0.1)) e |= kErrInvalid;
        double prev = 0.0;
        for (int64_t p = offsets[i]; p < offsets[i + 1]; ++p) {
            const double f = freq[p];
            if (!isfinite(f) || !(f > 0.0)) e |= kErrInvalid;
            if (p > offsets[i] && !(f > prev)) e |= kErrUnsorted;
            prev = f;
        }
    }
    if (i < n_dir) {
        const double x = sky[3 * (int64_t)i], y = sky[3 * (int64_t)i + 1],
                     z = sky[3 * (int64_t)i + 2];
        if (!(fabs(x) <= 1.000001 && fabs(y) <= 1.000001 && fabs(z) <= 1.000001))
            e |= kErrInvalid;
    }
    if (e) atomicOr(err, e);
}

// ---------------------------------------------------------------- a4 + a5 + profile
// One block per work item (direction, slab of 32 spin-down rows, tile of W
// frequency cells); a persistent grid strides over the items of all jobs.
//
// Shared memory holds the tile's counters H[L][row], L = s - (b0 - K + 1) for
// a stripe starting at cell s (so L in [0, W + K - 1) covers every stripe that
// touches the tile), row stride 32 words: lane l <-> row j0 + l <-> bank l.
//
// Accumulate: each warp takes 32 FFTs at a time.  Lane i binary-searches FFT
// i's (ascending) positions for the first peak that can reach the tile on any
// row of the slab; then, FFT by FFT, the warp loads 32 positions at once and,
// for each peak, every lane adds its own row's +1 (START: one atomic at the
// stripe start; DIFF: +1 at the first covered cell and -1 after the last).
// All 32 atomics of one instruction go to 32 different banks.
//
// Emit: lane l walks its row along f0 over a segment of the tile (one segment
// per warp): START sums a K-cell window of starts, DIFF takes a running sum
// with the other segments' totals as carry-in.  The count goes to the map
// (optional) and the warp's max over rows (smallest row on ties) to the
// direction's profile by a 64-bit atomicMax, which is order-independent.
template <int MODE>
__global__ void __launch_bounds__(1024, 1)
transform_kernel(const __grid_constant__ JobTable tbl, int64_t total_items, int32_t hist_words)
{
    extern __shared__ __align__(16) int32_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;

    for (int64_t item = blockIdx.x; item < total_items; item += gridDim.x) {
        int jb = 0;
        while (jb + 1 < tbl.n_jobs && item >= tbl.job[jb + 1].item_begin) ++jb;
        const TransformJob *J = &tbl.job[jb];
        const int64_t rem = item - J->item_begin;
        const int per_dir = J->n_slabs * J->n_tiles;
        const int d_rel = (int)(rem / per_dir);
        const int r2 = (int)(rem - (int64_t)d_rel * per_dir);
        const int slab = r2 / J->n_tiles;
        const int tile = r2 - slab * J->n_tiles;
        const int K = J->k_over, W = J->tile_cells, n_f0 = J->n_f0, n_fdot = J->n_fdot;
        const int n_fft = J->n_fft;
        const int j0 = slab * kRows;
        const int R = min(kRows, n_fdot - j0);
        const int b0 = tile * W;
        const int Wt = min(W, n_f0 - b0);
        const int E = Wt + K - 1;
        const int d_abs = J->dir_begin + d_rel;
        const int64_t *__restrict__ Ad = J->A + (int64_t)d_abs * J->n_peaks;
        const int64_t *__restrict__ offs = J->offsets;
        const int64_t *__restrict__ S0 = J->S0;
        const int64_t *__restrict__ Dt = J->D;
        const bool row_ok = lane < R;

        // zero the counters
        {
            int4 *h4 = reinterpret_cast<int4 *>(smem);
            const int n4 = (E * kRows) >> 2;
            for (int w = threadIdx.x; w < n4; w += blockDim.x) h4[w] = make_int4(0, 0, 0, 0);
        }
        __syncthreads();

        // accumulate
        const int64_t base_shift = (int64_t)(b0 - K + 1) * 4294967296LL;
        const int64_t e_fixed = (int64_t)E * 4294967296LL;
        const int nchunks = (n_fft + 31) >> 5;
        for (int c = warp; c < nchunks; c += nwarps) {
            const int i = (c << 5) + lane;
            int64_t q0 = 0, q1 = 0, hi = 0, cb = 0, dv = 0;
            if (i < n_fft) {
                const int64_t o0 = offs[i], o1 = offs[i + 1];
                dv = Dt[i];
                cb = S0[i] + (int64_t)j0 * dv + base_shift;
                const int64_t span = (int64_t)(R - 1) * dv;
                const int64_t lo = cb + (span < 0 ? span : 0);
                hi = cb + (span > 0 ? span : 0) + e_fixed;
                int64_t a = o0, b = o1;
                while (a < b) {
                    const int64_t m = (a + b) >> 1;
                    if (__ldg(Ad + m) < lo) a = m + 1; else b = m;
                }
                q0 = a;
                q1 = o1;
            }
            unsigned todo = __ballot_sync(kFull, q0 < q1);
            while (todo) {
                const int k = __ffs(todo) - 1;
                todo &= todo - 1;
                int64_t q = __shfl_sync(kFull, q0, k);
                const int64_t qe = __shfl_sync(kFull, q1, k);
                const int64_t h = __shfl_sync(kFull, hi, k);
                const int64_t off = __shfl_sync(kFull, cb, k) + (int64_t)lane * __shfl_sync(kFull, dv, k);
                for (;;) {
                    const int64_t idx = q + lane;
                    const int64_t av = (idx < qe) ? __ldg(Ad + idx) : LLONG_MAX;
                    const int n = __popc(__ballot_sync(kFull, av < h));
                    for (int t = 0; t < n; ++t) {
                        const int64_t a = __shfl_sync(kFull, av, t);
                        const int L = (int)((a - off) >> 32);
                        if (row_ok && (unsigned)L < (unsigned)E) {
                            if (MODE == FH_MODE_START) {
                                atomicAdd(&smem[L * kRows + lane], 1);
                            } else {
                                const int st = L - K + 1;
                                atomicAdd(&smem[(st > 0 ? st : 0) * kRows + lane], 1);
                                if (L + 1 < Wt) atomicAdd(&smem[(L + 1) * kRows + lane], -1);
                            }
                        }
                    }
                    if (n < 32) break;
                    q += 32;
                }
            }
        }
        __syncthreads();

        // emit counts, map and profile
        const int seg = (Wt + nwarps - 1) / nwarps;
        const int c0 = min(Wt, warp * seg);
        const int c1 = min(Wt, c0 + seg);
        int32_t *maprow = nullptr;
        if (J->maps != nullptr && row_ok)
            maprow = J->maps + ((int64_t)d_rel * n_fdot + j0 + lane) * n_f0 + b0;
        unsigned long long *prof =
            reinterpret_cast<unsigned long long *>(J->profile) + (int64_t)d_abs * n_f0 + b0;
        auto emit = [&](int c, int count) {
            if (maprow) maprow[c] = count;
            const int cm = __reduce_max_sync(kFull, row_ok ? count : INT_MIN);
            const unsigned rm = __reduce_min_sync(kFull, (row_ok && count == cm) ? (unsigned)lane : 32u);
            if (lane == (c & 31))
                atomicMax(prof + c, ((unsigned long long)(unsigned)cm << 32) |
                                        (0xFFFFFFFFull - (unsigned long long)(unsigned)(j0 + rm)));
        };
        if (MODE == FH_MODE_START) {
            int win = 0;
            if (c0 < c1)
                for (int L = c0; L < c0 + K - 1; ++L) win += smem[L * kRows + lane];
            for (int c = c0; c < c1; ++c) {
                win += smem[(c + K - 1) * kRows + lane];
                emit(c, win);
                win -= smem[c * kRows + lane];
            }
        } else {
            int32_t *segtot = smem + hist_words;
            int tot = 0;
            for (int c = c0; c < c1; ++c) tot += smem[c * kRows + lane];
            segtot[warp * 32 + lane] = tot;
            __syncthreads();
            int acc = 0;
            for (int w = 0; w < warp; ++w) acc += segtot[w * 32 + lane];
            for (int c = c0; c < c1; ++c) {
                acc += smem[c * kRows + lane];
                emit(c, acc);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- a6
// grid (n_sb, n_dir), 256 threads: greedy picks of one sub-band of one direction.
__global__ void __launch_bounds__(256) select_kernel(const SelectArgs a)
{
    __shared__ int picks[64];
    __shared__ unsigned long long pkey[64];
    __shared__ unsigned long long wkey[8];
    __shared__ int wcell[8];
    __shared__ int npick, stop;
    const int q = blockIdx.x, d_rel = blockIdx.y;
    const int lo = q * a.subband_cells;
    const int hi = min(a.n_f0, lo + a.subband_cells);
    const int d_abs = a.dir_begin + d_rel;
    const unsigned long long *prof =
        reinterpret_cast<const unsigned long long *>(a.profile) + (int64_t)d_abs * a.n_f0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) { npick = 0; stop = 0; }
    __syncthreads();
    for (int k = 0; k < a.top_k; ++k) {
        unsigned long long bk = 0ull;
        int bc = INT_MAX;
        const int np = npick;
        for (int b = lo + threadIdx.x; b < hi; b += blockDim.x) {
            bool ex = false;
            for (int m = 0; m < np; ++m) {
                const int dd = b > picks[m] ? b - picks[m] : picks[m] - b;
                if (dd <= a.excl) ex = true;
            }
            if (ex) continue;
            const unsigned long long key = prof[b];
            if (key > bk || (key == bk && b < bc)) { bk = key; bc = b; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long k2 = __shfl_down_sync(kFull, bk, o);
            const int c2 = __shfl_down_sync(kFull, bc, o);
            if (k2 > bk || (k2 == bk && c2 < bc)) { bk = k2; bc = c2; }
        }
        if (lane == 0) { wkey[warp] = bk; wcell[warp] = bc; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nw; ++w)
                if (wkey[w] > bk || (wkey[w] == bk && wcell[w] < bc)) { bk = wkey[w]; bc = wcell[w]; }
            if (bc == INT_MAX || bk == 0ull) {
                stop = 1;
            } else {
                const int count = (int)(unsigned)(bk >> 32);
                bool ok = count >= a.n_thr;
                for (int m = 0; m < npick && ok; ++m) {
                    const int dd = bc > picks[m] ? bc - picks[m] : picks[m] - bc;
                    if (dd < a.sep) ok = false;
                }
                if (!ok) {
                    stop = 1;
                } else {
                    picks[npick] = bc;
                    pkey[npick] = bk;
                    ++npick;
                }
            }
        }
        __syncthreads();
        if (stop) break;
    }
    const double np0 = __dmul_rn((double)a.n_fft, a.p0);
    const double sd = __dsqrt_rn(__dmul_rn(np0, __dsub_rn(1.0, a.p0)));
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

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_shift_tables(const double *t, int32_t n_fft, double t_ref, double kt,
                                double fdot_min, double fdot_step, int32_t n_fdot,
                                int64_t *S0, int64_t *D, int32_t *err, cudaStream_t s)
{
    if (n_fft <= 0) return cudaSuccess;
    const double f_last = fdot_min + (double)(n_fdot - 1) * fdot_step;
    const double absmax = fabs(fdot_min) > fabs(f_last) ? fabs(fdot_min) : fabs(f_last);
    shift_tables_kernel<<<(n_fft + 255) / 256, 256, 0, s>>>(t, n_fft, t_ref, kt, fdot_min,
                                                             fdot_step, absmax, S0, D, err);
    return cudaGetLastError();
}

cudaError_t launch_positions(const double *freq, const int64_t *offsets, const double *v,
                             const double *sky, int32_t n_fft, int64_t n_peaks, int32_t n_dir,
                             double f0_min, double kt, int32_t k_over, int64_t *A,
                             double *out_r, int32_t *err, cudaStream_t s)
{
    if (n_fft <= 0 || n_dir <= 0) return cudaSuccess;
    const double cshift = 0.5 - 0.5 * (double)k_over;
    dim3 grid((n_fft + kPosFfts - 1) / kPosFfts, n_dir);
    positions_kernel<<<grid, kPosThreads, 0, s>>>(freq, offsets, v, sky, n_fft, n_peaks, f0_min,
                                                  kt, cshift, A, out_r, err);
    return cudaGetLastError();
}

cudaError_t launch_sanitize_offsets(const int64_t *in, int32_t n_fft, int64_t n_peaks,
                                    int64_t *out, int32_t *err, cudaStream_t s)
{
    sanitize_offsets_kernel<<<1, 1024, 0, s>>>(in, n_fft, n_peaks, out, err);
    return cudaGetLastError();
}

cudaError_t launch_validate_device_inputs(const double *t, const double *freq,
                                          const int64_t *offsets, const double *v,
                                          const double *sky, int32_t n_fft, int32_t n_dir,
                                          int32_t *err, cudaStream_t s)
{
    const int n = n_fft > n_dir ? n_fft : n_dir;
    if (n <= 0) return cudaSuccess;
    validate_device_inputs_kernel<<<(n + 255) / 256, 256, 0, s>>>(t, freq, offsets, v, sky,
                                                                  n_fft, n_dir, err);
    return cudaGetLastError();
}

size_t transform_smem_bytes(int32_t tile_cells, int32_t k_over, int32_t mode, int32_t nwarps)
{
    size_t words = (size_t)(tile_cells + k_over - 1) * kRows;
    if (mode == FH_MODE_DIFF) words += (size_t)nwarps * 32;
    return words * sizeof(int32_t);
}

cudaError_t transform_prepare(int32_t mode, size_t smem)
{
    if (mode == FH_MODE_DIFF)
        return cudaFuncSetAttribute(transform_kernel<FH_MODE_DIFF>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaFuncSetAttribute(transform_kernel<FH_MODE_START>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int transform_blocks_per_sm(int32_t mode, int32_t nwarps, size_t smem)
{
    int n = 0;
    cudaError_t e;
    if (mode == FH_MODE_DIFF)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transform_kernel<FH_MODE_DIFF>,
                                                          nwarps * 32, smem);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, transform_kernel<FH_MODE_START>,
                                                          nwarps * 32, smem);
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_transform(int32_t mode, const JobTable &tbl, int64_t total_items,
                             int32_t grid, int32_t nwarps, size_t smem, cudaStream_t s)
{
    if (total_items <= 0) return cudaSuccess;
    int32_t hist_words = 0;
    for (int j = 0; j < tbl.n_jobs; ++j) {
        const int32_t w = (tbl.job[j].tile_cells + tbl.job[j].k_over - 1) * kRows;
        hist_words = w > hist_words ? w : hist_words;
    }
    if (mode == FH_MODE_DIFF)
        transform_kernel<FH_MODE_DIFF><<<grid, nwarps * 32, smem, s>>>(tbl, total_items, hist_words);
    else
        transform_kernel<FH_MODE_START><<<grid, nwarps * 32, smem, s>>>(tbl, total_items, hist_words);
    return cudaGetLastError();
}

cudaError_t launch_select(const SelectArgs &a, cudaStream_t s)
{
    if (a.n_dir <= 0 || a.n_sb <= 0) return cudaSuccess;
    dim3 grid(a.n_sb, a.n_dir);
    select_kernel<<<grid, 256, 0, s>>>(a);
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
