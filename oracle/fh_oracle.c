/*
 * Frequency-Hough (FH) oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU statement of what the FH hot path
 * computes (Astone et al., "Method for all-sky searches of continuous
 * gravitational wave signals using the frequency-Hough transform").  Only the
 * tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.  It
 * shares no code, header, table or helper with the CUDA library, and the
 * library never calls it.
 *
 * Arithmetic rules: IEEE-754 binary64 with round-to-nearest-even; every
 * floating-point operation below is rounded on its own, in the order written
 * (the file is compiled with -ffp-contract=off so that no multiply-add is
 * fused).  floor() is exact; conversions to int64 are exact for the ranges the
 * callers validate (|value| < 2^62).  Everything after the fixed-point
 * conversion is integer arithmetic.
 *
 * The steps, in the paper's order:
 *   a1  Doppler factor r = 1 / (1 + v.n)              (Eq. fdopp, Sec. II; Sec. VI)
 *   a2  corrected peak position in over-resolved cells, as 32.32 fixed point
 *                                                      (Sec. VI; Eq. freqres)
 *   a3  spin-down shift of each FFT for the first grid row and per row step
 *                                                      (Eq. uno; Eq. sdstep; t0 in Sec. VI)
 *   a4  stripe of each peak on each spin-down row: K cells starting at s;
 *       +1 at the start and -1 after the end in a differential row
 *                                                      (Eqs. due, ncount)
 *   a5  cumulative sum along f0 -> integer number counts (Eq. ncount)
 *   a6  per-sub-band candidate selection over all spin-down rows, with the
 *       second-order exclusion/separation rule         (Sec. VIII)
 *
 * Where the paper is loose (stripe width, rounding of the stripe start, cell
 * and frequency conventions, the selection rule's units) the reading taken is
 * restated in the comment of the step that uses it.
 *
 * Section numbers: II signal model, VI frequency-Hough transform, VII coarse
 * grid, VIII selection of first-level candidates, XII sensitivity (Eq. cr).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO32 4294967296.0

int fho_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void fho_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* floor(x / 2^32) for a signed 64-bit x, written as plain integer division. */
static int64_t floor_div_2_32(int64_t x)
{
    const int64_t q = 4294967296LL;
    if (x >= 0) return x / q;
    return -((-x + q - 1) / q);
}

/*
 * a1 -- Doppler factor (Eq. fdopp: f = f0 (1 + v.n / c); the peakmap is
 * corrected by dividing the observed frequency by that factor, Sec. VI).
 * v: n_fft x 3 detector velocities in units of c.  sky: n_dir x 3 unit vectors.
 * r: n_dir x n_fft, r[d][i] = 1 / (1 + ((v_x n_x + v_y n_y) + v_z n_z)).
 */
void fho_doppler_factor(int32_t n_fft, const double *v, int32_t n_dir,
                        const double *sky, double *r)
{
    for (int32_t d = 0; d < n_dir; ++d) {
        const double nx = sky[3 * (int64_t)d + 0];
        const double ny = sky[3 * (int64_t)d + 1];
        const double nz = sky[3 * (int64_t)d + 2];
        for (int32_t i = 0; i < n_fft; ++i) {
            const double px = v[3 * (int64_t)i + 0] * nx;
            const double py = v[3 * (int64_t)i + 1] * ny;
            const double pz = v[3 * (int64_t)i + 2] * nz;
            const double dot = (px + py) + pz;
            const double den = 1.0 + dot;
            r[(int64_t)d * n_fft + i] = 1.0 / den;
        }
    }
}

/*
 * a2 -- corrected position of every peak, in over-resolved cells (width
 * delta_f_H = 1 / (K T_FFT), Eq. freqres), as 32.32 fixed point.
 * With u = f r the Doppler-corrected frequency, the stripe centre in cell units
 * is x = (u - f0_min) K T_FFT.  A stripe is K cells wide (one FFT bin, Eq. due
 * with the input-plane bin width 1/T_FFT) and covers the cells whose centre
 * lies in (x - K/2, x + K/2]; its first cell is floor(x - K/2 + 1/2).  So
 *   a = (u - f0_min) * KT + (0.5 - 0.5 K),   A = floor(a * 2^32).
 * offsets: n_fft + 1 CSR offsets; freq: n_peaks; r: n_dir x n_fft (from a1);
 * A: n_dir x n_peaks.
 */
void fho_positions(int32_t n_fft, const int64_t *offsets, const double *freq,
                   int32_t n_dir, const double *r, double f0_min, double kt,
                   int32_t k_over, int64_t *A)
{
    const int64_t n_peaks = offsets[n_fft];
    const double c = 0.5 - 0.5 * (double)k_over;
    for (int32_t d = 0; d < n_dir; ++d) {
        for (int32_t i = 0; i < n_fft; ++i) {
            const double ri = r[(int64_t)d * n_fft + i];
            for (int64_t p = offsets[i]; p < offsets[i + 1]; ++p) {
                const double u = freq[p] * ri;
                const double x = u - f0_min;
                const double y = x * kt;
                const double a = y + c;
                A[(int64_t)d * n_peaks + p] = (int64_t)floor(a * TWO32);
            }
        }
    }
}

/*
 * a3 -- spin-down shift tables (Eq. uno: f0 = f - fdot (t - t0); rows
 * fdot_j = fdot_min + j * fdot_step, Eq. sdstep; t0 = t_ref, Sec. VI).
 * In cell units the shift of FFT i on row j is fdot_j * c_i with
 * c_i = (t_i - t_ref) * KT; it is realised in 32.32 fixed point as
 * S0_i + j * D_i with S0_i = floor(fdot_min c_i 2^32), D_i = floor(fdot_step c_i 2^32).
 */
void fho_shift_tables(int32_t n_fft, const double *t, double t_ref, double kt,
                      double fdot_min, double fdot_step, int64_t *S0, int64_t *D)
{
    for (int32_t i = 0; i < n_fft; ++i) {
        const double dt = t[i] - t_ref;
        const double c = dt * kt;
        const double s0 = fdot_min * c;
        const double dd = fdot_step * c;
        S0[i] = (int64_t)floor(s0 * TWO32);
        D[i] = (int64_t)floor(dd * TWO32);
    }
}

/* first cell of the stripe of peak p (FFT i) on row j */
static int64_t stripe_start(int64_t Ap, int64_t S0i, int64_t Di, int64_t j)
{
    const int64_t shift = S0i + j * Di;
    return floor_div_2_32(Ap - shift);
}

/*
 * a4 + a5 -- Hough map of one direction, by the differential method: on each
 * row, every peak adds +1 at its first cell inside [0, n_f0) and -1 at the
 * first cell after its stripe (when that cell is inside the map); the
 * cumulative sum along f0 then gives the number count of every cell
 * (Eq. ncount: +1 in every cell a stripe touches).
 * A: n_peaks positions of this direction (from a2).  rows: the n_rows row
 * indices to compute (NULL = all n_fdot rows in order).  map: n_rows x n_f0.
 * w: NULL for the plain map, or the adaptive map's integer weights of this
 * direction, one per FFT (Eq. ncountadap: n = sum_i w_i n_i, the FFT's peaks
 * adding w_i instead of 1; the weights are given already quantised to fixed
 * point, so the map stays an exact integer).
 */
void fho_hough_map(int32_t n_fft, const int64_t *offsets, const int64_t *A,
                   const int64_t *S0, const int64_t *D, int32_t k_over,
                   int32_t n_f0, int32_t n_rows, const int32_t *rows, const int32_t *w,
                   int32_t *map)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t q = 0; q < n_rows; ++q) {
        const int64_t j = rows ? rows[q] : q;
        int32_t *row = map + (int64_t)q * n_f0;
        memset(row, 0, sizeof(int32_t) * (size_t)n_f0);
        for (int32_t i = 0; i < n_fft; ++i) {
            const int32_t wi = w ? w[i] : 1;
            for (int64_t p = offsets[i]; p < offsets[i + 1]; ++p) {
                const int64_t s = stripe_start(A[p], S0[i], D[i], j);
                const int64_t e = s + k_over;
                if (s < n_f0 && e > 0) row[s > 0 ? s : 0] += wi;
                if (e > 0 && e < n_f0) row[e] -= wi;
            }
        }
        int32_t acc = 0;
        for (int32_t b = 0; b < n_f0; ++b) {
            acc += row[b];
            row[b] = acc;
        }
    }
}

/*
 * The same map by direct counting: every (peak, row) adds 1 (or its FFT's
 * weight w[i]) to each cell of [s, s + K) inside [0, n_f0).  For tiny inputs
 * only; it is the plain definition of the number count that the differential
 * method must reproduce.
 */
void fho_hough_map_direct(int32_t n_fft, const int64_t *offsets, const int64_t *A,
                          const int64_t *S0, const int64_t *D, int32_t k_over,
                          int32_t n_f0, int32_t n_fdot, const int32_t *w, int32_t *map)
{
    memset(map, 0, sizeof(int32_t) * (size_t)n_fdot * (size_t)n_f0);
    for (int32_t j = 0; j < n_fdot; ++j) {
        for (int32_t i = 0; i < n_fft; ++i) {
            const int32_t wi = w ? w[i] : 1;
            for (int64_t p = offsets[i]; p < offsets[i + 1]; ++p) {
                const int64_t s = stripe_start(A[p], S0[i], D[i], j);
                for (int64_t b = s; b < s + k_over; ++b)
                    if (b >= 0 && b < n_f0) map[(int64_t)j * n_f0 + b] += wi;
            }
        }
    }
}

/*
 * a6, first half -- profile over spin-down: for every cell b, the largest
 * count over all rows and the smallest row that reaches it (candidates are
 * taken "for all the possible spin-down values", Sec. VIII).
 */
void fho_profile(const int32_t *map, int32_t n_fdot, int32_t n_f0,
                 int32_t *pcount, int32_t *prow)
{
    for (int32_t b = 0; b < n_f0; ++b) {
        int32_t best = map[b];
        int32_t bj = 0;
        for (int32_t j = 1; j < n_fdot; ++j) {
            const int32_t c = map[(int64_t)j * n_f0 + b];
            if (c > best) {
                best = c;
                bj = j;
            }
        }
        pcount[b] = best;
        prow[b] = bj;
    }
}

/*
 * a6, second half -- sub-band selection (Sec. VIII).  The band is cut into
 * sub-bands of W cells (the last one may be shorter).  In each sub-band, up
 * to top_k picks are taken greedily: the k-th pick is the best cell (largest
 * count, then smallest row, then smallest cell) whose distance to every
 * earlier pick is larger than excl cells; selection in the sub-band stops
 * when no such cell exists, when the best one has count < n_thr, or when it
 * lies closer than sep cells to an earlier pick.
 * Output slots (n_sb x top_k): cell, row, count; -1 in all three when empty.
 */
void fho_select(const int32_t *pcount, const int32_t *prow, int32_t n_f0,
                int32_t subband_cells, int32_t top_k, int32_t excl, int32_t sep,
                int32_t n_thr, int32_t *out_cell, int32_t *out_row, int32_t *out_count)
{
    const int32_t n_sb = (n_f0 + subband_cells - 1) / subband_cells;
    for (int32_t q = 0; q < n_sb; ++q) {
        const int32_t lo = q * subband_cells;
        const int32_t hi = (lo + subband_cells < n_f0) ? lo + subband_cells : n_f0;
        int32_t npick = 0;
        for (int32_t k = 0; k < top_k; ++k) {
            out_cell[(int64_t)q * top_k + k] = -1;
            out_row[(int64_t)q * top_k + k] = -1;
            out_count[(int64_t)q * top_k + k] = -1;
        }
        for (int32_t k = 0; k < top_k; ++k) {
            int32_t bb = -1;
            for (int32_t b = lo; b < hi; ++b) {
                int excluded = 0;
                for (int32_t m = 0; m < npick; ++m) {
                    const int32_t pb = out_cell[(int64_t)q * top_k + m];
                    const int32_t dist = b > pb ? b - pb : pb - b;
                    if (dist <= excl) excluded = 1;
                }
                if (excluded) continue;
                if (bb < 0 || pcount[b] > pcount[bb] ||
                    (pcount[b] == pcount[bb] && prow[b] < prow[bb]))
                    bb = b;   /* b ascends, so equal (count, row) keeps the smaller cell */
            }
            if (bb < 0) break;
            if (pcount[bb] < n_thr) break;
            int too_close = 0;
            for (int32_t m = 0; m < npick; ++m) {
                const int32_t pb = out_cell[(int64_t)q * top_k + m];
                const int32_t dist = bb > pb ? bb - pb : pb - bb;
                if (dist < sep) too_close = 1;
            }
            if (too_close) break;
            out_cell[(int64_t)q * top_k + npick] = bb;
            out_row[(int64_t)q * top_k + npick] = prow[bb];
            out_count[(int64_t)q * top_k + npick] = pcount[bb];
            ++npick;
        }
    }
}
