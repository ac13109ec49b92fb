"""CPU oracle of peakmap construction and cleaning -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may use this module; the CUDA library never imports it and it never
imports the library.  Plain numpy, in the order the paper describes the steps:

* peak selection (Sec. "Peakmap", Eq. pm): R(i, j) = S_P(i, j) / S_AR(i, j) bin
  by bin (binary32, one IEEE division); a bin is a peak when R > theta and R is
  a local maximum, strictly above both neighbouring bins of the same FFT
  (the first and last bin of an FFT have one neighbour only and are never
  peaks);
* wandering-line veto (Sec. "Removal of spectral wandering lines"): the "gross
  histogram" counts the peaks of a low-resolution grid of Delta t_H x Delta f_H
  cells; every peak in a cell whose count is above the threshold is removed;
* constant-line veto by persistency (Sec. "Removal of spectral lines of
  constant frequency" with the robust statistic of App. "Robust statistic"):
  the number of FFTs with a peak in each frequency bin is histogrammed; with
  m1 = median and m2 = median(|x - m1|) / 0.6745 of those counts, every bin
  whose count exceeds m1 + k m2 loses all its peaks.

A peakmap here is binned: ``offsets`` (n_fft + 1, int64) and the band-relative
bin index of each peak (int32, ascending within an FFT); the frequency of bin b
is (k0 + b) / T_FFT (binary64).

Pins (``tests/test_oracle_peakmap_pins.py``): a pure-Python brute force of the
selection with hand cases (ramps, plateaus, edges, threshold ties); the
selected fraction of exponential noise against Eq. p0; the gross histogram of
noise against E_H = N p0 and sigma_H = sqrt(N p0 (1 - p0)) with the paper's
N = 2 Delta t_H Delta f_H = 864 example; an injected wandering line removed
cell by cell; hand-computed robust statistics and m2 -> sigma for normal
samples; injected constant lines removed bin by bin.
"""
from __future__ import annotations

import numpy as np

MAD_NORMAL = 0.6745   # App. "Robust statistic": m2 is the standard deviation of a normal law


def select_peaks(s_p, s_ar, theta: float):
    """Peaks of every FFT (Eq. pm): R > theta and a strict local maximum of R.

    s_p, s_ar: (n_fft, n_bins) spectra (binary32); theta is taken in binary32.
    Returns (offsets int64 (n_fft + 1), bins int32)."""
    s_p = np.ascontiguousarray(s_p, dtype=np.float32)
    s_ar = np.ascontiguousarray(s_ar, dtype=np.float32)
    n_fft, n_bins = s_p.shape
    with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
        # IEEE results for zero, tiny or non-finite spectra (inf, nan) are the
        # ratios the comparisons below see; no warning is raised for them
        r = s_p / s_ar                               # binary32, one rounding per bin
    th = np.float32(theta)
    sel = np.zeros((n_fft, n_bins), dtype=bool)
    if n_bins >= 3:
        mid = r[:, 1:-1]
        sel[:, 1:-1] = (mid > th) & (mid > r[:, :-2]) & (mid > r[:, 2:])
    counts = sel.sum(axis=1)
    offsets = np.zeros(n_fft + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    bins = np.nonzero(sel)[1].astype(np.int32)       # row-major: FFT by FFT, ascending bins
    return offsets, bins


def peak_frequencies(bins, k0: int, t_fft: float) -> np.ndarray:
    """Frequency of each peak's bin: (k0 + b) / T_FFT (binary64)."""
    return (np.float64(k0) + np.asarray(bins, dtype=np.float64)) / np.float64(t_fft)


def _gross_cells(t, offsets, bins, k0, t_fft, t0_h, dt_h, n_th, f0_h, df_h, n_fh):
    offsets = np.asarray(offsets, dtype=np.int64)
    n_fft = offsets.shape[0] - 1
    fft_of_peak = np.repeat(np.arange(n_fft), np.diff(offsets))
    it = np.floor((np.asarray(t, dtype=np.float64)[fft_of_peak] - t0_h) / dt_h)
    f = peak_frequencies(bins, k0, t_fft)
    jf = np.floor((f - f0_h) / df_h)
    inside = (it >= 0) & (it < n_th) & (jf >= 0) & (jf < n_fh)
    return it.astype(np.int64), jf.astype(np.int64), inside


def gross_histogram(t, offsets, bins, k0: int, t_fft: float, t0_h: float, dt_h: float,
                    n_th: int, f0_h: float, df_h: float, n_fh: int) -> np.ndarray:
    """The "gross histogram": peaks per (time cell, frequency cell), time cell
    floor((t_i - t0_h) / Delta t_H) of the FFT's start time, frequency cell
    floor((f - f0_h) / Delta f_H) of the peak's frequency; peaks outside the
    n_th x n_fh grid are not counted.  Returns int64 (n_th, n_fh)."""
    it, jf, inside = _gross_cells(t, offsets, bins, k0, t_fft, t0_h, dt_h, n_th, f0_h, df_h,
                                  n_fh)
    hist = np.zeros((n_th, n_fh), dtype=np.int64)
    np.add.at(hist, (it[inside], jf[inside]), 1)
    return hist


def filter_peaks(offsets, bins, keep):
    """The peakmap without the peaks where ``keep`` is False (order kept)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    keep = np.asarray(keep, dtype=bool)
    n_fft = offsets.shape[0] - 1
    fft_of_peak = np.repeat(np.arange(n_fft), np.diff(offsets))
    counts = np.bincount(fft_of_peak[keep], minlength=n_fft)
    out = np.zeros(n_fft + 1, dtype=np.int64)
    np.cumsum(counts, out=out[1:])
    return out, np.asarray(bins, dtype=np.int32)[keep]


def gross_veto(t, offsets, bins, k0: int, t_fft: float, t0_h: float, dt_h: float, n_th: int,
               f0_h: float, df_h: float, n_fh: int, threshold: int):
    """Wandering-line veto: remove every peak whose gross cell holds more than
    ``threshold`` peaks.  Returns (offsets, bins, hist)."""
    hist = gross_histogram(t, offsets, bins, k0, t_fft, t0_h, dt_h, n_th, f0_h, df_h, n_fh)
    it, jf, inside = _gross_cells(t, offsets, bins, k0, t_fft, t0_h, dt_h, n_th, f0_h, df_h,
                                  n_fh)
    keep = np.ones(it.shape[0], dtype=bool)
    keep[inside] = hist[it[inside], jf[inside]] <= threshold
    o, b = filter_peaks(offsets, bins, keep)
    return o, b, hist


def robust_stats(x):
    """App. "Robust statistic": m1 = median(x), m2 = median(|x - m1|) / c with
    c = 0.6745 (binary64; the median of an even count is the mean of the two
    middle values)."""
    x = np.asarray(x, dtype=np.float64)
    m1 = float(np.median(x))
    m2 = float(np.median(np.abs(x - m1))) / MAD_NORMAL
    return m1, m2


def persistency_veto(offsets, bins, n_bins: int, k_sigma: float):
    """Constant-line veto: count the FFTs with a peak in each bin, take the
    robust statistics of those counts and remove every peak of the bins whose
    count is above m1 + k m2.  Returns (offsets, bins, hist, m1, m2, thr)."""
    bins = np.asarray(bins, dtype=np.int32)
    hist = np.bincount(bins, minlength=n_bins).astype(np.int64)
    m1, m2 = robust_stats(hist)
    thr = m1 + k_sigma * m2
    vetoed = hist > thr
    o, b = filter_peaks(offsets, bins, ~vetoed[bins])
    return o, b, hist, m1, m2, thr
