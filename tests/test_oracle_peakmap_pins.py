"""Pins of the oracle's peakmap construction and cleaning (Sec. "Peakmap",
Eq. pm, Eq. p0; Sec. "Removal of spectral wandering lines"; Sec. "Removal of
spectral lines of constant frequency"; App. "Robust statistic") against facts
that do not come from the oracle code.  CPU only."""
import math

import numpy as np
import pytest

from paper_1407_8333_gb300 import synth


@pytest.fixture(scope="module")
def pm():
    import oracle
    return oracle.peakmap


@pytest.fixture(scope="module")
def th():
    from oracle import theory
    return theory


def brute_select(s_p, s_ar, theta):
    """Eq. pm by pure-Python loops: ratio bin by bin in binary32, above the
    threshold and above both neighbours."""
    out = []
    th = np.float32(theta)
    for i in range(s_p.shape[0]):
        r = [np.float32(s_p[i, j]) / np.float32(s_ar[i, j]) for j in range(s_p.shape[1])]
        row = []
        for j in range(1, len(r) - 1):
            if r[j] > th and r[j] > r[j - 1] and r[j] > r[j + 1]:
                row.append(j)
        out.append(row)
    return out


def as_rows(offsets, bins):
    return [list(bins[offsets[i]:offsets[i + 1]]) for i in range(len(offsets) - 1)]


def test_selection_by_brute_force(pm):
    s = synth.spectra_case(11, 9, 57, wander_amp=20.0, wander_f=(50.001, 50.005),
                           const_lines=(50.003,), signal_lambda=6.0)
    o, b = pm.select_peaks(s.s_p, s.s_ar, 2.5)
    assert as_rows(o, b) == brute_select(s.s_p, s.s_ar, 2.5)


def test_selection_hand_cases(pm):
    one = np.ones((1, 9), dtype=np.float32)
    cases = [
        ([0, 1, 2, 3, 4, 5, 6, 7, 8], []),                 # monotone ramp: no maximum
        ([0, 0, 0, 9, 0, 0, 0, 0, 0], [3]),                # a spike
        ([0, 0, 0, 2, 0, 0, 0, 0, 0], []),                 # a spike below theta
        ([0, 0, 9, 9, 0, 0, 0, 0, 0], []),                 # a plateau is no strict maximum
        ([9, 0, 0, 0, 0, 0, 0, 0, 9], []),                 # edge bins have one neighbour
        ([0, 5, 0, 6, 0, 0, 7, 1, 0], [1, 3, 6]),          # maxima one bin apart
        ([0, 2.5, 0, 0, 0, 0, 0, 0, 0], []),               # R equal to theta is not above it
    ]
    for vals, want in cases:
        sp = np.array([vals], dtype=np.float32)
        o, b = pm.select_peaks(sp, one, 2.5)
        assert list(b) == want, vals
    # the ratio, not the periodogram, is thresholded: halving S_AR doubles R
    sp = np.array([[0, 0, 0, 2, 0, 0, 0, 0, 0]], dtype=np.float32)
    _, b = pm.select_peaks(sp, one * np.float32(0.5), 2.5)
    assert list(b) == [3]


@pytest.mark.parametrize("theta", [1.5, 2.5, 3.5])
def test_noise_peak_fraction_is_eq_p0(pm, th, theta):
    """Exponential equalised noise: the selected fraction of interior bins is
    p0 = e^-theta - e^-2theta + e^-3theta / 3 (Eq. p0) within 5 binomial sigma."""
    n_fft, n_bins = 120, 8192
    s = synth.spectra_case(12, n_fft, n_bins)
    o, _ = pm.select_peaks(s.s_p, s.s_ar, theta)
    m = n_fft * (n_bins - 2)
    p = th.p0(theta)
    assert abs(o[-1] - m * p) < 5.0 * math.sqrt(m * p * (1.0 - p))


def test_gross_histogram_noise_matches_E_H_and_sigma_H(pm, th):
    """The paper's example: FFTs of 8192 s overlapping by half, Delta t_H = 12 h,
    Delta f_H = 0.01 Hz: N = 2 Delta t_H Delta f_H = 864, E_H = N p0 = 65 and
    sigma_H = sqrt(N p0 (1 - p0)) = 7.8 at theta = 2.5.  Over the full cells of
    a noise-only peakmap the mean and spread of the gross counts agree."""
    n = th.gross_points(43200.0, 0.01, 8192.0)
    e_h, s_h = th.gross_noise(n, th.p0(2.5))
    assert n == pytest.approx(864.0)
    assert round(e_h) == 65 and round(s_h, 1) == 7.8
    s = synth.spectra_case(13, 2 * 211, 8192)           # 20 days, 1 Hz
    o, b = pm.select_peaks(s.s_p, s.s_ar, 2.5)
    n_th, n_fh = 19, 99
    hist = pm.gross_histogram(s.t, o, b, s.k0, s.t_fft, 0.0, 43200.0, n_th, 50.0, 0.01, n_fh)
    # cells whose FFT and bin counts are both whole: mean count 864 p0 per cell
    counts = hist[:, 1:-1].astype(np.float64)
    assert abs(counts.mean() - e_h) < 0.02 * e_h
    # spread: binomial plus the 10 / 11 FFTs and 81 / 82 bins a cell can hold
    assert 0.85 * s_h < counts.std() < 1.25 * s_h


def test_gross_veto_removes_a_wandering_line_cell_by_cell(pm, th):
    """A line 15 bins wide (8 peaks per FFT) drifting over 0.13 Hz in 20 days:
    with the threshold at E_H + 4.5 sigma_H only cells the line crosses are
    vetoed, and most of the line's peaks go."""
    s = synth.spectra_case(14, 2 * 211, 2048, wander_amp=40.0, wander_f=(50.05, 50.18),
                           wander_width=15)
    o, b = pm.select_peaks(s.s_p, s.s_ar, 2.5)
    t0, dt, n_th, f0, df, n_fh = 0.0, 43200.0, 40, 50.0, 0.01, 25
    hist = pm.gross_histogram(s.t, o, b, s.k0, s.t_fft, t0, dt, n_th, f0, df, n_fh)
    e_h, s_h = th.gross_noise(th.gross_points(dt, df, s.t_fft), th.p0(2.5))
    thr = int(e_h + 4.5 * s_h)
    o2, b2, h2 = pm.gross_veto(s.t, o, b, s.k0, s.t_fft, t0, dt, n_th, f0, df, n_fh, thr)
    assert np.array_equal(h2, hist)
    # brute force: a peak survives iff its cell (if on the grid) holds <= thr peaks
    want = []
    for i in range(len(o) - 1):
        row = []
        for q in range(o[i], o[i + 1]):
            f = (s.k0 + b[q]) / s.t_fft
            it, jf = math.floor((s.t[i] - t0) / dt), math.floor((f - f0) / df)
            if 0 <= it < n_th and 0 <= jf < n_fh and hist[it, jf] > thr:
                continue
            row.append(b[q])
        want.append(row)
    assert as_rows(o2, b2) == want
    line_cells = set()
    line_peaks = removed = 0
    kept = as_rows(o2, b2)
    rows = as_rows(o, b)
    for i in range(len(s.t)):
        if s.wander_bins[i] < 0:
            continue
        for q in range(0, 15, 2):
            bb = int(s.wander_bins[i] + q)
            f = (s.k0 + bb) / s.t_fft
            line_cells.add((math.floor(s.t[i] / dt), math.floor((f - f0) / df)))
            if bb in rows[i]:
                line_peaks += 1
                removed += bb not in kept[i]
    vetoed = {tuple(int(x) for x in c) for c in np.argwhere(hist > thr)}
    assert vetoed and vetoed <= line_cells
    assert removed >= 0.8 * line_peaks


def test_robust_statistics_hand_cases(pm):
    m1, m2 = pm.robust_stats([1, 2, 3, 4, 100])
    assert m1 == 3.0 and m2 == pytest.approx(1.0 / 0.6745, rel=0, abs=1e-15)
    m1, m2 = pm.robust_stats([1, 2, 3, 4])           # even count: mean of the middle pair
    assert m1 == 2.5 and m2 == pytest.approx(1.0 / 0.6745, rel=0, abs=1e-15)
    m1, m2 = pm.robust_stats([7, 7, 7, 7])
    assert (m1, m2) == (7.0, 0.0)


def test_robust_dispersion_is_the_normal_sigma(pm):
    """c = 0.6745 makes m2 the standard deviation of a normal law."""
    u = synth.uniform(15, 1, np.arange(400000)).reshape(2, -1)
    g = np.sqrt(-2.0 * np.log1p(-u[0])) * np.cos(2.0 * np.pi * u[1])
    m1, m2 = pm.robust_stats(3.0 + 2.0 * g)
    assert abs(m1 - 3.0) < 0.02 and abs(m2 - 2.0) < 0.02


def test_persistency_veto_removes_constant_lines(pm):
    lines = (50.01, 50.1, 50.2)
    s = synth.spectra_case(16, 300, 2048, const_lines=lines, const_amp=40.0, const_frac=0.8)
    o, b = pm.select_peaks(s.s_p, s.s_ar, 2.5)
    o2, b2, hist, m1, m2, thr = pm.persistency_veto(o, b, 2048, 6.0)
    assert np.array_equal(hist, np.bincount(b, minlength=2048))
    vetoed = set(np.nonzero(hist > thr)[0])
    assert vetoed == set(int(x) for x in s.const_bins)
    want = [[x for x in row if x not in vetoed] for row in as_rows(o, b)]
    assert as_rows(o2, b2) == want
    # the noise counts are binomial(300, p0-ish): median near 300 p0
    assert abs(m1 - 300 * 0.0755) < 3.0


def constant_line_case():
    """A peakmap (built by the oracle's selection) with constant lines at 50.1
    and 50.4 Hz in 80 % of 400 FFTs, for the frequency-Hough transform without
    Doppler correction (v = 0) on three spin-down rows around 0."""
    import oracle
    s = synth.spectra_case(17, 400, 4096, const_lines=(50.1, 50.4), const_amp=40.0,
                           const_frac=0.8)
    o, b = oracle.peakmap.select_peaks(s.s_p, s.s_ar, 2.5)
    freq = oracle.peakmap.peak_frequencies(b, s.k0, s.t_fft)
    inp = synth.Inputs(w=None, t=s.t, offsets=o, freq=freq, v=np.zeros((len(s.t), 3)),
                       sky=np.array([[1.0, 0.0, 0.0]]))
    t_obs = s.t[-1] - s.t[0] + s.t_fft
    step = 1.0 / (s.t_fft * t_obs)
    pp = dict(t_fft=s.t_fft, k_over=10, f0_min=s.k0 / s.t_fft, n_f0=4096 * 10, fdot_min=-step,
              fdot_step=step, n_fdot=3, t_ref=0.5 * (s.t[0] + s.t[-1]), subband_cells=4096 * 10,
              top_k=2, excl_cells=40, sep_cells=80, n_thr=0, p0=0.0755)
    return s, inp, pp


def test_constant_lines_found_by_the_transform_without_doppler(oracle_mod):
    """Sec. "Removal of spectral lines of constant frequency", third option: the
    transform on the uncorrected peakmap (v = 0) puts the constant lines at
    spin-down 0 as the two strongest candidates, at their own frequencies."""
    s, inp, pp = constant_line_case()
    o = oracle_mod.search(inp, pp)
    rows = o["row"][0, 0, :2]
    f0 = np.sort(o["f0"][0, 0, :2])
    assert list(rows) == [1, 1]                       # the fdot = 0 row
    assert np.all(np.abs(f0 - np.array([50.1, 50.4])) < 1.0 / s.t_fft)
    assert np.all(o["count"][0, 0, :2] > 0.7 * len(s.t))
