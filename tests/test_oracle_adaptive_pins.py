"""Pins of the oracle's adaptive map (Eq. ncountadap: n = sum_i w_i n_i) and of
its critical ratio, against facts that do not come from the weighted code path.

CPU only.  The weights are integers in fixed point (W = rint(w 2^F), binary64,
ties to even), so every map stays exact.
"""
import math

import numpy as np
import pytest

from paper_1407_8333_gb300 import synth


def _steps(oracle, inp, pp):
    kt = float(pp["k_over"]) * float(pp["t_fft"])
    r = oracle.doppler_factor(inp.v, inp.sky)
    A = oracle.positions(inp.offsets, inp.freq, r, pp["f0_min"], kt, pp["k_over"])
    S0, D = oracle.shift_tables(inp.t, pp["t_ref"], kt, pp["fdot_min"], pp["fdot_step"])
    return kt, A, S0, D


def _map(oracle, inp, pp, A, S0, D, W=None, direct=False):
    if direct:
        return oracle.hough_map_direct(inp.offsets, A, S0, D, pp["k_over"], pp["n_f0"],
                                       pp["n_fdot"], weights=W)
    return oracle.hough_map(inp.offsets, A, S0, D, pp["k_over"], pp["n_f0"], pp["n_fdot"],
                            weights=W)


@pytest.fixture(scope="module")
def case(oracle_mod):
    inp, pp = synth.random_case(31, n_fft=24, n_bins=48, n_fdot=17, n_dir=1, p=0.3)
    kt, A, S0, D = _steps(oracle_mod, inp, pp)
    return inp, pp, A[0], S0, D


def test_unit_weights_give_the_plain_map(oracle_mod, case):
    inp, pp, A, S0, D = case
    n = inp.t.shape[0]
    assert np.array_equal(_map(oracle_mod, inp, pp, A, S0, D, np.ones(n, np.int32)),
                          _map(oracle_mod, inp, pp, A, S0, D))


def test_constant_weight_scales_the_map(oracle_mod, case):
    """A weight common to all FFTs (the paper's beam-pattern factor of one sky
    position) multiplies every pixel by the same number (Sec. VI)."""
    inp, pp, A, S0, D = case
    n = inp.t.shape[0]
    plain = _map(oracle_mod, inp, pp, A, S0, D)
    assert np.array_equal(_map(oracle_mod, inp, pp, A, S0, D, np.full(n, 37, np.int32)),
                          37 * plain)


def test_map_is_linear_in_the_weights(oracle_mod, case):
    inp, pp, A, S0, D = case
    n = inp.t.shape[0]
    rng = np.random.default_rng(5)
    w1 = rng.integers(0, 1000, n).astype(np.int32)
    w2 = rng.integers(0, 1000, n).astype(np.int32)
    assert np.array_equal(_map(oracle_mod, inp, pp, A, S0, D, w1 + w2),
                          _map(oracle_mod, inp, pp, A, S0, D, w1)
                          + _map(oracle_mod, inp, pp, A, S0, D, w2))


def test_zero_weights_equal_deleting_those_ffts(oracle_mod, case):
    """w_i = 0 removes FFT i from the sum: the same map as the plain transform of
    the peakmap without FFT i's peaks (a different peakmap, built here)."""
    inp, pp, A, S0, D = case
    n = inp.t.shape[0]
    keep = np.ones(n, bool)
    keep[[1, 4, 5, 13, 22]] = False
    w = keep.astype(np.int32)
    counts = np.diff(inp.offsets)
    off2 = np.concatenate([[0], np.cumsum(np.where(keep, counts, 0))]).astype(np.int64)
    A2 = np.concatenate([A[inp.offsets[i]:inp.offsets[i + 1]] for i in range(n) if keep[i]])
    plain2 = oracle_mod.hough_map(off2, A2, S0, D, pp["k_over"], pp["n_f0"], pp["n_fdot"])
    assert np.array_equal(_map(oracle_mod, inp, pp, A, S0, D, w), plain2)


@pytest.mark.parametrize("seed", [41, 42])
def test_weighted_differential_equals_weighted_direct(oracle_mod, seed):
    inp, pp = synth.random_case(seed, n_fft=15, n_bins=30, n_fdot=9, n_dir=1, p=0.4)
    kt, A, S0, D = _steps(oracle_mod, inp, pp)
    w = np.random.default_rng(seed).integers(0, 5000, inp.t.shape[0]).astype(np.int32)
    assert np.array_equal(_map(oracle_mod, inp, pp, A[0], S0, D, w),
                          _map(oracle_mod, inp, pp, A[0], S0, D, w, direct=True))


def test_weighted_count_by_python_brute_force(oracle_mod):
    """Independent brute force: the weighted number count of one cell is the sum
    of the weights of the peaks whose stripe covers it."""
    inp, pp = synth.random_case(43, n_fft=8, n_bins=20, n_fdot=5, n_dir=1, p=0.5)
    kt, A, S0, D = _steps(oracle_mod, inp, pp)
    w = np.arange(1, inp.t.shape[0] + 1, dtype=np.int32) * 3
    m = _map(oracle_mod, inp, pp, A[0], S0, D, w)
    K = pp["k_over"]
    ref = np.zeros_like(m)
    for i in range(inp.t.shape[0]):
        for p in range(inp.offsets[i], inp.offsets[i + 1]):
            for j in range(pp["n_fdot"]):
                s = (int(A[0][p]) - (int(S0[i]) + j * int(D[i]))) >> 32
                for b in range(max(s, 0), min(s + K, pp["n_f0"])):
                    ref[j, b] += w[i]
    assert np.array_equal(m, ref)


def test_quantisation_rounds_half_to_even(oracle_mod):
    W = oracle_mod.quantize_weights(np.array([[0.25, 0.75, 1.25, 1.75, 0.0, 3.1]]), 1)
    assert W.tolist() == [[0, 2, 2, 4, 0, 6]]
    W = oracle_mod.quantize_weights(np.array([[1.0, 0.5]]), 8)
    assert W.tolist() == [[256, 128]]


@pytest.mark.parametrize("bad", [[-1.0, 1.0], [np.nan, 1.0], [np.inf, 1.0]])
def test_quantisation_rejects_bad_weights(oracle_mod, bad):
    with pytest.raises(ValueError):
        oracle_mod.quantize_weights(np.array([bad]), 4)


def test_quantisation_rejects_a_sum_of_2_30(oracle_mod):
    """Counts are int32 and a cell takes at most two stripes of one FFT, so each
    direction's weights must sum below 2^30."""
    with pytest.raises(ValueError):
        oracle_mod.quantize_weights(np.array([[2.0 ** 29, 2.0 ** 29]]), 0)
    oracle_mod.quantize_weights(np.array([[2.0 ** 29, 2.0 ** 29 - 1.0]]), 0)


def test_adaptive_cr_reduces_to_eq_cr_and_is_scale_free(oracle_mod):
    """Unit weights: S1 = S2 = N and the adaptive CR is Eq. cr operation for
    operation; a common factor c on all weights multiplies n, S1 by c and S2 by
    c^2, leaving the CR unchanged."""
    N, p0 = 3164, 0.04
    cnt = np.array([[[150, 130, -1]]])
    cell = np.zeros_like(cnt)
    row = np.zeros_like(cnt)
    _, _, cr_plain = oracle_mod.report(cell, row, cnt, 50.0, 81920.0, 0.0, 1e-12, N, p0)
    _, _, cr_unit = oracle_mod.report(cell, row, cnt, 50.0, 81920.0, 0.0, 1e-12, N, p0,
                                      s1=[N], s2=[N])
    assert np.array_equal(cr_plain.view(np.uint64), cr_unit.view(np.uint64))
    c = 256
    _, _, cr_c = oracle_mod.report(cell, row, np.where(cnt >= 0, c * cnt, -1), 50.0, 81920.0,
                                   0.0, 1e-12, N, p0, s1=[c * N], s2=[c * c * N])
    assert np.allclose(cr_c, cr_unit, rtol=1e-12, atol=0)
    assert cr_plain[0, 0, 0] == pytest.approx((150 - N * p0) / math.sqrt(N * p0 * (1 - p0)),
                                              rel=1e-15)


def test_search_with_unit_weights_equals_plain_search(oracle_mod):
    inp, pp = synth.random_case(44, n_fft=20, n_bins=40, n_fdot=11, n_dir=2, p=0.3)
    a = oracle_mod.search(inp, pp, want_maps=True)
    b = oracle_mod.search(inp, pp, want_maps=True, weights=np.ones((2, 20)), frac_bits=0)
    for k in ("maps", "pcount", "prow", "cell", "row", "count"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["cr"].view(np.uint64), b["cr"].view(np.uint64))


def test_stripe_overlap_by_brute_force(oracle_mod):
    """stripe_overlap (the count bound's per-FFT factor) against its definition
    evaluated pair by pair: the most positions of one FFT inside a half-open
    window of K cells."""
    inp, pp = synth.dense_case(45, dense_ffts=(1, 4), n_dense=9, spacing_bins=0.23, n_fft=7,
                               n_bins=30, n_fdot=9, n_dir=1, p=0.4)
    kt, A, S0, D = _steps(oracle_mod, inp, pp)
    c = oracle_mod.stripe_overlap(inp.offsets, A[0], pp["k_over"])
    width = pp["k_over"] << 32
    for i in range(inp.t.shape[0]):
        a = [int(x) for x in A[0][inp.offsets[i]:inp.offsets[i + 1]]]
        best = max([sum(1 for y in a if x <= y < x + width) for x in a] or [0])
        assert c[i] == best
    assert c[1] >= 4 and c[4] >= 4          # the dense FFTs put >= 4 stripes on a cell


def test_count_bound_holds_on_dense_off_grid_peaks(oracle_mod):
    """Dense off-grid peaks: a cell takes more than two stripes of one FFT, yet
    no weighted count of the direct map exceeds count_bound, and one FFT alone
    reaches more than 2 W on some cell (so 2 sum(W) would not be a bound)."""
    inp, pp = synth.dense_case(46, dense_ffts=(2,), n_dense=10, spacing_bins=0.25, n_fft=6,
                               n_bins=30, n_fdot=9, n_dir=1, p=0.4)
    kt, A, S0, D = _steps(oracle_mod, inp, pp)
    w = (np.arange(inp.t.shape[0], dtype=np.int32) % 5 + 1) * 1000
    m = _map(oracle_mod, inp, pp, A[0], S0, D, w, direct=True)
    assert m.max() <= oracle_mod.count_bound(inp.offsets, A[0], pp["k_over"], w)
    only = np.zeros_like(w)
    only[2] = w[2]
    m2 = _map(oracle_mod, inp, pp, A[0], S0, D, only, direct=True)
    assert m2.max() > 2 * w[2]


def test_search_refuses_weights_whose_count_bound_reaches_2_31(oracle_mod):
    """Weights summing below 2^30 are refused when dense peaks of one FFT could
    carry a count to 2^31 (the same rule as the library's fh_set_weights); the
    same peakmap with smaller weights is searched, and its map equals direct
    counting."""
    inp, pp = synth.dense_case(47, dense_ffts=(1,), n_dense=12, spacing_bins=0.2, n_fft=5,
                               n_bins=30, n_fdot=9, n_dir=1, p=0.4)
    kt, A, S0, D = _steps(oracle_mod, inp, pp)
    c = oracle_mod.stripe_overlap(inp.offsets, A[0], pp["k_over"])
    assert c[1] >= 5
    n = inp.t.shape[0]
    big = np.ones((1, n))
    big[0, 1] = float(2 ** 29 - 16)           # sum < 2^30, but c[1] W[1] >= 2^31
    with pytest.raises(ValueError):
        oracle_mod.search(inp, pp, weights=big, frac_bits=0)
    ok = np.ones((1, n))
    ok[0, 1] = float((2 ** 31 - 1 - 64) // int(c[1]))
    o = oracle_mod.search(inp, pp, weights=ok, frac_bits=0, want_maps=True)
    W = oracle_mod.quantize_weights(ok, 0)
    assert np.array_equal(o["maps"][0], _map(oracle_mod, inp, pp, A[0], S0, D,
                                             W[0].astype(np.int32), direct=True))
