"""Peakmap construction and cleaning on the GPU, through the C ABI, against the
oracle (Sec. "Peakmap", Eq. pm; Sec. "Removal of spectral wandering lines";
Sec. "Removal of spectral lines of constant frequency"; App. "Robust
statistic").  Offsets, bins, histograms and the robust statistics bit for bit;
frequencies bit for bit (one binary64 division each)."""
import numpy as np
import pytest

from paper_1407_8333_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_8333_gb300 import build, fh as fhmod
    build.build()
    fhmod.load()
    return fhmod


@pytest.fixture(scope="module")
def pm():
    import oracle
    return oracle.peakmap


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(x):
    return x.cpu().numpy()


def gpu_select(fh, s, theta):
    o, b, f = fh.fh_peakmap_select(dev(s.s_p), dev(s.s_ar), theta, s.k0, s.t_fft)
    return host(o), host(b), host(f)


def check_select(fh, pm, s, theta):
    o, b, f = gpu_select(fh, s, theta)
    wo, wb = pm.select_peaks(s.s_p, s.s_ar, theta)
    assert np.array_equal(o, wo)
    assert np.array_equal(b, wb)
    assert np.array_equal(f.view(np.uint64), pm.peak_frequencies(wb, s.k0, s.t_fft).view(np.uint64))
    return o, b


@pytest.mark.parametrize("n_bins", [1, 2, 3, 31, 4096, 2 * 4096 + 777])
def test_select_matches_oracle(fh, pm, n_bins):
    """Segments of 4096 bins, a ragged last one, and the degenerate widths."""
    s = synth.spectra_case(21 + n_bins, 37, n_bins, wander_amp=30.0,
                           wander_f=(50.0 + 5 / 8192, 50.0 + max(6, n_bins - 9) / 8192),
                           wander_width=5, const_lines=(50.0 + (n_bins // 3) / 8192,),
                           signal_lambda=5.0)
    for theta in (1.0, 2.5, 4.0):
        check_select(fh, pm, s, theta)


def test_select_special_values_and_pitch(fh, pm):
    """Zero, infinite and NaN spectra divide as IEEE binary32 on both sides; a
    row pitch wider than the band is honoured."""
    import torch
    s = synth.spectra_case(30, 11, 300)
    sp, sa = s.s_p.copy(), s.s_ar.copy()
    sp[0, 10] = np.inf
    sa[1, 20] = 0.0
    sp[2, 30] = np.nan
    sa[3, 40] = np.inf
    sp[4, 50] = 1e-40          # subnormal
    sa[5, 60] = 1e-42
    sp[6, 70:73] = [3.0, 3.0, 2.0]
    wo, wb = pm.select_peaks(sp, sa, 2.5)
    wide_p = np.zeros((11, 333), np.float32)
    wide_a = np.ones((11, 333), np.float32)
    wide_p[:, :300], wide_a[:, :300] = sp, sa
    tp, ta = dev(wide_p)[:, :300], dev(wide_a)[:, :300]
    o, b, f = fh.fh_peakmap_select(tp, ta, 2.5, s.k0, s.t_fft)
    assert np.array_equal(host(o), wo) and np.array_equal(host(b), wb)
    torch.cuda.synchronize()


def test_select_capacity_error(fh, pm):
    s = synth.spectra_case(31, 5, 500)
    _, wb = pm.select_peaks(s.s_p, s.s_ar, 2.5)
    with pytest.raises(fh.FHError) as ei:
        fh.fh_peakmap_select(dev(s.s_p), dev(s.s_ar), 2.5, s.k0, s.t_fft, capacity=len(wb) - 1)
    assert ei.value.code == fh.FH_ERR_CAPACITY


def test_gross_veto_matches_oracle(fh, pm):
    s = synth.spectra_case(32, 2 * 211, 2048, wander_amp=40.0, wander_f=(50.05, 50.18),
                           wander_width=15)
    o, b = check_select(fh, pm, s, 2.5)
    grid = (0.0, 43200.0, 40, 50.0, 0.01, 25)
    for thr in (60, 90, 10 ** 6):
        wo, wb, wh = pm.gross_veto(s.t, o, b, s.k0, s.t_fft, *grid, thr)
        go, gb, gf, gh = fh.fh_peakmap_gross_veto(dev(s.t), dev(o), dev(b), s.k0, s.t_fft,
                                                  *grid, thr)
        assert np.array_equal(host(gh), wh)
        assert np.array_equal(host(go), wo) and np.array_equal(host(gb), wb)
        assert np.array_equal(host(gf), pm.peak_frequencies(wb, s.k0, s.t_fft))
    # a grid that covers only part of the peakmap: peaks off it are kept
    grid2 = (86400.0, 43200.0, 7, 50.03, 0.01, 6)
    wo, wb, wh = pm.gross_veto(s.t, o, b, s.k0, s.t_fft, *grid2, 70)
    go, gb, _, gh = fh.fh_peakmap_gross_veto(dev(s.t), dev(o), dev(b), s.k0, s.t_fft, *grid2, 70)
    assert np.array_equal(host(gh), wh)
    assert np.array_equal(host(go), wo) and np.array_equal(host(gb), wb)


@pytest.mark.parametrize("n_bins", [2048, 2047])
def test_persistency_veto_matches_oracle(fh, pm, n_bins):
    """Even and odd bin counts (median of a pair vs a single middle value)."""
    s = synth.spectra_case(33 + n_bins, 300, n_bins, const_lines=(50.01, 50.1, 50.2),
                           const_amp=40.0, const_frac=0.8)
    o, b = check_select(fh, pm, s, 2.5)
    for k in (2.0, 6.0):
        wo, wb, wh, m1, m2, thr = pm.persistency_veto(o, b, n_bins, k)
        go, gb, gf, gh, st = fh.fh_peakmap_persistency_veto(dev(o), dev(b), n_bins, k, s.k0,
                                                            s.t_fft)
        assert np.array_equal(host(gh), wh)
        assert st == (m1, m2, thr)
        assert np.array_equal(host(go), wo) and np.array_equal(host(gb), wb)
        assert np.array_equal(host(gf), pm.peak_frequencies(wb, s.k0, s.t_fft))


def test_robust_statistics_hand_case_on_device(fh):
    """Counts 0, 1, 1, 2, 9 (one FFT per peak): m1 = 1, |x - 1| = 1, 0, 0, 1, 8,
    m2 = 1 / 0.6745; with k = 5 the bin of 9 (> 1 + 5 / 0.6745 = 8.41) goes."""
    counts = [0, 1, 1, 2, 9]
    bins = np.concatenate([np.full(c, j, np.int32) for j, c in enumerate(counts)])
    offsets = np.arange(len(bins) + 1, dtype=np.int64)     # one peak per FFT
    go, gb, _, gh, st = fh.fh_peakmap_persistency_veto(dev(offsets), dev(bins), 5, 5.0, 0, 1.0)
    assert list(host(gh)) == counts
    assert st == (1.0, 1.0 / 0.6745, 1.0 + 5.0 * (1.0 / 0.6745))
    assert list(host(gb)) == [1, 2, 3, 3]


def test_cleaning_argument_and_csr_errors(fh):
    t = np.arange(4, dtype=np.float64)
    bins = np.array([1, 2, 3, 4], np.int32)
    bad = np.array([0, 3, 2, 4, 4], np.int64)             # decreasing offsets
    with pytest.raises(fh.FHError) as ei:
        fh.fh_peakmap_gross_veto(dev(t), dev(bad), dev(bins), 0, 1.0, 0.0, 1.0, 2, 0.0, 1.0, 2, 1)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG
    off = np.array([0, 1, 2, 3, 4], np.int64)
    with pytest.raises(fh.FHError) as ei:                  # bin 4 outside a 4-bin band
        fh.fh_peakmap_persistency_veto(dev(off), dev(bins), 4, 3.0, 0, 1.0)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG
    with pytest.raises(fh.FHError) as ei:                  # empty gross grid
        fh.fh_peakmap_gross_veto(dev(t), dev(off), dev(bins), 0, 1.0, 0.0, 1.0, 0, 0.0, 1.0, 2, 1)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG


def test_full_size_pipeline_matches_oracle(fh, pm):
    """The benchmark's peakmap workload: 3164 FFTs of 8192 s overlapping by half
    (150 days) x 8192 bins (1 Hz at 50 Hz), a signal track, a wandering line and
    two constant lines; selection, gross veto (12 h x 0.01 Hz, threshold 100) and
    persistency veto (k = 5), each compared in full."""
    s = synth.peakmap_workload()
    p = synth.PEAKMAP_PARAMS
    o, b = check_select(fh, pm, s, p["theta"])
    grid = (0.0, p["dt_h"], p["n_th"], p["f0_h"], p["df_h"], p["n_fh"])
    wo, wb, wh = pm.gross_veto(s.t, o, b, s.k0, s.t_fft, *grid, p["gross_thr"])
    go, gb, _, gh = fh.fh_peakmap_gross_veto(dev(s.t), dev(o), dev(b), s.k0, s.t_fft, *grid,
                                             p["gross_thr"])
    assert np.array_equal(host(gh), wh)
    assert np.array_equal(host(go), wo) and np.array_equal(host(gb), wb)
    wo2, wb2, wh2, m1, m2, thr = pm.persistency_veto(wo, wb, s.s_p.shape[1], p["k_sigma"])
    go2, gb2, _, gh2, st = fh.fh_peakmap_persistency_veto(go, gb, s.s_p.shape[1], p["k_sigma"],
                                                          s.k0, s.t_fft)
    assert np.array_equal(host(gh2), wh2) and st == (m1, m2, thr)
    assert np.array_equal(host(go2), wo2) and np.array_equal(host(gb2), wb2)
    # the disturbances are what the vetoes removed
    assert set(np.nonzero(wh2 > thr)[0]) == set(int(x) for x in s.const_bins)
    assert (wh > p["gross_thr"]).any()


def test_select_asynchronous_form(fh, pm):
    """With preallocated outputs the call does not synchronise; the total is
    offsets[n_fft] and peaks beyond the capacity are counted, not written;
    with or without a caller's workspace."""
    import torch
    s = synth.spectra_case(34, 23, 5000, wander_amp=30.0, wander_f=(50.05, 50.3), wander_width=7)
    wo, wb = pm.select_peaks(s.s_p, s.s_ar, 2.5)
    for cap in (len(wb) + 5, len(wb) // 2):
        out = (torch.empty(24, dtype=torch.int64, device="cuda"),
               torch.full((cap,), -1, dtype=torch.int32, device="cuda"),
               torch.empty(cap, dtype=torch.float64, device="cuda"))
        ws = torch.empty(fh.fh_peakmap_select_workspace(23, 5000), dtype=torch.uint8,
                         device="cuda") if cap % 2 else None
        o, b, f = fh.fh_peakmap_select(dev(s.s_p), dev(s.s_ar), 2.5, s.k0, s.t_fft, out=out,
                                       workspace=ws)
        torch.cuda.synchronize()
        assert np.array_equal(host(o), wo)
        k = min(cap, len(wb))
        assert np.array_equal(host(b)[:k], wb[:k])
        assert np.all(host(b)[k:] == -1)
        assert np.array_equal(host(f)[:k], pm.peak_frequencies(wb[:k], s.k0, s.t_fft))


def test_frequencies_for_a_t_fft_that_is_not_a_power_of_two(fh, pm):
    """A power-of-two T_FFT takes an exact multiply, any other the division;
    both give the IEEE quotient (k0 + b) / T_FFT, bit for bit."""
    for t_fft in (1800.0, 1024.0, 3.0):
        s = synth.spectra_case(35, 9, 700, t_fft=t_fft, f_lo=20.0)
        check_select(fh, pm, s, 2.0)
        o, b = pm.select_peaks(s.s_p, s.s_ar, 2.0)
        go, gb, gf, _ = fh.fh_peakmap_gross_veto(dev(s.t), dev(o), dev(b), s.k0, s.t_fft,
                                                 0.0, 5000.0, 4, 20.0, 0.05, 10, 3)
        wo, wb, _ = pm.gross_veto(s.t, o, b, s.k0, s.t_fft, 0.0, 5000.0, 4, 20.0, 0.05, 10, 3)
        assert np.array_equal(host(gb), wb)
        assert np.array_equal(host(gf).view(np.uint64),
                              pm.peak_frequencies(wb, s.k0, s.t_fft).view(np.uint64))


def test_select_captured_in_a_cuda_graph(fh, pm):
    """The asynchronous selection with a workspace allocates nothing, so it can
    be captured once and replayed; every replay gives the oracle's peakmap."""
    import torch
    s = synth.spectra_case(36, 40, 9000, wander_amp=30.0, wander_f=(50.1, 50.6), wander_width=9)
    wo, wb = pm.select_peaks(s.s_p, s.s_ar, 2.5)
    sp, sa = dev(s.s_p), dev(s.s_ar)
    cap = len(wb) + 64
    out = (torch.empty(41, dtype=torch.int64, device="cuda"),
           torch.empty(cap, dtype=torch.int32, device="cuda"),
           torch.empty(cap, dtype=torch.float64, device="cuda"))
    ws = torch.empty(fh.fh_peakmap_select_workspace(40, 9000), dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        fh.fh_peakmap_select(sp, sa, 2.5, s.k0, s.t_fft, out=out, workspace=ws, stream=st)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        fh.fh_peakmap_select(sp, sa, 2.5, s.k0, s.t_fft, out=out, workspace=ws, stream=st)
    for rep in range(3):
        out[0].fill_(-1)
        out[1].fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(host(out[0]), wo)
        assert np.array_equal(host(out[1])[:len(wb)], wb)
        assert np.array_equal(host(out[2])[:len(wb)], pm.peak_frequencies(wb, s.k0, s.t_fft))


def test_constant_lines_by_the_transform_without_doppler(fh, oracle_mod):
    """The third constant-line method (the transform at v = 0 near fdot = 0) is
    the library's ordinary path with zero velocities: its candidates equal the
    oracle's, the lines at spin-down 0."""
    import torch
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_peakmap_pins import constant_line_case
    s, inp, pp = constant_line_case()
    plan = fh.fh_create_plan(fh.make_desc(pp, inp.t.shape[0], 1, inp.n_peaks))
    try:
        args = [torch.from_numpy(np.ascontiguousarray(x)).cuda()
                for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        fh.fh_correct_doppler(plan, *args)
        fh.fh_transform(plan, 0, 1)
        cand = fh.fh_select_candidates(plan, 0, 1)
    finally:
        fh.fh_destroy_plan(plan)
    o = oracle_mod.search(inp, pp)
    for k in ("row", "cell", "count"):
        assert np.array_equal(cand[k][:2].astype(np.int64), o[k][0, 0, :2].astype(np.int64)), k
    assert list(cand["row"][:2]) == [1, 1]
