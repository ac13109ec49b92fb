"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results -- fixed-point positions, Hough maps, profiles, candidate
cells/rows/counts -- must match bit for bit.  The binary64 Doppler factors
must match bit for bit too (same IEEE operations in the same order, no FMA
on either side).  Reporting columns (f0, fdot, CR) are compared to 1e-12
relative, the tolerance stated for them.
"""
import math

import numpy as np
import pytest

from paper_1407_8333_gb300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12


@pytest.fixture(scope="module")
def fh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_8333_gb300 import build, fh as fhmod
    build.build()
    fhmod.load()
    return fhmod


def run_gpu(fh, inp, pp, mode=0, schedule=0, tile=0, warps=0, maps=True, device_inputs=True,
            autotune=False, checks=None, pinned=False):
    import torch
    n_fft = inp.t.shape[0]
    n_peaks = inp.n_peaks
    n_dir = inp.sky.shape[0]
    desc = fh.make_desc(pp, max(1, n_fft), n_dir, max(1, n_peaks), mode=mode, schedule=schedule,
                        tile_cells=tile, block_warps=warps)
    plan = fh.fh_create_plan(desc)
    try:
        if checks is not None:
            fh.fh_plan_set_input_checks(plan, checks)
        if device_inputs:
            args = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        elif pinned:
            # page-locked host arrays (read in place by the kernels for one direction)
            args = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
                    for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        else:
            args = [inp.t, inp.offsets, inp.freq, inp.v, inp.sky]
        r = torch.empty((n_dir, max(1, n_fft)), dtype=torch.float64, device="cuda")
        A = torch.empty((n_dir, max(1, n_peaks)), dtype=torch.int64, device="cuda")
        fh.fh_correct_doppler(plan, *args, out_r=r if n_fft else None,
                              out_A=A if n_peaks else None, n_peaks=n_peaks)
        if autotune:
            fh.fh_autotune(plan, 0, n_dir)
        m = (torch.full((n_dir, pp["n_fdot"], pp["n_f0"]), -7, dtype=torch.int32, device="cuda")
             if maps else None)
        fh.fh_transform(plan, 0, n_dir, m)
        prof = torch.empty((n_dir, pp["n_f0"]), dtype=torch.int64, device="cuda")
        fh.fh_copy_profile(plan, 0, n_dir, prof)
        cand = fh.fh_select_candidates(plan, 0, n_dir)
        torch.cuda.synchronize()
        out = dict(r=r.cpu().numpy()[:, :n_fft], A=A.cpu().numpy()[:, :n_peaks],
                   prof=prof.cpu().numpy().view(np.uint64), cand=cand,
                   launches=fh.fh_plan_launches(plan))
        if maps:
            out["maps"] = m.cpu().numpy()
        return out
    finally:
        fh.fh_destroy_plan(plan)


def oracle_profile_keys(pc, pr):
    return (pc.astype(np.uint64) << np.uint64(32)) | (np.uint64(0xFFFFFFFF) - pr.astype(np.uint64))


def compare(g, o, pp, n_fft, maps=True):
    assert np.array_equal(g["r"].view(np.uint64), o["r"].view(np.uint64))
    assert np.array_equal(g["A"], o["A"])
    if maps:
        assert np.array_equal(g["maps"], o["maps"])
    assert np.array_equal(g["prof"], oracle_profile_keys(o["pcount"], o["prow"]))
    n_dir = o["cell"].shape[0]
    c = g["cand"].reshape(n_dir, -1, pp["top_k"])
    assert np.array_equal(c["cell"], o["cell"])
    assert np.array_equal(c["row"], o["row"])
    assert np.array_equal(c["count"], o["count"])
    assert np.array_equal(c["dir"], np.broadcast_to(np.arange(n_dir)[:, None, None], c.shape))
    for k, ok in (("f0", "f0"), ("fdot", "fdot"), ("cr", "cr")):
        a, b = c[k], o[ok]
        same = (a == b) | (np.isnan(a) & np.isnan(b))
        close = np.abs(a - b) <= REL_TOL * np.maximum(np.abs(b), 1e-300)
        assert np.all(same | close), k


# ---------------------------------------------------------------- small randomised cases
CASES = [
    # seed, n_fft, n_bins, K, n_fdot, n_dir, tile, warps
    (1, 20, 40, 10, 7, 3, 96, 4),
    (2, 33, 57, 10, 45, 2, 100, 8),      # two slabs, ragged rows, ragged tile
    (3, 17, 64, 3, 33, 2, 64, 32),
    (4, 9, 31, 1, 5, 4, 32, 16),          # K = 1
    (5, 40, 128, 10, 70, 1, 0, 0),        # library default tile (single tile)
    (6, 64, 200, 7, 64, 2, 160, 8),
    (7, 14, 340, 10, 40, 2, 32, 8),       # 107 tiles: two passes of the window pre-pass
]


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("case", CASES)
def test_random_cases_bit_exact(fh, oracle_mod, mode, case):
    seed, n_fft, n_bins, K, n_fdot, n_dir, tile, warps = case
    inp, pp = synth.random_case(seed, n_fft=n_fft, n_bins=n_bins, k_over=K, n_fdot=n_fdot,
                                n_dir=n_dir, p=0.3, subband_bins=7, top_k=3,
                                excl_cells=2 * K, sep_cells=4 * K)
    o = oracle_mod.search(inp, pp, want_maps=True)
    g = run_gpu(fh, inp, pp, mode=mode, tile=tile, warps=warps)
    compare(g, o, pp, n_fft)


@pytest.mark.parametrize("schedule", [0, 1])
def test_schedules_agree_and_host_inputs(fh, oracle_mod, schedule):
    inp, pp = synth.random_case(8, n_fft=25, n_bins=90, k_over=10, n_fdot=40, n_dir=5, p=0.25)
    o = oracle_mod.search(inp, pp, want_maps=True)
    g = run_gpu(fh, inp, pp, schedule=schedule, tile=128, warps=8, device_inputs=False)
    compare(g, o, pp, 25)


def test_padded_rows_get_K_cells_per_peak(fh):
    """Invariant on the GPU map itself: with every stripe inside the map, each
    row of each direction sums to K * n_peaks (exact integer)."""
    inp, pp = synth.random_case(9, n_fft=50, n_bins=60, k_over=10, n_fdot=37, n_dir=3,
                                pad_bins=40, p=0.3)
    g = run_gpu(fh, inp, pp, tile=256)
    assert np.all(g["maps"].sum(axis=2, dtype=np.int64) == 10 * inp.n_peaks)


# ---------------------------------------------------------------- edge cases
def test_empty_peakmap(fh, oracle_mod):
    inp, pp = synth.random_case(10, n_fft=6, n_bins=20, p=0.0, n_dir=2)
    pp = dict(pp, p0=0.05)
    assert inp.n_peaks == 0
    o = oracle_mod.search(inp, pp, want_maps=True)
    g = run_gpu(fh, inp, pp, tile=64)
    assert not g["maps"].any()
    compare(g, o, pp, 6)


def test_single_fft_single_row(fh, oracle_mod):
    inp, pp = synth.random_case(11, n_fft=1, n_bins=50, n_fdot=1, n_dir=1, p=0.5, top_k=5,
                                excl_cells=0, sep_cells=0)
    o = oracle_mod.search(inp, pp, want_maps=True)
    g = run_gpu(fh, inp, pp, tile=64)
    compare(g, o, pp, 1)


def test_peaks_outside_band_are_clipped(fh, oracle_mod):
    """Map narrower than the supplied peaks: stripes crossing or beyond both
    edges are clipped exactly as the oracle clips them."""
    inp, pp = synth.random_case(12, n_fft=30, n_bins=40, margin=30, n_fdot=9, n_dir=2, p=0.4)
    pp = dict(pp, f0_min=pp["f0_min"] + 10 / pp["t_fft"], n_f0=pp["n_f0"] - 200)
    o = oracle_mod.search(inp, pp, want_maps=True)
    g = run_gpu(fh, inp, pp, tile=64, mode=1)
    compare(g, o, pp, 30)
    g2 = run_gpu(fh, inp, pp, tile=64, mode=2)
    compare(g2, o, pp, 30)


def test_selection_threshold_and_tiny_subbands(fh, oracle_mod):
    inp, pp = synth.random_case(13, n_fft=40, n_bins=30, n_fdot=11, n_dir=2, p=0.3,
                                subband_bins=1, top_k=4, excl_cells=3, sep_cells=5)
    pp = dict(pp, n_thr=14)
    o = oracle_mod.search(inp, pp, want_maps=True)
    g = run_gpu(fh, inp, pp, tile=96)
    compare(g, o, pp, 40)


def test_no_motion_closed_form_on_gpu(fh):
    """v = 0: the corrected position of a peak at FFT bin k (counted from
    f0_min) is exactly a = K k + (1 - K)/2, so its stripe starts at cell
    K k + floor((1-K)/2) (Eq. due; adjacent bins tile the f0 axis).  Read back
    through out_A."""
    inp, pp = synth.random_case(14, n_fft=12, n_bins=30, n_fdot=5, n_dir=1, off_grid=False,
                                doppler=False, p=0.5)
    g = run_gpu(fh, inp, pp, tile=64)
    K = pp["k_over"]
    k = np.rint(inp.freq * pp["t_fft"]).astype(np.int64) - int(round(pp["f0_min"] * pp["t_fft"]))
    assert np.array_equal(g["A"][0] >> 32, K * k + (1 - K) // 2)
    assert np.all((g["A"][0] & 0xFFFFFFFF) == (0 if K % 2 == 1 else 1 << 31))


# ---------------------------------------------------------------- invalid inputs
def test_host_input_errors(fh):
    inp, pp = synth.random_case(15, n_fft=10, n_bins=20, n_dir=1, p=0.5)
    desc = fh.make_desc(pp, 10, 1, inp.n_peaks)
    plan = fh.fh_create_plan(desc)
    try:
        f = inp.freq.copy()
        a, b = int(inp.offsets[2]), int(inp.offsets[2]) + 1
        f[a], f[b] = f[b], f[a]
        with pytest.raises(fh.FHError) as ei:
            fh.fh_correct_doppler(plan, inp.t, inp.offsets, f, inp.v, inp.sky)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        f = inp.freq.copy()
        f[3] = np.nan
        with pytest.raises(fh.FHError) as ei:
            fh.fh_correct_doppler(plan, inp.t, inp.offsets, f, inp.v, inp.sky)
        assert ei.value.code == fh.FH_ERR_INVALID_ARG
        # the edges of the host screen: +inf, 0, a negative value, and each of
        # them as the first or the last peak of an FFT
        first, last = int(inp.offsets[4]), int(inp.offsets[5]) - 1
        for where in (first, last):
            for bad_value in (np.inf, 0.0, -1.0, -0.0):
                f = inp.freq.copy()
                f[where] = bad_value
                with pytest.raises(fh.FHError) as ei:
                    fh.fh_correct_doppler(plan, inp.t, inp.offsets, f, inp.v, inp.sky)
                assert ei.value.code in (fh.FH_ERR_INVALID_ARG, fh.FH_ERR_UNSORTED), \
                    (where, bad_value)
        # equal neighbours are not strictly ascending
        f = inp.freq.copy()
        f[first + 1] = f[first]
        with pytest.raises(fh.FHError) as ei:
            fh.fh_correct_doppler(plan, inp.t, inp.offsets, f, inp.v, inp.sky)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        t = inp.t.copy()
        t[4] = t[3]
        with pytest.raises(fh.FHError) as ei:
            fh.fh_correct_doppler(plan, t, inp.offsets, inp.freq, inp.v, inp.sky)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        with pytest.raises(fh.FHError) as ei:      # transform before any correction
            fh.fh_transform(plan, 0, 1)
        assert ei.value.code == fh.FH_ERR_INVALID_ARG
    finally:
        fh.fh_destroy_plan(plan)
    bad = dict(pp, f0_min=pp["f0_min"] - 1e5)      # positions beyond 2^28 cells
    plan = fh.fh_create_plan(fh.make_desc(bad, 10, 1, inp.n_peaks))
    try:
        with pytest.raises(fh.FHError) as ei:
            fh.fh_correct_doppler(plan, inp.t, inp.offsets, inp.freq, inp.v, inp.sky)
        assert ei.value.code == fh.FH_ERR_RANGE
    finally:
        fh.fh_destroy_plan(plan)


def test_device_input_errors_are_reported_not_faulted(fh):
    """Unsorted frequencies and a broken CSR in DEVICE memory: the kernels clamp
    the offsets into a valid CSR (every read stays inside the arrays) and the
    device-side checks report the problem at the next synchronising call."""
    import torch
    inp, pp = synth.random_case(16, n_fft=10, n_bins=20, n_dir=1, p=0.5)
    plan = fh.fh_create_plan(fh.make_desc(pp, 10, 1, inp.n_peaks))
    try:
        f = inp.freq.copy()
        a = int(inp.offsets[3])
        f[a], f[a + 1] = f[a + 1], f[a]
        dev = lambda x: torch.from_numpy(x).cuda()
        fh.fh_correct_doppler(plan, dev(inp.t), dev(inp.offsets), dev(f), dev(inp.v), dev(inp.sky))
        fh.fh_transform(plan, 0, 1)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_select_candidates(plan, 0, 1)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        off = inp.offsets.copy()
        off[5] = inp.n_peaks + 1000          # out of range
        off[6] = -3                          # negative and decreasing
        fh.fh_correct_doppler(plan, dev(inp.t), dev(off), dev(inp.freq), dev(inp.v), dev(inp.sky),
                              n_peaks=inp.n_peaks)
        fh.fh_transform(plan, 0, 1)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_sync(plan)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        # every FFT's frequencies in descending order, and a NaN: the peak
        # windows can hold anything, so the transform must take its clamped
        # walk (every update inside the tile's counters)
        f = inp.freq.copy()
        for i in range(inp.t.shape[0]):
            a, b = int(inp.offsets[i]), int(inp.offsets[i + 1])
            f[a:b] = f[a:b][::-1]
        f[int(inp.offsets[2])] = np.nan
        fh.fh_correct_doppler(plan, dev(inp.t), dev(inp.offsets), dev(f), dev(inp.v), dev(inp.sky))
        fh.fh_transform(plan, 0, 1)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_select_candidates(plan, 0, 1)
        assert ei.value.code in (fh.FH_ERR_UNSORTED, fh.FH_ERR_INVALID_ARG)
        # the plan stays usable after the reported error
        fh.fh_correct_doppler(plan, dev(inp.t), dev(inp.offsets), dev(inp.freq), dev(inp.v),
                              dev(inp.sky))
        fh.fh_transform(plan, 0, 1)
        fh.fh_select_candidates(plan, 0, 1)
    finally:
        fh.fh_destroy_plan(plan)


def test_candidate_capacity_error(fh):
    import ctypes
    inp, pp = synth.random_case(17, n_fft=8, n_bins=20, n_dir=2, p=0.5)
    plan = fh.fh_create_plan(fh.make_desc(pp, 8, 2, inp.n_peaks))
    try:
        fh.fh_correct_doppler(plan, inp.t, inp.offsets, inp.freq, inp.v, inp.sky)
        fh.fh_transform(plan, 0, 2)
        n = ctypes.c_int64(0)
        small = np.zeros(3, dtype=fh.CANDIDATE_DTYPE)
        rc = fh.load().fh_select_candidates(plan, 0, 2, small.ctypes.data, 3, ctypes.byref(n), 0, None)
        assert rc == fh.FH_ERR_CAPACITY
        n_sb = -(-pp["n_f0"] // pp["subband_cells"])
        assert n.value == 2 * n_sb * pp["top_k"]
    finally:
        fh.fh_destroy_plan(plan)


# ---------------------------------------------------------------- the paper's workloads
def test_workload_nodoppler_100Hz_full(fh, oracle_mod):
    w = synth.WORKLOADS["nodoppler_T1024_N200_100Hz"]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    o = oracle_mod.search(inp, pp, want_maps=True)
    for mode in (1, 2):
        g = run_gpu(fh, inp, pp, mode=mode)
        compare(g, o, pp, w.n_fft)


def test_workload_sky_patch256_plain_vs_batched(fh, oracle_mod):
    w = synth.WORKLOADS["sky_patch256_T1024_N200_100Hz"]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    o = oracle_mod.search(inp, pp, want_maps=True)
    gb = run_gpu(fh, inp, pp, schedule=0)
    compare(gb, o, pp, w.n_fft)
    gp = run_gpu(fh, inp, pp, schedule=1, maps=False)
    compare(gp, o, pp, w.n_fft, maps=False)
    assert gp["launches"] > gb["launches"]


def test_workload_single_sky_50Hz_bench_configuration(fh, oracle_mod):
    """The benchmark's workload (T_FFT 8192 s, 150 days, 1169 x 81920 map) in the
    benchmark's launch configuration (autotuned tile): full map bit-exact."""
    w = synth.WORKLOADS["single_sky_T8192_150d_50Hz"]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    o = oracle_mod.search(inp, pp, want_maps=True)
    g = run_gpu(fh, inp, pp, autotune=True)
    compare(g, o, pp, w.n_fft)


def test_workload_highfreq_900Hz_sampled(fh, oracle_mod):
    """Largest workload (N = 61594 FFTs, ~26M peaks, 356 x 102400 map): two
    directions on the GPU; the oracle computes sampled rows of each and the
    candidates are checked against the profile the GPU reports."""
    import torch
    w = synth.WORKLOADS["highfreq_T1024_1yr_900Hz_64dir"]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    sub = synth.Inputs(w=w, t=inp.t, offsets=inp.offsets, freq=inp.freq, v=inp.v,
                       sky=np.ascontiguousarray(inp.sky[[w.line_dir, 40]]))
    g = run_gpu(fh, sub, pp, maps=True)
    kt = float(pp["k_over"]) * pp["t_fft"]
    r = oracle_mod.doppler_factor(sub.v, sub.sky)
    assert np.array_equal(g["r"].view(np.uint64), r.view(np.uint64))
    A = oracle_mod.positions(sub.offsets, sub.freq, r, pp["f0_min"], kt, pp["k_over"])
    assert np.array_equal(g["A"], A)
    S0, D = oracle_mod.shift_tables(sub.t, pp["t_ref"], kt, pp["fdot_min"], pp["fdot_step"])
    rows = np.array([0, 31, 32, 200, pp["n_fdot"] - 1], dtype=np.int32)
    for d in range(2):
        m = oracle_mod.hough_map(sub.offsets, A[d], S0, D, pp["k_over"], pp["n_f0"], rows=rows)
        assert np.array_equal(g["maps"][d][rows], m)
        pc, pr = oracle_mod.profile(g["maps"][d])
        assert np.array_equal(g["prof"][d], oracle_profile_keys(pc, pr))
        c, rr, n = oracle_mod.select(pc, pr, pp["subband_cells"], pp["top_k"], pp["excl_cells"],
                                     pp["sep_cells"], pp["n_thr"])
        cg = g["cand"].reshape(2, -1, pp["top_k"])[d]
        assert np.array_equal(cg["cell"], c) and np.array_equal(cg["count"], n)
    # the line direction recovers the injected line
    true_cell = int(math.floor((w.line_f0 - w.f_lo) * w.kt))
    q = true_cell // pp["subband_cells"]
    top = g["cand"].reshape(2, -1, pp["top_k"])[0, q, 0]
    assert abs(int(top["cell"]) - true_cell) <= w.k_over
    assert int(top["count"]) > 0.6 * w.n_fft


def test_workload_highfreq_900Hz_all_directions_bench_configuration(fh, oracle_mod):
    """The largest workload as the benchmark runs it: all 64 directions in one
    batched plan (window tables in groups of directions), autotuned tile.
    Three directions in different groups, the line's among them, are checked
    bit for bit against the oracle's full maps: profile keys and candidates
    (reporting columns to 1e-12)."""
    import torch
    w = synth.WORKLOADS["highfreq_T1024_1yr_900Hz_64dir"]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    n_dir = inp.sky.shape[0]
    dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
    plan = fh.fh_create_plan(fh.make_desc(pp, w.n_fft, n_dir, inp.n_peaks))
    try:
        fh.fh_correct_doppler(plan, *dev)
        fh.fh_autotune(plan, 0, n_dir)
        fh.fh_transform(plan, 0, n_dir)
        prof = torch.empty((n_dir, pp["n_f0"]), dtype=torch.int64, device="cuda")
        fh.fh_copy_profile(plan, 0, n_dir, prof)
        cand = fh.fh_select_candidates(plan, 0, n_dir).reshape(n_dir, -1, pp["top_k"])
        prof = prof.cpu().numpy().view(np.uint64)
    finally:
        fh.fh_destroy_plan(plan)
    kt = float(pp["k_over"]) * pp["t_fft"]
    S0, D = oracle_mod.shift_tables(inp.t, pp["t_ref"], kt, pp["fdot_min"], pp["fdot_step"])
    for d in sorted({w.line_dir, 30, 63}):
        r = oracle_mod.doppler_factor(inp.v, inp.sky[d:d + 1])
        A = oracle_mod.positions(inp.offsets, inp.freq, r, pp["f0_min"], kt, pp["k_over"])[0]
        m = oracle_mod.hough_map(inp.offsets, A, S0, D, pp["k_over"], pp["n_f0"], n_fdot=pp["n_fdot"])
        pc, pr = oracle_mod.profile(m)
        del m
        assert np.array_equal(prof[d], oracle_profile_keys(pc, pr)), d
        c, rr, n = oracle_mod.select(pc, pr, pp["subband_cells"], pp["top_k"], pp["excl_cells"],
                                     pp["sep_cells"], pp["n_thr"])
        assert np.array_equal(cand[d]["cell"], c) and np.array_equal(cand[d]["row"], rr)
        assert np.array_equal(cand[d]["count"], n) and np.all(cand[d]["dir"] == d)
        f0, fdot, cr = oracle_mod.report(c, rr, n, pp["f0_min"], kt, pp["fdot_min"],
                                         pp["fdot_step"], w.n_fft, pp["p0"])
        for got, want in ((cand[d]["f0"], f0), (cand[d]["fdot"], fdot), (cand[d]["cr"], cr)):
            assert np.all(np.abs(got - want) <= REL_TOL * np.maximum(np.abs(want), 1e-300))


@pytest.mark.parametrize("seed", [41, 42])
def test_host_inputs_checked_on_the_device_match_oracle(fh, oracle_mod, seed):
    """FH_CHECKS_DEVICE: host inputs copied and checked by the kernels give the
    same positions, maps, profiles and candidates as the oracle."""
    inp, pp = synth.random_case(seed, n_fft=33, n_bins=70, n_dir=3, p=0.4)
    g = run_gpu(fh, inp, pp, device_inputs=False, checks=fh.FH_CHECKS_DEVICE)
    o = oracle_mod.search(inp, pp, want_maps=True)
    compare(g, o, pp, inp.t.shape[0])


@pytest.mark.parametrize("seed, n_dir", [(43, 1), (44, 1), (45, 3)])
def test_pinned_host_inputs_match_oracle(fh, oracle_mod, seed, n_dir):
    """Page-locked host inputs (read in place by the kernels for one direction,
    copied for several), under host and under device checks: the oracle's
    positions, maps, profiles and candidates."""
    inp, pp = synth.random_case(seed, n_fft=41, n_bins=90, n_dir=n_dir, p=0.3)
    o = oracle_mod.search(inp, pp, want_maps=True)
    for checks in (fh.FH_CHECKS_HOST, fh.FH_CHECKS_DEVICE):
        g = run_gpu(fh, inp, pp, device_inputs=False, pinned=True, checks=checks)
        compare(g, o, pp, inp.t.shape[0])


def test_pinned_host_input_errors_checked_on_the_device(fh):
    """FH_CHECKS_DEVICE with page-locked host inputs read in place: unsorted
    frequencies and a broken CSR are reported at the next synchronising call,
    and the plan stays usable."""
    import torch
    inp, pp = synth.random_case(18, n_fft=12, n_bins=30, n_dir=1, p=0.5)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
    plan = fh.fh_create_plan(fh.make_desc(pp, 12, 1, inp.n_peaks))
    try:
        fh.fh_plan_set_input_checks(plan, fh.FH_CHECKS_DEVICE)
        f = pin(inp.freq)
        a = int(inp.offsets[4])
        f[a], f[a + 1] = f[a + 1], f[a]
        args = [pin(inp.t), pin(inp.offsets), f, pin(inp.v), pin(inp.sky)]
        fh.fh_correct_doppler(plan, *args)
        fh.fh_transform(plan, 0, 1)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_select_candidates(plan, 0, 1)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        off = pin(inp.offsets)
        off[6] = inp.n_peaks + 50
        fh.fh_correct_doppler(plan, args[0], off, pin(inp.freq), args[3], args[4],
                              n_peaks=inp.n_peaks)
        fh.fh_transform(plan, 0, 1)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_sync(plan)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        # valid page-locked inputs again: the oracle's candidates
        good = [pin(x) for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        fh.fh_correct_doppler(plan, *good)
        fh.fh_transform(plan, 0, 1)
        cand = fh.fh_select_candidates(plan, 0, 1)
    finally:
        fh.fh_destroy_plan(plan)
    import oracle
    o = oracle.search(inp, pp)
    c = cand.reshape(1, -1, pp["top_k"])
    assert np.array_equal(c["cell"], o["cell"]) and np.array_equal(c["count"], o["count"])


def test_host_input_errors_checked_on_the_device(fh):
    """FH_CHECKS_DEVICE: unsorted frequencies, a broken CSR, a NaN time and an
    infinite velocity in HOST memory are reported by the next synchronising
    call (no fault), and the plan stays usable."""
    inp, pp = synth.random_case(17, n_fft=10, n_bins=20, n_dir=1, p=0.5)
    plan = fh.fh_create_plan(fh.make_desc(pp, 10, 1, inp.n_peaks))
    try:
        fh.fh_plan_set_input_checks(plan, fh.FH_CHECKS_DEVICE)
        f = inp.freq.copy()
        a = int(inp.offsets[3])
        f[a], f[a + 1] = f[a + 1], f[a]
        fh.fh_correct_doppler(plan, inp.t, inp.offsets, f, inp.v, inp.sky)
        fh.fh_transform(plan, 0, 1)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_select_candidates(plan, 0, 1)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        off = inp.offsets.copy()
        off[5] = inp.n_peaks + 1000
        off[6] = -3
        fh.fh_correct_doppler(plan, inp.t, off, inp.freq, inp.v, inp.sky, n_peaks=inp.n_peaks)
        fh.fh_transform(plan, 0, 1)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_sync(plan)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        t = inp.t.copy()
        t[4] = np.nan
        fh.fh_correct_doppler(plan, t, inp.offsets, inp.freq, inp.v, inp.sky)
        fh.fh_transform(plan, 0, 1)
        with pytest.raises(fh.FHError):
            fh.fh_select_candidates(plan, 0, 1)
        v = inp.v.copy()
        v[2, 1] = np.inf
        fh.fh_correct_doppler(plan, inp.t, inp.offsets, inp.freq, v, inp.sky)
        fh.fh_transform(plan, 0, 1)
        with pytest.raises(fh.FHError):
            fh.fh_select_candidates(plan, 0, 1)
        fh.fh_correct_doppler(plan, inp.t, inp.offsets, inp.freq, inp.v, inp.sky)
        fh.fh_transform(plan, 0, 1)
        fh.fh_select_candidates(plan, 0, 1)
        with pytest.raises(fh.FHError):
            fh.fh_plan_set_input_checks(plan, 7)
    finally:
        fh.fh_destroy_plan(plan)


def test_windows_beyond_16_bits_are_looked_up(fh, oracle_mod):
    """A window table entry holds the window's first peak relative to its FFT's
    first and its count in 16 bits each; an FFT with 150,000 peaks 0.002 bins
    apart has windows whose count, and later whose start, do not fit, so the
    transform looks those windows up by binary search.  (The same peaks are also
    two to a cell, so packed counters do not apply to the job.)  Maps and
    candidates equal the oracle's."""
    inp, pp = synth.dense_case(91, dense_ffts=(2,), n_dense=150000, spacing_bins=0.002,
                               n_fft=6, n_bins=400, n_fdot=9, n_dir=1, p=0.2)
    assert int(inp.offsets[3] - inp.offsets[2]) == 150000
    o = oracle_mod.search(inp, pp, want_maps=True)
    for tile, warps in ((1024, 16), (1408, 8)):
        g = run_gpu(fh, inp, pp, tile=tile, warps=warps)
        compare(g, o, pp, inp.t.shape[0])


@pytest.mark.parametrize("mode", [1, 2])
def test_ffts_with_more_peaks_than_staged_are_read_from_global_memory(fh, oracle_mod, mode):
    """The window pre-pass stages each FFT's peak cells in shared memory up to
    a fixed count per FFT and direction (fewer when it stages the two
    directions of a pair); FFTs 1 and 3 here hold 900 and 1100 peaks, 0.3
    bins (3 cells) apart, beyond one or both limits, so their windows come from
    searches in global memory.  Three directions: one pair and one single
    direction in START mode.  Maps and candidates equal the oracle's."""
    inp, pp = synth.dense_case(93, dense_ffts=(1,), n_dense=900, spacing_bins=0.3,
                               n_fft=6, n_bins=400, n_fdot=40, n_dir=3, p=0.2)
    more, _ = synth.dense_case(93, dense_ffts=(3,), n_dense=1100, spacing_bins=0.3,
                               n_fft=6, n_bins=400, n_fdot=40, n_dir=3, p=0.2)
    counts = np.diff(inp.offsets)
    counts[3] = np.diff(more.offsets)[3]
    offsets = np.zeros(7, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    parts = [inp.freq[inp.offsets[i]:inp.offsets[i + 1]] if i != 3 else
             more.freq[more.offsets[3]:more.offsets[4]] for i in range(6)]
    inp = synth.Inputs(w=inp.w, t=inp.t, offsets=offsets, freq=np.concatenate(parts),
                       v=inp.v, sky=inp.sky)
    assert counts[1] == 900 and counts[3] == 1100
    o = oracle_mod.search(inp, pp, want_maps=True)
    for tile, warps in ((0, 0), (256, 8)):
        g = run_gpu(fh, inp, pp, mode=mode, tile=tile, warps=warps)
        compare(g, o, pp, inp.t.shape[0])


@pytest.mark.parametrize("n_fdot", [1, 2, 34, 35, 36, 40, 48, 49, 64])
def test_short_last_slab_every_width(fh, oracle_mod, n_fdot):
    """A last slab of R <= 16 rows is walked in 2^ceil(log2 R) steps with the
    row copies folded before the emit (1, 2, 3, 4, 8, 16 rows here; 17 and 32
    take the full walk), for a pair of directions and a single one (three
    directions), in START mode; maps, profiles and candidates equal the
    oracle's."""
    inp, pp = synth.random_case(500 + n_fdot, n_fft=24, n_bins=200, k_over=10, n_fdot=n_fdot,
                                n_dir=3, p=0.3)
    o = oracle_mod.search(inp, pp, want_maps=True)
    g = run_gpu(fh, inp, pp, mode=2, tile=320, warps=8)
    compare(g, o, pp, inp.t.shape[0])


@pytest.mark.parametrize("n_fdot", [33, 40, 63, 64, 65, 80, 96, 97, 130])
def test_one_direction_row_pairs(fh, oracle_mod, n_fdot):
    """One direction of a plain START map walks 64-row slabs with rows j0 + r and
    j0 + 32 + r in the two 16-bit halves of a counter word (the last slab's
    halves one after the other where they hold 32 rows or fewer); maps,
    profiles and candidates equal the oracle's, with the library's default
    tile and a narrow one (several tiles, a ragged last one)."""
    inp, pp = synth.random_case(700 + n_fdot, n_fft=30, n_bins=240, k_over=10, n_fdot=n_fdot,
                                n_dir=1, p=0.3)
    o = oracle_mod.search(inp, pp, want_maps=True)
    for tile, warps in ((0, 0), (352, 8)):
        g = run_gpu(fh, inp, pp, mode=2, tile=tile, warps=warps)
        compare(g, o, pp, inp.t.shape[0])


def test_row_pairs_dense_and_bad_device_inputs(fh, oracle_mod):
    """One direction in 64-row slabs when the paired counters do not apply:
    dense off-grid peaks (two stripes of one FFT can start in one cell, so the
    16-bit halves could overflow) walk the slab's two 32-row halves one after
    the other with whole-word counts, equal to the oracle; unsorted device
    frequencies make the transform take the clamped walk over the 64-row
    windows, reported at the next synchronising call, and the next valid call
    is equal to the oracle again."""
    import torch
    inp, pp = synth.dense_case(95, dense_ffts=(2, 5), n_dense=40, spacing_bins=0.05,
                               n_fft=12, n_bins=300, n_fdot=70, n_dir=1, p=0.2)
    o = oracle_mod.search(inp, pp, want_maps=True)
    compare(run_gpu(fh, inp, pp, mode=2), o, pp, inp.t.shape[0])
    clean, cpp = synth.random_case(96, n_fft=12, n_bins=300, n_fdot=70, n_dir=1, p=0.3)
    plan = fh.fh_create_plan(fh.make_desc(cpp, 12, 1, clean.n_peaks))
    try:
        dev = lambda x: torch.from_numpy(x).cuda()
        f = clean.freq.copy()
        for i in range(clean.t.shape[0]):
            a, b = int(clean.offsets[i]), int(clean.offsets[i + 1])
            f[a:b] = f[a:b][::-1]
        fh.fh_correct_doppler(plan, dev(clean.t), dev(clean.offsets), dev(f), dev(clean.v),
                              dev(clean.sky))
        fh.fh_transform(plan, 0, 1)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_sync(plan)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        fh.fh_correct_doppler(plan, *[dev(x) for x in (clean.t, clean.offsets, clean.freq,
                                                      clean.v, clean.sky)])
        m = torch.full((1, cpp["n_fdot"], cpp["n_f0"]), -7, dtype=torch.int32, device="cuda")
        fh.fh_transform(plan, 0, 1, m)
        torch.cuda.synchronize()
        assert np.array_equal(m.cpu().numpy(), oracle_mod.search(clean, cpp, want_maps=True)["maps"])
    finally:
        fh.fh_destroy_plan(plan)
