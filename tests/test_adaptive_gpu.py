"""Adaptive frequency-Hough map (Eq. ncountadap) on the GPU, through the C ABI,
against the oracle.

Weighted maps, profiles and candidate cells/rows/counts bit for bit; the
adaptive critical ratio to 1e-12 relative.  Small weights exercise the
transform's packed emit (counts below 2^26), large ones its unpacked path.
"""
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


def run_weighted(fh, inp, pp, weights, frac_bits, mode=0, maps=True, tile=0, warps=0):
    import torch
    n_fft = inp.t.shape[0]
    n_dir = inp.sky.shape[0]
    plan = fh.fh_create_plan(fh.make_desc(pp, n_fft, n_dir, max(1, inp.n_peaks), mode=mode,
                                          tile_cells=tile, block_warps=warps))
    try:
        dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        fh.fh_correct_doppler(plan, *dev)
        if weights is not None:
            fh.fh_set_weights(plan, weights, frac_bits)
        m = (torch.full((n_dir, pp["n_fdot"], pp["n_f0"]), -7, dtype=torch.int32, device="cuda")
             if maps else None)
        fh.fh_transform(plan, 0, n_dir, m)
        prof = torch.empty((n_dir, pp["n_f0"]), dtype=torch.int64, device="cuda")
        fh.fh_copy_profile(plan, 0, n_dir, prof)
        cand = fh.fh_select_candidates(plan, 0, n_dir)
        torch.cuda.synchronize()
        out = dict(prof=prof.cpu().numpy().view(np.uint64), cand=cand)
        if maps:
            out["maps"] = m.cpu().numpy()
        return out
    finally:
        fh.fh_destroy_plan(plan)


def check(g, o, pp, maps=True):
    if maps:
        assert np.array_equal(g["maps"], o["maps"])
    keys = (o["pcount"].astype(np.uint64) << np.uint64(32)) | \
           (np.uint64(0xFFFFFFFF) - o["prow"].astype(np.uint64))
    assert np.array_equal(g["prof"], keys)
    n_dir = o["cell"].shape[0]
    c = g["cand"].reshape(n_dir, -1, pp["top_k"])
    for k in ("cell", "row", "count"):
        assert np.array_equal(c[k], o[k]), k
    for k in ("f0", "fdot", "cr"):
        a, b = c[k], o[k]
        assert np.all((a == b) | (np.abs(a - b) <= REL_TOL * np.abs(b))), k


CASES = [
    # seed, n_fft, n_bins, n_fdot, n_dir, frac_bits, weight scale, mode, tile, warps
    (51, 30, 80, 37, 2, 4, 2.0, 0, 96, 8),        # packed emit
    (52, 41, 96, 45, 3, 20, 6.0, 0, 128, 16),     # count bound above 2^26: unpacked emit
    (53, 25, 64, 33, 2, 8, 3.0, 1, 100, 8),       # DIFF mode
    (54, 64, 200, 64, 1, 10, 1.0, 0, 0, 0),       # library default tile
]


@pytest.mark.parametrize("case", CASES)
def test_weighted_maps_and_candidates_bit_exact(fh, oracle_mod, case):
    seed, n_fft, n_bins, n_fdot, n_dir, F, scale, mode, tile, warps = case
    inp, pp = synth.random_case(seed, n_fft=n_fft, n_bins=n_bins, n_fdot=n_fdot, n_dir=n_dir,
                                p=0.3)
    w = scale * synth.uniform(seed, 77, np.arange(n_dir * n_fft)).reshape(n_dir, n_fft)
    w[:, ::7] = 0.0                       # some FFTs switched off
    o = oracle_mod.search(inp, pp, want_maps=True, weights=w, frac_bits=F)
    if F == 20:
        bounds = [oracle_mod.count_bound(inp.offsets, o["A"][d], pp["k_over"], o["W"][d])
                  for d in range(n_dir)]
        assert max(bounds) >= (1 << 26)
    g = run_weighted(fh, inp, pp, w, F, mode=mode, tile=tile, warps=warps)
    check(g, o, pp)


def test_unit_weights_equal_the_plain_map(fh, oracle_mod):
    inp, pp = synth.random_case(55, n_fft=33, n_bins=90, n_fdot=40, n_dir=2, p=0.3)
    a = run_weighted(fh, inp, pp, None, 0)
    b = run_weighted(fh, inp, pp, np.ones((2, 33)), 0)
    assert np.array_equal(a["maps"], b["maps"])
    assert np.array_equal(a["prof"], b["prof"])
    assert np.array_equal(a["cand"], b["cand"])


def test_new_peakmap_resets_weights_and_errors(fh):
    import torch
    inp, pp = synth.random_case(56, n_fft=20, n_bins=50, n_fdot=10, n_dir=1, p=0.3)
    plan = fh.fh_create_plan(fh.make_desc(pp, 20, 1, inp.n_peaks))
    try:
        dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        with pytest.raises(fh.FHError) as ei:            # no peakmap yet
            fh.fh_set_weights(plan, np.ones((1, 20)), 0)
        assert ei.value.code == fh.FH_ERR_INVALID_ARG
        fh.fh_correct_doppler(plan, *dev)
        fh.fh_transform(plan, 0, 1)
        plain = fh.fh_select_candidates(plan, 0, 1)
        for bad, code in ((np.full((1, 20), -1.0), fh.FH_ERR_INVALID_ARG),
                          (np.full((1, 20), np.nan), fh.FH_ERR_INVALID_ARG),
                          (np.ones((2, 20)), fh.FH_ERR_INVALID_ARG),       # wrong n_dir
                          (np.full((1, 20), 2.0 ** 26), fh.FH_ERR_RANGE)):  # sum >= 2^30
            with pytest.raises(fh.FHError) as ei:
                fh.fh_set_weights(plan, bad, 0)
            assert ei.value.code == code
        fh.fh_set_weights(plan, np.full((1, 20), 5.0), 0)
        fh.fh_transform(plan, 0, 1)
        five = fh.fh_select_candidates(plan, 0, 1)
        ok = plain["count"] >= 0
        assert np.array_equal(five["count"][ok], 5 * plain["count"][ok])
        fh.fh_correct_doppler(plan, *dev)                  # back to unit weights
        fh.fh_transform(plan, 0, 1)
        again = fh.fh_select_candidates(plan, 0, 1)
        assert np.array_equal(again, plain)
    finally:
        fh.fh_destroy_plan(plan)


def test_weighted_bench_workload_profile_and_candidates(fh, oracle_mod):
    """The 50 Hz benchmark workload, autotuned launch, weights of a beam-like
    daily modulation: profile and candidates against the oracle."""
    import torch
    w = synth.WORKLOADS["single_sky_T8192_150d_50Hz"]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    n = inp.t.shape[0]
    wts = (1.0 + 0.5 * np.cos(2 * np.pi * inp.t / 86164.09)).reshape(1, n)
    o = oracle_mod.search(inp, pp, weights=wts, frac_bits=12)
    plan = fh.fh_create_plan(fh.make_desc(pp, n, 1, inp.n_peaks))
    try:
        dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        fh.fh_correct_doppler(plan, *dev)
        fh.fh_autotune(plan, 0, 1)
        fh.fh_set_weights(plan, wts, 12)
        fh.fh_transform(plan, 0, 1)
        prof = torch.empty((1, pp["n_f0"]), dtype=torch.int64, device="cuda")
        fh.fh_copy_profile(plan, 0, 1, prof)
        cand = fh.fh_select_candidates(plan, 0, 1)
        g = dict(prof=prof.cpu().numpy().view(np.uint64), cand=cand)
    finally:
        fh.fh_destroy_plan(plan)
    check(g, o, pp, maps=False)


def _dense(seed):
    return synth.dense_case(seed, dense_ffts=(1, 5), n_dense=12, spacing_bins=0.2, n_fft=24,
                            n_bins=60, n_fdot=40, n_dir=2, p=0.3)


@pytest.mark.parametrize("mode,F,big", [(0, 4, 1.0), (0, 16, 1000.0), (1, 8, 40.0)])
def test_dense_off_grid_peaks_weighted_bit_exact(fh, oracle_mod, mode, F, big):
    """Dense off-grid peaks put several stripes of one FFT on a cell, so a count
    can exceed 2 sum(W); with a count bound below 2^31 both sides compute the
    map, equal bit for bit (packed emit, unpacked emit above 2^26, DIFF)."""
    inp, pp = _dense(61)
    n_fft = inp.t.shape[0]
    w = 1.0 + synth.uniform(61, 78, np.arange(2 * n_fft)).reshape(2, n_fft)
    w[:, 1] = big
    w[:, 5] = big
    o = oracle_mod.search(inp, pp, want_maps=True, weights=w, frac_bits=F)
    c = oracle_mod.stripe_overlap(inp.offsets, o["A"][0], pp["k_over"])
    assert c[1] >= 5 and c[5] >= 5
    assert int(o["maps"].max()) > 2 * int(o["W"][:, 1].max())   # more than two stripes
    g = run_weighted(fh, inp, pp, w, F, mode=mode, tile=96, warps=8)
    check(g, o, pp)


def test_dense_off_grid_peaks_large_weights_refused_on_both_sides(fh, oracle_mod):
    """The same peakmap with weights summing below 2^30 whose count bound
    reaches 2^31: the oracle raises and fh_set_weights returns FH_ERR_RANGE,
    and the plan still searches the same peakmap with admissible weights."""
    import torch
    inp, pp = _dense(62)
    n_fft = inp.t.shape[0]
    w = np.ones((2, n_fft))
    w[:, 1] = float(2 ** 29 - 4096)
    with pytest.raises(ValueError):
        oracle_mod.search(inp, pp, weights=w, frac_bits=0)
    plan = fh.fh_create_plan(fh.make_desc(pp, n_fft, 2, inp.n_peaks))
    try:
        dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        fh.fh_correct_doppler(plan, *dev)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_set_weights(plan, w, 0)
        assert ei.value.code == fh.FH_ERR_RANGE
        w2 = np.ones((2, n_fft))
        w2[:, 1] = 3.0
        fh.fh_set_weights(plan, w2, 0)
        m = torch.empty((2, pp["n_fdot"], pp["n_f0"]), dtype=torch.int32, device="cuda")
        fh.fh_transform(plan, 0, 2, m)
        torch.cuda.synchronize()
        o = oracle_mod.search(inp, pp, want_maps=True, weights=w2, frac_bits=0)
        assert np.array_equal(m.cpu().numpy(), o["maps"])
    finally:
        fh.fh_destroy_plan(plan)
