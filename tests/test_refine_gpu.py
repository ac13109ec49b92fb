"""Refined-grid search (Sec. "Refined Grid in the parameter space") on the GPU,
through the C ABI, against the oracle.

Refined direction, row, cell and count bit for bit; f0, spin-down and critical
ratio to 1e-12 relative.  Cases: random peakmaps with many candidates (several
transform batches), candidates at the edges of the coarse grid (the refined
band reaches outside it), spin-down refinements whose rows span one and
several 32-row slabs, and the 50 Hz line of the T_FFT = 8192 s workload on a
refined sky rectangle.
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


def gpu_refine(fh, inp, pp, cells, rows, sky_ref, k_fdot, checks=None):
    plan = fh.fh_create_plan(fh.make_desc(pp, inp.t.shape[0], 1, max(1, inp.n_peaks)))
    try:
        if checks is not None:
            fh.fh_plan_set_input_checks(plan, checks)
        return fh.fh_refine(plan, inp.t, inp.offsets, inp.freq, inp.v, cells, rows, sky_ref,
                            k_fdot)
    finally:
        fh.fh_destroy_plan(plan)


def check(g, o, n_cand):
    assert g.shape == (n_cand,)
    for k in ("dir", "row", "cell", "count"):
        assert np.array_equal(g[k].astype(np.int64), o[k]), k
    assert np.array_equal(g["subband"], np.arange(n_cand))
    assert np.all(g["rank"] == 0)
    for k in ("f0", "fdot", "cr"):
        np.testing.assert_allclose(g[k], o[k], rtol=REL_TOL, atol=0.0, err_msg=k)


def random_sky_ref(seed, n_cand, n_ref):
    u = synth.uniform(seed, 11, np.arange(2 * n_cand * n_ref)).reshape(n_cand, n_ref, 2)
    z = u[..., 0] * 2.0 - 1.0
    ph = u[..., 1] * 2.0 * np.pi
    r = np.sqrt(1.0 - z * z)
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=-1)


@pytest.mark.parametrize("k_fdot", [1, 3, 10])
def test_random_candidates_match_the_oracle(fh, oracle_mod, k_fdot):
    inp, pp = synth.random_case(301 + k_fdot, n_fft=40, n_bins=50, n_fdot=16, n_dir=1, p=0.4)
    n_cand, n_ref = 29, 5
    cu = synth.uniform(400 + k_fdot, 3, np.arange(2 * n_cand)).reshape(2, n_cand)
    cells = (cu[0] * pp["n_f0"]).astype(np.int32)
    rows = (cu[1] * pp["n_fdot"]).astype(np.int32)
    # the edges of the coarse grid: the refined band reaches outside it
    cells[:4] = [0, 1, pp["n_f0"] - 1, pp["n_f0"] // 2]
    rows[:4] = [0, pp["n_fdot"] - 1, 1, 0]
    sky = random_sky_ref(500 + k_fdot, n_cand, n_ref)
    sky[:, 0] = inp.sky[0]
    g = gpu_refine(fh, inp, pp, cells, rows, sky, k_fdot)
    o = oracle_mod.refine(inp, pp, cells, rows, sky, k_fdot)
    check(g, o, n_cand)


def test_many_rows_several_slabs(fh, oracle_mod):
    """K_fdot = 20: 80 refined rows, two full 32-row slabs and a ragged one."""
    inp, pp = synth.random_case(333, n_fft=24, n_bins=30, n_fdot=9, n_dir=1, p=0.5)
    cells = np.array([5, pp["n_f0"] // 3, pp["n_f0"] - 7], dtype=np.int32)
    rows = np.array([4, 2, 6], dtype=np.int32)
    sky = random_sky_ref(334, 3, 2)
    g = gpu_refine(fh, inp, pp, cells, rows, sky, 20)
    o = oracle_mod.refine(inp, pp, cells, rows, sky, 20)
    check(g, o, 3)


def test_no_candidates_and_argument_errors(fh):
    inp, pp = synth.random_case(335, n_fft=8, n_bins=10, n_fdot=5, n_dir=1)
    sky = np.zeros((0, 1, 3))
    out = gpu_refine(fh, inp, pp, np.zeros(0, np.int32), np.zeros(0, np.int32), sky, 2)
    assert out.shape == (0,)
    one = inp.sky[None, :1]
    for kf in (0, 65):
        with pytest.raises(fh.FHError) as ei:
            gpu_refine(fh, inp, pp, [3], [2], one, kf)
        assert ei.value.code == fh.FH_ERR_INVALID_ARG
    with pytest.raises(fh.FHError) as ei:      # no refined direction
        gpu_refine(fh, inp, pp, [3], [2], np.zeros((1, 0, 3)), 2)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG
    bad = inp.sky[None, :1] * 2.0               # not a unit vector
    with pytest.raises(fh.FHError) as ei:
        gpu_refine(fh, inp, pp, [3], [2], bad, 2)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG
    with pytest.raises(fh.FHError) as ei:      # candidate outside the fixed-point range
        gpu_refine(fh, inp, pp, [1 << 28], [2], one, 2)
    assert ei.value.code == fh.FH_ERR_RANGE


@pytest.mark.parametrize("k_fdot", [1, 4])
def test_the_50Hz_line_on_a_refined_sky(fh, oracle_mod, k_fdot):
    """The injected line of the T_FFT = 8192 s, 150 d workload: the coarse
    candidate of its subband, refined on a 3 x 3 sky rectangle around the
    coarse direction and K_fdot spin-down."""
    w = synth.WORKLOADS["single_sky_T8192_150d_50Hz"]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    o = oracle_mod.search(inp, pp)
    sb = int((w.line_f0 - w.f_lo) / w.subband_hz)
    # the line's subband and two of its neighbours, best candidate of each
    sbs = [sb, sb - 1, sb + 1]
    cells = np.array([int(o["cell"][0, s, 0]) for s in sbs], dtype=np.int32)
    rows = np.array([int(o["row"][0, s, 0]) for s in sbs], dtype=np.int32)
    n_d = synth.doppler_number(w.f_hi, w.t_fft)
    sky = np.stack([synth.refined_sky(inp.sky[0], n_d, 3)] * len(sbs))
    g = gpu_refine(fh, inp, pp, cells, rows, sky, k_fdot)
    r = oracle_mod.refine(inp, pp, cells, rows, sky, k_fdot)
    check(g, r, len(sbs))
    assert g["count"][0] >= int(o["count"][0, sb, 0])


def test_refine_with_device_checks(fh, oracle_mod):
    """FH_CHECKS_DEVICE: the same refined candidates; unsorted frequencies are
    reported by the call (it synchronises) as FH_ERR_UNSORTED."""
    inp, pp = synth.random_case(336, n_fft=30, n_bins=40, n_fdot=12, n_dir=1, p=0.4)
    cells = np.array([10, pp["n_f0"] // 2, pp["n_f0"] - 3], dtype=np.int32)
    rows = np.array([3, 6, 9], dtype=np.int32)
    sky = random_sky_ref(337, 3, 4)
    g = gpu_refine(fh, inp, pp, cells, rows, sky, 3, checks=fh.FH_CHECKS_DEVICE)
    check(g, oracle_mod.refine(inp, pp, cells, rows, sky, 3), 3)
    # the two highest peaks of one FFT swapped, far from candidates near the
    # bottom of the band: found by the check of every frequency, not only of
    # the peaks near the candidates
    f = inp.freq.copy()
    b = int(inp.offsets[5]) - 1
    f[b - 1], f[b] = f[b], f[b - 1]
    low = np.array([8, 12], dtype=np.int32)
    plan = fh.fh_create_plan(fh.make_desc(pp, inp.t.shape[0], 1, inp.n_peaks))
    try:
        fh.fh_plan_set_input_checks(plan, fh.FH_CHECKS_DEVICE)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_refine(plan, inp.t, inp.offsets, f, inp.v, low, rows[:2], sky[:2], 3)
        assert ei.value.code == fh.FH_ERR_UNSORTED
    finally:
        fh.fh_destroy_plan(plan)
