"""Pins of the oracle's refined-grid search (Sec. "Refined Grid in the parameter
space") against facts that do not come from the refinement code.  CPU only."""
import numpy as np
import pytest

from paper_1407_8333_gb300 import synth


def _coarse(oracle, inp, pp):
    kt = float(pp["k_over"]) * float(pp["t_fft"])
    r = oracle.doppler_factor(inp.v, inp.sky)
    A = oracle.positions(inp.offsets, inp.freq, r, pp["f0_min"], kt, pp["k_over"])
    S0, D = oracle.shift_tables(inp.t, pp["t_ref"], kt, pp["fdot_min"], pp["fdot_step"])
    return oracle.hough_map(inp.offsets, A[0], S0, D, pp["k_over"], pp["n_f0"], pp["n_fdot"])


@pytest.fixture(scope="module")
def small(oracle_mod):
    inp, pp = synth.random_case(71, n_fft=30, n_bins=60, n_fdot=24, n_dir=1, p=0.35)
    return inp, pp, _coarse(oracle_mod, inp, pp)


def test_k_fdot_1_on_the_coarse_direction_is_a_slice_of_the_coarse_map(oracle_mod, small):
    """With K_fdot = 1 and the coarse direction alone the refined grid is the
    coarse grid: rows j_c - 2 .. j_c + 1, cells b_c - K .. b_c + K."""
    inp, pp, coarse = small
    K = pp["k_over"]
    for cell, row in ((3 * K, 5), (pp["n_f0"] // 2, 12), (pp["n_f0"] - K - 1, pp["n_fdot"] - 2)):
        m = oracle_mod.refine_maps(inp, pp, cell, row, inp.sky[:1], 1)[0]
        assert np.array_equal(m, coarse[row - 2:row + 2, cell - K:cell + K + 1])


def test_every_k_fdot_th_refined_row_follows_a_coarse_row(oracle_mod, small):
    """Refined row m K_fdot and coarse row j_c - 2 + m differ in shift by less
    than K_fdot units of 2^-32 cell per FFT, which moves no stripe here."""
    inp, pp, coarse = small
    K, kf = pp["k_over"], 3
    cell, row = pp["n_f0"] // 2, 11
    m = oracle_mod.refine_maps(inp, pp, cell, row, inp.sky[:1], kf)[0]
    for q in range(4):
        assert np.array_equal(m[q * kf], coarse[row - 2 + q, cell - K:cell + K + 1])


def test_refined_map_by_python_brute_force(oracle_mod):
    """The refined map from its definition in exact integers: stripe start
    floor((A - (S0_i + (j_c - 2) D_i) - j' D'_i) / 2^32) - (b_c - K), K cells."""
    inp, pp = synth.random_case(72, n_fft=10, n_bins=24, n_fdot=9, n_dir=1, p=0.5)
    K, kf = pp["k_over"], 2
    cell, row = 2 * K + 3, 4
    kt = float(K) * float(pp["t_fft"])
    r = oracle_mod.doppler_factor(inp.v, inp.sky)
    A = oracle_mod.positions(inp.offsets, inp.freq, r, pp["f0_min"], kt, K)[0]
    S0, D = oracle_mod.shift_tables(inp.t, pp["t_ref"], kt, pp["fdot_min"], pp["fdot_step"])
    _, Dr = oracle_mod.shift_tables(inp.t, pp["t_ref"], kt, 0.0, pp["fdot_step"] / kf)
    ref = np.zeros((4 * kf, 2 * K + 1), dtype=np.int64)
    lo = cell - K
    for i in range(inp.t.shape[0]):
        for p in range(inp.offsets[i], inp.offsets[i + 1]):
            for j in range(4 * kf):
                s = ((int(A[p]) - int(S0[i]) - (row - 2) * int(D[i]) - j * int(Dr[i])) >> 32) - lo
                for b in range(max(s, 0), min(s + K, 2 * K + 1)):
                    ref[j, b] += 1
    m = oracle_mod.refine_maps(inp, pp, cell, row, inp.sky[:1], kf)[0]
    assert np.array_equal(m, ref)


def test_refinement_sharpens_the_spindown_of_the_50Hz_line(oracle_mod):
    """The 50 Hz workload's injected line (-3e-9 Hz/s) lies half-way between two
    coarse spin-down rows; with K_fdot = 4 its refined spin-down is within half
    a refined step of the truth, closer than the coarse one, and the refined
    count is at least the coarse one (the refined grid contains the coarse
    row)."""
    w = synth.WORKLOADS["single_sky_T8192_150d_50Hz"]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    o = oracle_mod.search(inp, pp)
    sb = int((w.line_f0 - w.f_lo) / w.subband_hz)
    cell, row, count = (int(o[k][0, sb, 0]) for k in ("cell", "row", "count"))
    coarse_fdot = float(o["fdot"][0, sb, 0])
    kf = 4
    ref = oracle_mod.refine(inp, pp, [cell], [row], inp.sky[None, :1], kf)
    step = pp["fdot_step"]
    assert abs(ref["fdot"][0] - w.line_fdot) <= step / kf / 2 + 1e-18
    assert abs(ref["fdot"][0] - w.line_fdot) < abs(coarse_fdot - w.line_fdot)
    assert ref["count"][0] >= count
    assert abs(ref["f0"][0] - w.line_f0) < 2.0 / w.t_fft


def test_refined_sky_includes_the_coarse_direction_and_its_count(oracle_mod):
    """The refined sky rectangle contains the coarse direction (its centre),
    so the refined count is at least the coarse candidate's count."""
    w = synth.WORKLOADS["single_sky_T8192_150d_50Hz"]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    o = oracle_mod.search(inp, pp)
    sb = int((w.line_f0 - w.f_lo) / w.subband_hz)
    cell, row, count = (int(o[k][0, sb, 0]) for k in ("cell", "row", "count"))
    sky = synth.refined_sky(inp.sky[0], synth.doppler_number(w.f_hi, w.t_fft), 3)
    assert np.array_equal(sky[4], inp.sky[0])
    ref = oracle_mod.refine(inp, pp, [cell], [row], sky[None], 1)
    assert ref["count"][0] >= count
