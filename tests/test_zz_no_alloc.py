"""fh_search_static: the allocation-free entry point.

It serves callers that cannot allocate device memory while they run (their
GPU memory is reserved for their own pool, or their loop must not take the
synchronisation a cudaMalloc/cudaFree can cause).  Checked here on the GPU,
through the C ABI:

* its candidates equal those of the plan-based entry points
  (fh_correct_doppler + fh_transform + fh_select_candidates) and those of the
  CPU oracle -- integers bit for bit, f0 / fdot / CR to 1e-12 relative -- on
  two calls in a row, the larger input first, so that anything the first call
  left in the shared scratch array would show up in the second; in both
  counting modes;
* the first call in the process takes at most the scratch array's size of
  device memory (the driver loads the array then), a later call none;
* a call with a broken CSR and unsorted frequencies in device memory reports
  them in device_status without faulting, and the next valid call (same
  scratch array) is right again;
* inputs beyond its fixed maximum sizes are refused with FH_ERR_TOO_LARGE.
"""
import math

import numpy as np
import pytest

from paper_1407_8333_gb300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12
# the fixed scratch array's size, as include/fh.h states it
SCRATCH_BYTES = 20_448_000
# the driver maps device memory in 2 MiB pages
PAGE = 2 << 20


@pytest.fixture(scope="module")
def fh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_8333_gb300 import build, fh as fhmod
    build.build()
    fhmod.load()
    return fhmod


def _dev(inp):
    import torch
    return [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]


def _plan_path(fh, inp, pp, mode):
    plan = fh.fh_create_plan(fh.make_desc(pp, max(1, inp.t.shape[0]), 1, max(1, inp.n_peaks),
                                          mode=mode))
    try:
        fh.fh_correct_doppler(plan, *_dev(inp))
        fh.fh_transform(plan, 0, 1)
        return fh.fh_select_candidates(plan, 0, 1)
    finally:
        fh.fh_destroy_plan(plan)


def _static_path(fh, dev, pp, out, status, mode):
    import torch
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    n = fh.fh_search_static(pp, *dev, out, status, mode=mode)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    got = out.cpu().numpy().view(fh.CANDIDATE_DTYPE)[:n].copy()
    return got, int(status.item()), free_before - free_after


def _same(a, b):
    for k in ("dir", "subband", "rank", "row", "cell", "count"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("f0", "fdot", "cr"):
        x, y = a[k], b[k]
        assert np.all((x == y) | (np.abs(x - y) <= REL_TOL * np.abs(y))), k


def _same_as_oracle(got, o, pp):
    c = got.reshape(1, -1, pp["top_k"])
    for k in ("cell", "row", "count"):
        assert np.array_equal(c[k], o[k]), k
    for k in ("f0", "fdot", "cr"):
        x, y = c[k], o[k]
        same = (x == y) | (np.isnan(x) & np.isnan(y))
        assert np.all(same | (np.abs(x - y) <= REL_TOL * np.abs(y))), k


def _cases():
    big_w = synth.WORKLOADS["sky_patch256_T1024_N200_100Hz"]
    big = synth.make_inputs(big_w)
    big = synth.Inputs(w=big_w, t=big.t, offsets=big.offsets, freq=big.freq, v=big.v,
                       sky=np.ascontiguousarray(big.sky[[big_w.line_dir]]))
    small, small_pp = synth.random_case(77, n_fft=30, n_bins=90, n_fdot=45, n_dir=1, p=0.3)
    return big_w, [(big, big_w.plan_params()), (small, small_pp)]


@pytest.mark.parametrize("mode", [1, 2])
def test_static_matches_plan_path_and_oracle_on_two_calls(fh, oracle_mod, mode):
    import torch
    big_w, cases = _cases()
    out = torch.empty(64 * 1024 * 48, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    first = None
    for k, (inp, pp) in enumerate(cases):
        want = _plan_path(fh, inp, pp, mode)
        o = oracle_mod.search(inp, pp)
        got, st, drop = _static_path(fh, _dev(inp), pp, out, status, mode)
        assert st == 0
        assert got.shape == want.shape
        _same(got, want)
        _same_as_oracle(got, o, pp)
        if k == 0:
            first = got
            # the first call of the process loads the scratch array (at most its
            # size, in whole pages); a call after it takes nothing
            assert drop <= (SCRATCH_BYTES + PAGE - 1) // PAGE * PAGE + PAGE
        else:
            assert drop == 0
    # the line case: the strongest candidate is the injected line (Sec. VI: a
    # signal adds about one count per FFT along its own f0 / fdot track)
    top = first[np.argmax(first["count"])]
    pp = cases[0][1]
    true_cell = int(math.floor((big_w.line_f0 - big_w.f_lo) * big_w.kt))
    assert abs(int(top["cell"]) - true_cell) <= big_w.k_over
    # the line's own row or a neighbour: over the 200 FFTs one row step moves a
    # stripe's end by about half a coarse bin, so neighbouring rows collect it too
    assert abs(float(top["fdot"]) - big_w.line_fdot) <= 1.5 * pp["fdot_step"]
    assert int(top["count"]) > 0.6 * big_w.n_fft


def test_static_reports_bad_device_inputs_then_recovers(fh, oracle_mod):
    """A broken CSR and unsorted frequencies in device memory: the kernels keep
    every read inside the arrays (sanitised CSR, clamped walk), device_status
    reports the problem, and the next valid call reuses the same scratch array
    and is right again."""
    import torch
    inp, pp = synth.random_case(79, n_fft=20, n_bins=60, n_fdot=40, n_dir=1, p=0.4)
    out = torch.empty(4096 * 48, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    dev = _dev(inp)
    off = inp.offsets.copy()
    off[5] = inp.n_peaks + 1000          # out of range
    off[6] = -3                          # negative and decreasing
    f = inp.freq.copy()
    for i in range(inp.t.shape[0]):      # every FFT's frequencies descending
        a, b = int(inp.offsets[i]), int(inp.offsets[i + 1])
        f[a:b] = f[a:b][::-1]
    bad = [dev[0], torch.from_numpy(off).cuda(), torch.from_numpy(f).cuda(), dev[3], dev[4]]
    _, st, _ = _static_path(fh, bad, pp, out, status, 0)
    assert st != 0
    got, st, drop = _static_path(fh, dev, pp, out, status, 0)
    assert st == 0 and drop == 0
    _same_as_oracle(got, oracle_mod.search(inp, pp), pp)


def test_static_refuses_sizes_beyond_its_maximum(fh):
    import torch
    inp, pp = synth.random_case(78, n_fft=10, n_bins=20, n_dir=1, p=0.3)
    dev = _dev(inp)
    out = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    too_wide = dict(pp, n_f0=(1 << 18) + 10)
    with pytest.raises(fh.FHError) as ei:
        fh.fh_search_static(too_wide, *dev, out)
    assert ei.value.code == fh.FH_ERR_TOO_LARGE
    with pytest.raises(fh.FHError) as ei:      # host memory is not accepted
        fh.fh_search_static(pp, inp.t, inp.offsets, inp.freq, inp.v, inp.sky, out)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG
