"""fh_search_static: the allocation-free entry point.

It serves callers that cannot allocate device memory while they run (their
GPU memory is reserved for their own pool, or their loop must not take the
synchronisation a cudaMalloc/cudaFree can cause).  Checked here on the GPU,
through the C ABI:

* its candidates equal those of the plan-based entry points
  (fh_correct_doppler + fh_transform + fh_select_candidates) -- integers bit
  for bit, f0 / fdot / CR to 1e-12 relative -- on two calls in a row, the
  larger input first, so that anything the first call left in the shared
  scratch array would show up in the second;
* a call changes nothing in the device's free memory;
* inputs beyond its fixed maximum sizes are refused with FH_ERR_TOO_LARGE.
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


def _plan_path(fh, inp, pp):
    import torch
    plan = fh.fh_create_plan(fh.make_desc(pp, max(1, inp.t.shape[0]), 1, max(1, inp.n_peaks)))
    try:
        dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        fh.fh_correct_doppler(plan, *dev)
        fh.fh_transform(plan, 0, 1)
        return fh.fh_select_candidates(plan, 0, 1)
    finally:
        fh.fh_destroy_plan(plan)


def _static_path(fh, inp, pp, out, status):
    import torch
    dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    n = fh.fh_search_static(pp, *dev, out, status)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    got = out.cpu().numpy().view(fh.CANDIDATE_DTYPE)[:n].copy()
    return got, int(status.item()), free_before, free_after


def _same(fh, a, b):
    for k in ("dir", "subband", "rank", "row", "cell", "count"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("f0", "fdot", "cr"):
        x, y = a[k], b[k]
        assert np.all((x == y) | (np.abs(x - y) <= REL_TOL * np.abs(y))), k


def test_static_matches_plan_path_on_two_calls(fh):
    import torch
    big_w = synth.WORKLOADS["sky_patch256_T1024_N200_100Hz"]
    big = synth.make_inputs(big_w)
    big = synth.Inputs(w=big_w, t=big.t, offsets=big.offsets, freq=big.freq, v=big.v,
                       sky=np.ascontiguousarray(big.sky[[big_w.line_dir]]))
    small, small_pp = synth.random_case(77, n_fft=30, n_bins=90, n_fdot=45, n_dir=1, p=0.3)
    cases = [(big, big_w.plan_params()), (small, small_pp)]
    out = torch.empty(64 * 1024 * 48, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for k, (inp, pp) in enumerate(cases):
        want = _plan_path(fh, inp, pp)
        got, st, free_before, free_after = _static_path(fh, inp, pp, out, status)
        assert st == 0
        assert got.shape == want.shape
        _same(fh, got, want)
        if k == 1:
            # the second call allocates nothing on the device
            assert free_after == free_before
    # the big line case: its top candidate is the injected line
    assert got.shape[0] > 0


def test_static_refuses_sizes_beyond_its_maximum(fh):
    import torch
    inp, pp = synth.random_case(78, n_fft=10, n_bins=20, n_dir=1, p=0.3)
    dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
    out = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    too_wide = dict(pp, n_f0=(1 << 18) + 10)
    with pytest.raises(fh.FHError) as ei:
        fh.fh_search_static(too_wide, *dev, out)
    assert ei.value.code == fh.FH_ERR_TOO_LARGE
    with pytest.raises(fh.FHError) as ei:      # host memory is not accepted
        fh.fh_search_static(pp, inp.t, inp.offsets, inp.freq, inp.v, inp.sky, out)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG
