"""A plan's step captured into a CUDA graph and replayed (batching row a7).

After one eager call of the same shape (which sizes the plan's window table),
fh_correct_doppler on device inputs, fh_transform and fh_select_candidates
into device memory enqueue only kernels, memsets and device copies, so the
sequence can be captured and replayed.  Checked here through the C ABI: each
replay's candidates equal a fresh eager plan's, bit for bit, and the CPU
oracle's (cells, rows and counts bit for bit; f0, fdot and CR to 1e-12
relative), including after the device inputs were overwritten in place (same
addresses, new contents).
"""
import numpy as np
import pytest

from paper_1407_8333_gb300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12


def _same_as_oracle(got, o, pp, n_dir):
    c = got.reshape(n_dir, -1, pp["top_k"])
    for k in ("cell", "row", "count"):
        assert np.array_equal(c[k], o[k]), k
    for k in ("f0", "fdot", "cr"):
        a, b = c[k], o[k]
        same = (a == b) | (np.isnan(a) & np.isnan(b))
        assert np.all(same | (np.abs(a - b) <= REL_TOL * np.abs(b))), k


@pytest.fixture(scope="module")
def fh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_8333_gb300 import build, fh as fhmod
    build.build()
    fhmod.load()
    return fhmod


def _eager(fh, inp, pp, n_dir, schedule):
    import torch
    plan = fh.fh_create_plan(fh.make_desc(pp, inp.t.shape[0], n_dir, inp.n_peaks,
                                          schedule=schedule))
    try:
        dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        fh.fh_correct_doppler(plan, *dev)
        fh.fh_transform(plan, 0, n_dir)
        return fh.fh_select_candidates(plan, 0, n_dir)
    finally:
        fh.fh_destroy_plan(plan)


@pytest.mark.parametrize("schedule", [0, 1])
def test_step_replays_from_a_cuda_graph(fh, oracle_mod, schedule):
    import torch
    inp, pp = synth.random_case(91, n_fft=48, n_bins=160, n_fdot=70, n_dir=3, p=0.3)
    n_dir = inp.sky.shape[0]
    # a second input of the same shape: frequencies one bin higher, other velocities
    inp2 = synth.Inputs(w=inp.w, t=inp.t, offsets=inp.offsets,
                        freq=inp.freq + 1.0 / pp["t_fft"], v=inp.v[::-1].copy(), sky=inp.sky)
    want = [_eager(fh, x, pp, n_dir, schedule) for x in (inp, inp2)]
    oracle = [oracle_mod.search(x, pp) for x in (inp, inp2)]

    plan = fh.fh_create_plan(fh.make_desc(pp, inp.t.shape[0], n_dir, inp.n_peaks,
                                          schedule=schedule))
    try:
        dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
        n_sb = -(-pp["n_f0"] // pp["subband_cells"])
        cand = torch.zeros(n_dir * n_sb * pp["top_k"] * 48, dtype=torch.uint8, device="cuda")
        s = torch.cuda.Stream()

        def step():
            fh.fh_correct_doppler(plan, *dev, stream=s)
            fh.fh_transform(plan, 0, n_dir, None, stream=s)
            fh.fh_select_candidates(plan, 0, n_dir, cand, stream=s)

        with torch.cuda.stream(s):
            step()                      # eager: sizes the plan's buffers
        torch.cuda.synchronize()
        launches = fh.fh_plan_launches(plan)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            step()
        captured = fh.fh_plan_launches(plan) - launches
        assert captured > 0

        def replay():
            cand.zero_()
            g.replay()
            torch.cuda.synchronize()
            fh.fh_sync(plan)            # device-side input checks stayed clean
            return cand.cpu().numpy().view(fh.CANDIDATE_DTYPE).copy()

        for k in range(2):
            got = replay()
            assert np.array_equal(got, want[0]), k
            _same_as_oracle(got, oracle[0], pp, n_dir)
        # new contents at the same addresses
        dev[2].copy_(torch.from_numpy(inp2.freq))
        dev[3].copy_(torch.from_numpy(inp2.v))
        got = replay()
        assert np.array_equal(got, want[1])
        _same_as_oracle(got, oracle[1], pp, n_dir)
        assert not np.array_equal(want[0], want[1])
    finally:
        torch.cuda.synchronize()
        fh.fh_destroy_plan(plan)
