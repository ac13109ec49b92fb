"""Serving (continuous batching) through fh_submit / fh_poll.

Each job's candidates must be bit-identical whether the job runs alone or in
a concurrent mix (integer results: tolerance 0), and equal to the oracle's.
Failure paths are made on the host: a job larger than the budget, invalid
inputs, a cancelled job, and a stuck (paused) queue that makes a bounded
drain time out -- no GPU fault is involved.
"""
import time

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


def _jobs():
    jobs = []
    for i, (n_fft, n_bins, K, n_fdot, n_dir) in enumerate(
            [(30, 80, 10, 40, 3), (50, 120, 10, 70, 1), (20, 64, 7, 33, 5), (64, 200, 10, 12, 2),
             (40, 90, 3, 50, 4), (25, 300, 10, 5, 7)]):
        inp, pp = synth.random_case(100 + i, n_fft=n_fft, n_bins=n_bins, k_over=K, n_fdot=n_fdot,
                                    n_dir=n_dir, p=0.3, top_k=3, excl_cells=2 * K, sep_cells=4 * K)
        jobs.append((inp, pp))
    return jobs


def _submit(fh, sv, inp, pp):
    return fh.fh_submit(sv, pp, inp.t, inp.offsets, inp.freq, inp.v, inp.sky)


def _wait(fh, sv, jid, timeout=120.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        st, out = fh.fh_poll(sv, jid)
        if st == fh.FH_JOB_DONE:
            return out
        time.sleep(0.002)
    raise AssertionError("job %d not done" % jid)


def test_alone_equals_mix_equals_oracle(fh, oracle_mod):
    jobs = _jobs()
    want = [oracle_mod.search(inp, pp) for inp, pp in jobs]
    # alone: one job at a time, one stream
    sv = fh.fh_server_create(1 << 30, 1)
    try:
        alone = [_wait(fh, sv, _submit(fh, sv, inp, pp)) for inp, pp in jobs]
    finally:
        fh.fh_server_destroy(sv)
    # mix: everything submitted at once, 3 streams, then a second wave while the
    # first is on the GPU
    sv = fh.fh_server_create(1 << 30, 3)
    try:
        ids = [_submit(fh, sv, inp, pp) for inp, pp in jobs[:3]]
        ids += [_submit(fh, sv, inp, pp) for inp, pp in jobs[3:]]
        fh.fh_server_drain(sv, 120.0)
        mix = [fh.fh_poll(sv, i)[1] for i in ids]
        stats = [fh.fh_job_get_stats(sv, i) for i in ids]
    finally:
        fh.fh_server_destroy(sv)
    for (inp, pp), a, m, o in zip(jobs, alone, mix, want):
        assert a.tobytes() == m.tobytes()
        c = m.reshape(inp.sky.shape[0], -1, pp["top_k"])
        assert np.array_equal(c["cell"], o["cell"])
        assert np.array_equal(c["row"], o["row"])
        assert np.array_equal(c["count"], o["count"])
    assert all(s["done_s"] >= s["start_s"] >= s["submit_s"] for s in stats)
    assert max(s["batch_jobs"] for s in stats) >= 2    # batching happened


def test_budget_admission_and_too_large(fh):
    (inp, pp) = _jobs()[0]
    sv = fh.fh_server_create(4096, 2)      # 4 KiB: this job cannot fit
    try:
        with pytest.raises(fh.FHError) as ei:
            _submit(fh, sv, inp, pp)
        assert ei.value.code == fh.FH_ERR_TOO_LARGE
    finally:
        fh.fh_server_destroy(sv)
    # a budget that fits one job at a time: everything still completes, one per batch
    sv = fh.fh_server_create(1 << 30, 4)
    try:
        jid = _submit(fh, sv, inp, pp)
        _wait(fh, sv, jid)
        need = fh.fh_job_get_stats(sv, jid)["device_bytes"]
    finally:
        fh.fh_server_destroy(sv)
    sv = fh.fh_server_create(int(need * 1.5), 4)
    try:
        ids = [_submit(fh, sv, inp, pp) for _ in range(4)]
        fh.fh_server_drain(sv, 60.0)
        st = [fh.fh_job_get_stats(sv, i) for i in ids]
        assert all(s["batch_jobs"] == 1 for s in st)
        outs = [fh.fh_poll(sv, i)[1].tobytes() for i in ids]
        assert len(set(outs)) == 1
    finally:
        fh.fh_server_destroy(sv)


def test_invalid_job_rejected_at_submit(fh):
    (inp, pp) = _jobs()[1]
    sv = fh.fh_server_create(1 << 30, 2)
    try:
        f = inp.freq.copy()
        f[[0, 1]] = f[[1, 0]]
        with pytest.raises(fh.FHError) as ei:
            fh.fh_submit(sv, pp, inp.t, inp.offsets, f, inp.v, inp.sky)
        assert ei.value.code == fh.FH_ERR_UNSORTED
        bad = dict(pp, k_over=0)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_submit(sv, bad, inp.t, inp.offsets, inp.freq, inp.v, inp.sky)
        assert ei.value.code == fh.FH_ERR_INVALID_ARG
        with pytest.raises(fh.FHError) as ei:
            fh.fh_poll(sv, 12345)
        assert ei.value.code == fh.FH_ERR_BAD_HANDLE
    finally:
        fh.fh_server_destroy(sv)


def test_stuck_queue_times_out_then_recovers_and_cancel(fh):
    (inp, pp) = _jobs()[2]
    sv = fh.fh_server_create(1 << 30, 2)
    try:
        fh.fh_server_pause(sv, True)         # simulated stuck admission
        a = _submit(fh, sv, inp, pp)
        b = _submit(fh, sv, inp, pp)
        t0 = time.time()
        with pytest.raises(fh.FHError) as ei:
            fh.fh_server_drain(sv, 0.3)
        assert ei.value.code == fh.FH_ERR_TIMEOUT
        assert 0.25 < time.time() - t0 < 5.0
        assert fh.fh_poll(sv, a)[0] == fh.FH_JOB_QUEUED
        fh.fh_cancel(sv, b)
        with pytest.raises(fh.FHError) as ei:
            fh.fh_poll(sv, b)
        assert ei.value.code == fh.FH_ERR_CANCELLED
        fh.fh_server_pause(sv, False)
        fh.fh_server_drain(sv, 60.0)
        assert fh.fh_poll(sv, a)[0] == fh.FH_JOB_DONE
        with pytest.raises(fh.FHError):
            fh.fh_cancel(sv, a)               # no longer queued
    finally:
        fh.fh_server_destroy(sv)


def test_destroy_with_queued_jobs(fh):
    (inp, pp) = _jobs()[3]
    sv = fh.fh_server_create(1 << 30, 1)
    fh.fh_server_pause(sv, True)
    for _ in range(3):
        _submit(fh, sv, inp, pp)
    fh.fh_server_destroy(sv)                 # cancels the queue, returns promptly


def test_served_jobs_of_the_stream_shapes_alone_mix_oracle(fh, oracle_mod):
    """One job of every shape the served stream draws (T_FFT 8192/4096/2048/1024 s
    x band 0.25/0.5/1/2 Hz, K = 10, the spin-down grid of 150 days: 1169 / 585 /
    293 / 147 rows) with 5 % of the FFTs and 1..32 directions: each job's
    candidates are the same bytes alone and in the concurrent mix, and equal the
    oracle's on a sampled direction (Sec. VIII: bands are searched
    independently)."""
    import math
    from paper_1407_8333_gb300 import serve
    pool = serve.make_job_pool(4, scale_fft=0.05)
    jobs = []
    for k, (shape, inp) in enumerate(sorted(pool.items())):
        w = inp.w
        n_dir = [1, 3, 7, 12, 19, 32, 5, 2][k % 8]
        grid = synth.ecliptic_grid(max(2.0, min(synth.doppler_number(w.f_hi, w.t_fft), 60.0)))
        idx = (7 * k + np.arange(n_dir)) % len(grid)
        jobs.append((shape, synth.Inputs(w=w, t=inp.t, offsets=inp.offsets, freq=inp.freq,
                                         v=inp.v, sky=np.ascontiguousarray(grid[idx]))))
    rows = {t: jobs_pp["n_fdot"] for t, jobs_pp in
            ((s[0], i.w.plan_params()) for s, i in jobs)}
    assert rows == {8192.0: 1169, 4096.0: 585, 2048.0: 293, 1024.0: 147}
    sv = fh.fh_server_create(8 << 30, 1)
    try:
        alone = [_wait(fh, sv, _submit(fh, sv, inp, inp.w.plan_params()), timeout=300.0)
                 for _, inp in jobs]
    finally:
        fh.fh_server_destroy(sv)
    sv = fh.fh_server_create(8 << 30, 4)
    try:
        ids = [_submit(fh, sv, inp, inp.w.plan_params()) for _, inp in jobs]
        fh.fh_server_drain(sv, 300.0)
        mix = [fh.fh_poll(sv, i)[1] for i in ids]
        stats = [fh.fh_job_get_stats(sv, i) for i in ids]
    finally:
        fh.fh_server_destroy(sv)
    assert max(s["batch_jobs"] for s in stats) >= 2    # batching happened
    for k, ((shape, inp), a, m) in enumerate(zip(jobs, alone, mix)):
        assert a.tobytes() == m.tobytes(), shape
        pp = inp.w.plan_params()
        n_dir = inp.sky.shape[0]
        d = (3 * k) % n_dir
        one = synth.Inputs(w=inp.w, t=inp.t, offsets=inp.offsets, freq=inp.freq, v=inp.v,
                           sky=np.ascontiguousarray(inp.sky[[d]]))
        o = oracle_mod.search(one, pp)
        c = m.reshape(n_dir, -1, pp["top_k"])[d]
        for key in ("cell", "row", "count"):
            assert np.array_equal(c[key], o[key][0]), (shape, key)
        assert not math.isnan(float(c["f0"][0, 0]))
