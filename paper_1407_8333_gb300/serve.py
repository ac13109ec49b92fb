"""Served mixed stream: Poisson arrivals of Hough jobs through fh_submit/fh_poll.

Job mix shaped after the paper's SFDB organisation (band widths 0.25/0.5/1/2 Hz,
T_FFT in {8192, 4096, 2048, 1024} s with band starts in the frequency range
that suits each T_FFT, T_obs = 150 days, spin-down -1e-8 .. +1e-9 Hz/s, sky
patches of 1..512 directions, peak probability 0.03..0.05).  A small pool of
peakmaps per (T_FFT, band width) is generated once and reused by the jobs of
that shape (only the sky patch and the arrival time differ), so the stream
measures the library, not the generator.

``run_stream`` reports p50/p99 latency (submit -> done) and aggregate updates/s
for the served form, and the same job list run one job at a time through the
plain form (a plan per job, one launch per sky direction) for comparison.
"""
from __future__ import annotations

import math
import statistics
import time

import numpy as np

from . import fh, synth

DAY = 86400.0
_T_RANGES = {8192.0: (32.0, 128.0), 4096.0: (128.0, 512.0), 2048.0: (256.0, 1024.0),
             1024.0: (512.0, 2048.0)}
_BANDS = (0.25, 0.5, 1.0, 2.0)


def job_workload(t_fft: float, band: float, f_lo: float, p: float, n_dir: int, seed: int,
                 t_obs_days: float = 150.0, n_fft: int = None) -> synth.Workload:
    t_obs = t_obs_days * DAY
    n = n_fft if n_fft is not None else int(math.floor(t_obs / (0.5 * t_fft)))
    return synth.Workload(
        name="job_T%d_B%g_f%g" % (t_fft, band, f_lo), t_fft=t_fft, n_fft=n, t_step=0.5 * t_fft,
        t_obs=t_obs, f_lo=f_lo, f_hi=f_lo + band, k_over=10, p_peak=p, fdot_lo=-1e-8,
        fdot_hi=1e-9, doppler=True, n_dir=n_dir, subband_hz=min(0.1, band), top_k=2,
        excl_bins=4, sep_bins=8, seed=seed)


def make_job_pool(seed: int, scale_fft: float = 1.0):
    """One peakmap per (T_FFT, band width) shape; ``scale_fft`` < 1 shortens T_obs."""
    rng_u = synth.uniform(seed, 9, np.arange(64))
    pool = {}
    k = 0
    for t in _T_RANGES:
        for b in _BANDS:
            lo, hi = _T_RANGES[t]
            f_lo = round(lo + (hi - lo - b) * float(rng_u[k]), 2)
            p = 0.03 + 0.02 * float(rng_u[k + 16])
            n = max(8, int(math.floor(150 * DAY / (0.5 * t)) * scale_fft))
            w = job_workload(t, b, f_lo, p, 1, seed * 100 + k, n_fft=n)
            pool[(t, b)] = synth.make_inputs(w)
            k += 1
    return pool


def job_list(seed: int, n_jobs: int, pool, max_dir: int = 512):
    """(shape, n_dir, sky) per job; n_dir log-uniform in [1, max_dir]."""
    u = synth.uniform(seed, 10, np.arange(4 * n_jobs)).reshape(n_jobs, 4)
    shapes = list(pool.keys())
    jobs = []
    for i in range(n_jobs):
        shape = shapes[int(u[i, 0] * len(shapes)) % len(shapes)]
        n_dir = int(round(math.exp(u[i, 1] * math.log(max_dir))))
        n_dir = max(1, min(max_dir, n_dir))
        inp = pool[shape]
        w = inp.w
        n_d = synth.doppler_number(w.f_hi, w.t_fft)
        grid = synth.ecliptic_grid(max(2.0, min(n_d, 60.0)))
        start = int(u[i, 2] * len(grid))
        idx = (start + np.arange(n_dir)) % len(grid)
        jobs.append((shape, n_dir, np.ascontiguousarray(grid[idx])))
    return jobs


def _updates(inp, n_dir):
    return inp.n_peaks * inp.w.n_fdot * n_dir


def _percentiles(lat):
    return 1e3 * float(np.percentile(lat, 50)), 1e3 * float(np.percentile(lat, 99))


def run_plain(pool, jobs, arrivals=None, plans=None):
    """Plain form: one job at a time in arrival order (a single FIFO queue), one
    launch per sky direction, a plan per job shape created beforehand.  Latency
    = completion - arrival."""
    import torch
    own = plans is None
    if own:
        plans = make_plain_plans(pool, max(n for _, n, _ in jobs))
    lat = []
    try:
        t0 = time.perf_counter()
        for k, (shape, n_dir, sky) in enumerate(jobs):
            at = 0.0 if arrivals is None else float(arrivals[k])
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            inp = pool[shape]
            plan = plans[shape]
            fh.fh_correct_doppler(plan, inp.t, inp.offsets, inp.freq, inp.v, sky)
            fh.fh_transform(plan, 0, n_dir)
            fh.fh_select_candidates(plan, 0, n_dir)
            lat.append(time.perf_counter() - t0 - at)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    finally:
        if own:
            for pl in plans.values():
                fh.fh_destroy_plan(pl)
    upd = sum(_updates(pool[s], n) for s, n, _ in jobs)
    p50, p99 = _percentiles(lat)
    return {"jobs": len(jobs), "wall_s": wall, "updates_per_s": upd / wall, "p50_ms": p50,
            "p99_ms": p99}


def make_plain_plans(pool, max_dir):
    plans = {}
    for shape, inp in pool.items():
        pp = inp.w.plan_params()
        plans[shape] = fh.fh_create_plan(fh.make_desc(pp, inp.w.n_fft, max_dir, inp.n_peaks,
                                                      schedule=fh.FH_SCHED_PLAIN))
    return plans


def run_served(pool, jobs, arrivals, budget_bytes: int, max_inflight: int = 4,
               timeout_s: float = 600.0):
    """Submit job i at arrivals[i] seconds, drain, return latency figures and results."""
    sv = fh.fh_server_create(budget_bytes, max_inflight)
    ids = []
    try:
        t0 = time.perf_counter()
        for (shape, n_dir, sky), at in zip(jobs, arrivals):
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            inp = pool[shape]
            ids.append(fh.fh_submit(sv, inp.w.plan_params(), inp.t, inp.offsets, inp.freq,
                                    inp.v, sky))
        fh.fh_server_drain(sv, timeout_s)
        wall = time.perf_counter() - t0
        stats = [fh.fh_job_get_stats(sv, i) for i in ids]
        results = [fh.fh_poll(sv, i)[1] for i in ids]
    finally:
        fh.fh_server_destroy(sv)
    lat = [s["done_s"] - s["submit_s"] for s in stats]
    upd = sum(s["updates"] for s in stats)
    first = min(s["submit_s"] for s in stats)
    last = max(s["done_s"] for s in stats)
    batches = {}
    for s in stats:
        batches.setdefault(s["batch"], s["batch_jobs"])
    p50, p99 = _percentiles(lat)
    return {"jobs": len(jobs), "wall_s": wall, "updates_per_s": upd / (last - first),
            "p50_ms": p50, "p99_ms": p99, "batches": len(batches),
            "mean_jobs_per_batch": statistics.mean(batches.values()),
            "max_inflight": max_inflight}, results


def run_stream(seconds: float = 8.0, seed: int = 4, scale_fft: float = 0.25, max_dir: int = 128,
               load: float = 0.7):
    """Served stream vs plain form on the same job list and the same arrivals.

    The served capacity is measured first with a burst (all jobs at t = 0);
    the Poisson arrival rate is then `load` x that capacity."""
    import torch
    pool = make_job_pool(seed, scale_fft=scale_fft)
    budget = int(0.5 * torch.cuda.get_device_properties(0).total_memory)
    burst = job_list(seed + 1, 48, pool, max_dir)
    cap, _ = run_served(pool, burst, np.zeros(len(burst)), budget)
    rate = load * cap["jobs"] / cap["wall_s"]
    n_jobs = max(16, min(600, int(seconds * rate)))
    jobs = job_list(seed, n_jobs, pool, max_dir)
    gaps = -np.log(1.0 - synth.uniform(seed, 11, np.arange(n_jobs))) / rate
    arrivals = np.cumsum(gaps) - gaps[0]
    served, _ = run_served(pool, jobs, arrivals, budget)
    plans = make_plain_plans(pool, max_dir)
    try:
        plain = run_plain(pool, jobs, arrivals, plans)
    finally:
        for pl in plans.values():
            fh.fh_destroy_plan(pl)
    return {"stream": ("Poisson arrivals at %.1f jobs/s (%.0f%% of the served burst capacity); "
                       "job shapes T_FFT {8192,4096,2048,1024} s x band {0.25,0.5,1,2} Hz, "
                       "T_obs 150 d x %.2g, 1..%d directions, p 0.03-0.05"
                       % (rate, 100 * load, scale_fft, max_dir)),
            "served_burst": cap, "served": served, "plain": plain,
            "p50_ratio_plain_over_served": plain["p50_ms"] / served["p50_ms"],
            "p99_ratio_plain_over_served": plain["p99_ms"] / served["p99_ms"],
            "speedup_updates_per_s": served["updates_per_s"] / plain["updates_per_s"]}
