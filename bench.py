#!/usr/bin/env python
"""Benchmark of the GB300 frequency-Hough path.

One step = one pass of the whole hot path over one batch of synthetic input:
Doppler correction + fixed-point positions + shift tables (fh_correct_doppler),
transform + profile (fh_transform), candidate selection (fh_select_candidates).

Default workload: one sky point at the paper's low-frequency scale --
T_FFT = 8192 s, half-interlaced over 150 days (3164 FFTs), 50-51 Hz with
K = 10 (81920 cells), spin-down -1e-8 .. +1e-9 Hz/s (1169 rows), peak
probability 0.04 (~1.18M peaks), top-5 per 0.1 Hz sub-band.

Printed: one JSON line (rank 0) with throughput in peak x spin-down updates/s
(device-resident inputs), the end-to-end figure through the C ABI with host
buffers, the roofline of the transform kernel, the oracle's CPU baseline,
SM clocks sampled during the timed region, the plain vs batched comparison
on a 256-direction sky patch and the served-stream latency figures.

``--impl reference`` times the CPU oracle (the benchmark's reference arm)
on the same workload instead.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FH peak×spindown updates/s, 1 GB300; served-job p50/p99 latency vs plain"
UNIT = "updates/s"
WORKLOAD = "single_sky_T8192_150d_50Hz"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-extras", action="store_true", help="skip batched/serving/cpu legs")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--legs", default="maps,adaptive,batched,serving,refine,peakmap,coincidences,"
                                      "highfreq,cpu",
                    help="extra legs to run after the timed step (comma list)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def config_of(w, extra=None):
    pp = w.plan_params()
    cfg = {"workload": w.name,
           "description": ("T_FFT=%g s, %d FFTs (start spacing %g s), band %.2f-%.2f Hz, K=%d "
                           "(%d cells), %d spin-down rows (%.3g..%.3g Hz/s), p=%.3g, %d sky "
                           "direction(s), top-%d per %.2g Hz" %
                           (w.t_fft, w.n_fft, w.t_step, w.f_lo, w.f_hi, w.k_over, pp["n_f0"],
                            pp["n_fdot"], pp["fdot_min"],
                            pp["fdot_min"] + (pp["n_fdot"] - 1) * pp["fdot_step"], w.p_peak,
                            w.n_dir, w.top_k, w.subband_hz)),
           "l2": "flushed between timed steps (256 MiB write)"}
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="fh_clocks_%d_" % self.gpu, suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(open(self.path)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax.append(float(row[2]))
            except ValueError:
                continue
            for n, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- helpers
def transform_traffic():
    """DRAM bytes per transform launch from the committed ncu summary, if the
    transform section of the kernel source is still the one that was profiled."""
    import hashlib
    import re
    try:
        src = open(os.path.join(ROOT, "paper_1407_8333_gb300", "csrc", "fh_kernels.cu")).read()
        a = src.index("// ---------------------------------------------------------------- a4 + a5 + profile")
        b = src.index("// ---------------------------------------------------------------- a6")
        sha = hashlib.sha1(src[a:b].encode()).hexdigest()
        md = open(os.path.join(ROOT, "profiles", "transform_single_sky_T8192_150d_50Hz.md")).read()
        m = re.search(r"traffic: dram_bytes_per_launch=(\d+) transform_source_sha1=([0-9a-f]+)", md)
        if m and m.group(2) == sha:
            return int(m.group(1))
    except (OSError, ValueError):
        pass
    return None


def peaks_path():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0}, "fallback"


def cpu_baseline_leg(inp, pp, budget_s=12.0, refine_args=None, peakmap=None, coinc=None,
                     highfreq=None):
    """The oracle as it stands, whole path a1-a6 on the same workload, with all
    host threads and with one (and, given refine_args = (cells, rows, sky_ref,
    k_fdot), its refined-grid search on a few of the workload's candidates;
    given highfreq = (inputs, params), one of the 900 Hz workload's 64
    directions, whose rate stands for all 64)."""
    import numpy as np
    import oracle
    oracle.build()
    ref = None
    if refine_args is not None:
        cells, rows, sky_ref, k_fdot = refine_args
        t0 = time.perf_counter()
        oracle.refine(inp, pp, cells, rows, sky_ref, k_fdot)
        dt = time.perf_counter() - t0
        ref = {"candidates_per_s": len(cells) / dt, "cores": oracle.num_threads(),
               "sample": "%d candidates, %d refined directions, K_fdot = %d, one run (%.2f s)"
                         % (len(cells), sky_ref.shape[1], k_fdot, dt)}
    upd = inp.n_peaks * pp["n_fdot"] * inp.sky.shape[0]
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        oracle.search(inp, pp)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s or len(times) >= 5:
            break
    best = min(times)
    out = {"value": upd / best, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": "whole path a1-a6 (maps, profile, selection) on the full workload, "
                     "1 direction, best of %d runs (%.2f s each)" % (len(times), best)}
    n_thr = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.search(inp, pp)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(n_thr)
    out["one_thread"] = {"value": upd / dt1, "unit": UNIT, "cores": 1,
                         "sample": "the same whole path on one thread, one run (%.2f s)" % dt1}
    if highfreq is not None:
        hinp, hpp = highfreq
        from paper_1407_8333_gb300 import synth
        d = hinp.w.line_dir
        one = synth.Inputs(w=hinp.w, t=hinp.t, offsets=hinp.offsets, freq=hinp.freq, v=hinp.v,
                           sky=np.ascontiguousarray(hinp.sky[[d]]))
        t0 = time.perf_counter()
        oracle.search(one, hpp)
        dth = time.perf_counter() - t0
        hupd = one.n_peaks * hpp["n_fdot"]
        out["highfreq"] = {"value": hupd / dth, "unit": UNIT, "cores": n_thr,
                           "sample": "whole path on direction %d of the 900 Hz workload's 64 "
                                     "(%.3g updates, one run, %.2f s); the per-update rate "
                                     "stands for all 64" % (d, hupd, dth)}
    if ref is not None:
        out["refine"] = ref
    if coinc is not None:
        a, b = coinc
        t0 = time.perf_counter()
        oracle.coincidence.cluster(a, 4.0)
        t1 = time.perf_counter()
        oracle.coincidence.coincidences(a, b, 1.0e6, 2.0e6, 1.5e6, (2, 2, 2, 2))
        t2 = time.perf_counter()
        out["coincidences"] = {"cluster_candidates_per_s": len(a) / (t1 - t0),
                               "coincidence_candidates_per_s": 2 * len(a) / (t2 - t1),
                               "cores": 1,
                               "sample": "%d candidates per set (numpy), one run each "
                                         "(%.2f s, %.2f s)" % (len(a), t1 - t0, t2 - t1)}
    if peakmap is not None:
        t0 = time.perf_counter()
        oracle.peakmap.select_peaks(peakmap.s_p, peakmap.s_ar, 2.5)
        dt = time.perf_counter() - t0
        n = peakmap.s_p.size
        out["peakmap"] = {"bins_per_s": n / dt, "cores": 1,
                          "sample": "peak selection of the whole peakmap workload (%d bins), "
                                    "numpy, one run (%.2f s)" % (n, dt)}
    return out


# ----------------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch

    from paper_1407_8333_gb300 import build, fh, replicas, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    fh.load()

    w = synth.WORKLOADS[args.workload]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    n_dir = inp.sky.shape[0]
    dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
    plan = fh.fh_create_plan(fh.make_desc(pp, w.n_fft, n_dir, inp.n_peaks))
    fh.fh_correct_doppler(plan, *dev)
    tile, warps = fh.fh_autotune(plan, 0, n_dir)
    n_sb = -(-pp["n_f0"] // pp["subband_cells"])
    cand = torch.empty(n_dir * n_sb * pp["top_k"] * 48, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    upd_step = inp.n_peaks * pp["n_fdot"] * n_dir

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        fh.fh_correct_doppler(plan, *dev, stream=stream)
        if ev:
            ev[1].record(stream)
        fh.fh_transform(plan, 0, n_dir, None, stream=stream)
        if ev:
            ev[2].record(stream)
        fh.fh_select_candidates(plan, 0, n_dir, cand, stream=stream)
        if ev:
            ev[3].record(stream)

    nvtx = torch.cuda.nvtx
    nvtx.range_push("warmup")
    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    nvtx.range_pop()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    # the library records events around its window pre-pass and transform kernel
    fh.fh_plan_set_timing(plan, True)
    l0 = fh.fh_plan_launches(plan)
    if world > 1:
        replicas.barrier()
    torch.cuda.synchronize()
    nvtx.range_push("timed")
    for k in range(args.steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize()
    nvtx.range_pop()
    if world > 1:
        replicas.barrier()
    launches = fh.fh_plan_launches(plan) - l0
    clocks = sampler.stop()
    n_groups, win_ms_sum, kern_ms_sum = fh.fh_plan_kernel_times(plan)
    fh.fh_plan_set_timing(plan, False)
    win_avg = win_ms_sum / n_groups
    kern_avg = kern_ms_sum / n_groups
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    tr_ms = [e[1].elapsed_time(e[2]) for e in evs]
    dop_ms = [e[0].elapsed_time(e[1]) for e in evs]
    sel_ms = [e[2].elapsed_time(e[3]) for e in evs]
    # the slowest replica's time (replicas: no data-path collective)
    total_ms = replicas.max_over_ranks(sum(step_ms))
    value = upd_step * args.steps * world / (total_ms * 1e-3)

    # roofline of the transform kernel (dominant): shared-memory atomics, one per
    # update, over that kernel's own event-timed launch duration
    atomic_peak, _ = fh.fh_bench_smem_atomics(0, 4096)
    tr_avg = statistics.mean(tr_ms)
    achieved_atom = upd_step / (kern_avg * 1e-3)
    peaks, peak_src = peaks_path()
    hbm_bytes = 8 * inp.n_peaks * n_dir + 8 * pp["n_f0"] * n_dir + 16 * w.n_fft
    roof = {"bound": "smem_atomic", "achieved": achieved_atom / 1e9, "peak": atomic_peak / 1e9,
            "unit": "Gatomic/s", "frac": achieved_atom / atomic_peak,
            "traffic": transform_traffic() if args.workload == WORKLOAD else None,
            "traffic_note": "dram__bytes_read+write per launch from profiles/transform_single_sky_T8192_150d_50Hz.md (null if the kernel changed since)",
            "kernel": "transform_kernel<FH_MODE_START>",
            "algorithmic": "1 shared-memory atomic per peak x spin-down update; %d updates per launch"
                           % upd_step,
            "peak_source": "own microbenchmark fh_bench_smem_atomics(0): conflict-free int32 "
                           "atomicAdd, all SMs, measured in this run",
            "duration_ms": kern_avg,
            "duration_note": "mean launch duration of transform_kernel over the timed steps, "
                             "CUDA events recorded by the library on the launching stream",
            "step_frac": upd_step / (tr_avg * 1e-3) / atomic_peak,
            "step_frac_note": "the same updates over fh_transform as a whole (window pre-pass "
                              "+ transform kernel)",
            "tile_cells": tile, "block_warps": warps}
    roof_hbm = {"bound": "hbm", "achieved": hbm_bytes / (kern_avg * 1e-3) / 1e9,
                "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                "frac": hbm_bytes / (kern_avg * 1e-3) / 1e9 / peaks.get("hbm_gbs"),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_src,
                "algorithmic": "8 B/peak (positions) + 8 B/cell (profile) + 16 B/FFT per launch"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "i64/i32 (f64 Doppler)",
           "data": "synthetic (seeded SplitMix64 peakmap, paper-shaped)",
           "config": config_of(w, {"parallelism": "replicas" if world > 1 else "single GPU",
                                   "inputs": "device-resident"}),
           "breakdown_ms": {"correct_doppler": statistics.mean(dop_ms),
                            "transform": tr_avg, "select": statistics.mean(sel_ms),
                            "transform_windows_kernel": win_avg,
                            "transform_kernel": kern_avg},
           "roofline": roof, "roofline_hbm": roof_hbm, "clocks": clocks,
           "gpu_launches": launches}

    # end to end through the C ABI with host buffers (pinned), H2D/D2H inside
    pinned = [torch.from_numpy(x).pin_memory().numpy() for x in
              (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
    # the host inputs are checked by the kernels (FH_CHECKS_DEVICE), so the
    # copies and the kernels start at once; errors would surface at the select
    fh.fh_plan_set_input_checks(plan, fh.FH_CHECKS_DEVICE)
    h2d = sum(x.nbytes for x in pinned)
    e2e_ms = []
    # page-locked candidate buffer: the read-back is one DMA, not a staged copy
    host_out = torch.zeros(n_dir * n_sb * pp["top_k"] * fh.CANDIDATE_DTYPE.itemsize,
                           dtype=torch.uint8).pin_memory().numpy().view(fh.CANDIDATE_DTYPE)
    for k in range(max(3, args.warmup) + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fh.fh_correct_doppler(plan, *pinned, stream=stream)
        fh.fh_transform(plan, 0, n_dir, None, stream=stream)
        fh.fh_select_candidates(plan, 0, n_dir, host_out, stream=stream)
        t1 = time.perf_counter()
        if k >= max(3, args.warmup):
            e2e_ms.append((t1 - t0) * 1e3)
    out["e2e"] = {"value": upd_step * len(e2e_ms) / (sum(e2e_ms) * 1e-3) * world, "unit": UNIT,
                  "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": host_out.nbytes,
                  "ms_per_step": statistics.mean(e2e_ms),
                  "input_checks": "device (FH_CHECKS_DEVICE): CSR, ordering, finiteness and "
                                  "range checked by the kernels, reported at the select",
                  "transfer": "page-locked host inputs read in place by the correction "
                              "kernels over the host link (one direction), candidates "
                              "read back into a page-locked buffer"}
    fh.fh_destroy_plan(plan)

    legs = set(args.legs.split(","))
    if rank == 0 and world == 1 and not args.no_extras:
        if "adaptive" in legs:
            out["adaptive"] = adaptive_leg(fh, inp, pp, dev, cand, flush, torch, args.steps)
        if "batched" in legs:
            out["batched_vs_plain"] = batched_vs_plain(fh, synth, torch)
        if "serving" in legs:
            try:
                out["serving"] = serving_leg(fh, synth, torch, args.serve_seconds)
            except Exception as e:  # report, do not hide
                out["serving"] = {"error": str(e)[:300]}
        ref_args = None
        if "refine" in legs:
            try:
                out["refine"], ref_args = refine_leg(fh, synth, w, inp, pp, host_out, args.steps)
            except Exception as e:  # report, do not hide
                out["refine"] = {"error": str(e)[:300]}
        if "peakmap" in legs:
            try:
                out["peakmap"] = peakmap_leg(fh, synth, torch, args.steps)
            except Exception as e:  # report, do not hide
                out["peakmap"] = {"error": str(e)[:300]}
        if "coincidences" in legs:
            try:
                out["coincidences"] = coincidence_leg(fh, synth, torch, args.steps)
            except Exception as e:  # report, do not hide
                out["coincidences"] = {"error": str(e)[:300]}
        if "maps" in legs:
            try:
                out["maps_written"] = maps_leg(fh, w, inp, pp, dev, flush, torch, args.steps)
            except Exception as e:  # report, do not hide
                out["maps_written"] = {"error": str(e)[:300]}
        hf_inputs = None
        if "highfreq" in legs:
            try:
                out["highfreq"], hf_inputs = highfreq_leg(fh, synth, torch, min(args.steps, 5))
            except Exception as e:  # report, do not hide
                out["highfreq"] = {"error": str(e)[:300]}
        if "cpu" in legs:
            out["cpu_baseline"] = cpu_baseline_leg(
                inp, pp, refine_args=ref_args,
                peakmap=synth.peakmap_workload() if "peakmap" in legs else None,
                coinc=coincidence_sets(synth, 5000, 1) if "coincidences" in legs else None,
                highfreq=hf_inputs)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def adaptive_leg(fh, inp, pp, dev, cand, flush, torch, steps):
    """The same workload as the adaptive map (Eq. ncountadap): weights with a
    sidereal-day modulation, 12 fraction bits, set after every correction (a
    new peakmap returns the plan to unit weights)."""
    import numpy as np
    n = inp.t.shape[0]
    w = (1.0 + 0.5 * np.cos(2 * np.pi * inp.t / 86164.09)).reshape(1, n)
    plan = fh.fh_create_plan(fh.make_desc(pp, n, 1, inp.n_peaks))
    try:
        fh.fh_correct_doppler(plan, *dev)
        fh.fh_autotune(plan, 0, 1)
        ts, kern = [], []
        fh.fh_plan_set_timing(plan, True)
        for k in range(3 + steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fh.fh_correct_doppler(plan, *dev)
            fh.fh_set_weights(plan, w, 12)
            fh.fh_transform(plan, 0, 1, None)
            fh.fh_select_candidates(plan, 0, 1, cand)
            e1.record()
            torch.cuda.synchronize()
            if k >= 3:
                ts.append(e0.elapsed_time(e1))
            if k == 2:
                fh.fh_plan_set_timing(plan, True)
        n_g, _, kms = fh.fh_plan_kernel_times(plan)
    finally:
        fh.fh_destroy_plan(plan)
    upd = inp.n_peaks * pp["n_fdot"]
    ms = statistics.mean(ts)
    return {"weights": "1 + 0.5 cos(2 pi t / sidereal day), 12 fraction bits",
            "ms_per_step": ms, "updates_per_s": upd / (ms * 1e-3),
            "transform_kernel_ms": kms / n_g}


def refine_leg(fh, synth, w, inp, pp, host_out, steps):
    """Refined-grid search (Sec. "Refined Grid in the parameter space") of every
    candidate the coarse step selected: a 3 x 3 refined sky rectangle around
    its direction, the spin-down step refined by 4, through the host API
    (host peakmap and candidates in, refined candidates out, copies included)."""
    import numpy as np
    cand = host_out[host_out["count"] >= 0]
    cells = cand["cell"].astype(np.int32)
    rows = cand["row"].astype(np.int32)
    n_d = synth.doppler_number(w.f_hi, w.t_fft)
    sky = np.stack([synth.refined_sky(inp.sky[int(c["dir"])], n_d, 3) for c in cand])
    k_fdot = 4
    import torch
    plan = fh.fh_create_plan(fh.make_desc(pp, inp.t.shape[0], 1, inp.n_peaks))
    # pinned host inputs, checked by the kernels (FH_CHECKS_DEVICE)
    pin = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
           for x in (inp.t, inp.offsets, inp.freq, inp.v, sky)]
    fh.fh_plan_set_input_checks(plan, fh.FH_CHECKS_DEVICE)
    try:
        ts = []
        for k in range(2 + steps):
            t0 = time.perf_counter()
            r = fh.fh_refine(plan, pin[0], pin[1], pin[2], pin[3], cells, rows, pin[4], k_fdot)
            if k >= 2:
                ts.append((time.perf_counter() - t0) * 1e3)
    finally:
        fh.fh_destroy_plan(plan)
    ms = statistics.median(ts)
    gain = r["count"].astype(np.int64) - cand["count"].astype(np.int64)
    res = {"n_cand": int(cand.shape[0]), "n_ref": int(sky.shape[1]), "k_fdot": k_fdot,
           "ms_per_call": ms, "candidates_per_s": cand.shape[0] / (ms * 1e-3),
           "count_gain_median": float(np.median(gain)) if gain.size else None,
           "inputs": "host (pinned) peakmap copied every call, checked by the kernels"}
    sel = slice(0, min(3, cand.shape[0]))
    return res, (cells[sel], rows[sel], sky[sel], k_fdot)


def peakmap_leg(fh, synth, torch, steps):
    """Peakmap construction (Eq. pm) and cleaning on the 150-day, 1 Hz workload
    (3164 FFTs x 8192 bins, 207 MB of binary32 spectra, more than L2): the
    selection timed on the device around its asynchronous call (three kernels);
    the two vetoes as host calls (each synchronises)."""
    p = synth.PEAKMAP_PARAMS
    s = synth.peakmap_workload()
    sp = torch.from_numpy(s.s_p).cuda()
    sa = torch.from_numpy(s.s_ar).cuda()
    t = torch.from_numpy(s.t).cuda()
    n_fft, n_bins = s.s_p.shape
    cap = n_fft * n_bins // 4
    out = (torch.empty(n_fft + 1, dtype=torch.int64, device="cuda"),
           torch.empty(cap, dtype=torch.int32, device="cuda"),
           torch.empty(cap, dtype=torch.float64, device="cuda"))
    ws = torch.empty(fh.fh_peakmap_select_workspace(n_fft, n_bins), dtype=torch.uint8,
                     device="cuda")
    # back-to-back selections between one pair of events (the host enqueues
    # faster than the device runs them, so the device time is measured);
    # 207 MB of input per call is more than L2 holds
    for k in range(3):
        fh.fh_peakmap_select(sp, sa, p["theta"], s.k0, s.t_fft, out=out, workspace=ws)
    torch.cuda.synchronize()
    ms = []
    for rep in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(max(1, steps)):
            fh.fh_peakmap_select(sp, sa, p["theta"], s.k0, s.t_fft, out=out, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1) / max(1, steps))
    n_peaks = int(out[0][-1].item())
    o, b = out[0], out[1][:n_peaks]
    grid = (0.0, p["dt_h"], p["n_th"], p["f0_h"], p["df_h"], p["n_fh"])
    g_ms, c_ms = [], []
    for k in range(2 + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        go, gb, _, gh = fh.fh_peakmap_gross_veto(t, o, b, s.k0, s.t_fft, *grid, p["gross_thr"])
        t1 = time.perf_counter()
        po, pb, _, ph, st = fh.fh_peakmap_persistency_veto(go, gb, n_bins, p["k_sigma"], s.k0,
                                                           s.t_fft)
        t2 = time.perf_counter()
        if k >= 2:
            g_ms.append((t1 - t0) * 1e3)
            c_ms.append((t2 - t1) * 1e3)
    sel = statistics.median(ms)
    alg = 8 * n_fft * n_bins + 12 * n_peaks
    peaks, src = peaks_path()
    gbs = alg / (sel * 1e-3) / 1e9
    return {"workload": "peakmap_T8192_150d_1Hz: 3164 FFTs x 8192 bins, theta 2.5, "
                        "gross 12 h x 0.01 Hz (threshold 100), persistency k = 5",
            "select_ms": sel, "bins_per_s": n_fft * n_bins / (sel * 1e-3),
            "n_peaks": n_peaks, "after_gross": int(gb.shape[0]),
            "after_persistency": int(pb.shape[0]),
            "gross_veto_ms": statistics.median(g_ms),
            "persistency_veto_ms": statistics.median(c_ms),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs"),
                         "unit": "GB/s", "frac": gbs / peaks.get("hbm_gbs"),
                         "algorithmic": "8 B per bin (two binary32 spectra) + 12 B per peak "
                                        "(bin, frequency) per selection",
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % src,
                         "duration_note": "CUDA events around back-to-back asynchronous "
                                          "fh_peakmap_select calls with a workspace, per "
                                          "call (median of 3 runs)"}}


def coincidence_sets(synth, n, bands, seed=51):
    """Two candidate sets of n each over `bands` 1 Hz bands at 100 Hz (T_FFT
    1024 s, sky uniform, 100 spin-down rows), n / 100 sources present in both
    (the second set at its own reference time, 1e6 s later), n / 50 clusters
    of 6 per set."""
    import numpy as np
    seeds = synth.candidate_set(seed, 0, n // 100, band=float(bands))[:, :4]
    later = seeds.copy()
    later[:, 2] += later[:, 3] * 1.0e6
    a = synth.candidate_set(seed, 1, n, band=float(bands), signals=seeds, clusters=n // 50,
                            cluster_size=6)
    b = synth.candidate_set(seed, 2, n, band=float(bands), signals=later, clusters=n // 50,
                            cluster_size=6)
    return np.ascontiguousarray(a), np.ascontiguousarray(b)


def coincidence_leg(fh, synth, torch, steps):
    """Clustering (d <= 4, Eq. norm) and coincidences (windows of 2 bins in
    every parameter, frequencies at the common time) through the host API
    (device candidates; each call synchronises)."""
    res = {}
    for n, bands in ((100000, 1), (1000000, 10)):
        a, b = coincidence_sets(synth, n, bands)
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        c_ms, k_ms, q_ms = [], [], []
        lab_b, _ = fh.fh_cluster(db, 4.0)
        for k in range(2 + steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lab, ncl = fh.fh_cluster(da, 4.0)
            t1 = time.perf_counter()
            pairs, m1, m2 = fh.fh_coincidences(da, db, 1.0e6, 2.0e6, 1.5e6, (2, 2, 2, 2))
            t2 = time.perf_counter()
            rows, _ = fh.fh_cluster_coincidences(da, db, 1.0e6, 2.0e6, 1.5e6, lab, lab_b, pairs)
            t3 = time.perf_counter()
            if k >= 2:
                c_ms.append((t1 - t0) * 1e3)
                k_ms.append((t2 - t1) * 1e3)
                q_ms.append((t3 - t2) * 1e3)
        cm, km = statistics.median(c_ms), statistics.median(k_ms)
        res["%dk_x_%dHz" % (n // 1000, bands)] = {
            "n_per_set": n, "clusters": ncl, "pairs": int(pairs.shape[0]),
            "coincident_in_set1": int((m1 > 0).sum().item()),
            "cluster_ms": cm, "coincidence_ms": km, "cluster_pairs": int(rows.shape[0]),
            "cluster_coincidence_ms": statistics.median(q_ms),
            "cluster_candidates_per_s": n / (cm * 1e-3),
            "coincidence_candidates_per_s": 2 * n / (km * 1e-3)}
    res["workload"] = ("two sets per size, sky uniform, f in 1 Hz bands at 100 Hz "
                       "(T_FFT 1024 s), 1 % common sources, 2 % clusters of 6")
    return res


def batched_vs_plain(fh, synth, torch):
    """256-direction sky patch (T_FFT 1024 s, 200 FFTs, 100-101 Hz): one launch
    per direction vs one persistent launch over all directions, each issued
    eagerly and replayed from a CUDA graph."""
    import numpy as np
    w = synth.WORKLOADS["sky_patch256_T1024_N200_100Hz"]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    n_dir = inp.sky.shape[0]
    dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
    upd = inp.n_peaks * pp["n_fdot"] * n_dir
    n_sb = -(-pp["n_f0"] // pp["subband_cells"])
    cand = torch.empty(n_dir * n_sb * pp["top_k"] * 48, dtype=torch.uint8, device="cuda")
    res = {"workload": w.name, "updates_per_step": upd}
    for name, sched in (("plain", fh.FH_SCHED_PLAIN), ("batched", fh.FH_SCHED_BATCHED)):
        plan = fh.fh_create_plan(fh.make_desc(pp, w.n_fft, n_dir, inp.n_peaks, schedule=sched))
        if sched == fh.FH_SCHED_BATCHED:
            fh.fh_correct_doppler(plan, *dev)
            fh.fh_autotune(plan, 0, n_dir)
        ts = []
        for k in range(13):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fh.fh_correct_doppler(plan, *dev)
            fh.fh_transform(plan, 0, n_dir, None)
            fh.fh_select_candidates(plan, 0, n_dir, cand)
            e1.record()
            torch.cuda.synchronize()
            if k >= 3:
                ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        res[name] = {"ms_per_step": ms, "updates_per_s": upd / (ms * 1e-3)}
        # the same step captured once into a CUDA graph and replayed
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            fh.fh_correct_doppler(plan, *dev, stream=s)
            fh.fh_transform(plan, 0, n_dir, None, stream=s)
            fh.fh_select_candidates(plan, 0, n_dir, cand, stream=s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            fh.fh_correct_doppler(plan, *dev, stream=s)
            fh.fh_transform(plan, 0, n_dir, None, stream=s)
            fh.fh_select_candidates(plan, 0, n_dir, cand, stream=s)
        ts = []
        for k in range(13):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            if k >= 3:
                ts.append(e0.elapsed_time(e1))
        fh.fh_sync(plan)
        ms = statistics.median(ts)
        res[name + "_graph"] = {"ms_per_step": ms, "updates_per_s": upd / (ms * 1e-3)}
        del g
        fh.fh_destroy_plan(plan)
    res["speedup"] = res["plain"]["ms_per_step"] / res["batched"]["ms_per_step"]
    res["speedup_graph"] = res["plain_graph"]["ms_per_step"] / res["batched_graph"]["ms_per_step"]
    return res


def maps_leg(fh, w, inp, pp, dev, flush, torch, steps):
    """The benchmark step in its second mode: the full number-count map
    (n_fdot x n_f0 int32 per direction, 383 MB here) written to HBM by the
    transform's emit as well as the profile and candidates.  Same inputs, L2
    flushed between steps, CUDA events."""
    n_dir = inp.sky.shape[0]
    maps = torch.empty((n_dir, pp["n_fdot"], pp["n_f0"]), dtype=torch.int32, device="cuda")
    n_sb = -(-pp["n_f0"] // pp["subband_cells"])
    cand = torch.empty(n_dir * n_sb * pp["top_k"] * 48, dtype=torch.uint8, device="cuda")
    plan = fh.fh_create_plan(fh.make_desc(pp, w.n_fft, n_dir, inp.n_peaks))
    try:
        fh.fh_correct_doppler(plan, *dev)
        tile, warps = fh.fh_autotune(plan, 0, n_dir)
        ts = []
        for k in range(3 + steps):
            if k == 3:
                fh.fh_plan_set_timing(plan, True)
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fh.fh_correct_doppler(plan, *dev)
            fh.fh_transform(plan, 0, n_dir, maps)
            fh.fh_select_candidates(plan, 0, n_dir, cand)
            e1.record()
            torch.cuda.synchronize()
            if k >= 3:
                ts.append(e0.elapsed_time(e1))
        ng, win_sum, kern_sum = fh.fh_plan_kernel_times(plan)
        fh.fh_plan_set_timing(plan, False)
    finally:
        fh.fh_destroy_plan(plan)
    upd = inp.n_peaks * pp["n_fdot"] * n_dir
    ms = statistics.mean(ts)
    kern = kern_sum / len(ts)
    map_bytes = 4 * pp["n_fdot"] * pp["n_f0"] * n_dir
    return {"mode": "maps written to HBM (int32) plus profile and candidates",
            "ms_per_step": ms, "updates_per_s": upd / (ms * 1e-3),
            "transform_kernel_ms": kern, "map_bytes": map_bytes,
            "map_write_gbs": map_bytes / (kern * 1e-3) / 1e9,
            "tile_cells": tile, "block_warps": warps, "steps": len(ts)}


def highfreq_leg(fh, synth, torch, steps):
    """The largest single-GPU workload: T_FFT 1024 s over a year (61594 FFTs,
    ~26.5M peaks), band 900-910 Hz, 356 x 102400 map, 64 sky directions in one
    batched plan (13.6 GB of positions).  Correction + transform + selection,
    device-resident inputs (far larger than L2), CUDA events."""
    w = synth.WORKLOADS["highfreq_T1024_1yr_900Hz_64dir"]
    t0 = time.perf_counter()
    inp = synth.make_inputs(w)
    gen_s = time.perf_counter() - t0
    pp = w.plan_params()
    n_dir = inp.sky.shape[0]
    dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
    upd = inp.n_peaks * pp["n_fdot"] * n_dir
    n_sb = -(-pp["n_f0"] // pp["subband_cells"])
    cand = torch.empty(n_dir * n_sb * pp["top_k"] * 48, dtype=torch.uint8, device="cuda")
    plan = fh.fh_create_plan(fh.make_desc(pp, w.n_fft, n_dir, inp.n_peaks))
    try:
        fh.fh_correct_doppler(plan, *dev)
        tile, warps = fh.fh_autotune(plan, 0, n_dir)
        ts = []
        n_warm = 2
        for k in range(n_warm + steps):
            if k == n_warm:
                fh.fh_plan_set_timing(plan, True)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            fh.fh_correct_doppler(plan, *dev)
            fh.fh_transform(plan, 0, n_dir, None)
            e[1].record()
            fh.fh_select_candidates(plan, 0, n_dir, cand)
            e[2].record()
            torch.cuda.synchronize()
            if k >= n_warm:
                ts.append((e[0].elapsed_time(e[2]), e[0].elapsed_time(e[1])))
        _, win_sum, kern_sum = fh.fh_plan_kernel_times(plan)
        fh.fh_plan_set_timing(plan, False)
    finally:
        fh.fh_destroy_plan(plan)
    ms = statistics.mean(t for t, _ in ts)
    return ({"workload": w.name, "n_peaks": inp.n_peaks, "n_dir": n_dir,
            "map": [pp["n_fdot"], pp["n_f0"]], "updates_per_step": upd,
            "ms_per_step": ms, "updates_per_s": upd / (ms * 1e-3),
            "correct_plus_transform_ms": statistics.mean(t for _, t in ts),
            "transform_kernel_ms": kern_sum / len(ts), "window_kernel_ms": win_sum / len(ts),
            "tile_cells": tile, "block_warps": warps, "steps": len(ts),
            "input_generation_s": gen_s}, (inp, pp))


def serving_leg(fh, synth, torch, seconds):
    from paper_1407_8333_gb300 import serve
    return serve.run_stream(seconds=seconds, seed=4)


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1407_8333_gb300 import synth
    oracle.build()
    if world > 1:
        # torchrun gives every worker one OpenMP thread; only this rank works here
        oracle.set_num_threads(os.cpu_count() or 1)
    w = synth.WORKLOADS[args.workload]
    inp = synth.make_inputs(w)
    pp = w.plan_params()
    upd = inp.n_peaks * pp["n_fdot"] * inp.sky.shape[0]
    for _ in range(args.warmup):
        oracle.search(inp, pp)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.search(inp, pp)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = upd * args.steps / total
    sample = ("whole path a1-a6 of the workload per step (1 direction, all %d rows), "
              "%d steps" % (pp["n_fdot"], args.steps))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "i64/i32 (f64 Doppler)", "data": "synthetic (seeded SplitMix64 peakmap)",
           "config": config_of(w, {"inputs": "host memory"}), "impl": "reference",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
