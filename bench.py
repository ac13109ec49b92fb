#!/usr/bin/env python
"""Benchmark of the GB300 frequency-Hough path.

One step = one pass of the whole hot path over one batch of synthetic input:
Doppler correction + fixed-point positions + shift tables (fh_correct_doppler),
transform + profile (fh_transform), candidate selection (fh_select_candidates).

Default workload, the largest single-GPU configuration: T_FFT = 1024 s,
half-interlaced over one year (61594 FFTs), 900-910 Hz with K = 10 (102400
cells), spin-down -1e-8 .. +1e-9 Hz/s (356 rows), peak probability 0.04
(~26.5M peaks), 64 sky directions in one plan, top-2 per 0.1 Hz sub-band.

Printed: one JSON line (rank 0) with throughput in peak x spin-down updates/s
(device-resident inputs), the end-to-end figure through the C ABI with host
buffers, the roofline of the transform kernel, the oracle's CPU baseline,
SM clocks sampled during the timed region, and legs: the 50 Hz single-sky
workload measured the same way, maps written, the adaptive map, plain vs
batched on a 256-direction sky patch, the served stream's latency figures,
refinement, peakmap construction and coincidences.  The line ends with a
short ``summary`` object.

``--impl reference`` times the CPU oracle (the benchmark's reference arm)
on a bounded sample of the same workload instead.
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
WORKLOAD = "highfreq_T1024_1yr_900Hz_64dir"
SMALL_WORKLOAD = "single_sky_T8192_150d_50Hz"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--dirs", type=int, default=0,
                    help="use only the workload's first N sky directions (profiling slices)")
    ap.add_argument("--no-extras", action="store_true", help="skip batched/serving/cpu legs")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--legs", default="single_sky,maps,adaptive,batched,serving,refine,peakmap,"
                                      "coincidences,cpu",
                    help="extra legs to run after the timed step (comma list)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def config_of(w, extra=None, n_dir=None):
    pp = w.plan_params()
    cfg = {"workload": w.name,
           "description": ("T_FFT=%g s, %d FFTs (start spacing %g s), band %.2f-%.2f Hz, K=%d "
                           "(%d cells), %d spin-down rows (%.3g..%.3g Hz/s), p=%.3g, %d sky "
                           "direction(s), top-%d per %.2g Hz" %
                           (w.t_fft, w.n_fft, w.t_step, w.f_lo, w.f_hi, w.k_over, pp["n_f0"],
                            pp["n_fdot"], pp["fdot_min"],
                            pp["fdot_min"] + (pp["n_fdot"] - 1) * pp["fdot_step"], w.p_peak,
                            n_dir or w.n_dir, w.top_k, w.subband_hz)),
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
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "transform_traffic.json")


def transform_source_sha1():
    """SHA-1 of the transform kernel's source: from its first helper (the cell
    of a fixed-point position) to the end of the a4 + a5 + profile section."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_1407_8333_gb300", "csrc", "fh_kernels.cu")).read()
    a = src.index("// Cell of a 32.32 fixed-point position")
    b = src.index("// ---------------------------------------------------------------- a6")
    return hashlib.sha1(src[a:b].encode()).hexdigest()


def transform_traffic(workload):
    """DRAM bytes per transform launch of `workload` from the committed ncu
    figures (profiles/transform_traffic.json), if the transform section of the
    kernel source is still the one that was profiled; else None."""
    try:
        rec = json.load(open(TRAFFIC_JSON)).get(workload)
        if rec and rec.get("transform_source_sha1") == transform_source_sha1():
            return rec
    except (OSError, ValueError):
        pass
    return None


def peaks_path():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0}, "fallback"


def oracle_sample(w, inp):
    """The bounded CPU sample of a workload: its line direction (or its only one)."""
    import numpy as np
    from paper_1407_8333_gb300 import synth
    if inp.sky.shape[0] == 1:
        return inp
    d = w.line_dir
    return synth.Inputs(w=w, t=inp.t, offsets=inp.offsets, freq=inp.freq, v=inp.v,
                        sky=np.ascontiguousarray(inp.sky[[d]]))


def cpu_baseline_leg(w, inp, pp, budget_s=12.0, small=None, refine_args=None, peakmap=None,
                     coinc=None):
    """The oracle as it stands, whole path a1-a6 on a bounded sample of the
    workload (one direction of it; the per-update rate stands for all), with
    all host threads; one thread on the 50 Hz workload `small` = (w, inputs,
    params); given refine_args = (cells, rows, sky_ref, k_fdot), its
    refined-grid search on a few candidates."""
    import oracle
    oracle.build()
    one = oracle_sample(w, inp)
    upd = one.n_peaks * pp["n_fdot"]
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        oracle.search(one, pp)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s or len(times) >= 3:
            break
    best = min(times)
    out = {"value": upd / best, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": "whole path a1-a6 (maps, profile, selection) on direction %d of the "
                     "workload's %d (%.3g updates), best of %d runs (%.2f s each); the "
                     "per-update rate stands for all directions"
                     % (w.line_dir if inp.sky.shape[0] > 1 else 0, inp.sky.shape[0], upd,
                        len(times), best)}
    n_thr = oracle.num_threads()
    if small is not None:
        sw, sinp, spp = small
        supd = sinp.n_peaks * spp["n_fdot"] * sinp.sky.shape[0]
        t0 = time.perf_counter()
        oracle.search(sinp, spp)
        dts = time.perf_counter() - t0
        oracle.set_num_threads(1)
        try:
            t0 = time.perf_counter()
            oracle.search(sinp, spp)
            dt1 = time.perf_counter() - t0
        finally:
            oracle.set_num_threads(n_thr)
        out["single_sky"] = {"value": supd / dts, "unit": UNIT, "cores": n_thr,
                             "sample": "whole path on the 50 Hz workload %s, one run (%.2f s)"
                                       % (sw.name, dts)}
        out["one_thread"] = {"value": supd / dt1, "unit": UNIT, "cores": 1,
                             "sample": "the same 50 Hz path on one thread, one run (%.2f s)"
                                       % dt1}
    if refine_args is not None:
        cells, rows, sky_ref, k_fdot = refine_args
        sinp, spp = small[1], small[2]
        t0 = time.perf_counter()
        oracle.refine(sinp, spp, cells, rows, sky_ref, k_fdot)
        dt = time.perf_counter() - t0
        out["refine"] = {"candidates_per_s": len(cells) / dt, "cores": n_thr,
                         "sample": "%d candidates, %d refined directions, K_fdot = %d, one run "
                                   "(%.2f s)" % (len(cells), sky_ref.shape[1], k_fdot, dt)}
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


def measure_step(fh, torch, w, inp, pp, dev, steps, warmup, flush, world=1, clocks=False):
    """Time `steps` steps (correction + transform + selection over every
    direction, device-resident inputs, L2 flushed between steps) with CUDA
    events on the launching stream; the library's events give the window
    pre-pass and transform kernel durations.  Returns the step figures, the
    transform's roofline against the live shared-atomic peak, the plan and
    its autotuned tile."""
    from paper_1407_8333_gb300 import replicas
    n_dir = inp.sky.shape[0]
    plan = fh.fh_create_plan(fh.make_desc(pp, w.n_fft, n_dir, inp.n_peaks))
    fh.fh_correct_doppler(plan, *dev)
    tile, warps = fh.fh_autotune(plan, 0, n_dir)
    n_sb = -(-pp["n_f0"] // pp["subband_cells"])
    cand = torch.empty(n_dir * n_sb * pp["top_k"] * 48, dtype=torch.uint8, device="cuda")
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
    for _ in range(max(3, warmup)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    nvtx.range_pop()
    sampler = None
    if clocks:
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    fh.fh_plan_set_timing(plan, True)
    l0 = fh.fh_plan_launches(plan)
    if world > 1:
        replicas.barrier()
    torch.cuda.synchronize()
    nvtx.range_push("timed")
    for k in range(steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize()
    nvtx.range_pop()
    if world > 1:
        replicas.barrier()
    launches = fh.fh_plan_launches(plan) - l0
    clk = sampler.stop() if sampler else None
    n_groups, win_ms_sum, kern_ms_sum = fh.fh_plan_kernel_times(plan)
    fh.fh_plan_set_timing(plan, False)
    groups_per_step = n_groups // steps
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    tr_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_ms = replicas.max_over_ranks(sum(step_ms)) if world > 1 else sum(step_ms)
    kern_launch = kern_ms_sum / n_groups          # one transform launch (a direction group)
    upd_launch = upd_step / groups_per_step
    atomic_peak, _ = fh.fh_bench_smem_atomics(0, 4096)
    achieved = upd_launch / (kern_launch * 1e-3)
    tr_avg = statistics.mean(tr_ms)
    traffic = transform_traffic(w.name)
    peaks, peak_src = peaks_path()
    hbm_bytes = 8 * inp.n_peaks * n_dir + 8 * pp["n_f0"] * n_dir + 16 * w.n_fft
    roof = {"bound": "smem_atomic", "achieved": achieved / 1e9, "peak": atomic_peak / 1e9,
            "unit": "Gatomic/s", "frac": achieved / atomic_peak,
            "traffic": traffic["dram_bytes_per_launch"] if traffic else None,
            "traffic_note": ("dram__bytes_read+write per transform launch (%s) from "
                             "profiles/transform_traffic.json; null if the kernel changed since"
                             % (traffic or {}).get("how", "ncu")),
            "kernel": "transform_kernel<FH_MODE_START>",
            "algorithmic": "1 shared-memory atomic per peak x spin-down update; %d updates per "
                           "launch (%d direction(s) per launch, %d launch(es) per step)"
                           % (upd_launch, n_dir // groups_per_step, groups_per_step),
            "peak_source": "own microbenchmark fh_bench_smem_atomics(0): conflict-free int32 "
                           "atomicAdd, all SMs, measured in this run",
            "duration_ms": kern_launch,
            "duration_note": "mean launch duration of transform_kernel over the timed steps, "
                             "CUDA events recorded by the library on the launching stream",
            "step_frac": upd_step / (tr_avg * 1e-3) / atomic_peak,
            "step_frac_note": "the same updates over fh_transform as a whole (window pre-pass "
                              "+ transform kernel)",
            "tile_cells": tile, "block_warps": warps}
    roof_hbm = {"bound": "hbm",
                "achieved": hbm_bytes / (kern_ms_sum / steps * 1e-3) / 1e9,
                "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                "frac": hbm_bytes / (kern_ms_sum / steps * 1e-3) / 1e9 / peaks.get("hbm_gbs"),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_src,
                "algorithmic": "8 B/peak/direction (positions) + 8 B/cell/direction (profile) "
                               "+ 16 B/FFT per step"}
    # the correction (a1-a3) is bound by the GPU's binary64 rate: its algorithmic
    # operations per step over its event-timed duration, against fh_bench_fp64
    fp64_peak, _ = fh.fh_bench_fp64(4096)
    corr_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    fp64_ops = 4 * inp.n_peaks * n_dir + 7 * w.n_fft * n_dir + 6 * w.n_fft
    roof_fp64 = {"bound": "fp64", "achieved": fp64_ops / (corr_ms * 1e-3) / 1e9,
                 "peak": fp64_peak / 1e9, "unit": "Gop/s",
                 "frac": fp64_ops / (corr_ms * 1e-3) / fp64_peak,
                 "kernel": "correct_kernel (one launch per fh_correct_doppler call)",
                 "algorithmic": "4 binary64 operations per (peak, direction): f r, - f0_min, "
                                "x KT, + (0.5 - 0.5 K); 7 per (FFT, direction): v.n (3 "
                                "multiplies, 2 adds), 1 + v.n, 1 / den; 6 per FFT: the shift "
                                "tables; %d per step" % fp64_ops,
                 "peak_source": "own microbenchmark fh_bench_fp64: independent IEEE multiply "
                                "and add chains on every SM, measured in this run",
                 "duration_ms": corr_ms,
                 "duration_note": "CUDA events around fh_correct_doppler (one 32-byte memset "
                                  "and the correction kernel)"}
    res = {"updates_per_step": upd_step, "ms_per_step": total_ms / steps,
           "value": upd_step * steps * world / (total_ms * 1e-3),
           "breakdown_ms": {"correct_doppler": statistics.mean(e[0].elapsed_time(e[1])
                                                               for e in evs),
                            "transform": tr_avg,
                            "select": statistics.mean(e[2].elapsed_time(e[3]) for e in evs),
                            "transform_windows_kernel": win_ms_sum / steps,
                            "transform_kernel": kern_ms_sum / steps},
           "roofline": roof, "roofline_hbm": roof_hbm, "roofline_correction": roof_fp64,
           "gpu_launches": launches,
           "clocks": clk}
    return res, plan, cand, (tile, warps)


def measure_e2e(fh, torch, inp, pp, plan, flush, steps, warmup, world=1):
    """The same step end to end through the C ABI: page-locked host inputs in,
    candidates back into a page-locked host buffer, copies inside the timed
    region; the inputs are checked by the kernels (FH_CHECKS_DEVICE)."""
    n_dir = inp.sky.shape[0]
    n_sb = -(-pp["n_f0"] // pp["subband_cells"])
    pinned = [torch.from_numpy(x).pin_memory().numpy() for x in
              (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
    fh.fh_plan_set_input_checks(plan, fh.FH_CHECKS_DEVICE)
    h2d = sum(x.nbytes for x in pinned)
    stream = torch.cuda.current_stream()
    host_out = torch.zeros(n_dir * n_sb * pp["top_k"] * fh.CANDIDATE_DTYPE.itemsize,
                           dtype=torch.uint8).pin_memory().numpy().view(fh.CANDIDATE_DTYPE)
    ms = []
    for k in range(max(3, warmup) + steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fh.fh_correct_doppler(plan, *pinned, stream=stream)
        fh.fh_transform(plan, 0, n_dir, None, stream=stream)
        fh.fh_select_candidates(plan, 0, n_dir, host_out, stream=stream)
        t1 = time.perf_counter()
        if k >= max(3, warmup):
            ms.append((t1 - t0) * 1e3)
    fh.fh_plan_set_input_checks(plan, fh.FH_CHECKS_HOST)
    upd = inp.n_peaks * pp["n_fdot"] * n_dir
    return {"value": upd * len(ms) / (sum(ms) * 1e-3) * world, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": host_out.nbytes,
            "ms_per_step": statistics.mean(ms),
            "input_checks": "device (FH_CHECKS_DEVICE): CSR, ordering, finiteness and "
                            "range checked by the kernels, reported at the select",
            "transfer": ("page-locked host inputs read in place by the correction kernels "
                         "over the host link" if n_dir == 1 else
                         "page-locked host inputs copied once per call (several directions "
                         "read them)") + ", candidates read back into a page-locked buffer"}, \
        host_out


# ----------------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch

    from paper_1407_8333_gb300 import build, fh, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    fh.load()

    w = synth.WORKLOADS[args.workload]
    inp = synth.make_inputs(w)
    if args.dirs > 0:
        inp = synth.Inputs(w=w, t=inp.t, offsets=inp.offsets, freq=inp.freq, v=inp.v,
                           sky=np.ascontiguousarray(inp.sky[:args.dirs]))
    pp = w.plan_params()
    dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    m, plan, _, _ = measure_step(fh, torch, w, inp, pp, dev, args.steps, args.warmup, flush,
                                 world=world, clocks=True)
    e2e, _ = measure_e2e(fh, torch, inp, pp, plan, flush, args.steps, args.warmup, world)
    fh.fh_destroy_plan(plan)
    del dev

    out = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "i64/i32 (f64 Doppler)",
           "data": "synthetic (seeded SplitMix64 peakmap, paper-shaped)",
           "config": config_of(w, n_dir=inp.sky.shape[0]),
           "inputs": "device-resident" + (" (larger than L2)" if inp.n_peaks * 8 > (256 << 20)
                                          else ""),
           "parallelism": "replicas" if world > 1 else "single GPU",
           "breakdown_ms": m["breakdown_ms"], "roofline": m["roofline"],
           "roofline_hbm": m["roofline_hbm"], "roofline_correction": m["roofline_correction"],
           "clocks": m["clocks"],
           "gpu_launches": m["gpu_launches"], "e2e": e2e}

    legs = set(args.legs.split(","))
    small = None
    ref_args = None
    if rank == 0 and world == 1 and not args.no_extras:
        if "single_sky" in legs or "cpu" in legs or "refine" in legs:
            sw = synth.WORKLOADS[SMALL_WORKLOAD]
            sinp = synth.make_inputs(sw)
            small = (sw, sinp, sw.plan_params())
        if "single_sky" in legs:
            try:
                out["single_sky"], host_out = single_sky_leg(fh, torch, small, args, flush)
                if "refine" in legs:
                    out["refine"], ref_args = refine_leg(fh, synth, sw, sinp, small[2],
                                                         host_out, args.steps)
            except Exception as e:  # report, do not hide
                out["single_sky"] = {"error": str(e)[:300]}
        if "adaptive" in legs:
            try:
                out["adaptive"] = adaptive_leg(fh, small, flush, torch, args.steps)
            except Exception as e:  # report, do not hide
                out["adaptive"] = {"error": str(e)[:300]}
        if "batched" in legs:
            out["batched_vs_plain"] = batched_vs_plain(fh, synth, torch)
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
                out["maps_written"] = maps_leg(fh, small, flush, torch, args.steps)
            except Exception as e:  # report, do not hide
                out["maps_written"] = {"error": str(e)[:300]}
        if "serving" in legs:
            try:
                out["serving"] = serving_leg(fh, synth, torch, args.serve_seconds)
            except Exception as e:  # report, do not hide
                out["serving"] = {"error": str(e)[:300]}
        if "cpu" in legs:
            out["cpu_baseline"] = cpu_baseline_leg(
                w, inp, pp, small=small, refine_args=ref_args,
                peakmap=synth.peakmap_workload() if "peakmap" in legs else None,
                coinc=coincidence_sets(synth, 5000, 1) if "coincidences" in legs else None)
    out["summary"] = summary_of(out)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def summary_of(out):
    """The figures a reader wants first, kept short (the line's last key)."""
    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d
    r = out.get("roofline", {})
    return {"workload": out["config"]["workload"], "updates_per_s": out["value"],
            "ms_per_step": out["ms_per_step"], "transform_frac": r.get("frac"),
            "transform_ms_per_launch": r.get("duration_ms"),
            "correction_fp64_frac": g(out, "roofline_correction", "frac"),
            "e2e_updates_per_s": g(out, "e2e", "value"),
            "single_sky_updates_per_s": g(out, "single_sky", "value"),
            "single_sky_transform_frac": g(out, "single_sky", "roofline", "frac"),
            "batched_over_plain": g(out, "batched_vs_plain", "speedup"),
            "serving_p50_ms": g(out, "serving", "served", "p50_ms"),
            "serving_p99_ms": g(out, "serving", "served", "p99_ms"),
            "plain_p50_ms": g(out, "serving", "plain", "p50_ms"),
            "plain_p99_ms": g(out, "serving", "plain", "p99_ms"),
            "serving_over_plain_updates": g(out, "serving", "speedup_updates_per_s"),
            "oracle_updates_per_s": g(out, "cpu_baseline", "value")}


def single_sky_leg(fh, torch, small, args, flush):
    """The 50 Hz single-sky workload (T_FFT 8192 s over 150 days, 3164 FFTs,
    1169 x 81920 map, one direction), measured like the headline: step, the
    transform's roofline, and end to end through the C ABI."""
    sw, sinp, spp = small
    dev = [torch.from_numpy(x).cuda() for x in (sinp.t, sinp.offsets, sinp.freq, sinp.v,
                                                 sinp.sky)]
    m, plan, _, _ = measure_step(fh, torch, sw, sinp, spp, dev, args.steps, args.warmup, flush)
    try:
        e2e, host_out = measure_e2e(fh, torch, sinp, spp, plan, flush, args.steps, args.warmup)
    finally:
        fh.fh_destroy_plan(plan)
    m.pop("clocks", None)
    m["workload"] = sw.name
    m["e2e"] = e2e
    return m, host_out


def adaptive_leg(fh, small, flush, torch, steps):
    """The 50 Hz workload as the adaptive map (Eq. ncountadap): weights with a
    sidereal-day modulation, 12 fraction bits, set after every correction (a
    new peakmap returns the plan to unit weights)."""
    import numpy as np
    sw, inp, pp = small
    dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
    n_sb = -(-pp["n_f0"] // pp["subband_cells"])
    cand = torch.empty(n_sb * pp["top_k"] * 48, dtype=torch.uint8, device="cuda")
    n = inp.t.shape[0]
    w = (1.0 + 0.5 * np.cos(2 * np.pi * inp.t / 86164.09)).reshape(1, n)
    plan = fh.fh_create_plan(fh.make_desc(pp, n, 1, inp.n_peaks))
    try:
        fh.fh_correct_doppler(plan, *dev)
        # the launch shape of the weighted map (its own autotuner entry)
        fh.fh_set_weights(plan, w, 12)
        fh.fh_autotune(plan, 0, 1)
        ts = []
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
    return {"workload": sw.name, "weights": "1 + 0.5 cos(2 pi t / sidereal day), 12 fraction bits",
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


def maps_leg(fh, small, flush, torch, steps):
    """The 50 Hz step in its second mode: the full number-count map
    (n_fdot x n_f0 int32, 383 MB) written to HBM by the transform's emit as
    well as the profile and candidates.  Same inputs, L2 flushed between steps,
    CUDA events."""
    w, inp, pp = small
    n_dir = inp.sky.shape[0]
    dev = [torch.from_numpy(x).cuda() for x in (inp.t, inp.offsets, inp.freq, inp.v, inp.sky)]
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
    return {"workload": w.name,
            "mode": "maps written to HBM (int32) plus profile and candidates",
            "ms_per_step": ms, "updates_per_s": upd / (ms * 1e-3),
            "transform_kernel_ms": kern, "map_bytes": map_bytes,
            "map_write_gbs": map_bytes / (kern * 1e-3) / 1e9,
            "tile_cells": tile, "block_warps": warps, "steps": len(ts)}


def serving_leg(fh, synth, torch, seconds):
    """The served mixed stream at its stated size: T_obs = 150 days, 1..512
    directions per job, Poisson arrivals at 70 % of the served capacity."""
    from paper_1407_8333_gb300 import serve
    return serve.run_stream(seconds=seconds, seed=4, scale_fft=1.0, max_dir=512, load=0.7)


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
    one = oracle_sample(w, inp)
    upd = one.n_peaks * pp["n_fdot"]
    for _ in range(args.warmup):
        oracle.search(one, pp)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.search(one, pp)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = upd * args.steps / total
    sample = ("whole path a1-a6 (maps, profile, selection) per step on direction %d of the "
              "workload's %d (all %d rows, %.3g updates), %d steps; the per-update rate stands "
              "for all directions" % (w.line_dir if inp.sky.shape[0] > 1 else 0,
                                      inp.sky.shape[0], pp["n_fdot"], upd, args.steps))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "i64/i32 (f64 Doppler)",
           "data": "synthetic (seeded SplitMix64 peakmap, paper-shaped)",
           "config": config_of(w), "inputs": "host memory", "impl": "reference",
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
