"""Thin ctypes binding of libfh (``include/fh.h``), same entry-point names.

Argument marshalling only: every step of the frequency-Hough path runs in the
library's CUDA kernels.  Arrays are passed as raw pointers: numpy arrays (host
memory, ``FH_MEM_HOST``) or CUDA tensors (device memory, ``FH_MEM_DEVICE``,
via ``data_ptr()``); streams are ``torch.cuda.Stream`` objects, raw handles or
None (legacy default stream).  The library must have been built
(``paper_1407_8333_gb300.build.build()``); loading fails loudly otherwise --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

FH_OK = 0
FH_ERR_INVALID_ARG = -1
FH_ERR_UNSORTED = -2
FH_ERR_RANGE = -3
FH_ERR_NOMEM = -4
FH_ERR_TOO_LARGE = -5
FH_ERR_CUDA = -6
FH_ERR_TIMEOUT = -7
FH_ERR_NOT_READY = -8
FH_ERR_CANCELLED = -9
FH_ERR_BAD_HANDLE = -10
FH_ERR_CAPACITY = -11
FH_MEM_HOST, FH_MEM_DEVICE = 0, 1
FH_MODE_AUTO, FH_MODE_DIFF, FH_MODE_START = 0, 1, 2
FH_SCHED_BATCHED, FH_SCHED_PLAIN = 0, 1
FH_JOB_QUEUED, FH_JOB_RUNNING, FH_JOB_DONE, FH_JOB_FAILED, FH_JOB_CANCELLED = 0, 1, 2, 3, 4

_i32, _i64, _f64, _P = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class fh_peakmap(ctypes.Structure):
    _fields_ = [("n_fft", _i32), ("n_peaks", _i64), ("t_fft", _P), ("offsets", _P),
                ("freq", _P), ("mem_kind", _i32)]


class fh_plan_desc(ctypes.Structure):
    _fields_ = [("t_fft", _f64), ("k_over", _i32), ("f0_min", _f64), ("n_f0", _i32),
                ("fdot_min", _f64), ("fdot_step", _f64), ("n_fdot", _i32), ("t_ref", _f64),
                ("subband_cells", _i32), ("top_k", _i32), ("excl_cells", _i32),
                ("sep_cells", _i32), ("n_thr", _i32), ("p0", _f64), ("max_fft", _i32),
                ("max_dir", _i32), ("max_peaks", _i64), ("mode", _i32), ("schedule", _i32),
                ("tile_cells", _i32), ("block_warps", _i32)]


class fh_candidate(ctypes.Structure):
    _fields_ = [("dir", _i32), ("subband", _i32), ("rank", _i32), ("row", _i32),
                ("cell", _i32), ("count", _i32), ("f0", _f64), ("fdot", _f64), ("cr", _f64)]


CANDIDATE_DTYPE = np.dtype([("dir", "<i4"), ("subband", "<i4"), ("rank", "<i4"),
                            ("row", "<i4"), ("cell", "<i4"), ("count", "<i4"),
                            ("f0", "<f8"), ("fdot", "<f8"), ("cr", "<f8")])
assert CANDIDATE_DTYPE.itemsize == ctypes.sizeof(fh_candidate) == 48


class fh_job_desc(ctypes.Structure):
    _fields_ = [("plan", fh_plan_desc), ("peaks", fh_peakmap), ("v_over_c", _P),
                ("sky_n", _P), ("n_dir", _i32)]


class fh_job_stats(ctypes.Structure):
    _fields_ = [("submit_s", _f64), ("start_s", _f64), ("done_s", _f64), ("updates", _i64),
                ("device_bytes", _i64), ("batch", _i32), ("batch_jobs", _i32)]


class FHError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__("%s failed (%d): %s" % (func, code, msg))
        self.code = code


_lib = None
_lock = threading.Lock()

_SIGS = {
    "fh_create_plan": ([ctypes.POINTER(fh_plan_desc), ctypes.POINTER(_P)], ctypes.c_int),
    "fh_destroy_plan": ([_P], ctypes.c_int),
    "fh_plan_device_bytes": ([ctypes.POINTER(fh_plan_desc)], _i64),
    "fh_correct_doppler": ([_P, ctypes.POINTER(fh_peakmap), _P, _P, _i32, _P, _P, _P], ctypes.c_int),
    "fh_transform": ([_P, _i32, _i32, _P, _P], ctypes.c_int),
    "fh_copy_profile": ([_P, _i32, _i32, _P, _P], ctypes.c_int),
    "fh_select_candidates": ([_P, _i32, _i32, _P, _i64, ctypes.POINTER(_i64), _i32, _P], ctypes.c_int),
    "fh_sync": ([_P, _P], ctypes.c_int),
    "fh_autotune": ([_P, _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), _P], ctypes.c_int),
    "fh_plan_launches": ([_P], _i64),
    "fh_set_weights": ([_P, _P, _i32, _i32, _P], ctypes.c_int),
    "fh_peakmap_select": ([_P, _P, _i32, _i32, _i64, ctypes.c_float, _i64, _f64, _P, _P, _P,
                           _i64, _P, _P, _i64, _P], ctypes.c_int),
    "fh_peakmap_select_workspace": ([_i32, _i32], _i64),
    "fh_peakmap_gross_veto": ([_P, _P, _P, _i32, _i64, _i64, _f64, _f64, _f64, _i32, _f64, _f64,
                               _i32, _i32, _P, _P, _P, _P, _i64, _P, _P], ctypes.c_int),
    "fh_peakmap_persistency_veto": ([_P, _P, _i32, _i64, _i32, _f64, _i64, _f64, _P, _P, _P, _P,
                                     _P, _i64, _P, _P], ctypes.c_int),
    "fh_cluster": ([_P, _i32, _f64, _P, _P, _P], ctypes.c_int),
    "fh_coincidences": ([_P, _i32, _f64, _P, _i32, _f64, _f64, _P, _P, _i64, _P, _P, _P, _P],
                        ctypes.c_int),
    "fh_plan_set_input_checks": ([_P, _i32], ctypes.c_int),
    "fh_cluster_coincidences": ([_P, _i32, _f64, _P, _P, _i32, _f64, _P, _f64, _P, _i64, _P, _P,
                                 _i64, _P, _P], ctypes.c_int),
    "fh_refine": ([_P, ctypes.POINTER(fh_peakmap), _P, _P, _P, _i32, _P, _i32, _i32, _P, _i64, _P],
                  ctypes.c_int),
    "fh_plan_set_timing": ([_P, _i32], ctypes.c_int),
    "fh_plan_kernel_times": ([_P, ctypes.POINTER(_i64), ctypes.POINTER(_f64), ctypes.POINTER(_f64)],
                             ctypes.c_int),
    "fh_server_create": ([_i64, _i32, ctypes.POINTER(_P)], ctypes.c_int),
    "fh_server_destroy": ([_P], ctypes.c_int),
    "fh_submit": ([_P, ctypes.POINTER(fh_job_desc), ctypes.POINTER(_i64)], ctypes.c_int),
    "fh_poll": ([_P, _i64, ctypes.POINTER(_i32), _P, _i64, ctypes.POINTER(_i64)], ctypes.c_int),
    "fh_job_get_stats": ([_P, _i64, ctypes.POINTER(fh_job_stats)], ctypes.c_int),
    "fh_cancel": ([_P, _i64], ctypes.c_int),
    "fh_server_drain": ([_P, _f64], ctypes.c_int),
    "fh_server_pause": ([_P, _i32], ctypes.c_int),
    "fh_search_static": ([ctypes.POINTER(fh_plan_desc), ctypes.POINTER(fh_peakmap), _P, _P, _P, _i64,
                          ctypes.POINTER(_i64), _P, _P], ctypes.c_int),
    "fh_bench_smem_atomics": ([_i32, _i32, ctypes.POINTER(_f64), ctypes.POINTER(_f64), _P], ctypes.c_int),
    "fh_bench_fp64": ([_i32, ctypes.POINTER(_f64), ctypes.POINTER(_f64), _P], ctypes.c_int),
    "fh_last_error": ([], ctypes.c_char_p),
    "fh_version": ([], ctypes.c_char_p),
}


def lib_path() -> str:
    return _build.LIB


def load(path: str = None):
    """Load libfh.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or _build.LIB
            if not os.path.exists(p):
                raise RuntimeError("libfh.so not found at %s: build it with "
                                   "paper_1407_8333_gb300.build.build()" % p)
            lib = ctypes.CDLL(p)
            for name, (args, res) in _SIGS.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def exported_symbols() -> list:
    return list(_SIGS.keys())


def _check(rc: int, func: str, ok=(FH_OK,)):
    if rc not in ok:
        raise FHError(rc, func, load().fh_last_error().decode(errors="replace"))
    return rc


# ---------------------------------------------------------------- marshalling
def _is_torch(x) -> bool:
    return hasattr(x, "data_ptr") and hasattr(x, "is_cuda")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError("unsupported buffer type %r" % type(x))


def _mem_kind(x) -> int:
    if _is_torch(x):
        if not x.is_cuda:
            raise ValueError("CPU tensors are not accepted; pass numpy arrays for host memory")
        return FH_MEM_DEVICE
    return FH_MEM_HOST


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def make_desc(params: dict, max_fft: int, max_dir: int, max_peaks: int, mode: int = FH_MODE_AUTO,
              schedule: int = FH_SCHED_BATCHED, tile_cells: int = 0, block_warps: int = 0) -> fh_plan_desc:
    d = fh_plan_desc()
    for k in ("t_fft", "f0_min", "fdot_min", "fdot_step", "t_ref", "p0"):
        setattr(d, k, float(params[k]))
    for k in ("k_over", "n_f0", "n_fdot", "subband_cells", "top_k", "excl_cells", "sep_cells",
              "n_thr"):
        setattr(d, k, int(params[k]))
    d.max_fft, d.max_dir, d.max_peaks = int(max_fft), int(max_dir), int(max(1, max_peaks))
    d.mode, d.schedule = int(mode), int(schedule)
    d.tile_cells, d.block_warps = int(tile_cells), int(block_warps)
    return d


def make_peakmap(t, offsets, freq, n_peaks: int = None) -> fh_peakmap:
    kind = _mem_kind(offsets)
    pm = fh_peakmap()
    pm.n_fft = int(offsets.shape[0] - 1)
    pm.n_peaks = int(n_peaks if n_peaks is not None else
                     (offsets[-1] if kind == FH_MEM_HOST else freq.shape[0]))
    pm.t_fft = _ptr(t)
    pm.offsets = _ptr(offsets)
    pm.freq = _ptr(freq)
    pm.mem_kind = kind
    return pm


# ---------------------------------------------------------------- entry points
def fh_version() -> str:
    return load().fh_version().decode()


def fh_last_error() -> str:
    return load().fh_last_error().decode(errors="replace")


def fh_plan_device_bytes(desc: fh_plan_desc) -> int:
    return int(load().fh_plan_device_bytes(ctypes.byref(desc)))


def fh_create_plan(desc: fh_plan_desc) -> ctypes.c_void_p:
    h = _P()
    _check(load().fh_create_plan(ctypes.byref(desc), ctypes.byref(h)), "fh_create_plan")
    return h


def fh_destroy_plan(plan) -> None:
    _check(load().fh_destroy_plan(plan), "fh_destroy_plan")


def fh_correct_doppler(plan, t, offsets, freq, v_over_c, sky_n, out_r=None, out_A=None,
                       stream=None, n_peaks: int = None) -> None:
    pm = make_peakmap(t, offsets, freq, n_peaks)
    n_dir = int(sky_n.shape[0])
    _check(load().fh_correct_doppler(plan, ctypes.byref(pm), _ptr(v_over_c), _ptr(sky_n), n_dir,
                                     _ptr(out_r), _ptr(out_A), _stream(stream)),
           "fh_correct_doppler")


def fh_transform(plan, dir_begin: int, n_dir: int, out_maps=None, stream=None) -> None:
    _check(load().fh_transform(plan, int(dir_begin), int(n_dir), _ptr(out_maps), _stream(stream)),
           "fh_transform")


def fh_copy_profile(plan, dir_begin: int, n_dir: int, out, stream=None) -> None:
    """Enqueue a device-to-device copy of the profile into ``out`` (a CUDA
    tensor or a raw device address); host arrays are refused, since the copy
    is asynchronous."""
    if isinstance(out, np.ndarray) or (_is_torch(out) and not out.is_cuda):
        raise TypeError("fh_copy_profile writes device memory: pass a CUDA tensor")
    _check(load().fh_copy_profile(plan, int(dir_begin), int(n_dir), _ptr(out), _stream(stream)),
           "fh_copy_profile")


def fh_select_candidates(plan, dir_begin: int, n_dir: int, out=None, stream=None):
    """Candidate slots; ``out`` = None -> a new numpy structured array (host)."""
    n = _i64(0)
    if out is None:
        load().fh_select_candidates(plan, int(dir_begin), int(n_dir), None, 0, ctypes.byref(n), 0,
                                    _stream(stream))
        out = np.zeros(int(n.value), dtype=CANDIDATE_DTYPE)
    kind = _mem_kind(out)
    cap = (out.numel() * out.element_size() // 48) if kind == FH_MEM_DEVICE else out.shape[0]
    _check(load().fh_select_candidates(plan, int(dir_begin), int(n_dir), _ptr(out), int(cap),
                                       ctypes.byref(n), kind, _stream(stream)),
           "fh_select_candidates")
    return out


def fh_sync(plan, stream=None) -> None:
    _check(load().fh_sync(plan, _stream(stream)), "fh_sync")


def fh_autotune(plan, dir_begin: int, n_dir: int, stream=None) -> tuple:
    w, nw = _i32(0), _i32(0)
    _check(load().fh_autotune(plan, int(dir_begin), int(n_dir), ctypes.byref(w), ctypes.byref(nw),
                              _stream(stream)), "fh_autotune")
    return int(w.value), int(nw.value)


def fh_plan_launches(plan) -> int:
    return int(load().fh_plan_launches(plan))


FH_CHECKS_HOST, FH_CHECKS_DEVICE = 0, 1


def fh_plan_set_input_checks(plan, where: int) -> None:
    """FH_CHECKS_HOST (default) or FH_CHECKS_DEVICE for host inputs."""
    _check(load().fh_plan_set_input_checks(plan, int(where)), "fh_plan_set_input_checks")


def _dev_ptr(x):
    return None if x is None else ctypes.c_void_p(x.data_ptr())


def _ws_bytes(w) -> int:
    return 0 if w is None else int(w.numel() * w.element_size())


def fh_peakmap_select_workspace(n_fft: int, n_bins: int) -> int:
    return int(load().fh_peakmap_select_workspace(int(n_fft), int(n_bins)))


def fh_peakmap_select(s_p, s_ar, theta: float, k0: int, t_fft: float, capacity: int = None,
                      want_freq: bool = True, stream=None, out=None, workspace=None):
    """Peaks of device spectra (torch float32, (n_fft, n_bins), rows contiguous).
    Returns (offsets int64, bins int32, freq float64 or None) on the device.
    With ``out`` = (offsets, bins, freq) preallocated, the call is asynchronous
    and returns those buffers whole (the total is offsets[n_fft]); ``workspace``
    (a device uint8 tensor of fh_peakmap_select_workspace bytes) avoids the
    call's own scratch allocation."""
    import torch
    n_fft, n_bins = int(s_p.shape[0]), int(s_p.shape[1])
    if s_p.stride(1) != 1 or s_ar.stride(1) != 1 or s_p.stride(0) != s_ar.stride(0):
        raise ValueError("s_p and s_ar need unit-stride rows of the same pitch")
    if out is not None:
        offsets, bins, freq = out
        _check(load().fh_peakmap_select(_dev_ptr(s_p), _dev_ptr(s_ar), n_fft, n_bins,
                                        int(s_p.stride(0)), float(theta), int(k0), float(t_fft),
                                        _dev_ptr(offsets), _dev_ptr(bins), _dev_ptr(freq),
                                        int(bins.shape[0]), None, _dev_ptr(workspace),
                                        _ws_bytes(workspace), _stream(stream)),
               "fh_peakmap_select")
        return offsets, bins, freq
    cap = int(capacity) if capacity is not None else max(1, n_fft * max(0, n_bins - 1) // 2)
    dev = s_p.device
    offsets = torch.empty(n_fft + 1, dtype=torch.int64, device=dev)
    bins = torch.empty(cap, dtype=torch.int32, device=dev)
    freq = torch.empty(cap, dtype=torch.float64, device=dev) if want_freq else None
    n = ctypes.c_int64(0)
    _check(load().fh_peakmap_select(_dev_ptr(s_p), _dev_ptr(s_ar), n_fft, n_bins,
                                    int(s_p.stride(0)), float(theta), int(k0), float(t_fft),
                                    _dev_ptr(offsets), _dev_ptr(bins), _dev_ptr(freq), cap,
                                    ctypes.byref(n), _dev_ptr(workspace), _ws_bytes(workspace),
                                    _stream(stream)), "fh_peakmap_select")
    k = n.value
    return offsets, bins[:k], (freq[:k] if freq is not None else None)


def fh_peakmap_gross_veto(t, offsets, bins, k0: int, t_fft: float, t0_h: float, dt_h: float,
                          n_th: int, f0_h: float, df_h: float, n_fh: int, threshold: int,
                          want_freq: bool = True, stream=None):
    """Wandering-line veto of a device peakmap.  Returns (offsets, bins, freq,
    hist (n_th, n_fh) int32) on the device."""
    import torch
    dev = offsets.device
    n_fft = int(offsets.shape[0]) - 1
    n_peaks = int(bins.shape[0])
    hist = torch.empty((int(n_th), int(n_fh)), dtype=torch.int32, device=dev)
    o2 = torch.empty(n_fft + 1, dtype=torch.int64, device=dev)
    cap = max(1, n_peaks)
    b2 = torch.empty(cap, dtype=torch.int32, device=dev)
    f2 = torch.empty(cap, dtype=torch.float64, device=dev) if want_freq else None
    n = ctypes.c_int64(0)
    _check(load().fh_peakmap_gross_veto(_dev_ptr(t), _dev_ptr(offsets), _dev_ptr(bins), n_fft,
                                        n_peaks, int(k0), float(t_fft), float(t0_h), float(dt_h),
                                        int(n_th), float(f0_h), float(df_h), int(n_fh),
                                        int(threshold), _dev_ptr(hist), _dev_ptr(o2),
                                        _dev_ptr(b2), _dev_ptr(f2), cap, ctypes.byref(n),
                                        _stream(stream)), "fh_peakmap_gross_veto")
    k = n.value
    return o2, b2[:k], (f2[:k] if f2 is not None else None), hist


def fh_peakmap_persistency_veto(offsets, bins, n_bins: int, k_sigma: float, k0: int,
                                t_fft: float, want_freq: bool = True, stream=None):
    """Constant-line veto of a device peakmap.  Returns (offsets, bins, freq,
    hist (n_bins) int32, (m1, m2, thr))."""
    import torch
    dev = offsets.device
    n_fft = int(offsets.shape[0]) - 1
    n_peaks = int(bins.shape[0])
    hist = torch.empty(int(n_bins), dtype=torch.int32, device=dev)
    o2 = torch.empty(n_fft + 1, dtype=torch.int64, device=dev)
    cap = max(1, n_peaks)
    b2 = torch.empty(cap, dtype=torch.int32, device=dev)
    f2 = torch.empty(cap, dtype=torch.float64, device=dev) if want_freq else None
    stats = (ctypes.c_double * 3)()
    n = ctypes.c_int64(0)
    _check(load().fh_peakmap_persistency_veto(_dev_ptr(offsets), _dev_ptr(bins), n_fft, n_peaks,
                                              int(n_bins), float(k_sigma), int(k0), float(t_fft),
                                              _dev_ptr(hist), ctypes.cast(stats, _P),
                                              _dev_ptr(o2), _dev_ptr(b2), _dev_ptr(f2), cap,
                                              ctypes.byref(n),
                                              _stream(stream)), "fh_peakmap_persistency_veto")
    k = n.value
    return o2, b2[:k], (f2[:k] if f2 is not None else None), hist, tuple(stats)


def fh_cluster_coincidences(c1, c2, t_ref1: float, t_ref2: float, t_c: float, label1, label2,
                            pairs, stream=None):
    """The nearest coincident pair of each coincident pair of clusters: rows
    (cluster 1, cluster 2, i, j) ((k, 4) device int32) and distances."""
    torch = _torch()
    a, b = _cands(c1), _cands(c2)
    pairs = pairs.contiguous()  # kept referenced for the call
    n_pairs = int(pairs.shape[0])
    cap = max(1, n_pairs)
    out = torch.empty((cap, 4), dtype=torch.int32, device=a.device)
    dist = torch.empty(cap, dtype=torch.float64, device=a.device)
    n = ctypes.c_int64(0)
    _check(load().fh_cluster_coincidences(_dev_ptr(a), int(a.shape[0]), float(t_ref1),
                                          _dev_ptr(label1), _dev_ptr(b), int(b.shape[0]),
                                          float(t_ref2), _dev_ptr(label2), float(t_c),
                                          _dev_ptr(pairs), n_pairs, _dev_ptr(out),
                                          _dev_ptr(dist), cap, ctypes.byref(n), _stream(stream)),
           "fh_cluster_coincidences")
    return out[:n.value], dist[:n.value]


def _cands(c):
    """A device tensor of candidate records: (n, 8) float64, rows in the order
    lam, beta, f, fdot, dlam, dbeta, df, dfdot."""
    if c.dtype != _torch().float64 or c.dim() != 2 or c.shape[1] != 8 or not c.is_contiguous():
        raise ValueError("candidates: a contiguous (n, 8) float64 device tensor")
    return c


def _torch():
    import torch
    return torch


def fh_cluster(cands, d_max: float, stream=None):
    """Cluster labels (device int32, the smallest index of each cluster) and the
    number of clusters."""
    torch = _torch()
    c = _cands(cands)
    n = int(c.shape[0])
    label = torch.empty(max(1, n), dtype=torch.int32, device=c.device)
    nc = ctypes.c_int32(0)
    _check(load().fh_cluster(_dev_ptr(c), n, float(d_max), _dev_ptr(label), ctypes.byref(nc),
                             _stream(stream)), "fh_cluster")
    return label[:n], int(nc.value)


def fh_coincidences(c1, c2, t_ref1: float, t_ref2: float, t_c: float, win, capacity: int = None,
                    stream=None):
    """Coincident pairs ((k, 2) device int32, (i, j) order) and the partner
    counts of both sets."""
    torch = _torch()
    a, b = _cands(c1), _cands(c2)
    n1, n2 = int(a.shape[0]), int(b.shape[0])
    w = (ctypes.c_double * 4)(*[float(x) for x in win])
    cap = int(capacity) if capacity is not None else max(1, 4 * (n1 + n2))
    while True:
        pairs = torch.empty((cap, 2), dtype=torch.int32, device=a.device)
        m1 = torch.empty(max(1, n1), dtype=torch.int32, device=a.device)
        m2 = torch.empty(max(1, n2), dtype=torch.int32, device=a.device)
        n = ctypes.c_int64(0)
        rc = load().fh_coincidences(_dev_ptr(a), n1, float(t_ref1), _dev_ptr(b), n2,
                                    float(t_ref2), float(t_c), ctypes.cast(w, _P),
                                    _dev_ptr(pairs), cap, ctypes.byref(n), _dev_ptr(m1),
                                    _dev_ptr(m2), _stream(stream))
        if rc == FH_ERR_CAPACITY and capacity is None:
            cap = int(n.value)
            continue
        _check(rc, "fh_coincidences")
        return pairs[:n.value], m1[:n1], m2[:n2]


def fh_refine(plan, t, offsets, freq, v_over_c, cells, rows, sky_ref, k_fdot: int,
              stream=None) -> np.ndarray:
    """Refined candidates (host arrays in, structured array out), one per
    coarse candidate; sky_ref is n_cand x n_ref x 3."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    freq = np.ascontiguousarray(freq, dtype=np.float64)
    v = np.ascontiguousarray(v_over_c, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    sky = np.ascontiguousarray(sky_ref, dtype=np.float64)
    n_cand, n_ref = int(sky.shape[0]), int(sky.shape[1])
    pm = make_peakmap(t, offsets, freq)
    out = np.zeros(n_cand, dtype=CANDIDATE_DTYPE)
    _check(load().fh_refine(plan, ctypes.byref(pm), v.ctypes.data_as(_P),
                            cells.ctypes.data_as(_P), rows.ctypes.data_as(_P), n_cand,
                            sky.ctypes.data_as(_P), n_ref, int(k_fdot), out.ctypes.data_as(_P),
                            n_cand, _stream(stream)), "fh_refine")
    return out


def fh_set_weights(plan, w, frac_bits: int = 0, stream=None) -> None:
    """Adaptive weights (n_dir x n_fft host reals, or None for the plain map)."""
    if w is None:
        _check(load().fh_set_weights(plan, None, 0, 0, _stream(stream)), "fh_set_weights")
        return
    w = np.ascontiguousarray(w, dtype=np.float64)
    if w.ndim != 2:
        raise ValueError("weights must be n_dir x n_fft")
    _check(load().fh_set_weights(plan, w.ctypes.data_as(_P), int(w.shape[0]), int(frac_bits),
                                 _stream(stream)), "fh_set_weights")


def fh_plan_set_timing(plan, on: bool = True) -> None:
    _check(load().fh_plan_set_timing(plan, 1 if on else 0), "fh_plan_set_timing")


def fh_plan_kernel_times(plan) -> tuple:
    """(groups, window pre-pass ms, transform kernel ms), summed over the groups
    recorded since timing was switched on."""
    n = _i64(0)
    w = ctypes.c_double(0.0)
    t = ctypes.c_double(0.0)
    _check(load().fh_plan_kernel_times(plan, ctypes.byref(n), ctypes.byref(w), ctypes.byref(t)),
           "fh_plan_kernel_times")
    return int(n.value), float(w.value), float(t.value)


def fh_bench_smem_atomics(variant: int = 0, iters: int = 4096, stream=None) -> tuple:
    r, ms = _f64(0), _f64(0)
    _check(load().fh_bench_smem_atomics(int(variant), int(iters), ctypes.byref(r), ctypes.byref(ms),
                                        _stream(stream)), "fh_bench_smem_atomics")
    return float(r.value), float(ms.value)


def fh_bench_fp64(iters: int = 4096, stream=None) -> tuple:
    """(binary64 operations per second, ms) of the multiply + add chains."""
    r, ms = _f64(0), _f64(0)
    _check(load().fh_bench_fp64(int(iters), ctypes.byref(r), ctypes.byref(ms), _stream(stream)),
           "fh_bench_fp64")
    return float(r.value), float(ms.value)


def fh_search_static(params: dict, t, offsets, freq, v_over_c, sky_n, out, device_status=None,
                     stream=None, mode: int = FH_MODE_AUTO, tile_cells: int = 0,
                     block_warps: int = 0) -> int:
    """One direction, no device allocation; all arrays are CUDA tensors.  Returns n_out."""
    desc = make_desc(params, 1, 1, 1, mode=mode, tile_cells=tile_cells, block_warps=block_warps)
    pm = make_peakmap(t, offsets, freq, n_peaks=int(freq.shape[0]))
    n = _i64(0)
    cap = out.numel() * out.element_size() // 48
    _check(load().fh_search_static(ctypes.byref(desc), ctypes.byref(pm), _ptr(v_over_c), _ptr(sky_n),
                                   _ptr(out), int(cap), ctypes.byref(n), _ptr(device_status),
                                   _stream(stream)), "fh_search_static")
    return int(n.value)


# ---- serving
def fh_server_create(device_mem_budget: int, max_inflight: int = 4):
    h = _P()
    _check(load().fh_server_create(int(device_mem_budget), int(max_inflight), ctypes.byref(h)),
           "fh_server_create")
    return h


def fh_server_destroy(server) -> None:
    _check(load().fh_server_destroy(server), "fh_server_destroy")


def fh_submit(server, params: dict, t, offsets, freq, v_over_c, sky_n, mode: int = FH_MODE_AUTO,
              tile_cells: int = 0) -> int:
    jd = fh_job_desc()
    jd.plan = make_desc(params, 1, 1, 1, mode=mode, tile_cells=tile_cells)
    jd.peaks = make_peakmap(t, offsets, freq)
    jd.v_over_c = _ptr(v_over_c)
    jd.sky_n = _ptr(sky_n)
    jd.n_dir = int(sky_n.shape[0])
    jid = _i64(0)
    _check(load().fh_submit(server, ctypes.byref(jd), ctypes.byref(jid)), "fh_submit")
    return int(jid.value)


def fh_poll(server, job_id: int, out: np.ndarray = None):
    """(state, candidates or None).  Raises on a failed job."""
    st = _i32(0)
    n = _i64(0)
    cap = 0 if out is None else out.shape[0]
    rc = load().fh_poll(server, int(job_id), ctypes.byref(st), _ptr(out), cap, ctypes.byref(n))
    if rc == FH_ERR_NOT_READY:
        return int(st.value), None
    if rc == FH_ERR_CAPACITY and out is None:
        out = np.zeros(int(n.value), dtype=CANDIDATE_DTYPE)
        rc = load().fh_poll(server, int(job_id), ctypes.byref(st), _ptr(out), out.shape[0],
                            ctypes.byref(n))
    _check(rc, "fh_poll")
    return int(st.value), out


def fh_job_get_stats(server, job_id: int) -> dict:
    s = fh_job_stats()
    _check(load().fh_job_get_stats(server, int(job_id), ctypes.byref(s)), "fh_job_get_stats")
    return {k: getattr(s, k) for k, _ in fh_job_stats._fields_}


def fh_cancel(server, job_id: int) -> None:
    _check(load().fh_cancel(server, int(job_id)), "fh_cancel")


def fh_server_drain(server, timeout_s: float) -> None:
    _check(load().fh_server_drain(server, float(timeout_s)), "fh_server_drain")


def fh_server_pause(server, paused: bool) -> None:
    _check(load().fh_server_pause(server, int(bool(paused))), "fh_server_pause")
