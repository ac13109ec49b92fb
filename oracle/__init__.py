"""CPU oracle of the frequency-Hough hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product (the CUDA library and its Python
binding) never imports, links or calls it, and it never imports the product.
It shares no code with the CUDA path; the only common module is the seeded
input generator, which holds none of the method's arithmetic.

The arithmetic lives in ``fh_oracle.c`` (plain C, IEEE binary64 in the order
written, ``-ffp-contract=off``), steps a1-a6 of the hot path, each citing the
passage of the paper it follows.  This module compiles it with gcc on first
use and wraps it with numpy arrays; the reporting columns of a candidate
(f0, fdot, critical ratio, Eq. cr) are computed here with numpy in binary64.

Pins (checked by ``tests/test_oracle_pins.py`` against facts independent of
this code): direct counting and an independent Python brute force on tiny
inputs; exact rational evaluation of the stripe start; the no-Doppler closed
form s = K k - K/2; the K-cells-per-peak row invariant; the binomial law of the
noise-only count (Eqs. phmsig, houghmean) including the paper's
N = 61594 / p0 = 0.0755 figures; injected-line recovery; selection against
sort-and-take-k and hand-computed cases.  Nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

from . import coincidence  # noqa: F401  (candidate clustering and coincidences)
from . import peakmap  # noqa: F401  (peakmap construction and cleaning)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfh_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.fho_num_threads.restype = ctypes.c_int
            lib.fho_set_num_threads.argtypes = [ctypes.c_int]
            lib.fho_doppler_factor.argtypes = [i32, P, i32, P, P]
            lib.fho_positions.argtypes = [i32, P, P, i32, P, f64, f64, i32, P]
            lib.fho_shift_tables.argtypes = [i32, P, f64, f64, f64, f64, P, P]
            lib.fho_hough_map.argtypes = [i32, P, P, P, P, i32, i32, i32, P, P, P]
            lib.fho_hough_map_direct.argtypes = [i32, P, P, P, P, i32, i32, i32, P, P]
            lib.fho_profile.argtypes = [P, i32, i32, P, P]
            lib.fho_select.argtypes = [P, P, i32, i32, i32, i32, i32, i32, P, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(_load().fho_num_threads())


def set_num_threads(n: int) -> None:
    _load().fho_set_num_threads(int(n))


# ---------------------------------------------------------------- a1 .. a3
def doppler_factor(v: np.ndarray, sky: np.ndarray) -> np.ndarray:
    """a1: r[d, i] = 1 / (1 + v_i . n_d)  (Eq. fdopp)."""
    v = _c(v, np.float64).reshape(-1, 3)
    sky = _c(sky, np.float64).reshape(-1, 3)
    r = np.empty((sky.shape[0], v.shape[0]), dtype=np.float64)
    _load().fho_doppler_factor(v.shape[0], _p(v), sky.shape[0], _p(sky), _p(r))
    return r


def positions(offsets, freq, r, f0_min: float, kt: float, k_over: int) -> np.ndarray:
    """a2: 32.32 fixed-point first-cell positions A[d, p] (Sec. VI, Eq. freqres)."""
    offsets = _c(offsets, np.int64)
    freq = _c(freq, np.float64)
    r = _c(r, np.float64)
    n_fft = offsets.shape[0] - 1
    r = r.reshape(-1, n_fft)
    A = np.empty((r.shape[0], int(offsets[-1])), dtype=np.int64)
    _load().fho_positions(n_fft, _p(offsets), _p(freq), r.shape[0], _p(r),
                          float(f0_min), float(kt), int(k_over), _p(A))
    return A


def shift_tables(t, t_ref: float, kt: float, fdot_min: float, fdot_step: float):
    """a3: (S0, D) int64 per FFT (Eqs. uno, sdstep)."""
    t = _c(t, np.float64)
    S0 = np.empty(t.shape[0], dtype=np.int64)
    D = np.empty(t.shape[0], dtype=np.int64)
    _load().fho_shift_tables(t.shape[0], _p(t), float(t_ref), float(kt), float(fdot_min),
                             float(fdot_step), _p(S0), _p(D))
    return S0, D


# ---------------------------------------------------------------- a4 + a5
def hough_map(offsets, A_dir, S0, D, k_over: int, n_f0: int, n_fdot: int = None,
              rows=None, weights=None) -> np.ndarray:
    """a4 + a5: number counts of one direction (differential +1/-1, cumulative
    sum); with ``weights`` (n_fft integers, already quantised) the adaptive
    map of Eq. ncountadap: each FFT's peaks add its weight instead of 1."""
    offsets = _c(offsets, np.int64)
    A_dir = _c(A_dir, np.int64)
    S0 = _c(S0, np.int64)
    D = _c(D, np.int64)
    if rows is None:
        n_rows = int(n_fdot)
        rp = None
    else:
        rows = _c(rows, np.int32)
        n_rows = rows.shape[0]
        rp = _p(rows)
    wp = None
    if weights is not None:
        weights = _c(weights, np.int32)
        wp = _p(weights)
    m = np.empty((n_rows, int(n_f0)), dtype=np.int32)
    _load().fho_hough_map(offsets.shape[0] - 1, _p(offsets), _p(A_dir), _p(S0), _p(D),
                          int(k_over), int(n_f0), n_rows, rp, wp, _p(m))
    return m


def hough_map_direct(offsets, A_dir, S0, D, k_over: int, n_f0: int, n_fdot: int,
                     weights=None) -> np.ndarray:
    """Direct per-cell counting (tiny inputs): the plain definition of Eq. ncount
    (Eq. ncountadap with ``weights``)."""
    offsets = _c(offsets, np.int64)
    A_dir = _c(A_dir, np.int64)
    S0 = _c(S0, np.int64)
    D = _c(D, np.int64)
    wp = None
    if weights is not None:
        weights = _c(weights, np.int32)
        wp = _p(weights)
    m = np.empty((int(n_fdot), int(n_f0)), dtype=np.int32)
    _load().fho_hough_map_direct(offsets.shape[0] - 1, _p(offsets), _p(A_dir), _p(S0),
                                 _p(D), int(k_over), int(n_f0), int(n_fdot), wp, _p(m))
    return m


# Each direction's quantised weights sum below 2^30 (a cell of a bin-grid
# peakmap takes at most two stripes of one FFT, so its weighted counts stay
# below 2^31).  Off-grid peakmaps can put more stripes of one FFT on a cell;
# ``count_bound`` bounds every count of any peakmap and ``search`` refuses
# weights whose bound reaches 2^31.
WEIGHT_SUM_LIMIT = (1 << 30) - 1
COUNT_LIMIT = 1 << 31


def stripe_overlap(offsets, A_dir, k_over: int) -> np.ndarray:
    """Per FFT, the largest number of its stripes that can cover one cell on
    any row: the most of its positions inside a half-open window of K cells.

    Two stripes of one FFT (Eq. due: K cells from s = floor((A - shift)/2^32))
    share a cell only if s_q - s_p <= K - 1, which forces A_q - A_p < K 2^32;
    so the stripes on a common cell have positions within less than K cells
    of the smallest, whatever the row.  (For a bin-grid peakmap this is 1 or
    2; dense off-grid peaks give more.)"""
    offsets = np.asarray(offsets, dtype=np.int64)
    A_dir = np.asarray(A_dir, dtype=np.int64)
    width = int(k_over) << 32
    n_fft = offsets.shape[0] - 1
    c = np.zeros(n_fft, dtype=np.int64)
    for i in range(n_fft):
        a = A_dir[int(offsets[i]):int(offsets[i + 1])]
        if a.shape[0] == 0:
            continue
        # for each peak p, the first q with A_q >= A_p + K 2^32 (positions ascending)
        q = np.searchsorted(a, a + width, side="left")
        c[i] = int((q - np.arange(a.shape[0])).max())
    return c


def count_bound(offsets, A_dir, k_over: int, W=None) -> int:
    """An upper bound of every count of one direction's map (Eq. ncountadap):
    sum over FFTs of its weight (1 for the plain map) times stripe_overlap."""
    c = stripe_overlap(offsets, A_dir, k_over)
    if W is None:
        return int(c.sum())
    return int(sum(int(w) * int(x) for w, x in zip(np.asarray(W).ravel(), c)))


def quantize_weights(w, frac_bits: int) -> np.ndarray:
    """Adaptive weights (Eq. ncountadap) as integers: W = rint(w 2^F), binary64,
    ties to even.  Weights must be finite and >= 0 and each direction's sum of
    W below 2^30 (so that no count can leave int32)."""
    w = np.asarray(w, dtype=np.float64)
    if not (0 <= int(frac_bits) <= 24):
        raise ValueError("frac_bits must be in [0, 24]")
    if not np.all(np.isfinite(w)) or np.any(w < 0):
        raise ValueError("weights must be finite and >= 0")
    W = np.rint(w * float(2 ** int(frac_bits)))
    if np.any(W.reshape(W.shape[0] if W.ndim > 1 else 1, -1).sum(axis=1) > WEIGHT_SUM_LIMIT):
        raise ValueError("a direction's quantised weights sum to 2^30 or more")
    return W.astype(np.int64)


# ---------------------------------------------------------------- a6
def profile(hmap: np.ndarray):
    """Max count over rows per cell, and the smallest row reaching it (Sec. VIII)."""
    hmap = _c(hmap, np.int32)
    n_fdot, n_f0 = hmap.shape
    pc = np.empty(n_f0, dtype=np.int32)
    pr = np.empty(n_f0, dtype=np.int32)
    _load().fho_profile(_p(hmap), n_fdot, n_f0, _p(pc), _p(pr))
    return pc, pr


def select(pcount, prow, subband_cells: int, top_k: int, excl: int, sep: int, n_thr: int):
    """Greedy per-sub-band picks (Sec. VIII); arrays (n_sb, top_k), -1 when empty."""
    pcount = _c(pcount, np.int32)
    prow = _c(prow, np.int32)
    n_f0 = pcount.shape[0]
    n_sb = (n_f0 + subband_cells - 1) // subband_cells
    cell = np.empty((n_sb, top_k), dtype=np.int32)
    row = np.empty((n_sb, top_k), dtype=np.int32)
    cnt = np.empty((n_sb, top_k), dtype=np.int32)
    _load().fho_select(_p(pcount), _p(prow), n_f0, int(subband_cells), int(top_k), int(excl),
                       int(sep), int(n_thr), _p(cell), _p(row), _p(cnt))
    return cell, row, cnt


def report(cell, row, cnt, f0_min: float, kt: float, fdot_min: float, fdot_step: float,
           n_fft: int, p0: float, s1=None, s2=None):
    """Reporting columns of each pick, binary64: cell-centre frequency, row
    spin-down and critical ratio CR = (n - N p0) / sqrt(N p0 (1 - p0)) (Eq. cr).
    Adaptive map (``s1``, ``s2`` = per-direction sums of the integer weights
    and of their squares): mean p0 S1 and variance p0 (1 - p0) S2 of the
    weighted noise count, CR = (n - S1 p0) / sqrt((S2 p0) (1 - p0)); for unit
    weights S1 = S2 = N and this is Eq. cr, operation for operation."""
    cell = np.asarray(cell)
    row = np.asarray(row)
    cnt = np.asarray(cnt)
    valid = cnt >= 0
    f0 = np.where(valid, f0_min + (cell.astype(np.float64) + 0.5) / kt, 0.0)
    fdot = np.where(valid, fdot_min + row.astype(np.float64) * fdot_step, 0.0)
    if s1 is None:
        np0 = float(n_fft) * p0
        var = np0 * (1.0 - p0)
    else:
        shape = (-1,) + (1,) * (cnt.ndim - 1)
        np0 = (np.asarray(s1, dtype=np.int64).astype(np.float64) * p0).reshape(shape)
        var = ((np.asarray(s2, dtype=np.int64).astype(np.float64) * p0) * (1.0 - p0)).reshape(shape)
    cr = np.where(valid, (cnt.astype(np.float64) - np0) / np.sqrt(var), 0.0)
    return f0, fdot, cr


# ---------------------------------------------------------------- whole path
def search(inp, params: dict, want_maps: bool = False, dirs=None, weights=None,
           frac_bits: int = 0):
    """Steps a1-a6 for every direction of ``inp`` (a synth.Inputs).

    Returns a dict with r, A, S0, D, per-direction profiles, candidate arrays
    (n_dir, n_sb, top_k) and, if asked, the maps (n_dir, n_fdot, n_f0).  With
    ``weights`` (n_dir x n_fft reals) the adaptive map (Eq. ncountadap) of the
    weights quantised by ``quantize_weights(weights, frac_bits)``.
    """
    kt = float(params["k_over"]) * float(params["t_fft"])
    sky = inp.sky if dirs is None else inp.sky[np.asarray(dirs)]
    r = doppler_factor(inp.v, sky)
    A = positions(inp.offsets, inp.freq, r, params["f0_min"], kt, params["k_over"])
    S0, D = shift_tables(inp.t, params["t_ref"], kt, params["fdot_min"], params["fdot_step"])
    out = dict(r=r, A=A, S0=S0, D=D, pcount=[], prow=[], cell=[], row=[], count=[])
    maps = []
    W = None
    if weights is not None:
        W = quantize_weights(np.asarray(weights, dtype=np.float64).reshape(sky.shape[0], -1),
                             frac_bits)
        for d in range(sky.shape[0]):
            if count_bound(inp.offsets, A[d], params["k_over"], W[d]) >= COUNT_LIMIT:
                raise ValueError("direction %d: weighted counts could reach 2^31 (dense peaks "
                                 "of one FFT under large weights)" % d)
        out["W"] = W
        out["s1"] = W.sum(axis=1)
        out["s2"] = (W * W).sum(axis=1)
    for d in range(sky.shape[0]):
        m = hough_map(inp.offsets, A[d], S0, D, params["k_over"], params["n_f0"],
                      params["n_fdot"], weights=None if W is None else W[d])
        pc, pr = profile(m)
        c, rr, n = select(pc, pr, params["subband_cells"], params["top_k"],
                          params["excl_cells"], params["sep_cells"], params["n_thr"])
        out["pcount"].append(pc)
        out["prow"].append(pr)
        out["cell"].append(c)
        out["row"].append(rr)
        out["count"].append(n)
        if want_maps:
            maps.append(m)
        del m
    for k in ("pcount", "prow", "cell", "row", "count"):
        out[k] = np.stack(out[k])
    f0, fdot, cr = report(out["cell"], out["row"], out["count"], params["f0_min"], kt,
                          params["fdot_min"], params["fdot_step"], inp.t.shape[0],
                          params["p0"], out.get("s1"), out.get("s2"))
    out.update(f0=f0, fdot=fdot, cr=cr)
    if want_maps:
        out["maps"] = np.stack(maps)
    return out


# ---------------------------------------------------------------- refined grid
def refine_maps(inp, params: dict, cell: int, row: int, sky_dirs, k_fdot: int):
    """Refined-grid FH maps around one coarse candidate (cell b_c, row j_c of
    the coarse grid), Sec. "Refined Grid in the parameter space".

    Frequency: the same K-over-resolved cells, +-1 coarse bin around the
    candidate: cells b_c - K .. b_c + K (refined cell 0 = coarse cell b_c - K).
    Spin-down: step fdot_step / K_fdot, 2 K_fdot rows below the coarse value and
    2 K_fdot - 1 above (4 K_fdot rows): refined row 0 lies on coarse row
    j_c - 2, i.e. its shift is S0_i + (j_c - 2) D_i, and a refined row step is
    D'_i = floor((fdot_step / K_fdot) c_i 2^32).  Sky: the given refined
    directions.  Every peak of the peakmap takes part.
    Returns maps (n_ref, 4 K_fdot, 2 K + 1)."""
    K = int(params["k_over"])
    kt = float(K) * float(params["t_fft"])
    sky_dirs = np.asarray(sky_dirs, dtype=np.float64).reshape(-1, 3)
    S0, D = shift_tables(inp.t, params["t_ref"], kt, params["fdot_min"], params["fdot_step"])
    _, Dr = shift_tables(inp.t, params["t_ref"], kt, 0.0,
                         float(params["fdot_step"]) / float(k_fdot))
    lo = int(cell) - K
    S0r = S0 + (int(row) - 2) * D + (np.int64(lo) << np.int64(32))
    r = doppler_factor(inp.v, sky_dirs)
    A = positions(inp.offsets, inp.freq, r, params["f0_min"], kt, K)
    return np.stack([hough_map(inp.offsets, A[d], S0r, Dr, K, 2 * K + 1, 4 * int(k_fdot))
                     for d in range(sky_dirs.shape[0])])


def refine(inp, params: dict, cells, rows, sky_ref, k_fdot: int):
    """One refined candidate per coarse candidate (cells[c], rows[c]): the cell
    of largest count of refine_maps over all refined directions sky_ref[c],
    rows and cells (ties: smallest direction, then row, then cell).

    Returns arrays per candidate: dir, row, cell (coarse-grid index), count,
    f0 = f0_min + (cell + 0.5) / KT, fdot = (fdot_min + (j_c - 2) fdot_step) +
    row (fdot_step / K_fdot) and CR (Eq. cr), binary64.
    """
    K = int(params["k_over"])
    kt = float(K) * float(params["t_fft"])
    cells = np.asarray(cells, dtype=np.int64)
    rows = np.asarray(rows, dtype=np.int64)
    sky_ref = np.asarray(sky_ref, dtype=np.float64)
    n_cand = sky_ref.shape[0]
    step_ref = float(params["fdot_step"]) / float(k_fdot)
    out = {k: np.zeros(n_cand, dtype=np.int64) for k in ("dir", "row", "cell", "count")}
    for k in ("f0", "fdot", "cr"):
        out[k] = np.zeros(n_cand)
    for c in range(n_cand):
        maps = refine_maps(inp, params, int(cells[c]), int(rows[c]), sky_ref[c], k_fdot)
        cnt = int(maps.max())
        d, j, b = (int(x) for x in np.argwhere(maps == cnt)[0])   # lexicographic: dir, row, cell
        lo = int(cells[c]) - K
        out["dir"][c], out["row"][c], out["cell"][c], out["count"][c] = d, j, lo + b, cnt
        out["f0"][c] = params["f0_min"] + (float(lo + b) + 0.5) / kt
        fdot_lo = params["fdot_min"] + float(int(rows[c]) - 2) * params["fdot_step"]
        out["fdot"][c] = fdot_lo + float(j) * step_ref
        np0 = float(inp.t.shape[0]) * params["p0"]
        out["cr"][c] = (float(cnt) - np0) / math.sqrt(np0 * (1.0 - params["p0"]))
    return out
