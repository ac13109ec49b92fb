"""Seeded synthetic inputs for the frequency-Hough (FH) transform.

This module produces the *inputs* of the method -- peakmaps, detector
velocities, sky directions and the grid parameters a caller passes to a plan --
and nothing of the method's own arithmetic (no Doppler correction, no stripe
mapping, no counting, no selection).  Both the CUDA library and the CPU oracle
are fed from here, so that the two sides see bit-identical inputs.

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).  Draw
``i`` of stream ``(seed, stream)`` is ``mix(key + (i + 1) * GAMMA)`` with the
published SplitMix64 finaliser ``mix``; so any draw can be recomputed from its
counter alone, in any language and in any order.

Shapes follow the paper's workloads:

* peaks are (FFT start time, FFT bin) pairs (peakmap definition, Sec. V) with
  frequencies exactly ``k / T_FFT``; each bin is a peak independently with
  probability ``p`` (the i.i.d. stand-in for threshold + local maximum selection);
* FFT start times are ``i * T_FFT`` or half-interlaced ``i * T_FFT / 2``
  (short-FFT database, Sec. IV);
* the spin-down grid has step ``delta_f / T_obs`` (Eq. sdstep, K_fdot = 1) and
  contains fdot = 0;
* the frequency grid is over-resolved by ``K`` (Eq. freqres);
* the detector velocity is a 30 km/s circular orbit plus a 0.46 km/s diurnal
  term (the v_orb + v_rot of Eq. fdopp), in units of c, ecliptic frame;
* sky directions are points of the ecliptic grid of Sec. VII.C / App. A2.

The paper analysed Virgo VSR2/VSR4 peakmaps; those data are not available, so
these seeded peakmaps stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace
from typing import Optional

import numpy as np

# --------------------------------------------------------------------------
# SplitMix64 counter generator
# --------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of one independent stream: the mixed (seed, stream) pair."""
    base = ((int(seed) & 0xFFFFFFFFFFFF) << 16) | (int(stream) & 0xFFFF)
    z = np.array([(base + 0x9E3779B97F4A7C15) & _MASK64], dtype=np.uint64)
    return _mix(z)[0]


def draws_u64(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Raw 64-bit draws for the given counters (any integer array)."""
    key = stream_key(seed, stream)
    c = np.asarray(counters).astype(np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + (c + np.uint64(1)) * _GAMMA)


def uniform(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of the draw."""
    return (draws_u64(seed, stream, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _threshold_u64(p: float) -> np.uint64:
    """Integer threshold t with P(draw < t) = p (to 2^-64)."""
    if p <= 0.0:
        return np.uint64(0)
    if p >= 1.0:
        return np.uint64(_MASK64)
    return np.uint64(int(p * 2.0 ** 64))


# streams
_S_PEAKS, _S_LINE, _S_PHASE, _S_SKY = 1, 2, 3, 4

C_KMS = 299792.458
V_ORB_KMS = 30.0
V_ROT_KMS = 0.46
OMEGA_ORB = 2.0 * math.pi / (365.25636 * 86400.0)
OMEGA_ROT = 2.0 * math.pi / 86164.09
EPSILON = math.radians(23.44)
DAY = 86400.0


# --------------------------------------------------------------------------
# Workload description
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    """One FH workload: peakmap shape, grids, sky patch and selection rule."""
    name: str
    t_fft: float              # FFT duration [s]
    n_fft: int                # number of FFTs
    t_step: float             # spacing of FFT start times [s]
    t_obs: float              # observation span that sets the spin-down step [s]
    f_lo: float               # band lower edge [Hz] (= cell 0 lower edge)
    f_hi: float               # band upper edge [Hz]
    k_over: int = 10          # frequency over-resolution K
    p_peak: float = 0.05      # probability that an FFT bin is a peak
    fdot_lo: float = 0.0      # spin-down range [Hz/s]; the grid contains 0
    fdot_hi: float = 0.0
    n_fdot_sym: int = 0       # if > 0: rows (j - n_fdot_sym) * step, j = 0..2*n_fdot_sym
    line_f0: Optional[float] = None   # injected line: source frequency at t_ref [Hz]
    line_fdot: float = 0.0            # injected line spin-down [Hz/s]
    line_presence: float = 0.9        # probability that the line is a peak in an FFT
    line_dir: int = 0                 # sky direction index that carries the line
    doppler: bool = False     # detector motion on (else v = 0)
    n_dir: int = 1            # number of sky directions
    subband_hz: float = 0.1   # candidate sub-band width [Hz]
    top_k: int = 1            # picks per sub-band
    excl_bins: int = 0        # exclusion half-width, in coarse (1/T_FFT) bins
    sep_bins: int = 0         # minimum separation, in coarse bins
    n_thr: int = 0            # minimum count of a pick
    seed: int = 1

    # ---- grids (the caller's plan parameters) ----
    @property
    def kt(self) -> float:
        return float(self.k_over) * self.t_fft

    @property
    def n_f0(self) -> int:
        return int(round((self.f_hi - self.f_lo) * self.t_fft)) * self.k_over

    @property
    def fdot_step(self) -> float:
        return (1.0 / self.t_fft) / self.t_obs

    @property
    def fdot_rows(self) -> tuple:
        """(j0, n_fdot): row j has fdot = (j - j0) * step."""
        if self.n_fdot_sym > 0:
            return self.n_fdot_sym, 2 * self.n_fdot_sym + 1
        step = self.fdot_step
        j0 = int(math.ceil(-self.fdot_lo / step - 1e-9)) if self.fdot_lo < 0 else 0
        jhi = int(math.floor(self.fdot_hi / step + 1e-9)) if self.fdot_hi > 0 else 0
        return j0, j0 + jhi + 1

    @property
    def n_fdot(self) -> int:
        return self.fdot_rows[1]

    @property
    def fdot_min(self) -> float:
        return -self.fdot_rows[0] * self.fdot_step

    @property
    def t_ref(self) -> float:
        return 0.5 * (0.0 + (self.n_fft - 1) * self.t_step)

    @property
    def subband_cells(self) -> int:
        return int(round(self.subband_hz * self.kt))

    @property
    def margin_bins(self) -> int:
        """FFT bins supplied beyond each band edge so that every band cell is complete."""
        j0, n = self.fdot_rows
        fmax = max(abs(self.fdot_min), abs(self.fdot_min + (n - 1) * self.fdot_step))
        drift = fmax * 0.5 * (self.n_fft - 1) * self.t_step
        dop = self.f_hi * (V_ORB_KMS + V_ROT_KMS) / C_KMS if self.doppler else 0.0
        return int(math.ceil((drift + dop) * self.t_fft)) + 1

    def plan_params(self) -> dict:
        j0, n_fdot = self.fdot_rows
        return dict(
            t_fft=self.t_fft, k_over=self.k_over, f0_min=self.f_lo, n_f0=self.n_f0,
            fdot_min=self.fdot_min, fdot_step=self.fdot_step, n_fdot=n_fdot,
            t_ref=self.t_ref, subband_cells=self.subband_cells, top_k=self.top_k,
            excl_cells=self.excl_bins * self.k_over, sep_cells=self.sep_bins * self.k_over,
            n_thr=self.n_thr, p0=self.p_peak)

    @property
    def bins(self) -> tuple:
        k_lo = int(round(self.f_lo * self.t_fft)) - self.margin_bins
        k_hi = int(round(self.f_hi * self.t_fft)) + self.margin_bins
        return k_lo, k_hi

    def expected_peaks(self) -> float:
        k_lo, k_hi = self.bins
        return self.n_fft * (k_hi - k_lo) * self.p_peak


# --------------------------------------------------------------------------
# Named workloads (sizes of the paper's configurations)
# --------------------------------------------------------------------------
def _n_half_interlaced(t_fft: float, t_obs: float) -> int:
    return int(math.floor(t_obs / (0.5 * t_fft)))


WORKLOADS = {
    # T_FFT = 1024 s, 200 FFTs back to back, 100-101 Hz, no detector motion,
    # 21 spin-down rows centred on 0, injected line 100.37 Hz / -2e-10 Hz/s.
    "nodoppler_T1024_N200_100Hz": Workload(
        name="nodoppler_T1024_N200_100Hz", t_fft=1024.0, n_fft=200, t_step=1024.0,
        t_obs=200 * 1024.0, f_lo=100.0, f_hi=101.0, k_over=10, p_peak=0.05,
        n_fdot_sym=10, line_f0=100.37, line_fdot=-2e-10, line_presence=0.9,
        doppler=False, n_dir=1, subband_hz=0.1, top_k=2, excl_bins=4, sep_bins=8, seed=1),
    # T_FFT = 8192 s, half-interlaced over 150 days, 50-51 Hz, one sky point,
    # spin-down -1e-8 .. +1e-9 Hz/s, p = 0.04, top-5 per 0.1 Hz.
    "single_sky_T8192_150d_50Hz": Workload(
        name="single_sky_T8192_150d_50Hz", t_fft=8192.0,
        n_fft=_n_half_interlaced(8192.0, 150 * DAY), t_step=4096.0, t_obs=150 * DAY,
        f_lo=50.0, f_hi=51.0, k_over=10, p_peak=0.04, fdot_lo=-1e-8, fdot_hi=1e-9,
        line_f0=50.3137, line_fdot=-3e-9, line_presence=0.9, doppler=True, n_dir=1,
        subband_hz=0.1, top_k=5, excl_bins=4, sep_bins=8, seed=2),
    # The 100 Hz peakmap with detector motion, 256 directions of the ecliptic
    # grid around a seeded centre; the line is Doppler-modulated for one of them.
    "sky_patch256_T1024_N200_100Hz": Workload(
        name="sky_patch256_T1024_N200_100Hz", t_fft=1024.0, n_fft=200, t_step=1024.0,
        t_obs=200 * 1024.0, f_lo=100.0, f_hi=101.0, k_over=10, p_peak=0.05,
        n_fdot_sym=10, line_f0=100.37, line_fdot=-2e-10, line_presence=0.9,
        line_dir=37, doppler=True, n_dir=256, subband_hz=0.1, top_k=2, excl_bins=4,
        sep_bins=8, seed=3),
    # T_FFT = 1024 s, half-interlaced over one year (N = 61594, the paper's N),
    # 900-910 Hz, spin-down -1e-8 .. +1e-9 Hz/s, 64 directions.
    "highfreq_T1024_1yr_900Hz_64dir": Workload(
        name="highfreq_T1024_1yr_900Hz_64dir", t_fft=1024.0, n_fft=61594, t_step=512.0,
        t_obs=365 * DAY, f_lo=900.0, f_hi=910.0, k_over=10, p_peak=0.04,
        fdot_lo=-1e-8, fdot_hi=1e-9, line_f0=903.21, line_fdot=-1e-9, line_presence=0.9,
        line_dir=5, doppler=True, n_dir=64, subband_hz=0.1, top_k=2, excl_bins=4,
        sep_bins=8, seed=5),
}


# --------------------------------------------------------------------------
# Sky directions: ecliptic grid (Sec. VII.C, App. A2)
# --------------------------------------------------------------------------
def doppler_number(f0: float, t_fft: float) -> float:
    """N_D = f0 * Omega_orb * R_orb * T_FFT / c (Eq. ND): Doppler band in FFT bins."""
    return f0 * (V_ORB_KMS / C_KMS) * t_fft


def _lat_walk(n_d: float, k: float, m: int) -> float:
    b = math.pi / 2
    for _ in range(m):
        s = math.sin(b)
        if s <= 0.0:
            return -1.0
        b = b - k / (n_d * s)
    return b


def ecliptic_grid(n_d: float) -> np.ndarray:
    """Unit vectors of the coarse sky grid for Doppler number ``n_d``.

    Latitudes are walked from the pole with step k / (N_D sin(beta)) and the
    constant k <= 1 is bisected so that the walk lands exactly on the equator;
    the southern half mirrors the northern one.  On each latitude the longitude
    step is the largest submultiple of 2*pi not above 1 / (N_D cos(beta)).
    """
    m = 0
    b = math.pi / 2
    while b > 0.0:
        b = b - 1.0 / (n_d * math.sin(b))
        m += 1
    lo, hi = 0.0, 1.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if _lat_walk(n_d, mid, m) > 0.0:
            lo = mid
        else:
            hi = mid
    k = lo
    lats = [math.pi / 2]
    b = math.pi / 2
    for _ in range(m - 1):
        b = b - k / (n_d * math.sin(b))
        lats.append(b)
    lats.append(0.0)
    lats = lats + [-x for x in reversed(lats[:-1])]
    pts = []
    for beta in lats:
        nl = max(1, int(math.ceil(2.0 * math.pi * n_d * math.cos(beta) - 1e-12)))
        for l in range(nl):
            lam = 2.0 * math.pi * l / nl
            pts.append((math.cos(beta) * math.cos(lam), math.cos(beta) * math.sin(lam),
                        math.sin(beta)))
    return np.asarray(pts, dtype=np.float64)


def refined_sky(n_hat, n_d: float, k_sky: int) -> np.ndarray:
    """Refined sky directions around a coarse direction (Sec. "Refined grid in
    the sky"): a k_sky x k_sky rectangle in ecliptic (lambda, beta) centred on
    it, k_sky = 2 N_layers + 1 odd, whose steps are the local coarse-grid
    spacings of ecliptic_grid divided by k_sky: beta step 1 / (N_D sin(beta)),
    longitude step 2 pi / ceil(2 pi N_D cos(beta)).  Rows of beta, then lambda;
    the centre (the coarse direction) is index (k_sky^2 - 1) / 2."""
    x, y, z = (float(c) for c in np.asarray(n_hat, dtype=np.float64).reshape(3))
    beta = math.asin(max(-1.0, min(1.0, z)))
    lam = math.atan2(y, x)
    db = min(1.0 / (n_d * max(abs(math.sin(beta)), 1e-3)), math.pi / 8)
    dl = 2.0 * math.pi / max(1, int(math.ceil(2.0 * math.pi * n_d * math.cos(beta) - 1e-12)))
    half = (int(k_sky) - 1) // 2
    pts = []
    for b in range(-half, half + 1):
        bb = beta + b * db / k_sky
        for a in range(-half, half + 1):
            ll = lam + a * dl / k_sky
            pts.append((math.cos(bb) * math.cos(ll), math.cos(bb) * math.sin(ll), math.sin(bb)))
    pts = np.asarray(pts, dtype=np.float64)
    pts[(k_sky * k_sky - 1) // 2] = (x, y, z)   # the coarse direction itself, exactly
    return pts


def pair_order(sky: np.ndarray) -> np.ndarray:
    """An order of the directions that lists them in neighbouring pairs (entries
    2u and 2u + 1): repeatedly the remaining direction farthest from the patch's
    centroid with its nearest remaining neighbour (ties: lower index).  A sky
    patch scanned this way keeps each pair's Doppler shifts within about one
    input bin of each other."""
    n = sky.shape[0]
    if n < 3:
        return np.arange(n)
    cen = sky.mean(axis=0)
    cen = cen / np.linalg.norm(cen)
    ang = np.arccos(np.clip(sky @ sky.T, -1.0, 1.0))
    rem = list(range(n))
    order = []
    while len(rem) > 1:
        a = min(rem, key=lambda i: (float(sky[i] @ cen), i))
        rem.remove(a)
        b = min(rem, key=lambda j: (float(ang[a, j]), j))
        rem.remove(b)
        order += [a, b]
    order += rem
    return np.asarray(order)


def sky_patch(w: Workload) -> np.ndarray:
    """``w.n_dir`` grid directions nearest a seeded centre, shape (n_dir, 3),
    listed in neighbouring pairs (``pair_order``)."""
    if not w.doppler and w.n_dir == 1:
        return np.array([[1.0, 0.0, 0.0]])
    n_d = doppler_number(w.f_hi, w.t_fft)
    grid = ecliptic_grid(n_d)
    u = uniform(w.seed, _S_SKY, np.arange(2))
    beta_c = math.asin(2.0 * u[0] - 1.0) * 0.8
    lam_c = 2.0 * math.pi * u[1]
    c = np.array([math.cos(beta_c) * math.cos(lam_c), math.cos(beta_c) * math.sin(lam_c),
                  math.sin(beta_c)])
    dots = grid @ c
    order = np.lexsort((np.arange(len(grid)), -dots))
    if w.n_dir > len(grid):
        raise ValueError("sky patch larger than the grid")
    patch = grid[order[: w.n_dir]]
    return np.ascontiguousarray(patch[pair_order(patch)])


# --------------------------------------------------------------------------
# Detector velocity (units of c, ecliptic frame), one vector per FFT
# --------------------------------------------------------------------------
def fft_times(w: Workload) -> np.ndarray:
    return np.arange(w.n_fft, dtype=np.float64) * w.t_step


def velocities(w: Workload) -> np.ndarray:
    n = w.n_fft
    if not w.doppler:
        return np.zeros((n, 3), dtype=np.float64)
    ph = uniform(w.seed, _S_PHASE, np.arange(2)) * 2.0 * math.pi
    t = fft_times(w) + 0.5 * w.t_fft
    a = OMEGA_ORB * t + ph[0]
    d = OMEGA_ROT * t + ph[1]
    vo = V_ORB_KMS / C_KMS
    vr = V_ROT_KMS / C_KMS
    v = np.empty((n, 3), dtype=np.float64)
    v[:, 0] = -vo * np.sin(a) - vr * np.sin(d)
    v[:, 1] = vo * np.cos(a) + vr * math.cos(EPSILON) * np.cos(d)
    v[:, 2] = vr * math.sin(EPSILON) * np.cos(d)
    return v


# --------------------------------------------------------------------------
# Peakmap
# --------------------------------------------------------------------------
@dataclass
class Inputs:
    """Arrays a caller hands to the library (all C-contiguous)."""
    w: Workload
    t: np.ndarray        # (n_fft,) f64 FFT start times [s]
    offsets: np.ndarray  # (n_fft + 1,) i64 CSR offsets of the peaks of each FFT
    freq: np.ndarray     # (n_peaks,) f64 peak frequencies [Hz], ascending within an FFT
    v: np.ndarray        # (n_fft, 3) f64 detector velocity / c
    sky: np.ndarray      # (n_dir, 3) f64 unit vectors

    @property
    def n_peaks(self) -> int:
        return int(self.offsets[-1])


def line_bins(w: Workload, v: np.ndarray, sky: np.ndarray, t: np.ndarray) -> tuple:
    """FFT bin of the injected line in each FFT and its presence mask.

    Forward signal model only (what the detector records): the source frequency
    f0 + fdot (t - t_ref) seen through the Doppler factor (1 + v.n) of Eq. fdopp.
    """
    if w.line_f0 is None:
        return np.zeros(w.n_fft, dtype=np.int64), np.zeros(w.n_fft, dtype=bool)
    n = sky[w.line_dir]
    f_src = w.line_f0 + w.line_fdot * (t - w.t_ref)
    f_obs = f_src * (1.0 + v @ n)
    k = np.rint(f_obs * w.t_fft).astype(np.int64)
    present = draws_u64(w.seed, _S_LINE, np.arange(w.n_fft)) < _threshold_u64(w.line_presence)
    return k, present


def make_inputs(w: Workload, chunk_cells: int = 1 << 24) -> Inputs:
    """Generate the seeded peakmap, velocities and sky patch of a workload."""
    t = fft_times(w)
    v = velocities(w)
    sky = sky_patch(w)
    k_lo, k_hi = w.bins
    nb = k_hi - k_lo
    thr = _threshold_u64(w.p_peak)
    lk, lp = line_bins(w, v, sky, t)
    counts = np.zeros(w.n_fft, dtype=np.int64)
    pieces = []
    rows = max(1, chunk_cells // nb)
    for i0 in range(0, w.n_fft, rows):
        i1 = min(w.n_fft, i0 + rows)
        ctr = (np.arange(i0, i1, dtype=np.int64)[:, None] * nb
               + np.arange(nb, dtype=np.int64)[None, :])
        mask = draws_u64(w.seed, _S_PEAKS, ctr) < thr
        for i in range(i0, i1):
            if lp[i] and k_lo <= lk[i] < k_hi:
                mask[i - i0, lk[i] - k_lo] = True
        ii, kk = np.nonzero(mask)
        counts[i0:i1] = np.bincount(ii, minlength=i1 - i0)
        pieces.append(kk.astype(np.int64) + k_lo)
    bins = np.concatenate(pieces) if pieces else np.zeros(0, dtype=np.int64)
    offsets = np.zeros(w.n_fft + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    freq = bins.astype(np.float64) / w.t_fft
    return Inputs(w=w, t=np.ascontiguousarray(t), offsets=offsets,
                  freq=np.ascontiguousarray(freq), v=np.ascontiguousarray(v),
                  sky=np.ascontiguousarray(sky))


def small(w: Workload, **changes) -> Workload:
    """A copy of ``w`` with some fields changed (for reduced test cases)."""
    return replace(w, **changes)


# --------------------------------------------------------------------------
# Small randomised cases (off-grid frequencies, random motion and sky)
# --------------------------------------------------------------------------
_S_CASE = 7


def random_case(seed: int, n_fft: int = 20, n_bins: int = 40, k_over: int = 10,
                n_fdot: int = 7, n_dir: int = 3, p: float = 0.3, t_fft: float = 1024.0,
                k0: int = 51200, margin: int = 4, off_grid: bool = True,
                doppler: bool = True, pad_bins: int = 0, subband_bins: int = 8,
                top_k: int = 2, excl_cells: int = 20, sep_cells: int = 40,
                n_thr: int = 0, vmax: float = 1e-4) -> tuple:
    """A small seeded case: (Inputs, plan parameter dict).

    Frequencies are (k + jitter) / T_FFT with |jitter| < 0.3 when ``off_grid``
    (so that no stripe edge falls exactly on a cell boundary), FFTs are
    half-interlaced, the velocity components are uniform in [-vmax, vmax]/sqrt(3)
    and the sky directions are uniform on the sphere.  ``pad_bins`` widens the
    map on both sides beyond the supplied peaks.
    """
    ctr = 0

    def u(n):
        nonlocal ctr
        x = uniform(seed, _S_CASE, np.arange(ctr, ctr + n))
        ctr += n
        return x

    t_step = 0.5 * t_fft
    t = np.arange(n_fft, dtype=np.float64) * t_step
    t_obs = n_fft * t_step
    nb = n_bins + 2 * margin
    mask = u(n_fft * nb).reshape(n_fft, nb) < p
    jit = (u(n_fft * nb).reshape(n_fft, nb) - 0.5) * 0.6 if off_grid else np.zeros((n_fft, nb))
    kk = np.arange(k0 - margin, k0 + n_bins + margin, dtype=np.float64)[None, :] + jit
    freq = (kk / t_fft)[mask]
    counts = mask.sum(axis=1)
    offsets = np.zeros(n_fft + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    if doppler:
        v = (u(3 * n_fft).reshape(n_fft, 3) * 2.0 - 1.0) * (vmax / math.sqrt(3.0))
    else:
        v = np.zeros((n_fft, 3))
    zz = u(n_dir) * 2.0 - 1.0
    ph = u(n_dir) * 2.0 * math.pi
    rr = np.sqrt(1.0 - zz * zz)
    sky = np.stack([rr * np.cos(ph), rr * np.sin(ph), zz], axis=1)
    fdot_step = (1.0 / t_fft) / t_obs
    params = dict(t_fft=t_fft, k_over=k_over, f0_min=(k0 - pad_bins) / t_fft,
                  n_f0=(n_bins + 2 * pad_bins) * k_over,
                  fdot_min=-(n_fdot // 2) * fdot_step, fdot_step=fdot_step, n_fdot=n_fdot,
                  t_ref=0.5 * (n_fft - 1) * t_step, subband_cells=subband_bins * k_over,
                  top_k=top_k, excl_cells=excl_cells, sep_cells=sep_cells, n_thr=n_thr, p0=p)
    w = Workload(name="random_case_%d" % seed, t_fft=t_fft, n_fft=n_fft, t_step=t_step,
                 t_obs=t_obs, f_lo=k0 / t_fft, f_hi=(k0 + n_bins) / t_fft, k_over=k_over,
                 p_peak=p, doppler=doppler, n_dir=n_dir, seed=seed)
    inp = Inputs(w=w, t=t, offsets=offsets, freq=np.ascontiguousarray(freq),
                 v=np.ascontiguousarray(v), sky=np.ascontiguousarray(sky))
    return inp, params


def dense_case(seed: int, dense_ffts=(1,), n_dense: int = 12, spacing_bins: float = 0.2,
               **kw) -> tuple:
    """``random_case`` with the peaks of the FFTs ``dense_ffts`` replaced by
    ``n_dense`` off-grid peaks ``spacing_bins`` apart (ascending, inside the
    band): an accepted but non-bin-grid peakmap on which several stripes of
    one FFT cover the same cell (the adaptive map's count bound must hold)."""
    inp, params = random_case(seed, **kw)
    t_fft = params["t_fft"]
    k0 = int(round(inp.w.f_lo * t_fft))
    parts, counts = [], []
    for i in range(inp.t.shape[0]):
        if i in dense_ffts:
            start = k0 + 2.0 + 0.37 * (i % 3)
            f = (start + spacing_bins * np.arange(n_dense)) / t_fft
        else:
            f = inp.freq[int(inp.offsets[i]):int(inp.offsets[i + 1])]
        parts.append(f)
        counts.append(f.shape[0])
    offsets = np.zeros(inp.t.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    out = Inputs(w=inp.w, t=inp.t, offsets=offsets,
                 freq=np.ascontiguousarray(np.concatenate(parts)), v=inp.v, sky=inp.sky)
    return out, params


# --------------------------------------------------------------------------
# Spectra for peakmap construction (periodogram and AR average spectrum)
# --------------------------------------------------------------------------
_S_SPEC_E, _S_SPEC_G = 8, 9


@dataclass
class Spectra:
    """Per-FFT spectra of one band: s_p (periodogram) and s_ar (average
    spectrum estimate), both (n_fft, n_bins) binary32; t (n_fft) FFT start
    times; bin b of the band is frequency (k0 + b) / t_fft."""
    s_p: np.ndarray
    s_ar: np.ndarray
    t: np.ndarray
    k0: int
    t_fft: float
    wander_bins: np.ndarray   # per FFT, the wandering line's bin (-1: none)
    const_bins: np.ndarray    # bins of the constant lines
    signal_bins: np.ndarray   # per FFT, the signal track's bin (-1: none)


def spectra_case(seed: int, n_fft: int, n_bins: int, t_fft: float = 8192.0,
                 f_lo: float = 50.0, interlaced: bool = True, signal_lambda: float = 0.0,
                 signal_f0: float = None, signal_fdot: float = 0.0, wander_amp: float = 0.0,
                 wander_f: tuple = None, wander_width: int = 1, const_lines: tuple = (),
                 const_amp: float = 40.0,
                 const_frac: float = 0.8) -> Spectra:
    """Seeded spectra with the statistics the peakmap section describes:
    s_ar a smooth positive curve over the band and s_p = s_ar x, where x is the
    equalised periodogram, exponential with mean 1 for noise and normalised
    non-central chi^2 with 2 degrees of freedom and non-centrality lambda
    (mean 1 + lambda / 2) in the bins of a signal track f0 + fdot (t - t_mid).

    Disturbances: a wandering line (``wander_width`` bins per FFT drifting
    between the two frequencies of ``wander_f``, x = wander_amp in every other
    one of them, so that each is a local maximum) and constant lines at
    the frequencies ``const_lines`` (x = const_amp in a fraction const_frac of
    the FFTs).  Draws: SplitMix64 counter streams; exponentials as -log(1 - u),
    Gaussians by Box-Muller."""
    k0 = int(round(f_lo * t_fft))
    step = 0.5 * t_fft if interlaced else t_fft
    t = np.arange(n_fft, dtype=np.float64) * step
    m = n_fft * n_bins
    u = uniform(seed, _S_SPEC_E, np.arange(m)).reshape(n_fft, n_bins)
    x = -np.log1p(-u)
    j = np.arange(n_bins, dtype=np.float64)
    s_ar = (1.0 + 0.3 * np.sin(2.0 * np.pi * j / max(n_bins, 1)) + 0.1 * j / max(n_bins, 1))
    s_ar = np.broadcast_to(s_ar, (n_fft, n_bins)) * (1.0 + 0.05 * np.cos(
        2.0 * np.pi * t / max(t[-1], 1.0)))[:, None]
    sig = np.full(n_fft, -1, dtype=np.int64)
    if signal_lambda > 0.0:
        f0 = f_lo + 0.5 * n_bins / t_fft if signal_f0 is None else signal_f0
        tm = 0.5 * (t[0] + t[-1])
        sig = np.rint((f0 + signal_fdot * (t - tm)) * t_fft).astype(np.int64) - k0
        ok = (sig >= 0) & (sig < n_bins)
        g = uniform(seed, _S_SPEC_G, np.arange(4 * n_fft)).reshape(4, n_fft)
        r = np.sqrt(-2.0 * np.log1p(-g[0]))
        g1 = r * np.cos(2.0 * np.pi * g[1])
        g2 = r * np.sin(2.0 * np.pi * g[1])
        xs = ((np.sqrt(signal_lambda) + g1) ** 2 + g2 ** 2) / 2.0
        rows = np.nonzero(ok)[0]
        x[rows, sig[rows]] = xs[rows]
        sig[~ok] = -1
    wand = np.full(n_fft, -1, dtype=np.int64)
    if wander_amp > 0.0 and wander_f is not None:
        fa, fb = wander_f
        ph = np.arange(n_fft) / max(n_fft - 1, 1)
        fw = fa + (fb - fa) * (0.5 - 0.5 * np.cos(np.pi * ph))
        wand = np.rint(fw * t_fft).astype(np.int64) - k0
        for q in range(0, int(wander_width), 2):
            wb = wand + q
            rows = np.nonzero((wb >= 0) & (wb < n_bins))[0]
            x[rows, wb[rows]] = wander_amp
        wand[(wand < 0) | (wand >= n_bins)] = -1
    cb = np.array([int(round(f * t_fft)) - k0 for f in const_lines], dtype=np.int64)
    if cb.size:
        on = uniform(seed, _S_SPEC_G + 1, np.arange(n_fft * cb.size)).reshape(n_fft, cb.size)
        for q, b in enumerate(cb):
            if 0 <= b < n_bins:
                rows = np.nonzero(on[:, q] < const_frac)[0]
                x[rows, b] = const_amp
    s_ar32 = s_ar.astype(np.float32)
    s_p32 = (s_ar * x).astype(np.float32)
    return Spectra(s_p=np.ascontiguousarray(s_p32), s_ar=np.ascontiguousarray(s_ar32), t=t,
                   k0=k0, t_fft=float(t_fft), wander_bins=wand, const_bins=cb,
                   signal_bins=sig)


# The peakmap workload: 150 days of FFTs of 8192 s overlapping by half (3164),
# a 1 Hz band at 50 Hz (8192 bins), threshold theta = 2.5 (p0 = 0.0755), a
# gross grid of 12 h x 0.01 Hz with the veto at E_H + 4.5 sigma_H (65 + 35),
# persistency veto at m1 + 5 m2.
PEAKMAP_PARAMS = dict(n_fft=3164, n_bins=8192, t_fft=8192.0, f_lo=50.0, theta=2.5,
                      dt_h=43200.0, n_th=300, df_h=0.01, f0_h=50.0, n_fh=100, gross_thr=100,
                      k_sigma=5.0)


def peakmap_workload(seed: int = 41) -> Spectra:
    """Spectra of the peakmap workload: noise, a signal track (lambda = 3,
    50.3 Hz, -1e-9 Hz/s), a wandering line 15 bins wide drifting from 50.55 to
    50.75 Hz, constant lines at 50.123 and 50.877 Hz in 80 % of the FFTs."""
    p = PEAKMAP_PARAMS
    return spectra_case(seed, p["n_fft"], p["n_bins"], t_fft=p["t_fft"], f_lo=p["f_lo"],
                        signal_lambda=3.0, signal_f0=50.3, signal_fdot=-1e-9,
                        wander_amp=40.0, wander_f=(50.55, 50.75), wander_width=15,
                        const_lines=(50.123, 50.877), const_amp=40.0, const_frac=0.8)


# --------------------------------------------------------------------------
# Candidate sets (clustering and coincidences)
# --------------------------------------------------------------------------
_S_CAND = 12
CAND_FIELDS = ("lam", "beta", "f", "fdot", "dlam", "dbeta", "df", "dfdot")


def candidates_on_grid(seed: int, stream: int, n: int, m) -> np.ndarray:
    """n candidates drawn uniformly on a grid of m = (m_lam, m_beta, m_f,
    m_fdot) cells, as (n, 8) float64 rows in CAND_FIELDS order: every width is
    one cell; longitude cells cover the circle (value = cell 2 pi / m_lam), the
    other values are the cell indices."""
    u = uniform(seed, 100 + stream, np.arange(4 * n)).reshape(4, n)
    cells = [np.floor(u[q] * m[q]) for q in range(4)]
    out = np.empty((n, 8))
    out[:, 0] = cells[0] * (2.0 * math.pi / m[0])
    out[:, 1], out[:, 2], out[:, 3] = cells[1], cells[2], cells[3]
    out[:, 4] = 2.0 * math.pi / m[0]
    out[:, 5:8] = 1.0
    return out


def candidate_set(seed: int, stream: int, n: int, f_lo: float = 100.0, band: float = 1.0,
                  t_fft: float = 1024.0, n_d: float = None, fdot_step: float = None,
                  fdot_rows: int = 100, clusters: int = 0, cluster_size: int = 8,
                  signals: np.ndarray = None, jitter: float = 0.5) -> np.ndarray:
    """A set of n candidates in the shape of the search's output, (n, 8) rows
    in CAND_FIELDS order: sky directions uniform on the sphere with the coarse
    widths of the App. A2 grid at Doppler number n_d (beta: 1 / (N_D |sin beta|),
    at most pi / 8; lambda: 2 pi / ceil(2 pi N_D cos beta)); f uniform in the
    band, width 1 / T_FFT; fdot on fdot_rows rows of fdot_step below zero.
    ``clusters`` groups of ``cluster_size`` candidates within about a bin of a
    seed candidate, and ``signals`` (rows of lam, beta, f, fdot) repeated with
    up to ``jitter`` bins of noise, replace the first rows."""
    if n_d is None:
        n_d = doppler_number(f_lo + band, t_fft)
    if fdot_step is None:
        fdot_step = 1.0 / (t_fft * 3.15e7)
    u = uniform(seed, _S_CAND + stream, np.arange(6 * n)).reshape(6, n)
    lam = u[0] * 2.0 * math.pi
    beta = np.arcsin(u[1] * 2.0 - 1.0)
    f = f_lo + u[2] * band
    fdot = -np.floor(u[3] * fdot_rows) * fdot_step

    def widths(b):
        db = np.minimum(1.0 / (n_d * np.maximum(np.abs(np.sin(b)), 1e-3)), math.pi / 8)
        dl = 2.0 * math.pi / np.maximum(1.0, np.ceil(2.0 * math.pi * n_d * np.cos(b) - 1e-12))
        return dl, db

    rows = []
    k = 0
    sig = np.zeros((0, 4)) if signals is None else np.asarray(signals, np.float64).reshape(-1, 4)
    for s in sig:
        rows.append(s)
    for c in range(clusters):
        rows.append(np.array([lam[c], beta[c], f[c], fdot[c]]))
        for q in range(cluster_size - 1):
            rows.append(None)   # filled below, near the seed
    out = np.empty((n, 8))
    out[:, 0], out[:, 1], out[:, 2], out[:, 3] = lam, beta, f, fdot
    j = uniform(seed, _S_CAND + 50 + stream, np.arange(4 * n)).reshape(4, n) * 2.0 - 1.0
    seed_row = None
    for r, v in enumerate(rows[:n]):
        if v is not None:
            out[r, :4] = v
            seed_row = out[r, :4].copy()
            if r < len(sig):
                seed_row = None
        elif seed_row is not None:
            dl, db = widths(seed_row[1])
            out[r, 0] = np.mod(seed_row[0] + j[0, r] * dl, 2.0 * math.pi)
            out[r, 1] = np.clip(seed_row[1] + j[1, r] * db, -math.pi / 2, math.pi / 2)
            out[r, 2] = seed_row[2] + j[2, r] / t_fft
            out[r, 3] = seed_row[3] + np.round(j[3, r]) * fdot_step
    dl, db = widths(out[:, 1])
    for r in range(min(len(sig), n)):
        out[r, 0] = np.mod(out[r, 0] + jitter * j[0, r] * dl[r], 2.0 * math.pi)
        out[r, 1] = np.clip(out[r, 1] + jitter * j[1, r] * db[r], -math.pi / 2, math.pi / 2)
        out[r, 2] += jitter * j[2, r] / t_fft
        out[r, 3] += np.round(jitter * j[3, r]) * fdot_step
    dl, db = widths(out[:, 1])
    out[:, 4], out[:, 5] = dl, db
    out[:, 6] = 1.0 / t_fft
    out[:, 7] = fdot_step
    return out
