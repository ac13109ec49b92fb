"""The seeded synthetic inputs (`paper_1407_8333_gb300/synth.py`) against the
recipe they follow: the SplitMix64 mixer's published outputs, the workload
sizes, peakmaps on the FFT bin grid with the stated peak probability and line
presence, detector velocities of the stated magnitude, unit sky vectors and
the App. A2 sky grid's number of points (2 pi N_D^2 in the limit).  CPU only;
no method arithmetic is involved."""
import math

import numpy as np
import pytest

from paper_1407_8333_gb300 import synth


def test_splitmix64_reference_outputs():
    """The first outputs of SplitMix64 (Steele, Lea, Flood 2014) from state 0:
    mix(gamma), mix(2 gamma), mix(3 gamma)."""
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        z = np.array([g, g * np.uint64(2), g * np.uint64(3)], dtype=np.uint64)
    got = [int(x) for x in synth._mix(z)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("name, n_fft, n_f0, n_fdot, n_dir", [
    ("nodoppler_T1024_N200_100Hz", 200, 10240, 21, 1),
    ("single_sky_T8192_150d_50Hz", 3164, 81920, 1169, 1),
    ("sky_patch256_T1024_N200_100Hz", 200, 10240, 21, 256),
    ("highfreq_T1024_1yr_900Hz_64dir", 61594, 102400, 356, 64),
])
def test_workload_sizes(name, n_fft, n_f0, n_fdot, n_dir):
    w = synth.WORKLOADS[name]
    pp = w.plan_params()
    assert (w.n_fft, pp["n_f0"], pp["n_fdot"], w.n_dir) == (n_fft, n_f0, n_fdot, n_dir)
    # K T is an exact integer and the spin-down step is delta f / T_obs (Eq. sdstep)
    assert float(pp["k_over"]) * pp["t_fft"] == round(float(pp["k_over"]) * pp["t_fft"])
    assert pp["fdot_step"] == pytest.approx(1.0 / (w.t_fft * w.t_obs), rel=1e-15)


@pytest.mark.parametrize("name", ["nodoppler_T1024_N200_100Hz", "sky_patch256_T1024_N200_100Hz",
                                  "single_sky_T8192_150d_50Hz"])
def test_peakmap_recipe(name):
    w = synth.WORKLOADS[name]
    inp = synth.make_inputs(w)
    k_lo, k_hi = w.bins
    nb = k_hi - k_lo
    # FFT start times i * t_step
    assert np.array_equal(inp.t, np.arange(w.n_fft) * w.t_step)
    # frequencies exactly on the bin grid k / T_FFT, ascending within each FFT,
    # inside the band plus its margins
    k = inp.freq * w.t_fft
    assert np.array_equal(k, np.rint(k))
    k = k.astype(np.int64)
    assert k.min() >= k_lo and k.max() < k_hi
    for i in range(0, w.n_fft, max(1, w.n_fft // 50)):
        a, b = inp.offsets[i], inp.offsets[i + 1]
        assert np.all(np.diff(k[a:b]) > 0)
    # peak probability p: binomial count within 5 sigma (the line adds at most n_fft)
    cells = w.n_fft * nb
    mean = cells * w.p_peak
    sigma = math.sqrt(cells * w.p_peak * (1 - w.p_peak))
    assert abs(inp.n_peaks - mean) < 5 * sigma + w.n_fft
    # the line is a peak in about 90 % of the FFTs at its Doppler-shifted bin
    lk, lp = synth.line_bins(w, inp.v, inp.sky, inp.t)
    hit = np.zeros(w.n_fft, dtype=bool)
    for i in range(w.n_fft):
        a, b = inp.offsets[i], inp.offsets[i + 1]
        hit[i] = np.any(k[a:b] == lk[i])
    expect = w.line_presence + (1 - w.line_presence) * w.p_peak
    se = math.sqrt(expect * (1 - expect) / w.n_fft)
    assert abs(hit.mean() - expect) < 5 * se
    assert np.all(hit[lp])
    # velocity: orbit 30 km/s plus diurnal 0.46 km/s, in units of c
    speed = np.linalg.norm(inp.v, axis=1)
    if w.doppler:
        lo = (synth.V_ORB_KMS - synth.V_ROT_KMS) / synth.C_KMS
        hi = (synth.V_ORB_KMS + synth.V_ROT_KMS) / synth.C_KMS
        assert np.all(speed >= lo * (1 - 1e-12)) and np.all(speed <= hi * (1 + 1e-12))
    else:
        assert np.all(speed == 0.0)
    # unit sky vectors
    assert np.allclose(np.linalg.norm(inp.sky, axis=1), 1.0, atol=1e-12, rtol=0)


def test_inputs_are_reproducible():
    w = synth.WORKLOADS["sky_patch256_T1024_N200_100Hz"]
    a, b = synth.make_inputs(w), synth.make_inputs(w)
    for x, y in zip((a.t, a.offsets, a.freq, a.v, a.sky), (b.t, b.offsets, b.freq, b.v, b.sky)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("f0, t_fft", [(101.0, 1024.0), (51.0, 8192.0), (910.0, 1024.0)])
def test_sky_grid_size_and_symmetry(f0, t_fft):
    """App. A2: rings K / (N_D sin beta) apart with 2 pi N_D cos(beta) points
    each, i.e. 2 pi N_D^2 / K points for large N_D (Eq. Nsky's 4 pi N_D^2 is
    twice that: a reading of the paper), of unit length, the southern half
    mirroring the northern one."""
    n_d = synth.doppler_number(f0, t_fft)
    g = synth.ecliptic_grid(n_d)
    assert 1.0 < len(g) / (2 * math.pi * n_d * n_d) < 1.3
    assert np.allclose(np.linalg.norm(g, axis=1), 1.0, atol=1e-12, rtol=0)
    z = np.sort(g[:, 2])
    assert np.allclose(z, -z[::-1], atol=1e-12)


def test_sky_grid_tends_to_two_pi_nd_squared():
    """The ratio to 2 pi N_D^2 falls towards 1 as N_D grows (the discreteness
    of the rings near the poles and the equator fades)."""
    r = [len(synth.ecliptic_grid(n_d)) / (2 * math.pi * n_d * n_d) for n_d in (10, 40, 150)]
    assert r[0] > r[1] > r[2] and 1.0 < r[2] < 1.05
