"""Closed forms of the paper used to pin the oracle -- TEST INFRASTRUCTURE ONLY.

Each function restates one equation of the paper in binary64:

* ``p0``           noise peak probability, threshold + local maximum (Eq. p0, Sec. V)
* ``binomial``     mean and standard deviation of a noise-only number count
                   (Eqs. phmsig, houghmean, Sec. VI)
* ``critical_ratio``   CR = (n - N p0) / sqrt(N p0 (1 - p0))   (Eq. cr, Sec. XII)
* ``n_thr_gauss``  count threshold for a false-alarm probability (Eq. nthr_gauss)
* ``cr_thr``       CR threshold for N_cand of N_tot points (Eq. crthr)
* ``n_tot``        number of coarse parameter-space points (Eq. Ntot, Sec. VIII)
* ``n_coinc``      expected number of candidates of set 1 with at least one
                   coincidence in set 2 (App. "Theory of coincidences")
* ``gross_points`` points N of one gross-histogram cell and its noise mean and
                   standard deviation E_H = N p0, sigma_H = sqrt(N p0 (1 - p0))
                   (Sec. "Removal of spectral wandering lines")
"""
from __future__ import annotations

import math

from scipy.special import erfcinv


def p0(theta: float) -> float:
    """Eq. p0: integral over x > theta of e^-x (1 - e^-x)^2."""
    return math.exp(-theta) - math.exp(-2.0 * theta) + math.exp(-3.0 * theta) / 3.0


def binomial(n: int, eta: float) -> tuple:
    """Eq. houghmean: (mu, sigma) = (N eta, sqrt(N eta (1 - eta)))."""
    mu = n * eta
    return mu, math.sqrt(mu * (1.0 - eta))


def critical_ratio(count: float, n: int, p: float) -> float:
    """Eq. cr."""
    return (count - n * p) / math.sqrt(n * p * (1.0 - p))


def n_thr_gauss(n: int, p: float, pfa: float) -> float:
    """Eq. nthr_gauss: N p0 + sqrt(2 N p0 (1 - p0)) erfc^-1(2 P_fa)."""
    return n * p + math.sqrt(2.0 * n * p * (1.0 - p)) * float(erfcinv(2.0 * pfa))


def cr_thr(n_cand: float, n_tot: float) -> float:
    """Eq. crthr: sqrt(2) erfc^-1(2 N_cand / N_tot)."""
    return math.sqrt(2.0) * float(erfcinv(2.0 * n_cand / n_tot))


def n_tot(k_f: float, k_sky: float, t_fft: float, dt: float, t_obs: float,
          tau_min: float) -> tuple:
    """Eq. Ntot with the product over orders j <= j_max whose N_sd^(j) >= 1 (Eq. Nsd).

    Returns (N_tot, j_max)."""
    base = t_fft / dt
    j_max = 0
    prod = 1.0
    j = 1
    while base * (t_obs / tau_min) ** j >= 1.0:
        j_max = j
        prod *= (t_obs / tau_min) ** j
        j += 1
    return 5.6 * math.pi * 1e-9 * k_f * k_sky * base ** (3 + j_max) * prod, j_max


def gross_points(dt_h: float, df_h: float, t_fft: float, interlaced: bool = True) -> float:
    """N = (Delta t_H / T_FFT)(Delta f_H / delta f) points per gross cell, delta f =
    1 / T_FFT; FFTs overlapping by half double it (N = 2 Delta t_H Delta f_H)."""
    n = (dt_h / t_fft) * (df_h * t_fft)
    return 2.0 * n if interlaced else n


def gross_noise(n_points: float, p: float) -> tuple:
    """(E_H, sigma_H) = (N p0, sqrt(N p0 (1 - p0))) of a noise-only gross cell."""
    return n_points * p, math.sqrt(n_points * p * (1.0 - p))


def n_coinc(n1: int, n2: int, w, m) -> float:
    """App. "Theory of coincidences": N_coinc,1 = N1 (1 - exp(-N2 prod_j w_j / m_j)),
    w_j the total coincidence window and m_j the cells of parameter j."""
    prod = 1.0
    for wj, mj in zip(w, m):
        prod *= wj / mj
    return n1 * (1.0 - math.exp(-n2 * prod))
