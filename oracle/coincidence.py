"""CPU oracle of candidate clustering and coincidences -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may use this module; the CUDA library never imports it and it never
imports the library.  Plain numpy and Python, in the order the paper states
the steps (Sec. "Candidate clustering and coincidences"; App. "Theory of
coincidences"):

* a candidate is (lambda, beta, f, fdot) with the widths of its coarse bins
  (d_lambda, d_beta, d_f, d_fdot); the difference of two candidates in one
  parameter, in bins, is k = |x2 - x1| / ((dx1 + dx2) / 2) (the mean width of
  the two), with longitudes compared the short way around the circle;
* distance (Eq. norm): d = sqrt(k_lambda^2 + k_beta^2 + k_f^2 + k_fdot^2);
* a cluster: the candidates linked by chains of distances d <= d_max (every
  member is within d_max of at least one other member), labelled by its
  smallest candidate index;
* coincidences between two sets: each candidate's frequency is referred to a
  common time, f' = f + fdot (t_c - t_ref); two candidates coincide when, in
  every parameter, k <= the caller's window (in bins, the sum of the two sets'
  half-windows n_1 + n_2 of the appendix);
* coincidences among clusters: two clusters coincide when at least one pair of
  their members does, and each coincident pair of clusters keeps only its
  nearest coincident pair (smallest distance at the common time; ties to the
  smallest (i, j)).

Every number is binary64 in the order written (numpy evaluates the array
expressions operation by operation, no fused multiply-add).

Pins (``tests/test_oracle_coincidence_pins.py``): hand-computed distances
(Pythagorean triples, mean widths, the longitude wrap), single-linkage chains
and the d = d_max boundary, clusters equal to scipy's connected components of
the d <= d_max graph, a pure-Python brute force of the coincidences, the
reference-time shift, and the appendix's expected number of coincidences
N_1 (1 - exp(-N_2 prod w_j / m_j)) on uniformly drawn candidates.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi
FIELDS = ("lam", "beta", "f", "fdot", "dlam", "dbeta", "df", "dfdot")
CAND_DTYPE = np.dtype([(k, np.float64) for k in FIELDS])


def as_cands(x) -> np.ndarray:
    """Structured array of candidates (a (n, 8) float array in FIELDS order is
    accepted)."""
    x = np.asarray(x)
    if x.dtype == CAND_DTYPE:
        return x
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 8)
    return x.view(CAND_DTYPE).reshape(-1)


def bins_apart(x1, x2, w1, w2, wrap: bool = False):
    """k = |x2 - x1| / ((w1 + w2) * 0.5); a longitude difference above pi is
    taken the other way round, 2 pi - |x2 - x1|."""
    a = np.abs(np.asarray(x2, np.float64) - np.asarray(x1, np.float64))
    if wrap:
        a = np.where(a > np.pi, TWO_PI - a, a)
    return a / ((np.asarray(w1, np.float64) + np.asarray(w2, np.float64)) * 0.5)


def param_bins(c1, c2):
    """(k_lambda, k_beta, k_f, k_fdot) between candidates c1 and c2 (broadcast)."""
    return (bins_apart(c1["lam"], c2["lam"], c1["dlam"], c2["dlam"], wrap=True),
            bins_apart(c1["beta"], c2["beta"], c1["dbeta"], c2["dbeta"]),
            bins_apart(c1["f"], c2["f"], c1["df"], c2["df"]),
            bins_apart(c1["fdot"], c2["fdot"], c1["dfdot"], c2["dfdot"]))


def distance(c1, c2):
    """Eq. norm: sqrt(((k_l^2 + k_b^2) + k_f^2) + k_fd^2)."""
    kl, kb, kf, kd = param_bins(c1, c2)
    return np.sqrt(((kl * kl + kb * kb) + kf * kf) + kd * kd)


def cluster(cands, d_max: float):
    """Cluster labels (the smallest index of each cluster) and the number of
    clusters: a breadth-first walk of the graph whose edges are the pairs with
    distance <= d_max."""
    c = as_cands(cands)
    n = c.shape[0]
    label = np.full(n, -1, dtype=np.int64)
    for s in range(n):
        if label[s] >= 0:
            continue
        label[s] = s
        queue = [s]
        while queue:
            i = queue.pop()
            near = np.nonzero(distance(c[i], c) <= d_max)[0]
            for j in near:
                if label[j] < 0:
                    label[j] = s
                    queue.append(int(j))
    return label, int(np.count_nonzero(label == np.arange(n)))


def shift_to(cands, t_ref: float, t_c: float) -> np.ndarray:
    """The candidates with f referred to time t_c: f + fdot (t_c - t_ref)."""
    c = as_cands(cands).copy()
    c["f"] = c["f"] + c["fdot"] * (np.float64(t_c) - np.float64(t_ref))
    return c


def coincidences(cands1, cands2, t_ref1: float, t_ref2: float, t_c: float, win):
    """Coincident pairs (i of set 1, j of set 2), sorted by (i, j), and the
    number of partners of every candidate of each set.  win: the four windows
    (lambda, beta, f, fdot) in bins."""
    a = shift_to(cands1, t_ref1, t_c)
    b = shift_to(cands2, t_ref2, t_c)
    w = [np.float64(x) for x in win]
    pairs = []
    n1 = np.zeros(a.shape[0], dtype=np.int64)
    n2 = np.zeros(b.shape[0], dtype=np.int64)
    for i in range(a.shape[0]):
        kl, kb, kf, kd = param_bins(a[i], b)
        hit = np.nonzero((kl <= w[0]) & (kb <= w[1]) & (kf <= w[2]) & (kd <= w[3]))[0]
        for j in hit:
            pairs.append((i, int(j)))
        n1[i] = hit.size
        n2[hit] += 1
    p = np.array(pairs, dtype=np.int64).reshape(-1, 2)
    return p, n1, n2


def cluster_coincidences(cands1, cands2, t_ref1: float, t_ref2: float, t_c: float, label1,
                         label2, pairs):
    """Each coincident pair of clusters (label1[i], label2[j]) with its nearest
    coincident pair (i, j) and their distance, in the order of those pairs.
    Returns (rows (k, 4) int64: cluster 1, cluster 2, i, j; distances (k,))."""
    a = shift_to(cands1, t_ref1, t_c)
    b = shift_to(cands2, t_ref2, t_c)
    best = {}
    for i, j in np.asarray(pairs, dtype=np.int64).reshape(-1, 2):
        d = float(distance(a[i], b[j]))
        key = (int(label1[i]), int(label2[j]))
        cand = (d, int(i), int(j))
        if key not in best or cand < best[key]:
            best[key] = cand
    reps = sorted((i, j, key, d) for key, (d, i, j) in best.items())
    rows = np.array([(key[0], key[1], i, j) for i, j, key, d in reps], dtype=np.int64)
    return rows.reshape(-1, 4), np.array([d for *_, d in reps], dtype=np.float64)
