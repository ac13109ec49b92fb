"""Pins of the oracle's candidate clustering and coincidences (Sec. "Candidate
clustering and coincidences", Eq. norm; App. "Theory of coincidences") against
facts that do not come from the oracle code.  CPU only."""
import math

import numpy as np
import pytest

from paper_1407_8333_gb300 import synth


@pytest.fixture(scope="module")
def co():
    import oracle
    return oracle.coincidence


def cand(lam=0.0, beta=0.0, f=0.0, fdot=0.0, dlam=1.0, dbeta=1.0, df=1.0, dfdot=1.0):
    return [lam, beta, f, fdot, dlam, dbeta, df, dfdot]


def test_distance_hand_cases(co):
    C = co.as_cands
    # Pythagorean triples in bins: (3, 4) -> 5, (1, 2, 2, 4) -> 5
    assert co.distance(C(cand()), C(cand(f=3.0, fdot=4.0)))[0] == 5.0
    assert co.distance(C(cand()), C(cand(lam=1.0, beta=2.0, f=2.0, fdot=4.0)))[0] == 5.0
    # the mean of the two widths: widths 1 and 3, difference 4 -> 2 bins
    assert co.distance(C(cand(df=1.0)), C(cand(f=4.0, df=3.0)))[0] == 2.0
    # longitudes the short way round: 0.01 and 2 pi - 0.01 are 0.02 apart
    d = co.distance(C(cand(lam=0.01, dlam=0.02)), C(cand(lam=2 * math.pi - 0.01, dlam=0.02)))[0]
    assert d == pytest.approx(1.0, rel=1e-12)
    # and the plain difference below pi is not wrapped
    d = co.distance(C(cand(lam=1.0, dlam=0.5)), C(cand(lam=3.0, dlam=0.5)))[0]
    assert d == 4.0


def test_single_linkage_chain_and_boundary(co):
    """A - B and B - C within d_max, A - C not: one cluster (Sec. "Candidate
    clustering and coincidences": each member within d_max of at least one
    other); d == d_max links."""
    c = co.as_cands([cand(f=0.0), cand(f=3.0), cand(f=6.0), cand(f=10.0), cand(f=20.0)])
    lab, n = co.cluster(c, 4.0)
    assert list(lab) == [0, 0, 0, 0, 4] and n == 2
    lab, n = co.cluster(c, 3.999)
    assert list(lab) == [0, 0, 0, 3, 4] and n == 3
    lab, n = co.cluster(c, 2.0)
    assert list(lab) == [0, 1, 2, 3, 4] and n == 5


def test_clusters_are_the_connected_components(co):
    """Against scipy's connected components of the d <= d_max graph, labels
    renamed to the smallest member."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    c = co.as_cands(synth.candidate_set(3, 0, 700, clusters=12, cluster_size=6))
    d = np.array([co.distance(c[i], c) for i in range(len(c))])
    for d_max in (2.0, 4.0):
        n, comp = connected_components(csr_matrix(d <= d_max), directed=False)
        want = np.array([np.nonzero(comp == comp[i])[0].min() for i in range(len(c))])
        lab, nc = co.cluster(c, d_max)
        assert nc == n and np.array_equal(lab, want)


def brute_coincidences(a, b, ta, tb, tc, win):
    out = []
    for i in range(len(a)):
        for j in range(len(b)):
            ok = True
            fa = a[i][2] + a[i][3] * (tc - ta)
            fb = b[j][2] + b[j][3] * (tc - tb)
            for q, (x, y, wx, wy) in enumerate(((a[i][0], b[j][0], a[i][4], b[j][4]),
                                                (a[i][1], b[j][1], a[i][5], b[j][5]),
                                                (fa, fb, a[i][6], b[j][6]),
                                                (a[i][3], b[j][3], a[i][7], b[j][7]))):
                dx = abs(y - x)
                if q == 0 and dx > math.pi:
                    dx = 2 * math.pi - dx
                if dx / ((wx + wy) * 0.5) > win[q]:
                    ok = False
            if ok:
                out.append((i, j))
    return out


def test_coincidences_by_brute_force(co):
    seeds = synth.candidate_set(4, 0, 64, clusters=8, cluster_size=8)[::8, :4]
    a = synth.candidate_set(4, 1, 150, signals=seeds)
    b = synth.candidate_set(4, 2, 170, signals=seeds)
    for win in ((1, 1, 1, 1), (2, 2, 3, 2)):
        p, n1, n2 = co.coincidences(a, b, 1e6, 2e6, 1.5e6, win)
        want = brute_coincidences(a.tolist(), b.tolist(), 1e6, 2e6, 1.5e6, win)
        assert [tuple(x) for x in p] == want
        assert n1.sum() == n2.sum() == len(want)
    # the injected signals are found
    p, _, _ = co.coincidences(a, b, 0.0, 0.0, 0.0, (2, 2, 2, 2))
    assert {(i, i) for i in range(8)} <= {tuple(x) for x in p}


def test_reference_time_shift(co):
    """Frequencies are compared at the common time: f + fdot (t_c - t_ref)."""
    a = co.as_cands([cand(f=100.0, fdot=-1.0, df=0.5)])
    b = co.as_cands([cand(f=90.0, fdot=-1.0, df=0.5)])     # the same source 10 s later
    p, _, _ = co.coincidences(a, b, 0.0, 10.0, 0.0, (1, 1, 1, 1))
    assert p.tolist() == [[0, 0]]
    p, _, _ = co.coincidences(a, b, 0.0, 0.0, 0.0, (1, 1, 1, 1))
    assert p.tolist() == []


@pytest.mark.parametrize("m, win_cells, n", [((20, 20, 20, 20), (0, 0, 0, 0), 4000),
                                             ((100, 100, 200, 100), (2, 1, 3, 2), 6000)])
def test_expected_number_of_coincidences(co, th, m, win_cells, n):
    """App. "Theory of coincidences": uniform candidates on m_j cells and total
    windows w_j = 2 n_j + 1: N_coinc,1 = N1 (1 - exp(-N2 prod w_j / m_j)), about
    100 expected here, within 4 binomial sigma (cells at the edges of the
    linear parameters see part of the window: a factor 1 - n_j (n_j + 1) /
    (m_j w_j) each; longitude is a circle)."""
    a = synth.candidates_on_grid(5, 1, n, m)
    b = synth.candidates_on_grid(5, 2, n, m)
    _, c1, c2 = co.coincidences(a, b, 0.0, 0.0, 0.0, win_cells)
    w = [2 * q + 1 for q in win_cells]
    want = th.n_coinc(n, n, w, m)
    edge = 1.0
    for q, wj, mj in zip(win_cells[1:], w[1:], m[1:]):
        edge *= 1.0 - q * (q + 1) / (mj * wj)
    assert 80 < want < 130
    for got in (np.count_nonzero(c1), np.count_nonzero(c2)):
        assert abs(got - want * edge) < 4.0 * math.sqrt(want)


def test_cluster_coincidences_keep_the_nearest_pair(co):
    """Clusters {0, 1} and {2} of set 1, {0} and {1, 2} of set 2; pairs
    (0, 0), (1, 0), (1, 1), (2, 2): cluster pairs (0, 0) keeps the nearer of
    (0, 0) and (1, 0), (0, 1) keeps (1, 1), (2, 1) keeps (2, 2)."""
    a = co.as_cands([cand(f=0.0), cand(f=3.0), cand(f=20.0)])
    b = co.as_cands([cand(f=2.0), cand(f=3.5), cand(f=20.0)])
    rows, d = co.cluster_coincidences(a, b, 0.0, 0.0, 0.0, [0, 0, 2], [0, 1, 1],
                                      [(0, 0), (1, 0), (1, 1), (2, 2)])
    assert rows.tolist() == [[0, 0, 1, 0], [0, 1, 1, 1], [2, 1, 2, 2]]
    assert d.tolist() == [1.0, 0.5, 0.0]
    # ties go to the smallest (i, j)
    b2 = co.as_cands([cand(f=1.0), cand(f=4.0), cand(f=20.0)])
    rows, _ = co.cluster_coincidences(a, b2, 0.0, 0.0, 0.0, [0, 0, 2], [0, 0, 1],
                                      [(0, 0), (1, 1)])
    assert rows.tolist() == [[0, 0, 0, 0]]


def test_cluster_coincidences_by_brute_force(co):
    seeds = synth.candidate_set(6, 0, 64, clusters=8, cluster_size=8)[::8, :4]
    a = synth.candidate_set(6, 1, 300, signals=seeds, clusters=20, cluster_size=5)
    b = synth.candidate_set(6, 2, 280, signals=seeds, clusters=20, cluster_size=5)
    la, _ = co.cluster(a, 4.0)
    lb, _ = co.cluster(b, 4.0)
    p, _, _ = co.coincidences(a, b, 1e6, 2e6, 1.5e6, (3, 3, 3, 3))
    rows, d = co.cluster_coincidences(a, b, 1e6, 2e6, 1.5e6, la, lb, p)
    al, bl = a.tolist(), b.tolist()
    best = {}
    for i, j in p.tolist():
        fa = al[i][2] + al[i][3] * (1.5e6 - 1e6)
        fb = bl[j][2] + bl[j][3] * (1.5e6 - 2e6)
        ks = []
        for q, (x, y, wx, wy) in enumerate(((al[i][0], bl[j][0], al[i][4], bl[j][4]),
                                            (al[i][1], bl[j][1], al[i][5], bl[j][5]),
                                            (fa, fb, al[i][6], bl[j][6]),
                                            (al[i][3], bl[j][3], al[i][7], bl[j][7]))):
            dx = abs(y - x)
            if q == 0 and dx > math.pi:
                dx = 2 * math.pi - dx
            ks.append(dx / ((wx + wy) * 0.5))
        dist = math.sqrt(((ks[0] ** 2 + ks[1] ** 2) + ks[2] ** 2) + ks[3] ** 2)
        key = (int(la[i]), int(lb[j]))
        if key not in best or (dist, i, j) < best[key]:
            best[key] = (dist, i, j)
    want = sorted((i, j, k) for k, (dd, i, j) in best.items())
    assert [tuple(r) for r in rows.tolist()] == [(k[0], k[1], i, j) for i, j, k in want]
    assert len(rows) < len(p)      # clusters merge pairs


@pytest.fixture(scope="module")
def th():
    from oracle import theory
    return theory
