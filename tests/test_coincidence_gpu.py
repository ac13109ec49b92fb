"""Candidate clustering and coincidences on the GPU, through the C ABI, against
the oracle (Sec. "Candidate clustering and coincidences", Eq. norm; App.
"Theory of coincidences").  Labels, cluster counts, pairs and partner counts
bit for bit."""
import math

import numpy as np
import pytest

from paper_1407_8333_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_8333_gb300 import build, fh as fhmod
    build.build()
    fhmod.load()
    return fhmod


@pytest.fixture(scope="module")
def co():
    import oracle
    return oracle.coincidence


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def check_cluster(fh, co, c, d_max):
    lab, n = fh.fh_cluster(dev(c), d_max)
    want, wn = co.cluster(c, d_max)
    assert n == wn
    assert np.array_equal(lab.cpu().numpy(), want)
    return want


def check_coinc(fh, co, a, b, ta, tb, tc, win):
    p, m1, m2 = fh.fh_coincidences(dev(a), dev(b), ta, tb, tc, win)
    wp, w1, w2 = co.coincidences(a, b, ta, tb, tc, win)
    assert np.array_equal(p.cpu().numpy(), wp.reshape(-1, 2))
    assert np.array_equal(m1.cpu().numpy(), w1) and np.array_equal(m2.cpu().numpy(), w2)
    return wp


@pytest.mark.parametrize("n, clusters", [(1, 0), (2, 0), (37, 3), (1500, 30)])
def test_cluster_matches_oracle(fh, co, n, clusters):
    c = synth.candidate_set(41 + n, 0, n, clusters=clusters, cluster_size=7)
    for d_max in (0.0, 1.5, 4.0, 9.0):
        check_cluster(fh, co, c, d_max)


def test_cluster_degenerate_geometries(fh, co):
    c = synth.candidate_set(42, 0, 400, clusters=10)
    # every candidate at one frequency: a single bucket
    same = c.copy()
    same[:, 2] = 123.456
    check_cluster(fh, co, same, 3.0)
    # longitudes on both sides of 0 / 2 pi
    wrap = c.copy()
    wrap[:, 0] = np.where(np.arange(400) % 2 == 0, 0.0005 * np.arange(400) % 0.01,
                          2 * math.pi - 0.0005 * np.arange(400) % 0.01)
    check_cluster(fh, co, wrap, 4.0)
    # duplicates and an enormous d_max (one cluster)
    dup = np.concatenate([c[:50], c[:50]])
    check_cluster(fh, co, dup, 0.0)
    lab = check_cluster(fh, co, c, 1e300)
    assert np.all(lab == 0)


@pytest.mark.parametrize("win", [(0, 0, 0, 0), (1, 1, 1, 1), (2, 2, 3, 2)])
def test_coincidences_match_oracle(fh, co, win):
    seeds = synth.candidate_set(43, 0, 80, clusters=10, cluster_size=8)[::8, :4]
    a = synth.candidate_set(43, 1, 900, signals=seeds, clusters=5)
    b = synth.candidate_set(43, 2, 1100, signals=seeds, clusters=5)
    check_coinc(fh, co, a, b, 3.0e6, 4.5e6, 3.7e6, win)
    check_coinc(fh, co, a, b, 0.0, 0.0, 0.0, win)


def test_coincidences_on_a_grid_and_edge_cases(fh, co):
    m = (40, 30, 50, 20)
    a = synth.candidates_on_grid(44, 1, 3000, m)
    b = synth.candidates_on_grid(44, 2, 2500, m)
    for win in ((0, 0, 0, 0), (1, 0, 2, 1)):
        check_coinc(fh, co, a, b, 0.0, 0.0, 0.0, win)
    # empty sets
    p, m1, m2 = fh.fh_coincidences(dev(a[:0]), dev(b), 0.0, 0.0, 0.0, (1, 1, 1, 1))
    assert p.shape[0] == 0 and np.all(m2.cpu().numpy() == 0)
    p, m1, m2 = fh.fh_coincidences(dev(a), dev(b[:0]), 0.0, 0.0, 0.0, (1, 1, 1, 1))
    assert p.shape[0] == 0 and np.all(m1.cpu().numpy() == 0)
    # a window so wide that everything coincides
    check_coinc(fh, co, a[:60], b[:70], 0.0, 0.0, 0.0, (1e300, 1e300, 1e300, 1e300))


def test_capacity_and_invalid_candidates(fh):
    a = synth.candidates_on_grid(45, 1, 300, (5, 5, 5, 5))
    with pytest.raises(fh.FHError) as ei:
        fh.fh_coincidences(dev(a), dev(a), 0.0, 0.0, 0.0, (0, 0, 0, 0), capacity=10)
    assert ei.value.code == fh.FH_ERR_CAPACITY
    bad = a.copy()
    bad[7, 6] = 0.0            # a zero frequency width
    with pytest.raises(fh.FHError) as ei:
        fh.fh_cluster(dev(bad), 2.0)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG
    bad[7, 6] = 1.0
    bad[9, 2] = np.nan
    with pytest.raises(fh.FHError) as ei:
        fh.fh_coincidences(dev(bad), dev(a), 0.0, 0.0, 0.0, (1, 1, 1, 1))
    assert ei.value.code == fh.FH_ERR_INVALID_ARG
    with pytest.raises(fh.FHError) as ei:
        fh.fh_cluster(dev(a), -1.0)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG


def test_twenty_thousand_candidates(fh, co):
    """Sets the size of one band's output (10^4 - 10^5 candidates)."""
    seeds = synth.candidate_set(46, 0, 400, clusters=50, cluster_size=8)[::8, :4]
    # the same sources seen by the second set at its own reference time 1e6 s later
    later = seeds.copy()
    later[:, 2] += later[:, 3] * 1.0e6
    a = synth.candidate_set(46, 1, 20000, signals=seeds, clusters=200, cluster_size=6)
    b = synth.candidate_set(46, 2, 20000, signals=later, clusters=200, cluster_size=6)
    check_cluster(fh, co, a, 4.0)
    wp = check_coinc(fh, co, a, b, 1.0e6, 2.0e6, 1.5e6, (2, 2, 2, 2))
    assert {(i, i) for i in range(50)} <= {tuple(x) for x in wp}


def test_cluster_coincidences_match_oracle(fh, co):
    """Clusters of both sets, their coincident pairs, and the nearest pair of
    each coincident pair of clusters: rows and distances equal the oracle's."""
    import torch
    seeds = synth.candidate_set(47, 0, 160, clusters=20, cluster_size=8)[::8, :4]
    later = seeds.copy()
    later[:, 2] += later[:, 3] * 1.0e6
    a = synth.candidate_set(47, 1, 3000, signals=seeds, clusters=60, cluster_size=6)
    b = synth.candidate_set(47, 2, 2800, signals=later, clusters=60, cluster_size=6)
    da, db = dev(a), dev(b)
    la, _ = fh.fh_cluster(da, 4.0)
    lb, _ = fh.fh_cluster(db, 4.0)
    pairs, _, _ = fh.fh_coincidences(da, db, 1.0e6, 2.0e6, 1.5e6, (3, 3, 3, 3))
    rows, dist = fh.fh_cluster_coincidences(da, db, 1.0e6, 2.0e6, 1.5e6, la, lb, pairs)
    wla, _ = co.cluster(a, 4.0)
    wlb, _ = co.cluster(b, 4.0)
    wp, _, _ = co.coincidences(a, b, 1.0e6, 2.0e6, 1.5e6, (3, 3, 3, 3))
    wrows, wd = co.cluster_coincidences(a, b, 1.0e6, 2.0e6, 1.5e6, wla, wlb, wp)
    assert np.array_equal(rows.cpu().numpy(), wrows)
    assert np.array_equal(dist.cpu().numpy().view(np.uint64), wd.view(np.uint64))
    assert len(wrows) < len(wp)
    # pairs out of (i, j) order, or out of range, are refused
    bad = pairs.flip(0).contiguous()
    if bad.shape[0] > 1:
        with pytest.raises(fh.FHError) as ei:
            fh.fh_cluster_coincidences(da, db, 1.0e6, 2.0e6, 1.5e6, la, lb, bad)
        assert ei.value.code == fh.FH_ERR_INVALID_ARG
    out = torch.tensor([[0, 5000]], dtype=torch.int32, device="cuda")
    with pytest.raises(fh.FHError) as ei:
        fh.fh_cluster_coincidences(da, db, 1.0e6, 2.0e6, 1.5e6, la, lb, out)
    assert ei.value.code == fh.FH_ERR_INVALID_ARG
