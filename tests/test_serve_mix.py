"""The served stream's job mix (`paper_1407_8333_gb300/serve.py`), host side
only: 16 job shapes (T_FFT in {8192, 4096, 2048, 1024} s x band width in
{0.25, 0.5, 1, 2} Hz), band starts inside the frequency range of each T_FFT,
peak probability in [0.03, 0.05], half-interlaced FFTs over 150 days (scaled),
and sky patches of 1 .. max_dir grid directions, log-uniform.  CPU only."""
import math

import numpy as np
import pytest

from paper_1407_8333_gb300 import serve


@pytest.fixture(scope="module")
def pool():
    return serve.make_job_pool(7, scale_fft=0.005)


def test_job_pool_shapes(pool):
    assert set(pool) == {(t, b) for t in (8192.0, 4096.0, 2048.0, 1024.0)
                         for b in (0.25, 0.5, 1.0, 2.0)}
    for (t, b), inp in pool.items():
        w = inp.w
        lo, hi = serve._T_RANGES[t]
        assert lo <= w.f_lo and w.f_hi <= hi + 1e-9
        assert w.f_hi - w.f_lo == b and w.t_fft == t and w.t_step == t / 2
        assert 0.03 <= w.p_peak <= 0.05
        assert w.n_fft == max(8, int(math.floor(150 * 86400.0 / (0.5 * t)) * 0.005))
        assert inp.sky.shape == (1, 3)


def test_job_list_directions(pool):
    jobs = serve.job_list(8, 160, pool, max_dir=128)
    n = np.array([j[1] for j in jobs])
    assert n.min() >= 1 and n.max() <= 128
    # log-uniform on [1, 128]: the median near sqrt(128) ~ 11, both ends reached
    assert 6 <= np.median(n) <= 20 and (n <= 2).any() and (n >= 100).any()
    for shape, nd, sky in jobs[:50]:
        assert shape in pool and sky.shape == (nd, 3)
        assert np.allclose(np.linalg.norm(sky, axis=1), 1.0, atol=1e-12, rtol=0)
    # the same seed gives the same list
    again = serve.job_list(8, 160, pool, max_dir=128)
    assert all(a[0] == b[0] and a[1] == b[1] and np.array_equal(a[2], b[2])
               for a, b in zip(jobs, again))
