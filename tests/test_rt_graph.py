"""The random graphs of the real-time table (CPU only).

The paper's real-time table (Sec. 3.1.1, Table "RT") sweeps the connection density of the
network: each cell connected to a given fraction of the others.  The benchmark draws such
graphs with a pair hash (bench.rt_graph): the pair {i, j} is a junction with probability
`density`, decided once for both orders.  These checks hold for any correct draw: the CSR
is well formed, symmetric, free of self loops, rows ascending, the realised density is
within a few standard deviations of the asked one, and the draw is a function of the seed.

The table's sizes come from a search over step times (bench.rt_search); on synthetic step
time curves it must land within 2 % of the threshold a brute-force scan finds.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def dense_of(n, row_ptr, col):
    A = np.zeros((n, n), bool)
    for i in range(n):
        A[i, col[row_ptr[i]:row_ptr[i + 1]]] = True
    return A


@pytest.mark.parametrize("n,density", [(1, 0.5), (2, 1.0), (97, 0.25), (300, 0.5), (257, 0.75), (64, 1.0)])
def test_rt_graph_is_a_symmetric_csr_of_the_asked_density(n, density):
    rp, col = bench.rt_graph(torch, n, density, seed=5, device="cpu")
    assert rp.dtype == np.int32 and col.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == len(col) and np.all(np.diff(rp) >= 0)
    for i in range(n):
        r = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(r) > 0), "row not strictly ascending"
        assert np.all((r >= 0) & (r < n))
    A = dense_of(n, rp, col)
    assert not A.diagonal().any(), "self loop"
    assert (A == A.T).all(), "not symmetric"
    pairs = n * (n - 1) // 2
    if pairs:
        got = A.sum() / 2
        sd = np.sqrt(pairs * density * (1 - density))
        assert abs(got - density * pairs) <= 5 * sd + 1e-9


def test_rt_graph_full_density_is_all_to_all():
    n = 50
    rp, col = bench.rt_graph(torch, n, 1.0, seed=9, device="cpu")
    A = dense_of(n, rp, col)
    assert (A == ~np.eye(n, dtype=bool)).all()


def test_rt_graph_depends_on_the_seed_only():
    a = bench.rt_graph(torch, 200, 0.3, seed=5, device="cpu")
    b = bench.rt_graph(torch, 200, 0.3, seed=5, device="cpu")
    c = bench.rt_graph(torch, 200, 0.3, seed=6, device="cpu")
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[1], c[1])


# ---- the size search behind the real-time table --------------------------------------

def _threshold(t_of_n, limit=50.0, q=64, hi=1 << 24):
    """Largest multiple of q with t(N) <= limit, by brute force over multiples of q."""
    best = None
    n = q
    while n <= hi and t_of_n(n) <= limit:
        best = n
        n += q
    return best


@pytest.mark.parametrize("p,n_star,n0", [(2, 18700, 16384), (2, 10400, 9216), (1, 1_200_000, 1 << 20),
                                         (1, 2_290_000, 1 << 21), (2, 3000, 20000)])
def test_rt_search_lands_within_two_percent_of_the_threshold(p, n_star, n0):
    a = 47.0 / n_star ** p
    t = lambda n: 3.0 + a * n ** p
    best, tried = bench.rt_search(t, n0, p)
    assert best is not None and t(best) <= 50.0
    truth = _threshold(t, q=64, hi=4 * n_star)
    assert truth * 0.98 <= best <= truth
    assert all(n % 64 == 0 for n in tried) and len(tried) <= 11


def test_rt_search_with_an_overhead_the_model_does_not_know():
    """A fixed cost other than the model's 3 us and a little measurement noise: the bracket
    still closes on the threshold."""
    rng = np.random.default_rng(0)
    t = lambda n: 9.0 + 41.0 * (n / 12000.0) ** 2 * (1.0 + 0.002 * rng.standard_normal())
    best, tried = bench.rt_search(t, 6000, 2)
    assert best is not None and tried[best] <= 50.0
    assert 0.97 * 12000 <= best <= 12000 * 1.01
    bigger = [n for n, v in tried.items() if n > best]
    assert bigger and all(tried[n] > 50.0 for n in bigger)


def test_rt_search_when_no_size_meets_the_limit():
    best, tried = bench.rt_search(lambda n: 60.0 + n * 1e-6, 4096, 1)
    assert best is None and min(tried) == 64


def test_rt_search_when_every_size_meets_the_limit():
    best, tried = bench.rt_search(lambda n: 10.0, 4096, 1)
    assert best == max(tried) and best > 4096
