"""The random graphs of the real-time table (CPU only).

The paper's real-time table (Sec. 3.1.1, Table "RT") sweeps the connection density of the
network: each cell connected to a given fraction of the others.  The benchmark draws such
graphs with a pair hash (bench.rt_graph): the pair {i, j} is a junction with probability
`density`, decided once for both orders.  These checks hold for any correct draw: the CSR
is well formed, symmetric, free of self loops, rows ascending, the realised density is
within a few standard deviations of the asked one, and the draw is a function of the seed.
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
