"""The synthetic input recipes match the workloads they stand for (sizes, densities,
weights, pulse windows and seeds of the five configurations), and are deterministic."""
import numpy as np
import pytest

from paper_1612_01501_gb300 import inputs


def _pulse_steps(p):
    cells, beg, end, amp = p
    return np.asarray(cells), np.asarray(beg), np.asarray(end), np.asarray(amp)


def test_c1_recipe():
    """64 cells all-to-all, g_c = 0.04, jitter within +-5 mV from seed 0, 6 uA/cm^2 to cells
    0-7 from 100 to 110 ms, 1 s = 20 000 steps of 50 us."""
    c = inputs.config("c1")
    assert c["n"] == 64 and c["kind"] == "dense" and c["g"] == np.float32(0.04)
    assert c["n_steps"] == 20000
    assert np.abs(c["jitter"]).max() <= 5.0 and np.abs(c["jitter"]).max() > 4.0
    cells, beg, end, amp = _pulse_steps(c["pulses"])
    assert sorted(cells.tolist()) == list(range(8))
    assert set(beg.tolist()) == {2000} and set(end.tolist()) == {2200} and set(amp.tolist()) == {6.0}
    assert np.array_equal(inputs.config("c1")["jitter"], c["jitter"])       # seeded


def test_c2_recipe():
    """8192 cells all-to-all, g_c = 0.04 / N * 64 = 3.125e-4, no evoked input, 200 ms."""
    c = inputs.config("c2")
    assert c["n"] == 8192 and c["pulses"] is None and c["n_steps"] == 4000
    assert c["g"] == np.float32(0.04 / 8192 * 64) == np.float32(3.125e-4)
    assert np.abs(c["jitter"]).max() <= 5.0
    assert not np.array_equal(c["jitter"][:64], inputs.config("c1")["jitter"])   # seed 1, not seed 0


@pytest.mark.parametrize("k", [10, 100])
def test_c3_recipe(k):
    """65 536 cells, symmetric random CSR with mean degree close to k (no self loops, rows
    ascending), one weight 0.04 * 64 / k, a seeded ~20 % of cells pulsed 50-60 ms."""
    c = inputs.config("c3", k=k)
    n, rp, col = c["n"], c["row_ptr"], c["col"]
    assert n == 65536 and rp.dtype == np.int32 and col.dtype == np.int32
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert (rows != col).all()
    same_row = rows[1:] == rows[:-1]
    assert (col[1:][same_row] > col[:-1][same_row]).all()
    fwd = set(zip(rows.tolist(), col.tolist()))
    assert all((j, i) in fwd for i, j in list(fwd)[:20000])                # symmetric
    assert abs(len(col) / n - k) <= 0.05 * k
    assert np.all(c["w"] == np.float32(0.04 * 64 / k))
    cells, beg, end, amp = _pulse_steps(c["pulses"])
    assert 0.18 <= len(np.unique(cells)) / n <= 0.22
    assert set(beg.tolist()) == {1000} and set(end.tolist()) == {1200} and set(amp.tolist()) == {6.0}


def test_batch_recipe():
    """256 networks, sizes log-uniform in [32, 4096], even dense / odd CSR with k in
    [8, 256], g_c in [0.01, 0.08], network b seeded with 1000 + b; each network's first
    ceil(n / 8) cells pulsed 20-30 ms."""
    specs = inputs.batch_specs()
    assert len(specs) == 256
    ns = np.array([s["n"] for s in specs])
    assert ns.min() >= 32 and ns.max() <= 4096
    logn = np.log(ns)
    assert abs(np.median(logn) - 0.5 * (np.log(32) + np.log(4096))) < 0.5   # log-uniform centre
    assert all(s["kind"] == ("dense" if b % 2 == 0 else "csr") for b, s in enumerate(specs))
    assert all(8 <= s["k"] <= 256 for s in specs if s["kind"] == "csr")
    assert all(0.01 <= s["g_ref"] <= 0.08 for s in specs)
    assert [s["seed"] for s in specs] == list(range(1000, 1256))
    net = inputs.batch_network(specs[1])
    cells, beg, end, _ = _pulse_steps(net["pulses"])
    assert len(cells) == (specs[1]["n"] + 7) // 8 and set(beg.tolist()) == {400} and set(end.tolist()) == {600}


def test_generator_is_deterministic_and_uniform():
    a = inputs.uniform(inputs.stream_seed(7, "x"), 200000)
    b = inputs.uniform(inputs.stream_seed(7, "x"), 200000)
    c = inputs.uniform(inputs.stream_seed(7, "y"), 200000)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.005 and abs(a.var() - 1 / 12) < 0.002
    # a window of the counter stream equals the same window of a longer draw
    assert np.array_equal(inputs.uniform(inputs.stream_seed(7, "x"), 100, offset=500), a[500:600])
