"""Allocation failures, injected on the host.

`ion_debug_fail_alloc(k)` makes the device allocation after the next k ones report
out-of-memory.  For every k up to the number of allocations a handle makes (creation,
trace buffer, pulse table, persistent buffers, autotuner save area), the failing call must
return ION_ERR_OOM, leave nothing allocated once the handle is destroyed, and leave the
library usable: a clean run afterwards reproduces the one taken before (bit for bit, or,
where the autotuner may choose another launch shape, to rounding).
No device fault is involved: the failure is a status code returned before cudaMalloc.
"""
import numpy as np
import pytest

from paper_1612_01501_gb300 import inputs
from paper_1612_01501_gb300 import ion

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01501_gb300 import build
    build.build()
    return torch


def _pulses(n):
    cells = np.arange(0, n, max(1, n // 16), dtype=np.int32)
    return cells, np.full(len(cells), 1, np.int64), np.full(len(cells), 3, np.int64), np.full(len(cells), 4.0, np.float32)


def _state(n, seed):
    S = ion.ion_default_state(n)
    S[0] = (S[0] + inputs.vdend_jitter(n, seed)).astype(np.float32)
    return S


def _case(name):
    """(n, create(), extra(h)) of one handle recipe."""
    if name == "dense_graph":
        n = 4096
        return n, lambda S: ion.ion_create(n, ion.DENSE_UNIFORM, g=inputs.junction_weight(0.04, n), init_state=S), None
    if name == "dense_persistent":
        n = 8192
        return n, lambda S: ion.ion_create(n, ion.DENSE_UNIFORM, g=inputs.junction_weight(0.04, n), init_state=S,
                                           flags=ion.FLAG_KAHAN | ion.FLAG_PERSISTENT | ion.FLAG_HALF_WORK), None
    if name == "csr_staged":
        n = 40000
        rp, col = inputs.random_symmetric_csr(n, 300, 3)
        w = np.full(len(col), inputs.junction_weight(0.04, 300), np.float32)
        return n, lambda S: ion.ion_create(n, ion.CSR, row_ptr=rp, col=col, w=w, init_state=S,
                                           tune=dict(csr_staging=2)), None
    if name == "csr_autotune":
        n = 3000
        rp, col = inputs.random_symmetric_csr(n, 10, 4)
        rows = np.repeat(np.arange(n), np.diff(rp))
        a, b = np.minimum(rows, col).astype(np.int64), np.maximum(rows, col).astype(np.int64)
        w = (0.01 + 0.04 * ((a * 7919 + b * 104729) % 1000) / 1000.0).astype(np.float32)   # symmetric
        return n, lambda S: ion.ion_create(n, ion.CSR, row_ptr=rp, col=col, w=w, init_state=S), \
            lambda h: ion.ion_autotune(h, 2)
    if name == "matrix":
        n = 1024
        W = np.random.default_rng(5).uniform(0.0, 2e-4, (n, n)).astype(np.float32)
        W = np.triu(W, 1) + np.triu(W, 1).T
        return n, lambda S: ion.ion_create(n, ion.DENSE_MATRIX, w=W, init_state=S), None
    if name == "sgj_dense":
        n = 4096
        return n, lambda S: ion.ion_create(n, ion.DENSE_UNIFORM, g=inputs.junction_weight(0.04, n), init_state=S,
                                           flags=ion.FLAG_KAHAN | ion.FLAG_SGJ), None
    if name == "batch":
        rp, col = inputs.random_symmetric_csr(2000, 20, 6)
        nets = [dict(n=1500, kind=ion.DENSE_UNIFORM, g=3e-4),
                dict(n=2000, kind=ion.CSR, row_ptr=rp, col=col, w=np.full(len(col), 2e-3, np.float32)),
                dict(n=500, kind=ion.NO_GJ)]
        return 4000, lambda S: ion.ion_create_batch(nets, init_state=S), lambda h: ion.ion_autotune(h, 2)
    if name == "surrogate":
        from oracle import mlp
        p = mlp.init_params(5, scale=1.0)
        lo, hi = np.log(1.36), np.log(13.5)     # the [Ca] range the surrogate tests normalise by
        wts = ion.weights_from_dict({k: v.astype(np.float32) for k, v in p.items()},
                                    in_shift=(mlp.V_CENTER, 0.5 * (lo + hi)), in_scale=(1 / mlp.V_HALF, 2 / (hi - lo)))
        n = 4096
        return n, lambda S: ion.ion_create(n, ion.DENSE_UNIFORM, g=inputs.junction_weight(0.04, n), init_state=S,
                                           flags=ion.FLAG_KAHAN | ion.FLAG_SURROGATE, surrogate=wts), None
    raise KeyError(name)


def _run(n, create, extra, S):
    """Create, trace, pulse, (tune), step, read; returns the state.  Destroys on any error."""
    h = create(S)
    try:
        ion.ion_set_trace(h, 1, 8)
        ion.ion_set_input(h, _pulses(n))
        if extra is not None:
            extra(h)
        ion.ion_step(h, 5)
        ion.ion_sync(h)
        return ion.ion_read_state(h, n)
    finally:
        ion.ion_destroy(h)


CASES = ["dense_graph", "dense_persistent", "csr_staged", "csr_autotune", "matrix", "sgj_dense", "batch",
         "surrogate"]


@pytest.mark.parametrize("name", CASES)
def test_injected_allocation_failure(torch_cuda, name):
    torch = torch_cuda
    n, create, extra = _case(name)
    S = _state(n, 11)
    ref = _run(n, create, extra, S)            # also warms the context and the allocator
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    failed = 0
    for k in range(128):
        ion.ion_debug_fail_alloc(k)
        try:
            _run(n, create, extra, S)
        except ion.IonError as e:
            assert e.status == ion.ERR_OOM, f"allocation {k}: {e}"
            failed += 1
            continue
        finally:
            ion.ion_debug_fail_alloc(-1)
        break                                   # k is past the last allocation: the run completed
    else:
        pytest.fail("more than 128 device allocations in one run")
    assert failed >= 3, failed
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 <= 16 << 20, (free0 - free1) / 2**20
    again = _run(n, create, extra, S)
    if name in ("csr_autotune", "batch"):   # the tuner may pick another launch shape: another summation order
        np.testing.assert_allclose(again, ref, rtol=1e-4, atol=1e-4)
    else:
        assert np.array_equal(again, ref)
