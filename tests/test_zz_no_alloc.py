"""The allocation-free dense gap-current entry point, checked against ion_gj_dense (two
calls in a row) and against the FP64 oracle (up to the largest size its array holds).

ion_gj_dense_noalloc serves callers that cannot allocate device memory (a loop with a
hard per-step deadline, code inside a stream capture, hosts that own all device memory);
its scratch is a fixed array inside the library instead of an allocation.  This file is
collected last on purpose, and it also passes when run alone in a fresh process."""
import numpy as np
import pytest

from paper_1612_01501_gb300 import inputs
from paper_1612_01501_gb300 import ion

from helpers import sum_abs_dv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01501_gb300 import build
    build.build()
    return torch


def test_noalloc_matches_allocating_entry_point_twice(torch_cuda):
    """Two calls in a row (different sizes, so the second reuses the array the first left
    behind), each compared with ion_gj_dense within the tolerance of the dense
    primitive's parity test: 2e-6 * g * sum_j |V_i - V_j|."""
    torch = torch_cuda
    for n, seed in ((1000, 41), (8192 + 77, 42)):
        vd = (-60.0 + inputs.vdend_jitter(n, seed, 20.0)).astype(np.float32)
        g = inputs.junction_weight(0.04, n)
        v = torch.from_numpy(vd).cuda()
        ic_ref = torch.empty(n, dtype=torch.float32, device="cuda")
        ic_new = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        ion.ion_gj_dense(v, g, ic_ref)
        ion.ion_gj_dense_noalloc(v, g, ic_new)
        torch.cuda.synchronize()
        a = ic_new.cpu().numpy()
        b = ic_ref.cpu().numpy()
        tol = 2e-6 * g * sum_abs_dv(vd) + 1e-30
        assert np.all(np.isfinite(a))
        assert np.all(np.abs(a - b) <= tol), (n, (np.abs(a - b) / tol).max())


@pytest.mark.parametrize("n", [1000, 65536])
def test_noalloc_matches_the_oracle(torch_cuda, O, n):
    """Against the FP64 oracle (not only the other CUDA entry point), at a small size and at
    the largest size the fixed array holds (65 536 cells, no padding), same bound as the
    dense primitive's parity test: 2e-6 * g * sum_j |V_i - V_j|."""
    torch = torch_cuda
    vd = (-60.0 + inputs.vdend_jitter(n, 43 + n, 20.0)).astype(np.float32)
    g = inputs.junction_weight(0.04, n)
    v = torch.from_numpy(vd).cuda()
    ic = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    ion.ion_gj_dense_noalloc(v, g, ic)
    torch.cuda.synchronize()
    got = ic.cpu().numpy().astype(np.float64)
    ref = O.gj_dense(vd.astype(np.float64), g, threads=max(1, O.max_threads()))
    tol = 2e-6 * g * sum_abs_dv(vd) + 1e-30
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= tol), (n, (np.abs(got - ref) / tol).max())


def test_noalloc_rejects_sizes_beyond_its_array(torch_cuda):
    torch = torch_cuda
    n = 65536 + 1
    v = torch.zeros(n, dtype=torch.float32, device="cuda")
    ic = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(ion.IonError) as ei:
        ion.ion_gj_dense_noalloc(v, 0.01, ic)
    assert ei.value.status == ion.ERR_INVALID_ARG
