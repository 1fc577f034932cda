"""Persistent dense launches (one cooperative launch per ion_step call, state in
registers, a bounded grid barrier per step) against the per-step path and the oracle,
and the barrier's timeout path (forced with the debug delay hook, no GPU fault)."""
import numpy as np
import pytest

from paper_1612_01501_gb300 import inputs
from paper_1612_01501_gb300 import ion

from helpers import TRAJ_MV, initial_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01501_gb300 import build
    build.build()
    return torch


def _run(n, g, S0, steps, flags, pulses=None, chunks=1, **kw):
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=g, init_state=S0, flags=flags, **kw) as sim:
        if pulses is not None:
            sim.set_input(pulses)
        for _ in range(chunks):
            sim.step(steps // chunks)
        return sim.state(), sim.launches


def test_persistent_full_work_bitwise_equals_step_launches(cuda, O):
    cfg = inputs.config("c2")
    S0 = initial_state(O, cfg)
    a, la = _run(cfg["n"], cfg["g"], S0, 300, ion.FLAG_KAHAN, chunks=3)
    b, lb = _run(cfg["n"], cfg["g"], S0, 300, ion.FLAG_KAHAN | ion.FLAG_PERSISTENT, chunks=3)
    np.testing.assert_array_equal(a, b)
    assert lb < la / 10        # one launch (+ one counter advance) per ion_step call


def test_persistent_half_work_matches_step_launches(cuda, O):
    """Each unordered pair evaluated once: a different summation order, so close, not equal."""
    cfg = inputs.config("c2")
    S0 = initial_state(O, cfg)
    a, _ = _run(cfg["n"], cfg["g"], S0, 300, ion.FLAG_KAHAN, chunks=3)
    b, lb = _run(cfg["n"], cfg["g"], S0, 300, ion.FLAG_KAHAN | ion.FLAG_PERSISTENT | ion.FLAG_HALF_WORK, chunks=3)
    assert np.abs(a[:3] - b[:3]).max() <= 1e-3
    assert lb == 6


@pytest.mark.parametrize("n,tune", [(8192, None), (4096, None), (1000, dict(dense_rows_per_warp=2, dense_warps=8,
                                                                           dense_col_splits=1)),
                                    (3001, dict(dense_rows_per_warp=4, dense_warps=16, dense_col_splits=2))])
def test_half_work_one_step_matches_oracle(cuda, O, n, tune):
    """One step of the half-work kernel (odd and even grids, one or two column splits)
    from an identical state, against the FP64 oracle (per-step bound 1e-5)."""
    from helpers import STEP_RTOL, step_rel_err, sum_abs_dv
    g = inputs.junction_weight(0.04, n)
    cfg = dict(n=n, jitter=inputs.vdend_jitter(n, 77))
    S0 = initial_state(O, cfg)
    Sw, _ = O.run(S0.astype(np.float64), 20, kind=O.DENSE, g=g, threads=max(1, O.max_threads()))
    Sw32 = Sw.astype(np.float32)
    ref, _ = O.run(Sw32.astype(np.float64), 1, kind=O.DENSE, g=g, threads=max(1, O.max_threads()))
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=g, init_state=Sw32,
                        flags=ion.FLAG_KAHAN | ion.FLAG_PERSISTENT | ion.FLAG_HALF_WORK, tune=tune) as sim:
        sim.step(1)
        got = sim.state()
    err = step_rel_err(got, ref, g * sum_abs_dv(Sw32[0]))
    assert err.max() <= STEP_RTOL, err.max(axis=1)


@pytest.mark.parametrize("n", [64, 100, 1000])
def test_persistent_matches_oracle_trajectory(cuda, O, n):
    cfg = dict(n=n, kind="dense", g=inputs.junction_weight(0.04, n), jitter=inputs.vdend_jitter(n, 5),
               pulses=inputs.pulses(np.arange(min(8, n)), 10.0, 20.0, 6.0))
    S0 = initial_state(O, cfg)
    got, _ = _run(n, cfg["g"], S0, 1000, ion.FLAG_KAHAN | ion.FLAG_PERSISTENT, pulses=cfg["pulses"], chunks=4)
    ref, _ = O.run(S0.astype(np.float64), 1000, kind=O.DENSE, g=cfg["g"], pulses=cfg["pulses"],
                   threads=max(1, O.max_threads()))
    assert np.abs(got[:3] - ref[:3]).max() <= TRAJ_MV


def test_persistent_trace_matches_step_trace(cuda, O):
    cfg = inputs.config("validation")
    n = cfg["n"]
    S0 = initial_state(O, cfg)
    out = []
    for flags in (ion.FLAG_KAHAN, ion.FLAG_KAHAN | ion.FLAG_PERSISTENT):
        with ion.Simulation(n, ion.DENSE_UNIFORM, g=cfg["g"], init_state=S0, flags=flags) as sim:
            sim.set_input(cfg["pulses"])
            ion.ion_set_trace(sim.h, 1, 3000)
            sim.step(3000)
            out.append(ion.ion_read_trace(sim.h, n, 3000))
    a = O.spike_steps(out[0][:, 0])
    b = O.spike_steps(out[1][:, 0])
    assert len(a) >= 2 and np.array_equal(a, b)


def test_grid_barrier_timeout_is_reported_not_hung(cuda, O):
    """One CTA sleeps 200 ms before its first barrier while the barrier bound is 1 ms:
    the other CTAs give up, raise the abort word and return; the launch ends and the host
    sees ION_ERR_TIMEOUT.  The handle's context stays usable afterwards."""
    n = 1000
    S0 = O.default_state(n).astype(np.float32)
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=0.01, init_state=S0, flags=ion.FLAG_KAHAN | ion.FLAG_PERSISTENT,
                        barrier_timeout_ns=1_000_000, debug_delay_ns=200_000_000) as sim:
        sim.step(5)
        with pytest.raises(ion.IonError) as ei:
            sim.sync()
        assert ei.value.status == ion.ERR_TIMEOUT
    # a fresh handle on the same context works
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=0.01, init_state=S0, flags=ion.FLAG_KAHAN | ion.FLAG_PERSISTENT) as s2:
        s2.step(5)
        s2.sync()


def test_half_work_barrier_timeout_is_reported(cuda, O):
    n = 4096        # several CTAs: the half-work kernel, two bounded barriers per step
    S0 = O.default_state(n).astype(np.float32)
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=0.001, init_state=S0,
                        flags=ion.FLAG_KAHAN | ion.FLAG_PERSISTENT | ion.FLAG_HALF_WORK,
                        barrier_timeout_ns=1_000_000, debug_delay_ns=200_000_000) as sim:
        sim.step(5)
        with pytest.raises(ion.IonError) as ei:
            sim.sync()
        assert ei.value.status == ion.ERR_TIMEOUT


@pytest.mark.parametrize("half", [False, True])
def test_grid_barrier_counter_wraps_past_2_to_32(cuda, O, half):
    """The barrier's 32-bit arrival counter starts 300 arrivals below 2^32 (test hook), so it
    and the barrier targets wrap within the first steps, as they do after ~2^32 arrivals of
    a long launch.  The comparison is modulo 2^32: the states equal those of a launch whose
    counter starts at 0, bit for bit."""
    cfg = inputs.config("c2")
    S0 = initial_state(O, cfg)
    flags = ion.FLAG_KAHAN | ion.FLAG_PERSISTENT | (ion.FLAG_HALF_WORK if half else 0)
    a, _ = _run(cfg["n"], cfg["g"], S0, 200, flags, chunks=2)
    b, _ = _run(cfg["n"], cfg["g"], S0, 200, flags, chunks=2, debug_barrier_base=(1 << 32) - 300)
    np.testing.assert_array_equal(a, b)
