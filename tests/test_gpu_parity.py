"""GPU path vs the FP64 oracle on identical seeded inputs (every test needs a GB300).

Bars (spec tolerances): one step from an identical FP32 state has relative error
<= 1e-5 (floors: 1 mV, 1e-3 for gates); voltages stay within 0.1 mV of the oracle over the
first 100 ms; spike times agree within one step over 1 s.  Gap-current primitives are held
to 2e-6 of sum_j |dV_ij| (the scale of the FP32 rounding of the scaled voltages).
"""
import numpy as np
import pytest

from paper_1612_01501_gb300 import inputs
from paper_1612_01501_gb300 import ion

from helpers import STEP_RTOL, TRAJ_MV, V_FIELDS, csr_abs_scale, initial_state, step_rel_err, sum_abs_dv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01501_gb300 import build
    build.build()
    return torch


def _threads(O):
    return max(1, O.max_threads())


# ------------------------------------------------------------------ model pieces

def test_rates_match_oracle(torch_cuda, O):
    worst_x = worst_t = 0.0
    for ca in (0.5, 3.7, 20.0, 800.0):
        for V in np.arange(-100.0, 60.0, 0.37):
            V32 = float(np.float32(V))
            xg, tg = ion.ion_rates(V32, ca)
            xo, to = O.rates(V32, float(np.float32(ca)))
            worst_x = max(worst_x, np.max(np.abs(xg - xo) / np.maximum(np.abs(xo), 1e-3)))
            m = to > 0
            worst_t = max(worst_t, np.max(np.abs(tg[m] - to[m]) / to[m]))
    assert worst_x < 2e-6, worst_x
    assert worst_t < 2e-6, worst_t


def test_default_state_matches_oracle(torch_cuda, O):
    g = ion.ion_default_state(5)
    o = O.default_state(5)
    assert step_rel_err(g, o).max() < 2e-6


# ------------------------------------------------------------------ gap-junction primitives

@pytest.mark.parametrize("n", [1, 2, 63, 1000, 8192, 16461])
@pytest.mark.parametrize("kahan", [True, False])
def test_gj_dense_primitive(torch_cuda, O, n, kahan):
    torch = torch_cuda
    vd = (-60.0 + inputs.vdend_jitter(n, 100 + n, 20.0)).astype(np.float32)
    g = inputs.junction_weight(0.04, max(n, 1))
    ic = torch.empty(n, dtype=torch.float32, device="cuda")
    ion.ion_gj_dense(torch.from_numpy(vd).cuda(), g, ic, kahan=kahan)
    torch.cuda.synchronize()
    ref = O.gj_dense(vd.astype(np.float64), float(np.float32(g)), threads=_threads(O))
    tol = 2e-6 * g * sum_abs_dv(vd) + 1e-30
    err = np.abs(ic.cpu().numpy() - ref)
    assert np.all(err <= tol), (err / tol).max()


@pytest.mark.parametrize("n,k", [(5000, 10), (5000, 100), (3001, 1000), (100, 0)])
def test_gj_csr_primitive(torch_cuda, O, n, k):
    torch = torch_cuda
    rp, col = inputs.random_symmetric_csr(n, k, 7)
    w = inputs.uniform(inputs.stream_seed(k, "w"), len(col), 0.001, 0.05).astype(np.float32)
    vd = (-60.0 + inputs.vdend_jitter(n, 9, 20.0)).astype(np.float32)
    ic = torch.empty(n, dtype=torch.float32, device="cuda")
    T = lambda a: torch.from_numpy(a).cuda()
    ion.ion_gj_csr(T(vd), T(rp), T(col) if len(col) else torch.zeros(1, dtype=torch.int32, device="cuda"),
                   T(w) if len(w) else None, 0.0, ic)
    torch.cuda.synchronize()
    ref = O.gj_csr(rp, col, w.astype(np.float64), vd.astype(np.float64))
    rows = np.repeat(np.arange(n), np.diff(rp))
    scale = np.bincount(rows, weights=w * np.abs(vd[rows] - vd[col]), minlength=n) if len(col) else np.zeros(n)
    err = np.abs(ic.cpu().numpy() - ref)
    assert np.all(err <= 2e-6 * scale + 1e-30)


# ------------------------------------------------------------------ one step from an identical state

def _one_step_case(O, name, n, kind, g=0.0, rp=None, col=None, w=None, warm=50, **kw):
    cfg = dict(n=n, jitter=inputs.vdend_jitter(n, 31))
    S0 = initial_state(O, cfg)
    k_or = {O.DENSE: O.DENSE, O.CSR: O.CSR, O.NOGJ: O.NOGJ}[kind]
    wd = None if w is None else w.astype(np.float64)
    # warm the state up with the oracle so every variable is off its steady state
    Sw, _ = O.run(S0.astype(np.float64), warm, kind=k_or, g=g, row_ptr=rp, col=col, w=wd, threads=_threads(O))
    Sw32 = Sw.astype(np.float32)
    iapp = inputs.uniform(inputs.stream_seed(n, "iapp"), n, 0.0, 4.0).astype(np.float32)
    ref, _ = O.run(Sw32.astype(np.float64), 1, kind=k_or, g=g, row_ptr=rp, col=col, w=wd, t0=0,
                   iapp_dense=iapp[None, :], threads=_threads(O))
    ikind = {O.DENSE: ion.DENSE_UNIFORM, O.CSR: ion.CSR, O.NOGJ: ion.NO_GJ}[kind]
    with ion.Simulation(n, ikind, g=g, row_ptr=rp, col=col, w=w, init_state=Sw32, **kw) as sim:
        sim.step(1, dense=iapp[None, :])
        got = sim.state()
    if kind == O.DENSE:
        scale = g * sum_abs_dv(Sw32[0])
    elif kind == O.CSR:
        scale = csr_abs_scale(rp, col, w, Sw32[0])
    else:
        scale = None
    return step_rel_err(got, ref, scale)


@pytest.mark.parametrize("n", [1, 64, 300, 8192])
@pytest.mark.parametrize("flags", [ion.FLAG_KAHAN, ion.FLAG_KAHAN | ion.FLAG_SPLIT])
def test_one_step_dense(torch_cuda, O, n, flags):
    g = inputs.junction_weight(0.04, n)
    err = _one_step_case(O, "dense", n, O.DENSE, g=float(np.float32(g)), flags=flags)
    assert err.max() <= STEP_RTOL, (err.max(axis=1))


@pytest.mark.parametrize("k", [10, 100, 1000])
def test_one_step_csr_c3(torch_cuda, O, k):
    cfg = inputs.config("c3", k=k)
    err = _one_step_case(O, "csr", cfg["n"], O.CSR, rp=cfg["row_ptr"], col=cfg["col"], w=cfg["w"], warm=5)
    assert err.max() <= STEP_RTOL, err.max(axis=1)


def test_one_step_csr_empty_rows_and_split(torch_cuda, O):
    n = 1000
    rp, col = inputs.random_symmetric_csr(n, 2, 5)      # many isolated cells
    w = np.full(len(col), 0.05, np.float32)
    for flags in (ion.FLAG_KAHAN, ion.FLAG_KAHAN | ion.FLAG_SPLIT):
        err = _one_step_case(O, "csr", n, O.CSR, rp=rp, col=col, w=w, flags=flags)
        assert err.max() <= STEP_RTOL


def test_one_step_no_gj(torch_cuda, O):
    err = _one_step_case(O, "nogj", 777, O.NOGJ)
    assert err.max() <= STEP_RTOL


def _sample_pulses(pulses, sample):
    """The pulse table restricted to the sampled cells, renumbered 0..len(sample)-1."""
    cells, beg, end, amp = pulses
    m = np.isin(cells, sample)
    return (np.searchsorted(sample, cells[m]).astype(np.int32), beg[m], end[m], amp[m])


def test_k3_cell_update_at_2p22_sampled(torch_cuda, O):
    """The cell update alone on 2^22 uncoupled cells (NGJ), in the launch configuration
    the benchmark times (graph replay of 100 steps).  Cells are independent, so the oracle
    follows a seeded sample of them: one step from an identical warmed state while their
    pulses are on, then 299 more steps."""
    cfg = inputs.config("k3")
    n = cfg["n"]
    S = initial_state(O, cfg)
    rng = np.random.default_rng(5)
    sample = np.unique(np.concatenate([[0, 1, n - 1], rng.choice(n, 1021, replace=False)])).astype(np.int64)
    sp = _sample_pulses(cfg["pulses"], sample)
    assert len(sp[0]) > 100                                   # some sampled cells are pulsed
    warm, _ = O.run(S[:, sample].astype(np.float64), 50, kind=O.NOGJ, t0=0, pulses=sp, threads=_threads(O))
    S[:, sample] = warm.astype(np.float32)                    # both sides start from the warmed sample
    t0 = inputs.step_of_ms(5.0)                               # first step of the pulses
    with ion.Simulation(n, ion.NO_GJ, init_state=S, graph_steps=100, flags=ion.FLAG_KAHAN) as sim:
        sim.set_input(cfg["pulses"])
        ion.ion_set_step_count(sim.h, t0)
        sim.step(1)
        got1 = sim.state()[:, sample]
        sim.step(299)
        got2 = sim.state()[:, sample]
    ref1, _ = O.run(S[:, sample].astype(np.float64), 1, kind=O.NOGJ, t0=t0, pulses=sp, threads=_threads(O))
    assert step_rel_err(got1, ref1).max() <= STEP_RTOL
    ref2, _ = O.run(ref1, 299, kind=O.NOGJ, t0=t0 + 1, pulses=sp, threads=_threads(O))
    dv = np.abs(got2[list(V_FIELDS)].astype(np.float64) - ref2[list(V_FIELDS)]).max()
    assert dv <= TRAJ_MV, dv


# ------------------------------------------------------------------ trajectories

def _run_both(O, cfg, n_steps, chunk, kind="dense", trace=False, **kw):
    """Run GPU and oracle side by side in chunks; yield (t, gpu_state, oracle_state)."""
    n = cfg["n"]
    S0 = initial_state(O, cfg)
    k_or = O.DENSE if cfg["kind"] == "dense" else O.CSR
    ikind = ion.DENSE_UNIFORM if cfg["kind"] == "dense" else ion.CSR
    Sref = S0.astype(np.float64)
    sim = ion.Simulation(n, ikind, g=cfg.get("g", 0.0), row_ptr=cfg.get("row_ptr"), col=cfg.get("col"),
                         w=cfg.get("w"), init_state=S0, **kw)
    if cfg.get("pulses") is not None:
        sim.set_input(cfg["pulses"])
    wd = None if cfg.get("w") is None else cfg["w"].astype(np.float64)
    t = 0
    try:
        while t < n_steps:
            c = min(chunk, n_steps - t)
            sim.step(c)
            Sref, tr = O.run(Sref, c, kind=k_or, g=cfg.get("g", 0.0), row_ptr=cfg.get("row_ptr"), col=cfg.get("col"),
                             w=wd, t0=t, pulses=cfg.get("pulses"), trace_cells=np.arange(n) if trace else None,
                             threads=_threads(O))
            t += c
            yield t, sim, Sref, tr
    finally:
        sim.close()


def test_c1_voltages_within_0p1mv_over_100ms(torch_cuda, O):
    cfg = inputs.config("c1")
    worst = 0.0
    for t, sim, Sref, _ in _run_both(O, cfg, 2000, 100):
        got = sim.state()
        worst = max(worst, np.abs(got[:3] - Sref[:3]).max())
    assert worst <= TRAJ_MV, worst


def _spike_times_case(O, cfg):
    n = cfg["n"]
    S0 = initial_state(O, cfg)
    _, otr = O.run(S0.astype(np.float64), 20000, kind=O.DENSE, g=cfg["g"], pulses=cfg["pulses"],
                   trace_cells=np.arange(n), threads=_threads(O))
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=cfg["g"], init_state=S0) as sim:
        sim.set_input(cfg["pulses"])
        ion.ion_set_trace(sim.h, 1, 20000)
        sim.step(20000)
        gtr = ion.ion_read_trace(sim.h, n, 20000)
    assert gtr.shape == otr.shape
    total = 0
    for c in range(n):
        a = O.spike_steps(gtr[:, c])
        b = O.spike_steps(otr[:, c])
        assert len(a) == len(b), (c, a, b)
        assert np.all(np.abs(a - b) <= 1), (c, a, b)
        total += len(b)
    return total


def test_c1_spike_times_over_1s(torch_cuda, O):
    """The 64-cell network for 1 s.  Under this cell model the pulse to 8 of 64 cells
    drains through the 56 unpulsed partners (g = 0.04 each) and no cell fires, so this
    checks that neither side fires; the spiking variant below carries the spike times."""
    assert _spike_times_case(O, inputs.config("c1")) == 0


def test_spike_times_over_1s_spiking_network(torch_cuda, O):
    """The 64-cell network with every cell pulsed three times: every cell fires bursts
    (about 1000 spikes in 1 s) and every spike time agrees within one step."""
    total = _spike_times_case(O, inputs.config("c1_spiking"))
    assert total >= 16 * 64, total


def test_validation_experiment_spikes(torch_cuda, O):
    """Sec. 3: identical cells + a pulse to all: every cell spikes, in step, on the GPU as
    in the oracle (spike times within one step), and the GPU cells stay bitwise equal."""
    cfg = inputs.config("validation")
    n = cfg["n"]
    S0 = initial_state(O, cfg)
    Sref, otr = O.run(S0.astype(np.float64), 4000, kind=O.DENSE, g=cfg["g"], pulses=cfg["pulses"],
                      trace_cells=np.arange(n), threads=_threads(O))
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=cfg["g"], init_state=S0) as sim:
        sim.set_input(cfg["pulses"])
        ion.ion_set_trace(sim.h, 1, 4000)
        sim.step(4000)
        gtr = ion.ion_read_trace(sim.h, n, 4000)
        S = sim.state()
    assert np.all(S == S[:, :1])
    a = O.spike_steps(gtr[:, 0])
    b = O.spike_steps(otr[:, 0])
    assert len(a) >= 2 and len(a) == len(b) and np.all(np.abs(a - b) <= 1), (a, b)


def test_c2_first_20ms(torch_cuda, O):
    """8192-cell all-to-all network, checked against the FP64 oracle on its first 20 ms."""
    cfg = inputs.config("c2")
    worst = 0.0
    for t, sim, Sref, _ in _run_both(O, cfg, 400, 100):
        got = sim.state()
        worst = max(worst, np.abs(got[:3] - Sref[:3]).max())
    assert worst <= TRAJ_MV, worst


@pytest.mark.parametrize("k", [10, 100, 1000])
def test_c3_trajectory(torch_cuda, O, k):
    """The 65 536-cell sparse network at each density for the first 100 ms (2000 steps,
    the pulse to ~20 % of the cells at 50-60 ms included), checked every 25 ms."""
    cfg = inputs.config("c3", k=k)
    worst = 0.0
    for t, sim, Sref, _ in _run_both(O, cfg, 2000, 500):
        got = sim.state()
        d = np.abs(got[:3] - Sref[:3]).max()
        assert d <= TRAJ_MV, (t, d)
        worst = max(worst, d)
    print(f"k = {k}: worst |dV| over 100 ms {worst:.2e} mV")


# ------------------------------------------------------------------ runtime behaviour

def test_graph_replay_bitwise_equals_direct_launches(torch_cuda, O):
    cfg = inputs.config("c1")
    S0 = initial_state(O, cfg)
    out = []
    for flags in (ion.FLAG_KAHAN, ion.FLAG_KAHAN | ion.FLAG_NO_GRAPH):
        with ion.Simulation(64, ion.DENSE_UNIFORM, g=cfg["g"], init_state=S0, flags=flags, graph_steps=40) as sim:
            sim.set_input(cfg["pulses"])
            sim.step(2123)
            out.append(sim.state())
    np.testing.assert_array_equal(out[0], out[1])


def test_checkpoint_restart_bitwise(torch_cuda, O):
    """2n steps straight == n steps, save (state + step count), restore in a new handle, n steps."""
    cfg = inputs.config("c3", k=10)
    S0 = initial_state(O, cfg)
    kw = dict(row_ptr=cfg["row_ptr"], col=cfg["col"], w=cfg["w"])
    with ion.Simulation(cfg["n"], ion.CSR, init_state=S0, **kw) as a:
        a.set_input(cfg["pulses"])
        a.step(1101)
        mid, t_mid = a.state(), a.t
        a.step(1100)
        straight = a.state()
    with ion.Simulation(cfg["n"], ion.CSR, init_state=mid, **kw) as b:
        ion.ion_set_step_count(b.h, t_mid)
        b.set_input(cfg["pulses"])
        b.step(1100)
        resumed = b.state()
    np.testing.assert_array_equal(straight, resumed)


def test_nonfinite_state_is_reported(torch_cuda, O):
    n = 8
    S0 = O.default_state(n).astype(np.float32)
    with ion.Simulation(n, ion.NO_GJ, init_state=S0) as sim:
        sim.set_input(inputs.pulses(np.arange(n), 0.0, 50.0, 5000.0))   # drives explicit Euler to overflow
        sim.step(1000)
        with pytest.raises(ion.IonError) as ei:
            sim.sync()
        assert ei.value.status == ion.ERR_NONFINITE


def test_write_then_read_roundtrip(torch_cuda, O):
    n = 333
    S = initial_state(O, dict(n=n, jitter=inputs.vdend_jitter(n, 3)))
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=0.01) as sim:
        sim.step(3)                 # odd step count: V_dend lives in the second slot
        sim.write(S)
        np.testing.assert_array_equal(sim.state(), S)
        sim.write(S[5] * 0 + 0.25, field=5)
        assert np.all(sim.state(5) == 0.25)


@pytest.mark.parametrize("sw,rows", [(1, 37), (2, 256), (8, 100), (32, 7)])
def test_csr_launch_shapes_agree(torch_cuda, O, sw, rows):
    """Every lanes-per-row / rows-per-CTA choice gives the oracle's step (ragged CTAs)."""
    n = 3001
    rp, col = inputs.random_symmetric_csr(n, 24, 13)
    w = np.full(len(col), inputs.junction_weight(0.04, 24), np.float32)
    err = _one_step_case(O, "csr", n, O.CSR, rp=rp, col=col, w=w, warm=5,
                         tune=dict(csr_lanes_per_row=sw, csr_rows_per_cta=rows))
    assert err.max() <= STEP_RTOL


def test_gj_csr_unaligned_and_unweighted(torch_cuda, O):
    """Index/weight arrays that are not 16-byte aligned take the scalar-load path; a NULL
    weight array means every weight is g_c."""
    torch = torch_cuda
    n = 4000
    rp, col = inputs.random_symmetric_csr(n, 50, 17)
    vd = (-60.0 + inputs.vdend_jitter(n, 19, 20.0)).astype(np.float32)
    w = inputs.uniform(inputs.stream_seed(3, "w"), len(col), 0.001, 0.05).astype(np.float32)
    T = lambda a: torch.from_numpy(a).cuda()
    col_u = torch.zeros(len(col) + 1, dtype=torch.int32, device="cuda")
    col_u[1:] = T(col)
    w_u = torch.zeros(len(col) + 1, dtype=torch.float32, device="cuda")
    w_u[1:] = T(w)
    ic = torch.empty(n, dtype=torch.float32, device="cuda")
    ion.ion_gj_csr(T(vd), T(rp), col_u[1:], w_u[1:], 0.0, ic)
    torch.cuda.synchronize()
    ref = O.gj_csr(rp, col, w.astype(np.float64), vd.astype(np.float64))
    scale = csr_abs_scale(rp, col, w, vd)
    assert np.all(np.abs(ic.cpu().numpy() - ref) <= 2e-6 * scale + 1e-30)
    g = 0.02
    ion.ion_gj_csr(T(vd), T(rp), T(col), None, g, ic)
    torch.cuda.synchronize()
    ref = O.gj_csr(rp, col, np.full(len(col), np.float64(np.float32(g))), vd.astype(np.float64))
    scale = csr_abs_scale(rp, col, np.full(len(col), g), vd)
    assert np.all(np.abs(ic.cpu().numpy() - ref) <= 2e-6 * scale + 1e-30)


@pytest.mark.parametrize("n,k,staging", [(40000, 64, 0), (40000, 64, 1), (3001, 40, 2), (70000, 12, 2)])
def test_csr_shared_memory_staging(torch_cuda, O, n, k, staging):
    """V_dend staged in shared memory chunk by chunk (two or three 128 KB chunks, or one),
    or gathered through L1/L2: both match the oracle's step."""
    rp, col = inputs.random_symmetric_csr(n, k, 23)
    w = np.full(len(col), inputs.junction_weight(0.04, k), np.float32)
    err = _one_step_case(O, "csr", n, O.CSR, rp=rp, col=col, w=w, warm=3, tune=dict(csr_staging=staging))
    assert err.max() <= STEP_RTOL


@pytest.mark.parametrize("n,k,staging", [(3001, 48, 1), (3001, 12, 1), (3001, 24, 2), (70000, 40, 1), (70000, 300, 2)])
@pytest.mark.parametrize("weights", ["uniform", "random", "as_given"])
def test_csr_compact_layouts(torch_cuda, O, n, k, staging, weights):
    """The compact CSR layouts (16-bit columns; one scalar for bitwise-equal weights) and
    the layout as given all reproduce the oracle's step; the handle reports what it
    streams per edge: 16-bit columns when V_dend is staged in chunks, or n <= 65 536 with
    rows of at least 32 edges on average."""
    rp, col = inputs.random_symmetric_csr(n, k, 29)
    g = inputs.junction_weight(0.04, k)
    if weights == "random":
        w = (g * inputs.uniform(inputs.stream_seed(n, "edge_w"), len(col), 0.5, 1.5)).astype(np.float32)
    else:
        w = np.full(len(col), g, np.float32)
    flags = ion.FLAG_KAHAN | (ion.FLAG_CSR_AS_GIVEN if weights == "as_given" else 0)
    tune = dict(csr_staging=staging)
    with ion.Simulation(n, ion.CSR, row_ptr=rp, col=col, w=w, flags=flags, tune=tune) as sim:
        lay = ion.ion_csr_layout(sim.h)
    assert lay["staged"] == (1 if staging == 2 else 0)
    if weights == "as_given":
        assert lay == dict(index_bytes=4, weight_bytes=4, staged=lay["staged"])
    else:
        deg = len(col) / n
        assert lay["index_bytes"] == (2 if (staging == 2 or (n <= 65536 and deg >= 32)) else 4)
        assert lay["weight_bytes"] == (0 if weights == "uniform" else 4)
    err = _one_step_case(O, "csr", n, O.CSR, rp=rp, col=col, w=w, warm=3, flags=flags, tune=tune)
    assert err.max() <= STEP_RTOL, err.max(axis=1)


@pytest.mark.parametrize("n,k", [(40000, 600), (70000, 300), (40000, 64)])
def test_csr_bank_order(torch_cuda, O, n, k):
    """16-bit columns stored in shared-memory bank order (ion_tune.csr_bank_order; staged
    kernel at 32, 16 and 8 lanes per row) reproduce the oracle's step, and over 30 steps
    differ from the sorted order only by rounding (but do differ: the order is applied)."""
    rp, col = inputs.random_symmetric_csr(n, k, 31)
    w = np.full(len(col), inputs.junction_weight(0.04, k), np.float32)
    tune = dict(csr_staging=2, csr_bank_order=1)
    err = _one_step_case(O, "csr", n, O.CSR, rp=rp, col=col, w=w, warm=3, tune=tune)
    assert err.max() <= STEP_RTOL, err.max(axis=1)
    S0 = ion.ion_default_state(n)
    S0[0] = (S0[0] + inputs.vdend_jitter(n, 31)).astype(np.float32)
    out = []
    for tu in (tune, dict(csr_staging=2)):
        with ion.Simulation(n, ion.CSR, row_ptr=rp, col=col, w=w, init_state=S0, tune=tu) as sim:
            assert ion.ion_csr_layout(sim.h)["staged"] == 1
            sim.step(30)
            out.append(sim.state())
    assert np.isfinite(out[0]).all()
    assert np.abs(out[0][:3] - out[1][:3]).max() <= 1e-3
    assert not np.array_equal(out[0], out[1])


# ------------------------------------------------------------------ SGJ use case (linear junctions)

def _sgj_one_step(O, n, kind, g=0.0, rp=None, col=None, w=None, tune=None, layout=None):
    cfg = dict(n=n, jitter=inputs.vdend_jitter(n, 41))
    S0 = initial_state(O, cfg)
    k_or = O.DENSE_SGJ if kind == O.DENSE else O.CSR_SGJ
    wd = None if w is None else w.astype(np.float64)
    Sw, _ = O.run(S0.astype(np.float64), 30, kind=k_or, g=g, row_ptr=rp, col=col, w=wd, threads=_threads(O))
    Sw32 = Sw.astype(np.float32)
    iapp = inputs.uniform(inputs.stream_seed(n, "iapp_sgj"), n, 0.0, 4.0).astype(np.float32)
    ref, _ = O.run(Sw32.astype(np.float64), 1, kind=k_or, g=g, row_ptr=rp, col=col, w=wd, t0=0,
                   iapp_dense=iapp[None, :], threads=_threads(O))
    ikind = ion.DENSE_UNIFORM if kind == O.DENSE else ion.CSR
    kw = {} if tune is None else dict(tune=tune)
    with ion.Simulation(n, ikind, g=g, row_ptr=rp, col=col, w=w, init_state=Sw32,
                        flags=ion.FLAG_KAHAN | ion.FLAG_SGJ, **kw) as sim:
        if layout is not None:
            layout.update(ion.ion_csr_layout(sim.h))
        sim.step(1, dense=iapp[None, :])
        got = sim.state()
    scale = g * sum_abs_dv(Sw32[0]) if kind == O.DENSE else csr_abs_scale(rp, col, w, Sw32[0])
    return step_rel_err(got, ref, scale)


@pytest.mark.parametrize("n", [1, 300, 8192, 20000])     # up to 16 384 cells: one launch per step; 20 000: two
def test_sgj_dense_one_step(torch_cuda, O, n):
    err = _sgj_one_step(O, n, O.DENSE, g=float(np.float32(inputs.junction_weight(0.04, n))))
    assert err.max() <= STEP_RTOL, err.max(axis=1)


# (cells, mean degree, weights, staging asked (0: the default), expected layout): 16-bit
# columns for networks of at most 65 536 cells with rows of 32 or more edges (the compact
# kernels with the linear term), staged chunk by chunk when asked or when rows are long
# (the default stages rows of 64 or more edges that keep 32 or more per 32 768-cell chunk),
# 32-bit columns read by eight lanes per row otherwise
@pytest.mark.parametrize("n,k,weights,staging,index_bytes,staged", [
    (65536, 100, "uniform", 0, 2, 1), (2000, 64, "random", 1, 2, 0), (40000, 64, "uniform", 2, 2, 1),
    (40000, 48, "random", 2, 2, 1), (1000, 7, "random", 0, 4, 0)])
def test_sgj_csr_one_step(torch_cuda, O, n, k, weights, staging, index_bytes, staged):
    rp, col = inputs.random_symmetric_csr(n, k, 17)
    g = inputs.junction_weight(0.04, k)
    w = np.full(len(col), g, np.float32)
    if weights == "random":
        w = (w * inputs.uniform(inputs.stream_seed(n, "sgj_w"), len(col), 0.5, 1.5)).astype(np.float32)
    lay = {}
    tune = dict(csr_staging=staging) if staging else None
    err = _sgj_one_step(O, n, O.CSR, rp=rp, col=col, w=w, tune=tune, layout=lay)
    assert lay["index_bytes"] == index_bytes and lay["staged"] == staged, lay
    assert err.max() <= STEP_RTOL, err.max(axis=1)


@pytest.mark.parametrize("kind", ["rgj", "sgj"])
def test_staged_csr_with_rows_of_thousands_of_edges(torch_cuda, O, kind):
    """A 4096-cell network with about 63 % of all pairs connected (rows of ~2600 edges, one
    chunk): the staged kernel keeps the unpadded layout for such rows with the exponential
    junction and the padded one with the linear junction; both reproduce the oracle's step."""
    n = 4096
    rp, col = inputs.random_symmetric_csr(n, n, 31)   # n/2 draws per cell: ~63 % of all pairs
    assert len(col) / n > 1500
    g = inputs.junction_weight(0.04, len(col) / n)
    w = np.full(len(col), g, np.float32)
    if kind == "sgj":
        lay = {}
        err = _sgj_one_step(O, n, O.CSR, rp=rp, col=col, w=w, tune=dict(csr_staging=2), layout=lay)
    else:
        lay = None
        err = _one_step_case(O, "csr", n, O.CSR, rp=rp, col=col, w=w, warm=3, tune=dict(csr_staging=2))
    assert err.max() <= STEP_RTOL, err.max(axis=1)
    if lay is not None:
        assert lay["staged"] == 1 and lay["index_bytes"] == 2


def test_sgj_csr_trajectory_on_the_staged_kernel(torch_cuda, O):
    """Linear junctions through the staged compact kernel (two chunks) for 20 ms: within
    0.1 mV of the oracle."""
    n, k = 40000, 40
    rp, col = inputs.random_symmetric_csr(n, k, 23)
    g = inputs.junction_weight(0.04, k)
    cfg = dict(n=n, jitter=inputs.vdend_jitter(n, 43))
    S0 = initial_state(O, cfg)
    pulses = inputs.pulses(inputs.random_subset(n, 0.2, 43), 2.0, 12.0, 6.0)
    with ion.Simulation(n, ion.CSR, row_ptr=rp, col=col, w=np.full(len(col), g, np.float32), init_state=S0,
                        flags=ion.FLAG_KAHAN | ion.FLAG_SGJ, tune=dict(csr_staging=2)) as sim:
        assert ion.ion_csr_layout(sim.h)["staged"] == 1
        sim.set_input(pulses)
        sim.step(400)
        got = sim.state()
    ref, _ = O.run(S0.astype(np.float64), 400, kind=O.CSR_SGJ, g=g, row_ptr=rp, col=col,
                   w=np.full(len(col), g, np.float64), pulses=pulses, threads=_threads(O))
    assert np.abs(got[:3] - ref[:3]).max() <= TRAJ_MV


def test_sgj_c1_trajectory_100ms(torch_cuda, O):
    """The 64-cell network with linear junctions: within 0.1 mV of the oracle for 100 ms."""
    cfg = inputs.config("c1")
    n = cfg["n"]
    S0 = initial_state(O, cfg)
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=cfg["g"], init_state=S0, flags=ion.FLAG_KAHAN | ion.FLAG_SGJ) as sim:
        sim.set_input(cfg["pulses"])
        sim.step(2000)
        got = sim.state()
    ref, _ = O.run(S0.astype(np.float64), 2000, kind=O.DENSE_SGJ, g=cfg["g"], pulses=cfg["pulses"],
                   threads=_threads(O))
    assert np.abs(got[:3] - ref[:3]).max() <= TRAJ_MV


# ------------------------------------------------------------------ dense N x N weight matrix

def _matrix(n, seed):
    g = inputs.junction_weight(0.04, n)
    return (g * inputs.uniform(inputs.stream_seed(seed, "matrix_w"), n * n, 0.0, 2.0)).astype(np.float32).reshape(n, n)


@pytest.mark.parametrize("n,R", [(1, 0), (300, 0), (3001, 1), (3001, 2), (3001, 4), (9000, 0)])
def test_matrix_one_step(torch_cuda, O, n, R):
    """One step with an asymmetric random weight matrix (one or two V_dend tiles, a ragged
    last CTA) from an identical state, against the FP64 oracle; the I_c floor is the
    scale of its terms, sum_j |W_ij| |dV_ij|."""
    W = _matrix(n, 50)
    cfg = dict(n=n, jitter=inputs.vdend_jitter(n, 51))
    S0 = initial_state(O, cfg)
    Wd = W.astype(np.float64)
    Sw, _ = O.run(S0.astype(np.float64), 5, kind=O.MATRIX, w=Wd, threads=_threads(O))
    Sw32 = Sw.astype(np.float32)
    ref, _ = O.run(Sw32.astype(np.float64), 1, kind=O.MATRIX, w=Wd, threads=_threads(O))
    tune = dict(dense_rows_per_warp=R) if R else None    # 0: the library's choice
    with ion.Simulation(n, ion.DENSE_MATRIX, w=W, init_state=Sw32, tune=tune) as sim:
        sim.step(1)
        got = sim.state()
    vd = Sw32[0].astype(np.float64)
    scale = np.array([np.abs(Wd[i]) @ np.abs(vd[i] - vd) for i in range(n)])
    err = step_rel_err(got, ref, scale)
    assert err.max() <= STEP_RTOL, err.max(axis=1)


def test_matrix_from_device_tensor_and_uniform_matches_dense(torch_cuda, O):
    """A device-resident matrix is copied like a host one, and a uniform matrix gives the
    uniform dense network's trajectory (different summation order: close, not equal)."""
    torch = torch_cuda
    n = 1000
    g = float(np.float32(inputs.junction_weight(0.04, n)))
    cfg = dict(n=n, jitter=inputs.vdend_jitter(n, 52))
    S0 = initial_state(O, cfg)
    Wt = torch.full((n, n), g, dtype=torch.float32, device="cuda")
    with ion.Simulation(n, ion.DENSE_MATRIX, w=Wt, init_state=S0) as sim:
        sim.step(400)
        a = sim.state()
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=g, init_state=S0) as sim:
        sim.step(400)
        b = sim.state()
    assert np.abs(a[:3] - b[:3]).max() <= 1e-3


# ------------------------------------------------------------------ asynchronous trace drain

def test_trace_async_drain_matches_sync_read(torch_cuda, O):
    """V_axon samples drained asynchronously (copy stream, pinned buffer, steps enqueued
    behind the copy) equal the synchronous reads of an identical run, through a ring of
    600 samples drained every 500 steps (it wraps, and later steps must wait for the copy
    still reading the slots they overwrite)."""
    torch = torch_cuda
    cfg = inputs.config("c1_spiking")
    n, rounds, per = cfg["n"], 6, 500
    S0 = initial_state(O, cfg)
    outs = []
    for mode in ("async", "sync"):
        with ion.Simulation(n, ion.DENSE_UNIFORM, g=cfg["g"], init_state=S0) as sim:
            sim.set_input(cfg["pulses"])
            ion.ion_set_trace(sim.h, 1, 600)
            if mode == "async":
                buf = torch.empty((rounds * per, n), dtype=torch.float32).pin_memory()
                got = 0
                for r in range(rounds):
                    sim.step(per)
                    got += ion.ion_read_trace_async(sim.h, buf[got:], rounds * per - got)
                ion.ion_trace_wait(sim.h)
                assert got == rounds * per
                outs.append(buf.numpy().copy())
            else:
                parts = []
                for r in range(rounds):
                    sim.step(per)
                    parts.append(ion.ion_read_trace(sim.h, n, per))
                outs.append(np.concatenate(parts))
    np.testing.assert_array_equal(outs[0], outs[1])
    assert len(O.spike_steps(outs[0][:, 0])) >= 2       # the drained trace holds real spikes


# ------------------------------------------------------------------ the configuration the bench times

@pytest.mark.parametrize("workload", ["c2", "c3_k100"])
def test_autotuned_full_size_one_step(torch_cuda, O, workload):
    """The full-size network after ion_autotune (as bench.py runs it: graph replay of 100
    steps), one step from an identical warmed state against the FP64 oracle."""
    cfg = inputs.config("c2") if workload == "c2" else inputs.config("c3", k=100)
    n = cfg["n"]
    S0 = initial_state(O, cfg)
    dense = cfg["kind"] == "dense"
    kind = O.DENSE if dense else O.CSR
    kw = dict(g=cfg["g"]) if dense else dict(row_ptr=cfg["row_ptr"], col=cfg["col"], w=cfg["w"])
    wd = None if dense else cfg["w"].astype(np.float64)
    Sw, _ = O.run(S0.astype(np.float64), 3, kind=kind, g=cfg.get("g", 0.0), row_ptr=cfg.get("row_ptr"),
                  col=cfg.get("col"), w=wd, threads=_threads(O))
    Sw32 = Sw.astype(np.float32)
    ref, _ = O.run(Sw32.astype(np.float64), 1, kind=kind, g=cfg.get("g", 0.0), row_ptr=cfg.get("row_ptr"),
                   col=cfg.get("col"), w=wd, t0=3, threads=_threads(O))
    with ion.Simulation(n, ion.DENSE_UNIFORM if dense else ion.CSR, init_state=Sw32, graph_steps=100, **kw) as sim:
        table = ion.ion_autotune(sim.h, 10)
        assert sim.t == 0
        ion.ion_set_step_count(sim.h, 3)
        sim.step(1)
        got = sim.state()
    scale = cfg["g"] * sum_abs_dv(Sw32[0]) if dense else csr_abs_scale(cfg["row_ptr"], cfg["col"], cfg["w"], Sw32[0])
    err = step_rel_err(got, ref, scale)
    assert err.max() <= STEP_RTOL, (table, err.max(axis=1))


# ------------------------------------------------------------------ resources

def test_create_destroy_loop_does_not_leak(torch_cuda, O):
    """Twenty create/step/destroy cycles of a dense, a CSR (compact and staged) and a
    matrix network leave the device's free memory where it was (within 64 MB)."""
    torch = torch_cuda
    rp, col = inputs.random_symmetric_csr(40000, 300, 3)
    w = np.full(len(col), inputs.junction_weight(0.04, 300), np.float32)
    W = np.full((2048, 2048), 1e-4, np.float32)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(20):
        for make in (lambda: ion.Simulation(8192, ion.DENSE_UNIFORM, g=3e-4),
                     lambda: ion.Simulation(40000, ion.CSR, row_ptr=rp, col=col, w=w, tune=dict(csr_staging=2)),
                     lambda: ion.Simulation(2048, ion.DENSE_MATRIX, w=W)):
            with make() as sim:
                ion.ion_set_trace(sim.h, 1, 8)
                sim.step(3)
                sim.sync()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 <= 64 << 20, (free0 - free1) / 2**20


@pytest.mark.parametrize("case", ["dense", "csr", "csr_staged", "matrix", "no_gj", "sgj_dense", "batch"])
def test_programmatic_launches_match_ordinary_launches(torch_cuda, case):
    """Per-step kernels launched with programmatic stream serialization (the default) give
    the same bits as ordinary launches, over graph replays and direct launches."""
    n = 6000
    S0 = ion.ion_default_state(n)
    S0[0] = (S0[0] + inputs.vdend_jitter(n, 21)).astype(np.float32)
    g = inputs.junction_weight(0.04, n)
    if case in ("csr", "csr_staged"):
        rp, col = inputs.random_symmetric_csr(n, 120, 5)
        w = np.full(len(col), inputs.junction_weight(0.04, 120), np.float32)
        tune = dict(csr_staging=2) if case == "csr_staged" else None
        make = lambda fl: ion.ion_create(n, ion.CSR, row_ptr=rp, col=col, w=w, init_state=S0, flags=fl, tune=tune)
    elif case == "matrix":
        W = np.full((n, n), g, np.float32)
        make = lambda fl: ion.ion_create(n, ion.DENSE_MATRIX, w=W, init_state=S0, flags=fl)
    elif case == "no_gj":
        make = lambda fl: ion.ion_create(n, ion.NO_GJ, init_state=S0, flags=fl)
    elif case == "sgj_dense":
        make = lambda fl: ion.ion_create(n, ion.DENSE_UNIFORM, g=g, init_state=S0, flags=fl | ion.FLAG_SGJ)
    elif case == "batch":
        rp, col = inputs.random_symmetric_csr(3000, 20, 6)
        nets = [dict(n=3000, kind=ion.DENSE_UNIFORM, g=inputs.junction_weight(0.04, 3000)),
                dict(n=3000, kind=ion.CSR, row_ptr=rp, col=col, w=np.full(len(col), 2e-3, np.float32))]
        make = lambda fl: ion.ion_create_batch(nets, init_state=S0, flags=fl)
    else:
        make = lambda fl: ion.ion_create(n, ion.DENSE_UNIFORM, g=g, init_state=S0, flags=fl)
    pul = (np.array([0, 17, 4000], np.int32), np.array([2, 5, 40], np.int64), np.array([30, 60, 90], np.int64),
           np.array([6.0, 4.0, 5.0], np.float32))
    out = []
    for extra in (0, ion.FLAG_NO_PDL):
        h = make(ion.FLAG_KAHAN | extra)
        try:
            ion.ion_set_input(h, pul)
            ion.ion_set_trace(h, 1, 130)
            ion.ion_step(h, 100)        # graph replays
            ion.ion_step(h, 27)         # direct launches
            ion.ion_sync(h)
            out.append((ion.ion_read_state(h, n), ion.ion_read_trace(h, n, 127)))
        finally:
            ion.ion_destroy(h)
    assert np.isfinite(out[0][0]).all()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


# ------------------------------------------------------------------ per-cell constants

def _cell_params(O, n, seed):
    """(NCELLPARAMS, n) per-cell constants: the table's conductances and area ratios scaled
    by U(0.7, 1.3), its reversal potentials shifted by U(-3, 3) mV, per cell."""
    rng = np.random.default_rng(seed)
    base = O.model_default()[:O.NCELLPARAMS]
    cp = np.repeat(base[:, None], n, axis=1)
    for p in range(O.NCELLPARAMS):
        if O.PARAMS[p].startswith("V_"):
            cp[p] += rng.uniform(-3.0, 3.0, n)
        else:
            cp[p] *= rng.uniform(0.7, 1.3, n)
    return cp.astype(np.float32)


@pytest.mark.parametrize("kind", ["dense", "csr", "no_gj"])
def test_per_cell_constants_one_step(torch_cuda, O, kind):
    """One step from an identical FP32 state with every cell owning its constants (the FP32
    values are what both sides read)."""
    n = 3001
    cp = _cell_params(O, n, 21)
    S0 = O.default_state(n)
    S0[O.F["V_dend"]] += inputs.vdend_jitter(n, 22, 8.0)
    S0[O.F["g_CaL"]] = np.linspace(0.5, 1.0, n)
    S0 = S0.astype(np.float32)
    kw, okw, scale = {}, {}, None
    if kind == "dense":
        g = inputs.junction_weight(0.04, n)
        ikind, kw, okw = ion.DENSE_UNIFORM, dict(g=g), dict(kind=O.DENSE, g=g)
        scale = g * sum_abs_dv(S0[0])
    elif kind == "csr":
        rp, col = inputs.random_symmetric_csr(n, 40, 23)
        w = np.full(len(col), inputs.junction_weight(0.04, 40), np.float32)
        ikind, kw = ion.CSR, dict(row_ptr=rp, col=col, w=w)
        okw = dict(kind=O.CSR, row_ptr=rp, col=col, w=w.astype(np.float64))
        scale = csr_abs_scale(rp, col, w, S0[0])
    else:
        ikind, okw = ion.NO_GJ, dict(kind=O.NOGJ)
    with ion.Simulation(n, ikind, init_state=S0, cell_params=cp, **kw) as sim:
        sim.step(1)
        got = sim.state()
    ref, _ = O.run(S0.astype(np.float64), 1, cell_params=cp.astype(np.float64), threads=_threads(O), **okw)
    err = step_rel_err(got, ref, scale)
    assert err.max() <= STEP_RTOL, err.max(axis=1)
    # the constants matter: the same step with the table's constants differs
    ref_table, _ = O.run(S0.astype(np.float64), 1, threads=_threads(O), **okw)
    assert np.abs(ref_table[1] - ref[1]).max() > 1e-3


def test_per_cell_constants_trajectory_100ms(torch_cuda, O):
    """The 64-cell all-to-all network (C1 inputs) with heterogeneous cells for 100 ms:
    voltages within 0.1 mV of the oracle."""
    cfg = inputs.config("c1")
    n = cfg["n"]
    cp = _cell_params(O, n, 31)
    S0 = initial_state(O, cfg)
    Sref = S0.astype(np.float64)
    worst = 0.0
    with ion.Simulation(n, ion.DENSE_UNIFORM, g=cfg["g"], init_state=S0, cell_params=cp) as sim:
        sim.set_input(cfg["pulses"])
        t = 0
        for _ in range(4):
            sim.step(500)
            Sref, _ = O.run(Sref, 500, kind=O.DENSE, g=cfg["g"], t0=t, pulses=cfg["pulses"],
                            cell_params=cp.astype(np.float64), threads=_threads(O))
            t += 500
            worst = max(worst, float(np.abs(sim.state()[:3] - Sref[:3]).max()))
    assert worst <= TRAJ_MV, worst


def test_per_cell_constants_rejected_where_unsupported(torch_cuda, O):
    n = 100
    cp = _cell_params(O, n, 41)
    bad = cp.copy()
    bad[O.P["p1"], 7] = 1.5
    nan = cp.copy()
    nan[O.P["g_Na_s"], 3] = np.nan
    for c, kw, code in ((bad, dict(kind=ion.NO_GJ), ion.ERR_INVALID_ARG),
                        (nan, dict(kind=ion.NO_GJ), ion.ERR_INVALID_ARG),
                        (cp, dict(kind=ion.DENSE_UNIFORM, g=0.01, flags=ion.FLAG_KAHAN | ion.FLAG_PERSISTENT),
                         ion.ERR_UNSUPPORTED),
                        (cp, dict(kind=ion.DENSE_UNIFORM, g=0.01, flags=ion.FLAG_KAHAN | ion.FLAG_SGJ),
                         ion.ERR_UNSUPPORTED)):
        with pytest.raises(ion.IonError) as ei:
            ion.ion_create(n, cell_params=c, **kw)
        assert ei.value.status == code
    with pytest.raises(ion.IonError) as ei:
        ion.ion_create_batch([dict(n=n, kind=ion.NO_GJ)], cell_params=cp)
    assert ei.value.status == ion.ERR_UNSUPPORTED


# ------------------------------------------------------------------ half-work CSR

@pytest.mark.parametrize("n,k,weights", [(5000, 10, "uniform"), (5000, 100, "random"), (3001, 1000, "uniform"),
                                         (65536, 100, "uniform")])
def test_csr_half_work_one_step(torch_cuda, O, n, k, weights):
    """Each stored pair evaluated once (upper triangle; the mirrored term through a
    per-edge slot, gathered per row in a fixed order): one step from an identical state
    against the oracle, at uniform and random symmetric weights."""
    rp, col = inputs.random_symmetric_csr(n, k, 51)
    w = np.full(len(col), inputs.junction_weight(0.04, k), np.float32)
    if weights == "random":   # symmetric: the weight of a pair from its smaller and larger cell
        rows = np.repeat(np.arange(n), np.diff(rp))
        lo, hi = np.minimum(rows, col).astype(np.uint64), np.maximum(rows, col).astype(np.uint64)
        h = (lo * np.uint64(2654435761) + hi * np.uint64(40503)) % np.uint64(1000)
        w = (w * (0.5 + h.astype(np.float64) / 1000.0)).astype(np.float32)
    err = _one_step_case(O, "csr", n, O.CSR, rp=rp, col=col, w=w, warm=3, flags=ion.FLAG_KAHAN | ion.FLAG_HALF_WORK)
    assert err.max() <= STEP_RTOL, err.max(axis=1)


def test_csr_half_work_trajectory_matches_full_pass(torch_cuda, O):
    """The 65 536-cell k = 100 network with its pulse, 600 steps: the half-work pass stays
    within the trajectory bound of the oracle, like the full pass."""
    cfg = inputs.config("c3", k=100)
    worst = 0.0
    for t, sim, Sref, _ in _run_both(O, cfg, 600, 300, flags=ion.FLAG_KAHAN | ion.FLAG_HALF_WORK):
        worst = max(worst, float(np.abs(sim.state()[:3] - Sref[:3]).max()))
    assert worst <= TRAJ_MV, worst


def test_csr_half_work_needs_symmetric_weights(torch_cuda, O):
    n = 200
    rp, col = inputs.random_symmetric_csr(n, 8, 52)
    w = np.linspace(0.01, 0.02, len(col)).astype(np.float32)   # not symmetric
    with pytest.raises(ion.IonError) as ei:
        ion.ion_create(n, ion.CSR, row_ptr=rp, col=col, w=w, flags=ion.FLAG_KAHAN | ion.FLAG_HALF_WORK)
    assert ei.value.status == ion.ERR_UNSUPPORTED
