"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Paper: Smaragdos et al., "BrainFrame" (arXiv 1612.01501).
  Sec. 2.2  -- synchronous explicit step (delta = 50 us), 19 state words (Table "reqs").
  Alg. 1    -- realistic gap junction (read as the odd form (0.8 e^{-dV^2/100} + 0.2) dV).
  Sec. 3    -- validation: identical cells, a short pulse to all, a complex spike in all.
Cell-model constants are the published three-compartment IO cell; their parity with the
publication is unpinned, so the cell-model pins below check each mechanism against
closed forms of the model's own definition (half-activation points, reversal
potentials, linear invariants, exact solutions of reduced systems).
"""
import math

import numpy as np
import pytest

from paper_1612_01501_gb300 import inputs

DT = 0.05


# ------------------------------------------------------------------ gap junctions

def test_gj_zero_when_all_equal(O):
    vd = np.full(37, -61.25)
    assert np.all(O.gj_dense(vd, 0.3) == 0.0)
    rp, col = inputs.random_symmetric_csr(37, 6, 5)
    assert np.all(O.gj_csr(rp, col, np.full(len(col), 0.7), vd) == 0.0)


def test_gj_two_cell_closed_form(O):
    # dV = 10: (0.8 e^{-1} + 0.2) * 10 = 2 + 8/e
    ic = O.gj_dense(np.array([10.0, 0.0]), 1.0)
    assert ic[0] == pytest.approx(4.943035529371539, rel=1e-15)
    assert ic[1] == -ic[0]                                  # I_ij = -I_ji exactly
    # large dV: e^{-100} vanishes, the current is the linear part 0.2 dV
    ic = O.gj_dense(np.array([100.0, 0.0]), 0.25)
    assert ic[0] == pytest.approx(0.25 * 20.0, rel=1e-15)
    # small dV: slope (0.8 + 0.2) = 1 at the origin
    ic = O.gj_dense(np.array([1e-4, 0.0]), 2.0)
    assert ic[0] == pytest.approx(2.0 * 1e-4, rel=1e-9)


def test_gj_three_cell_closed_form(O):
    # V = (0, 10, 20), g = 0.5: Ic_0 = 0.5 (-(2 + 8/e) - (4 + 16 e^{-4})), Ic_1 = 0, Ic_2 = -Ic_0
    ic = O.gj_dense(np.array([0.0, 10.0, 20.0]), 0.5)
    assert ic[0] == pytest.approx(-4.618042875795643, rel=1e-14)
    assert abs(ic[1]) < 1e-15
    assert ic[2] == pytest.approx(4.618042875795643, rel=1e-14)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_gj_brute_force_tiny(O, n):
    """Brute force over every ordered pair of a 2-4 cell network."""
    vd = inputs.uniform(inputs.stream_seed(n, "bf"), n, -80.0, 20.0)
    g = 0.037
    ref = np.zeros(n)
    for i in range(n):
        for j in range(n):
            d = vd[i] - vd[j]
            ref[i] += g * (0.8 * math.exp(-(d * d) / 100.0) + 0.2) * d
    np.testing.assert_allclose(O.gj_dense(vd, g), ref, rtol=1e-13, atol=1e-15)
    # the same network as an explicit CSR complete graph (no self loops)
    rp = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.int32)
    col = np.array([j for i in range(n) for j in range(n) if j != i], np.int32)
    np.testing.assert_allclose(O.gj_csr(rp, col, np.full(len(col), g), vd), ref, rtol=1e-13, atol=1e-15)


def test_gj_network_sum_vanishes(O):
    """Antisymmetric pair terms + symmetric weights: sum_i Ic_i = 0 up to roundoff."""
    n = 500
    vd = -60.0 + inputs.vdend_jitter(n, 11, 20.0)
    ic = O.gj_dense(vd, 0.01)
    assert abs(ic.sum()) < 1e-12 * np.abs(ic).sum() * n
    rp, col = inputs.random_symmetric_csr(n, 20, 3)
    ic = O.gj_csr(rp, col, np.full(len(col), 0.05), vd)
    assert abs(ic.sum()) < 1e-12 * np.abs(ic).sum() * n


def test_gj_odd_and_linear_in_weight(O):
    vd = -60.0 + inputs.vdend_jitter(50, 4)
    a = O.gj_dense(vd, 0.02)
    b = O.gj_dense(-vd, 0.02)       # flipping every voltage flips every current
    np.testing.assert_allclose(a, -b, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(O.gj_dense(vd, 0.06), 3.0 * a, rtol=1e-14, atol=1e-14)


def test_csr_symmetric_generator():
    rp, col = inputs.random_symmetric_csr(300, 10, 9)
    n = 300
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(col >= 0) and np.all(col < n) and np.all(rows != col)
    pairs = set(zip(rows.tolist(), col.tolist()))
    assert all((j, i) in pairs for i, j in pairs)
    for i in range(n):
        seg = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(seg) > 0)
    assert 8.0 < len(col) / n <= 10.0


# ------------------------------------------------------------------ rate functions

def test_half_activation_points(O):
    G = {g: i for i, g in enumerate(O.GATES)}
    cases = [("m_s", -30.0), ("m_a", -30.0), ("h_s", -70.0), ("h_a", -60.0), ("k", -61.0),
             ("l", -85.5), ("n_s", -3.0), ("q", -80.0)]
    for gate, v in cases:
        xi, _ = O.rates(v, 1.0)
        assert xi[G[gate]] == pytest.approx(0.5, abs=1e-15), gate
    # rising gates rise, falling gates fall
    lo, _ = O.rates(-90.0, 1.0)
    hi, _ = O.rates(20.0, 1.0)
    for gate in ("m_s", "k", "n_s", "r", "x_s", "x_a", "m_a"):
        assert hi[G[gate]] > lo[G[gate]], gate
    for gate in ("h_s", "h_a", "l", "q"):
        assert hi[G[gate]] < lo[G[gate]], gate


def test_time_constants_closed_form(O):
    G = {g: i for i, g in enumerate(O.GATES)}
    for v in (-100.0, -40.0, 30.0):
        assert O.rates(v, 1.0)[1][G["k"]] == 1.0
    assert O.rates(-40.0, 1.0)[1][G["h_s"]] == pytest.approx(3.0, rel=1e-15)
    assert O.rates(-40.0, 1.0)[1][G["h_a"]] == pytest.approx(1.5, rel=1e-15)
    assert O.rates(-50.0, 1.0)[1][G["n_s"]] == pytest.approx(52.0, rel=1e-15)
    # tau_l(-84) = 20 e^{76/30} / 2 + 35
    assert O.rates(-84.0, 1.0)[1][G["l"]] == pytest.approx(160.95420976379947, rel=1e-14)
    # tau_q(-80) = 1 / (e^{6.88-14.6} + e^{-5.6-1.87})
    assert O.rates(-80.0, 1.0)[1][G["q"]] == pytest.approx(986.3986469274646, rel=1e-13)


def test_alpha_beta_gates_closed_form(O):
    G = {g: i for i, g in enumerate(O.GATES)}
    # x gate at V = -25: alpha has a removable singularity with limit 1.3; beta = 1.69 e^{-0.125}
    xi, ta = O.rates(-25.0, 1.0)
    for g in ("x_s", "x_a"):
        assert xi[G[g]] == pytest.approx(0.4657128304845378, rel=1e-14)
        assert ta[G[g]] == pytest.approx(0.3582406388342599, rel=1e-14)
    # x gate at V = -35: alpha = 1.3 / (e - 1), beta = 1.69
    xi, ta = O.rates(-35.0, 1.0)
    assert xi[G["x_s"]] == pytest.approx(0.30923693409438974, rel=1e-14)
    assert ta[G["x_s"]] == pytest.approx(0.4087355419559824, rel=1e-14)
    # r gate at V = -8.5: beta has a removable singularity with limit 0.1
    xi, ta = O.rates(-8.5, 1.0)
    assert xi[G["r"]] == pytest.approx(0.8235966168358252, rel=1e-14)
    assert ta[G["r"]] == pytest.approx(8.82016915820874, rel=1e-14)
    # r gate at V = 5: alpha = 1.7 / 2, beta = 0.27 / (e^{2.7} - 1)
    xi, ta = O.rates(5.0, 1.0)
    assert xi[G["r"]] == pytest.approx(0.9776263588044646, rel=1e-14)
    assert ta[G["r"]] == pytest.approx(5.750743287085085, rel=1e-14)
    # continuity across both singular points
    for v0, g in ((-25.0, "x_s"), (-8.5, "r")):
        a = O.rates(v0 - 1e-7, 1.0)[0][G[g]]
        b = O.rates(v0, 1.0)[0][G[g]]
        c = O.rates(v0 + 1e-7, 1.0)[0][G[g]]
        assert abs(a - b) < 1e-7 and abs(c - b) < 1e-7


def test_calcium_gate_closed_form(O):
    G = {g: i for i, g in enumerate(O.GATES)}
    xi, ta = O.rates(-60.0, 0.0)
    assert xi[G["s"]] == 0.0 and ta[G["s"]] == pytest.approx(1.0 / 0.015, rel=1e-15)
    xi, ta = O.rates(-60.0, 250.0)       # alpha = 0.005
    assert xi[G["s"]] == pytest.approx(0.25, rel=1e-14) and ta[G["s"]] == pytest.approx(50.0, rel=1e-14)
    xi, ta = O.rates(-60.0, 1e4)         # alpha saturates at 0.01
    assert xi[G["s"]] == pytest.approx(0.4, rel=1e-14) and ta[G["s"]] == pytest.approx(40.0, rel=1e-14)


# ------------------------------------------------------------------ cell update

def _model_only(O, keep=(), **override):
    """Model table with every conductance and g_int zeroed except those in `keep`."""
    P = O.model_default()
    for name in ("g_int", "g_CaH", "g_KCa", "g_h", "g_ld", "g_CaL", "g_Na_s", "g_Kdr_s", "g_K_s",
                 "g_ls", "g_Na_a", "g_K_a", "g_la"):
        if name not in keep:
            P[O.P[name]] = 0.0
    for k, v in override.items():
        P[O.P[k]] = v
    return P


def _state(O, n=1, **vals):
    S = O.default_state(n)
    for k, v in vals.items():
        S[O.F[k]] = v
    return S


def test_leak_only_hand_step(O):
    P = _model_only(O, keep=("g_ld", "g_ls", "g_la"))
    S = _state(O, V_dend=-60.0, V_soma=-60.0, V_axon=-60.0, g_CaL=0.0)
    Sn = O.cell_step(S, model=P)
    # dV/dt = -0.016 (V - 10) = 1.12 mV/ms; V' = -60 + 0.05 * 1.12
    for f in ("V_dend", "V_soma", "V_axon"):
        assert Sn[O.F[f], 0] == pytest.approx(-59.944, abs=1e-13)


def test_coupling_only_is_jacobi_and_conservative(O):
    P = _model_only(O, keep=("g_int",))
    S = _state(O, V_dend=10.0, V_soma=0.0, V_axon=0.0, g_CaL=0.0)
    Sn = O.cell_step(S, model=P)
    assert Sn[O.F["V_dend"], 0] == pytest.approx(9.913333333333334, abs=1e-14)   # 10 - 0.05 (0.13/0.75) 10
    assert Sn[O.F["V_soma"], 0] == pytest.approx(0.26, abs=1e-14)                # 0.05 (0.13/0.25) 10
    assert Sn[O.F["V_axon"], 0] == 0.0      # uses the step-t soma voltage (0), not the new one
    # Q = (1-p1) V_d + p1 V_s + p1 p2/(1-p2) V_a is conserved; all voltages reach Q / sum(weights)
    w = np.array([0.75, 0.25, 0.25 * 0.15 / 0.85])
    Sf, _ = O.run(S, 20000, kind=O.NOGJ, model=P)
    V = Sf[[O.F["V_dend"], O.F["V_soma"], O.F["V_axon"]], 0]
    assert w @ V == pytest.approx(7.5, abs=1e-11)
    np.testing.assert_allclose(V, 7.183098591549295, atol=1e-9)


def test_channel_hand_values(O):
    # delayed-rectifier K alone: V_s = 0, n = 0.5: I = 9 * 0.5^4 * 75 = 42.1875
    P = _model_only(O, keep=("g_Kdr_s",))
    Sn = O.cell_step(_state(O, V_soma=0.0, n_s=0.5, g_CaL=0.0), model=P)
    assert Sn[O.F["V_soma"], 0] == pytest.approx(-2.109375, abs=1e-13)
    # soma Na alone, h = 1, V_s = 0: I = 150 m_inf(0)^3 (0 - 55), m_inf(0) = 1/(1+e^{-30/5.5})
    P = _model_only(O, keep=("g_Na_s",))
    Sn = O.cell_step(_state(O, V_soma=0.0, h_s=1.0, g_CaL=0.0), model=P)
    assert Sn[O.F["V_soma"], 0] == pytest.approx(407.2523848855162, rel=1e-13)
    assert Sn[O.F["m_s"], 0] == pytest.approx(0.9957413929480899, rel=1e-14)
    # high-threshold Ca alone: V_d = 0, r = 0.5, [Ca] = 1: I_CaH = 4.5 * 0.25 * (0 - 120) = -135
    P = _model_only(O, keep=("g_CaH",))
    Sn = O.cell_step(_state(O, V_dend=0.0, r=0.5, Ca=1.0, g_CaL=0.0), model=P)
    assert Sn[O.F["I_CaH"], 0] == pytest.approx(-135.0, abs=1e-12)
    assert Sn[O.F["V_dend"], 0] == pytest.approx(0.05 * 135.0, abs=1e-12)
    assert Sn[O.F["Ca"], 0] == pytest.approx(1.0 + 0.05 * (3.0 * 135.0 - 0.075), abs=1e-12)


@pytest.mark.parametrize("chan,comp,vrev,gate", [
    ("g_CaH", "V_dend", 120.0, {"r": 0.5}), ("g_KCa", "V_dend", -75.0, {"s": 0.5}),
    ("g_h", "V_dend", -43.0, {"q": 0.5}), ("g_ld", "V_dend", 10.0, {}),
    ("g_CaL", "V_soma", 120.0, {"k": 0.5, "l": 0.5}), ("g_Na_s", "V_soma", 55.0, {"h_s": 0.5}),
    ("g_Kdr_s", "V_soma", -75.0, {"n_s": 0.5}), ("g_K_s", "V_soma", -75.0, {"x_s": 0.5}),
    ("g_ls", "V_soma", 10.0, {}), ("g_Na_a", "V_axon", 55.0, {"h_a": 0.5}),
    ("g_K_a", "V_axon", -75.0, {"x_a": 0.5}), ("g_la", "V_axon", 10.0, {})])
def test_each_current_vanishes_at_its_reversal(O, chan, comp, vrev, gate):
    P = _model_only(O, keep=(chan,))
    vals = {"V_dend": 0.0, "V_soma": 0.0, "V_axon": 0.0, comp: vrev, **gate}
    vals["g_CaL"] = 0.68 if chan == "g_CaL" else 0.0
    S = _state(O, **vals)
    Sn = O.cell_step(S, model=P)
    assert Sn[O.F[comp], 0] == S[O.F[comp], 0]
    # and away from it the current drives V towards the reversal potential
    vals[comp] = vrev - 7.0
    S = _state(O, **vals)
    assert O.cell_step(S, model=P)[O.F[comp], 0] > vrev - 7.0


def test_gate_relaxation_closed_form(O):
    """With every conductance off V is constant and each gate follows the linear
    recurrence x_{n+1} = x_n + dt (x_inf - x_n) / tau, i.e. x_n = x_inf (1 - (1 - dt/tau)^n)."""
    P = _model_only(O, ca_out=0.0)      # and [Ca] held constant (no decay, no influx)
    S = _state(O, V_dend=-52.0, V_soma=-47.0, V_axon=-65.0, Ca=2.5, g_CaL=0.0)
    for g in ("r", "s", "q", "k", "l", "h_s", "n_s", "x_s", "h_a", "x_a"):
        S[O.F[g]] = 0.0
    n = 150
    Sf, _ = O.run(S, n, kind=O.NOGJ, model=P)
    comp = {"r": -52.0, "s": -52.0, "q": -52.0, "k": -47.0, "l": -47.0, "h_s": -47.0, "n_s": -47.0,
            "x_s": -47.0, "h_a": -65.0, "x_a": -65.0}
    G = {g: i for i, g in enumerate(O.GATES)}
    for g, v in comp.items():
        xi, ta = O.rates(v, 2.5)
        want = xi[G[g]] * (1.0 - (1.0 - DT / ta[G[g]]) ** n)
        assert Sf[O.F[g], 0] == pytest.approx(want, rel=1e-11, abs=1e-15), g


def test_calcium_decay_closed_form(O):
    P = _model_only(O)         # g_CaH = 0, so I_CaH = 0: pure decay [Ca]_n = [Ca]_0 (1 - 0.075 dt)^n
    S = _state(O, V_dend=-60.0, V_soma=-60.0, V_axon=-60.0, Ca=5.0, r=0.3, g_CaL=0.0)
    Sf, _ = O.run(S, 400, kind=O.NOGJ, model=P)
    assert Sf[O.F["Ca"], 0] == pytest.approx(5.0 * (1.0 - 0.075 * DT) ** 400, rel=1e-12)


def test_gap_current_enters_as_outward_dendritic_current(O):
    """A coupled step equals the uncoupled step with I_app lowered by I_c (sign and
    placement of the gap current); all fields but the stored I_c agree."""
    n = 4
    S = O.default_state(n)
    S[O.F["V_dend"]] += np.array([-3.0, 1.0, 4.0, -0.5])
    ic = O.gj_dense(S[O.F["V_dend"]], 0.05)
    iapp = np.array([0.0, 2.0, 0.0, 1.0])
    a = O.cell_step(S, ic=ic, iapp=iapp)
    b = O.cell_step(S, ic=None, iapp=iapp - ic)
    keep = [f for f in range(O.NF) if f != O.F["I_c"]]
    np.testing.assert_allclose(a[keep], b[keep], rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal(a[O.F["I_c"]], ic)
    # two cells at different V_dend, no ionic currents: coupling pulls them together
    P = _model_only(O)
    S2 = _state(O, 2, V_dend=np.array([-50.0, -70.0]), g_CaL=0.0)
    Sf, _ = O.run(S2, 200, kind=O.DENSE, g=0.05, model=P)
    d0 = 20.0
    d1 = Sf[O.F["V_dend"], 0] - Sf[O.F["V_dend"], 1]
    assert 0.0 < d1 < d0
    assert Sf[O.F["V_dend"]].sum() == pytest.approx(-120.0, abs=1e-10)


def test_default_state_high_threshold_calcium_current(O):
    """The default state's I_CaH is the dendritic high-threshold Ca current of the resting
    state: g_CaH r_inf(-60)^2 (V_0 - V_Ca) = 4.5 r^2 (-60 - 120).  At -60 mV the r gate's
    alpha = 1.7 / (1 + e^{65/13.9}) = 0.0156873... and its beta (0.02 (V + 8.5) over
    e^{(V + 8.5)/5} - 1, here -1.03 / (e^{-10.3} - 1)) = 1.0300346..., so r_inf = 0.0150014...
    and I_CaH = -0.182285 uA/cm^2 (worked out by hand to six figures)."""
    S = O.default_state(3)
    r = S[O.F["r"], 0]
    assert r == pytest.approx(0.0150014, abs=5e-8)
    assert np.all(S[O.F["I_CaH"]] == pytest.approx(-0.182285, abs=5e-7))
    P = O.model_default()
    assert S[O.F["I_CaH"], 0] == pytest.approx(P[O.P["g_CaH"]] * r * r * (P[O.P["V_0"]] - P[O.P["V_Ca"]]), rel=1e-15)
    assert np.all(S[O.F["I_c"]] == 0.0)


# ------------------------------------------------------------------ network invariants

def test_identical_cells_stay_identical(O):
    n = 12
    S = O.default_state(n)
    pul = inputs.pulses(np.arange(n), 5.0, 15.0, 6.0)
    for kind, g in ((O.NOGJ, 0.0), (O.DENSE, 0.04)):
        Sf, tr = O.run(S, 1000, kind=kind, g=g, pulses=pul, trace_cells=np.arange(n))
        assert np.all(Sf == Sf[:, :1]), kind
        assert np.all(tr == tr[:, :1])


def test_openmp_is_bitwise_serial(O):
    n = 96
    S = O.default_state(n)
    S[O.F["V_dend"]] += inputs.vdend_jitter(n, 3)
    a, _ = O.run(S, 50, kind=O.DENSE, g=0.01, threads=1)
    b, _ = O.run(S, 50, kind=O.DENSE, g=0.01, threads=4)
    np.testing.assert_array_equal(a, b)


def test_c1_gates_stay_in_unit_interval(O):
    cfg = inputs.config("c1")
    S = O.default_state(cfg["n"])
    S[O.F["V_dend"]] += cfg["jitter"]
    S = S.astype(np.float32).astype(np.float64)
    gates = [O.F[g] for g in ("r", "s", "q", "k", "l", "m_s", "h_s", "n_s", "x_s", "m_a", "h_a", "x_a")]
    t = 0
    for _ in range(40):          # the full 1 s in chunks of 500 steps
        S, _ = O.run(S, 500, kind=O.DENSE, g=cfg["g"], t0=t, pulses=cfg["pulses"], threads=4)
        t += 500
        assert np.all(S[gates] >= 0.0) and np.all(S[gates] <= 1.0)
        assert np.all(np.isfinite(S))


def test_validation_experiment_complex_spike_in_every_cell(O):
    """Sec. 3: identical initial states and a pulse to every cell for about 500 steps
    give a complex spike in every cell, all in step (synchronous)."""
    cfg = inputs.config("validation")
    n = cfg["n"]
    S = O.default_state(n)
    Sf, tr = O.run(S, 4000, kind=O.DENSE, g=cfg["g"], pulses=cfg["pulses"], trace_cells=np.arange(n),
                   threads=4)
    sp = [O.spike_steps(tr[:, c]) for c in range(n)]
    assert all(len(s) >= 2 for s in sp)                     # a burst: several spikes per cell
    assert all(np.array_equal(s, sp[0]) for s in sp)        # all cells in step
    assert sp[0][0] >= 2000                                  # not before the pulse onset


# ---- simplified gap junctions (SGJ use case, Sec. 2.3.2): w (V_i - V_j) per connection

def test_sgj_two_cells_by_hand(O):
    ic = O.gj_dense_sgj(np.array([-60.0, -50.0]), 0.1)
    np.testing.assert_allclose(ic, [-1.0, 1.0], rtol=0, atol=1e-12)


def test_sgj_dense_closed_form_and_zero_sum(O):
    rng = np.random.default_rng(3)
    vd = rng.uniform(-70, -40, 257)
    g = 0.013
    ic = O.gj_dense_sgj(vd, g)
    np.testing.assert_allclose(ic, g * (len(vd) * vd - vd.sum()), rtol=0, atol=1e-9)
    assert abs(ic.sum()) <= 1e-9 * g * np.abs(vd).sum() * len(vd)


def test_sgj_is_the_small_dv_limit_of_rgj(O):
    """The RGJ term (0.8 e^{-dV^2/100} + 0.2) dV tends to dV: for |dV| <= 1e-3 mV the two
    junction forms agree to 1e-7 relative (the next term is 0.008 dV^3)."""
    rng = np.random.default_rng(4)
    vd = -60.0 + rng.uniform(-1e-3, 1e-3, 64)
    a = O.gj_dense(vd, 0.02)
    b = O.gj_dense_sgj(vd, 0.02)
    assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max()


def test_sgj_csr_complete_graph_equals_dense_and_conserves(O):
    n = 40
    rp = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.int32)
    col = np.array([j for i in range(n) for j in range(n) if j != i], np.int32)
    vd = np.random.default_rng(5).uniform(-65, -45, n)
    a = O.gj_csr_sgj(rp, col, np.full(len(col), 0.03), vd)
    np.testing.assert_allclose(a, O.gj_dense_sgj(vd, 0.03), rtol=0, atol=1e-12)
    rp2, col2 = inputs.random_symmetric_csr(500, 12, 6)
    vd2 = np.random.default_rng(6).uniform(-65, -45, 500)
    ic = O.gj_csr_sgj(rp2, col2, np.full(len(col2), 0.05), vd2)
    assert abs(ic.sum()) <= 1e-10 * np.abs(ic).sum()


def test_sgj_run_uses_the_linear_junction(O):
    """One step of kind DENSE_SGJ equals the cell update fed with the SGJ current."""
    n = 30
    S = O.default_state(n)
    S[O.F["V_dend"]] += np.linspace(-5, 5, n)
    ref = O.cell_step(S, ic=O.gj_dense_sgj(S[O.F["V_dend"]], 0.02))
    got, _ = O.run(S, 1, kind=O.DENSE_SGJ, g=0.02)
    np.testing.assert_array_equal(got, ref)


# ---- dense N x N weight matrix (programmed connectivity with every pair stored, Sec. 2.3)

def test_matrix_uniform_equals_dense_uniform(O):
    vd = np.random.default_rng(7).uniform(-70, -40, 123)
    W = np.full((123, 123), 0.017)
    np.testing.assert_allclose(O.gj_matrix(W, vd), O.gj_dense(vd, 0.017), rtol=1e-13, atol=1e-13)


def test_matrix_equals_weighted_complete_csr(O):
    """Any matrix equals the CSR of the complete graph with the same off-diagonal weights
    (the diagonal pair contributes exactly zero whatever its weight)."""
    n = 60
    rng = np.random.default_rng(8)
    W = rng.uniform(0.0, 0.1, (n, n))
    vd = rng.uniform(-70, -40, n)
    rp = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.int32)
    col = np.array([j for i in range(n) for j in range(n) if j != i], np.int32)
    w = np.array([W[i, j] for i in range(n) for j in range(n) if j != i])
    np.testing.assert_allclose(O.gj_matrix(W, vd), O.gj_csr(rp, col, w, vd), rtol=1e-13, atol=1e-13)


def test_matrix_two_cells_by_hand_and_symmetric_conservation(O):
    W = np.array([[5.0, 0.3], [0.7, 9.0]])
    vd = np.array([-60.0, -50.0])
    t = (0.8 * np.exp(-1.0) + 0.2) * 10.0        # term(+10); term(-10) = -t
    np.testing.assert_allclose(O.gj_matrix(W, vd), [-0.3 * t, 0.7 * t], rtol=1e-14)
    rng = np.random.default_rng(9)
    A = rng.uniform(0, 0.05, (80, 80))
    ic = O.gj_matrix(A + A.T, rng.uniform(-70, -40, 80))
    assert abs(ic.sum()) <= 1e-12 * np.abs(ic).sum()


# ------------------------------------------------------------------ per-cell constants

def _per_cell_tables(O, n, seed):
    """n model tables whose per-cell entries (0..19) are the defaults scaled by U(0.7, 1.3)
    (conductances and area ratios) or shifted by U(-3, 3) mV (reversal potentials)."""
    rng = np.random.default_rng(seed)
    base = O.model_default()
    tabs = np.repeat(base[None, :], n, axis=0)
    for p in range(O.NCELLPARAMS):
        if O.PARAMS[p].startswith("V_"):
            tabs[:, p] += rng.uniform(-3.0, 3.0, n)
        else:
            tabs[:, p] *= rng.uniform(0.7, 1.3, n)
    return tabs


def test_per_cell_constants_equal_to_the_table_change_nothing(O):
    n = 40
    cfg = inputs.config("c1")
    S = O.default_state(n)
    S[O.F["V_dend"]] += inputs.vdend_jitter(n, 4)
    cp = np.repeat(O.model_default()[:O.NCELLPARAMS, None], n, axis=1)
    a, _ = O.run(S, 200, kind=O.DENSE, g=0.01, pulses=inputs.pulses(np.arange(8), 2.0, 6.0, 6.0))
    b, _ = O.run(S, 200, kind=O.DENSE, g=0.01, pulses=inputs.pulses(np.arange(8), 2.0, 6.0, 6.0), cell_params=cp)
    np.testing.assert_array_equal(a, b)


def test_per_cell_constants_equal_one_table_per_cell(O):
    """Uncoupled cells with per-cell constants evolve exactly as each cell run alone with a
    model table holding its constants (brute force over the cells; catches a transposed or
    shifted per-cell layout)."""
    n = 9
    tabs = _per_cell_tables(O, n, 11)
    S = O.default_state(n)
    S[O.F["V_dend"]] += inputs.vdend_jitter(n, 5)
    S[O.F["g_CaL"]] = np.linspace(0.5, 1.1, n)
    pul = inputs.pulses(np.arange(n), 1.0, 4.0, 6.0)
    cp = tabs[:, :O.NCELLPARAMS].T.copy()
    cp[O.P["g_CaL"]] = 1e9            # never read: g_CaL comes from the state
    got, _ = O.run(S, 300, kind=O.NOGJ, pulses=pul, cell_params=cp)
    for i in range(n):
        ref, _ = O.run(S[:, i:i + 1], 300, kind=O.NOGJ, model=tabs[i],
                       pulses=inputs.pulses(np.array([0]), 1.0, 4.0, 6.0))
        np.testing.assert_array_equal(got[:, i], ref[:, 0])


def test_per_cell_leak_conductance_hand_step(O):
    """A leak-only cell whose own g_ld is doubled: one step moves V_dend twice as far
    towards V_L as in a cell with the table's g_ld (by hand: 0.05 * 0.016 * 70 = 0.056 mV)."""
    P = _model_only(O, keep=("g_ld",))
    S = _state(O, 2, V_dend=-60.0, V_soma=-60.0, V_axon=-60.0, g_CaL=0.0)
    cp = np.repeat(P[:O.NCELLPARAMS, None], 2, axis=1)
    cp[O.P["g_ld"], 1] *= 2.0
    Sn = O.cell_step(S, model=P, cell_params=cp)
    assert Sn[O.F["V_dend"], 0] == pytest.approx(-59.944, abs=1e-13)
    assert Sn[O.F["V_dend"], 1] == pytest.approx(-59.888, abs=1e-13)
