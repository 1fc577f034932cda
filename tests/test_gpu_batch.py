"""Batched networks (one launch per step over many networks) against the FP64 oracle run
of each network alone, plus the autotuner (it must leave the simulation untouched)."""
import numpy as np
import pytest

from paper_1612_01501_gb300 import inputs
from paper_1612_01501_gb300 import ion

from helpers import STEP_RTOL, TRAJ_MV, csr_abs_scale, step_rel_err, sum_abs_dv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01501_gb300 import build
    build.build()
    return torch


def _nets(specs):
    out = []
    for sp in specs:
        b = inputs.batch_network(sp)
        b["spec"] = sp
        out.append(b)
    return out


def _batch_inputs(O, nets):
    """Concatenated FP32 initial state and pulse table in the batch's cell numbering."""
    states, cells, beg, end, amp = [], [], [], [], []
    off = 0
    for b in nets:
        S = O.default_state(b["n"])
        S[O.F["V_dend"]] += b["jitter"]
        states.append(S.astype(np.float32))
        p = b["pulses"]
        cells.append(p[0] + off)
        beg.append(p[1]); end.append(p[2]); amp.append(p[3])
        off += b["n"]
    S0 = np.concatenate(states, axis=1)
    pul = (np.concatenate(cells).astype(np.int32), np.concatenate(beg), np.concatenate(end), np.concatenate(amp))
    return S0, pul


def _ion_nets(nets):
    out = []
    for b in nets:
        if b["kind"] == "dense":
            out.append(dict(n=b["n"], kind=ion.DENSE_UNIFORM, g=b["g"]))
        elif b["kind"] == "csr":
            out.append(dict(n=b["n"], kind=ion.CSR, row_ptr=b["row_ptr"], col=b["col"], w=b["w"]))
        else:
            out.append(dict(n=b["n"], kind=ion.NO_GJ))
    return out


def _oracle_net(O, b, S0, steps, pulses):
    kind = {"dense": O.DENSE, "csr": O.CSR, "nogj": O.NOGJ}[b["kind"]]
    return O.run(S0.astype(np.float64), steps, kind=kind, g=b.get("g", 0.0), row_ptr=b.get("row_ptr"),
                 col=b.get("col"), w=None if b.get("w") is None else b["w"].astype(np.float64), pulses=pulses,
                 threads=max(1, O.max_threads()))[0]


def _mixed_specs():
    return [dict(n=37, kind="dense", k=37, g_ref=0.03, seed=5), dict(n=300, kind="csr", k=12, g_ref=0.05, seed=6),
            dict(n=1000, kind="dense", k=1000, g_ref=0.08, seed=7), dict(n=257, kind="csr", k=100, g_ref=0.02, seed=8),
            dict(n=4096, kind="dense", k=4096, g_ref=0.01, seed=9), dict(n=33, kind="csr", k=8, g_ref=0.04, seed=10)]


def test_batch_matches_each_network_alone(cuda, O):
    nets = _nets(_mixed_specs())
    S0, pul = _batch_inputs(O, nets)
    with_h = ion.ion_create_batch(_ion_nets(nets), init_state=S0)
    try:
        ion.ion_set_input(with_h, pul)
        ion.ion_step(with_h, 600)            # pulses at 20-30 ms = steps 400..600
        got = ion.ion_read_state(with_h, S0.shape[1])
    finally:
        ion.ion_destroy(with_h)
    off = 0
    for b in nets:
        n = b["n"]
        ref = _oracle_net(O, b, S0[:, off:off + n], 600, b["pulses"])
        assert np.abs(got[:3, off:off + n] - ref[:3]).max() <= TRAJ_MV, (b["spec"], np.abs(got[:3, off:off + n] - ref[:3]).max())
        off += n


@pytest.mark.parametrize("layout", ["compact", "random_weights", "as_given"])
def test_batch_one_step_error(cuda, O, layout):
    """One step of every network from an identical state.  CSR networks run in the compact
    layout (16-bit local columns, V_dend staged in shared memory, one scalar weight), with
    random per-edge weights (compact columns, weight array), or as given (32-bit columns)."""
    nets = _nets(_mixed_specs())
    if layout == "random_weights":
        for b in nets:
            if b["kind"] == "csr":
                u = inputs.uniform(inputs.stream_seed(b["n"], "edge_w"), len(b["w"]), 0.5, 1.5)
                b["w"] = (b["w"] * u).astype(np.float32)
    S0, pul = _batch_inputs(O, nets)
    flags = ion.FLAG_KAHAN | (ion.FLAG_CSR_AS_GIVEN if layout == "as_given" else 0)
    h = ion.ion_create_batch(_ion_nets(nets), init_state=S0, flags=flags)
    try:
        ion.ion_step(h, 1)
        got = ion.ion_read_state(h, S0.shape[1])
    finally:
        ion.ion_destroy(h)
    off = 0
    for b in nets:
        n = b["n"]
        ref = _oracle_net(O, b, S0[:, off:off + n], 1, None)
        if b["kind"] == "dense":
            scale = b["g"] * sum_abs_dv(S0[0, off:off + n])
        else:
            scale = csr_abs_scale(b["row_ptr"], b["col"], b["w"], S0[0, off:off + n])
        err = step_rel_err(got[:, off:off + n], ref, scale)
        assert err.max() <= STEP_RTOL, (b["spec"], err.max(axis=1))
        off += n


def _c4_spread(nets, per_kind=16):
    """Indices of `per_kind` dense and `per_kind` CSR networks of the 256-network batch at
    evenly spaced size ranks (smallest and largest of each kind included)."""
    pick = []
    for kind in ("dense", "csr"):
        idx = sorted((i for i, b in enumerate(nets) if b["kind"] == kind), key=lambda i: nets[i]["n"])
        ranks = np.unique(np.round(np.linspace(0, len(idx) - 1, per_kind)).astype(int))
        pick += [idx[r] for r in ranks]
    return pick


def test_c4_all_256_networks_one_step(cuda, O):
    """One step of every network of the 256-network batch from an identical FP32 state,
    each against the oracle run of that network alone (per-step relative error bar)."""
    nets = _nets(inputs.batch_specs())
    S0, pul = _batch_inputs(O, nets)
    h = ion.ion_create_batch(_ion_nets(nets), init_state=S0, graph_steps=50)
    try:
        ion.ion_step(h, 1)
        got = ion.ion_read_state(h, S0.shape[1])
    finally:
        ion.ion_destroy(h)
    offs = np.concatenate([[0], np.cumsum([b["n"] for b in nets])])
    worst = 0.0
    for i, b in enumerate(nets):
        sl = slice(offs[i], offs[i + 1])
        ref = _oracle_net(O, b, S0[:, sl], 1, None)
        if b["kind"] == "dense":
            scale = b["g"] * sum_abs_dv(S0[0, sl])
        else:
            scale = csr_abs_scale(b["row_ptr"], b["col"], b["w"], S0[0, sl])
        err = step_rel_err(got[:, sl], ref, scale)
        assert err.max() <= STEP_RTOL, (i, b["spec"], err.max(axis=1))
        worst = max(worst, float(err.max()))
    print(f"256 networks, one step: worst relative error {worst:.2e}")


def test_c4_trajectories_100ms_on_32_networks(cuda, O):
    """The whole batch for 100 ms (2000 steps, pulses at 20-30 ms) in graph replays;
    16 dense and 16 CSR networks spanning the size range stay within 0.1 mV of their
    oracle runs at every 25 ms checkpoint."""
    nets = _nets(inputs.batch_specs())
    S0, pul = _batch_inputs(O, nets)
    offs = np.concatenate([[0], np.cumsum([b["n"] for b in nets])])
    pick = _c4_spread(nets)
    assert len(pick) == 32
    refs = {i: S0[:, offs[i]:offs[i + 1]].astype(np.float64) for i in pick}
    h = ion.ion_create_batch(_ion_nets(nets), init_state=S0, graph_steps=50)
    worst = 0.0
    try:
        ion.ion_set_input(h, pul)
        t = 0
        for _ in range(4):
            ion.ion_step(h, 500)
            got = ion.ion_read_state(h, S0.shape[1])
            assert np.all(np.isfinite(got))
            for i in pick:
                b = nets[i]
                kind = {"dense": O.DENSE, "csr": O.CSR}[b["kind"]]
                refs[i], _ = O.run(refs[i], 500, kind=kind, g=b.get("g", 0.0), row_ptr=b.get("row_ptr"),
                                   col=b.get("col"), w=None if b.get("w") is None else b["w"].astype(np.float64),
                                   t0=t, pulses=b["pulses"], threads=max(1, O.max_threads()))
                d = np.abs(got[:3, offs[i]:offs[i + 1]] - refs[i][:3]).max()
                assert d <= TRAJ_MV, (t + 500, i, b["spec"], d)
                worst = max(worst, float(d))
            t += 500
    finally:
        ion.ion_destroy(h)
    print(f"32 networks over 100 ms: worst |dV| {worst:.2e} mV")


def test_autotune_leaves_state_untouched_and_results_agree(cuda, O):
    nets = _nets(_mixed_specs())
    S0, pul = _batch_inputs(O, nets)
    h = ion.ion_create_batch(_ion_nets(nets), init_state=S0)
    try:
        ion.ion_set_input(h, pul)
        ion.ion_step(h, 10)
        before = ion.ion_read_state(h, S0.shape[1])
        table = ion.ion_autotune(h, 5)
        assert ion.ion_step_count(h) == 10
        np.testing.assert_array_equal(ion.ion_read_state(h, S0.shape[1]), before)
        assert table["dense_rows_per_warp"] in (1, 2, 4, 8) and 1 <= table["csr_rows_per_cta"] <= 256
        ion.ion_step(h, 590)
        got = ion.ion_read_state(h, S0.shape[1])
    finally:
        ion.ion_destroy(h)
    off = 0
    for b in nets:
        n = b["n"]
        ref = _oracle_net(O, b, S0[:, off:off + n], 600, b["pulses"])
        assert np.abs(got[:3, off:off + n] - ref[:3]).max() <= TRAJ_MV
        off += n


@pytest.mark.parametrize("kind", ["dense", "csr", "csr_large"])
def test_autotune_single_network(cuda, O, kind):
    """The autotuner on one network leaves it untouched and the tuned shape stays exact.
    csr_large: V_dend staging takes more than 48 KB of shared memory (every lanes-per-row
    candidate of the staged kernel must be allowed it)."""
    n = 20000 if kind == "csr_large" else 4000
    if kind == "dense":
        kw = dict(kind=ion.DENSE_UNIFORM, g=inputs.junction_weight(0.04, n))
    else:
        rp, col = inputs.random_symmetric_csr(n, 60, 4)
        kw = dict(kind=ion.CSR, row_ptr=rp, col=col, w=np.full(len(col), inputs.junction_weight(0.04, 60), np.float32))
    S0 = O.default_state(n)
    S0[0] += inputs.vdend_jitter(n, 4)
    S0 = S0.astype(np.float32)
    sim = ion.Simulation(n, init_state=S0, **kw)
    try:
        table = ion.ion_autotune(sim.h, 5)
        assert sim.t == 0
        np.testing.assert_array_equal(sim.state(), S0)
        sim.step(100)
        got = sim.state()
    finally:
        sim.close()
    assert any(v != 0 for v in table.values())
    b = dict(kind="dense" if kind == "dense" else "csr", g=kw.get("g", 0.0), row_ptr=kw.get("row_ptr"),
             col=kw.get("col"), w=kw.get("w"))
    ref = _oracle_net(O, b, S0, 100, None)
    assert np.abs(got[:3] - ref[:3]).max() <= TRAJ_MV


# ------------------------------------------------------------------ persistent batches

def test_persistent_batch_bitwise_equals_step_launches(cuda, O):
    """One cooperative launch per ion_step call (pieces dealt to resident CTAs, per-network
    arrival counters) gives the per-step launches' states bit for bit, with pulses, over
    several calls of different lengths."""
    nets = _nets(_mixed_specs())
    S0, pul = _batch_inputs(O, nets)
    out = []
    for flags in (ion.FLAG_KAHAN, ion.FLAG_KAHAN | ion.FLAG_PERSISTENT):
        h = ion.ion_create_batch(_ion_nets(nets), init_state=S0, flags=flags, graph_steps=50)
        try:
            ion.ion_set_input(h, pul)
            for k in (1, 299, 300, 7):
                ion.ion_step(h, k)
            out.append(ion.ion_read_state(h, S0.shape[1]))
            launches = ion.ion_launch_count(h)
        finally:
            ion.ion_destroy(h)
    np.testing.assert_array_equal(out[0], out[1])
    assert launches == 8      # a kernel and a counter advance per call


@pytest.mark.parametrize("R", [1, 2, 4])
def test_persistent_batch_shapes_one_step(cuda, O, R):
    """One step of the mixed batch through the persistent kernel at each dense row count,
    against the oracle (per-step bar)."""
    nets = _nets(_mixed_specs())
    S0, _ = _batch_inputs(O, nets)
    h = ion.ion_create_batch(_ion_nets(nets), init_state=S0, flags=ion.FLAG_KAHAN | ion.FLAG_PERSISTENT,
                             tune=dict(dense_rows_per_warp=R))
    try:
        ion.ion_step(h, 1)
        got = ion.ion_read_state(h, S0.shape[1])
    finally:
        ion.ion_destroy(h)
    off = 0
    for b in nets:
        n = b["n"]
        ref = _oracle_net(O, b, S0[:, off:off + n], 1, None)
        scale = b["g"] * sum_abs_dv(S0[0, off:off + n]) if b["kind"] == "dense" else \
            csr_abs_scale(b["row_ptr"], b["col"], b["w"], S0[0, off:off + n])
        err = step_rel_err(got[:, off:off + n], ref, scale)
        assert err.max() <= STEP_RTOL, (R, b["spec"], err.max(axis=1))
        off += n


def test_persistent_c4_all_256_networks(cuda, O):
    """The 256-network batch in the persistent form: 100 steps equal the per-step launches
    bit for bit, and one step of every network meets the per-step bar against the oracle."""
    nets = _nets(inputs.batch_specs())
    S0, pul = _batch_inputs(O, nets)
    res = []
    for flags in (ion.FLAG_KAHAN, ion.FLAG_KAHAN | ion.FLAG_PERSISTENT):
        h = ion.ion_create_batch(_ion_nets(nets), init_state=S0, flags=flags, graph_steps=50)
        try:
            ion.ion_step(h, 1)
            one = ion.ion_read_state(h, S0.shape[1])
            ion.ion_set_input(h, pul)
            ion.ion_step(h, 100)
            res.append((one, ion.ion_read_state(h, S0.shape[1])))
        finally:
            ion.ion_destroy(h)
    np.testing.assert_array_equal(res[0][1], res[1][1])
    got = res[1][0]
    offs = np.concatenate([[0], np.cumsum([b["n"] for b in nets])])
    for i, b in enumerate(nets):
        sl = slice(offs[i], offs[i + 1])
        ref = _oracle_net(O, b, S0[:, sl], 1, None)
        scale = b["g"] * sum_abs_dv(S0[0, sl]) if b["kind"] == "dense" else \
            csr_abs_scale(b["row_ptr"], b["col"], b["w"], S0[0, sl])
        err = step_rel_err(got[:, sl], ref, scale)
        assert err.max() <= STEP_RTOL, (i, b["spec"], err.max(axis=1))


def test_persistent_batch_wait_timeout_is_reported(cuda, O):
    """CTA 0 sleeps 200 ms before its first piece while a wait is bounded by 1 ms: the
    CTAs waiting for its network's arrivals give up, raise the abort word and return; the
    host sees ION_ERR_TIMEOUT and the context stays usable."""
    specs = [dict(n=4096, kind="dense", k=4096, g_ref=0.02, seed=31), dict(n=2000, kind="dense", k=2000,
                                                                           g_ref=0.02, seed=32)]
    nets = _nets(specs)
    S0, _ = _batch_inputs(O, nets)
    h = ion.ion_create_batch(_ion_nets(nets), init_state=S0, flags=ion.FLAG_KAHAN | ion.FLAG_PERSISTENT,
                             barrier_timeout_ns=1_000_000, debug_delay_ns=200_000_000)
    try:
        ion.ion_step(h, 5)
        with pytest.raises(ion.IonError) as ei:
            ion.ion_sync(h)
        assert ei.value.status == ion.ERR_TIMEOUT
    finally:
        ion.ion_destroy(h)
    h = ion.ion_create_batch(_ion_nets(nets), init_state=S0, flags=ion.FLAG_KAHAN | ion.FLAG_PERSISTENT)
    try:
        ion.ion_step(h, 5)
        ion.ion_sync(h)
    finally:
        ion.ion_destroy(h)
