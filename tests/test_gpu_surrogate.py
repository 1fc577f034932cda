"""Learned surrogate of the rate functions: GPU training kernels against the FP64 MLP
oracle (gradients), tensor-core inference against an FP64 forward pass, the trained
network against the exact rate functions, and a simulation with learned rates against the
exact FP32 method (trace and spike-time error are reported, with loose bounds)."""
import numpy as np
import pytest

from oracle import mlp
from paper_1612_01501_gb300 import inputs
from paper_1612_01501_gb300 import ion

pytestmark = pytest.mark.gpu
CA_RANGE = (1.36, 13.5)       # the [Ca] seen in 1 s of the 64-cell network, widened x0.5 / x2


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01501_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def trained(cuda):
    w, loss = ion.ion_surrogate_train(n_samples=1 << 20, epochs=100, batch=2048, lr=2e-3, seed=7, v_lo=-100.0,
                                      v_hi=50.0, ca_lo=CA_RANGE[0], ca_hi=CA_RANGE[1])
    print(f"surrogate training: final normalised loss {loss:.3e}")
    return w, loss


@pytest.mark.parametrize("B", [128, 300])
def test_training_gradients_match_fp64_oracle(cuda, B):
    rng = np.random.default_rng(B)
    p = mlp.init_params(5, scale=1.5)
    x = rng.uniform(-1, 1, (B, 2)).astype(np.float32)
    t = rng.normal(0, 1, (B, 24)).astype(np.float32)
    mask = np.ones(24, np.float32)
    mask[[11, 19]] = 0.0
    w = ion.weights_from_dict({k: v.astype(np.float32) for k, v in p.items()})
    L, g = ion.ion_surrogate_grad(w, x, t, mask)
    p32 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    Lr, gr = mlp.loss_and_grads(p32, x.astype(np.float64), t.astype(np.float64), mask.astype(np.float64))
    assert L == pytest.approx(Lr, rel=1e-5)
    # every entry: |g - g_ref| <= 1e-4 |g_ref| + 1e-6 max|g_ref of its block|.  The floor is
    # the FP32 rounding of a sum of B sample terms (about B * 2^-24 of the largest term, so
    # 2e-5 at B = 300); a wrong entry, even a single bias, exceeds it
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        scale = np.abs(gr[k]).max()
        err = np.abs(g[k] - gr[k]) - (1e-4 * np.abs(gr[k]) + 1e-6 * scale)
        worst = np.unravel_index(np.argmax(err), err.shape)
        assert err.max() <= 0.0, (k, worst, float(g[k][worst]), float(gr[k][worst]), scale)


def _bf16(x):
    """Round to BF16 (nearest, ties to even) through FP32, as the device packs FP32 values."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _ulp_bf16(x):
    """Spacing of BF16 numbers at |x| (8 significant bits)."""
    a = np.maximum(np.abs(np.asarray(x, np.float64)), 2.0 ** -126)
    return 2.0 ** (np.floor(np.log2(a)) - 7)


def bf16_forward_with_bound(p, x, out_scale, out_shift):
    """The inference arithmetic written out in FP64 (BF16 layer-2/3 weights; every tanh
    input and output rounded to BF16; FP32 accumulation), and a per-output bound on how far
    the device may be from it: each tanh may differ by its input's rounding plus two BF16
    units of its output (the hardware tanh is an approximation), propagated through the
    BF16 weights, plus FP32 accumulation of 64 products."""
    w2, w3 = _bf16(p["w2"]), _bf16(p["w3"])
    z1 = x @ p["w1"].T + p["b1"]
    z1b = _bf16(z1)
    h1 = _bf16(np.tanh(z1b))
    d1 = _ulp_bf16(z1) + 2 * _ulp_bf16(h1)
    z2 = h1 @ w2.T + p["b2"]
    d2 = d1 @ np.abs(w2).T + 2.0 ** -22 * (np.abs(h1) @ np.abs(w2).T + np.abs(p["b2"]))
    h2 = _bf16(np.tanh(_bf16(z2)))
    dh2 = d2 + _ulp_bf16(z2) + 2 * _ulp_bf16(h2)
    y = (h2 @ w3.T + p["b3"]) * out_scale + out_shift
    dy = np.abs(out_scale) * (dh2 @ np.abs(w3).T + 2.0 ** -22 * (np.abs(h2) @ np.abs(w3).T + np.abs(p["b3"])))
    return y, dy


def test_tensor_core_inference_matches_bf16_reference(cuda):
    """tcgen05 inference (ion_surrogate_eval) against the BF16 arithmetic written out in
    FP64, within the bound that arithmetic implies (a few BF16 units per activation), at
    sizes that leave a ragged last 128-row tile."""
    p = mlp.init_params(9, scale=1.0)
    rng = np.random.default_rng(1)
    lo, hi = np.log(CA_RANGE[0]), np.log(CA_RANGE[1])
    for n in (1000, 128, 1):
        V = rng.uniform(-100, 50, n).astype(np.float32)
        ca = np.exp(rng.uniform(lo, hi, n)).astype(np.float32)
        oscale = rng.uniform(0.5, 2.0, 24).astype(np.float32)
        oshift = rng.uniform(-1.0, 1.0, 24).astype(np.float32)
        p32 = {k: v.astype(np.float32) for k, v in p.items()}
        w = ion.weights_from_dict(p32, in_shift=(mlp.V_CENTER, 0.5 * (lo + hi)), in_scale=(1 / mlp.V_HALF, 2 / (hi - lo)),
                                  out_shift=oshift, out_scale=oscale)
        got = ion.ion_surrogate_eval(w, V, ca)
        x = np.stack([(V.astype(np.float64) - np.float32(mlp.V_CENTER)) * np.float32(1 / mlp.V_HALF),
                      (np.log(ca.astype(np.float64)) - np.float32(0.5 * (lo + hi))) * np.float32(2 / (hi - lo))], 1)
        ref, bound = bf16_forward_with_bound({k: v.astype(np.float64) for k, v in p32.items()}, x,
                                             oscale.astype(np.float64), oshift.astype(np.float64))
        ratio = np.abs(got - ref) / (bound + 1e-12)
        print(f"n = {n}: max |err| / bound = {ratio.max():.3f}, max |err| {np.abs(got - ref).max():.2e}")
        assert np.all(np.isfinite(got))
        assert ratio.max() <= 1.0, (n, np.unravel_index(np.argmax(ratio), ratio.shape), ratio.max())


def test_tcgen05_and_warp_mma_cell_updates_agree(cuda, O):
    """The two tensor-core paths of the learned cell update (tcgen05 with TMEM accumulators,
    the default, and warp-level mma.sync) evaluate the same BF16 network: one step of a
    ragged 1000-cell network from the same state agrees.  The two accumulate the 64-term
    layer sums in different orders, so a hidden activation can round to a neighbouring
    BF16 value (2^-8 relative); through one step that moves a gate by at most ~1e-3 of its
    floor, and leaves the voltages (which use the step-t gates) equal."""
    p = mlp.init_params(3, scale=1.0)
    lo, hi = np.log(CA_RANGE[0]), np.log(CA_RANGE[1])
    w = ion.weights_from_dict({k: v.astype(np.float32) for k, v in p.items()},
                              in_shift=(mlp.V_CENTER, 0.5 * (lo + hi)), in_scale=(1 / mlp.V_HALF, 2 / (hi - lo)),
                              out_shift=np.full(24, -1.0, np.float32), out_scale=np.full(24, 0.5, np.float32))
    n = 1000
    S0 = O.default_state(n)
    S0[0] += inputs.vdend_jitter(n, 5, 10.0)
    S0 = S0.astype(np.float32)
    out = []
    for flags in (ion.FLAG_KAHAN | ion.FLAG_SURROGATE, ion.FLAG_KAHAN | ion.FLAG_SURROGATE | ion.FLAG_SURROGATE_WARP_MMA):
        with ion.Simulation(n, ion.DENSE_UNIFORM, g=inputs.junction_weight(0.04, n), init_state=S0, flags=flags,
                            surrogate=w) as sim:
            sim.step(1)
            out.append(sim.state())
    d = np.abs(out[0].astype(np.float64) - out[1]) / np.maximum(np.abs(out[1]), 1e-3)
    assert np.all(out[0][:4] == out[1][:4])      # voltages and [Ca] use the step-t state only
    assert d.max() <= 2e-3, d.max(axis=1)


def test_trained_surrogate_fits_the_rate_functions(trained, O):
    w, loss = trained
    assert loss < 2e-3
    rng = np.random.default_rng(11)
    V = rng.uniform(-100, 50, 4000).astype(np.float32)
    ca = np.exp(rng.uniform(np.log(CA_RANGE[0]), np.log(CA_RANGE[1]), 4000)).astype(np.float32)
    got = ion.ion_surrogate_eval(w, V, ca)
    ref, mask = mlp.gate_targets(V, ca)
    xinf_err = np.abs(mlp.sigmoid(got[:, 0::2]) - mlp.sigmoid(ref[:, 0::2]))
    logit_err = np.abs(got[:, 0::2] - ref[:, 0::2])
    lntau_err = np.abs(got[:, 1::2] - ref[:, 1::2])[:, mask[1::2] > 0]
    print(f"x_inf |err| mean {xinf_err.mean():.2e} max {xinf_err.max():.2e}; logit |err| mean "
          f"{logit_err.mean():.2e}; ln tau |err| mean {lntau_err.mean():.2e} max {lntau_err.max():.2e}")
    assert xinf_err.mean() < 5e-3 and xinf_err.max() < 0.1
    assert lntau_err.mean() < 0.05


def _learned_vs_exact(w, O, pul, n=4096, steps=2000):
    """A 4096-cell k = 100 network run with exact and with learned rates from the same
    state: (exact trace, learned trace, learned final state), V_axon of every cell."""
    rp, col = inputs.random_symmetric_csr(n, 100, 2)
    wts = np.full(len(col), inputs.junction_weight(0.04, 100), np.float32)
    S0 = O.default_state(n)
    S0[0] += inputs.vdend_jitter(n, 2)
    S0 = S0.astype(np.float32)
    out = []
    for flags, kw in ((ion.FLAG_KAHAN, {}), (ion.FLAG_KAHAN | ion.FLAG_SURROGATE, dict(surrogate=w))):
        with ion.Simulation(n, ion.CSR, row_ptr=rp, col=col, w=wts, init_state=S0, flags=flags, **kw) as sim:
            sim.set_input(pul)
            ion.ion_set_trace(sim.h, 1, steps)
            sim.step(steps)
            out.append((sim.state(), ion.ion_read_trace(sim.h, n, steps)))
    return out[0][1], out[1][1], out[1][0]


def test_learned_rates_subthreshold(trained, O):
    """The workload's input (a 10 ms pulse to 20 % of the cells, which drains into their
    neighbours without firing): learned and exact V_axon traces stay within a few mV."""
    w, _ = trained
    n = 4096
    te, ts, Ss = _learned_vs_exact(w, O, inputs.pulses(inputs.random_subset(n, 0.2, 2), 50.0, 60.0, 6.0))
    assert np.all(np.isfinite(Ss))
    trace_rms = float(np.sqrt(np.mean((te.astype(np.float64) - ts) ** 2)))
    print(f"subthreshold: V_axon trace rms {trace_rms:.3f} mV, max {np.abs(te - ts).max():.3f} mV")
    assert trace_rms < 5.0


def test_learned_rates_spiking(trained, O):
    """Every cell pulsed at 50-60 ms: both methods fire a burst in every sampled cell, with
    spike counts within one of each other and first spikes within 0.5 ms on average (the
    surrogate changes the model, it is not a rounding error)."""
    w, _ = trained
    n = 4096
    te, ts, Ss = _learned_vs_exact(w, O, inputs.pulse_windows(np.arange(n), [(50.0, 60.0)], 6.0))
    assert np.all(np.isfinite(Ss))
    trace_rms = float(np.sqrt(np.mean((te.astype(np.float64) - ts) ** 2)))
    se = [O.spike_steps(te[:, c]) for c in range(0, n, 64)]
    ss = [O.spike_steps(ts[:, c]) for c in range(0, n, 64)]
    same = [len(a) == len(b) for a, b in zip(se, ss)]
    first = np.array([abs(int(a[0]) - int(b[0])) for a, b in zip(se, ss) if len(a) and len(b)])
    dstep = np.concatenate([np.abs(a - b) for a, b in zip(se, ss) if len(a) == len(b)] or [np.zeros(0)])
    print(f"spiking: V_axon trace rms {trace_rms:.3f} mV, spikes {sum(map(len, se))} vs "
          f"{sum(map(len, ss))} (64 sampled cells), same count in {sum(same)}/64 cells, first-spike "
          f"|dt| max {first.max() if len(first) else -1} mean {first.mean() if len(first) else -1:.2f} steps, "
          f"matched |dt| max {dstep.max() if len(dstep) else 0} steps")
    assert all(len(a) >= 1 for a in se) and all(len(b) >= 1 for b in ss)    # every sampled cell fires
    # the learned rates change the model, not only the rounding: the stated bound is the
    # burst's spike count within one spike of the exact method in every sampled cell and
    # its first spike within 10 steps (0.5 ms) on average, 20 at most (measured on the
    # tcgen05 path: one spike more in every sampled cell, first spikes 8.6 steps apart on
    # average, 9 at most)
    counts = np.array([len(b) - len(a) for a, b in zip(se, ss)])
    assert np.all(np.abs(counts) <= 1), counts
    assert len(first) == len(se) and first.mean() <= 10.0 and first.max() <= 20, first


def test_surrogate_gain_is_reported(trained, O):
    """What the learned rate functions gain on this GPU: both paths time the same 4096-cell
    network with the same gap-current kernel (the direct CSR kernel, which the surrogate
    path uses; the exact path is held to it by turning V_dend staging off), so the ratio
    compares the learned rate functions with the exact ones.  The exact functions are
    cheap on the SFU, so the surrogate is slower here; the test holds the ratio to the
    stated floor."""
    import time
    w, _ = trained
    n = 4096
    rp, col = inputs.random_symmetric_csr(n, 100, 2)
    wts = np.full(len(col), inputs.junction_weight(0.04, 100), np.float32)
    S0 = O.default_state(n)
    S0[0] += inputs.vdend_jitter(n, 2)
    S0 = S0.astype(np.float32)
    rate = {}
    for name, flags, kw in (("exact", ion.FLAG_KAHAN, dict(tune=dict(csr_staging=1))),
                            ("surrogate", ion.FLAG_KAHAN | ion.FLAG_SURROGATE, dict(surrogate=w))):
        with ion.Simulation(n, ion.CSR, row_ptr=rp, col=col, w=wts, init_state=S0, flags=flags, **kw) as sim:
            sim.step(200)
            sim.sync()
            t0 = time.perf_counter()
            sim.step(2000)
            sim.sync()
            rate[name] = n * 2000 / (time.perf_counter() - t0)
            assert np.all(np.isfinite(sim.state()))
    gain = rate["surrogate"] / rate["exact"]
    print(f"cell-steps/s: exact {rate['exact']:.3e}, surrogate {rate['surrogate']:.3e}, gain {gain:.2f}x")
    # the stated result on this GPU: the learned rates cost about twice the exact ones
    # (0.46-0.49x measured on the full C5 network: 192 tanh.bf16x2 per cell-step against
    # ~36 SFU operations); this guards against a regression beyond that
    assert gain >= 0.3, gain
