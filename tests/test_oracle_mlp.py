"""Pins of the FP64 surrogate-MLP oracle: its analytic gradients against central finite
differences (independent of the backward formulas), and its targets against the rate
functions' closed forms."""
import numpy as np
import pytest

from oracle import mlp


def test_mlp_gradients_match_finite_differences(O):
    rng = np.random.default_rng(3)
    p = mlp.init_params(1)
    x = rng.uniform(-1, 1, (7, 2))
    t = rng.normal(0, 1, (7, 24))
    mask = np.ones(24)
    mask[[11, 19]] = 0.0
    L, g = mlp.loss_and_grads(p, x, t, mask)
    h = 1e-4      # truncation ~h^2, roundoff ~eps/h: both far below the tolerance here
    for name in ("w1", "b1", "w2", "b2", "w3", "b3"):
        flat = p[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for k in idx:
            old = flat[k]
            flat[k] = old + h
            Lp, _ = mlp.loss_and_grads(p, x, t, mask)
            flat[k] = old - h
            Lm, _ = mlp.loss_and_grads(p, x, t, mask)
            flat[k] = old
            num = (Lp - Lm) / (2 * h)
            assert g[name].reshape(-1)[k] == pytest.approx(num, rel=1e-6, abs=1e-11), (name, k)


def test_targets_follow_rate_functions(O):
    out, mask = mlp.gate_targets([-30.0, -80.0], [1.0, 1.0])
    G = {g: i for i, g in enumerate(O.GATES)}
    assert out[0, 2 * G["m_s"]] == pytest.approx(0.0, abs=1e-12)   # logit(m_inf(-30)) = logit(1/2)
    assert out[1, 2 * G["q"]] == pytest.approx(0.0, abs=1e-12)     # q_inf(-80) = 1/2
    assert mlp.sigmoid(mlp.gate_targets([-47.0], [1.0])[0][0, 2 * G["h_s"]]) == pytest.approx(
        O.rates(-47.0, 1.0)[0][G["h_s"]], rel=1e-12)
    assert out[0, 2 * G["k"] + 1] == 0.0                          # ln(tau_k) = ln 1
    assert mask[2 * G["m_s"] + 1] == 0 and mask[2 * G["m_a"] + 1] == 0 and mask.sum() == 22
