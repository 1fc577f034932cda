"""FP64 reference of the rate-function surrogate MLP (test infrastructure only).

The surrogate stands in for the channel rate functions of the cell model (the gates'
steady states x_inf and time constants tau, Sec. 2.2 of the paper; the surrogate itself
is not in the paper).  Network: inputs (v, c) -> 64 tanh units -> 64 tanh units -> 24
linear outputs, weights row-major [out][in].  Training objective: mean over samples and
unmasked outputs of the squared error, in normalised units.

Only the tests import this module; the library never does.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _O

N_IN, N_HID, N_OUT = 2, 64, 24
V_CENTER, V_HALF = -25.0, 75.0          # V in [-100, 50] mV -> [-1, 1]


def init_params(seed: int, scale: float = 1.0):
    """Deterministic weights for tests (not the training initialisation)."""
    rng = np.random.default_rng(seed)
    return {
        "w1": rng.normal(0, scale / np.sqrt(N_IN), (N_HID, N_IN)), "b1": rng.normal(0, 0.1, N_HID),
        "w2": rng.normal(0, scale / np.sqrt(N_HID), (N_HID, N_HID)), "b2": rng.normal(0, 0.1, N_HID),
        "w3": rng.normal(0, scale / np.sqrt(N_HID), (N_OUT, N_HID)), "b3": rng.normal(0, 0.1, N_OUT),
    }


def forward(p, x):
    """x: (B, 2) normalised inputs -> (y (B, 24), cache)."""
    z1 = x @ p["w1"].T + p["b1"]
    h1 = np.tanh(z1)
    z2 = h1 @ p["w2"].T + p["b2"]
    h2 = np.tanh(z2)
    y = h2 @ p["w3"].T + p["b3"]
    return y, (x, h1, h2)


def loss_and_grads(p, x, t, mask):
    """Masked MSE L = sum_{s,o} mask_o (y_so - t_so)^2 / (B * sum(mask)) and dL/dparams."""
    B = x.shape[0]
    y, (x, h1, h2) = forward(p, x)
    m = np.asarray(mask, np.float64)
    denom = B * m.sum()
    e = (y - t) * m
    L = float((e * e).sum() / denom)
    d3 = 2.0 * e / denom                      # dL/dy
    g = {"w3": d3.T @ h2, "b3": d3.sum(0)}
    d2 = (d3 @ p["w3"]) * (1.0 - h2 * h2)     # through tanh
    g["w2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ p["w2"]) * (1.0 - h1 * h1)
    g["w1"] = d1.T @ x
    g["b1"] = d1.sum(0)
    return L, g


LOGIT_MAX = 15.0


def gate_targets(V, ca):
    """Raw targets of every sample from the FP64 rate functions: for gate g, output 2g is
    logit(x_inf) clipped to +-15 and output 2g+1 is ln(tau) (masked for the instantaneous
    gates m_s, m_a)."""
    V = np.atleast_1d(np.asarray(V, np.float64))
    ca = np.atleast_1d(np.asarray(ca, np.float64))
    out = np.zeros((len(V), N_OUT))
    mask = np.ones(N_OUT)
    for s in range(len(V)):
        xi, ta = _O.rates(V[s], ca[s])
        with np.errstate(divide="ignore"):
            lg = np.log(xi) - np.log1p(-np.minimum(xi, 1.0 - 1e-16))
        out[s, 0::2] = np.clip(lg, -LOGIT_MAX, LOGIT_MAX)
        out[s, 1::2] = np.log(np.where(ta > 0, ta, 1.0))
    for gname in ("m_s", "m_a"):
        mask[2 * _O.GATES.index(gname) + 1] = 0.0
    return out, mask


def normalise_inputs(V, ca, ca_lo, ca_hi):
    lc, lh = np.log(ca_lo), np.log(ca_hi)
    return np.stack([(np.asarray(V, np.float64) - V_CENTER) / V_HALF,
                     (np.log(np.asarray(ca, np.float64)) - 0.5 * (lc + lh)) / (0.5 * (lh - lc))], axis=1)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-np.asarray(z, np.float64)))
