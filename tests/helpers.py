"""Shared test helpers: initial states fed identically to both sides, and the per-step
error measure (one step from an identical FP32 state, relative with per-field floors)."""
import numpy as np

# floors of the relative error: voltages 1 mV, [Ca] 1, gates 1e-3, g_CaL 1e-3,
# currents 1e-2 uA/cm^2
FLOORS = np.array([1.0, 1.0, 1.0, 1.0] + [1e-3] * 12 + [1e-3, 1e-2, 1e-2])
STEP_RTOL = 1e-5        # per-step state relative error bound for the FP32 path
TRAJ_MV = 0.1           # |dV| bound over the first 100 ms
V_FIELDS = (0, 1, 2)


def initial_state(O, cfg, model=None):
    """Oracle default state + the config's V_dend jitter, rounded to FP32 (the values both
    sides start from), returned as float32 (19, n)."""
    S = O.default_state(cfg["n"], model)
    S[O.F["V_dend"]] += cfg["jitter"]
    return S.astype(np.float32)


def step_rel_err(S_gpu, S_ref, ic_scale=None):
    """|S_gpu - S_ref| / max(|S_ref|, floor) per field and cell.

    The gap current I_c is a sum of terms of both signs that can cancel; its error is
    measured against the scale of its terms, ic_scale_i = sum_j w_ij |dV_ij| (when
    given), the quantity the FP32 rounding of the individual terms is proportional to.
    """
    S_gpu = np.asarray(S_gpu, np.float64)
    S_ref = np.asarray(S_ref, np.float64)
    den = np.maximum(np.abs(S_ref), FLOORS[:, None])
    if ic_scale is not None:
        den[18] = np.maximum(den[18], np.asarray(ic_scale, np.float64))
    return np.abs(S_gpu - S_ref) / den


def csr_abs_scale(row_ptr, col, w, vd):
    """sum_{e in row i} w_e |V_i - V_col(e)| for every row i."""
    n = len(row_ptr) - 1
    vd = np.asarray(vd, np.float64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    if len(col) == 0:
        return np.zeros(n)
    return np.bincount(rows, weights=np.asarray(w, np.float64) * np.abs(vd[rows] - vd[col]), minlength=n)


def sum_abs_dv(vd):
    """sum_j |V_i - V_j| for every i (O(n log n) via sorting)."""
    vd = np.asarray(vd, np.float64)
    order = np.argsort(vd)
    s = vd[order]
    n = len(s)
    pre = np.concatenate([[0.0], np.cumsum(s)])
    k = np.arange(n)
    tot = s * k - pre[:-1] + (pre[-1] - pre[1:]) - s * (n - 1 - k)
    out = np.empty(n)
    out[order] = tot
    return out
