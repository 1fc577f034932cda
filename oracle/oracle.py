"""ctypes front of the FP64 oracle in ``ion_oracle.c`` (test infrastructure only).

The arithmetic lives in the C file; this module only builds it, marshals numpy arrays
and adds the trace post-processing the tests use (spike extraction).  Nothing in the
product library imports it.

Paper: Smaragdos et al., "BrainFrame" (arXiv 1612.01501), Sec. 2.2 (cell and step),
Algorithm 1 (realistic gap junction), Table "reqs" (19 state words per cell).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ion_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# state field order (mirrors the enum in ion_oracle.c)
FIELDS = ("V_dend", "V_soma", "V_axon", "Ca", "r", "s", "q", "k", "l", "m_s", "h_s",
          "n_s", "x_s", "m_a", "h_a", "x_a", "g_CaL", "I_CaH", "I_c")
NF = len(FIELDS)
F = {name: i for i, name in enumerate(FIELDS)}
# gate order of or_rates
GATES = ("r", "s", "q", "k", "l", "m_s", "h_s", "n_s", "x_s", "m_a", "h_a", "x_a")
NG = len(GATES)
# constants-table order
PARAMS = ("g_int", "p1", "p2", "g_CaH", "g_KCa", "g_h", "g_ld", "g_CaL", "g_Na_s",
          "g_Kdr_s", "g_K_s", "g_ls", "g_Na_a", "g_K_a", "g_la", "V_Na", "V_K", "V_Ca",
          "V_h", "V_L", "C_m", "ca_in", "ca_out", "V_0", "Ca_0")
P = {name: i for i, name in enumerate(PARAMS)}
NCELLPARAMS = 20   # per-cell constants: table entries 0..19 (g_CaL's row unused)

DENSE, CSR, NOGJ, DENSE_SGJ, CSR_SGJ, MATRIX = 0, 1, 2, 3, 4, 5   # SGJ: linear junctions (Sec. 2.3.2)
DT_MS = 0.05  # Sec. 2.2: delta = 50 us


def build(force: bool = False) -> str:
    """Compile ion_oracle.c into liboracle.so (gcc, FP64, OpenMP over cells)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_FLOP_SRC = os.path.join(os.path.dirname(_SRC), "flop_count.cpp")
_FLOP_EXE = os.path.join(os.path.dirname(_SRC), "flop_count")


def build_flop_count(force: bool = False) -> str:
    """Compile flop_count.cpp: this oracle's source with every double replaced by an
    operation-counting number type (g++; the oracle's C needs -fpermissive as C++)."""
    stale = not os.path.exists(_FLOP_EXE) or any(os.path.getmtime(p) > os.path.getmtime(_FLOP_EXE)
                                                  for p in (_FLOP_SRC, _SRC))
    if force or stale:
        tmp = _FLOP_EXE + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fpermissive", "-w", "-o", tmp, _FLOP_SRC, "-lm"])
        os.replace(tmp, _FLOP_EXE)
    return _FLOP_EXE


def op_counts() -> dict:
    """Operation counts of one cell step, one dense gap-junction pair and one SGJ edge."""
    out = subprocess.check_output([build_flop_count()], text=True)
    return {k: float(v) for k, v in (line.split() for line in out.splitlines())}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            lp = ctypes.POINTER(ctypes.c_int64)
            fp = ctypes.POINTER(ctypes.c_float)
            L.or_nfields.restype = ctypes.c_int
            L.or_nparams.restype = ctypes.c_int
            L.or_ngates.restype = ctypes.c_int
            L.or_max_threads.restype = ctypes.c_int
            L.or_model_default.argtypes = [dp]
            L.or_rates.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp]
            L.or_default_state.argtypes = [ctypes.c_int, dp, dp]
            L.or_gj_dense.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, ctypes.c_int]
            L.or_gj_csr.argtypes = [ctypes.c_int, ip, ip, dp, dp, dp, ctypes.c_int]
            L.or_gj_dense_sgj.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, ctypes.c_int]
            L.or_gj_matrix.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int]
            L.or_gj_csr_sgj.argtypes = [ctypes.c_int, ip, ip, dp, dp, dp, ctypes.c_int]
            L.or_cell_step.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp, dp, dp, dp, ctypes.c_int]
            L.or_run.restype = ctypes.c_int
            L.or_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ip, ip, dp, dp, dp,
                                 ctypes.c_double, dp, ctypes.c_int64, ctypes.c_int64, fp,
                                 ctypes.c_int, ip, lp, lp, dp, ctypes.c_int, ip, dp, ctypes.c_int]
            assert L.or_nfields() == NF and L.or_nparams() == len(PARAMS) and L.or_ngates() == NG
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if a is not None else None


def _l(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if a is not None else None


def _f(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if a is not None else None


def max_threads() -> int:
    return int(lib().or_max_threads())


def model_default() -> np.ndarray:
    out = np.zeros(len(PARAMS), np.float64)
    lib().or_model_default(_d(out))
    return out


def rates(V: float, ca: float):
    """(x_inf[12], tau[12]) of every gate at voltage V and calcium ca."""
    xi = np.zeros(NG)
    ta = np.zeros(NG)
    lib().or_rates(float(V), float(ca), _d(xi), _d(ta))
    return xi, ta


def default_state(n: int, model=None) -> np.ndarray:
    """(19, n) FP64 default state (every cell identical)."""
    model = model_default() if model is None else np.ascontiguousarray(model, np.float64)
    S = np.zeros((NF, n), np.float64)
    lib().or_default_state(int(n), _d(model), _d(S))
    return S


def gj_dense(vd, g: float, threads: int = 1) -> np.ndarray:
    vd = np.ascontiguousarray(vd, np.float64)
    ic = np.zeros_like(vd)
    lib().or_gj_dense(len(vd), _d(vd), float(g), _d(ic), int(threads))
    return ic


def gj_csr(row_ptr, col, w, vd, threads: int = 1) -> np.ndarray:
    row_ptr = np.ascontiguousarray(row_ptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.float64)
    vd = np.ascontiguousarray(vd, np.float64)
    ic = np.zeros_like(vd)
    lib().or_gj_csr(len(vd), _i(row_ptr), _i(col), _d(w), _d(vd), _d(ic), int(threads))
    return ic


def gj_matrix(W, vd, threads: int = 1) -> np.ndarray:
    """Dense N x N weights: Ic_i = sum_j W[i, j] (0.8 e^{-dV^2/100} + 0.2) dV."""
    vd = np.ascontiguousarray(vd, np.float64)
    W = np.ascontiguousarray(W, np.float64)
    assert W.shape == (len(vd), len(vd))
    ic = np.zeros_like(vd)
    lib().or_gj_matrix(len(vd), _d(W), _d(vd), _d(ic), int(threads))
    return ic


def gj_dense_sgj(vd, g: float, threads: int = 1) -> np.ndarray:
    """SGJ use case: Ic_i = g * sum_j (V_i - V_j)."""
    vd = np.ascontiguousarray(vd, np.float64)
    ic = np.zeros_like(vd)
    lib().or_gj_dense_sgj(len(vd), _d(vd), float(g), _d(ic), int(threads))
    return ic


def gj_csr_sgj(row_ptr, col, w, vd, threads: int = 1) -> np.ndarray:
    """SGJ use case: Ic_i = sum over row i of w_e (V_i - V_col)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.float64)
    vd = np.ascontiguousarray(vd, np.float64)
    ic = np.zeros_like(vd)
    lib().or_gj_csr_sgj(len(vd), _i(row_ptr), _i(col), _d(w), _d(vd), _d(ic), int(threads))
    return ic


def _cell_params(cell_params, n):
    """Per-cell constants as a contiguous (NCELLPARAMS, n) float64 array, or None."""
    if cell_params is None:
        return None
    cp = np.ascontiguousarray(cell_params, np.float64)
    assert cp.shape == (NCELLPARAMS, n), cp.shape
    return cp


def cell_step(S, ic=None, iapp=None, model=None, dt: float = DT_MS, threads: int = 1,
              cell_params=None) -> np.ndarray:
    """One explicit-Euler cell update of every cell, with the gap current given.
    cell_params: None or (NCELLPARAMS, n) per-cell constants (table entries 0..19; the
    g_CaL row is not read, g_CaL being a state field)."""
    S = np.ascontiguousarray(S, np.float64)
    n = S.shape[1]
    cp = _cell_params(cell_params, n)
    model = model_default() if model is None else np.ascontiguousarray(model, np.float64)
    ic = None if ic is None else np.ascontiguousarray(ic, np.float64)
    iapp = None if iapp is None else np.ascontiguousarray(iapp, np.float64)
    Sn = np.zeros_like(S)
    lib().or_cell_step(n, _d(model), _d(cp), float(dt), _d(S), _d(ic), _d(iapp), _d(Sn), int(threads))
    return Sn


def run(S0, n_steps: int, kind: int = DENSE, g: float = 0.0, row_ptr=None, col=None, w=None,
        model=None, dt: float = DT_MS, t0: int = 0, iapp_dense=None, pulses=None,
        trace_cells=None, threads: int = 1, cell_params=None):
    """Advance S0 (19, n) by n_steps; returns (S_final, trace or None).

    pulses: None or a tuple (cell[int32], t_begin[int64], t_end[int64], amp[float64]).
    trace_cells: indices whose V_axon is recorded after every step, shape (n_steps, len).
    """
    S = np.array(S0, np.float64, order="C", copy=True)
    n = S.shape[1]
    cp = _cell_params(cell_params, n)
    model = model_default() if model is None else np.ascontiguousarray(model, np.float64)
    if kind == MATRIX:
        w = np.ascontiguousarray(w, np.float64)
        assert w.shape == (n, n)
    if kind in (CSR, CSR_SGJ):
        row_ptr = np.ascontiguousarray(row_ptr, np.int32)
        col = np.ascontiguousarray(col, np.int32)
        w = np.ascontiguousarray(w, np.float64)
    if iapp_dense is not None:
        iapp_dense = np.ascontiguousarray(iapp_dense, np.float32)
        assert iapp_dense.shape == (n_steps, n)
    if pulses is not None:
        pc = np.ascontiguousarray(pulses[0], np.int32)
        pb = np.ascontiguousarray(pulses[1], np.int64)
        pe = np.ascontiguousarray(pulses[2], np.int64)
        pa = np.ascontiguousarray(pulses[3], np.float64)
        npul = len(pc)
    else:
        pc = pb = pe = pa = None
        npul = 0
    if trace_cells is not None:
        tc = np.ascontiguousarray(trace_cells, np.int32)
        tr = np.zeros((n_steps, len(tc)), np.float64)
    else:
        tc = tr = None
    rc = lib().or_run(n, int(kind), float(g), _i(row_ptr), _i(col), _d(w), _d(model), _d(cp), float(dt),
                      _d(S), int(t0), int(n_steps), _f(iapp_dense), npul, _i(pc), _l(pb), _l(pe),
                      _d(pa), 0 if tc is None else len(tc), _i(tc), _d(tr), int(threads))
    if rc != 0:
        raise MemoryError("oracle could not allocate its step buffers")
    return S, tr


def spike_steps(trace_col, threshold: float = 0.0, rearm: float = -30.0) -> np.ndarray:
    """Spike times of one V_axon trace, as step indices.

    A spike is an upward crossing of `threshold` by V_axon (the first sample >= it), and
    the detector re-arms once V_axon falls below `rearm`.  (The paper names the axon
    voltage as the cell output but defines no spike; this is the reading used.)
    """
    out = []
    armed = True
    for t, v in enumerate(np.asarray(trace_col)):
        if armed and v >= threshold:
            out.append(t)
            armed = False
        elif not armed and v < rearm:
            armed = True
    return np.asarray(out, np.int64)
