"""Python binding of libion.so (include/ion.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does nothing but
convert numpy arrays / torch tensors to pointers, call it, and raise `IonError` on a
non-OK status.  All arithmetic runs in the library's CUDA kernels; if libion.so is
missing this module raises on import of the library -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libion.so")

NFIELDS, NPARAMS, NGATES, NCELLPARAMS = 19, 25, 12, 20
FIELDS = ("V_dend", "V_soma", "V_axon", "Ca", "r", "s", "q", "k", "l", "m_s", "h_s", "n_s", "x_s",
          "m_a", "h_a", "x_a", "g_CaL", "I_CaH", "I_c")
FIELD = {f: i for i, f in enumerate(FIELDS)}
FIELD_ALL = -1
GATES = ("r", "s", "q", "k", "l", "m_s", "h_s", "n_s", "x_s", "m_a", "h_a", "x_a")

OK, ERR_INVALID_ARG, ERR_BAD_CSR, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ("OK", "INVALID_ARG", "BAD_CSR", "OOM", "CUDA", "NONFINITE", "TIMEOUT", "UNSUPPORTED")
DENSE_UNIFORM, CSR, NO_GJ, DENSE_MATRIX = 0, 1, 2, 3
HOST, DEVICE = 0, 1
FLAG_KAHAN, FLAG_PERSISTENT, FLAG_SURROGATE, FLAG_CHECKS, FLAG_NO_GRAPH, FLAG_SPLIT, FLAG_HALF_WORK = 1, 2, 4, 8, 16, 32, 64
FLAG_CSR_AS_GIVEN = 128
FLAG_SGJ = 256           # SGJ use case: linear junctions w (V_i - V_j)
FLAG_NO_PDL = 512        # ordinary launches instead of programmatic dependent launches
FLAG_SURROGATE_WARP_MMA = 1024   # surrogate MLP on warp-level mma.sync instead of tcgen05
INPUT_NONE, INPUT_PULSES, INPUT_DENSE = 0, 1, 2
MLP_IN, MLP_HID, MLP_OUT = 2, 64, 24

c_i32p = ctypes.POINTER(ctypes.c_int32)
c_i64p = ctypes.POINTER(ctypes.c_int64)
c_f32p = ctypes.POINTER(ctypes.c_float)


class IonError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"ION_ERR_{name}: {msg}")
        self.status = status


class ion_net(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int32), ("kind", ctypes.c_int32)]


class ion_conn(ctypes.Structure):
    _fields_ = [("g_c", ctypes.c_float), ("row_ptr", c_i32p), ("col_idx", c_i32p), ("weight", c_f32p),
                ("nnz", ctypes.c_int64), ("mem", ctypes.c_int32)]


class ion_model(ctypes.Structure):
    _fields_ = [("v", ctypes.c_double * NPARAMS)]


class ion_params(ctypes.Structure):
    _fields_ = [("dt_ms", ctypes.c_double), ("model", ctypes.POINTER(ion_model)), ("flags", ctypes.c_uint32),
                ("surrogate", ctypes.c_void_p), ("check_every", ctypes.c_int32), ("graph_steps", ctypes.c_int32),
                ("barrier_timeout_ns", ctypes.c_uint64), ("cuda_stream", ctypes.c_void_p),
                ("tune", ctypes.c_void_p), ("debug_delay_ns", ctypes.c_int64), ("cell_params", c_f32p),
                ("debug_barrier_base", ctypes.c_uint32)]


class ion_input(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("mem", ctypes.c_int32), ("dense", c_f32p), ("n_pulses", ctypes.c_int32),
                ("pulse_cell", c_i32p), ("pulse_begin", c_i64p), ("pulse_end", c_i64p), ("pulse_amp", c_f32p)]


class ion_tune(ctypes.Structure):
    _fields_ = [("dense_rows_per_warp", ctypes.c_int32), ("dense_warps", ctypes.c_int32),
                ("dense_col_splits", ctypes.c_int32), ("csr_lanes_per_row", ctypes.c_int32),
                ("csr_rows_per_cta", ctypes.c_int32), ("csr_lanes_scale", ctypes.c_int32),
                ("csr_staging", ctypes.c_int32), ("csr_bank_order", ctypes.c_int32)]


class ion_surrogate_weights(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_float * (MLP_HID * MLP_IN)), ("b1", ctypes.c_float * MLP_HID),
                ("w2", ctypes.c_float * (MLP_HID * MLP_HID)), ("b2", ctypes.c_float * MLP_HID),
                ("w3", ctypes.c_float * (MLP_OUT * MLP_HID)), ("b3", ctypes.c_float * MLP_OUT),
                ("in_shift", ctypes.c_float * MLP_IN), ("in_scale", ctypes.c_float * MLP_IN),
                ("out_shift", ctypes.c_float * MLP_OUT), ("out_scale", ctypes.c_float * MLP_OUT)]


class ion_train_cfg(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int64), ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("lr", ctypes.c_float), ("seed", ctypes.c_uint64), ("v_lo", ctypes.c_float), ("v_hi", ctypes.c_float),
                ("ca_lo", ctypes.c_float), ("ca_hi", ctypes.c_float), ("cuda_stream", ctypes.c_void_p)]


# entry point -> (restype, argtypes); the complete list of symbols include/ion.h declares
_SIGS = {
    "ion_model_default": (None, [ctypes.POINTER(ion_model)]),
    "ion_rates": (ctypes.c_int, [ctypes.c_float, ctypes.c_float, c_f32p, c_f32p]),
    "ion_default_state": (ctypes.c_int, [ctypes.POINTER(ion_model), ctypes.c_int32, c_f32p]),
    "ion_create": (ctypes.c_int, [ctypes.POINTER(ion_net), ctypes.POINTER(ion_conn), ctypes.POINTER(ion_params),
                                  c_f32p, ctypes.POINTER(ctypes.c_void_p)]),
    "ion_create_batch": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ion_net), ctypes.POINTER(ion_conn),
                                        ctypes.POINTER(ion_params), c_f32p, ctypes.POINTER(ctypes.c_void_p)]),
    "ion_set_input": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ion_input)]),
    "ion_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ion_input)]),
    "ion_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "ion_read_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_f32p, ctypes.c_int64]),
    "ion_write_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_f32p, ctypes.c_int64]),
    "ion_state_device_ptr": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "ion_set_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]),
    "ion_read_trace": (ctypes.c_int, [ctypes.c_void_p, c_f32p, ctypes.c_int64, c_i64p]),
    "ion_read_trace_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, c_i64p]),
    "ion_trace_wait": (ctypes.c_int, [ctypes.c_void_p]),
    "ion_step_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "ion_debug_fail_alloc": (ctypes.c_int, [ctypes.c_int32]),
    "ion_csr_bank_order": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_void_p]),
    "ion_csr_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "ion_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ion_tune)]),
    "ion_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "ion_set_step_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "ion_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "ion_destroy": (None, [ctypes.c_void_p]),
    "ion_gj_dense": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.c_void_p]),
    "ion_gj_dense_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p,
                                            ctypes.c_int32, ctypes.c_void_p]),
    "ion_gj_csr": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "ion_cell_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ion_model), ctypes.c_double, ctypes.c_void_p]),
    "ion_probe_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_double)]),
    "ion_surrogate_train": (ctypes.c_int, [ctypes.POINTER(ion_train_cfg), ctypes.POINTER(ion_surrogate_weights),
                                           c_f32p]),
    "ion_surrogate_grad": (ctypes.c_int, [ctypes.POINTER(ion_surrogate_weights), c_f32p, c_f32p, c_f32p,
                                          ctypes.c_int32, ctypes.POINTER(ion_surrogate_weights), c_f32p]),
    "ion_surrogate_eval": (ctypes.c_int, [ctypes.POINTER(ion_surrogate_weights), c_f32p, c_f32p, ctypes.c_int64,
                                          c_f32p]),
}

_lib = None


def lib():
    """The loaded libion.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libion.so not built ({LIB_PATH}); run paper_1612_01501_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st: int, handle=None):
    if st != OK:
        msg = lib().ion_last_error(handle)
        raise IonError(st, msg.decode() if msg else "")


def _ptr(a, ctype):
    """Pointer to a numpy array (host) or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.cast(ctypes.c_void_p(a.data_ptr()), ctypes.POINTER(ctype))
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


# ---- model -------------------------------------------------------------------------

def ion_model_default() -> np.ndarray:
    m = ion_model()
    lib().ion_model_default(ctypes.byref(m))
    return np.array(m.v[:], np.float64)


def _model_struct(model):
    if model is None:
        return None
    m = ion_model()
    m.v[:] = [float(x) for x in np.asarray(model, np.float64)]
    return m


def ion_rates(V: float, ca: float):
    xi = np.zeros(NGATES, np.float32)
    ta = np.zeros(NGATES, np.float32)
    _check(lib().ion_rates(float(V), float(ca), _ptr(xi, ctypes.c_float), _ptr(ta, ctypes.c_float)))
    return xi, ta


def ion_default_state(n: int, model=None) -> np.ndarray:
    out = np.zeros((NFIELDS, n), np.float32)
    m = _model_struct(model)
    _check(lib().ion_default_state(ctypes.byref(m) if m else None, int(n), _ptr(out, ctypes.c_float)))
    return out


# ---- handles -------------------------------------------------------------------------

def _conn_struct(kind, g=0.0, row_ptr=None, col=None, w=None):
    c = ion_conn()
    c.g_c = float(g)
    keep = []
    if kind == CSR:
        dev = _is_device(row_ptr)
        if not dev:
            row_ptr = np.ascontiguousarray(row_ptr, np.int32)
            col = np.ascontiguousarray(col, np.int32)
            w = None if w is None else np.ascontiguousarray(w, np.float32)
        keep += [row_ptr, col, w]
        c.row_ptr = _ptr(row_ptr, ctypes.c_int32)
        c.col_idx = _ptr(col, ctypes.c_int32)
        c.weight = _ptr(w, ctypes.c_float)
        c.nnz = int(len(col) if not dev else col.numel())
        c.mem = DEVICE if dev else HOST
    elif kind == DENSE_MATRIX:   # w: n x n row-major weights (host array or device tensor)
        dev = _is_device(w)
        if not dev:
            w = np.ascontiguousarray(w, np.float32)
        keep.append(w)
        c.weight = _ptr(w, ctypes.c_float)
        c.mem = DEVICE if dev else HOST
    return c, keep


def _params_struct(dt_ms=0.05, model=None, flags=FLAG_KAHAN, stream=None, graph_steps=0, tune=None,
                   surrogate=None, check_every=0, barrier_timeout_ns=0, debug_delay_ns=0, cell_params=None,
                   debug_barrier_base=0):
    p = ion_params()
    p.dt_ms = float(dt_ms)
    m = _model_struct(model)
    p.model = ctypes.pointer(m) if m is not None else None
    p.flags = int(flags)
    p.graph_steps = int(graph_steps)
    p.check_every = int(check_every)
    p.barrier_timeout_ns = int(barrier_timeout_ns)
    p.debug_delay_ns = int(debug_delay_ns)
    p.debug_barrier_base = int(debug_barrier_base) & 0xFFFFFFFF
    p.cuda_stream = ctypes.c_void_p(stream) if stream else None
    keep = [m]
    if cell_params is not None:   # (NCELLPARAMS, n) host array, ion_param row order
        cp = np.ascontiguousarray(cell_params, np.float32)
        assert cp.ndim == 2 and cp.shape[0] == NCELLPARAMS
        p.cell_params = _ptr(cp, ctypes.c_float)
        keep.append(cp)
    if tune is not None:
        t = ion_tune(*[int(tune.get(k, 0)) for k, _ in ion_tune._fields_])
        p.tune = ctypes.cast(ctypes.pointer(t), ctypes.c_void_p)
        keep.append(t)
    if surrogate is not None:
        p.surrogate = ctypes.cast(ctypes.pointer(surrogate), ctypes.c_void_p)
        keep.append(surrogate)
    return p, keep


def ion_create(n: int, kind: int, g: float = 0.0, row_ptr=None, col=None, w=None, init_state=None, **params):
    """Create a handle (returns the opaque pointer as an int)."""
    net = ion_net(int(n), int(kind))
    conn, k1 = _conn_struct(kind, g, row_ptr, col, w)
    p, k2 = _params_struct(**params)
    st = None
    if init_state is not None:
        st = np.ascontiguousarray(init_state, np.float32)
        assert st.size == NFIELDS * n
    h = ctypes.c_void_p()
    _check(lib().ion_create(ctypes.byref(net), ctypes.byref(conn) if kind != NO_GJ else None, ctypes.byref(p),
                            _ptr(st, ctypes.c_float), ctypes.byref(h)))
    del k1, k2
    return h.value


def ion_create_batch(nets, init_state=None, **params):
    """nets: list of dicts (n, kind, g, row_ptr, col, w) -> handle."""
    arr_n = (ion_net * len(nets))()
    arr_c = (ion_conn * len(nets))()
    keep = []
    for b, d in enumerate(nets):
        arr_n[b] = ion_net(int(d["n"]), int(d["kind"]))
        c, k = _conn_struct(d["kind"], d.get("g", 0.0), d.get("row_ptr"), d.get("col"), d.get("w"))
        arr_c[b] = c
        keep += k
    p, k2 = _params_struct(**params)
    st = None if init_state is None else np.ascontiguousarray(init_state, np.float32)
    h = ctypes.c_void_p()
    _check(lib().ion_create_batch(len(nets), arr_n, arr_c, ctypes.byref(p), _ptr(st, ctypes.c_float), ctypes.byref(h)))
    del keep, k2
    return h.value


def _input_struct(pulses=None, dense=None):
    inp = ion_input()
    keep = []
    if dense is not None:
        inp.kind = INPUT_DENSE
        if _is_device(dense):
            inp.mem = DEVICE
        else:
            dense = np.ascontiguousarray(dense, np.float32)
            inp.mem = HOST
        inp.dense = _ptr(dense, ctypes.c_float)
        keep.append(dense)
    elif pulses is not None:
        inp.kind = INPUT_PULSES
        inp.mem = HOST
        cells = np.ascontiguousarray(pulses[0], np.int32)
        beg = np.ascontiguousarray(pulses[1], np.int64)
        end = np.ascontiguousarray(pulses[2], np.int64)
        amp = np.ascontiguousarray(pulses[3], np.float32)
        inp.n_pulses = len(cells)
        inp.pulse_cell = _ptr(cells, ctypes.c_int32)
        inp.pulse_begin = _ptr(beg, ctypes.c_int64)
        inp.pulse_end = _ptr(end, ctypes.c_int64)
        inp.pulse_amp = _ptr(amp, ctypes.c_float)
        keep += [cells, beg, end, amp]
    else:
        inp.kind = INPUT_NONE
    return inp, keep


def ion_set_input(h, pulses=None):
    inp, keep = _input_struct(pulses=pulses)
    _check(lib().ion_set_input(h, ctypes.byref(inp)), h)


def ion_step(h, n_steps: int, dense=None):
    """Advance n_steps (asynchronous).  dense: [n_steps, n] evoked input for this call."""
    if dense is None:
        _check(lib().ion_step(h, int(n_steps), None), h)
    else:
        inp, keep = _input_struct(dense=dense)
        _check(lib().ion_step(h, int(n_steps), ctypes.byref(inp)), h)


def ion_sync(h):
    _check(lib().ion_sync(h), h)


def ion_read_state(h, n: int, field: int = FIELD_ALL) -> np.ndarray:
    out = np.zeros((NFIELDS, n) if field == FIELD_ALL else (n,), np.float32)
    _check(lib().ion_read_state(h, int(field), _ptr(out, ctypes.c_float), out.size), h)
    return out


def ion_write_state(h, state, field: int = FIELD_ALL):
    a = np.ascontiguousarray(state, np.float32)
    _check(lib().ion_write_state(h, int(field), _ptr(a, ctypes.c_float), a.size), h)


def ion_state_device_ptr(h, field: int) -> int:
    p = ctypes.c_void_p()
    _check(lib().ion_state_device_ptr(h, int(field), ctypes.byref(p)), h)
    return p.value


def ion_set_trace(h, stride: int, capacity: int):
    _check(lib().ion_set_trace(h, int(stride), int(capacity)), h)


def ion_read_trace(h, n: int, max_samples: int) -> np.ndarray:
    out = np.zeros((max_samples, n), np.float32)
    got = ctypes.c_int64()
    _check(lib().ion_read_trace(h, _ptr(out, ctypes.c_float), int(max_samples), ctypes.byref(got)), h)
    return out[:got.value]


def ion_read_trace_async(h, out, max_samples: int) -> int:
    """Queue the copy of the recorded samples into `out` (a pinned host tensor or a numpy
    array of at least max_samples x n floats, kept alive by the caller until
    ion_trace_wait); returns the number of samples queued."""
    got = ctypes.c_int64()
    ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    _check(lib().ion_read_trace_async(h, ctypes.c_void_p(ptr), int(max_samples), ctypes.byref(got)), h)
    return got.value


def ion_trace_wait(h):
    _check(lib().ion_trace_wait(h), h)


def ion_autotune(h, steps: int = 20) -> dict:
    """Time candidate launch shapes and keep the fastest; returns the chosen table."""
    t = ion_tune()
    _check(lib().ion_autotune(h, int(steps), ctypes.byref(t)), h)
    return {k: int(getattr(t, k)) for k, _ in ion_tune._fields_}


def ion_csr_layout(h) -> dict:
    """Bytes per stored edge the handle streams (index, weight) and whether V_dend is staged."""
    ib, wb, st = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().ion_csr_layout(h, ctypes.byref(ib), ctypes.byref(wb), ctypes.byref(st)), h)
    return {"index_bytes": ib.value, "weight_bytes": wb.value, "staged": st.value}


def ion_csr_bank_order(row_ptr, col, chunk: int, lanes_per_row: int) -> np.ndarray:
    """Bank-ordered edge permutation of a sorted host CSR (see the header)."""
    rp = np.ascontiguousarray(row_ptr, np.int32)
    c = np.ascontiguousarray(col, np.int32)
    perm = np.zeros(max(1, int(rp[-1])), np.int32)
    _check(lib().ion_csr_bank_order(len(rp) - 1, rp.ctypes.data, c.ctypes.data, int(chunk), int(lanes_per_row),
                                    perm.ctypes.data))
    return perm[:int(rp[-1])]


def ion_debug_fail_alloc(after: int):
    """Test hook: make the device allocation after the next `after` ones fail once (-1 disarms)."""
    lib().ion_debug_fail_alloc(int(after))


def ion_step_count(h) -> int:
    return int(lib().ion_step_count(h))


def ion_set_step_count(h, t: int):
    _check(lib().ion_set_step_count(h, int(t)), h)


def ion_launch_count(h) -> int:
    return int(lib().ion_launch_count(h))


def ion_last_error(h=None) -> str:
    m = lib().ion_last_error(h)
    return m.decode() if m else ""


def ion_destroy(h):
    if h:
        lib().ion_destroy(h)


# ---- single-launch primitives (torch CUDA tensors) -------------------------------------

def _stream(stream):
    return ctypes.c_void_p(stream) if stream else None


def ion_gj_dense(vdend, g: float, ic, kahan: bool = True, stream=None):
    _check(lib().ion_gj_dense(vdend.data_ptr(), int(vdend.numel()), float(g), ic.data_ptr(), int(bool(kahan)),
                              _stream(stream)))


def ion_gj_dense_noalloc(vdend, g: float, ic, kahan: bool = True, stream=None):
    """ion_gj_dense without any allocation (fixed scratch array of 65536 floats per device)."""
    _check(lib().ion_gj_dense_noalloc(vdend.data_ptr(), int(vdend.numel()), float(g), ic.data_ptr(),
                                      int(bool(kahan)), _stream(stream)))


def ion_gj_csr(vdend, row_ptr, col, w, g: float, ic, stream=None):
    _check(lib().ion_gj_csr(vdend.data_ptr(), int(vdend.numel()), row_ptr.data_ptr(), col.data_ptr(),
                            None if w is None else w.data_ptr(), float(g), ic.data_ptr(), _stream(stream)))


def ion_cell_update(state, n: int, ic=None, iapp=None, model=None, dt_ms: float = 0.05, stream=None):
    m = _model_struct(model)
    _check(lib().ion_cell_update(state.data_ptr(), int(n), None if ic is None else ic.data_ptr(),
                                 None if iapp is None else iapp.data_ptr(), ctypes.byref(m) if m else None,
                                 float(dt_ms), _stream(stream)))


def ion_probe_peak(what: int, iters: int = 4096, stream=None) -> float:
    """Measured ops/s of the SFU ex2 (what=0) or the FP32 FMA pipe (what=1)."""
    r = ctypes.c_double()
    _check(lib().ion_probe_peak(int(what), int(iters), _stream(stream), ctypes.byref(r)))
    return float(r.value)


# ---- surrogate ---------------------------------------------------------------------------

def ion_surrogate_train(n_samples=1_000_000, epochs=20, batch=1024, lr=1e-3, seed=0, v_lo=-100.0, v_hi=50.0,
                        ca_lo=1.0, ca_hi=20.0, stream=None):
    cfg = ion_train_cfg(int(n_samples), int(epochs), int(batch), float(lr), int(seed), float(v_lo), float(v_hi),
                        float(ca_lo), float(ca_hi), _stream(stream))
    w = ion_surrogate_weights()
    loss = ctypes.c_float()
    _check(lib().ion_surrogate_train(ctypes.byref(cfg), ctypes.byref(w), ctypes.byref(loss)))
    return w, float(loss.value)


_WFIELDS = ("w1", "b1", "w2", "b2", "w3", "b3")


def weights_from_dict(p: dict, in_shift=(0.0, 0.0), in_scale=(1.0, 1.0), out_shift=None, out_scale=None):
    """ion_surrogate_weights from arrays w1 (64,2), b1, w2 (64,64), b2, w3 (24,64), b3."""
    w = ion_surrogate_weights()
    for k in _WFIELDS:
        getattr(w, k)[:] = [float(v) for v in np.asarray(p[k], np.float32).reshape(-1)]
    w.in_shift[:] = list(map(float, in_shift))
    w.in_scale[:] = list(map(float, in_scale))
    w.out_shift[:] = [0.0] * MLP_OUT if out_shift is None else list(map(float, out_shift))
    w.out_scale[:] = [1.0] * MLP_OUT if out_scale is None else list(map(float, out_scale))
    return w


def weights_to_dict(w) -> dict:
    shapes = {"w1": (MLP_HID, MLP_IN), "b1": (MLP_HID,), "w2": (MLP_HID, MLP_HID), "b2": (MLP_HID,),
              "w3": (MLP_OUT, MLP_HID), "b3": (MLP_OUT,)}
    d = {k: np.array(getattr(w, k)[:], np.float32).reshape(shapes[k]) for k in _WFIELDS}
    for k in ("in_shift", "in_scale", "out_shift", "out_scale"):
        d[k] = np.array(getattr(w, k)[:], np.float32)
    return d


def ion_surrogate_grad(w, x, t, mask):
    """(loss, gradient dict) of one batch, computed by the training kernels."""
    x = np.ascontiguousarray(x, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    mask = np.ascontiguousarray(mask, np.float32)
    g = ion_surrogate_weights()
    L = ctypes.c_float()
    _check(lib().ion_surrogate_grad(ctypes.byref(w), _ptr(x, ctypes.c_float), _ptr(t, ctypes.c_float),
                                    _ptr(mask, ctypes.c_float), int(x.shape[0]), ctypes.byref(g), ctypes.byref(L)))
    return float(L.value), weights_to_dict(g)


def ion_surrogate_eval(w, V, ca) -> np.ndarray:
    V = np.ascontiguousarray(V, np.float32)
    ca = np.ascontiguousarray(ca, np.float32)
    out = np.zeros((len(V), MLP_OUT), np.float32)
    _check(lib().ion_surrogate_eval(ctypes.byref(w), _ptr(V, ctypes.c_float), _ptr(ca, ctypes.c_float), len(V),
                                    _ptr(out, ctypes.c_float)))
    return out


class Simulation:
    """Owning wrapper of one handle (destroyed with the object)."""

    def __init__(self, n, kind, **kw):
        self.n = int(n)
        self.h = ion_create(n, kind, **kw)

    def step(self, n_steps, dense=None):
        ion_step(self.h, n_steps, dense)

    def set_input(self, pulses=None):
        ion_set_input(self.h, pulses)

    def state(self, field=FIELD_ALL):
        return ion_read_state(self.h, self.n, field)

    def write(self, state, field=FIELD_ALL):
        ion_write_state(self.h, state, field)

    def sync(self):
        ion_sync(self.h)

    @property
    def t(self):
        return ion_step_count(self.h)

    @property
    def launches(self):
        return ion_launch_count(self.h)

    def close(self):
        if self.h:
            ion_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
