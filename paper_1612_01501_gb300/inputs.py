"""Seeded synthetic inputs for InfOli networks.

This module holds random numbers and graph structure only -- none of the method's
arithmetic -- so that the CUDA path and the FP64 oracle can be fed identical inputs.
Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its published
definition and used in counter form: the k-th draw of a stream with seed s is
mix(s + (k + 1) * 0x9E3779B97F4A7C15).

The workload shapes follow the paper's use cases (Sec. 2.3: dense all-to-all RGJ
networks and user-programmed connectivity; Sec. 3: 96-7680-cell networks, a short
current pulse as the validation input) at the sizes of the five benchmark
configurations (64 and 8192 dense cells, 65 536 sparse cells, a batch of 256 uneven
networks, and the surrogate's sampling ranges).
"""
from __future__ import annotations

import zlib

import numpy as np

DT_MS = 0.05                       # Sec. 2.2: delta = 50 us
GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, name: str) -> np.uint64:
    """Seed of the named sub-stream of `seed` (independent draws per purpose)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + GAMMA * np.uint64(1 + zlib.crc32(name.encode()))
    return _mix(np.array([z]))[0]


def splitmix64(seed, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+n-1 of the splitmix64 sequence started at `seed` (uint64)."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(seed) + k * GAMMA)


def uniform(seed, n: int, lo: float = 0.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [lo, hi): the top 53 bits of each draw scaled by 2^-53."""
    u = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


# ---- per-cell inputs -------------------------------------------------------------

def vdend_jitter(n: int, seed: int, amp_mv: float = 5.0) -> np.ndarray:
    """Per-cell offsets added to the default dendritic voltage, uniform in +-amp_mv."""
    return uniform(stream_seed(seed, "vdend_jitter"), n, -amp_mv, amp_mv)


def random_subset(n: int, frac: float, seed: int, name: str = "pulse_subset") -> np.ndarray:
    """Sorted int32 indices of the cells whose draw falls below `frac` (about frac * n)."""
    u = uniform(stream_seed(seed, name), n)
    return np.nonzero(u < frac)[0].astype(np.int32)


def step_of_ms(t_ms: float) -> int:
    return int(round(t_ms / DT_MS))


def pulses(cells, t0_ms: float, t1_ms: float, amp: float):
    """Pulse table (cell int32, t_begin int64, t_end int64, amp float32), steps [t0, t1)."""
    cells = np.asarray(cells, np.int32)
    m = len(cells)
    return (cells, np.full(m, step_of_ms(t0_ms), np.int64), np.full(m, step_of_ms(t1_ms), np.int64),
            np.full(m, amp, np.float32))


def pulse_windows(cells, windows, amp: float):
    """One pulse per cell and window [(t0_ms, t1_ms), ...], concatenated window by window."""
    P = [pulses(cells, a, b, amp) for a, b in windows]
    return tuple(np.concatenate([p[q] for p in P]) for q in range(4))


# ---- connectivity ----------------------------------------------------------------

def random_symmetric_csr(n: int, k: int, seed: int):
    """Symmetric random graph, no self loops, rows sorted ascending (int32 CSR).

    Each cell draws k/2 partners uniformly from the other n-1 cells; every drawn pair
    is stored in both directions and duplicates are merged, so the mean degree is close
    to k (the exact nnz is whatever the draw gives).
    """
    if n < 2 or k <= 0:
        return np.zeros(n + 1, np.int32), np.zeros(0, np.int32)
    half = max(1, k // 2)
    src = np.repeat(np.arange(n, dtype=np.int64), half)
    u = uniform(stream_seed(seed, "csr_partners"), n * half)
    dst = np.minimum((u * (n - 1)).astype(np.int64), n - 2)
    dst = dst + (dst >= src)                      # skip the cell itself
    key = np.concatenate([src * n + dst, dst * n + src])
    key = np.unique(key)                          # sorted by (row, col), duplicates merged
    rows = (key // n).astype(np.int64)
    cols = (key % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    if row_ptr[-1] >= 2 ** 31:
        raise ValueError("graph too large for int32 CSR")
    return row_ptr.astype(np.int32), cols


def junction_weight(g_ref: float, neighbours: float) -> float:
    """Per-junction weight for a network whose cells have `neighbours` partners.

    The coupling is quoted for a 64-partner cell (0.04 mS/cm^2 for the 64-cell
    all-to-all network); larger networks keep the same total coupling per cell,
    g = g_ref * 64 / neighbours (the 8192-cell dense network uses 0.04 / 8192 * 64).
    """
    return float(np.float32(g_ref * 64.0 / neighbours))


# ---- the five workloads ----------------------------------------------------------

def config(name: str, k: int | None = None, n: int | None = None) -> dict:
    """Synthetic input bundle of one workload.

    Keys: n, kind ('dense' | 'csr' | 'ngj'), g (dense weight), row_ptr/col/w (CSR), jitter
    (added to V_dend), pulses (or None), n_steps.
    """
    if name == "c1":   # 64 cells all-to-all, g_c = 0.04, pulse 6 uA/cm^2 to cells 0-7 at 100-110 ms
        n = 64
        return dict(name=name, n=n, kind="dense", g=float(np.float32(0.04)), jitter=vdend_jitter(n, 0),
                    pulses=pulses(np.arange(8), 100.0, 110.0, 6.0), n_steps=20000)
    if name == "c2":   # 8192 cells all-to-all, g_c = 0.04 / N * 64, I_app = 0, 200 ms
        n = 8192
        return dict(name=name, n=n, kind="dense", g=junction_weight(0.04, n), jitter=vdend_jitter(n, 1),
                    pulses=None, n_steps=4000)
    if name == "c3":   # 65 536 cells, random symmetric CSR with k neighbours, seed 2
        n = 65536
        k = 100 if k is None else k
        row_ptr, col = random_symmetric_csr(n, k, 2)
        w = np.full(len(col), junction_weight(0.04, k), np.float32)
        sub = random_subset(n, 0.2, 2)
        return dict(name=f"{name}_k{k}", n=n, kind="csr", k=k, row_ptr=row_ptr, col=col, w=w,
                    jitter=vdend_jitter(n, 2), pulses=pulses(sub, 50.0, 60.0, 6.0), n_steps=4000)
    if name == "k3":   # uncoupled cells (NGJ, Sec. 2.3.3): the cell update alone, default 2^22 cells
        n = (1 << 22) if n is None else n
        sub = random_subset(n, 0.2, 3)
        return dict(name=f"{name}_n{n}", n=n, kind="ngj", jitter=vdend_jitter(n, 3),
                    pulses=pulses(sub, 5.0, 15.0, 6.0), n_steps=400)
    if name == "c2_matrix":   # 8192 cells, every pair weighted: W_ij = g_c(N) * U(0, 2), seed 1
        n = 8192
        g = junction_weight(0.04, n)
        W = (g * uniform(stream_seed(1, "matrix_w"), n * n, 0.0, 2.0)).astype(np.float32).reshape(n, n)
        return dict(name=name, n=n, kind="matrix", W=W, jitter=vdend_jitter(n, 1), pulses=None, n_steps=4000)
    if name == "c1_spiking":   # c1 with every cell pulsed at 100-110, 400-410 and 700-710 ms
        n = 64
        cells = np.arange(n)
        return dict(name=name, n=n, kind="dense", g=float(np.float32(0.04)), jitter=vdend_jitter(n, 0),
                    pulses=pulse_windows(cells, [(100.0, 110.0), (400.0, 410.0), (700.0, 710.0)], 6.0),
                    n_steps=20000)
    if name == "c3_spiking":   # the c3 network with every cell pulsed at 50-60 and 500-510 ms
        base = config("c3", k=k)
        base.update(name=f"c3_spiking_k{base['k']}",
                    pulses=pulse_windows(np.arange(base["n"]), [(50.0, 60.0), (500.0, 510.0)], 6.0))
        return base
    if name == "validation":   # Sec. 3: identical cells, a pulse to all cells for 500 steps
        n = 64
        return dict(name=name, n=n, kind="dense", g=float(np.float32(0.04)), jitter=np.zeros(n),
                    pulses=pulses(np.arange(n), 100.0, 125.0, 6.0), n_steps=20000)
    raise KeyError(name)


def batch_specs(n_nets: int = 256, seed_base: int = 1000, n_lo: int = 32, n_hi: int = 4096,
                k_lo: int = 8, k_hi: int = 256, g_lo: float = 0.01, g_hi: float = 0.08):
    """Specs of the batched sweep: sizes log-uniform in [n_lo, n_hi], even-numbered
    networks dense and odd-numbered CSR with k uniform in [k_lo, k_hi], g_c uniform in
    [g_lo, g_hi], network b seeded with seed_base + b."""
    out = []
    for b in range(n_nets):
        s = seed_base + b
        u = uniform(stream_seed(s, "batch_spec"), 3)
        n = int(round(np.exp(np.log(n_lo) + u[0] * (np.log(n_hi) - np.log(n_lo)))))
        n = min(max(n, n_lo), n_hi)
        g_ref = g_lo + u[1] * (g_hi - g_lo)
        if b % 2 == 0:
            out.append(dict(n=n, kind="dense", k=n, g_ref=g_ref, seed=s))
        else:
            k = int(min(k_lo + int(u[2] * (k_hi - k_lo + 1)), k_hi))
            out.append(dict(n=n, kind="csr", k=k, g_ref=g_ref, seed=s))
    return out


def batch_network(spec: dict) -> dict:
    """Input bundle of one network of the batched sweep (pulse: cells [0, ceil(n/8))
    get 6 uA/cm^2 from 20 to 30 ms)."""
    n, s = spec["n"], spec["seed"]
    bundle = dict(n=n, kind=spec["kind"], jitter=vdend_jitter(n, s),
                  pulses=pulses(np.arange((n + 7) // 8), 20.0, 30.0, 6.0))
    if spec["kind"] == "dense":
        bundle["g"] = junction_weight(spec["g_ref"], n)
    else:
        k = min(spec["k"], n - 1)
        row_ptr, col = random_symmetric_csr(n, k, s)
        bundle.update(row_ptr=row_ptr, col=col, w=np.full(len(col), junction_weight(spec["g_ref"], k), np.float32))
    return bundle


def surrogate_samples(n: int, seed: int, v_lo: float = -100.0, v_hi: float = 50.0,
                      ca_lo: float = 1.0, ca_hi: float = 20.0):
    """Training inputs of the rate-function surrogate: V uniform in [v_lo, v_hi] mV and
    [Ca] log-uniform in [ca_lo, ca_hi]; returned as float32 arrays (V, Ca)."""
    v = uniform(stream_seed(seed, "surrogate_v"), n, v_lo, v_hi)
    lc = uniform(stream_seed(seed, "surrogate_ca"), n, np.log(ca_lo), np.log(ca_hi))
    return v.astype(np.float32), np.exp(lc).astype(np.float32)
