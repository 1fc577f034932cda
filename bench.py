"""Benchmark of the InfOli hot path on one GB300 (or N independent replicas).

Default workload: the 8192-cell all-to-all network (RGJ at 100 % density), FP32 state in
SoA layout, g_c = 0.04 / N * 64, V_dend jittered +-5 mV from seed 1, no evoked input.  One
bench step simulates 200 ms = 4000 time steps of 50 us from the same initial state.
Metric: cell-timesteps/s (and gap-junction pair evaluations/s, N^2 per time step).

`--workload` selects another configuration for a secondary line (c1: 64 dense cells for
1 s; c3_k10 / c3_k100 / c3_k1000: 65 536 cells with random symmetric CSR connectivity;
c4: 256 uneven networks in one batch; c5: the k = 100 network for 1 s with the learned
rate-function surrogate against the exact FP32 method; k3: the cell update alone on 2^22
uncoupled cells, with a sweep of sizes from 2^16; c2_sgj: the 8192-cell network with the
simplified linear junctions of the SGJ use case; c2_matrix: 8192 cells with an N x N
weight matrix streamed from HBM every step).
`--impl reference` times the FP64 CPU oracle instead (a bounded sample, all host cores).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-timesteps/s"
L2_FLUSH_BYTES = 512 << 20           # > 129 MB L2
WORKLOADS = {
    "c2": dict(name="c2_dense_8192_allToAll_200ms", cfg="c2", steps=4000),
    "c1": dict(name="c1_dense_64_allToAll_1s", cfg="c1", steps=20000),
    "c3_k10": dict(name="c3_csr_65536_k10_200ms", cfg="c3", k=10, steps=4000),
    "c3_k100": dict(name="c3_csr_65536_k100_200ms", cfg="c3", k=100, steps=4000),
    "c3_k1000": dict(name="c3_csr_65536_k1000_200ms", cfg="c3", k=1000, steps=4000),
    "c4": dict(name="c4_batch_256_nets_logU32-4096_half_dense_100ms", cfg="c4", steps=2000),
    "c5": dict(name="c5_surrogate_csr_65536_k100_1s", cfg="c3", k=100, steps=20000),
    "k3": dict(name="k3_cell_update_ngj_4194304_20ms", cfg="k3", n=1 << 22, steps=400),
    "c2_sgj": dict(name="c2_sgj_dense_8192_linearGJ_200ms", cfg="c2", steps=4000, sgj=True),
    "c2_matrix": dict(name="c2_matrix_dense_8192_NxN_weights_100ms", cfg="c2_matrix", steps=2000),
    "rt": dict(name="rt_largest_real_time_network_per_use_case", cfg="rt", steps=2000),
}
# The use cases of the paper's real-time table (Sec. 3.1.1, Table "RT"): junction model
# (RGJ: the exponential junction, SGJ: linear, NGJ: none), connection density, the model
# exponent of the step time in N (pairs or edges grow as N^2, the rest as N) and a first
# size to measure.
RT_CASES = (("RGJ", 1.00, 2, 16384), ("RGJ", 0.75, 2, 9216), ("RGJ", 0.50, 2, 11264), ("RGJ", 0.25, 2, 15360),
            ("SGJ", 1.00, 1, 1 << 20), ("SGJ", 0.75, 2, 6144), ("SGJ", 0.50, 2, 7168), ("SGJ", 0.25, 2, 10240),
            ("NGJ", 0.00, 1, 1 << 21))
RT_LIMIT_US = 50.0   # one time step of 50 us computed in at most 50 us (Sec. 2.2)
K3_SWEEP = (1 << 16, 1 << 18, 1 << 20, 1 << 22)
# DRAM bytes (read + write) per launch of the line's dominant kernel, from one ncu capture
# of that kernel in its current form (the summaries under profiles/ give the commands);
# None where no capture matches the line's kernel and shape
# (bytes per launch, source, launch shape the capture used: autotuner fields that must match)
TRAFFIC = {   # an entry is removed when its kernel changes, until it is captured again
    ("c2", "dense_step_kernel"): (532224, "profiles/dense_step_kernel_c2_8192.md",
                                  dict(dense_rows_per_warp=4, dense_warps=28, dense_col_splits=2)),
    ("k3", "cell_step_kernel"): (275259392 + 241500416, "profiles/cell_step_kernel_k3_4194304.md", {}),
    ("c3_k10", "csr_step_kernel"): (7211520, "profiles/csr_step_kernel_c3_k10.md",
                                    dict(csr_lanes_per_row=1, csr_rows_per_cta=128)),
    # captured at 32 lanes per row: the DRAM bytes are those of the padded layout (each
    # index byte and state word read once), the same for any lane count
    ("c3_k1000", "csr_chunk_step_kernel"): (135862784 + 2681600, "profiles/csr_chunk_step_kernel_c3_k1000.md",
                                            dict(csr_staging=2)),
    # captured with 8-row dense tiles: the DRAM bytes (state, CSR indices; V_dend tiles
    # come from L2) are read once per step whatever the tile shape
    ("c3_k100", "csr_chunk_step_kernel"): (18866432, "profiles/csr_chunk_step_kernel_c3_k100.md", dict(csr_staging=2)),
    ("c2_sgj", "sgj_dense_update_kernel"): (517376, "profiles/sgj_dense_update_kernel_c2_sgj_8192.md", {}),
    ("c4", "batch_step_kernel"): (44903168 + 71936, "profiles/batch_step_kernel_c4.md", {}),
    ("c5", "surrogate_tc_kernel"): (4612352, "profiles/surrogate_tc_kernel_c5.md", {}),
    # captured at one row per warp: every weight is streamed once whatever the rows per warp
    ("c2_matrix", "matrix_step_kernel"): (272269312 + 5144320, "profiles/matrix_step_kernel_c2_matrix_8192.md", {}),
}


def traffic_for(key, kernel, variant, tune, dense_shape=""):
    """(DRAM bytes per launch, summary) of the line's kernel from TRAFFIC, or None: only for
    the graph-replayed variants (the surrogate line's included) and only when the launch
    shape the line runs (the autotuner's table, or --dense-shape) matches every field the
    capture fixes."""
    tr = TRAFFIC.get((key, kernel))
    if tr is None or variant not in ("graph", "exact", "surrogate"):
        return None
    shape = dict(tune or {})
    if dense_shape:
        R, W, GJ = (int(x) for x in dense_shape.split(","))
        shape.update(dense_rows_per_warp=R, dense_warps=W, dense_col_splits=GJ)
    if not all(shape.get(f) == v for f, v in tr[2].items()):
        return None
    return tr[0], tr[1]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--sim-steps", type=int, default=0, help="time steps per bench step (0: the workload's)")
    ap.add_argument("--variant", default="auto",
                    choices=["auto", "graph", "persistent", "persistent_half", "graph_csr_as_given", "graph_csr_half"])
    ap.add_argument("--no-extra", action="store_true", help="skip the CPU baseline and the e2e leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch shapes")
    ap.add_argument("--dense-shape", default="", help="R,W,GJ: a fixed dense launch shape (no autotuning)")
    return ap.parse_args()


def replica_reduce(ms_local: float, cells_local: float, pg=None):
    """Whole-job figures of N independent replicas: the slowest rank's time bounds the job
    and the cells of all ranks count (weak scaling: every rank runs a full workload).
    Returns (value = total cells / max time, max time in ms).  pg: torch.distributed or None."""
    ms, cells = float(ms_local), float(cells_local)
    if pg is not None:
        import torch
        dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        c = torch.tensor([cells], dtype=torch.float64, device=dev)
        pg.all_reduce(c, op=pg.ReduceOp.SUM)
        ms, cells = float(t.item()), float(c.item())
    return cells / (ms * 1e-3), ms


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [[x.strip() for x in line.split(",")] for line in open(self.f.name)]
        rows = [r for r in rows if len(r) >= 9]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        num = lambda x: x.replace(".", "").isdigit()
        sm = [float(r[1]) for r in rows if num(r[1])]
        mx = [float(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def hbm_peak():
    """Measured copy bandwidth of this machine's GB300 (GB/s), else the earlier measurement."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6792.4


def k3_sweep(ion, torch, stream, flush, sim_steps, warmup, known, peak):
    """Cell update alone (uncoupled cells) at each size of K3_SWEEP: us per time step and
    GB/s of algorithmic bytes (132 B of state + the pulse table per cell).  Sizes already
    timed are passed in `known` ({n: seconds per time step})."""
    from paper_1612_01501_gb300 import inputs
    out = {}
    for n in K3_SWEEP:
        cfg = inputs.config("k3", n=n)
        per = known.get(n)
        if per is None:
            S0 = ion.ion_default_state(n)
            S0[0] = (S0[0].astype(np.float64) + cfg["jitter"]).astype(np.float32)
            with ion.Simulation(n, ion.NO_GJ, init_state=S0, stream=stream, graph_steps=100) as sim:
                sim.set_input(cfg["pulses"])
                for _ in range(warmup):
                    sim.step(sim_steps)
                reps, ms = 3, 0.0
                for r in range(reps):
                    flush.fill_(float(r))
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    sim.step(sim_steps)
                    b.record()
                    torch.cuda.synchronize()
                    ms += a.elapsed_time(b)
                sim.sync()
            per = ms * 1e-3 / (reps * sim_steps)
        by = 132 * n + 4 * (n + 1) + 20 * len(cfg["pulses"][0])
        out[str(n)] = {"us_per_timestep": per * 1e6, "gb_per_s": by / per / 1e9, "frac": by / per / 1e9 / peak,
                       "state_mb": 80 * n / 1e6}
    return out


class SpikeLog:
    """Spike times of every cell from streamed V_axon samples: an upward crossing of 0 mV
    (the first sample at or above it), re-armed once V_axon falls below -30 mV."""

    def __init__(self, n):
        self.armed = np.ones(n, bool)
        self.t = 0
        self.cells, self.steps = [], []

    def feed(self, trace):
        for row in trace:
            fire = self.armed & (row >= 0.0)
            idx = np.flatnonzero(fire)
            if len(idx):
                self.cells.append(idx)
                self.steps.append(np.full(len(idx), self.t, np.int64))
            self.armed = (self.armed & ~fire) | (~self.armed & (row < -30.0))
            self.t += 1

    def sorted(self):
        c = np.concatenate(self.cells) if self.cells else np.zeros(0, np.int64)
        t = np.concatenate(self.steps) if self.steps else np.zeros(0, np.int64)
        o = np.lexsort((t, c))
        return c[o], t[o]


def compare_runs(ion, sim_a, sim_b, reset, n, steps, chunk=2000):
    """Run two handles side by side from the same state with V_axon traced every step;
    return the trace error and the spike-time agreement of b against a.  Spikes are
    matched in order within each cell whose spike counts agree."""
    logs = [SpikeLog(n), SpikeLog(n)]
    sq, mx, cnt = 0.0, 0.0, 0
    for sim in (sim_a, sim_b):
        reset(sim)
        ion.ion_set_trace(sim.h, 1, chunk)
    done = 0
    while done < steps:
        c = min(chunk, steps - done)
        tr = []
        for sim, log in zip((sim_a, sim_b), logs):
            sim.step(c)
            t = ion.ion_read_trace(sim.h, n, c)
            log.feed(t)
            tr.append(t)
        d = tr[0].astype(np.float64) - tr[1]
        sq += float((d * d).sum())
        mx = max(mx, float(np.abs(d).max()))
        cnt += d.size
        done += c
    for sim in (sim_a, sim_b):
        ion.ion_set_trace(sim.h, 0, 0)
    (ca, ta), (cb, tb) = logs[0].sorted(), logs[1].sorted()
    na, nb = np.bincount(ca, minlength=n), np.bincount(cb, minlength=n)
    same = na == nb
    da = np.abs(ta[same[ca]] - tb[same[cb]])
    return {"v_axon_rms_mV": (sq / max(cnt, 1)) ** 0.5, "v_axon_max_abs_mV": mx,
            "spikes_exact": int(len(ca)), "spikes_surrogate": int(len(cb)),
            "spiking_cells_exact": int((na > 0).sum()),
            "cells_same_spike_count_frac": float(same.mean()),
            "spikes_within_1_step_frac": float((da <= 1).sum() / max(len(ca), 1)),
            "matched_max_abs_dstep": int(da.max()) if len(da) else 0,
            "matched_mean_abs_dstep": float(da.mean()) if len(da) else 0.0,
            "compared_steps": int(steps)}


def rt_graph(torch, n: int, density: float, seed: int, device: str = "cuda"):
    """Symmetric random graph of the real-time table: each unordered pair {i, j} is a
    junction with probability `density`, decided by a 32-bit integer hash of (seed, i, j)
    (the same for both orders); no self loops; rows sorted.  Drawn on the device in blocks
    of rows and returned as host int32 CSR."""
    dev = torch.device(device)
    M = 0xFFFFFFFF
    thr = int(density * 2 ** 32)
    j = torch.arange(n, device=dev, dtype=torch.int64)[None, :]
    counts, cols = [], []
    B = max(1, (1 << 26) // n)
    for i0 in range(0, n, B):
        i = torch.arange(i0, min(n, i0 + B), device=dev, dtype=torch.int64)[:, None]
        h = (torch.minimum(i, j) * n + torch.maximum(i, j) + seed * 0x9E3779B1) & M
        h = h ^ (h >> 16)
        h = (h * 0x7FEB352D) & M
        h = h ^ (h >> 15)
        h = (h * 0x846CA68B) & M
        h = h ^ (h >> 16)
        m = (h < thr) & (i != j)
        counts.append(m.sum(dim=1))
        cols.append(torch.nonzero(m)[:, 1].to(torch.int32))
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(torch.cat(counts), 0)
    return row_ptr.to(torch.int32).cpu().numpy(), torch.cat(cols).cpu().numpy()


def rt_search(time_at, n0, p, limit=RT_LIMIT_US, quantum=64):
    """The largest size N (a multiple of `quantum`) with time_at(N) <= limit, for a step time
    that grows with N.  Measure n0; then up to four model steps: fit t(N) = 3 + a N^p to the
    last measurement and measure the size predicted for 0.98 x limit; then bisect the
    bracket [largest size within the limit, smallest size over it] until it is within 2 %
    or one quantum (halving or growing by 10 % while one side is missing).  Returns
    (largest size within the limit or None, {size: time} of every measurement)."""
    tried = {}

    def measure(N):
        N = max(quantum, int(round(N / float(quantum))) * quantum)
        if N not in tried:
            tried[N] = time_at(N)
        return N, tried[N]

    def sides():
        return [k for k, v in tried.items() if v <= limit], [k for k, v in tried.items() if v > limit]

    N, t = measure(n0)
    for _ in range(4):   # model steps
        a = max(t - 3.0, 0.05) / float(N) ** p
        N, t = measure(((0.98 * limit - 3.0) / a) ** (1.0 / p))
        ok, bad = sides()
        if ok and bad and min(bad) <= 1.02 * max(ok):
            break
    for _ in range(6):   # bisection
        ok, bad = sides()
        if not ok:
            measure(min(tried) // 2)
            continue
        if not bad:
            measure(max(ok) * 1.1)
            continue
        lo, hi = max(ok), min(bad)
        if hi <= 1.02 * lo or hi - lo <= quantum:
            break
        measure((lo + hi) / 2)
    ok, _ = sides()
    return (max(ok) if ok else None), tried


def rt_table(ion, torch, stream, warmup):
    """Largest network whose time step is computed within 50 us, per use case of the
    paper's real-time table, on one GPU, steps back to back (CUDA-graph replay).  Each
    size is measured over 2000 steps after `warmup` x 200 untimed ones (rt_search picks
    the sizes).  Also: per-step latency with the host in the loop at that size (each
    step's evoked input written from host memory, V_axon read back)."""
    from paper_1612_01501_gb300 import inputs
    rows = []
    for model, dens, p, n0 in RT_CASES:
        launches = {}

        def time_at(N):
            flags = ion.FLAG_KAHAN | (ion.FLAG_SGJ if model == "SGJ" else 0)
            kw = {}
            if model == "NGJ":
                kind = ion.NO_GJ
            elif dens >= 1.0:
                kind, kw = ion.DENSE_UNIFORM, dict(g=inputs.junction_weight(0.04, N))
            else:
                rp, col = rt_graph(torch, N, dens, seed=5)
                kind = ion.CSR
                kw = dict(row_ptr=rp, col=col, w=np.full(len(col), inputs.junction_weight(0.04, dens * N),
                                                       np.float32))
            S0 = ion.ion_default_state(N)
            S0[0] = (S0[0].astype(np.float64) + inputs.vdend_jitter(N, 1)).astype(np.float32)
            with ion.Simulation(N, kind, init_state=S0, stream=stream, graph_steps=100, flags=flags, **kw) as sim:
                for _ in range(max(1, warmup)):
                    sim.step(200)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                l0 = sim.launches
                a.record()
                sim.step(2000)
                b.record()
                torch.cuda.synchronize()
                sim.sync()
                launches[N] = sim.launches - l0
                return a.elapsed_time(b) * 1e3 / 2000

        best, tried = rt_search(time_at, n0, p)
        row = {"use_case": f"{model} ({int(round(dens * 100))} %)", "max_cells": best,
               "us_per_timestep": tried.get(best), "launches_timed": launches.get(best, 0),
               "measured_us_per_timestep": {str(k): round(v, 3) for k, v in sorted(tried.items())}}
        if best is not None:
            row.update(host_loop_latency(ion, torch, stream, model, dens, best))
        rows.append(row)
    return rows


def host_loop_latency(ion, torch, stream, model, dens, N, n_steps=1000):
    """Wall time of one closed-loop step at N cells: the step's evoked input (N floats)
    from host memory, one time step, V_axon (N floats) back to the host."""
    from paper_1612_01501_gb300 import inputs
    flags = ion.FLAG_KAHAN | (ion.FLAG_SGJ if model == "SGJ" else 0)
    kw = {}
    if model == "NGJ":
        kind = ion.NO_GJ
    elif dens >= 1.0:
        kind, kw = ion.DENSE_UNIFORM, dict(g=inputs.junction_weight(0.04, N))
    else:
        rp, col = rt_graph(torch, N, dens, seed=5)
        kind = ion.CSR
        kw = dict(row_ptr=rp, col=col, w=np.full(len(col), inputs.junction_weight(0.04, dens * N), np.float32))
    iapp = torch.zeros((1, N), dtype=torch.float32).pin_memory()
    out = torch.empty(N, dtype=torch.float32).pin_memory()
    lat = []
    with ion.Simulation(N, kind, stream=stream, graph_steps=100, flags=flags, **kw) as sim:
        h = sim.h
        for k in range(n_steps + 50):
            t0 = time.perf_counter()
            ion.ion_step(h, 1, dense=iapp.numpy())
            ion._check(ion.lib().ion_read_state(h, ion.FIELD["V_axon"], ion._ptr(out, ion.ctypes.c_float), N), h)
            t1 = time.perf_counter()
            if k >= 50:
                lat.append((t1 - t0) * 1e6)
        sim.sync()
    lat.sort()
    return {"host_loop_us_median": lat[len(lat) // 2], "host_loop_us_p99": lat[int(0.99 * len(lat))],
            "host_loop_bytes_per_step": 8 * N}


def run_rt(args, ion, torch, rank, world, local, pg):
    """The real-time table (one JSON line): the line's value is the cell-timestep rate of
    the largest real-time RGJ network at 100 % density; `rt_table` holds every use case."""
    stream = torch.cuda.current_stream().cuda_stream
    if pg:
        pg.barrier()
    clocks = Clocks(local)
    clocks.start()
    rows = rt_table(ion, torch, stream, args.warmup)
    ck = clocks.stop()
    head = rows[0]
    us = head["us_per_timestep"] or float("nan")
    # cell-timesteps of the 2000 timed steps at that size, slowest replica's time
    value, _ = replica_reduce(us * 2000 * 1e-3, (head["max_cells"] or 0) * 2000, pg)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": 2000, "warmup": args.warmup, "ms_per_step": us * 1e-3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOADS["rt"]["name"], "parallelism": f"replicas x{world}",
                           "l2": "not flushed: each size runs 2000 consecutive time steps, as in real time"},
                "real_time": {"limit_us": RT_LIMIT_US, "criterion": "one 50 us time step computed in <= 50 us"},
                "rt_table": rows, "clocks": ck,
                "gpu_launches": sum(r.get("launches_timed", 0) for r in rows)}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def load_workload(key):
    """Input bundle of a workload (seeded, synthetic) as the oracle and the GPU see it."""
    from paper_1612_01501_gb300 import inputs
    w = WORKLOADS[key]
    if w["cfg"] == "c4":
        nets = [inputs.batch_network(sp) for sp in inputs.batch_specs()]
        off, cells, beg, end, amp = 0, [], [], [], []
        for b in nets:
            p = b["pulses"]
            cells.append(p[0] + off); beg.append(p[1]); end.append(p[2]); amp.append(p[3])
            off += b["n"]
        pul = (np.concatenate(cells).astype(np.int32), np.concatenate(beg), np.concatenate(end), np.concatenate(amp))
        return dict(n=off, kind="batch", nets=nets, jitter=np.concatenate([b["jitter"] for b in nets]), pulses=pul)
    return inputs.config(w["cfg"], k=w.get("k"), n=w.get("n"))


def cpu_baseline(key, sample_steps, single_thread_steps=0):
    """FP64 oracle on all host cores: `sample_steps` time steps of the workload (and, if
    single_thread_steps > 0, that many more on one core, reported beside it)."""
    import oracle as O
    cfg = load_workload(key)
    threads = O.max_threads()
    jobs = cfg["nets"] if cfg["kind"] == "batch" else [cfg]
    runs = []
    for b in jobs:
        S = O.default_state(b["n"])
        S[O.F["V_dend"]] += b["jitter"]
        S = S.astype(np.float32).astype(np.float64)
        kind = {"dense": O.DENSE, "csr": O.CSR, "ngj": O.NOGJ, "matrix": O.MATRIX}[b["kind"]]
        if WORKLOADS[key].get("sgj"):
            kind = {O.DENSE: O.DENSE_SGJ, O.CSR: O.CSR_SGJ}[kind]
        wt = b.get("W") if b["kind"] == "matrix" else b.get("w")
        kw = dict(kind=kind, g=b.get("g", 0.0), row_ptr=b.get("row_ptr"), col=b.get("col"),
                  w=None if wt is None else wt.astype(np.float64), threads=threads)
        runs.append((S, kw))
    O.run(runs[0][0], 1, **runs[0][1])        # warm caches and the thread pool
    t0 = time.perf_counter()
    for S, kw in runs:
        O.run(S, sample_steps, **kw)
    dt = time.perf_counter() - t0
    v = cfg["n"] * sample_steps / dt
    out = {"value": v, "unit": METRIC, "cores": threads, "kind": "oracle",
           "sample": f"{sample_steps} time steps of {WORKLOADS[key]['name']} (FP64, OpenMP over cells)",
           "seconds": dt}
    if single_thread_steps > 0:
        t0 = time.perf_counter()
        for S, kw in runs:
            O.run(S, single_thread_steps, **dict(kw, threads=1))
        d1 = time.perf_counter() - t0
        out["single_core"] = {"value": cfg["n"] * single_thread_steps / d1, "unit": METRIC, "cores": 1,
                              "sample": f"{single_thread_steps} time steps, one thread"}
    return out


def reference_sample_steps(key):
    return {"c2": 8, "c1": 2000, "c4": 3, "k3": 3, "c2_matrix": 4}.get(key, 20)


def run_reference(args, rank):
    """The reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    k = reference_sample_steps(args.workload)
    runs = [cpu_baseline(args.workload, k) for _ in range(args.warmup + args.steps)][args.warmup:]
    t = sum(r["seconds"] for r in runs)
    n = load_workload(args.workload)["n"]
    v = n * k * len(runs) / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(runs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["name"], "n_cells": n, "timesteps_per_step": k,
                       "note": f"bounded sample: {k} time steps per bench step"},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": runs[0]["cores"], "kind": "oracle",
                             "sample": f"{k} time steps of {WORKLOADS[args.workload]['name']} per bench step"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    torch.cuda.set_device(local)
    # a dedicated stream: the library's steps and the timing events must share it
    # (the default stream's handle is 0, which the library reads as "no stream given")
    torch.cuda.set_stream(torch.cuda.Stream())
    from paper_1612_01501_gb300 import build as B
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
        if rank == 0:
            B.build()
        pg.barrier()
    else:
        B.build()
    from paper_1612_01501_gb300 import ion

    key = args.workload
    wl = WORKLOADS[key]
    if key == "rt":
        return run_rt(args, ion, torch, rank, world, local, pg)
    sim_steps = args.sim_steps or wl["steps"]
    cfg = load_workload(key)
    n = cfg["n"]
    dense = cfg["kind"] == "dense"
    batch = cfg["kind"] == "batch"
    ngj = cfg["kind"] == "ngj"
    S0 = ion.ion_default_state(n)
    S0[0] = (S0[0].astype(np.float64) + cfg["jitter"]).astype(np.float32)
    tune_table = None
    stream = torch.cuda.current_stream().cuda_stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    surrogate = None
    surrogate_info = {}
    if key == "c5":
        t0 = time.perf_counter()
        surrogate, loss = ion.ion_surrogate_train(n_samples=1 << 20, epochs=100, batch=2048, lr=2e-3, seed=7,
                                                  v_lo=-100.0, v_hi=50.0, ca_lo=1.36, ca_hi=13.5, stream=stream)
        surrogate_info = {"train_seconds": time.perf_counter() - t0, "train_samples": 1 << 20, "epochs": 100,
                          "final_loss_normalised": loss}

    def make_sim(flags):
        nonlocal tune_table
        if wl.get("sgj"):
            flags |= ion.FLAG_SGJ
        if batch:
            specs = [dict(n=b["n"], kind=ion.DENSE_UNIFORM, g=b["g"]) if b["kind"] == "dense" else
                     dict(n=b["n"], kind=ion.CSR, row_ptr=b["row_ptr"], col=b["col"], w=b["w"]) for b in cfg["nets"]]
            sim = ion.Simulation.__new__(ion.Simulation)
            sim.n = n
            sim.h = ion.ion_create_batch(specs, init_state=S0, stream=stream, graph_steps=100, flags=flags)
            sim.set_input(cfg["pulses"])
            if not args.no_autotune:
                tune_table = ion.ion_autotune(sim.h, 20)  # project-written autotuner: time the tile shapes
            return sim
        if ngj:
            kind, kw = ion.NO_GJ, {}
        elif cfg["kind"] == "matrix":
            kind, kw = ion.DENSE_MATRIX, dict(w=cfg["W"])
        elif dense:
            kind, kw = ion.DENSE_UNIFORM, dict(g=cfg["g"])
        else:
            kind, kw = ion.CSR, dict(row_ptr=cfg["row_ptr"], col=cfg["col"], w=cfg["w"])
        if flags & ion.FLAG_SURROGATE:
            kw["surrogate"] = surrogate
        if args.dense_shape and kind == ion.DENSE_UNIFORM:
            R, W, GJ = (int(x) for x in args.dense_shape.split(","))
            kw["tune"] = dict(dense_rows_per_warp=R, dense_warps=W, dense_col_splits=GJ)
        sim = ion.Simulation(n, kind, init_state=S0, stream=stream, graph_steps=100, flags=flags, **kw)
        if cfg.get("pulses") is not None:
            sim.set_input(cfg["pulses"])
        if not (flags & (ion.FLAG_PERSISTENT | ion.FLAG_SURROGATE)) and kind in (ion.DENSE_UNIFORM, ion.CSR,
                                                                                 ion.DENSE_MATRIX) \
                and not args.no_autotune and not args.dense_shape:
            tune_table = ion.ion_autotune(sim.h, 20)    # launch shape timed on this network (state restored)
        return sim

    def reset(sim):
        sim.write(S0)
        ion.ion_set_step_count(sim.h, 0)

    def warm(flags):
        """A handle of one variant after args.warmup untimed bench steps."""
        sim = make_sim(flags)
        for _ in range(args.warmup):
            reset(sim)
            sim.step(sim_steps)
        torch.cuda.synchronize()
        return sim

    def trial(sim, reps=2):
        """Median time (ms) of `reps` bench steps: the variant choice, made before and apart
        from the timed region."""
        out = []
        for k in range(reps):
            flush.fill_(float(k))
            reset(sim)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            sim.step(sim_steps)
            b.record()
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.median(out)

    def timed(sim):
        """Time args.steps bench steps of one variant (each from the same state and t = 0)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(local)
        clocks.start()
        launches0 = sim.launches
        for k in range(args.steps):
            flush.fill_(float(k))                       # evict L2 between timed steps
            reset(sim)                                  # same initial state every step (untimed)
            ev[k][0].record()
            sim.step(sim_steps)
            ev[k][1].record()
        torch.cuda.synchronize()
        ck = clocks.stop()
        launches = sim.launches - launches0
        ms = sum(a.elapsed_time(b) for a, b in ev)
        sim.sync()                                      # the run stayed finite
        return ms, launches, ck

    cand = [("graph", ion.FLAG_KAHAN),
            ("graph_ordinary_launches", ion.FLAG_KAHAN | ion.FLAG_NO_PDL)]   # without programmatic launches
    if batch:   # every network's steps in one cooperative launch per ion_step call
        cand.append(("persistent", ion.FLAG_KAHAN | ion.FLAG_PERSISTENT))
    if dense and not wl.get("sgj"):
        cand.append(("persistent", ion.FLAG_KAHAN | ion.FLAG_PERSISTENT))
        if n > 144:   # multi-CTA networks: the half-work pass as well as the full pass
            cand.append(("persistent_half", ion.FLAG_KAHAN | ion.FLAG_PERSISTENT | ion.FLAG_HALF_WORK))
    if cfg["kind"] == "csr" and key != "c5":   # the CSR as given (32-bit columns, per-edge weights) too
        cand.append(("graph_csr_as_given", ion.FLAG_KAHAN | ion.FLAG_CSR_AS_GIVEN))
        cand.append(("graph_csr_half", ion.FLAG_KAHAN | ion.FLAG_HALF_WORK))   # each stored pair once
    if args.variant != "auto":
        cand = [c for c in cand if c[0] == args.variant]
    if key == "c5":
        cand = [("exact", ion.FLAG_KAHAN), ("surrogate", ion.FLAG_KAHAN | ion.FLAG_SURROGATE)]
    # The reported variant is chosen on trial steps after the warm-up, before the timed
    # region; only that variant is timed (c5 times both: the surrogate is the line, the
    # exact method its comparison).
    variants, best, best_sim = {}, None, None
    for name, flags in cand:
        tune_table = None
        sim_v = warm(flags)
        variants[name] = dict(trial_ms=trial(sim_v), tune=tune_table, flags=flags)
        if key == "c5":
            variants[name]["sim"] = sim_v
        elif best is None or variants[name]["trial_ms"] < variants[best]["trial_ms"]:
            if best_sim is not None:
                best_sim.close()
            best, best_sim = name, sim_v
        else:
            sim_v.close()
    if key == "c5":
        best = "surrogate"
        for name in ("exact", "surrogate"):
            ms_v, l_v, ck_v = timed(variants[name]["sim"])
            variants[name].update(ms=ms_v, launches=l_v, clocks=ck_v)
    else:
        ms_v, l_v, ck_v = timed(best_sim)
        variants[best].update(sim=best_sim, ms=ms_v, launches=l_v, clocks=ck_v)
    if key == "c5":   # the line reports the surrogate; the exact method is its comparison
        best = "surrogate"
        surrogate_info.update({
            "exact_cell_timesteps_per_s": n * sim_steps * args.steps / (variants["exact"]["ms"] * 1e-3),
            "speedup_vs_exact": variants["exact"]["ms"] / variants["surrogate"]["ms"]})
        surrogate_info.update(compare_runs(ion, variants["exact"]["sim"], variants["surrogate"]["sim"], reset,
                                           n, sim_steps))
        # the workload's pulse reaches 20 % of the cells and drains into their neighbours
        # (no cell fires); the spike times are compared on the same network with every
        # cell pulsed at 50-60 ms and 500-510 ms
        from paper_1612_01501_gb300 import inputs
        spiking = inputs.config("c3_spiking", k=wl["k"])
        for name in ("exact", "surrogate"):
            variants[name]["sim"].set_input(spiking["pulses"])
        surrogate_info["spiking_comparison"] = dict(
            workload="c3_spiking_csr_65536_k100_1s (every cell pulsed at 50-60 and 500-510 ms)",
            **compare_runs(ion, variants["exact"]["sim"], variants["surrogate"]["sim"], reset, n, sim_steps))
        for name in ("exact", "surrogate"):
            variants[name]["sim"].set_input(cfg["pulses"])
    sim, ms, launches, ck = (variants[best][k] for k in ("sim", "ms", "launches", "clocks"))
    for k, v in variants.items():
        if k != best and v.get("sim") is not None:
            v["sim"].close()

    cell_steps = n * sim_steps * args.steps * world
    value, ms = replica_reduce(ms, n * sim_steps * args.steps, pg)   # slowest rank, cells of all ranks
    per_step_s = ms * 1e-3 / (sim_steps * args.steps)
    if batch:
        # one ex2 per dense pair and per CSR edge; the SFU rate bounds the mix
        work = sum(b["n"] ** 2 if b["kind"] == "dense" else len(b["col"]) for b in cfg["nets"])
        peak = ion.ion_probe_peak(0, 4096, stream)
        achieved = work / per_step_s
        roof = {"bound": "alu", "unit": "ex2/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                "traffic": None, "kernel": "batch_persist_kernel" if best == "persistent" else "batch_step_kernel",
                "peak_source": "measured SFU ex2 rate (ion_probe_peak) in the same process",
                "us_per_timestep": per_step_s * 1e6}
        extra = {"pair_evals_per_s": sum(b["n"] ** 2 for b in cfg["nets"] if b["kind"] == "dense") / per_step_s,
                 "edges_per_s": sum(len(b["col"]) for b in cfg["nets"] if b["kind"] == "csr") / per_step_s,
                 "autotuned": tune_table, "n_networks": len(cfg["nets"])}
    elif cfg["kind"] == "matrix":
        # HBM: the padded weight matrix (4 B per stored pair) streams every step, plus the
        # cell state (132 B per cell)
        n_pad = (n + 255) // 256 * 256
        bytes_step = 4 * n * n_pad + 132 * n
        achieved = bytes_step / per_step_s / 1e9
        peak = hbm_peak()
        roof = {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                "traffic": None, "kernel": "matrix_step_kernel", "algorithmic_bytes_per_timestep": bytes_step,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs", "us_per_timestep": per_step_s * 1e6}
        extra = {"pair_evals_per_s": value * n}
    elif dense and wl.get("sgj"):
        # linear junctions: O(N) per step (the sum of V_dend, then each cell's update): the
        # state (132 B per cell) and one read of V_dend by the partial sums
        bytes_step = 132 * n + 4 * n
        achieved = bytes_step / per_step_s / 1e9
        peak = hbm_peak()
        roof = {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                "traffic": None, "kernel": "sgj_dense_update_kernel",
                "algorithmic_bytes_per_timestep": bytes_step, "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                "us_per_timestep": per_step_s * 1e6,
                "note": "latency-bound: one short launch per step on an L2-resident state"}
        extra = {"pair_evals_per_s": value * n}
    elif dense:
        # SFU-bound: one ex2 per pair evaluation (N^2 per time step); the half-work kernel
        # evaluates each unordered pair once (N^2 / 2 ex2 per time step)
        half = best == "persistent_half"
        ex2_step = n * n / 2 if half else n * n
        peak = ion.ion_probe_peak(0, 4096, stream)
        achieved = ex2_step / per_step_s
        roof = {"bound": "alu", "unit": "ex2/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                "traffic": None, "kernel": {"persistent": "dense_persist_kernel",
                           "persistent_half": "dense_half_kernel"}.get(best, "dense_step_kernel"),
                "peak_source": "measured SFU ex2 rate (ion_probe_peak) in the same process",
                "ffma_peak_per_s": ion.ion_probe_peak(1, 4096, stream), "us_per_timestep": per_step_s * 1e6,
                "ex2_per_timestep": ex2_step}
        extra = {"pair_evals_per_s": value * n}
    elif ngj:
        # HBM: per time step the cell state (15 words read + 18 written) and the pulse
        # table (4 B offset per cell + 20 B per pulse, 20 % of cells pulsed)
        bytes_step = 132 * n + 4 * (n + 1) + 20 * len(cfg["pulses"][0])
        achieved = bytes_step / per_step_s / 1e9
        peak = hbm_peak()
        roof = {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                "traffic": None, "kernel": "cell_step_kernel", "algorithmic_bytes_per_timestep": bytes_step,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs", "us_per_timestep": per_step_s * 1e6,
                "note": "state (%.0f MB) larger than L2 (129 MB)" % (80 * n / 1e6)}
        extra = {"sweep": k3_sweep(ion, torch, stream, flush, sim_steps, args.warmup, {n: per_step_s}, peak)}
    elif key == "c5":
        # the surrogate's cell kernel: 3 MLP evaluations per cell on the tensor cores
        flops = 3 * 2 * (2 * 64 + 64 * 64 + 64 * 24)
        achieved = n * flops / per_step_s / 1e12
        # the kernel runs inside a seconds-long step: the sustained bf16 rate is its peak
        peak, src = 1700.0, "fallback (sustained bf16 of an earlier GB300 measurement)"
        try:
            peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops_sustained"])
            src = "MEASURED_PEAKS.json bf16_tflops_sustained"
        except (OSError, KeyError, ValueError):
            pass
        roof = {"bound": "tensor", "unit": "TFLOP/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                "traffic": None, "kernel": "surrogate_tc_kernel",
                "kernels": "surrogate_tc_kernel (tcgen05 MLP + cell update) after the gap-current kernel",
                "peak_source": src, "us_per_timestep": per_step_s * 1e6,
                "mlp_flop_per_cell_step": flops}
        # the MLP's two hidden layers end in tanh: 3 x 128 per cell-step, paired in
        # tanh.approx.bf16x2, whose measured issue rate bounds the kernel before the MMAs do
        tanh2 = 3 * 128 // 2
        tpk = ion.ion_probe_peak(2, 4096, stream)
        roof["tanh_bf16x2"] = {"per_cell_step": tanh2, "achieved": n * tanh2 / per_step_s, "peak": tpk,
                               "frac": n * tanh2 / per_step_s / tpk,
                               "peak_source": "measured tanh.approx.bf16x2 rate (ion_probe_peak) in the same process"}
        extra = {"surrogate": surrogate_info}
    else:
        # HBM: per time step the CSR as the handle stores it (index + weight bytes per edge,
        # 4 B per row pointer, 4 B per row and interior chunk boundary when staged), the cell
        # state (15 words read + 18 written) and the pulse table (8 B per cell on average)
        nnz = len(cfg["col"])
        lay = ion.ion_csr_layout(sim.h)
        n_pad = (n + 255) // 256 * 256
        if lay["staged"]:         # row pointers + interior chunk boundaries
            ptr_bytes = 4 * (n + 1) + 4 * n * ((n_pad + 32767) // 32768 - 1)
        else:
            ptr_bytes = 4 * (n + 1)
        bytes_step = (lay["index_bytes"] + lay["weight_bytes"]) * nnz + ptr_bytes + 132 * n + 8 * n
        achieved = bytes_step / per_step_s / 1e9
        peak = hbm_peak()
        roof = {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                "traffic": None,
                "kernel": "csr_chunk_step_kernel" if lay["staged"] else "csr_step_kernel",
                "algorithmic_bytes_per_timestep": bytes_step,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs", "us_per_timestep": per_step_s * 1e6,
                "note": "working set fits in L2 (129 MB)" if bytes_step < 100e6 else "streams from HBM",
                "csr_layout": lay}
        extra = {"edges_per_s": value / n * nnz, "nnz": nnz}

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"], "n_cells": n, "timesteps_per_step": sim_steps,
                       "parallelism": f"replicas x{world}", "l2": "flushed (512 MB write) between timed steps"},
            "roofline": roof,
            "variants": {k: {"trial_ms_per_step": v["trial_ms"],
                             **({"ms_per_step": v["ms"] / args.steps} if "ms" in v else {})}
                         for k, v in variants.items()},
            "variant": best,
            "variant_choice": "fastest median of 2 trial steps after the warm-up, before the timed region",
            "gpu_launches": int(launches),
            "clocks": ck,
        }
        tr = traffic_for(key, roof.get("kernel"), best, variants[best]["tune"], args.dense_shape)
        if tr is not None:
            roof["traffic"] = tr[0]
            roof["traffic_source"] = tr[1] + " (one ncu capture of this kernel; the summary names its launch shape)"
        # the paper's real-time criterion: one time step (50 us of biological time) computed
        # in at most 50 us of wall time
        line["real_time"] = {"us_per_timestep": roof["us_per_timestep"], "limit_us": 50.0,
                             "met": roof["us_per_timestep"] <= 50.0}
        if variants[best]["tune"] is not None and "autotuned" not in extra:
            line["autotuned"] = variants[best]["tune"]
        line.update(extra)
    if not args.no_extra:
        # e2e through the public API with pinned host buffers (H2D state in, D2H state out)
        S_pin = torch.from_numpy(S0.copy()).pin_memory()
        out_pin = torch.empty_like(S_pin).pin_memory()
        e2e_steps = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ion.ion_write_state(sim.h, S_pin.numpy())
            ion.ion_set_step_count(sim.h, 0)
            sim.step(sim_steps)
            out_pin.numpy()[:] = ion.ion_read_state(sim.h, n)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_value, _ = replica_reduce(e2e_s * 1e3, n * sim_steps * e2e_steps, pg)
        if rank == 0:
            line["e2e"] = {"value": e2e_value, "unit": METRIC,
                           "h2d_bytes_per_step": int(S0.nbytes), "d2h_bytes_per_step": int(S0.nbytes)}
            ks = reference_sample_steps(key) if key != "c2" else 3
            cpu = cpu_baseline(key, ks, single_thread_steps=max(1, ks // 4))
            line["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "single_core")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
