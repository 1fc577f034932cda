"""Benchmark of the InfOli hot path on one GB300 (or N independent replicas).

Workload (default): the 8192-cell all-to-all network (RGJ at 100 % density), FP32 state
in SoA layout, g_c = 0.04 / N * 64, V_dend jittered +-5 mV from seed 1, no evoked input;
one bench step simulates 200 ms = 4000 time steps of 50 us.  Metric: cell-timesteps/s
(and gap-junction pair evaluations/s, N^2 per time step).

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead (on a
bounded sample of the same workload, all host cores).
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
WORKLOAD = "c2_dense_8192_allToAll_200ms"
N_CELLS = 8192
STEPS_PER_BENCH_STEP = 4000          # 200 ms of simulated time
L2_FLUSH_BYTES = 512 << 20           # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sim-steps", type=int, default=STEPS_PER_BENCH_STEP)
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary configuration lines")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def c2_initial_state():
    """FP32 initial state of the workload, computed by the library on the device."""
    from paper_1612_01501_gb300 import inputs, ion
    S = ion.ion_default_state(N_CELLS)
    S[0] = (S[0].astype(np.float64) + inputs.vdend_jitter(N_CELLS, 1)).astype(np.float32)
    return S


def cpu_baseline(sample_steps: int = 3, reps: int = 1):
    """FP64 oracle on the host cores: `sample_steps` time steps of the same workload."""
    import oracle as O
    from paper_1612_01501_gb300 import inputs
    cfg = inputs.config("c2")
    S = O.default_state(N_CELLS)
    S[O.F["V_dend"]] += cfg["jitter"]
    S = S.astype(np.float32).astype(np.float64)
    threads = O.max_threads()
    O.run(S, 1, kind=O.DENSE, g=cfg["g"], threads=threads)        # warm caches / thread pool
    t0 = time.perf_counter()
    for _ in range(reps):
        O.run(S, sample_steps, kind=O.DENSE, g=cfg["g"], threads=threads)
    dt = time.perf_counter() - t0
    v = N_CELLS * sample_steps * reps / dt
    return {"value": v, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"{sample_steps * reps} time steps of the 8192-cell dense network (FP64, OpenMP over cells)",
            "pair_evals_per_s": v * N_CELLS, "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    steps = []
    import oracle as O
    O.build()
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(sample_steps=8)
        if k >= args.warmup:
            steps.append(r)
    t = sum(r["seconds"] for r in steps)
    cells = N_CELLS * 8 * len(steps)
    v = cells / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_cells": N_CELLS, "timesteps_per_step": 8,
                       "note": "bounded sample: 8 time steps per bench step"},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": steps[0]["cores"], "kind": "oracle",
                             "sample": "8 time steps of the 8192-cell dense network per bench step"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    # a dedicated stream: the library's steps and the timing events must share it
    # (the default stream's handle is 0, which the library reads as "no stream given")
    torch.cuda.set_stream(torch.cuda.Stream())
    from paper_1612_01501_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
        pg.barrier()
        B.build()
    from paper_1612_01501_gb300 import inputs, ion

    stream = torch.cuda.current_stream().cuda_stream
    S0 = c2_initial_state()
    g = inputs.junction_weight(0.04, N_CELLS)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def measure(flags):
        """Time args.steps bench steps (4000 time steps each) of one variant."""
        sim = ion.Simulation(N_CELLS, ion.DENSE_UNIFORM, g=g, init_state=S0, stream=stream, graph_steps=100,
                             flags=flags)
        for _ in range(args.warmup):
            sim.write(S0)
            sim.step(args.sim_steps)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(local)
        clocks.start()
        launches0 = sim.launches
        for k in range(args.steps):
            flush.fill_(float(k))                       # evict L2 between timed steps
            sim.write(S0)                               # same initial state every step (untimed)
            ev[k][0].record()
            sim.step(args.sim_steps)
            ev[k][1].record()
        torch.cuda.synchronize()
        ck = clocks.stop()
        launches = sim.launches - launches0
        ms = sum(a.elapsed_time(b) for a, b in ev)
        if pg:
            t = torch.tensor([ms], device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            ms = float(t.item())
        sim.sync()                                      # the run stayed finite
        return sim, ms, launches, ck

    variants = {}
    for name, flags in (("graph", ion.FLAG_KAHAN), ("persistent", ion.FLAG_KAHAN | ion.FLAG_PERSISTENT)):
        sim_v, ms_v, l_v, ck_v = measure(flags)
        variants[name] = dict(sim=sim_v, ms=ms_v, launches=l_v, clocks=ck_v)
    best = min(variants, key=lambda k: variants[k]["ms"])
    sim, ms, launches, ck = (variants[best][k] for k in ("sim", "ms", "launches", "clocks"))
    for k, v in variants.items():
        if k != best:
            v["sim"].close()

    cell_steps = N_CELLS * args.sim_steps * args.steps * world
    value = cell_steps / (ms * 1e-3)
    pair_evals_s = value * N_CELLS
    # roofline of the dense kernel: SFU-bound, one ex2 per pair evaluation.  The timed
    # region is (almost) all dense-kernel time: per time step one fused launch (graph
    # variant) or one slice of the persistent launch.
    per_step_s = ms * 1e-3 / (args.sim_steps * args.steps)
    ex2_peak = ion.ion_probe_peak(0, 4096, stream)
    ffma_peak = ion.ion_probe_peak(1, 4096, stream)
    achieved_ex2 = N_CELLS * N_CELLS / per_step_s

    # e2e through the public API with pinned host buffers (H2D state in, D2H state out)
    S_pin = torch.from_numpy(S0.copy()).pin_memory()
    out_pin = torch.empty_like(S_pin).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ion.ion_write_state(sim.h, S_pin.numpy())
        sim.step(args.sim_steps)
        out_pin.numpy()[:] = ion.ion_read_state(sim.h, N_CELLS)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = N_CELLS * args.sim_steps * e2e_steps * world / e2e_s

    extra = {}
    if rank == 0:
        cpu = cpu_baseline(sample_steps=3)
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_cells": N_CELLS, "timesteps_per_step": args.sim_steps,
                       "g_c": g, "parallelism": f"replicas x{world}", "l2": "flushed (512 MB write) between timed steps"},
            "pair_evals_per_s": pair_evals_s,
            "roofline": {"bound": "alu", "unit": "ex2/s", "achieved": achieved_ex2, "peak": ex2_peak,
                         "frac": achieved_ex2 / ex2_peak, "traffic": None,
                         "kernel": "dense_persist_kernel" if best == "persistent" else "dense_step_kernel",
                         "peak_source": "measured SFU ex2 probe (ion_probe_peak), same clock",
                         "ffma_peak_per_s": ffma_peak, "us_per_timestep": per_step_s * 1e6},
            "variants": {k: {"ms_per_step": v["ms"] / args.steps,
                             "cell_timesteps_per_s": cell_steps / (v["ms"] * 1e-3)} for k, v in variants.items()},
            "variant": best,
            "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": int(S0.nbytes),
                    "d2h_bytes_per_step": int(S0.nbytes)},
            "gpu_launches": int(launches),
            "clocks": ck,
        }
        line.update({k: v for k, v in extra.items() if k not in line})
        print(json.dumps(line), flush=True)
    sim.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
