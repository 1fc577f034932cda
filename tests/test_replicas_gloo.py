"""The multi-process (replicas) path of bench.py on CPU: two gloo ranks, each timing its own
replica; the job's value divides the cells of both ranks by the slower rank's time."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_time_and_cells(tmp_path):
    script = tmp_path / "rank.py"
    script.write_text(textwrap.dedent(f"""
        import os, sys, json
        sys.path.insert(0, {ROOT!r})
        import torch.distributed as dist
        import bench
        dist.init_process_group("gloo")
        r = dist.get_rank()
        ms_local = [10.0, 25.0][r]            # rank 1 is the slow replica
        cells_local = [1000.0, 1000.0][r]
        value, ms = bench.replica_reduce(ms_local, cells_local, dist)
        if r == 0:
            print(json.dumps({{"value": value, "ms": ms}}))
        dist.barrier()
        dist.destroy_process_group()
    """))
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
                          "--master-addr", "127.0.0.1", "--master-port", env["MASTER_PORT"], str(script)],
                         capture_output=True, text=True, env=env, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    import json
    line = [l for l in out.stdout.splitlines() if l.startswith("{")][-1]
    d = json.loads(line)
    assert d["ms"] == 25.0
    assert abs(d["value"] - 2000.0 / 0.025) < 1e-6


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    v, ms = bench.replica_reduce(20.0, 500.0, None)
    assert ms == 20.0 and abs(v - 500.0 / 0.02) < 1e-9
