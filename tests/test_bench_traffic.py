"""The bench's DRAM-traffic figures (CPU only).

A bench line reports `roofline.traffic` (DRAM bytes per launch of its dominant kernel)
only from an ncu capture of that kernel, and only when the line runs the launch shape the
capture fixed; otherwise the figure is null.  These checks pin that rule and that every
figure names a summary that exists under profiles/.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

C2_SHAPE = dict(dense_rows_per_warp=4, dense_warps=28, dense_col_splits=2)


def test_every_traffic_figure_names_an_existing_summary_and_a_workload():
    for (key, kernel), (nbytes, source, shape) in bench.TRAFFIC.items():
        assert key in bench.WORKLOADS, key
        assert nbytes > 0 and isinstance(shape, dict)
        assert os.path.isfile(os.path.join(ROOT, source)), source
        assert kernel in open(os.path.join(ROOT, source)).read(), (kernel, source)


def test_traffic_only_for_the_captured_launch_shape():
    assert bench.traffic_for("c2", "dense_step_kernel", "graph", C2_SHAPE)[0] > 0
    other = dict(C2_SHAPE, dense_warps=24)
    assert bench.traffic_for("c2", "dense_step_kernel", "graph", other) is None
    assert bench.traffic_for("c2", "dense_step_kernel", "graph", None) is None
    # --dense-shape stands in for the autotuner's table
    assert bench.traffic_for("c2", "dense_step_kernel", "graph", None, "4,28,2")[0] > 0
    assert bench.traffic_for("c2", "dense_step_kernel", "graph", None, "2,28,2") is None


@pytest.mark.parametrize("variant", ["persistent", "persistent_half", "graph_csr_as_given", "graph_csr_half"])
def test_no_traffic_for_variants_that_run_other_kernels(variant):
    assert bench.traffic_for("c2", "dense_step_kernel", variant, C2_SHAPE) is None
    assert bench.traffic_for("c3_k1000", "csr_chunk_step_kernel", variant, dict(csr_staging=2)) is None


def test_no_traffic_for_an_uncaptured_kernel():
    assert bench.traffic_for("c1", "dense_persist_kernel", "persistent", None) is None
    assert bench.traffic_for("c3_k1000", "csr_step_kernel", "graph", dict(csr_staging=1)) is None


def test_staged_csr_traffic_needs_the_staged_layout():
    assert bench.traffic_for("c3_k1000", "csr_chunk_step_kernel", "graph", dict(csr_staging=2, csr_lanes_per_row=8))
    assert bench.traffic_for("c3_k1000", "csr_chunk_step_kernel", "graph", dict(csr_staging=0)) is None
