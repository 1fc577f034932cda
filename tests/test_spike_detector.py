"""Pins of the spike detector behind every spike-time check (CPU only).

The paper names the axon voltage as the cell's output (Table "reqs": one axon-output word
per cell) but defines no spike.  The reading used throughout: a spike is an upward
crossing of 0 mV by V_axon, timed at the first sample at or above 0 mV, and the detector
re-arms only once V_axon has fallen below -30 mV.  A cell at rest (-60 mV) is armed, so
a trace that starts above threshold reports a spike at sample 0.

Each case below is a hand-built trace with its answer worked out by reading the trace,
so that a detector that re-arms at the wrong level, compares strictly, or starts disarmed
fails one of them.  The same cases are run through the streaming detector the benchmark
uses for its surrogate comparison (bench.SpikeLog), which is a separate implementation.
"""
import numpy as np
import pytest

from oracle.oracle import spike_steps

REST = -60.0

CASES = [
    # (name, trace, expected spike steps)
    ("flat_rest", [REST] * 8, []),
    ("single_crossing", [REST, -20.0, -1.0, 5.0, 20.0, -10.0, -50.0, REST], [3]),
    ("sample_exactly_at_zero", [REST, -5.0, 0.0, 10.0, -40.0], [2]),
    ("just_below_zero_is_no_spike", [REST, -1e-6, -0.5, REST], []),
    ("starts_above_threshold", [10.0, 30.0, -10.0, -40.0, REST], [0]),
    # after a spike, a dip to -29 mV does not re-arm: the second peak is not a spike
    ("dip_to_minus_29_does_not_rearm", [REST, 5.0, -29.0, 8.0, -29.0, 12.0, REST], [1]),
    # a dip to -31 mV re-arms: the second peak is a spike
    ("dip_to_minus_31_rearms", [REST, 5.0, -31.0, 8.0, REST], [1, 3]),
    # exactly -30 mV does not re-arm (re-arming needs V < -30)
    ("dip_to_exactly_minus_30_does_not_rearm", [REST, 5.0, -30.0, 8.0, REST], [1]),
    # two bursts: each burst has several peaks that never fall below -30 mV between them,
    # and the cell repolarises to rest between the bursts
    ("two_bursts",
     [REST, -40.0, 2.0, -20.0, 4.0, -25.0, 1.0, -45.0, REST, REST, -35.0, 0.5, -10.0, 3.0, -70.0, REST],
     [2, 11]),
    # a slow rise spends several samples above 0 mV: one spike at the first of them
    ("plateau_above_threshold", [REST, -10.0, 0.1, 0.2, 0.3, 0.2, -35.0, REST], [2]),
]


@pytest.mark.parametrize("name,trace,expected", CASES, ids=[c[0] for c in CASES])
def test_oracle_spike_detector(name, trace, expected):
    got = spike_steps(np.asarray(trace, np.float64))
    assert got.dtype == np.int64
    assert got.tolist() == expected


@pytest.mark.parametrize("name,trace,expected", CASES, ids=[c[0] for c in CASES])
def test_streaming_detector_agrees(name, trace, expected):
    """bench.SpikeLog (one row per time step, many cells at once, fed in chunks) finds the
    same spikes; the cases are laid side by side as cells of one trace matrix."""
    bench = pytest.importorskip("bench")
    log = bench.SpikeLog(2)
    tr = np.stack([np.asarray(trace, np.float32), np.full(len(trace), REST, np.float32)], axis=1)
    half = len(trace) // 2
    log.feed(tr[:half])
    log.feed(tr[half:])
    cells, steps = log.sorted()
    assert steps[cells == 0].tolist() == expected
    assert steps[cells == 1].tolist() == []


def test_float32_trace_thresholds():
    """Float32 samples are compared as given: the largest float32 below 0 is no spike, and
    the detector sees -30 mV rounded to float32 as -30 exactly (no re-arm)."""
    below = np.nextafter(np.float32(0.0), np.float32(-1.0))
    assert spike_steps(np.array([REST, below, REST], np.float32)).tolist() == []
    assert spike_steps(np.array([REST, 1.0, np.float32(-30.0), 1.0], np.float32)).tolist() == [1]
