"""Checks of the oracle's structure against the numbers the paper prints (Table "reqs",
Sec. 2.2; SGJ count, Sec. 2.3.2; time step, Sec. 2.2)."""
import json
import os

import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table_reqs.json")))


def test_state_words(O):
    assert O.NF == GOLD["neuron_state_words"] == 19


def test_conductance_count(O):
    # 12 maximal conductances + g_int + two area ratios + 5 reversal potentials
    cond = [p for p in O.PARAMS[:20]]
    assert len(cond) == GOLD["neuron_conductances"]
    assert sum(p.startswith("g_") for p in cond) == 13 and sum(p.startswith("V_") for p in cond) == 5
    assert O.PARAMS[20] == "C_m"


def test_flop_model_counts_n_squared_pairs():
    """859 N + 12 N^2 C: at N = 96, C = 1 the gap junctions are 57 % of the work, which
    holds for the N^2 pair count used by the pair-evaluation metric."""
    n = 96
    gj = GOLD["gap_junction_flop_per_connection"] * n * n
    cell = GOLD["cell_compartment_flop"] * n
    assert round(100 * gj / (gj + cell)) == GOLD["gj_share_percent_96_cells_all_to_all"]
    assert round(100 * cell / (gj + cell)) == GOLD["compartment_share_percent_96_cells_all_to_all"]
    assert GOLD["cell_compartment_flop"] + GOLD["gap_junction_flop_per_connection"] == GOLD["flop_single_cell_with_one_gj"]


def test_time_step(O):
    assert O.DT_MS * 1000.0 == pytest.approx(GOLD["time_step_us"])
