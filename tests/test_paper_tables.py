"""Checks of the oracle's structure against the numbers the paper prints (Table "reqs",
Sec. 2.2; SGJ count, Sec. 2.3.2; time step, Sec. 2.2)."""
import json
import os

import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table_reqs.json")))


def test_state_words(O):
    assert O.NF == GOLD["neuron_state_words"] == 19


def test_conductance_count(O):
    """Table "reqs" lists 20 conductances per neuron.  The three-compartment model used here
    has 13: the 12 maximal channel conductances (4 dendritic, 5 somatic, 3 axonal) and the
    inter-compartment conductance g_int.  The remaining per-cell constants of the table's
    first 20 entries are two area ratios (p1, p2) and five reversal potentials, which are
    not conductances.  The gap to the paper's count is a documented mismatch (the paper
    prints no equations to resolve it), so this pins the model's own count and the paper's
    number separately rather than reconciling them."""
    cond = [p for p in O.PARAMS if p.startswith("g_")]
    assert cond == ["g_int", "g_CaH", "g_KCa", "g_h", "g_ld", "g_CaL", "g_Na_s", "g_Kdr_s", "g_K_s", "g_ls",
                    "g_Na_a", "g_K_a", "g_la"]
    assert len(cond) == 13
    assert GOLD["neuron_conductances"] == 20             # the paper's figure, not reached by the model
    assert [p for p in O.PARAMS[:20] if not p.startswith("g_")] == ["p1", "p2", "V_Na", "V_K", "V_Ca", "V_h", "V_L"]
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


def test_operation_counts_against_the_paper(O):
    """Operation counts of the oracle (soft pin: the paper does not say how it counts an
    exponential).  The gap-junction term is exactly 7 arithmetic operations and one
    exponential per ordered pair (V_i - V_j, its square, / 100, exp, x 0.8, + 0.2, x dV,
    accumulate); the paper's 12 then prices an exponential at 5.  At that price the
    oracle's cell step lands near the paper's 859 per neuron (it evaluates all 12 rate
    functions in each compartment, so it over-counts), and an SGJ connection costs 3
    operations against the paper's 4."""
    c = O.op_counts()
    gj_arith = c["gj_pair_add"] + c["gj_pair_mul"] + c["gj_pair_div"]
    assert (c["gj_pair_add"], c["gj_pair_mul"], c["gj_pair_div"], c["gj_pair_exp"]) == (3, 3, 1, 1)
    exp_price = GOLD["gap_junction_flop_per_connection"] - gj_arith
    assert exp_price == 5
    cell = c["cell_add"] + c["cell_mul"] + c["cell_div"] + c["cell_minmax"] + exp_price * c["cell_exp"]
    print(f"cell step: {c['cell_add']:.0f} add, {c['cell_mul']:.0f} mul, {c['cell_div']:.0f} div, "
          f"{c['cell_exp']:.0f} exp -> {cell:.0f} FLOP at 5 per exp (paper: {GOLD['cell_compartment_flop']})")
    assert 0.5 * GOLD["cell_compartment_flop"] <= cell <= 1.5 * GOLD["cell_compartment_flop"]
    sgj = c["sgj_edge_add"] + c["sgj_edge_mul"]
    assert (c["sgj_edge_add"], c["sgj_edge_mul"], c["sgj_edge_exp"]) == (2, 1, 0)
    assert sgj <= GOLD["sgj_flop_per_connection"]
