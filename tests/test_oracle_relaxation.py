"""Pins of the oracle's relaxation matrices (Eq. 4 with Eq. 11, the orthogonal reading, D3Q15).

Each non-conserved moment, perturbed alone on a uniform rest state with G = 0,
must decay by (1 - s_k) per step with the rate the golden table assigns to its
basis polynomial; six distinct rates make every rate group distinguishable.
A planted swap of s_q and s_pi in the oracle must fail the same check.
"""

import numpy as np
import pytest

from oracle import d3q15 as D
from oracle import lbm_oracle as L
from relaxation_pin import (SIX_RATES, basis, decay_error, non_conserved_rows, perturbed_rest_state,
                            rate_table)

GRID = (3, 3, 3)
EPS = 1e-3
RHO0 = 0.7
STEPS = 1
CASES = {  # golden operator name -> (oracle module, oracle operator, velocities, rest weights)
    "nonorth": (L, "nonorth", L.E, L.W_LATTICE),
    "orth": (L, "orth", L.E, L.W_LATTICE),
    "nonorth15": (D, "nonorth", D.E, D.W_LATTICE),
}


def _worst_error(op_name, step_fn=None):
    mod, oop, E, w = CASES[op_name]
    p = L.Params(grid=GRID, operator=oop, eos="none", G=0.0, **SIX_RATES)
    step = step_fn or mod.step
    worst = 0.0
    for k in non_conserved_rows(op_name):
        f0 = perturbed_rest_state(op_name, E, w, k, EPS, RHO0, GRID)
        f = f0
        for _ in range(STEPS):
            f = step(p, f)
        worst = max(worst, decay_error(op_name, E, f0, f, k, EPS, SIX_RATES, STEPS))
    return worst


def test_golden_table_matches_the_paper_counts():
    # Eq. 11: four conserved rows, one s_e, five s_nu, six s_q, three s_pi
    names = [r for _, _, r in rate_table("nonorth")]
    assert [names.count(s) for s in ("conserved", "s_e", "s_nu", "s_q", "s_pi")] == [4, 1, 5, 6, 3]
    names = [r for _, _, r in rate_table("orth")]
    assert [names.count(s) for s in ("conserved", "s_e", "s_eps", "s_q", "s_nu", "s_pi", "s_m")] == [4, 1, 1, 3, 5, 2, 3]
    names = [r for _, _, r in rate_table("nonorth15")]
    assert [names.count(s) for s in ("conserved", "s_e", "s_nu", "s_q", "s_pi")] == [4, 1, 5, 4, 1]


@pytest.mark.parametrize("op_name", ["nonorth", "orth", "nonorth15"])
def test_golden_basis_spans_the_oracle_basis(op_name):
    """The golden polynomials are the oracle's rows, row for row."""
    mod, oop, E, _ = CASES[op_name]
    M_oracle = mod.nonorth_matrix() if op_name == "nonorth15" else L.matrix(L.Params(operator=oop))
    assert np.array_equal(basis(op_name, E), M_oracle)


@pytest.mark.parametrize("op_name", ["nonorth", "orth", "nonorth15"])
def test_each_moment_decays_with_its_own_rate(op_name):
    assert _worst_error(op_name) < 1e-13


def test_relaxation_diagonal_names_each_rate_once():
    """The oracle's diagonal, with six distinct rates, is the golden table's rate column."""
    for op_name, (mod, oop, _, _) in CASES.items():
        p = L.Params(grid=GRID, operator=oop, **SIX_RATES)
        lam = mod.relaxation(p)
        want = [1.0 if r == "conserved" else SIX_RATES[r] for _, _, r in rate_table(op_name)]
        np.testing.assert_array_equal(lam, want)


@pytest.mark.parametrize("op_name", ["nonorth", "orth"])
def test_planted_swap_of_s_q_and_s_pi_fails_the_pin(op_name, monkeypatch):
    """A mistake planted in the oracle (s_q and s_pi exchanged) is caught by the decay check."""
    real = L.relaxation

    def swapped(p):
        return real(p.with_(s_q=p.s_pi, s_pi=p.s_q))

    monkeypatch.setattr(L, "relaxation", swapped)
    assert _worst_error(op_name) > 1e-2 * EPS


def test_planted_swap_in_d3q15_fails_the_pin(monkeypatch):
    real = D.relaxation
    monkeypatch.setattr(D, "relaxation", lambda p: real(p.with_(s_q=p.s_pi, s_pi=p.s_q)))
    assert _worst_error("nonorth15") > 1e-2 * EPS
