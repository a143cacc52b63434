"""Closed-form pin of which relaxation rate acts on which moment (Eq. 4, Eq. 11).

On a uniform rest state with no interaction force (G = 0), perturb exactly one
non-conserved moment m_k by eps.  Density and momentum do not change, so the
equilibrium moments and the forcing moments stay those of the rest state, the
field stays uniform (streaming moves nothing), and Eq. 4 leaves

    m_k(t) - m_k(0) = (1 - s_k)^t eps,   every other moment unchanged,

with s_k the rate the paper assigns to the polynomial of row k.  The basis is
built here from the polynomials listed in ``tests/golden/relaxation_rates.txt``
(not from the oracle's matrices), so the check covers both the placement of
the rows and the rate each one relaxes with.  With six distinct rates any
crossing of two rate groups changes some decay factor.
"""

from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

# six distinct rates: a rate placed on the wrong moment group changes a decay factor
SIX_RATES = dict(s_e=0.8, s_nu=1.3, s_q=1.15, s_pi=0.9, s_eps=1.4, s_m=1.7)


def rate_table(operator: str):
    """[(row, polynomial, rate name)] of one operator from the golden file."""
    rows = []
    with open(os.path.join(HERE, "golden", "relaxation_rates.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            op, k, poly, rate = line.split()
            if op == operator:
                rows.append((int(k), poly, rate))
    assert [r[0] for r in rows] == list(range(len(rows)))
    return rows


def basis(operator: str, E: np.ndarray) -> np.ndarray:
    """Rows of the golden polynomials evaluated at the velocities E (one row per direction of E)."""
    e = np.asarray(E, dtype=np.float64)
    env = {"ex": e[:, 0], "ey": e[:, 1], "ez": e[:, 2], "e2": (e * e).sum(1)}
    rows = []
    for _, poly, _ in rate_table(operator):
        v = eval(poly, {"__builtins__": {}}, dict(env))
        rows.append(np.broadcast_to(np.asarray(v, dtype=np.float64), (len(e),)).copy())
    return np.array(rows)


def expected_factors(operator: str, rates: dict, steps: int) -> np.ndarray:
    """(1 - s_k)^steps per row; 1 for the conserved rows."""
    out = []
    for _, _, rate in rate_table(operator):
        out.append(1.0 if rate == "conserved" else (1.0 - rates[rate]) ** steps)
    return np.array(out)


def perturbed_rest_state(operator: str, E, w_lattice, k: int, eps: float, rho0: float, grid):
    """Uniform f = w rho0 + eps M^-1 e_k on a (Nz, Ny, Nx) grid, populations first."""
    M = basis(operator, E)
    f = np.asarray(w_lattice, dtype=np.float64) * rho0 + eps * np.linalg.solve(M, np.eye(len(E))[k])
    return np.broadcast_to(f.reshape(-1, 1, 1, 1), (len(E),) + tuple(grid[::-1])).copy()


def decay_error(operator: str, E, f0: np.ndarray, f1: np.ndarray, k: int, eps: float, rates: dict,
                steps: int) -> float:
    """Largest deviation, over rows and nodes, of M f1 - M f0 from eps ((1 - s_k)^steps - 1) e_k.

    f0 is the perturbed state (m_k = rest value + eps), f1 the state ``steps`` steps later.
    """
    M = basis(operator, E)
    dm = np.tensordot(M, f1 - f0, axes=(1, 0))  # (Q, Nz, Ny, Nx)
    want = np.zeros(len(E))
    want[k] = eps * (expected_factors(operator, rates, steps)[k] - 1.0)
    return float(np.max(np.abs(dm - want.reshape(-1, 1, 1, 1))))


def non_conserved_rows(operator: str):
    return [k for k, _, rate in rate_table(operator) if rate != "conserved"]
