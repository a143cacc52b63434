"""Plain FP64 numpy restatement of the D3Q15 non-orthogonal MRT variant.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper builds its non-orthogonal operator on D3Q19 and states that the
D3Q15 model "can be constructed in a similar way" (Sec. II A) without giving
it.  This module is that construction, read as follows (every reading is
pinned in ``tests/test_oracle_d3q15.py``):

* Velocities: rest, the six axis directions in the order of Eq. 2, then the
  eight corners (+-1, +-1, +-1) with opposite pairs adjacent.
* Basis (Eqs. 7-10 carried over): the raw monomials of Eqs. 7-10 evaluated
  on the D3Q15 velocities.  On D3Q15 the third-order pairs e_x^2 e_y and
  e_y e_z^2 (and the two other pairs like it) are the same vector, and the
  three fourth-order vectors of Eq. 10 are one (the corner indicator); in
  their place D3Q15 carries e_x e_y e_z, which is zero on every D3Q19
  velocity.  Rows: 1, e_x, e_y, e_z | |e|^2, 3e_x^2-|e|^2, e_y^2-e_z^2,
  e_x e_y, e_x e_z, e_y e_z | e_x^2 e_y, e_x e_y^2, e_x^2 e_z, e_x e_y e_z |
  e_x^2 e_y^2.  M has 133 non-zero entries and M^-1 101.
* Equilibria and forcing moments: each row takes the Eq. 13 / Eq. 14 value
  of the D3Q19 rows whose vector it is on D3Q15, the mean of them where
  several coincide (the fourth-order row: phi + (2/3) rho c_s^2 |u|^2 and
  (4/3) c_s^2 F.u); e_x e_y e_z takes its second-order Maxwellian moment
  and forcing, both zero.  Rows 0-13 then equal M f_eq and M G of the
  standard second-order D3Q15 equilibrium and Guo forcing.
* Relaxation (Eq. 11 carried over): 1 on the conserved moments, s_e on
  |e|^2, s_nu on the five other second-order rows, s_q on the four
  third-order rows, s_pi on the fourth-order row.
* Interaction force (Eq. 15): weights 1/3 on the axes and 1/24 on the
  corners, the D3Q15 weights whose second- and fourth-order sums equal those
  of the D3Q19 weights 1/6, 1/12 the paper gives, so the force has the same
  leading-order expansion and the sigma term of Eq. 16 carries over.

Everything else (equation of state, pseudopotential, Eq. 16 term, initial
fields) is lattice independent and taken from ``lbm_oracle``.
"""

from __future__ import annotations

import numpy as np

from . import lbm_oracle as L

Q = 15
CS2 = L.CS2

# one row per direction: (e_x, e_y, e_z)
E = np.array(
    [
        [0, 0, 0],
        [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
        [1, 1, 1], [-1, -1, -1], [1, 1, -1], [-1, -1, 1],
        [1, -1, 1], [-1, 1, -1], [-1, 1, 1], [1, -1, -1],
    ],
    dtype=np.int64,
)

# interaction-force weights (Eq. 15 on D3Q15)
W_FORCE = np.array([0.0] + [1.0 / 3.0] * 6 + [1.0 / 24.0] * 8)

# weights of the standard second-order D3Q15 equilibrium (rest state f = w rho)
W_LATTICE = np.array([2.0 / 9.0] + [1.0 / 9.0] * 6 + [1.0 / 72.0] * 8)


def nonorth_matrix() -> np.ndarray:
    """M of the D3Q15 non-orthogonal operator, rows from the monomials listed above."""
    e = E.astype(np.float64)
    ex, ey, ez = e[:, 0], e[:, 1], e[:, 2]
    e2 = ex * ex + ey * ey + ez * ez
    rows = [
        np.ones(Q), ex, ey, ez,
        e2, 3 * ex * ex - e2, ey * ey - ez * ez,
        ex * ey, ex * ez, ey * ez,
        ex * ex * ey, ex * ey * ey, ex * ex * ez, ex * ey * ez,
        ex * ex * ey * ey,
    ]
    return np.array(rows, dtype=np.float64)


def relaxation(p: L.Params) -> np.ndarray:
    """Diagonal of Lambda (Eq. 11 carried over to the 15 rows)."""
    return np.array([1, 1, 1, 1, p.s_e] + [p.s_nu] * 5 + [p.s_q] * 4 + [p.s_pi], dtype=np.float64)


SHEAR_ROWS = [5, 6, 7, 8, 9]


def meq(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Equilibrium moments: Eq. 13 rows as they fall on D3Q15."""
    ux, uy, uz = u
    uu = ux * ux + uy * uy + uz * uz
    phi = rho * CS2 * CS2 * (1 - 1.5 * uu)
    zero = np.zeros_like(rho)
    return np.stack([
        rho, rho * ux, rho * uy, rho * uz,
        rho + rho * uu,
        rho * (2 * ux * ux - uy * uy - uz * uz),
        rho * (uy * uy - uz * uz),
        rho * ux * uy, rho * ux * uz, rho * uy * uz,
        rho * CS2 * uy, rho * CS2 * ux, rho * CS2 * uz,
        zero,
        phi + 2.0 / 3.0 * rho * CS2 * uu,
    ])


def forcing(F: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Forcing moments: Eq. 14 rows as they fall on D3Q15."""
    Fx, Fy, Fz = F
    ux, uy, uz = u
    Fu = Fx * ux + Fy * uy + Fz * uz
    zero = np.zeros_like(Fx)
    return np.stack([
        zero, Fx, Fy, Fz,
        2 * Fu,
        2 * (2 * Fx * ux - Fy * uy - Fz * uz),
        2 * (Fy * uy - Fz * uz),
        Fx * uy + Fy * ux, Fx * uz + Fz * ux, Fy * uz + Fz * uy,
        CS2 * Fy, CS2 * Fx, CS2 * Fz,
        zero,
        4.0 / 3.0 * CS2 * Fu,
    ])


def feq_standard(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Standard second-order D3Q15 equilibrium, shape (15, ...)."""
    eu = np.tensordot(E.astype(np.float64), u, axes=(1, 0))
    uu = (u * u).sum(axis=0)
    w = W_LATTICE.reshape((Q,) + (1,) * rho.ndim)
    return w * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * uu)


def guo_force_velocity_space(F: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Guo's forcing term on D3Q15: w_alpha [3(e - u) + 9 (e.u) e] . F."""
    e = E.astype(np.float64)
    eu = np.tensordot(e, u, axes=(1, 0))
    eF = np.tensordot(e, F, axes=(1, 0))
    uF = (u * F).sum(axis=0)
    w = W_LATTICE.reshape((Q,) + (1,) * (F.ndim - 1))
    return w * (3 * (eF - uF) + 9 * eu * eF)


def _apply(M: np.ndarray, v: np.ndarray) -> np.ndarray:
    return (M @ v.reshape(Q, -1)).reshape(v.shape)


def interaction_force(psi: np.ndarray, G: float) -> np.ndarray:
    """Eq. 15 with the D3Q15 weights: F = -G psi(x) sum_a w_a psi(x + e_a) e_a."""
    acc = np.zeros((3,) + psi.shape)
    for a in range(1, Q):
        nb = W_FORCE[a] * L.shifted(psi, E[a])
        for d in range(3):
            if E[a, d] != 0:
                acc[d] += E[a, d] * nb
    return -G * psi * acc


def density(f: np.ndarray) -> np.ndarray:
    """Eq. 6: rho = sum_alpha f_alpha."""
    return f.sum(axis=0)


def velocity(f: np.ndarray, rho: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Eq. 6: rho u = sum_alpha e_alpha f_alpha + F/2."""
    j = np.tensordot(E.astype(np.float64).T, f, axes=(1, 0))
    return (j + 0.5 * F) / rho


def stream(fstar: np.ndarray) -> np.ndarray:
    """Eq. 5: f_alpha(x + e_alpha, t+1) = f*_alpha(x, t), periodic."""
    out = np.empty_like(fstar)
    for a in range(Q):
        ex, ey, ez = (int(c) for c in E[a])
        out[a] = np.roll(fstar[a], shift=(ez, ey, ex), axis=(0, 1, 2))
    return out


def collide(p: L.Params, f, rho, u, F, psi) -> np.ndarray:
    """Eq. 4 in the D3Q15 moment space, then f* = M^-1 m*."""
    M = nonorth_matrix()
    Minv = np.linalg.inv(M)
    m = _apply(M, f)
    S = forcing(F, u)
    if p.sigma != 0.0:
        S[4] = S[4] + L.sigma_term(p, F, psi)
    lam = relaxation(p)
    Lm = np.broadcast_to(lam.reshape((Q,) + (1,) * rho.ndim), (Q,) + rho.shape).copy()
    if p.nu_l is not None:
        snu = L.shear_rate_field(p, rho)
        for k in SHEAR_ROWS:
            Lm[k] = snu
    mstar = m - Lm * (m - meq(rho, u)) + (1 - Lm / 2) * S
    return _apply(Minv, mstar)


def macroscopic(p: L.Params, f: np.ndarray):
    """rho, u, psi and F of a post-streaming state (Eqs. 6 and 15)."""
    rho = density(f)
    psi = L.pseudopotential(rho, p)
    F = interaction_force(psi, p.G)
    return rho, velocity(f, rho, F), psi, F


def step(p: L.Params, f: np.ndarray) -> np.ndarray:
    """One time step t -> t+1 of the post-streaming state (Eqs. 3-6, 15)."""
    rho, u, psi, F = macroscopic(p, f)
    return stream(collide(p, f, rho, u, F, psi))


def run(p: L.Params, f: np.ndarray, steps: int) -> np.ndarray:
    for _ in range(steps):
        f = step(p, f)
    return f


def equilibrium_state(p: L.Params, rho, u=None) -> np.ndarray:
    """f = M^-1 m_eq(rho, u) (u = 0 if omitted)."""
    rho = np.asarray(rho, dtype=np.float64)
    if u is None:
        u = np.zeros((3,) + rho.shape)
    return _apply(np.linalg.inv(nonorth_matrix()), meq(rho, u))


def total_mass(f: np.ndarray) -> float:
    return float(density(f).sum())


def total_momentum(p: L.Params, f: np.ndarray) -> np.ndarray:
    rho, u, _, _ = macroscopic(p, f)
    return (rho * u).reshape(3, -1).sum(axis=1)
