"""Plain FP64 numpy restatement of the D3Q19 pseudopotential MRT-LB step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): imported by the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``, never by
the product package.

Every array of populations has shape ``(19, Nz, Ny, Nx)``: direction first,
then z, y, x (x fastest), matching node index ``i = x + Nx*(y + Ny*z)``.
Directions follow the order of Eq. 2.  Lattice units: dt = dx = c = 1 and
c_s^2 = 1/3 (Sec. II B, Eq. 13).

What each piece follows:

* velocities ................................ Eq. 2
* non-orthogonal transformation matrix ..... Eqs. 7-10 (printed as Eq. 12);
  its inverse is taken with ``numpy.linalg.inv`` (printed in App. A)
* relaxation matrix ......................... Eq. 11
* equilibrium moments, forcing moments ...... Eqs. 13, 14; Eq. 16 (sigma term)
* collision in moment space ................. Eq. 4
* streaming ................................. Eq. 5
* density and velocity ...................... Eq. 6
* interaction force ......................... Eq. 15 (weights 1/6, 1/12)
* pseudopotentials .......................... Sec. II B (exp and sqrt forms)
* Carnahan-Starling equation of state ....... Eq. 58
* droplet initial density ................... Eq. 59
* flat liquid slab .......................... Sec. IV D (interfaces at lo, hi)

The orthogonal operator the paper compares against (Sec. II B, Sec. IV) is not
printed there.  Reading used: the D3Q19 orthogonal basis of d'Humieres et al.
(the paper's Ref. 11), evaluated at the Eq. 2 velocities; its equilibria are
M_o f_eq and its forcing moments M_o G with the standard second-order
equilibrium f_eq and Guo's forcing term G; its relaxation matrix applies the
same rates to the matching moment groups.  With this reading M_o and M_o^-1
both have the 213 non-zero entries the paper quotes.  Parity of this operator
with the authors' own code is unpinned beyond physics-level agreement.
"""

from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

Q = 19
CS2 = 1.0 / 3.0  # c_s^2, Eq. 13

# Eq. 2, one row per direction alpha = 0..18: (e_x, e_y, e_z).
E = np.array(
    [
        [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
        [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
        [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1],
    ],
    dtype=np.int64,
).T

# Weights of the interaction force, Eq. 15: 1/6 on the axes, 1/12 on the
# diagonals (the rest direction carries e = 0 and never contributes).
W_FORCE = np.array([0.0] + [1.0 / 6.0] * 6 + [1.0 / 12.0] * 12)

# Weights of the standard second-order D3Q19 equilibrium.  The paper never
# writes f_eq out; these are needed only for the orthogonal reading above and
# for the forcing term G in velocity space.
W_LATTICE = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)


# --------------------------------------------------------------------------
# Transformation matrices
# --------------------------------------------------------------------------
def _components():
    e = E.astype(np.float64)
    return e[:, 0], e[:, 1], e[:, 2]


def nonorth_matrix() -> np.ndarray:
    """Non-orthogonal M, rows built from the basis vectors of Eqs. 7-10."""
    ex, ey, ez = _components()
    e2 = ex * ex + ey * ey + ez * ez
    rows = [
        np.ones(Q), ex, ey, ez,                                   # Eq. 7
        e2, 3 * ex * ex - e2, ey * ey - ez * ez,                  # Eq. 8
        ex * ey, ex * ez, ey * ez,
        ex * ex * ey, ex * ey * ey, ex * ex * ez,                 # Eq. 9
        ex * ez * ez, ey * ey * ez, ey * ez * ez,
        ex * ex * ey * ey, ex * ex * ez * ez, ey * ey * ez * ez,  # Eq. 10
    ]
    return np.array(rows, dtype=np.float64)


def orth_matrix() -> np.ndarray:
    """Orthogonal D3Q19 M_o (d'Humieres et al. basis) at the Eq. 2 ordering.

    Rows: rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww,
    pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z.
    """
    ex, ey, ez = _components()
    e2 = ex * ex + ey * ey + ez * ez
    rows = [
        np.ones(Q),
        19 * e2 - 30,
        (21 * e2 * e2 - 53 * e2 + 24) / 2,
        ex, (5 * e2 - 9) * ex,
        ey, (5 * e2 - 9) * ey,
        ez, (5 * e2 - 9) * ez,
        3 * ex * ex - e2, (3 * e2 - 5) * (3 * ex * ex - e2),
        ey * ey - ez * ez, (3 * e2 - 5) * (ey * ey - ez * ez),
        ex * ey, ey * ez, ex * ez,
        (ey * ey - ez * ez) * ex, (ez * ez - ex * ex) * ey, (ex * ex - ey * ey) * ez,
    ]
    return np.array(rows, dtype=np.float64)


def inverse(M: np.ndarray) -> np.ndarray:
    """M^-1 by numpy's LU solve (App. A prints it for the non-orthogonal M)."""
    return np.linalg.inv(M)


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Params:
    """Everything one run needs.  Rates are relaxation rates s (not times).

    Non-orthogonal operator, Eq. 11: s_e (moment 4), s_nu (5-9), s_q (10-15),
    s_pi (16-18).  Orthogonal operator: s_e (e), s_eps (eps), s_q (q_i),
    s_nu (p_ij), s_pi (pi_xx, pi_ww), s_m (m_i).
    """

    grid: tuple = (32, 32, 32)  # (Nx, Ny, Nz)
    operator: str = "nonorth"  # "nonorth" | "orth"
    eos: str = "cs"  # "cs" | "exp" | "none"
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    T: float = 0.0
    psi0: float = 1.0
    rho0: float = 1.0
    G: float = -1.0
    s_e: float = 1.1
    s_nu: float = 1.0
    s_q: float = 1.1
    s_pi: float = 1.1
    s_eps: float = 1.1
    s_m: float = 1.1
    sigma: float = 0.0
    # density-dependent shear viscosity (Sec. IV D, last paragraph): nu varies
    # linearly in rho from nu_v at rho_v to nu_l at rho_l, clamped between the
    # two; s_nu(rho) = 1 / (3 nu + 1/2).  Off when nu_l is None.
    nu_l: float | None = None
    nu_v: float | None = None
    rho_l_nu: float = 1.0
    rho_v_nu: float = 0.0

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


def critical_temperature(a: float, b: float, R: float) -> float:
    """T_c of the Carnahan-Starling EOS as the paper states it (Sec. IV D)."""
    return 0.37733 * a / (b * R)


def relaxation(p: Params) -> np.ndarray:
    """Diagonal of Lambda for the chosen operator (Eq. 11 for non-orth)."""
    if p.operator == "nonorth":
        d = [1, 1, 1, 1, p.s_e] + [p.s_nu] * 5 + [p.s_q] * 6 + [p.s_pi] * 3
    elif p.operator == "orth":
        d = [1, p.s_e, p.s_eps, 1, p.s_q, 1, p.s_q, 1, p.s_q,
             p.s_nu, p.s_pi, p.s_nu, p.s_pi, p.s_nu, p.s_nu, p.s_nu,
             p.s_m, p.s_m, p.s_m]
    else:
        raise ValueError(f"unknown operator {p.operator!r}")
    return np.array(d, dtype=np.float64)


def shear_rate_field(p: Params, rho: np.ndarray) -> np.ndarray:
    """s_nu at every node: constant, or from the density-dependent viscosity."""
    if p.nu_l is None:
        return np.full(np.shape(rho), p.s_nu)
    t = (np.asarray(rho) - p.rho_v_nu) / (p.rho_l_nu - p.rho_v_nu)
    nu = p.nu_v + t * (p.nu_l - p.nu_v)
    nu = np.clip(nu, min(p.nu_l, p.nu_v), max(p.nu_l, p.nu_v))
    return 1.0 / (3.0 * nu + 0.5)


SHEAR_ROWS = {"nonorth": [5, 6, 7, 8, 9], "orth": [9, 11, 13, 14, 15]}


def matrix(p: Params) -> np.ndarray:
    return nonorth_matrix() if p.operator == "nonorth" else orth_matrix()


# --------------------------------------------------------------------------
# Equilibria and forcing
# --------------------------------------------------------------------------
def feq_standard(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Standard second-order D3Q19 equilibrium, shape (19, ...)."""
    eu = np.tensordot(E.astype(np.float64), u, axes=(1, 0))  # (19, ...)
    uu = (u * u).sum(axis=0)
    w = W_LATTICE.reshape((Q,) + (1,) * rho.ndim)
    return w * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * uu)


def guo_force_velocity_space(F: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Guo's forcing term G_alpha = w_alpha [3(e - u) + 9 (e.u) e] . F."""
    e = E.astype(np.float64)
    eu = np.tensordot(e, u, axes=(1, 0))
    eF = np.tensordot(e, F, axes=(1, 0))
    uF = (u * F).sum(axis=0)
    w = W_LATTICE.reshape((Q,) + (1,) * (F.ndim - 1))
    return w * (3 * (eF - uF) + 9 * eu * eF)


def meq_nonorth(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Equilibrium moments of the non-orthogonal operator, Eq. 13."""
    ux, uy, uz = u
    uu = ux * ux + uy * uy + uz * uz
    phi = rho * CS2 * CS2 * (1 - 1.5 * uu)
    return np.stack([
        rho, rho * ux, rho * uy, rho * uz,
        rho + rho * uu,
        rho * (2 * ux * ux - uy * uy - uz * uz),
        rho * (uy * uy - uz * uz),
        rho * ux * uy, rho * ux * uz, rho * uy * uz,
        rho * CS2 * uy, rho * CS2 * ux, rho * CS2 * uz,
        rho * CS2 * ux, rho * CS2 * uz, rho * CS2 * uy,
        phi + rho * CS2 * (ux * ux + uy * uy),
        phi + rho * CS2 * (ux * ux + uz * uz),
        phi + rho * CS2 * (uy * uy + uz * uz),
    ])


def forcing_nonorth(F: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Forcing moments S of the non-orthogonal operator, Eq. 14."""
    Fx, Fy, Fz = F
    ux, uy, uz = u
    zero = np.zeros_like(Fx)
    return np.stack([
        zero, Fx, Fy, Fz,
        2 * (Fx * ux + Fy * uy + Fz * uz),
        2 * (2 * Fx * ux - Fy * uy - Fz * uz),
        2 * (Fy * uy - Fz * uz),
        Fx * uy + Fy * ux, Fx * uz + Fz * ux, Fy * uz + Fz * uy,
        CS2 * Fy, CS2 * Fx, CS2 * Fz, CS2 * Fx, CS2 * Fz, CS2 * Fy,
        2 * CS2 * (ux * Fx + uy * Fy),
        2 * CS2 * (ux * Fx + uz * Fz),
        2 * CS2 * (uy * Fy + uz * Fz),
    ])


def _apply(M: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Matrix (19x19) times a field of 19-vectors, shape (19, ...)."""
    return (M @ v.reshape(Q, -1)).reshape(v.shape)


def meq_orth(rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Orthogonal-operator equilibria: M_o f_eq (reading stated above)."""
    return _apply(orth_matrix(), feq_standard(rho, u))


def forcing_orth(F: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Orthogonal-operator forcing moments: M_o G (Guo's G)."""
    return _apply(orth_matrix(), guo_force_velocity_space(F, u))


def sigma_term(p: Params, F: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """The extra part of S_4 in Eq. 16: 6 sigma |F_m|^2 / (psi^2 (1/s_e - 1/2))."""
    F2 = (F * F).sum(axis=0)
    return 6.0 * p.sigma * F2 / (psi * psi * (1.0 / p.s_e - 0.5))


# --------------------------------------------------------------------------
# Equation of state and pseudopotential
# --------------------------------------------------------------------------
class EOSDomainError(ValueError):
    """The density left the domain where psi is defined (Sec. IV D)."""


def pressure_cs(rho: np.ndarray, p: Params) -> np.ndarray:
    """Carnahan-Starling p_EOS, Eq. 58, with eta = b rho / 4."""
    eta = p.b * rho / 4.0
    return rho * p.R * p.T * (1 + eta + eta * eta - eta ** 3) / (1 - eta) ** 3 - p.a * rho * rho


def pseudopotential(rho: np.ndarray, p: Params) -> np.ndarray:
    """psi(rho): square-root form with the CS EOS, or the exponential form.

    sqrt form: psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2)), c = 1.
    exp form: psi = psi_0 exp(-rho_0 / rho).  "none": psi = 0 (no force).
    """
    rho = np.asarray(rho, dtype=np.float64)
    if p.eos == "none":
        return np.zeros_like(rho)
    if np.any(~np.isfinite(rho)) or np.any(rho <= 0):
        raise EOSDomainError("density must be positive and finite")
    if p.eos == "exp":
        return p.psi0 * np.exp(-p.rho0 / rho)
    if p.eos != "cs":
        raise ValueError(f"unknown eos {p.eos!r}")
    if np.any(p.b * rho / 4.0 >= 1.0):
        raise EOSDomainError("Carnahan-Starling packing fraction b*rho/4 >= 1")
    radicand = 2.0 * (pressure_cs(rho, p) - rho * CS2) / p.G
    if np.any(radicand < 0):
        raise EOSDomainError("negative radicand in the square-root pseudopotential")
    return np.sqrt(radicand)


def eos_pressure(rho: np.ndarray, p: Params) -> np.ndarray:
    """Bulk pressure of the model: p_EOS for CS; rho/3 + G psi^2/2 otherwise."""
    if p.eos == "cs":
        return pressure_cs(np.asarray(rho, dtype=np.float64), p)
    psi = pseudopotential(rho, p)
    return np.asarray(rho) * CS2 + 0.5 * p.G * psi * psi


# --------------------------------------------------------------------------
# Field operations
# --------------------------------------------------------------------------
def shifted(field: np.ndarray, e) -> np.ndarray:
    """g(x) = field(x + e) on the periodic box; field has shape (Nz, Ny, Nx)."""
    ex, ey, ez = (int(c) for c in e)
    return np.roll(field, shift=(-ez, -ey, -ex), axis=(0, 1, 2))


def interaction_force(psi: np.ndarray, G: float) -> np.ndarray:
    """Eq. 15: F(x) = -G psi(x) sum_alpha w_alpha psi(x + e_alpha) e_alpha."""
    acc = np.zeros((3,) + psi.shape)
    for a in range(1, Q):
        nb = W_FORCE[a] * shifted(psi, E[a])
        for d in range(3):
            if E[a, d] != 0:
                acc[d] += E[a, d] * nb
    return -G * psi * acc


def density(f: np.ndarray) -> np.ndarray:
    """Eq. 6: rho = sum_alpha f_alpha."""
    return f.sum(axis=0)


def velocity(f: np.ndarray, rho: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Eq. 6: rho u = sum_alpha e_alpha f_alpha + F/2."""
    j = np.tensordot(E.astype(np.float64).T, f, axes=(1, 0))  # (3, ...)
    return (j + 0.5 * F) / rho


def stream(fstar: np.ndarray) -> np.ndarray:
    """Eq. 5: f_alpha(x + e_alpha, t+1) = f*_alpha(x, t), periodic."""
    out = np.empty_like(fstar)
    for a in range(Q):
        ex, ey, ez = (int(c) for c in E[a])
        out[a] = np.roll(fstar[a], shift=(ez, ey, ex), axis=(0, 1, 2))
    return out


def collide(p: Params, f: np.ndarray, rho: np.ndarray, u: np.ndarray,
            F: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Eq. 4 followed by f* = M^-1 m*: the collision in moment space."""
    M = matrix(p)
    Minv = inverse(M)
    lam = relaxation(p)
    m = _apply(M, f)
    if p.operator == "nonorth":
        meq = meq_nonorth(rho, u)
        S = forcing_nonorth(F, u)
        if p.sigma != 0.0:
            S[4] = S[4] + sigma_term(p, F, psi)
    else:
        meq = meq_orth(rho, u)
        G = guo_force_velocity_space(F, u)
        if p.sigma != 0.0:
            # Eq. 16 carried over to the orthogonal basis: the same change of
            # the post-collision populations, M_o (M^-1 delta_4) in moments.
            G = G + np.multiply.outer(inverse(nonorth_matrix())[:, 4], sigma_term(p, F, psi))
        S = _apply(orth_matrix(), G)
    L = np.broadcast_to(lam.reshape((Q,) + (1,) * rho.ndim), (Q,) + rho.shape).copy()
    if p.nu_l is not None:
        snu = shear_rate_field(p, rho)
        for k in SHEAR_ROWS[p.operator]:
            L[k] = snu
    mstar = m - L * (m - meq) + (1 - L / 2) * S
    return _apply(Minv, mstar)


def macroscopic(p: Params, f: np.ndarray):
    """rho, u, psi and F of a post-streaming state (Eqs. 6 and 15)."""
    rho = density(f)
    psi = pseudopotential(rho, p)
    F = interaction_force(psi, p.G)
    u = velocity(f, rho, F)
    return rho, u, psi, F


def step(p: Params, f: np.ndarray) -> np.ndarray:
    """One time step t -> t+1 of the post-streaming state f_bar (Eqs. 3-6, 15)."""
    rho, u, psi, F = macroscopic(p, f)
    return stream(collide(p, f, rho, u, F, psi))


def run(p: Params, f: np.ndarray, steps: int) -> np.ndarray:
    for _ in range(steps):
        f = step(p, f)
    return f


def equilibrium_state(p: Params, rho: np.ndarray, u=None) -> np.ndarray:
    """f = M^-1 m_eq(rho, u) for the chosen operator (u = 0 if omitted)."""
    rho = np.asarray(rho, dtype=np.float64)
    if u is None:
        u = np.zeros((3,) + rho.shape)
    meq = meq_nonorth(rho, u) if p.operator == "nonorth" else meq_orth(rho, u)
    return _apply(inverse(matrix(p)), meq)


# --------------------------------------------------------------------------
# Initial density fields
# --------------------------------------------------------------------------
def _coords(grid):
    nx, ny, nz = grid
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def _min_image(d: np.ndarray, n: int) -> np.ndarray:
    d = np.abs(d)
    return np.minimum(d, n - d)


def droplet_density(grid, centre, R, W, rho_l, rho_v) -> np.ndarray:
    """Eq. 59 with r the periodic minimum-image distance to the centre."""
    x, y, z = _coords(grid)
    dx = _min_image(x - centre[0], grid[0])
    dy = _min_image(y - centre[1], grid[1])
    dz = _min_image(z - centre[2], grid[2])
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r - R) / W)


def slab_density(grid, axis, lo, hi, W, rho_l, rho_v) -> np.ndarray:
    """Liquid slab between planes lo and hi along one axis (Sec. IV D)."""
    coord = _coords(grid)[axis]
    return rho_v + 0.5 * (rho_l - rho_v) * (np.tanh(2.0 * (coord - lo) / W)
                                             - np.tanh(2.0 * (coord - hi) / W))


# --------------------------------------------------------------------------
# Diagnostics (Sec. IV B and IV D)
# --------------------------------------------------------------------------
def total_mass(f: np.ndarray) -> float:
    return float(density(f).sum())


def total_momentum(p: Params, f: np.ndarray) -> np.ndarray:
    rho, u, _, _ = macroscopic(p, f)
    return (rho * u).reshape(3, -1).sum(axis=1)
