"""Pins for equilibria, forcing moments and the collision (Eqs. 4, 13, 14, 16)."""

import numpy as np
import pytest

from oracle import lbm_oracle as L

RNG = np.random.default_rng(1805)


def _rand_state(n=7):
    rho = RNG.uniform(0.05, 2.0, n)
    u = RNG.uniform(-0.1, 0.1, (3, n))
    F = RNG.uniform(-0.01, 0.01, (3, n))
    return rho, u, F


def test_standard_equilibrium_moments_textbook():
    rho, u, _ = _rand_state()
    feq = L.feq_standard(rho, u)
    e = L.E.astype(float)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-15)
    assert np.allclose(np.tensordot(e.T, feq, 1), rho * u, rtol=0, atol=1e-15)
    pi = np.einsum("ai,aj,an->ijn", e, e, feq)
    want = np.einsum("ij,n->ijn", np.eye(3), rho / 3) + np.einsum("n,in,jn->ijn", rho, u, u)
    assert np.max(np.abs(pi - want)) < 1e-15


def test_guo_forcing_moments_textbook():
    rho, u, F = _rand_state()
    G = L.guo_force_velocity_space(F, u)
    e = L.E.astype(float)
    assert np.max(np.abs(G.sum(0))) < 1e-17
    assert np.max(np.abs(np.tensordot(e.T, G, 1) - F)) < 1e-17
    pi = np.einsum("ai,aj,an->ijn", e, e, G)
    want = np.einsum("in,jn->ijn", u, F) + np.einsum("in,jn->ijn", F, u)
    assert np.max(np.abs(pi - want)) < 1e-17


def test_eq13_matches_M_feq_up_to_second_order_moments():
    """Rows 0-15 of Eq. 13 are M f_eq; rows 16-18 are the paper's own choice."""
    rho, u, _ = _rand_state()
    M = L.nonorth_matrix()
    direct = M @ L.feq_standard(rho, u)
    meq = L.meq_nonorth(rho, u)
    assert np.max(np.abs(direct[:16] - meq[:16])) < 1e-15
    # The fourth-order rows differ from M f_eq by rho (u_i^2 + u_j^2)/6.
    ux, uy, uz = u
    diff = direct[16:] - meq[16:]
    want = rho * np.stack([ux * ux + uy * uy, ux * ux + uz * uz, uy * uy + uz * uz]) / 6
    assert np.max(np.abs(diff - want)) < 1e-15


def test_eq14_matches_M_guo_up_to_second_order_moments():
    _, u, F = _rand_state()
    M = L.nonorth_matrix()
    direct = M @ L.guo_force_velocity_space(F, u)
    S = L.forcing_nonorth(F, u)
    assert np.max(np.abs(direct[:16] - S[:16])) < 1e-17


def test_orth_equilibria_closed_form():
    rho, u, _ = _rand_state()
    ux, uy, uz = u
    uu = ux * ux + uy * uy + uz * uz
    pxx = 2 * ux * ux - uy * uy - uz * uz
    pww = uy * uy - uz * uz
    want = rho * np.stack([
        np.ones_like(ux), -11 + 19 * uu, 3 - 5.5 * uu,
        ux, -2 / 3 * ux, uy, -2 / 3 * uy, uz, -2 / 3 * uz,
        pxx, -pxx / 2, pww, -pww / 2, ux * uy, uy * uz, ux * uz,
        0 * ux, 0 * ux, 0 * ux])
    assert np.max(np.abs(L.meq_orth(rho, u) - want)) < 1e-14


def test_orth_forcing_closed_form():
    _, u, F = _rand_state()
    ux, uy, uz = u
    Fx, Fy, Fz = F
    Fu = Fx * ux + Fy * uy + Fz * uz
    axx = 2 * Fx * ux - Fy * uy - Fz * uz
    aww = Fy * uy - Fz * uz
    z = 0 * Fx
    want = np.stack([z, 38 * Fu, -11 * Fu, Fx, -2 / 3 * Fx, Fy, -2 / 3 * Fy, Fz, -2 / 3 * Fz,
                     2 * axx, -axx, 2 * aww, -aww, Fx * uy + Fy * ux, Fy * uz + Fz * uy,
                     Fx * uz + Fz * ux, z, z, z])
    assert np.max(np.abs(L.forcing_orth(F, u) - want)) < 1e-16


@pytest.mark.parametrize("op", ["nonorth", "orth"])
def test_equilibrium_is_fixed_point_without_force(op):
    p = L.Params(operator=op, s_e=0.8, s_nu=1.3, s_q=1.2, s_pi=0.9, s_eps=1.4, s_m=1.7)
    rho, u, _ = _rand_state()
    f = L.equilibrium_state(p, rho, u)
    F = np.zeros_like(u)
    fstar = L.collide(p, f, rho, u, F, np.ones_like(rho))
    assert np.max(np.abs(fstar - f)) < 1e-15


@pytest.mark.parametrize("op", ["nonorth", "orth"])
def test_collision_conserves_mass_and_adds_force(op):
    p = L.Params(operator=op, s_e=0.8, s_nu=1.3, s_q=1.2, s_pi=0.9, s_eps=1.4, s_m=1.7)
    rho, u, F = _rand_state()
    f = L.equilibrium_state(p, rho, u) + RNG.normal(0, 1e-3, (19, rho.size))
    rho = f.sum(0)
    u = L.velocity(f, rho, F)
    fstar = L.collide(p, f, rho, u, F, np.ones_like(rho))
    e = L.E.astype(float)
    assert np.max(np.abs(fstar.sum(0) - rho)) < 1e-14
    # Eq. 4 with Lambda = 1 on j and S_1..3 = F: j* = rho u + F/2 = j + F.
    assert np.max(np.abs(np.tensordot(e.T, fstar, 1) - np.tensordot(e.T, f, 1) - F)) < 1e-15


def test_operators_agree_at_rest_and_differ_in_motion():
    rho, u, F = _rand_state()
    zero = np.zeros_like(u)
    out = {}
    for op in ("nonorth", "orth"):
        p = L.Params(operator=op)
        f = L.equilibrium_state(L.Params(operator="nonorth"), rho) + 1e-3 * RNG.normal(size=(19, rho.size))
        out[op] = (L.collide(p, f, rho, zero, zero, np.ones_like(rho)),
                   L.collide(p, L.feq_standard(rho, u), rho, u, F, np.ones_like(rho)))
    assert not np.allclose(out["nonorth"][1], out["orth"][1], atol=1e-10)


def test_sigma_term_changes_only_moment_4():
    p = L.Params(sigma=0.105, s_e=0.8)
    rho, u, F = _rand_state()
    psi = RNG.uniform(0.1, 1.0, rho.size)
    f = L.feq_standard(rho, u)
    a = L.collide(p, f, rho, u, F, psi)
    b = L.collide(p.with_(sigma=0.0), f, rho, u, F, psi)
    dm = L.nonorth_matrix() @ (a - b)
    delta = 6 * 0.105 * (F * F).sum(0) / (psi * psi * (1 / 0.8 - 0.5))
    want = np.zeros_like(dm)
    want[4] = (1 - 0.8 / 2) * delta
    assert np.max(np.abs(dm - want)) < 1e-15
    # The orthogonal reading carries the same velocity-space change.
    po = p.with_(operator="orth")
    fo = L.collide(po, f, rho, u, F, psi) - L.collide(po.with_(sigma=0.0), f, rho, u, F, psi)
    dmo = L.orth_matrix() @ fo
    lam = L.relaxation(po)
    want_o = (1 - lam[:, None] / 2) * np.multiply.outer(np.array([0, 19, -16] + [0] * 16, float), delta)
    # (differences of two collisions: round-off of |M_o f| ~ 30 |f| eps)
    assert np.max(np.abs(dmo - want_o)) < 1e-13
