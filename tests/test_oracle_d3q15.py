"""Pins for the D3Q15 variant of the oracle (Sec. II A: "constructed in a similar way").

The paper gives no D3Q15 model, so each pin checks the construction against
something fixed outside it: the textbook D3Q15 lattice conditions, the paper's
own D3Q19 rows (restated in ``lbm_oracle`` and pinned there against Eqs. 12-14),
exact rational inverses, invariants and the closed-form viscosities of Eq. 54.
"""

from fractions import Fraction

import numpy as np
import pytest
from scipy.optimize import curve_fit

from oracle import d3q15 as D
from oracle import lbm_oracle as L
from oracle import maxwell

RNG = np.random.default_rng(1805)


def _droplet(grid=(16, 16, 16), T_over_Tc=0.8, R=4.0, W=2.0, **kw):
    p = L.Params(grid=grid, T=T_over_Tc * L.critical_temperature(1.0, 4.0, 1.0), **kw)
    rl, rv = maxwell.coexistence_cs(T_over_Tc)
    rho = L.droplet_density(grid, tuple(n / 2 for n in grid), R, W, rl, rv)
    return p, D.equilibrium_state(p, rho)


# ---------------------------------------------------------------- lattice
def test_velocities_are_the_d3q15_set_with_opposites_adjacent():
    v = {tuple(int(c) for c in r) for r in D.E}
    want = {(0, 0, 0)} | {tuple(s * (i == k) for k in range(3)) for i in range(3) for s in (1, -1)}
    want |= {(a, b, c) for a in (1, -1) for b in (1, -1) for c in (1, -1)}
    assert len(D.E) == 15 and v == want
    for a in range(1, 15, 2):
        assert np.all(D.E[a] == -D.E[a + 1])
    # the rest and axis directions are those of Eq. 2, in its order
    assert np.all(D.E[:7] == L.E[:7])


def _tensor_sums(w, e):
    e = e.astype(np.float64)
    s2 = np.einsum("a,ai,aj->ij", w, e, e)
    s4 = np.einsum("a,ai,aj,ak,al->ijkl", w, e, e, e, e)
    s1 = np.einsum("a,ai->i", w, e)
    s3 = np.einsum("a,ai,aj,ak->ijk", w, e, e, e)
    return s1, s2, s3, s4


def test_equilibrium_weights_meet_the_textbook_isotropy_conditions():
    # sum w = 1, sum w e e = c_s^2 I, sum w e e e e = c_s^4 (dd + dd + dd), odd sums 0
    s1, s2, s3, s4 = _tensor_sums(D.W_LATTICE, D.E)
    d = np.eye(3)
    iso4 = (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)) / 9
    assert abs(D.W_LATTICE.sum() - 1) < 1e-15
    assert np.max(np.abs(s2 - d / 3)) < 1e-15 and np.max(np.abs(s4 - iso4)) < 1e-15
    assert np.max(np.abs(s1)) == 0 and np.max(np.abs(s3)) == 0


def test_force_weights_have_the_d3q19_weights_second_and_fourth_order_sums():
    q15 = _tensor_sums(D.W_FORCE, D.E)
    q19 = _tensor_sums(L.W_FORCE, L.E)
    for a, b in zip(q15, q19):
        assert np.max(np.abs(a - b)) < 1e-15
    assert abs(q15[1][0, 0] - 1) < 1e-15  # sum w e_x e_x = 1: F = -G psi grad psi to leading order


# ---------------------------------------------------------------- matrix
def _exact(M):
    return [[Fraction(int(round(v))) for v in row] for row in M]


def _exact_inverse(A):
    n = len(A)
    aug = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if aug[r][c] != 0)
        aug[c], aug[piv] = aug[piv], aug[c]
        pv = aug[c][c]
        aug[c] = [v / pv for v in aug[c]]
        for r in range(n):
            if r != c and aug[r][c] != 0:
                k = aug[r][c]
                aug[r] = [a - k * b for a, b in zip(aug[r], aug[c])]
    return [row[n:] for row in aug]


def test_matrix_is_invertible_and_numpy_inverse_is_the_exact_one():
    M = D.nonorth_matrix()
    Minv_exact = _exact_inverse(_exact(M))
    Minv = np.linalg.inv(M)
    assert np.max(np.abs(Minv - np.array([[float(v) for v in r] for r in Minv_exact]))) < 1e-15
    assert int((M != 0).sum()) == 133
    assert sum(v != 0 for r in Minv_exact for v in r) == 101


def test_rows_agree_with_eq12_on_the_shared_velocities():
    # D3Q15 row k and D3Q19 row k19 are the same monomial: equal on rest + axes
    pairs = [(k, k) for k in range(13)] + [(14, 16)]
    M15, M19 = D.nonorth_matrix(), L.nonorth_matrix()
    for k, k19 in pairs:
        assert np.all(M15[k, :7] == M19[k19, :7])
    assert np.all(M15[13, :7] == 0)  # e_x e_y e_z vanishes off the corners


def test_coinciding_eq9_and_eq10_vectors_on_d3q15():
    e = D.E.astype(np.float64)
    ex, ey, ez = e.T
    M = D.nonorth_matrix()
    assert np.all(M[10] == ey * ez * ez) and np.all(M[11] == ex * ez * ez) and np.all(M[12] == ey * ey * ez)
    assert np.all(M[14] == ex * ex * ez * ez) and np.all(M[14] == ey * ey * ez * ez)


def test_rates_are_the_eq11_rates_of_the_coinciding_d3q19_rows():
    # distinct rates for every group, so a swapped assignment shows
    p = L.Params(s_e=0.71, s_nu=1.13, s_q=1.27, s_pi=0.93, s_eps=1.5, s_m=1.6)
    r15, r19 = D.relaxation(p), L.relaxation(p)
    for k in range(10):
        assert r15[k] == r19[k]
    for k, pair in ((10, (10, 15)), (11, (11, 13)), (12, (12, 14))):
        assert all(r15[k] == r19[k19] for k19 in pair)
    assert all(r15[14] == r19[k19] for k19 in (16, 17, 18))
    assert r15[13] == p.s_q  # e_x e_y e_z: third order, the Eq. 11 third-order rate
    assert L.relaxation(p)[10] == p.s_q and L.relaxation(p)[16] == p.s_pi  # Eq. 11 itself


# ---------------------------------------------------------------- equilibria, forcing
def test_rest_state_is_the_textbook_weights():
    rho = RNG.uniform(0.1, 2.0, 7)
    f = D.equilibrium_state(L.Params(), rho)
    assert np.max(np.abs(f - np.multiply.outer(D.W_LATTICE, rho))) < 1e-15


def test_equilibria_rows_0_to_13_are_moments_of_the_textbook_equilibrium():
    rho = RNG.uniform(0.1, 2.0, 11)
    u = RNG.uniform(-0.1, 0.1, (3, 11))
    want = D._apply(D.nonorth_matrix(), D.feq_standard(rho, u))
    assert np.max(np.abs(D.meq(rho, u)[:14] - want[:14])) < 1e-15


def test_equilibria_rows_take_the_eq13_values_of_the_coinciding_d3q19_rows():
    rho = RNG.uniform(0.1, 2.0, 9)
    u = RNG.uniform(-0.1, 0.1, (3, 9))
    m15, m19 = D.meq(rho, u), L.meq_nonorth(rho, u)
    for k in range(10):
        assert np.max(np.abs(m15[k] - m19[k])) < 1e-15
    for k, pair in ((10, (10, 15)), (11, (11, 13)), (12, (12, 14))):
        for k19 in pair:
            assert np.max(np.abs(m15[k] - m19[k19])) < 1e-15
    assert np.max(np.abs(m15[14] - m19[16:19].mean(axis=0))) < 1e-15
    assert np.max(np.abs(m15[13])) == 0


def test_forcing_rows_0_to_13_are_moments_of_guo_forcing_and_row_14_the_eq14_mean():
    F = RNG.normal(0, 1e-3, (3, 8))
    u = RNG.uniform(-0.1, 0.1, (3, 8))
    S = D.forcing(F, u)
    want = D._apply(D.nonorth_matrix(), D.guo_force_velocity_space(F, u))
    assert np.max(np.abs(S[:14] - want[:14])) < 1e-16
    assert np.max(np.abs(S[14] - L.forcing_nonorth(F, u)[16:19].mean(axis=0))) < 1e-16


def test_equilibrium_is_a_fixed_point_without_force():
    p = L.Params(s_e=0.7, s_nu=1.3, s_q=1.1, s_pi=0.9)
    rho = RNG.uniform(0.1, 1.0, (3, 4, 5))
    u = RNG.uniform(-0.05, 0.05, (3, 3, 4, 5))
    f = D.equilibrium_state(p, rho, u)
    out = D.collide(p, f, rho, u, np.zeros_like(u), np.ones_like(rho))
    assert np.max(np.abs(out - f)) < 1e-15


def test_collision_conserves_mass_and_adds_the_force_to_momentum():
    p = L.Params()
    rho = RNG.uniform(0.1, 1.0, (2, 3, 4))
    f = D.equilibrium_state(p, rho) + RNG.normal(0, 1e-3, (15, 2, 3, 4))
    F = RNG.normal(0, 1e-3, (3, 2, 3, 4))
    rho = D.density(f)
    u = D.velocity(f, rho, F)
    out = D.collide(p, f, rho, u, F, np.ones_like(rho))
    j_in = np.tensordot(D.E.T.astype(float), f, axes=(1, 0))
    j_out = np.tensordot(D.E.T.astype(float), out, axes=(1, 0))
    assert np.max(np.abs(D.density(out) - rho)) < 1e-15
    assert np.max(np.abs(j_out - (j_in + F))) < 1e-15


# ---------------------------------------------------------------- streaming, force
def test_streaming_moves_each_population_along_its_velocity():
    for a in range(15):
        fstar = np.zeros((15, 3, 4, 5))
        fstar[a, 1, 2, 3] = 1.0
        out = D.stream(fstar)
        ex, ey, ez = D.E[a]
        assert out[a][((1 + ez) % 3, (2 + ey) % 4, (3 + ex) % 5)] == 1.0 and out.sum() == 1.0


def test_force_vanishes_for_uniform_psi_sums_to_zero_and_has_the_gradient_limit():
    assert np.max(np.abs(D.interaction_force(np.full((5, 6, 7), 0.3), -1.0))) == 0.0
    F = D.interaction_force(RNG.uniform(0.1, 1.0, (5, 6, 7)), -1.0)
    assert np.max(np.abs(F.reshape(3, -1).sum(1))) < 1e-13
    n = 64
    k = 2 * np.pi / n
    z = np.meshgrid(np.arange(n), np.arange(4), np.arange(4), indexing="ij")[0]
    psi = 1.0 + 0.1 * np.sin(k * z)
    F = D.interaction_force(psi, -1.7)
    want = 1.7 * psi * 0.1 * k * np.cos(k * z)
    assert np.max(np.abs(F[2] - want)) < 2 * k * k * np.max(np.abs(want))
    assert np.max(np.abs(F[:2])) < 1e-15


# ---------------------------------------------------------------- invariants
def test_mass_and_momentum_conserved():
    p, f = _droplet()
    m0, P0 = D.total_mass(f), D.total_momentum(p, f)
    f = D.run(p, f, 60)
    assert abs(D.total_mass(f) - m0) < 1e-13 * m0
    assert np.max(np.abs(D.total_momentum(p, f) - P0)) < 1e-13 * m0


def test_uniform_state_stays_uniform():
    p = L.Params(grid=(4, 5, 3), T=0.9 * L.critical_temperature(1, 4, 1))
    u = np.zeros((3, 3, 5, 4))
    u[0], u[1], u[2] = 0.01, -0.02, 0.005
    f0 = D.equilibrium_state(p, np.full((3, 5, 4), 0.2), u)
    f = D.run(p, f0, 10)
    assert np.max(f.reshape(15, -1).max(1) - f.reshape(15, -1).min(1)) < 1e-15
    assert np.max(np.abs(f - f0)) < 1e-14


def test_centred_droplet_keeps_mirror_and_axis_symmetry():
    p, f = _droplet()
    rho, u, _, _ = D.macroscopic(p, D.run(p, f, 30))
    idx = (-np.arange(16)) % 16
    assert np.max(np.abs(rho - rho[:, :, idx])) < 1e-13
    assert np.max(np.abs(rho - rho[:, idx, :])) < 1e-13
    assert np.max(np.abs(rho - rho[idx, :, :])) < 1e-13
    assert np.max(np.abs(rho - np.transpose(rho, (0, 2, 1)))) < 1e-13
    assert np.max(np.abs(rho - np.transpose(rho, (2, 1, 0)))) < 1e-13
    assert np.max(np.abs(u[0] + u[0][:, :, idx])) < 1e-13


def test_sqrt_pseudopotential_is_independent_of_G():
    p, f0 = _droplet()
    assert np.max(np.abs(D.run(p, f0, 15) - D.run(p.with_(G=-2.5), f0, 15))) < 1e-13


# ---------------------------------------------------------------- closed forms (Eq. 54)
@pytest.mark.parametrize("s_nu", [1.0, 1.6])
def test_shear_wave_decays_with_eq54_viscosity(s_nu):
    nz, steps = 64, 200
    p = L.Params(grid=(3, 3, nz), eos="none", G=0.0, s_nu=s_nu, s_e=0.9, s_q=1.2, s_pi=1.3)
    k = 2 * np.pi / nz
    z = np.broadcast_to(np.arange(nz)[:, None, None], (nz, 3, 3))
    u = np.zeros((3, nz, 3, 3))
    u[0] = 1e-3 * np.sin(k * z)
    f = D.equilibrium_state(p, np.ones((nz, 3, 3)), u)

    def amp(f):
        return 2 * np.mean(D.macroscopic(p, f)[1][0] * np.sin(k * z))

    ratio = amp(D.run(p, f, steps)) / amp(f)
    nu = (1 / s_nu - 0.5) / 3
    assert abs(ratio / np.exp(-nu * k * k * steps) - 1) < 0.003


def test_sound_wave_speed_and_bulk_viscosity_eq54():
    nz, steps, s_e, s_nu = 64, 400, 0.8, 1.2
    p = L.Params(grid=(3, 3, nz), eos="none", G=0.0, s_nu=s_nu, s_e=s_e, s_q=1.2, s_pi=1.3)
    k = 2 * np.pi / nz
    z = np.broadcast_to(np.arange(nz)[:, None, None], (nz, 3, 3))
    f = D.equilibrium_state(p, 1 + 1e-4 * np.cos(k * z))
    a = []
    for _ in range(steps):
        a.append(2 * np.mean((D.density(f) - 1) * np.cos(k * z)))
        f = D.step(p, f)
    t = np.arange(steps)
    popt, _ = curve_fit(lambda t, A, g, w, ph: A * np.exp(-g * t) * np.cos(w * t + ph),
                        t, np.array(a), p0=[1e-4, 1e-3, k / np.sqrt(3), 0.0])
    nu = (1 / s_nu - 0.5) / 3
    nu_b = 2.0 / 9.0 * (1 / s_e - 0.5)
    assert abs(popt[1] / (k * k / 2 * (4 * nu / 3 + nu_b)) - 1) < 0.01
    assert abs(popt[2] / (k / np.sqrt(3)) - 1) < 0.002


# ---------------------------------------------------------------- brute force
def test_vectorised_step_matches_brute_force_loops():
    p = L.Params(grid=(3, 4, 5), T=0.8 * L.critical_temperature(1, 4, 1), sigma=0.1)
    rho = RNG.uniform(0.05, 0.3, (5, 4, 3))
    u = RNG.uniform(-0.02, 0.02, (3, 5, 4, 3))
    f = D.equilibrium_state(p, rho, u) + RNG.normal(0, 1e-4, (15, 5, 4, 3))
    nx, ny, nz = p.grid
    M = D.nonorth_matrix()
    Minv = np.linalg.inv(M)
    lam = D.relaxation(p)
    e = [tuple(int(c) for c in r) for r in D.E]
    wF = [0.0] + [1 / 3] * 6 + [1 / 24] * 8
    rho = f.sum(axis=0)
    psi = L.pseudopotential(rho, p)
    out = np.zeros_like(f)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                S = [sum(wF[a] * psi[(z + e[a][2]) % nz, (y + e[a][1]) % ny, (x + e[a][0]) % nx] * e[a][d]
                         for a in range(1, 15)) for d in range(3)]
                F = [-p.G * psi[z, y, x] * s for s in S]
                r = rho[z, y, x]
                uu = [(sum(e[a][d] * f[a, z, y, x] for a in range(15)) + 0.5 * F[d]) / r for d in range(3)]
                m = [sum(M[k, a] * f[a, z, y, x] for a in range(15)) for k in range(15)]
                meq = D.meq(np.array([r]), np.array(uu)[:, None])[:, 0]
                Sm = D.forcing(np.array(F)[:, None], np.array(uu)[:, None])[:, 0]
                Sm[4] += 6 * p.sigma * sum(c * c for c in F) / (psi[z, y, x] ** 2 * (1 / p.s_e - 0.5))
                ms = [m[k] - lam[k] * (m[k] - meq[k]) + (1 - lam[k] / 2) * Sm[k] for k in range(15)]
                for a in range(15):
                    out[a, (z + e[a][2]) % nz, (y + e[a][1]) % ny, (x + e[a][0]) % nx] = \
                        sum(Minv[a, k] * ms[k] for k in range(15))
    assert np.max(np.abs(D.step(p, f) - out)) < 1e-15


# ---------------------------------------------------------------- physics (Eq. 16, Maxwell)
def test_flat_interface_coexistence_with_the_sigma_term_matches_maxwell_and_d3q19():
    # The force weights carry the D3Q19 second- and fourth-order sums, so the
    # sigma of Eq. 16 that makes D3Q19 thermodynamically consistent does the
    # same here: a slab at T = 0.8 T_c settles at the Maxwell densities (Sec. IV D
    # scatter: under 1 % for rho_L, a few % for rho_V) and at D3Q19's densities.
    p = L.Params(grid=(1, 1, 64), T=0.8 * L.critical_temperature(1, 4, 1), sigma=0.116,
                 s_nu=1.0, s_e=1.1, s_q=1.1, s_pi=1.1)
    rl, rv = maxwell.coexistence_cs(0.8)
    rho0 = L.slab_density(p.grid, 2, 16, 48, 2.0, rl, rv)
    r15 = D.density(D.run(p, D.equilibrium_state(p, rho0), 4000))
    r19 = L.density(L.run(p, L.equilibrium_state(p, rho0), 4000))
    assert abs(r15[32, 0, 0] / rl - 1) < 0.01 and abs(r15[0, 0, 0] / rv - 1) < 0.06
    assert abs(r15[32, 0, 0] / r19[32, 0, 0] - 1) < 1e-6 and abs(r15[0, 0, 0] / r19[0, 0, 0] - 1) < 1e-6
    without = D.density(D.run(p.with_(sigma=0.0), D.equilibrium_state(p, rho0), 2000))
    assert abs(without[0, 0, 0] / rv - 1) > 0.3  # the sigma term is what brings rho_V there
