"""Pins for the oracle's time step: streaming, force, invariants, closed forms."""

import numpy as np
import pytest
from scipy.optimize import curve_fit

from oracle import lbm_oracle as L
from oracle import maxwell

RNG = np.random.default_rng(20180522)
OPS = ["nonorth", "orth"]


def _droplet_params(grid=(16, 16, 16), op="nonorth", T_over_Tc=0.8):
    Tc = L.critical_temperature(1.0, 4.0, 1.0)
    return L.Params(grid=grid, operator=op, T=T_over_Tc * Tc)


def _droplet_state(p, R=4.0, W=2.0, T_over_Tc=0.8):
    rl, rv = maxwell.coexistence_cs(T_over_Tc)
    c = tuple(n / 2 for n in p.grid)
    rho = L.droplet_density(p.grid, c, R, W, rl, rv)
    return L.equilibrium_state(p, rho)


# ---------------------------------------------------------------- streaming
def test_streaming_moves_each_population_along_its_velocity():
    grid = (5, 4, 3)
    for a in range(19):
        fstar = np.zeros((19, 3, 4, 5))
        fstar[a, 1, 2, 3] = 1.0  # node (x, y, z) = (3, 2, 1)
        out = L.stream(fstar)
        ex, ey, ez = L.E[a]
        want = ((1 + ez) % 3, (2 + ey) % 4, (3 + ex) % 5)
        assert out[a][want] == 1.0 and out.sum() == 1.0


# ---------------------------------------------------------------- force (Eq. 15)
def test_force_vanishes_for_uniform_psi_and_sums_to_zero():
    psi = np.full((5, 6, 7), 0.37)
    assert np.max(np.abs(L.interaction_force(psi, -1.0))) == 0.0
    psi = RNG.uniform(0.1, 1.0, (5, 6, 7))
    F = L.interaction_force(psi, -1.0)
    assert np.max(np.abs(F.reshape(3, -1).sum(1))) < 1e-13


def test_force_is_minus_G_psi_grad_psi_for_long_waves():
    # sum_alpha w_alpha e_alpha e_alpha = I for the Eq. 15 weights, so
    # F = -G psi grad(psi) + O(k^2) for a smooth psi.
    n = 64
    k = 2 * np.pi / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(4), np.arange(4), indexing="ij")
    psi = 1.0 + 0.1 * np.sin(k * z)
    G = -1.7
    F = L.interaction_force(psi, G)
    want = -G * psi * 0.1 * k * np.cos(k * z)
    assert np.max(np.abs(F[2] - want)) < 2 * k * k * np.max(np.abs(want))
    assert np.max(np.abs(F[0])) < 1e-15 and np.max(np.abs(F[1])) < 1e-15


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("op", OPS)
def test_mass_and_momentum_conserved(op):
    p = _droplet_params(op=op)
    f = _droplet_state(p)
    m0 = L.total_mass(f)
    P0 = L.total_momentum(p, f)
    f = L.run(p, f, 60)
    assert abs(L.total_mass(f) - m0) < 1e-13 * m0
    assert np.max(np.abs(L.total_momentum(p, f) - P0)) < 1e-13 * m0


@pytest.mark.parametrize("op", OPS)
def test_uniform_state_stays_uniform(op):
    p = _droplet_params(grid=(4, 5, 3), op=op, T_over_Tc=0.9)
    rho = np.full((3, 5, 4), 0.2)
    u = np.zeros((3, 3, 5, 4))
    u[0], u[1], u[2] = 0.01, -0.02, 0.005
    f0 = L.equilibrium_state(p, rho, u)
    f = L.run(p, f0, 10)
    spread = f.reshape(19, -1).max(1) - f.reshape(19, -1).min(1)
    assert np.max(spread) < 1e-15  # still uniform, node by node
    assert np.max(np.abs(f - f0)) < 1e-14  # and still the same equilibrium


@pytest.mark.parametrize("op", OPS)
def test_centred_droplet_keeps_mirror_and_axis_symmetry(op):
    p = _droplet_params(op=op)
    f = L.run(p, _droplet_state(p), 30)
    rho, u, _, _ = L.macroscopic(p, f)
    n = 16
    idx = (-np.arange(n)) % n  # mirror about the centre node n/2
    assert np.max(np.abs(rho - rho[:, :, idx])) < 1e-13
    assert np.max(np.abs(rho - rho[:, idx, :])) < 1e-13
    assert np.max(np.abs(rho - np.transpose(rho, (0, 2, 1)))) < 1e-13
    assert np.max(np.abs(rho - np.transpose(rho, (2, 1, 0)))) < 1e-13
    assert np.max(np.abs(u[0] + u[0][:, :, idx])) < 1e-13


@pytest.mark.parametrize("op", OPS)
def test_sqrt_pseudopotential_is_independent_of_G(op):
    # psi ~ 1/sqrt(|G|) and F ~ G psi psi: the dynamics cannot depend on G.
    p = _droplet_params(op=op)
    f0 = _droplet_state(p)
    a = L.run(p, f0, 15)
    b = L.run(p.with_(G=-2.5), f0, 15)
    assert np.max(np.abs(a - b)) < 1e-13


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("s_nu", [1.0, 1.6])
def test_shear_wave_decays_with_eq54_viscosity(op, s_nu):
    nz, steps = 64, 200
    p = L.Params(grid=(3, 3, nz), operator=op, eos="none", G=0.0, s_nu=s_nu,
                 s_e=0.9, s_q=1.2, s_pi=1.3, s_eps=1.1, s_m=1.4)
    k = 2 * np.pi / nz
    z = np.broadcast_to(np.arange(nz)[:, None, None], (nz, 3, 3))
    u = np.zeros((3, nz, 3, 3))
    u[0] = 1e-3 * np.sin(k * z)
    f = L.equilibrium_state(p, np.ones((nz, 3, 3)), u)

    def amp(f):
        return 2 * np.mean(L.macroscopic(p, f)[1][0] * np.sin(k * z))

    a0 = amp(f)
    ratio = amp(L.run(p, f, steps)) / a0
    nu = (1 / s_nu - 0.5) / 3  # Eq. 54, mu = rho c_s^2 (1/s_nu - 1/2)
    assert abs(ratio / np.exp(-nu * k * k * steps) - 1) < 0.003


@pytest.mark.parametrize("op", OPS)
def test_sound_wave_speed_and_bulk_viscosity_eq54(op):
    nz, steps, s_e, s_nu = 64, 400, 0.8, 1.2
    p = L.Params(grid=(3, 3, nz), operator=op, eos="none", G=0.0, s_nu=s_nu, s_e=s_e,
                 s_q=1.2, s_pi=1.3, s_eps=1.1, s_m=1.4)
    k = 2 * np.pi / nz
    z = np.broadcast_to(np.arange(nz)[:, None, None], (nz, 3, 3))
    f = L.equilibrium_state(p, 1 + 1e-4 * np.cos(k * z))
    a = []
    for _ in range(steps):
        a.append(2 * np.mean((L.density(f) - 1) * np.cos(k * z)))
        f = L.step(p, f)
    t = np.arange(steps)
    popt, _ = curve_fit(lambda t, A, g, w, ph: A * np.exp(-g * t) * np.cos(w * t + ph),
                        t, np.array(a), p0=[1e-4, 1e-3, k / np.sqrt(3), 0.0])
    nu = (1 / s_nu - 0.5) / 3
    nu_b = 2.0 / 9.0 * (1 / s_e - 0.5)  # Eq. 54, mu_b = (2/3) rho c_s^2 (1/s_e - 1/2)
    assert abs(popt[1] / (k * k / 2 * (4 * nu / 3 + nu_b)) - 1) < 0.01
    assert abs(popt[2] / (k / np.sqrt(3)) - 1) < 0.002


# ---------------------------------------------------------------- brute force
def _brute_force_step(p, f):
    """One step with per-node loops and push streaming (tiny grids only)."""
    nx, ny, nz = p.grid
    M = L.matrix(p)
    Minv = L.inverse(M)
    lam = L.relaxation(p)
    e = [tuple(int(c) for c in r) for r in L.E]
    wF = [0.0] + [1 / 6] * 6 + [1 / 12] * 12
    rho = np.zeros((nz, ny, nx))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                rho[z, y, x] = sum(f[a, z, y, x] for a in range(19))
    psi = L.pseudopotential(rho, p)
    out = np.zeros_like(f)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                F = [0.0, 0.0, 0.0]
                for a in range(1, 19):
                    nb = psi[(z + e[a][2]) % nz, (y + e[a][1]) % ny, (x + e[a][0]) % nx]
                    for d in range(3):
                        F[d] += wF[a] * nb * e[a][d]
                F = [-p.G * psi[z, y, x] * c for c in F]
                r = rho[z, y, x]
                u = [(sum(e[a][d] * f[a, z, y, x] for a in range(19)) + 0.5 * F[d]) / r for d in range(3)]
                m = [sum(M[k, a] * f[a, z, y, x] for a in range(19)) for k in range(19)]
                uu, FF = np.array(u)[:, None], np.array(F)[:, None]
                if p.operator == "nonorth":
                    meq = L.meq_nonorth(np.array([r]), uu)[:, 0]
                    S = L.forcing_nonorth(FF, uu)[:, 0]
                else:
                    meq = L.meq_orth(np.array([r]), uu)[:, 0]
                    S = L.forcing_orth(FF, uu)[:, 0]
                ms = [m[k] - lam[k] * (m[k] - meq[k]) + (1 - lam[k] / 2) * S[k] for k in range(19)]
                for a in range(19):
                    val = sum(Minv[a, k] * ms[k] for k in range(19))
                    out[a, (z + e[a][2]) % nz, (y + e[a][1]) % ny, (x + e[a][0]) % nx] = val
    return out


@pytest.mark.parametrize("op", OPS)
def test_vectorised_step_matches_brute_force_loops(op):
    p = L.Params(grid=(3, 4, 5), operator=op, T=0.8 * L.critical_temperature(1, 4, 1))
    rho = RNG.uniform(0.05, 0.3, (5, 4, 3))
    u = RNG.uniform(-0.02, 0.02, (3, 5, 4, 3))
    f = L.equilibrium_state(p, rho, u) + RNG.normal(0, 1e-4, (19, 5, 4, 3))
    assert np.max(np.abs(L.step(p, f) - _brute_force_step(p, f))) < 1e-15


# ---------------------------------------------------------------- variable viscosity
@pytest.mark.parametrize("op", OPS)
def test_variable_viscosity_reduces_to_constant_when_equal(op):
    p = _droplet_params(op=op)
    f0 = _droplet_state(p)
    nu = (1 / p.s_nu - 0.5) / 3
    q = p.with_(nu_l=nu, nu_v=nu, rho_l_nu=0.3, rho_v_nu=0.02)
    assert np.max(np.abs(L.run(p, f0, 10) - L.run(q, f0, 10))) < 1e-15


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("phase", ["liquid", "vapour"])
def test_variable_viscosity_shear_wave_takes_the_phase_viscosity(op, phase):
    """A uniform fluid at rho_L (rho_V) decays with nu_L (nu_V): Eq. 54 with s_nu(rho)."""
    nz, steps = 64, 200
    rho_l, rho_v, nu_l, nu_v = 1.2, 0.8, 0.05, 0.2
    rho0 = rho_l if phase == "liquid" else rho_v
    p = L.Params(grid=(3, 3, nz), operator=op, eos="none", G=0.0, s_nu=1.0, s_e=0.9, s_q=1.2, s_pi=1.3,
                 s_eps=1.1, s_m=1.4, nu_l=nu_l, nu_v=nu_v, rho_l_nu=rho_l, rho_v_nu=rho_v)
    k = 2 * np.pi / nz
    z = np.broadcast_to(np.arange(nz)[:, None, None], (nz, 3, 3))
    u = np.zeros((3, nz, 3, 3))
    u[0] = 1e-4 * np.sin(k * z)
    f = L.equilibrium_state(p, np.full((nz, 3, 3), rho0), u)

    def amp(f):
        return 2 * np.mean(L.macroscopic(p, f)[1][0] * np.sin(k * z))

    ratio = amp(L.run(p, f, steps)) / amp(f)
    nu = nu_l if phase == "liquid" else nu_v
    assert abs(ratio / np.exp(-nu * k * k * steps) - 1) < 0.003
    assert np.allclose(L.shear_rate_field(p, np.array([2.0, 0.1])), [1 / (3 * nu_l + 0.5), 1 / (3 * nu_v + 0.5)])


# ---------------------------------------------------------------- initial fields
def test_droplet_profile_is_eq59_with_periodic_minimum_image():
    grid, c, R, W, rl, rv = (20, 16, 12), (10.0, 8.0, 6.0), 4.0, 2.0, 0.3, 0.02
    rho = L.droplet_density(grid, c, R, W, rl, rv)
    assert rho.shape == (12, 16, 20)
    # at the centre tanh(-2R/W); at distance R (node (14, 8, 6)) the mean of the phases
    assert abs(rho[6, 8, 10] - (0.5 * (rl + rv) + 0.5 * (rl - rv) * np.tanh(4.0))) < 1e-15
    assert abs(rho[6, 8, 14] - 0.5 * (rl + rv)) < 1e-15
    # the minimum image: x = 0 lies 10 from the centre either way, x = 19 lies 9 (through the boundary)
    d9 = 0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(2.0 * (9.0 - R) / W)
    assert abs(rho[6, 8, 19] - d9) < 1e-15 and abs(rho[6, 8, 1] - d9) < 1e-15
    # a centre off the grid by one period gives the same field
    assert np.max(np.abs(L.droplet_density(grid, (30.0, -8.0, 18.0), R, W, rl, rv) - rho)) < 1e-14


def test_slab_profile_between_its_planes():
    grid, lo, hi, W, rl, rv = (3, 2, 64), 16.0, 48.0, 2.0, 0.3, 0.02
    rho = L.slab_density(grid, 2, lo, hi, W, rl, rv)
    half = 0.5 * (rl - rv)
    assert abs(rho[32, 0, 0] - (rv + half * 2 * np.tanh(16.0))) < 1e-15  # mid-slab: liquid
    assert abs(rho[16, 1, 2] - (rv + half * (0.0 - np.tanh(-32.0)))) < 1e-15  # on the plane lo: the mean
    assert abs(rho[0, 0, 0] - (rv + half * (np.tanh(-16.0) - np.tanh(-48.0)))) < 1e-15  # vapour
    assert np.all(rho == rho[:, :1, :1])  # depends on z only
    assert np.allclose(L.slab_density((64, 2, 3), 0, lo, hi, W, rl, rv)[0, 0, :], rho[:, 0, 0], rtol=0, atol=0)
