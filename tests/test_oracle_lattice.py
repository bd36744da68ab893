"""Pins of the oracle's lattice Boltzmann part (Sec. 2, Eqs. 1-4) against
closed forms and conservation laws.  CPU only."""
import math

import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W


def test_velocity_set_is_d3q19(orc):
    e, t = orc.velocity_set()
    assert len({tuple(v) for v in e}) == 19
    n2 = (e * e).sum(1)
    assert sorted(n2.tolist()) == [0] + [1] * 6 + [2] * 12
    # weights by speed class (1/3, 1/18, 1/36)
    for v, w in zip(n2, t):
        assert w == {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[int(v)]
    # every vector has its opposite
    assert all(tuple(-v) in {tuple(u) for u in e} for v in e)


def test_lattice_isotropy(orc):
    """sum t = 1, sum t e = 0, sum t e_a e_b = delta/3,
    sum t e_a e_b e_c e_d = (dd + dd + dd)/9: the moments a D3Q19 set must
    have for Eq. 3 to recover Navier-Stokes."""
    e, t = orc.velocity_set()
    e = e.astype(float)
    assert abs(t.sum() - 1) < 1e-15
    assert np.abs(t @ e).max() < 1e-15
    d = np.eye(3)
    assert np.abs(np.einsum("i,ia,ib->ab", t, e, e) - d / 3).max() < 1e-15
    m4 = np.einsum("i,ia,ib,ic,id->abcd", t, e, e, e, e)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.abs(m4 - iso).max() < 1e-15


@pytest.mark.parametrize("rho,U", [(1.0, (0, 0, 0)), (1.03, (0.02, -0.05, 0.01)),
                                   (0.97, (0.1, 0.0, -0.07))])
def test_equilibrium_moments(orc, rho, U):
    """Eq. 3 (with rho): zeroth, first and second moments are rho, rho U and
    rho (delta/3 + U U) exactly."""
    e, _ = orc.velocity_set()
    U = np.asarray(U, float)
    feq = np.array([orc.equilibrium(i, rho, U) for i in range(19)])
    assert abs(feq.sum() - rho) < 1e-14
    assert np.abs(e.T @ feq - rho * U).max() < 1e-14
    P = np.einsum("i,ia,ib->ab", feq, e, e)
    assert np.abs(P - rho * (np.eye(3) / 3 + np.outer(U, U))).max() < 1e-14


def test_moments_recover_equilibrium_state(orc):
    rng = W.SplitMix64(11)
    shape = (3, 4, 5)
    rho = 1 + 0.05 * W.random_array(rng, shape)
    U = 0.05 * W.random_array(rng, (3,) + shape)
    f = orc.init_equilibrium(shape, rho, U)
    r2, U2 = orc.moments(f)
    assert np.abs(r2 - rho).max() < 1e-14
    assert np.abs(U2 - U).max() < 1e-14


def test_stream_moves_each_population_along_its_vector(orc):
    """Eq. 4 with periodic wrap: a single marked population at X ends at
    X + e_i (mod n)."""
    e, _ = orc.velocity_set()
    shape = (3, 4, 5)
    nz, ny, nx = shape
    for i in range(19):
        f = np.zeros((19,) + shape)
        f[i, 0, 3, 4] = 1.0
        g = orc.stream(f)
        z, y, x = (0 + e[i, 2]) % nz, (3 + e[i, 1]) % ny, (4 + e[i, 0]) % nx
        assert g[i, z, y, x] == 1.0 and g.sum() == 1.0


def test_collide_tau_one_gives_equilibrium(orc):
    """Eq. 2 with tau = 1 replaces f by Eq(rho, U + G)."""
    rng = W.SplitMix64(12)
    shape = (2, 3, 4)
    f = orc.init_equilibrium(shape) + 1e-3 * W.random_array(rng, (19,) + shape)
    rho, U = orc.moments(f)
    G = 1e-3 * W.random_array(rng, (3,) + shape)
    g = orc.collide(f, 1.0, rho, U, G)
    ref = orc.init_equilibrium(shape, rho, U + G)
    assert np.abs(g - ref).max() < 1e-15


def test_rest_state_is_invariant(orc):
    sim = orc.Simulation((6, 5, 4), 0.8)
    f0 = sim.f.copy()
    sim.step(10)
    # full populations in FP64: invariant up to the rounding of sum t_i
    assert np.abs(sim.f - f0).max() < 1e-16


def _perturbed(orc, shape, seed):
    rng = W.SplitMix64(seed)
    rho = 1 + 0.02 * W.random_array(rng, shape)
    U = 0.03 * W.random_array(rng, (3,) + shape)
    return orc.init_equilibrium(shape, rho, U) + 1e-4 * W.random_array(rng, (19,) + shape)


def test_mass_conserved_over_100_steps(orc):
    shape = (8, 8, 8)
    sim = orc.Simulation(shape, 0.7)
    sim.f = _perturbed(orc, shape, 13)
    m0 = sim.sums()[0]
    sim.step(100)
    assert abs(sim.sums()[0] - m0) / m0 < 1e-13


def test_momentum_increment_is_rho_G(orc):
    """Velocity-shift forcing (Sec. 2, step 3): the collision adds
    sum rho G to the total momentum; streaming preserves it."""
    shape = (6, 6, 6)
    rng = W.SplitMix64(14)
    f = _perturbed(orc, shape, 15)
    rho, U = orc.moments(f)
    G = 1e-3 * W.random_array(rng, (3,) + shape)
    p0 = orc.sums(f)[1:]
    g = orc.stream(orc.collide(f, 0.9, rho, U, G))
    p1 = orc.sums(g)[1:]
    expect = (rho[None] * G).reshape(3, -1).sum(1)
    assert np.abs((p1 - p0) - expect).max() < 1e-13


def test_uniform_force_accelerates_uniformly(orc):
    """A uniform G in a periodic box at rest: U(t) = t G exactly (each
    collision adds G to the velocity and the state stays uniform)."""
    G = np.array([1e-4, -2e-4, 5e-5])
    sim = orc.Simulation((4, 4, 4), 0.8, gbody=G)
    for t in range(1, 21):
        sim.step()
        rho, U = sim.fields()
        assert np.abs(rho - 1).max() < 1e-14
        assert np.abs(U - t * G[:, None, None, None]).max() < 1e-15 * t + 1e-16


def test_galilean_uniform_flow_stays_uniform(orc):
    shape = (4, 5, 6)
    U = np.zeros((3,) + shape)
    U[0], U[1], U[2] = 0.03, -0.02, 0.01
    sim = orc.Simulation(shape, 0.7)
    sim.f = orc.init_equilibrium(shape, None, U)
    sim.step(20)
    rho, U2 = sim.fields()
    assert np.abs(U2 - U).max() < 1e-15
    assert np.abs(rho - 1).max() < 1e-14


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_shear_wave_decays_at_lattice_viscosity(orc, tau):
    """u_x = A sin(2 pi y / n) decays as exp(-nu k^2 t), nu = (tau - 1/2)/3
    (BGK viscosity of Eq. 2); rate within 0.5% at n = 32, measured between
    t = 100 and t = 300 (after the start-up transient of an equilibrium
    initial state)."""
    n, A = 32, 1e-3
    y = np.arange(n)
    shape = (2, n, 2)
    U = np.zeros((3,) + shape)
    U[0] = (A * np.sin(2 * np.pi * y / n))[None, :, None]
    sim = orc.Simulation(shape, tau)
    sim.f = orc.init_equilibrium(shape, None, U)
    s = np.sin(2 * np.pi * y / n)

    def amp():
        _, U1 = sim.fields()
        return (U1[0, 0, :, 0] * s).sum() / (s * s).sum()

    sim.step(100)
    a1 = amp()
    sim.step(200)
    a2 = amp()
    rate = -math.log(a2 / a1) / 200
    nu = (tau - 0.5) / 3
    assert abs(rate / (nu * (2 * np.pi / n) ** 2) - 1) < 0.005
