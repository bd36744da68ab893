"""Pins of the oracle's learned warm start: the 16 per-point features
(orc_mlp_features) and the initial guess du_prev + V MLP(x)
(orc_learned_init), on cases worked by hand, and the oracle simulation's
learned mode against the modes it reduces to.

Hand-worked values use the two facts of the weighting function that hold for
both kernels (Sec. 3): the taps of one axis sum to 1 and their squares to
3/8.  Densities are counted on the 4x4x4 bricks of the lattice."""
import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W

V, L = 0.05, 16.0
SHAPE = (16, 16, 16)  # (nz, ny, nx)


def _zero_U():
    return np.zeros((3,) + SHAPE)


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
def test_single_point_at_known_radius_and_height(orc, kernel):
    """Fluid at rest, no previous force: u_i = 0, the slip is u_k; the point
    sits at radius 5 (3-4-5 triangle) and 2 cells below its body's centre."""
    c = np.array([[6.25, 5.5, 9.0]])
    x = c + np.array([[3.0, 4.0, -2.0]])
    ut = np.array([[0.01, -0.02, 0.0]])
    om = np.array([-0.004])
    F = orc.mlp_features(_zero_U(), x, ut, None, body=[0], centre=c, omega=om, kernel=kernel)
    ref = np.zeros(16)
    ref[3:6] = ut[0] / V
    ref[10] = 5.0 / L
    ref[11] = -2.0 / L
    ref[12] = 0.004 * 5.0 / V
    ref[13:16] = ut[0] / V
    # x = (9.25, 9.5, 7.0): taps 8..11, 8..11, 6..9 -> bricks x 2, y 2, z 1-2;
    # one support per brick
    ref[9] = 1.0 / 64.0
    assert np.abs(F[0] - ref).max() < 1e-15


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
def test_uniform_flow_and_previous_force_of_an_isolated_point(orc, kernel):
    """U0 uniform: I[U0] = U0 exactly (partition of unity).  With du_prev
    spread first, a single point sees its own correction through
    I[S[e]] = (3/8)^3 e at any position."""
    U0 = np.empty((3,) + SHAPE)
    u0 = np.array([0.02, -0.01, 0.005])
    U0[:] = u0[:, None, None, None]
    x = np.array([[7.3, 2.9, 11.61]])
    ut = np.array([[0.0, 0.03, 0.0]])
    dp = np.array([[0.4, -0.2, 0.1]])
    F = orc.mlp_features(U0, x, ut, dp, kernel=kernel)
    ui = u0 + (3.0 / 8.0) ** 3 * dp[0]
    assert np.allclose(F[0, 0:3], ui / V, rtol=0, atol=1e-14)
    assert np.allclose(F[0, 6:9], dp[0] / V, rtol=0, atol=1e-14)
    assert np.allclose(F[0, 13:16], (ut[0] - ui) / V, rtol=0, atol=1e-14)
    # no bodies: no radius, height or rotation speed
    assert np.all(F[0, 10:13] == 0.0)


def test_density_counts_supports_per_brick(orc):
    """A at (5.3, 5.3, 5.3): taps 4..7 on every axis, one brick (1,1,1).
    B at (7.5, 5.3, 5.3): taps 6..9 in x, bricks (1,1,1) and (2,1,1).
    C far away at (13.2, 13.2, 1.2): taps 12..15, 12..15, 0..3, one brick.
    Brick (1,1,1) holds two supports, the others one."""
    x = np.array([[5.3, 5.3, 5.3], [7.5, 5.3, 5.3], [13.2, 13.2, 1.2]])
    F = orc.mlp_features(_zero_U(), x, np.zeros((3, 3)))
    assert F[0, 9] == 2.0 / 64.0
    assert F[1, 9] == (2.0 + 1.0) / (2 * 64.0)
    assert F[2, 9] == 1.0 / 64.0


def test_density_across_the_periodic_seam(orc):
    """x = 0.2 has taps -1..2 in x, i.e. cells 15 and 0..2 (bricks 3 and 0);
    a second point at (14.5, 0.2, 0.2) has taps 13..16 -> cells 13..15, 0
    (bricks 3 and 0 again) and shares both bricks of the first in x; on y and
    z both points have taps -1..2 (bricks 3 and 0).  Each of the 8 bricks of
    either support holds both supports."""
    x = np.array([[0.2, 0.2, 0.2], [14.5, 0.2, 0.2]])
    F = orc.mlp_features(_zero_U(), x, np.zeros((2, 3)))
    assert F[0, 9] == 2.0 / 64.0 and F[1, 9] == 2.0 / 64.0
    # shifted by one brick in x the second point no longer meets the first
    x[1, 0] = 10.5  # taps 9..12: bricks 2 and 3, of which brick 3 is shared
    F = orc.mlp_features(_zero_U(), x, np.zeros((2, 3)))
    # first point: bricks x in {3, 0}, y, z in {3, 0}; shared: x = 3 (4 bricks)
    assert F[0, 9] == (4 * 2 + 4 * 1) / (8 * 64.0)
    assert F[1, 9] == (4 * 1 + 4 * 2) / (8 * 64.0)


def test_features_follow_the_rotation(orc):
    """Radius and height of every point of a rotating propeller stay those of
    its rest pose (rigid rotation about z), and the rotation speed is
    |omega| r, which is |u_k| up to the chord-to-arc factor
    2 sin(omega/2) / omega."""
    w = W.single_propeller()
    p = w.props
    for t in (0, 13):
        x, ut = orc.kinematics(p.xrest, p.body, p.centre, p.omega, p.phase, t)
        F = orc.mlp_features(np.zeros((3,) + w.shape), x, ut, body=p.body, centre=p.centre,
                             omega=p.omega)
        d = p.xrest - p.centre[p.body]
        assert np.allclose(F[:, 10] * L, np.hypot(d[:, 0], d[:, 1]), rtol=0, atol=1e-12)
        assert np.allclose(F[:, 11] * L, d[:, 2], rtol=0, atol=1e-12)
        om = np.abs(p.omega[p.body])
        chord = np.linalg.norm(ut, axis=1)
        # (u_k is a difference of positions near 16: ~1e-12 relative cancellation)
        assert np.allclose(F[:, 12] * V * 2 * np.sin(om / 2) / om, chord, rtol=1e-10, atol=0)


def test_learned_init_of_a_bias_only_network(orc):
    """All weights zero, output bias b3: MLP(x) = b3 for any x, so the
    initial guess is du_prev + V b3 (and V b3 without a previous force)."""
    P = np.zeros(orc.mlp_nparam())
    b3 = np.array([0.3, -0.7, 1.1])
    P[-3:] = b3
    rng = W.SplitMix64(301)
    feat = W.random_array(rng, (5, 16))
    dp = W.random_array(rng, (5, 3))
    assert np.array_equal(orc.learned_init(P, feat, dp), dp + V * b3)
    assert np.array_equal(orc.learned_init(P, feat, None), np.tile(V * b3, (5, 1)))


def test_learned_init_uses_the_network_output(orc):
    """One hidden path (W1[0,3] = a, W2[0,0] = b, W3[1,0] = 1): the initial
    guess moves only along y and by V s(b s(a x_3)) with the SiLU s."""
    P = np.zeros(orc.mlp_nparam())
    a, b = 0.9, 1.7
    P[3] = a
    P[1024 + 64] = b
    P[1024 + 64 + 4096 + 64 + 64] = 1.0  # W3[1][0]
    feat = np.zeros((2, 16))
    feat[:, 3] = [0.4, -1.2]  # u_k,x / V
    s = lambda v: v / (1.0 + np.exp(-v))
    du = orc.learned_init(P, feat, np.ones((2, 3)))
    assert np.allclose(du[:, 1], 1.0 + V * s(b * s(a * feat[:, 3])), rtol=0, atol=1e-15)
    assert np.all(du[:, 0] == 1.0) and np.all(du[:, 2] == 1.0)


def test_simulation_learned_mode_reduces_to_the_previous_force_start(orc):
    """With a network that outputs zero the learned start is exactly the
    previous-force start; with a constant output c it is shifted by V c at
    every step, which the oracle's recorded initial guess shows."""
    w = W.single_propeller(3)
    pts = w.props.as_dict()
    P = np.zeros(orc.mlp_nparam())
    a = orc.Simulation(w.shape, w.tau, pts, warm="previous").step(3)
    b = orc.Simulation(w.shape, w.tau, pts, warm="mlp", mlp=P).step(3)
    assert np.array_equal(a.f, b.f) and np.array_equal(a.du, b.du)
    assert b.features.shape == (w.props.n_points, 16)
    P[-3:] = [0.01, -0.02, 0.0]
    c = orc.Simulation(w.shape, w.tau, pts, warm="mlp", mlp=P).step(2)
    du1 = c.du.copy()
    c.step(1)
    assert np.allclose(c.du_init, du1 + V * P[-3:], rtol=0, atol=1e-15)
    # the features of that step: du_prev is the previous final du
    assert np.allclose(c.features[:, 6:9], du1 / V, rtol=0, atol=1e-15)


def test_simulation_learned_mode_first_step_features(orc):
    """At the first step (fluid at rest, no previous force) u_i = 0, so the
    slip features equal the surface-velocity features."""
    w = W.single_propeller(4)
    P = np.zeros(orc.mlp_nparam())
    s = orc.Simulation(w.shape, w.tau, w.props.as_dict(), warm="mlp", mlp=P).step(1)
    F = s.features
    assert np.abs(F[:, 0:3]).max() < 1e-15
    assert np.array_equal(F[:, 13:16], F[:, 3:6])
    assert np.all(F[:, 6:9] == 0.0)
    assert np.all(F[:, 9] >= 1.0 / 64.0)
