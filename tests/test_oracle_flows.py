"""End-to-end pins of the oracle's coupled LBM + IBM step (Sec. 2-3) on flows
with closed forms, and of the rigid-body kinematics of Alg. 1.  CPU only."""
import math

import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W


def _planes(nx, nz, m, y_and_u):
    """Two periodic sheets of m x m points at the given y, moving along x."""
    sp = nx / m
    xs, ut = [], []
    for yw, u in y_and_u:
        for i in range(m):
            for k in range(m):
                xs.append((sp * i + 0.3, yw, sp * k + 0.1))
                ut.append((u, 0.0, 0.0))
    xs, ut = np.array(xs), np.array(ut)
    return dict(x=xs, ut=ut, area=np.full(len(xs), sp * sp))


def test_couette_between_immersed_planes(orc):
    """Planes at y = 8 and y = 24 moving at -U_w and +U_w in a periodic box:
    the steady profile between them is linear (R^2 > 1 - 1e-9 on cells more
    than 2 from the planes), odd about the mid-plane, and the corrected field
    interpolated on the planes meets the wall speed.  The slope exceeds the
    sharp-wall value 2 U_w / 16 by the diffuse-interface thickening (less
    than 1.5 cells in total)."""
    ny, n, tau, Uw = 32, 4, 1.0, 0.01
    P = _planes(n, n, 6, ((8.0, -Uw), (24.0, Uw)))
    sim = orc.Simulation((n, ny, n), tau, P)
    sim.step(3000)
    rho, U = sim.fields()
    prof = U[0].mean(axis=(0, 2))
    assert np.abs(U[0] - prof[None, :, None]).max() < 1e-12  # x-z invariant
    y = np.arange(ny)
    sel = (y >= 11) & (y <= 21)
    c = np.polyfit(y[sel], prof[sel], 1)
    fit = np.polyval(c, y[sel])
    r2 = 1 - ((prof[sel] - fit) ** 2).sum() / ((prof[sel] - prof[sel].mean()) ** 2).sum()
    assert r2 > 1 - 1e-9
    assert abs(np.polyval(c, 16.0)) < 1e-9  # zero on the mid-plane
    assert np.abs(prof[16 + 1:24] + prof[16 - 1:8:-1]).max() < 1e-9  # odd
    slope = c[0]
    assert 2 * Uw / 16 < slope < 2 * Uw / (16 - 1.5)
    # no-slip reached by the fixed point (5 iterations, residual shrinking)
    eps_pt = sim.eps_pt[-1]
    assert np.all(np.diff(eps_pt) < 0) and eps_pt[-1] < 5e-3


def test_poiseuille_between_static_planes(orc):
    """Static planes at y = 8, 24 and a uniform body force g along x: in the
    bulk between them the steady profile is a parabola with curvature
    u'' = -g / nu, nu = (tau - 1/2)/3, and symmetric about the mid-plane."""
    ny, n, tau, g = 32, 4, 1.0, 1e-6
    P = _planes(n, n, 6, ((8.0, 0.0), (24.0, 0.0)))
    sim = orc.Simulation((n, ny, n), tau, P, gbody=(g, 0.0, 0.0))
    sim.step(4000)
    _, U = sim.fields()
    prof = U[0].mean(axis=(0, 2))
    nu = (tau - 0.5) / 3
    y = np.arange(ny)
    sel = (y >= 11) & (y <= 21)
    c = np.polyfit(y[sel], prof[sel], 2)
    assert abs(c[0] / (-g / (2 * nu)) - 1) < 1e-6
    assert abs(-c[1] / (2 * c[0]) - 16.0) < 1e-6  # vertex on the mid-plane
    resid = prof[sel] - np.polyval(c, y[sel])
    assert np.abs(resid).max() < 1e-3 * prof.max()


def _exact_sums(orc, f):
    """Mass and momentum of the populations, correctly rounded (fsum)."""
    e, _ = orc.velocity_set()
    m = math.fsum(f.ravel())
    p = [math.fsum((e[:, c, None, None, None] * f).ravel()) for c in range(3)]
    return np.array([m] + p)


def test_sums_match_correctly_rounded_sums(orc):
    """orc_sums adds in plain order: within n * 2^-53 * sum|f| of fsum."""
    w = W.single_propeller()
    sim = orc.Simulation(w.shape, w.tau, w.props.as_dict(), n_iter=5)
    sim.step(2)
    bound = sim.f.size * 2.0 ** -53 * np.abs(sim.f).sum()
    assert np.abs(sim.sums() - _exact_sums(orc, sim.f)).max() < bound


def test_propeller_step_conserves_mass_and_adds_rho_G(orc):
    """The coupled step with moving points: mass is conserved to roundoff;
    the momentum change over one step equals sum rho G with G the IBM force
    of that step (velocity-shift forcing).  One blade only, so that the net
    force is far from zero (a full propeller's cancels by symmetry).  Sums
    are taken correctly rounded so that only the step's own rounding shows."""
    w = W.single_propeller()
    P = w.props.as_dict()
    keep = slice(0, 90)  # blade 0
    P = dict(P, xrest=P["xrest"][keep], area=P["area"][keep], body=P["body"][keep])
    sim = orc.Simulation(w.shape, w.tau, P, n_iter=5)
    m0 = _exact_sums(orc, sim.f)
    for _ in range(4):
        before = _exact_sums(orc, sim.f)
        sim.step()
        after = _exact_sums(orc, sim.f)
        expect = [math.fsum((sim.rho * sim.G[c]).ravel()) for c in range(3)]
        assert np.abs(expect).max() > 1e-2
        assert np.abs((after[1:] - before[1:]) - expect).max() < 1e-12
    assert abs(_exact_sums(orc, sim.f)[0] - m0[0]) / m0[0] < 1e-14


def test_kinematics_rotates_rigidly(orc):
    """Alg. 1: x(t) = M(t) [x_rest, 1] is a rotation about z through each
    centre; distances to the axis and axial coordinates are preserved, the
    surface velocity is the backward difference, of length
    2 r sin(omega / 2), and after one period the points return."""
    w = W.single_propeller()
    p = w.props
    P = 90
    omega = np.array([2 * math.pi / P])
    x0, u0 = orc.kinematics(p.xrest, p.body, p.centre, omega, p.phase, 0)
    rr = np.hypot(*(p.xrest[:, :2] - p.centre[0, :2]).T)
    for t in (0, 1, 17, 45):
        x, ut = orc.kinematics(p.xrest, p.body, p.centre, omega, p.phase, t)
        assert np.abs(np.hypot(*(x[:, :2] - p.centre[0, :2]).T) - rr).max() < 1e-12
        assert np.abs(x[:, 2] - p.xrest[:, 2]).max() < 1e-13
        xp, _ = orc.kinematics(p.xrest, p.body, p.centre, omega, p.phase, t - 1)
        assert np.abs(ut - (x - xp)).max() < 1e-14
        assert np.abs(np.linalg.norm(ut, axis=1) - 2 * rr * math.sin(omega[0] / 2)).max() < 1e-13
        # counter-clockwise: (r x u)_z > 0
        d = x[:, :2] - p.centre[0, :2]
        assert np.all(d[:, 0] * ut[:, 1] - d[:, 1] * ut[:, 0] > 0)
    xP, _ = orc.kinematics(p.xrest, p.body, p.centre, omega, p.phase, P)
    assert np.abs(xP - x0).max() < 1e-12
    # t = 0 with phase phi0 is the rest pose rotated by phi0
    c, s = math.cos(p.phase[0]), math.sin(p.phase[0])
    d = p.xrest - p.centre[0]
    ref = p.centre[0] + np.stack([c * d[:, 0] - s * d[:, 1], s * d[:, 0] + c * d[:, 1], d[:, 2]], 1)
    assert np.abs(x0 - ref).max() < 1e-12


def test_poiseuille_with_conjugate_gradients(orc):
    """The same channel with the fixed point solved by conjugate gradients
    (5 iterations per step): the bulk is the same parabola (curvature -g/nu,
    vertex on the mid-plane), and the steady flow equals the paper loop's to
    within what their different 5-iterate forces leave (the planes' slip)."""
    ny, n, tau, g = 32, 4, 1.0, 1e-6
    P = _planes(n, n, 6, ((8.0, 0.0), (24.0, 0.0)))
    sims = [orc.Simulation((n, ny, n), tau, P, gbody=(g, 0.0, 0.0), solver=s)
            for s in ("cg", "mdf")]
    for sim in sims:
        sim.step(4000)
    prof, prof_m = (sim.fields()[1][0].mean(axis=(0, 2)) for sim in sims)
    nu = (tau - 0.5) / 3
    y = np.arange(ny)
    sel = (y >= 11) & (y <= 21)
    c = np.polyfit(y[sel], prof[sel], 2)
    assert abs(c[0] / (-g / (2 * nu)) - 1) < 1e-6
    assert abs(-c[1] / (2 * c[0]) - 16.0) < 1e-6
    assert np.abs(prof[sel] - np.polyval(c, y[sel])).max() < 1e-3 * prof.max()
    assert np.abs(prof - prof_m).max() < 2e-2 * prof_m.max()
