"""Pins of the oracle's immersed-boundary part (Sec. 3, Alg. 1-2): the
weighting function, interpolation, spreading and the multi-direct-forcing fixed
point, against closed forms, identities and a dense linear solve.  CPU only."""
import math
import os

import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "delta_values.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        kernel, r, expr = line.split()[:3]
        rows.append((kernel, float(r), eval(expr, {"sqrt": math.sqrt})))
    return rows


@pytest.mark.parametrize("kernel,r,value", _golden_rows())
def test_delta_golden_values(orc, kernel, r, value):
    assert abs(orc.delta(r, kernel) - value) < 1e-15
    assert abs(orc.delta(-r, kernel) - value) < 1e-15  # w depends on |r|


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
def test_delta_discrete_moments(orc, kernel):
    """Over the integer lattice, for any x: sum w = 1 (partition of unity),
    sum w^2 = 3/8, even and odd sub-sums 1/2; first moment zero for Peskin
    and bounded (|m1| <= 0.0211) but non-zero for the cosine kernel."""
    rng = W.SplitMix64(21)
    m1max = 0.0
    for _ in range(200):
        x = rng.uniform(-3.0, 3.0)
        X = np.arange(-8, 9)
        w = orc.delta(x - X, kernel)
        assert abs(w.sum() - 1) < 2e-16 * 8
        assert abs((w * w).sum() - 3 / 8) < 1e-15
        assert abs(w[X % 2 == 0].sum() - 0.5) < 1e-15
        m1 = ((X - x) * w).sum()
        m1max = max(m1max, abs(m1))
        if kernel == "peskin":
            assert abs(m1) < 1e-14
    if kernel == "cosine":
        assert 0.015 < m1max <= 0.0211


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
def test_delta_support_and_continuity(orc, kernel):
    r = np.linspace(0, 2.5, 2501)
    w = orc.delta(r, kernel)
    assert np.all(w[r >= 2] == 0) and np.all(w[r < 2] > 0)
    assert np.all(np.diff(w) <= 1e-15)  # decreasing with distance
    assert np.abs(np.diff(w)).max() < 2e-3  # continuous


def _rand_fields(seed, shape, n, margin=0.0):
    rng = W.SplitMix64(seed)
    U = W.random_array(rng, (3,) + shape)
    x = W.random_points(rng, n, shape, margin)
    g = W.random_array(rng, (n, 3))
    return U, x, g


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
def test_interpolation_of_constant_and_linear_fields(orc, kernel):
    shape = (9, 10, 11)
    _, x, _ = _rand_fields(22, shape, 40, margin=3.0)
    U = np.zeros((3,) + shape)
    U[0], U[1], U[2] = 0.3, -0.2, 0.7
    u = orc.interpolate(U, x, kernel)
    assert np.abs(u - [0.3, -0.2, 0.7]).max() < 1e-15
    if kernel == "peskin":
        # zero first moment: linear fields are interpolated exactly (away
        # from the periodic seam)
        Z, Y, X = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
        U[0], U[1], U[2] = X, 2 * Y - 1, Z + X
        u = orc.interpolate(U, x, kernel)
        ref = np.stack([x[:, 0], 2 * x[:, 1] - 1, x[:, 2] + x[:, 0]], 1)
        assert np.abs(u - ref).max() < 1e-13


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
def test_interpolation_spreading_adjoint(orc, kernel):
    """<I[U], g> = <U, S[g]>: interpolation and spreading use the same
    weights (Sec. 3), so they are adjoint; includes points across the
    periodic seam."""
    shape = (7, 8, 9)
    U, x, g = _rand_fields(23, shape, 64)
    lhs = (orc.interpolate(U, x, kernel) * g).sum()
    rhs = (U * orc.spread(shape, x, g, kernel)).sum()
    assert abs(lhs - rhs) < 1e-13 * max(1, abs(lhs))


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
def test_self_interaction_is_three_eighths_cubed(orc, kernel):
    """I[S[e]](k) for a single point = (sum_X w^2)^3 = (3/8)^3 at any
    position (separable weights, sum w^2 = 3/8)."""
    shape = (8, 8, 8)
    rng = W.SplitMix64(24)
    for _ in range(10):
        x = W.random_points(rng, 1, shape)
        F = orc.spread(shape, x, np.array([[1.0, 0.0, 0.0]]), kernel)
        u = orc.interpolate(F, x, kernel)
        assert abs(u[0, 0] - 0.052734375) < 1e-15
        assert abs(u[0, 1]) == 0 and abs(u[0, 2]) == 0


def test_spread_conserves_total_and_is_translation_invariant(orc):
    shape = (6, 7, 8)
    _, x, g = _rand_fields(25, shape, 30)
    F = orc.spread(shape, x, g)
    assert np.abs(F.reshape(3, -1).sum(1) - g.sum(0)).max() < 1e-13
    # integer shift of all points = periodic roll of the field
    F2 = orc.spread(shape, x + [3, -2, 5], g)
    assert np.abs(F2 - np.roll(F, (5, -2, 3), axis=(1, 2, 3))).max() < 1e-14


def _dense_A(orc, shape, x, kernel="cosine"):
    """A = I S as a (3n x 3n) matrix, built column by column."""
    n = len(x)
    A = np.zeros((3 * n, 3 * n))
    for j in range(3 * n):
        v = np.zeros((n, 3))
        v.reshape(-1)[j] = 1.0
        A[:, j] = orc.interpolate(orc.spread(shape, x, v, kernel), x, kernel).reshape(-1)
    return A


def _sheet(shape, spacing, y0=3.3):
    nz, ny, nx = shape
    pts = []
    for k in range(int(nz / spacing)):
        for i in range(int(nx / spacing)):
            pts.append((0.21 + spacing * i, y0, 0.37 + spacing * k))
    return np.array(pts)


def test_fixed_point_is_the_damped_richardson_iteration(orc):
    """With uniform s, the Sec. 3 loop is du_N = s sum_{n<N} (1 - sA)^n r0,
    r0 = u_t - I[U0] (first estimate includes g_0), and G = S[du]."""
    shape = (6, 8, 6)
    x = _sheet(shape, 0.7)
    n = len(x)
    rng = W.SplitMix64(26)
    U0 = 0.01 * W.random_array(rng, (3,) + shape)
    ut = 0.02 * W.random_array(rng, (n, 3))
    s = 0.49
    A = _dense_A(orc, shape, x)
    r0 = (ut - orc.interpolate(U0, x)).reshape(-1)
    for N in (1, 2, 5, 12):
        G, du, eps, _ = orc.ibm(U0, x, ut, np.full(n, s), n_iter=N)
        ref = np.zeros(3 * n)
        r = r0.copy()
        for _ in range(N):
            ref += s * r
            r = r - s * (A @ r)
        assert np.abs(du.reshape(-1) - ref).max() < 1e-14
        assert np.abs(G - orc.spread(shape, x, du)).max() < 1e-15
        assert len(eps) == N


def test_fixed_point_residual_is_monotone_and_converges_to_linear_solve(orc):
    """A = I S is a Gram matrix (S is the adjoint of I), so its eigenvalues
    are >= 0; for a sheet at spacing 0.7 it is singular (more points than the
    kernel resolves), at spacing 2 it is well conditioned (eigenvalues of a
    single separable kernel sum: in [0.036, 0.094]).  With s lambda in (0, 2)
    the Eulerian and pointwise residuals never increase, and the iterate
    reaches du = A^-1 r0."""
    shape = (6, 8, 6)
    lam07 = np.linalg.eigvalsh(_dense_A(orc, shape, _sheet(shape, 0.7)))
    assert lam07.min() > -1e-14 and lam07.min() < 1e-12 and lam07.max() < 1
    x = _sheet(shape, 2.0)
    n = len(x)
    rng = W.SplitMix64(27)
    U0 = 0.01 * W.random_array(rng, (3,) + shape)
    ut = 0.02 * W.random_array(rng, (n, 3))
    s = 10.0
    A = _dense_A(orc, shape, x)
    lam = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert 0.03 < lam.min() and lam.max() < 0.1
    G, du, eps, eps_pt = orc.ibm(U0, x, ut, np.full(n, s), n_iter=0, tol=1e-13,
                                 max_iter=4000)
    assert len(eps) < 4000
    assert np.all(np.diff(eps) <= 1e-15) and np.all(np.diff(eps_pt) <= 1e-15)
    r0 = (ut - orc.interpolate(U0, x)).reshape(-1)
    ref = np.linalg.solve(A, r0)
    assert np.abs(du.reshape(-1) - ref).max() < 1e-10 * np.abs(ref).max()
    # the converged corrected field meets the surface velocity
    assert np.abs(orc.interpolate(U0 + G, x) - ut).max() < 1e-12


def test_tolerance_mode_stops_at_first_iterate_below_tol(orc):
    shape = (6, 8, 6)
    x = _sheet(shape, 0.7)
    n = len(x)
    rng = W.SplitMix64(28)
    U0 = 0.01 * W.random_array(rng, (3,) + shape)
    ut = 0.02 * W.random_array(rng, (n, 3))
    _, _, eps_fixed, _ = orc.ibm(U0, x, ut, np.full(n, 0.49), n_iter=60)
    tol = 0.3
    assert eps_fixed[0] > tol > eps_fixed[-1]
    _, _, eps, _ = orc.ibm(U0, x, ut, np.full(n, 0.49), n_iter=0, tol=tol, max_iter=60)
    k = int(np.argmax(eps_fixed <= tol))
    assert len(eps) == k + 1 and np.allclose(eps, eps_fixed[:k + 1], rtol=0, atol=0)
    _, _, eps_cap, _ = orc.ibm(U0, x, ut, np.full(n, 0.49), n_iter=0, tol=1e-30, max_iter=7)
    assert len(eps_cap) == 7


def test_literal_and_consistent_forms_agree_when_s_is_one(orc):
    shape = (6, 8, 6)
    x = _sheet(shape, 0.7)
    n = len(x)
    rng = W.SplitMix64(29)
    U0 = 0.01 * W.random_array(rng, (3,) + shape)
    ut = 0.02 * W.random_array(rng, (n, 3))
    a = orc.ibm(U0, x, ut, np.ones(n), n_iter=5)
    b = orc.ibm(U0, x, ut, np.ones(n), n_iter=5, literal=True)
    assert np.abs(a[1] - b[1]).max() < 1e-16
    c = orc.ibm(U0, x, ut, np.full(n, 0.5), n_iter=5, literal=True)
    assert np.abs(a[1] - c[1]).max() > 1e-6  # s matters in the literal form


def test_warm_start_shifts_the_initial_field(orc):
    """A warm start du_init enters as U_0 = U0 + S[du_init]; starting from
    the N-iterate continues the same sequence (N + M iterations)."""
    shape = (6, 8, 6)
    x = _sheet(shape, 0.7)
    n = len(x)
    rng = W.SplitMix64(30)
    U0 = 0.01 * W.random_array(rng, (3,) + shape)
    ut = 0.02 * W.random_array(rng, (n, 3))
    s = np.full(n, 0.49)
    _, du3, _, _ = orc.ibm(U0, x, ut, s, n_iter=3)
    _, du5, _, _ = orc.ibm(U0, x, ut, s, n_iter=5)
    _, du32, _, _ = orc.ibm(U0, x, ut, s, n_iter=2, du_init=du3)
    assert np.abs(du32 - du5).max() < 1e-15
