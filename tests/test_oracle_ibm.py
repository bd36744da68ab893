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


# ---- conjugate gradients on the lattice form of the fixed point -------------

def _dense_B(orc, shape, x, s, kernel="cosine"):
    """B = S diag(s) I on one component of the lattice (cells x cells)."""
    nz, ny, nx = shape
    N = nx * ny * nz
    B = np.zeros((N, N))
    for j in range(N):
        E = np.zeros((3,) + tuple(shape))
        E[0].reshape(-1)[j] = 1.0
        y = orc.interpolate(E, x, kernel) * s[:, None]
        B[:, j] = orc.spread(shape, x, y, kernel)[0].reshape(-1)
    return B


def _energy(orc, E, x, s):
    """E . B E = sum_k s(k) |I[E](k)|^2."""
    y = orc.interpolate(E, x)
    return float((s[:, None] * y * y).sum())


def _sheet_case(seed, spacing=0.7, svals=(0.49,)):
    shape = (6, 8, 6)
    x = _sheet(shape, spacing)
    n = len(x)
    rng = W.SplitMix64(seed)
    U0 = 0.01 * W.random_array(rng, (3,) + shape)
    ut = 0.02 * W.random_array(rng, (n, 3))
    s = np.array([svals[k % len(svals)] for k in range(n)], dtype=np.float64)
    return shape, x, U0, ut, s


def test_cg_iterates_are_textbook_cg_on_the_lattice_system(orc):
    """The oracle's CG, run through point vectors, against scipy's CG on the
    dense lattice system B G = c (B = S diag(s) I per component, the three
    components one system), from a warm start, iterate by iterate."""
    sla = pytest.importorskip("scipy.sparse.linalg")
    shape, x, U0, ut, s = _sheet_case(40, svals=(0.49, 0.3, 0.6))
    n = len(x)
    rng = W.SplitMix64(41)
    du0 = 0.5 * W.random_array(rng, (n, 3))
    B1 = _dense_B(orc, shape, x, s)
    B = np.kron(np.eye(3), B1)
    c = orc.spread(shape, x, s[:, None] * (ut - orc.interpolate(U0, x))).reshape(-1)
    G0 = orc.spread(shape, x, du0).reshape(-1)
    ref = []
    sla.cg(B, c, x0=G0.copy(), rtol=0.0, atol=0.0, maxiter=8,
           callback=lambda xk: ref.append(xk.copy()))
    assert len(ref) == 8
    for k in (1, 2, 3, 5, 8):
        G, du, eps, _, _ = orc.ibm_cg(U0, x, ut, s, n_iter=k, du_init=du0)
        scale = np.abs(ref[k - 1]).max()
        assert np.abs(G.reshape(-1) - ref[k - 1]).max() < 1e-11 * scale
        # eps_j is the norm of the lattice residual c - B G_j over ||S[s u_t]||
        den = np.linalg.norm(orc.spread(shape, x, s[:, None] * ut))
        Gj = G0 if k == 1 else ref[k - 2]
        assert abs(eps[-1] - np.linalg.norm(c - B @ Gj) / den) < 1e-11 * eps[-1]


def test_cg_exact_after_as_many_iterations_as_distinct_eigenvalues(orc):
    """Points whose supports are disjoint: B restricted to them has the
    eigenvalues s(k) (3/8)^3, so with two distinct areas CG is exact after two
    iterations: du = (u_t - I[U0]) / (3/8)^3 (Sec. 3's single-point
    self-interaction), and the residual vanishes."""
    shape = (16, 16, 16)
    x = np.array([(2.3 + 8 * i, 3.6 + 8 * j, 1.1 + 8 * k)
                  for i in range(2) for j in range(2) for k in range(2)], dtype=np.float64)
    n = len(x)
    rng = W.SplitMix64(42)
    U0 = 0.01 * W.random_array(rng, (3,) + shape)
    ut = 0.02 * W.random_array(rng, (n, 3))
    s = np.array([0.49 if k % 2 else 1.3 for k in range(n)])
    b = ut - orc.interpolate(U0, x)
    G, du, eps, _, _ = orc.ibm_cg(U0, x, ut, s, n_iter=3)
    assert eps[0] > 0.1 and eps[1] > 1e-3 and eps[2] < 1e-14
    assert np.abs(du - b / (3 / 8) ** 3).max() < 1e-13 * np.abs(du).max()
    _, _, eps1, _, _ = orc.ibm_cg(U0, x, ut, np.full(n, 0.7), n_iter=2)
    assert eps1[1] < 1e-14  # one distinct eigenvalue: exact after one iteration


def test_cg_and_fixed_point_reach_the_same_force(orc):
    """On the singular 0.7-spacing sheet both methods converge to the one
    solution of B G = c in G_0 + range(B): CG in a few dozen iterations, the
    loop of Sec. 3 in ~20k."""
    shape, x, U0, ut, s = _sheet_case(28)
    Gc, duc, epsc, _, _ = orc.ibm_cg(U0, x, ut, s, n_iter=0, tol=1e-12, max_iter=500)
    Gm, dum, epsm, _ = orc.ibm(U0, x, ut, s, n_iter=0, tol=1e-12, max_iter=100000)
    assert len(epsc) < 60 and len(epsm) > 10000
    assert epsc[-1] <= 1e-12 and epsm[-1] <= 1e-12
    assert np.abs(Gc - Gm).max() < 1e-9 * np.abs(Gm).max()
    # converged: the corrected field meets the surface velocity in the sense
    # the kernel resolves (the lattice residual), not pointwise
    assert np.linalg.norm(orc.spread(shape, x, s[:, None] * (ut - orc.interpolate(U0 + Gc, x)))) \
        < 1e-11 * np.linalg.norm(orc.spread(shape, x, s[:, None] * ut))


def test_cg_energy_error_is_minimal_over_the_same_krylov_space(orc):
    """Uniform s: the loop of Sec. 3 and CG build G_n in the same affine
    Krylov space G_0 + K_n(B, R_0); CG's error in the energy norm of B is the
    minimum over it, so it never exceeds the loop's and never increases."""
    shape, x, U0, ut, s = _sheet_case(43)
    Gs, _, _, _, _ = orc.ibm_cg(U0, x, ut, s, n_iter=0, tol=1e-13, max_iter=500)
    prev = np.inf
    for n in range(1, 13):
        Gc = orc.ibm_cg(U0, x, ut, s, n_iter=n)[0]
        Gm = orc.ibm(U0, x, ut, s, n_iter=n)[0]
        ec, em = _energy(orc, Gc - Gs, x, s), _energy(orc, Gm - Gs, x, s)
        assert ec <= em * (1 + 1e-10) + 1e-30
        assert ec <= prev * (1 + 1e-10)
        prev = ec
    assert ec < 1e-2 * em  # 12 iterations: ~200x smaller


def test_cg_residual_recursion_is_the_residual_of_the_iterate(orc):
    """eps_n, carried by the recursion r_{n+1} = r_n - alpha y_n, equals the
    definition ||S[s (u_t - I[U0 + S[du_n]])]|| / ||S[s u_t]|| recomputed from
    the iterate du_n; u_interp = I[U0 + S[du_n]] of the last iterate."""
    shape, x, U0, ut, s = _sheet_case(44, svals=(0.49, 0.35))
    rng = W.SplitMix64(45)
    du0 = 0.3 * W.random_array(rng, (len(x), 3))
    _, _, eps, eps_pt, _ = orc.ibm_cg(U0, x, ut, s, n_iter=9, du_init=du0)
    den = np.linalg.norm(orc.spread(shape, x, s[:, None] * ut))
    for n in range(9):
        du_n = du0 if n == 0 else orc.ibm_cg(U0, x, ut, s, n_iter=n, du_init=du0)[1]
        ui = orc.interpolate(U0 + orc.spread(shape, x, du_n), x)
        e = np.linalg.norm(orc.spread(shape, x, s[:, None] * (ut - ui))) / den
        assert abs(eps[n] - e) < 1e-10 * e
        assert abs(eps_pt[n] - np.linalg.norm(ut - ui) / np.linalg.norm(ut)) < 1e-10 * eps_pt[n]
        if n:
            ui_last = orc.ibm_cg(U0, x, ut, s, n_iter=n + 1, du_init=du0)[4]
            assert np.abs(ui_last - ui).max() < 1e-12


def test_cg_tolerance_mode_stops_at_first_iterate_below_tol(orc):
    shape, x, U0, ut, s = _sheet_case(46)
    _, _, eps_fixed, _, _ = orc.ibm_cg(U0, x, ut, s, n_iter=30)
    tol = 0.05
    assert eps_fixed[0] > tol > eps_fixed[-1]
    _, _, eps, _, _ = orc.ibm_cg(U0, x, ut, s, n_iter=0, tol=tol, max_iter=30)
    k = int(np.argmax(eps_fixed <= tol))
    assert len(eps) == k + 1 and np.array_equal(eps, eps_fixed[:k + 1])
    _, _, eps_cap, _, _ = orc.ibm_cg(U0, x, ut, s, n_iter=0, tol=1e-30, max_iter=7)
    assert len(eps_cap) == 7
