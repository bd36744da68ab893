"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP32 arithmetic on O(1e-2) velocities; the bar for fields after
many steps is the relative L2 error 1e-5 on U; single operators are held to
a few FP32 ulps of their inputs' scale.
"""
import math

import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _lattice(gpu_lib, torch_cuda, shape, tau, **kw):
    return gpu_lib.Lattice(shape, tau, stream=torch_cuda.cuda.current_stream(), **kw)


def _perturbed(orc, shape, seed, amp=0.03):
    rng = W.SplitMix64(seed)
    rho = 1 + 0.02 * W.random_array(rng, shape)
    U = amp * W.random_array(rng, (3,) + shape)
    return orc.init_equilibrium(shape, rho, U) + 1e-4 * W.random_array(rng, (19,) + shape)


# ---------------------------------------------------------------- LBM only


@pytest.mark.parametrize("shape", [(4, 8, 12), (12, 20, 36), (8, 8, 4)])
def test_populations_roundtrip(gpu_lib, torch_cuda, orc, shape):
    f = _perturbed(orc, shape, 40)
    lat = _lattice(gpu_lib, torch_cuda, shape, 0.8)
    lat.set_populations(f)
    g = lat.populations()
    assert np.abs(g - f).max() < 1e-7  # FP32 deviations
    lat.close()


@pytest.mark.parametrize("shape,tau", [((12, 20, 36), 0.8), ((4, 8, 12), 0.6), ((8, 8, 8), 1.3)])
def test_collide_stream_matches_oracle_one_step(gpu_lib, torch_cuda, orc, shape, tau):
    """Eqs. 1-4 with a uniform body force (the forcing path of step 3) on a
    lattice whose cell count is not a multiple of the block size (ragged
    tail) and spans many blocks."""
    f = _perturbed(orc, shape, 41)
    gb = np.array([1e-4, -3e-5, 2e-5])
    lat = _lattice(gpu_lib, torch_cuda, shape, tau)
    lat.set_populations(f)
    lat.set_body_force(gb)
    lat.step(1, 5)
    g = lat.populations()
    rho, U = orc.moments(f)
    G = np.broadcast_to(gb[:, None, None, None], (3,) + shape).copy()
    ref = orc.stream(orc.collide(f, tau, rho, U, G))
    t = orc.velocity_set()[1]
    dev = ref - t[:, None, None, None]
    assert np.abs(g - ref).max() < 2e-7
    assert rel_l2(g - t[:, None, None, None], dev) < 2e-6
    lat.close()


def test_lbm_only_100_steps_and_mass(gpu_lib, torch_cuda, orc):
    shape = (16, 16, 16)
    f = _perturbed(orc, shape, 42)
    lat = _lattice(gpu_lib, torch_cuda, shape, 0.7)
    lat.set_populations(f)
    lat.step(100, 5)
    rho, U, _ = lat.fields()
    sim = orc.Simulation(shape, 0.7)
    sim.f = f.copy()
    sim.step(100)
    rho_o, U_o = sim.fields()
    assert rel_l2(U, U_o) < 1e-5
    # rho is returned in FP32: a few ulps of 1 (1.2e-7) absolute
    assert np.abs(rho - rho_o).max() < 5e-7
    s = lat.stats()
    # the FP64 sums are those of the populations the GPU holds ...
    dg = lat.deviations().astype(np.float64)
    e, _ = orc.velocity_set()
    exact = [dg.shape[1] * dg.shape[2] * dg.shape[3] + math.fsum(dg.ravel())] + [
        math.fsum((e[:, c, None, None, None] * dg).ravel()) for c in range(3)]
    assert abs(s["mass"] - exact[0]) < 1e-7
    assert np.abs(np.array(s["momentum"]) - exact[1:]).max() < 1e-7
    # ... and FP32 storage conserves mass to its rounding (1e-7 relative)
    m0 = orc.sums(f)[0]
    assert abs(s["mass"] - m0) / m0 < 1e-7
    assert s["step"] == 100
    lat.close()


# ---------------------------------------------------- operators (stateless)


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
@pytest.mark.parametrize("shape,n", [((8, 12, 16), 50), ((32, 32, 32), 3000)])
def test_interpolation_operator(gpu_lib, torch_cuda, orc, kernel, shape, n):
    torch = torch_cuda
    rng = W.SplitMix64(43)
    U = W.random_array(rng, (3,) + shape)
    x = W.random_points(rng, n, shape)
    x[:5] = [[0.01, 0.2, 0.3], [shape[2] - 0.01, 1.0, 2.0], [3.0, shape[1] - 0.5, 0.0],
             [-0.75, -1.25, shape[0] + 0.5], [2.0, 3.0, 1.0]]  # seams, outside, integer
    Ud = torch.tensor(U, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    ud = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    gpu_lib.interpolate_dev(Ud, xd, ud, kernel, torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref = orc.interpolate(U.astype(np.float32).astype(np.float64), x, kernel)
    assert np.abs(ud.cpu().numpy() - ref).max() < 2e-6


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
@pytest.mark.parametrize("shape,n,own", [((8, 12, 16), 50, True), ((32, 32, 32), 3000, False),
                                          ((4, 4, 8), 40, False)])
def test_spreading_operator(gpu_lib, torch_cuda, orc, kernel, shape, n, own):
    """Atomic-free gather spread vs the oracle's scatter (Alg. 2), including
    dims of one and two bricks where neighbour bins alias."""
    torch = torch_cuda
    rng = W.SplitMix64(44)
    x = W.random_points(rng, n, shape)
    v = W.random_array(rng, (n, 3))
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    vd = torch.tensor(v, dtype=torch.float32, device="cuda")
    F = torch.full((3,) + shape, 7.0, dtype=torch.float32, device="cuda")
    scratch = None
    if not own:
        nb = gpu_lib.spread_scratch_bytes(shape, n)
        scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    gpu_lib.spread_dev(xd, vd, F, kernel, scratch, torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref = orc.spread(shape, x, v.astype(np.float32).astype(np.float64), kernel)
    scale = np.abs(v).max() * 8
    assert np.abs(F.cpu().numpy() - ref).max() < 2e-6 * scale
    # deterministic: a second call is bitwise identical
    F2 = torch.empty_like(F)
    gpu_lib.spread_dev(xd, vd, F2, kernel, scratch, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.equal(F, F2)


# ------------------------------------------------------------ coupled step


def test_kinematics_matches_oracle(gpu_lib, torch_cuda, orc):
    """Positions x(t) = M(t) x_rest and u_k = x(t) - x(t-1) (Alg. 1): one
    iteration from a fluid at rest gives du = s u_k exactly."""
    w = W.dense_array_64()
    p = w.props
    lat = _lattice(gpu_lib, torch_cuda, w.shape, w.tau)
    lat.set_propellers(p)
    lat.set_time(37)
    lat.step(1, 1)
    x, u, du = lat.points()
    xo, uto = orc.kinematics(p.xrest, p.body, p.centre, p.omega, p.phase, 37)
    assert np.abs(x - xo).max() < 1e-12
    assert np.abs(u).max() == 0.0
    assert np.abs(du - p.area[:, None] * uto).max() < 1e-8
    lat.close()


def _run_pair(gpu_lib, torch_cuda, orc, w, steps, kernel="cosine", f0=None):
    lat = _lattice(gpu_lib, torch_cuda, w.shape, w.tau, delta=kernel)
    lat.set_propellers(w.props)
    sim = orc.Simulation(w.shape, w.tau, w.props.as_dict(), n_iter=w.n_iter, kernel=kernel)
    if f0 is not None:
        lat.set_populations(f0)
        sim.f = f0.copy()
    return lat, sim


def test_single_propeller_100_steps(gpu_lib, torch_cuda, orc):
    """32^3, tau 0.8, one propeller, 5 iterations, 100 steps: relative L2 of
    U below 1e-5 against the FP64 oracle, also at intermediate steps, and the
    IBM force and per-point corrections."""
    w = W.single_propeller()
    lat, sim = _run_pair(gpu_lib, torch_cuda, orc, w, 100)
    for chunk in (1, 9, 40, 50):
        lat.step(chunk, w.n_iter)
        sim.step(chunk)
        rho, U, G = lat.fields()
        rho_o, U_o = sim.fields()
        assert rel_l2(U, U_o) < 1e-5, (sim.t, rel_l2(U, U_o))
        assert np.abs(rho - rho_o).max() < 5e-7
        assert rel_l2(G, sim.G) < 1e-5
        _, _, du = lat.points()
        assert rel_l2(du, sim.du) < 1e-5
    s = lat.stats()
    assert s["step"] == 100 and s["last_ibm_iters"] == 5 and s["active_bricks"] > 0
    m0 = 32 ** 3
    assert abs(s["mass"] - m0) / m0 < 1e-9
    lat.close()


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
def test_dense_array_downscale_from_perturbed_state(gpu_lib, torch_cuda, orc, kernel):
    """64^3 array of 216 small propellers (supports of neighbours overlap in
    bins), started from a perturbed flow so that U0 is non-trivial; 10 steps."""
    w = W.dense_array_64()
    f0 = _perturbed(orc, w.shape, 45, amp=0.01)
    lat, sim = _run_pair(gpu_lib, torch_cuda, orc, w, 10, kernel, f0)
    lat.step(10, w.n_iter)
    sim.step(10)
    rho, U, G = lat.fields()
    rho_o, U_o = sim.fields()
    assert rel_l2(U, U_o) < 1e-5
    assert rel_l2(G, sim.G) < 1e-5
    lat.close()


def test_couette_planes_match_oracle(gpu_lib, torch_cuda, orc):
    """Static-position points with prescribed velocity (no bodies) in a box
    one brick wide: 300 steps."""
    ny, n, tau, Uw = 32, 4, 1.0, 0.01
    m = 6
    sp = n / m
    xs, ut = [], []
    for yw, u in ((8.0, -Uw), (24.0, Uw)):
        for i in range(m):
            for k in range(m):
                xs.append((sp * i + 0.3, yw, sp * k + 0.1))
                ut.append((u, 0.0, 0.0))
    xs, ut = np.array(xs), np.array(ut)
    P = dict(x=xs, ut=ut, area=np.full(len(xs), sp * sp))
    lat = _lattice(gpu_lib, torch_cuda, (n, ny, n), tau)
    lat.set_points(xs, ut, P["area"])
    sim = orc.Simulation((n, ny, n), tau, P)
    lat.step(300, 5)
    sim.step(300)
    _, U, _ = lat.fields()
    _, U_o = sim.fields()
    assert rel_l2(U, U_o) < 1e-5
    lat.close()


def test_deterministic_and_resumable(gpu_lib, torch_cuda, orc):
    w = W.single_propeller()
    a = _lattice(gpu_lib, torch_cuda, w.shape, w.tau)
    a.set_propellers(w.props)
    a.step(7, 5)
    state = a.save_state()
    a.step(5, 5)
    fa = a.populations()
    b = _lattice(gpu_lib, torch_cuda, w.shape, w.tau)
    b.set_propellers(w.props)
    b.step(12, 5)
    assert np.array_equal(fa, b.populations())  # run to run bitwise
    c = _lattice(gpu_lib, torch_cuda, w.shape, w.tau)
    c.load_state(state)
    assert c.time == 7
    c.step(5, 5)
    assert np.array_equal(fa, c.populations())  # resume bitwise
    for lat in (a, b, c):
        lat.close()


def test_timing_and_launch_counters(gpu_lib, torch_cuda):
    w = W.single_propeller()
    lat = _lattice(gpu_lib, torch_cuda, w.shape, w.tau)
    lat.set_propellers(w.props)
    lat.enable_timing(True)
    lat.step(3, 5)
    t = lat.timing()
    assert t["collide_stream"][1] == 3 and t["point_update"][1] == 15
    assert t["brick_spread"][1] == 15 and t["brick_init"][1] == 6 and t["pairs"][1] == 9
    assert t["collide_active"][1] == 0  # one collide over every cell (no overlap)
    assert all(ms >= 0 for ms, _ in t.values()) and t["collide_stream"][0] > 0
    # per step: kinematics, 3 pair kernels, moments + init, 5 x 2 iteration
    # kernels, collide-stream, stats
    assert lat.stats()["kernel_launches"] == 3 * (1 + 3 + 2 + 10 + 1 + 1)
    lat.close()


def test_bad_arguments_return_codes(gpu_lib, torch_cuda):
    lat = _lattice(gpu_lib, torch_cuda, (8, 8, 8), 0.8)
    with pytest.raises(gpu_lib.LbmError) as e:
        lat.set_points(np.array([[1.0, np.nan, 2.0]]))
    assert e.value.code == gpu_lib.LBM_ENONFINITE
    with pytest.raises(gpu_lib.LbmError) as e:
        lat.step(-1, 5)
    assert e.value.code == gpu_lib.LBM_EINVAL
    lat.set_points(np.array([[1.0, 2.0, 3.0]]), body=np.array([2]))
    with pytest.raises(gpu_lib.LbmError):
        lat.set_bodies(np.zeros((1, 3)), [0.1], [0.0])  # body 2 of 1
    with pytest.raises(gpu_lib.LbmError) as e:
        lat.load_state(np.zeros(16, np.uint8))
    assert e.value.code == gpu_lib.LBM_ESTATE
    lat.close()


def test_async_readback_matches_blocking(gpu_lib, torch_cuda):
    torch = torch_cuda
    w = W.single_propeller(2)
    a = _lattice(gpu_lib, torch, w.shape, w.tau, warm="previous")
    b = _lattice(gpu_lib, torch, w.shape, w.tau, warm="previous")
    n = w.props.n_points
    pin = lambda shape, dt: torch.zeros(shape, dtype=dt).pin_memory().numpy()
    x, u, du = pin((n, 3), torch.float64), pin((n, 3), torch.float32), pin((n, 3), torch.float32)
    sums = pin(4, torch.float64)
    sums[:] = 7.0
    a.sums_async(sums)  # no sums before the first step: left unchanged
    torch.cuda.current_stream().synchronize()
    assert np.all(sums == 7.0)
    for lat in (a, b):
        lat.set_propellers(w.props)
        lat.step(3, 5)
    a.points_async(x, u, du)
    a.sums_async(sums)
    a.step(1, 5)  # enqueued after the copies: they hold step 3's values
    torch.cuda.current_stream().synchronize()
    xb, ub, dub = b.points()
    sb = b.stats()
    assert np.array_equal(x, xb) and np.array_equal(u, ub) and np.array_equal(du, dub)
    assert sums[0] == sb["mass"] and tuple(sums[1:]) == sb["momentum"]
    a.points_async(du=du)
    a.sums_async(sums)
    torch.cuda.current_stream().synchronize()
    _, _, du4 = a.points()
    sa = a.stats()
    assert np.array_equal(du, du4) and not np.array_equal(du4, dub)
    assert sums[0] == sa["mass"] and tuple(sums[1:]) == sa["momentum"]
    for lat in (a, b):
        lat.close()


def test_non_finite_populations_are_refused_and_overflow_is_reported(gpu_lib, torch_cuda, orc):
    """Failure paths on the host: a NaN population given to
    lbm_write_populations is refused (LBM_ENONFINITE) and the state is left
    as it was; finite populations whose density overflows FP32 (two rest
    populations of 3e38 in one 128-cell partial sum) make the step's FP64 mass
    sum infinite, which lbm_read_stats reports as LBM_ENONFINITE."""
    shape = (8, 8, 8)
    lat = _lattice(gpu_lib, torch_cuda, shape, 0.8)
    f = orc.init_equilibrium(shape)
    bad = f.copy()
    bad[5, 3, 2, 1] = np.nan
    with pytest.raises(gpu_lib.LbmError) as e:
        lat.set_populations(bad)
    assert e.value.code == gpu_lib.LBM_ENONFINITE
    assert np.abs(lat.populations() - f).max() < 1e-7
    assert lat.step(1, 5) == gpu_lib.LBM_OK
    assert np.isfinite(lat.stats()["mass"])
    big = f.copy()
    big[0, 0, 0, 0] = big[0, 0, 0, 1] = 3e38  # rest population: not streamed
    lat.set_populations(big)
    assert lat.step(1, 5) == gpu_lib.LBM_OK  # does not wait for the GPU
    with pytest.raises(gpu_lib.LbmError) as e:
        lat.stats()
    assert e.value.code == gpu_lib.LBM_ENONFINITE
    lat.close()
