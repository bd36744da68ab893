"""The paper's two U pre-computation strategies (Sec. 5) beside the default
brick set: the box strategy (every cell of each body's bounding box, moved by
M(t)) and the kernel strategy (every point's support, duplicated cells).
They change only which cells get U0 and how often, so every step must be
bitwise the one of the brick set, which the oracle pins (relative L2 1e-5 on
U); the cases cover overlapping boxes, a box across the periodic seam, fixed
points moved by the caller, both solvers, tolerance mode and 16-bit
storage."""
import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W

pytestmark = pytest.mark.gpu

STRATEGIES = ["bricks", "box", "kernel"]


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _perturbed(orc, shape, seed, amp=0.01):
    rng = W.SplitMix64(seed)
    rho = 1 + 0.02 * W.random_array(rng, shape)
    U = amp * W.random_array(rng, (3,) + shape)
    return orc.init_equilibrium(shape, rho, U) + 1e-4 * W.random_array(rng, (19,) + shape)


def _run(gpu_lib, torch, w, strategy, steps, n_iter=5, f0=None, **kw):
    lat = gpu_lib.Lattice(w.shape, w.tau, stream=torch.cuda.current_stream(), **kw)
    lat.set_u0_strategy(strategy)
    assert lat.u0_strategy() == strategy
    lat.set_propellers(w.props)
    if f0 is not None:
        lat.set_populations(f0)
    for _ in range(steps):
        lat.step(1, n_iter)
    out = (lat.deviations(), lat.points()[2], lat.stats())
    lat.close()
    return out


def _seam_propeller():
    """One propeller of the 32^3 workload whose centre sits near a corner, so
    that its box (and its supports) wrap across the periodic seam in x and y."""
    w = W.single_propeller(11)
    p = w.props
    shift = np.array([3.5, 29.25, 0.0]) - p.centre[0]
    q = W.Propellers(p.xrest + shift, p.area, p.body, p.centre + shift, p.omega, p.phase,
                     p.blade_length, p.blade_width)
    return W.Workload("seam_propeller_32", w.shape, w.tau, q, w.n_iter, w.steps)


@pytest.mark.parametrize("case", ["single_propeller_32", "seam_propeller_32",
                                  "propeller_array_64"])
def test_strategies_are_bitwise_equal_and_match_oracle(gpu_lib, torch_cuda, orc, case):
    torch = torch_cuda
    f0 = None
    if case == "single_propeller_32":
        w, steps = W.single_propeller(10), 12
    elif case == "seam_propeller_32":
        w, steps = _seam_propeller(), 12
    else:
        w, steps = W.dense_array_64(), 4
        f0 = _perturbed(orc, w.shape, 401)
    res = {s: _run(gpu_lib, torch, w, s, steps, f0=f0) for s in STRATEGIES}
    for s in ("box", "kernel"):
        assert np.array_equal(res[s][0], res["bricks"][0]), s
        assert np.array_equal(res[s][1], res["bricks"][1]), s
        assert res[s][2]["mass"] == res["bricks"][2]["mass"]
    sim = orc.Simulation(w.shape, w.tau, w.props.as_dict(), n_iter=5)
    if f0 is not None:
        sim.f = f0.copy()
    sim.step(steps)
    t = orc.velocity_set()[1][:, None, None, None]
    _, U_o = sim.fields()
    f = res["kernel"][0].astype(np.float64) + t
    _, U = orc.moments(f)
    assert rel_l2(U, U_o) < 1e-5


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_strategies_with_16bit_storage(gpu_lib, torch_cuda, storage):
    torch = torch_cuda
    w = W.single_propeller(12)
    res = {s: _run(gpu_lib, torch, w, s, 6, storage=storage) for s in STRATEGIES}
    for s in ("box", "kernel"):
        assert np.array_equal(res[s][0], res["bricks"][0]), s


@pytest.mark.parametrize("solver", ["mdf", "cg"])
def test_strategies_in_tolerance_mode(gpu_lib, torch_cuda, solver):
    """Iterating to a residual target (previous step's force) with either
    solver: the same iteration counts and bitwise the same state."""
    torch = torch_cuda
    w = W.single_propeller(13)
    tol = 2e-3 if solver == "mdf" else 1e-4
    res = {}
    for s in STRATEGIES:
        lat = gpu_lib.Lattice(w.shape, w.tau, warm="previous", ibm_tol=tol, ibm_max_iter=3000,
                              stream=torch.cuda.current_stream(), solver=solver)
        lat.set_u0_strategy(s)
        lat.set_propellers(w.props)
        iters = []
        for _ in range(4):
            assert lat.step(1, 0) == gpu_lib.LBM_OK
            iters.append(lat.stats()["last_ibm_iters"])
        res[s] = (lat.deviations(), iters)
        lat.close()
    for s in ("box", "kernel"):
        assert res[s][1] == res["bricks"][1]
        assert np.array_equal(res[s][0], res["bricks"][0]), s


def test_box_follows_points_moved_by_the_caller(gpu_lib, torch_cuda, orc):
    """Fixed points without bodies (a sheet moved along x by the caller each
    step through ibm_update_points): the box strategy recomputes the box of
    the moved positions; bitwise the brick set's steps."""
    torch = torch_cuda
    shape = (24, 20, 28)
    xs = np.array([(6.3 + 0.7 * i, 9.1, 5.2 + 0.7 * k) for i in range(12) for k in range(14)])
    ut = np.tile([0.02, 0.0, 0.0], (len(xs), 1))
    area = np.full(len(xs), 0.49)
    out = {}
    for s in STRATEGIES:
        lat = gpu_lib.Lattice(shape, 0.7, stream=torch.cuda.current_stream())
        lat.set_u0_strategy(s)
        lat.set_points(xs, ut, area)
        X = xs.copy()
        for step in range(6):
            X = X + np.array([0.02, 0.0, 0.0]) * step
            lat.update_points(X)
            lat.step(1, 5)
        torch.cuda.synchronize()
        out[s] = lat.deviations()
        lat.close()
    for s in ("box", "kernel"):
        assert np.array_equal(out[s], out["bricks"]), s
    assert np.abs(out["bricks"]).max() > 0


def test_strategy_arguments_and_batches(gpu_lib, torch_cuda):
    torch = torch_cuda
    w = W.single_propeller(14)
    lat = gpu_lib.Lattice(w.shape, w.tau, stream=torch.cuda.current_stream())
    with pytest.raises(gpu_lib.LbmError) as e:
        gpu_lib._check(gpu_lib.load().lbm_set_u0_strategy(lat.h, 7), lat.h)
    assert e.value.code == gpu_lib.LBM_EINVAL
    assert lat.u0_strategy() == "bricks"
    lat.set_propellers(w.props)
    lat.set_u0_strategy("kernel")
    other = gpu_lib.Lattice(w.shape, w.tau, stream=torch.cuda.current_stream())
    other.set_propellers(w.props)
    batch = gpu_lib.Batch([lat, other])
    with pytest.raises(gpu_lib.LbmError) as e:
        batch.step(1, 5)
    assert e.value.code == gpu_lib.LBM_EINVAL
    batch.close()
    for h in (lat, other):
        h.close()
