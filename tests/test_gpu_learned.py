"""The learned warm start on the GPU against the FP64 oracle, element by
element: the 16 features of every point (mlp_features_kernel), the initial
guess du_prev + V MLP(x) (mlp_warm_kernel) inside whole fixed-count steps,
and the iteration gain of the trained network over the previous-force start.

Tolerances.  The features are FP32 functions of the FP32 state: velocities
(u ~ 0.05, stored as u / V with V = 0.05, so O(1)) agree to the FP32 drift of
the state over a few steps (~1e-6 relative to the largest value of the
group); the density is a ratio of small integers (one FP32 rounding); radius,
height and speed are FP64 values rounded to FP32.  Through the MLP, the BF16
weights and activations give at most 2e-2 relative error on its output
(test_gpu_mlp), so the learned part V MLP(x) of the initial guess carries at
most 2e-2 of its own norm; with a bias-only network the output is exact in
FP32 and the whole learned step is held to the plain FP32 bar (1e-5)."""
import numpy as np
import pytest

from paper_1904_02108_gb300 import learned
from paper_1904_02108_gb300 import workload as W

pytestmark = pytest.mark.gpu

V = 0.05


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


def _gpu_features(gpu_lib, torch, lat, n):
    X = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    lat.mlp_sample_dev(X, None)
    torch.cuda.synchronize()
    return X.cpu().numpy().astype(np.float64)


def _check_features(F, ref):
    groups = {"u_i": [0, 1, 2], "u_k": [3, 4, 5], "du_prev": [6, 7, 8], "slip": [13, 14, 15]}
    for name, cols in groups.items():
        scale = max(np.abs(ref[:, cols]).max(), 1e-3)
        err = np.abs(F[:, cols] - ref[:, cols]).max()
        assert err <= 2e-5 * scale, (name, err, scale)
    # density: small-integer ratios, one FP32 rounding
    assert np.abs(F[:, 9] - ref[:, 9]).max() <= 1e-7 * np.abs(ref[:, 9]).max()
    # radius, height, rotation speed: FP64 values rounded to FP32
    for c in (10, 11, 12):
        scale = max(np.abs(ref[:, c]).max(), 1e-6)
        assert np.abs(F[:, c] - ref[:, c]).max() <= 2e-7 * scale, c


@pytest.mark.parametrize("case", ["single_propeller_32", "propeller_array_64"])
@pytest.mark.parametrize("steps", [1, 4])
def test_features_match_oracle(gpu_lib, torch_cuda, orc, case, steps):
    """Features of the step after `steps - 1` steps from the previous-force
    start: the first step (no previous force, fluid at rest or perturbed) and
    a later one, on one propeller and on the 64^3 array of 216 propellers
    whose supports share bricks."""
    torch = torch_cuda
    if case == "single_propeller_32":
        w = W.single_propeller(7)
        f0 = None
    else:
        w = W.dense_array_64()
        f0 = _perturbed(orc, w.shape, 311)
    p = w.props
    lat = gpu_lib.Lattice(w.shape, w.tau, warm="previous",
                          stream=torch.cuda.current_stream())
    lat.set_propellers(p)
    lat.set_features(True)
    sim = orc.Simulation(w.shape, w.tau, p.as_dict(), warm="previous", n_iter=w.n_iter)
    if f0 is not None:
        lat.set_populations(f0)
        sim.f = f0.copy()
    lat.step(steps, w.n_iter)
    F = _gpu_features(gpu_lib, torch, lat, p.n_points)
    # the oracle's features of the same step, from its own state
    sim.step(steps - 1)
    _, U0 = sim.fields()
    x, ut = sim.positions()
    du_prev = sim.du.copy() if steps > 1 else None
    ref = orc.mlp_features(U0, x, ut, du_prev, body=p.body, centre=p.centre, omega=p.omega)
    _check_features(F, ref)
    if steps == 1:
        assert np.all(F[:, 6:9] == 0.0)
    lat.close()


def test_features_of_fixed_points_without_bodies(gpu_lib, torch_cuda, orc):
    """Points with a prescribed surface velocity and no bodies: radius,
    height and speed are zero; the rest as the oracle."""
    torch = torch_cuda
    shape = (16, 24, 32)
    rng = W.SplitMix64(312)
    n = 300
    x = W.random_points(rng, n, shape)
    ut = 0.03 * W.random_array(rng, (n, 3))
    area = 0.5 + 0.5 * np.abs(W.random_array(rng, (n,)))
    f0 = _perturbed(orc, shape, 313, amp=0.02)
    lat = gpu_lib.Lattice(shape, 0.7, warm="previous", stream=torch.cuda.current_stream())
    lat.set_points(x, ut, area)
    lat.set_populations(f0)
    lat.set_features(True)
    ut32 = ut.astype(np.float32).astype(np.float64)
    sim = orc.Simulation(shape, 0.7, dict(x=x, ut=ut32, area=area.astype(np.float32)),
                         warm="previous")
    sim.f = f0.copy()
    lat.step(3, 5)
    F = _gpu_features(gpu_lib, torch, lat, n)
    sim.step(2)
    _, U0 = sim.fields()
    ref = orc.mlp_features(U0, x, ut32, sim.du)
    _check_features(F, ref)
    assert np.all(F[:, 10:13] == 0.0)
    lat.close()


def _learned_pair(gpu_lib, torch, orc, w, P, f0=None):
    lat = gpu_lib.Lattice(w.shape, w.tau, warm="mlp", stream=torch.cuda.current_stream())
    lat.set_propellers(w.props)
    lat.set_mlp_weights(P.astype(np.float32))
    sim = orc.Simulation(w.shape, w.tau, w.props.as_dict(), warm="mlp",
                         mlp=P.astype(np.float32).astype(np.float64), n_iter=w.n_iter)
    if f0 is not None:
        lat.set_populations(f0)
        sim.f = f0.copy()
    return lat, sim


def test_learned_step_with_a_bias_only_network_matches_oracle(gpu_lib, torch_cuda, orc):
    """A network whose output is its bias b3 (exact in FP32): every learned
    step starts from du_prev + V b3 on both sides, so fields, forces and
    corrections after 10 fixed-count steps meet the FP32 bar of the plain
    method (relative L2 1e-5).  A wrong scale, sign or previous-force term in
    the initial guess would move du by V |b3| per step."""
    torch = torch_cuda
    w = W.single_propeller(8)
    P = np.zeros(learned.NPARAM)
    P[-3:] = [0.0625, -0.125, 0.03125]
    lat, sim = _learned_pair(gpu_lib, torch, orc, w, P)
    for chunk in (1, 4, 5):
        lat.step(chunk, w.n_iter)
        sim.step(chunk)
        _, U, G = lat.fields()
        _, U_o = sim.fields()
        _, _, du = lat.points()
        assert rel_l2(U, U_o) < 1e-5, (sim.t, rel_l2(U, U_o))
        assert rel_l2(G, sim.G) < 1e-5
        assert rel_l2(du, sim.du) < 1e-5
    lat.close()


@pytest.mark.parametrize("case", ["single_propeller_32", "propeller_array_64"])
def test_learned_step_with_a_random_network_matches_oracle(gpu_lib, torch_cuda, orc, case):
    """A random network (Glorot weights, non-zero biases) through the BF16
    tensor-core MLP: after each learned step the correction du differs from
    the oracle's by at most 2e-2 of the learned part V MLP(x) of the initial
    guess plus the FP32 bar on du, summed over the steps so far (the fixed
    point's iterations do not amplify an error of the initial guess: with the
    uniform s of a propeller, s A is symmetric with eigenvalues in [0, 1), so
    |1 - s A| <= 1; the previous step's error enters through du_prev)."""
    torch = torch_cuda
    if case == "single_propeller_32":
        w, f0 = W.single_propeller(9), None
    else:
        w = W.dense_array_64()
        f0 = _perturbed(orc, w.shape, 314)
    P = learned.init_params(315).astype(np.float64)
    P[1024:1088] = 0.05
    P[-3:] = [0.1, -0.05, 0.02]
    lat, sim = _learned_pair(gpu_lib, torch, orc, w, P, f0)
    bound = 0.0
    for _ in range(3):
        du_prev = sim.du.copy()
        lat.step(1, w.n_iter)
        sim.step(1)
        _, _, du = lat.points()
        learned_part = np.linalg.norm(sim.du_init - (du_prev if sim.t > 1 else 0.0))
        # the previous steps' differences carry over through du_prev
        bound += 2e-2 * learned_part + 1e-5 * np.linalg.norm(sim.du)
        err = np.linalg.norm(du.astype(np.float64) - sim.du)
        print("step %d: |du - du_oracle| = %.3g, bound %.3g, |V MLP| = %.3g, |du| = %.3g"
              % (sim.t, err, bound, learned_part, np.linalg.norm(sim.du)))
        assert err <= bound, (sim.t, err, bound)
    lat.close()
