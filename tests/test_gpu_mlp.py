"""The learned warm start: the BF16 tensor-core MLP kernels against the FP64
oracle (forward, loss, gradient), the Adam step, training, and what the
trained network gains over the method without it."""
import math

import numpy as np
import pytest

from paper_1904_02108_gb300 import learned
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


def _setup(torch, gpu_lib, n, seed):
    P = learned.init_params(seed)
    P[1024:1088] = 0.1  # non-zero biases
    P[-3:] = [0.2, -0.1, 0.05]
    rng = W.SplitMix64(seed + 1)
    X = W.random_array(rng, (n, 16)).astype(np.float32)
    T = W.random_array(rng, (n, 3)).astype(np.float32)
    Pd = torch.tensor(P, device="cuda")
    packed = torch.empty(gpu_lib.mlp_packed_bytes(), dtype=torch.uint8, device="cuda")
    gpu_lib.mlp_pack_dev(Pd, packed, torch.cuda.current_stream())
    return P, X, T, Pd, packed


@pytest.mark.parametrize("n", [1, 1000, 5000])
def test_forward_matches_oracle(gpu_lib, torch_cuda, orc, n):
    torch = torch_cuda
    P, X, _, Pd, packed = _setup(torch, gpu_lib, n, 81)
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    gpu_lib.mlp_forward_dev(Xd, packed, Yd, torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref = orc.mlp_forward(P.astype(np.float64), X.astype(np.float64))
    # BF16 weights and activations: 2^-8 relative per rounding
    assert rel_l2(Yd.cpu().numpy(), ref) < 2e-2


@pytest.mark.parametrize("n", [1000, 4096])
def test_gradient_matches_oracle(gpu_lib, torch_cuda, orc, n):
    torch = torch_cuda
    P, X, T, Pd, packed = _setup(torch, gpu_lib, n, 82)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    grad = torch.zeros_like(Pd)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    scratch = torch.empty(gpu_lib.mlp_grad_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    gpu_lib.mlp_loss_grad_dev(Xd, Td, Pd, packed, grad, loss, scratch, torch.cuda.current_stream())
    torch.cuda.synchronize()
    L, g = orc.mlp_loss_grad(P.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    gg = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - L) < 1e-2 * L
    assert rel_l2(gg, g) < 2e-2
    # every block of the gradient, not only the largest ones
    offs = [0, 1024, 1088, 5184, 5248, 5440, 5443]
    for a, b in zip(offs[:-1], offs[1:]):
        assert rel_l2(gg[a:b], g[a:b]) < 5e-2, (a, b)


def test_adam_step(gpu_lib, torch_cuda):
    torch = torch_cuda
    n = 5443
    rng = W.SplitMix64(83)
    P = W.random_array(rng, (n,)).astype(np.float32)
    m = 0.1 * W.random_array(rng, (n,)).astype(np.float32)
    v = np.abs(0.01 * W.random_array(rng, (n,))).astype(np.float32)
    gr = W.random_array(rng, (n,)).astype(np.float32)
    Pd, md, vd, gd = (torch.tensor(a, device="cuda") for a in (P, m, v, gr))
    gpu_lib.mlp_adam_dev(Pd, md, vd, gd, 3, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8,
                         stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    m1 = 0.9 * m + 0.1 * gr
    v1 = 0.999 * v + 0.001 * gr * gr
    ref = P - 1e-2 * (m1 / (1 - 0.9 ** 3)) / (np.sqrt(v1 / (1 - 0.999 ** 3)) + 1e-8)
    assert np.abs(Pd.cpu().numpy() - ref).max() < 1e-5


def test_training_fits_a_teacher_network(gpu_lib, torch_cuda, orc):
    """Targets from a fixed random MLP (the FP64 oracle as teacher): Adam on
    the GPU kernels cuts the loss by more than 20x."""
    torch = torch_cuda
    teacher = learned.init_params(91)
    rng = W.SplitMix64(92)
    X = W.random_array(rng, (32768, 16)).astype(np.float32)
    T = orc.mlp_forward(teacher.astype(np.float64), X.astype(np.float64)).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    P, losses = learned.train(Xd, Td, epochs=60, batch=4096, lr=3e-3, seed=93)
    assert losses[-1] < losses[0] / 20, losses


def test_learned_start_needs_fewer_iterations(gpu_lib, torch_cuda):
    """Trained on trajectories of single propellers with fresh seeds, the
    network's starting guess reaches the residual target in fewer fixed-point
    iterations than both the zero start and the previous-force start (which
    the learned start corrects: du_prev + V MLP(x)) on a held-out propeller,
    and the converged step still meets the target."""
    torch = torch_cuda
    tol = 1e-3
    train_w = [W.single_propeller(5000 + i) for i in range(4)]
    X, T = learned.generate(train_w, steps=40, tol=tol, max_iter=3000, samples_per_step=360)
    P, losses = learned.train(X, T, epochs=40, batch=2048, lr=2e-3)
    assert losses[-1] < losses[0]
    held = W.single_propeller(6000)
    iters = {}
    for warm in ("zero", "previous", "mlp"):
        lat = gpu_lib.Lattice(held.shape, held.tau, warm=warm, ibm_tol=tol, ibm_max_iter=3000,
                              stream=torch.cuda.current_stream())
        lat.set_propellers(held.props)
        if warm == "mlp":
            lat.set_mlp_weights(P)
        total = 0
        for _ in range(20):
            assert lat.step(1, 0) == gpu_lib.LBM_OK
            total += lat.stats()["last_ibm_iters"]
            assert lat.residuals()[-1] <= tol
        iters[warm] = total
        lat.close()
    print("iterations to eps <= %g over 20 steps: %s" % (tol, iters))
    assert iters["mlp"] < iters["zero"]
    assert iters["mlp"] < iters["previous"]
