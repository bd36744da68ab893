"""Learned warm start of the fixed point: training data from solver
trajectories and the training loop, on the GPU through the library's own
MLP kernels (mlp_loss_grad_dev, mlp_adam_dev).  Device memory comes from
PyTorch; every forward, backward and optimizer step runs in liblbmibm.so.

Data: the solver advances propeller workloads in tolerance mode from the
previous step's force; at every step it records each point's features and
the target (final du - previous du) / V (ibm_read_mlp_sample_dev), of which a
random subset of points is kept.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding
from . import workload as W

NPARAM = binding.MLP_NPARAM


def init_params(seed: int = 7):
    """Glorot-uniform weights, zero biases, as a host FP32 vector."""
    rng = W.SplitMix64(seed)
    parts = []
    for fan_in, fan_out in ((16, 64), (64, 64), (64, 3)):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        parts.append(W.random_array(rng, (fan_out * fan_in,), -lim, lim))
        parts.append(np.zeros(fan_out))
    P = np.concatenate(parts).astype(np.float32)
    assert P.size == NPARAM
    return P


def generate(workloads, steps, tol=1e-4, max_iter=2000, samples_per_step=4096, seed=0,
             storage="f32", skip=2, solver="mdf"):
    """Runs each workload for `steps` steps (tolerance mode, previous-force
    start, with the paper's loop ("mdf") or conjugate gradients ("cg") on the
    fixed point) and returns device tensors X [N,16], T [N,3]."""
    import torch
    st = torch.cuda.current_stream()
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    xs, ts = [], []
    for w in workloads:
        lat = binding.Lattice(w.shape, w.tau, storage=storage, warm="previous", ibm_tol=tol,
                              ibm_max_iter=max_iter, stream=st, solver=solver)
        lat.set_propellers(w.props)
        lat.set_features(True)
        n = w.props.n_points
        X = torch.empty((n, 16), dtype=torch.float32, device="cuda")
        T = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        for s in range(steps):
            lat.step(1, 0)
            if s < skip:  # the first steps start from nothing
                continue
            lat.mlp_sample_dev(X, T)
            k = min(samples_per_step, n)
            idx = torch.randperm(n, device="cuda", generator=g)[:k]
            xs.append(X[idx].clone())
            ts.append(T[idx].clone())
        lat.close()
    return torch.cat(xs), torch.cat(ts)


def train(X, T, epochs=20, batch=16384, lr=2e-3, seed=7, P0=None, log=None):
    """Adam on the mean 0.5 |MLP(x) - t|^2; returns (P cuda FP32, losses)."""
    import torch
    st = torch.cuda.current_stream()
    P = torch.tensor(init_params(seed) if P0 is None else P0, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    grad = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    packed = torch.empty(binding.mlp_packed_bytes(), dtype=torch.uint8, device="cuda")
    binding.mlp_pack_dev(P, packed, st)
    scratch = torch.empty(binding.mlp_grad_scratch_bytes(batch), dtype=torch.uint8, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    n = X.shape[0]
    step = 0
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        tot = 0.0
        nb = 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb, tb = X[idx].contiguous(), T[idx].contiguous()
            binding.mlp_loss_grad_dev(xb, tb, P, packed, grad, loss, scratch, st)
            step += 1
            binding.mlp_adam_dev(P, m, v, grad, step, lr=lr, packed=packed, stream=st)
            tot += float(loss.item()) if nb % 16 == 0 else 0.0
            nb += 1
        losses.append(tot / max(1, (nb + 15) // 16))
        if log:
            log("epoch %d loss %.4g" % (ep, losses[-1]))
    return P, losses
