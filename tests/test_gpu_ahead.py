"""Steps prepared ahead against steps taken one call at a time.

Within one lbm_step call of several eager steps, the library builds the
next step's kinematics and pair lists while the current step collides (a
second stream and a second brick map).  That changes when work runs, not
what it computes, so a call of n steps must leave bitwise the same
populations, point values, FP64 sums, forces and step counter as n calls of
one step (which never prepare ahead), for every solver, warm start, U0
strategy, storage and iteration mode, and the same kernel count.
"""
import numpy as np
import pytest

from paper_1904_02108_gb300 import learned, workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _pair(gpu_lib, torch_cuda, w, setup, **kw):
    st = torch_cuda.cuda.current_stream()
    lats = []
    for _ in range(2):
        lat = gpu_lib.Lattice(w.shape, w.tau, stream=st, **kw)
        setup(lat)
        lats.append(lat)
    return lats


def _same(a, b):
    assert np.array_equal(a.populations(), b.populations())
    pa, pb = a.points(), b.points()
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y)
    _, _, Ga = a.fields()
    _, _, Gb = b.fields()
    assert np.array_equal(Ga, Gb)
    sa, sb = a.stats(), b.stats()
    for k in ("mass", "momentum", "step", "kernel_launches", "last_ibm_iters", "active_bricks"):
        assert sa[k] == sb[k], k


CASES = {
    "array64_loop": dict(kw=dict(warm="previous"), n_iter=5),
    "array64_zero_start": dict(kw=dict(warm="zero"), n_iter=5),
    "array64_cg": dict(kw=dict(warm="previous", solver="cg"), n_iter=5),
    "array64_bf16": dict(kw=dict(warm="previous", storage="bf16"), n_iter=5),
    "array64_f16_box": dict(kw=dict(warm="previous", storage="f16"), n_iter=5, u0="box"),
    "array64_kernel_u0": dict(kw=dict(warm="previous"), n_iter=5, u0="kernel"),
    "array64_tolerance": dict(kw=dict(warm="previous", ibm_tol=1e-3, ibm_max_iter=400),
                              n_iter=0),
    "array64_cg_tolerance": dict(kw=dict(warm="previous", solver="cg", ibm_tol=1e-4,
                                         ibm_max_iter=400), n_iter=0),
    "array64_learned": dict(kw=dict(warm="mlp"), n_iter=5, mlp=True),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_one_call_of_n_steps_is_n_calls_of_one(gpu_lib, torch_cuda, case):
    cfg = CASES[case]
    w = W.dense_array_64()

    def setup(lat):
        lat.set_propellers(w.props)
        if cfg.get("u0"):
            lat.set_u0_strategy(cfg["u0"])
        if cfg.get("mlp"):
            lat.set_mlp_weights(learned.init_params(315).astype(np.float32))

    a, b = _pair(gpu_lib, torch_cuda, w, setup, **cfg["kw"])
    a.step(6, cfg["n_iter"])
    for _ in range(6):
        b.step(1, cfg["n_iter"])
    _same(a, b)
    # a second call starts from the first call's last step
    a.step(3, cfg["n_iter"])
    for _ in range(3):
        b.step(1, cfg["n_iter"])
    _same(a, b)
    a.close()
    b.close()


def test_points_moved_between_calls(gpu_lib, torch_cuda):
    """Points without bodies, moved by the caller between calls (each call's
    first step reads the new positions; the steps after it are prepared
    ahead) and with targets: bitwise the single-step sequence."""
    rng = W.SplitMix64(77)
    shape = (32, 32, 32)
    X0 = W.random_points(rng, 900, shape, margin=2.0)
    U = 0.02 * W.random_array(rng, (900, 3))
    st = torch_cuda.cuda.current_stream()
    lats = [gpu_lib.Lattice(shape, 0.7, warm="previous", stream=st) for _ in range(2)]
    for lat in lats:
        lat.set_points(X0, U)
    a, b = lats
    for call in range(3):
        X = X0 + 0.37 * call
        a.update_points(X)
        b.update_points(X)
        a.step(4, 5)
        for _ in range(4):
            b.step(1, 5)
        _same(a, b)
    a.close()
    b.close()


@pytest.mark.parametrize("mode", ["fixed", "loop_to_tol", "cg_to_tol"])
def test_uploads_start_the_next_step(gpu_lib, torch_cuda, mode):
    """Mapped transfers, one step per call, the rest pose of rotating bodies
    uploaded from page-locked memory before every step (the next step's
    kinematics and pair lists then start at the upload, beside the step
    before it), with read-outs of fields, points and stats between the
    steps: bitwise the same as copies and blocking calls; with the fixed
    count, and iterating the paper's loop or conjugate gradients to a
    residual target."""
    torch = torch_cuda
    w = W.dense_array_64()
    st = torch.cuda.current_stream()
    kw = dict(warm="previous")
    n_iter = 5
    if mode != "fixed":
        kw.update(ibm_tol=1e-3, ibm_max_iter=400, solver="cg" if mode == "cg_to_tol" else "mdf")
        n_iter = 0
    a, b = (gpu_lib.Lattice(w.shape, w.tau, stream=st, **kw) for _ in range(2))
    for lat in (a, b):
        lat.set_propellers(w.props)
    a.set_host_io("mapped")
    X = torch.from_numpy(np.ascontiguousarray(w.props.xrest)).pin_memory().numpy()
    L = gpu_lib.load()
    for k in range(6):
        gpu_lib._check(L.ibm_update_points(a.h, len(X), gpu_lib._ptr(X), None), a.h)
        b.update_points(w.props.xrest)
        a.step(1, n_iter)
        b.step(1, n_iter)
        if k % 2:
            _same(a, b)
    _same(a, b)
    a.close()
    b.close()
