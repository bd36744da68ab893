"""The split step (the cells outside the step's active bricks collide while
the IBM stages run; the active bricks' cells collide after the IBM loop)
against one collide over every cell after the loop.  Every cell's arithmetic
is the same, so the populations and the force agree bitwise; only the
grouping of the FP64 partial sums of mass and momentum differs."""
import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _pair(gpu_lib, torch, w, **kw):
    lats = []
    for on in (True, False):
        lat = gpu_lib.Lattice(w.shape, w.tau, stream=torch.cuda.current_stream(), **kw)
        lat.set_overlap(on)
        lat.set_propellers(w.props)
        lats.append(lat)
    return lats


def _same_sums(lat, sa, sb):
    """Both sums add each cell's FP32 terms in warps of 32 (then in FP64), the
    split step grouping the active bricks' cells differently: each warp sum
    is within 31 eps32 of its terms' absolute sum, so the two results are
    within 32 eps32 of the terms' absolute sum over the lattice."""
    eps = 2.0 ** -24
    rho, U, G = (np.asarray(a, np.float64) for a in lat.fields())
    tol_m = 32 * eps * np.abs(rho - 1).sum() + 1e-9
    assert abs(sa["mass"] - sb["mass"]) <= tol_m
    for c, (a, b) in enumerate(zip(sa["momentum"], sb["momentum"])):
        tol = 32 * eps * np.abs(rho * (U[c] + G[c])).sum() + 1e-12
        assert abs(a - b) <= tol


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_split_step_is_bitwise_single_collide(gpu_lib, torch_cuda, storage):
    w = W.single_propeller(1)
    a, b = _pair(gpu_lib, torch_cuda, w, storage=storage, warm="previous")
    a.step(9, 5)
    b.step(9, 5)
    assert np.array_equal(a.deviations(), b.deviations())
    ra, Ua, Ga = a.fields()
    rb, Ub, Gb = b.fields()
    assert np.array_equal(Ga, Gb) and np.array_equal(Ua, Ub)
    sa, sb = a.stats(), b.stats()
    assert sa["step"] == sb["step"] == 9 and sa["active_bricks"] == sb["active_bricks"] > 0
    _same_sums(a, sa, sb)
    assert sa["kernel_launches"] == sb["kernel_launches"] + 9  # the second collide
    for lat in (a, b):
        lat.close()


def test_split_step_many_propellers_and_body_force(gpu_lib, torch_cuda):
    # propellers close to the periodic boundary: active bricks wrap around
    props = W.propellers([(3.0, 30.0, 20.0), (28.0, 2.5, 30.0), (16.0, 16.0, 38.5)], 7.0, 2.0,
                         0.05, [0.0, 1.0, 2.0])
    w = W.Workload("wrap", (40, 36, 32), 0.7, props, 5)
    a, b = _pair(gpu_lib, torch_cuda, w)
    for lat in (a, b):
        lat.set_body_force((2e-6, -1e-6, 0.0))
        lat.step(7, 5)
    assert np.array_equal(a.deviations(), b.deviations())
    _same_sums(a, a.stats(), b.stats())
    for lat in (a, b):
        lat.close()


def test_split_step_in_captured_graphs(gpu_lib, torch_cuda):
    w = W.single_propeller(2)
    a, b = _pair(gpu_lib, torch_cuda, w, warm="previous")
    c = gpu_lib.Lattice(w.shape, w.tau, stream=torch_cuda.cuda.current_stream(),
                        warm="previous")
    c.set_propellers(w.props)
    c.set_overlap(True)
    c.set_graph(True)  # split inside the captures
    for lat in (a, b, c):
        lat.step(11, 5)
    assert np.array_equal(a.deviations(), c.deviations())
    assert np.array_equal(b.deviations(), c.deviations())
    assert a.stats()["mass"] == c.stats()["mass"]
    for lat in (a, b, c):
        lat.close()


def test_split_step_tolerance_mode(gpu_lib, torch_cuda):
    w = W.single_propeller(0)
    a, b = _pair(gpu_lib, torch_cuda, w, warm="previous", ibm_tol=1e-5, ibm_max_iter=300)
    for lat in (a, b):
        lat.step(4, 0)
    assert np.array_equal(a.deviations(), b.deviations())
    sa, sb = a.stats(), b.stats()
    assert sa["last_ibm_iters"] == sb["last_ibm_iters"] > 0
    assert sa["last_residual"] == sb["last_residual"]
    for lat in (a, b):
        lat.close()


def test_overlap_switch_mid_run(gpu_lib, torch_cuda):
    w = W.single_propeller(3)
    a, b = _pair(gpu_lib, torch_cuda, w, warm="previous")
    a.step(3, 5)
    b.step(3, 5)
    a.set_overlap(False)
    b.set_overlap(True)
    a.step(4, 5)
    b.step(4, 5)
    assert np.array_equal(a.deviations(), b.deviations())
    for lat in (a, b):
        lat.close()
