"""Launch shapes and the autotuner: no result depends on the launch shape
(populations, point corrections and FP64 sums are bitwise equal under any
shape), and autotuning leaves the lattice exactly where it was."""
import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W

pytestmark = pytest.mark.gpu

OTHER = dict(collide_block=128, brick_blocks=152 * 8, point_block=512, moments_spb=1,
             sort_blocks=152 * 8, collide_staged=1, sort_blocks_ahead=1)
WIDE = dict(collide_block=256, brick_blocks=152 * 32, point_block=128, moments_spb=2,
            sort_blocks=152 * 64, sort_blocks_ahead=152 * 64)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _pair_lattice(gpu_lib, torch, **kw):
    w = W.propellers([(12.0, 20.0, 14.0), (34.0, 20.0, 30.0)], 8.0, 2.0, 0.04, [0.3, 1.9])
    lat = gpu_lib.Lattice((44, 40, 48), 0.7, stream=torch.cuda.current_stream(), **kw)
    lat.set_propellers(w)
    return lat


def _same(a, b):
    assert np.array_equal(a.populations(), b.populations())
    sa, sb = a.stats(), b.stats()
    assert sa["step"] == sb["step"]
    assert sa["mass"] == sb["mass"] and sa["momentum"] == sb["momentum"]
    assert np.array_equal(a.points()[2], b.points()[2])


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("shape", [OTHER, WIDE])
def test_results_do_not_depend_on_the_launch_shape(gpu_lib, torch_cuda, storage, shape):
    a = _pair_lattice(gpu_lib, torch_cuda, storage=storage, warm="previous")
    b = _pair_lattice(gpu_lib, torch_cuda, storage=storage, warm="previous")
    b.set_launch_shape(**shape)
    assert b.launch_shape() == {**a.launch_shape(), **shape}
    a.step(7, 5)
    b.step(7, 5)
    _same(a, b)
    for lat in (a, b):
        lat.close()


def test_autotune_leaves_the_lattice_unchanged(gpu_lib, torch_cuda):
    a = _pair_lattice(gpu_lib, torch_cuda, warm="previous")
    b = _pair_lattice(gpu_lib, torch_cuda, warm="previous")
    a.step(3, 5)
    b.step(3, 5)
    chosen = a.autotune(n_ibm_iter=5, steps_per_trial=2)
    assert a.launch_shape() == chosen
    assert chosen["collide_block"] in (128, 256)
    assert chosen["moments_spb"] in (1, 2, 4)
    assert chosen["collide_staged"] == 2  # (FP32 storage: not a candidate, the default kept)
    assert a.stats()["step"] == 3
    a.step(4, 5)
    b.step(4, 5)
    _same(a, b)
    for lat in (a, b):
        lat.close()


def test_launch_shape_rejects_values_out_of_range(gpu_lib, torch_cuda):
    lat = _pair_lattice(gpu_lib, torch_cuda)
    for bad in (dict(collide_block=512), dict(point_block=1024), dict(moments_spb=8),
                dict(brick_blocks=0), dict(sort_blocks=-1), dict(collide_staged=3),
                dict(sort_blocks_ahead=0)):
        with pytest.raises(gpu_lib.LbmError):
            lat.set_launch_shape(**bad)
    lat.close()


def test_batch_autotune_keeps_batch_equal_to_single_stepping(gpu_lib, torch_cuda):
    torch = torch_cuda
    specs = [W.single_propeller(7), W.single_propeller(8)]
    mk = lambda w: gpu_lib.Lattice(w.shape, w.tau, warm="previous",
                                   stream=torch.cuda.current_stream())
    single = [mk(w) for w in specs]
    batched = [mk(w) for w in specs]
    for lat, w in zip(single + batched, specs + specs):
        lat.set_propellers(w.props)
    for lat in single:
        lat.step(5, 5)
    batch = gpu_lib.Batch(batched)
    batch.step(2, 5)
    chosen = batch.autotune(n_ibm_iter=5, steps_per_trial=2)
    assert batch.launch_shape() == chosen
    batch.step(3, 5)
    for s, b in zip(single, batched):
        _same(s, b)
    batch.close()
    for lat in single + batched:
        lat.close()


def test_update_points_moves_the_points_without_a_reset(gpu_lib, torch_cuda):
    """ibm_update_points with the same positions changes nothing; with moved
    positions it matches a lattice given those positions by ibm_set_points
    (zero warm start, so the reset there makes no difference)."""
    import numpy as np
    torch = torch_cuda
    rng = W.SplitMix64(71)
    x0 = W.random_points(rng, 400, (32, 32, 32))
    x1 = x0 + 0.3 * W.random_array(rng, x0.shape)
    ut = 0.02 * W.random_array(rng, x0.shape)
    mk = lambda: gpu_lib.Lattice((32, 32, 32), 0.8, stream=torch.cuda.current_stream())
    a, b, c = mk(), mk(), mk()
    for lat in (a, b, c):
        lat.set_points(x0, ut)
        lat.step(3, 5)
    a.update_points(x0)  # unchanged positions
    for lat in (a, b, c):
        lat.step(2, 5)
    assert np.array_equal(a.populations(), b.populations())
    a.update_points(x1, ut)
    c.set_points(x1, ut)
    a.step(2, 5)
    c.step(2, 5)
    assert np.array_equal(a.populations(), c.populations())
    assert np.array_equal(a.points()[2], c.points()[2])
    with pytest.raises(gpu_lib.LbmError):
        a.update_points(x1[:10])
    for lat in (a, b, c):
        lat.close()
