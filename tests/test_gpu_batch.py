"""Captured steps (CUDA graphs) and batches of uneven lattices advanced by one
launch per stage: both must give bitwise the results of plain per-lattice
stepping, which the oracle parity tests pin."""
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


def _domains():
    """Three uneven domains: a propeller in 32^3, two in 48x40x44, and an
    empty 20x24x16 box with a body force."""
    a = W.single_propeller(3)
    b = W.propellers([(12.0, 20.0, 14.0), (34.0, 20.0, 30.0)], 8.0, 2.0, 0.04, [0.3, 1.9])
    return [(a.shape, 0.8, a.props, None), ((44, 40, 48), 0.7, b, None),
            ((16, 24, 20), 0.9, None, (1e-5, 0.0, 0.0))]


def _make(gpu_lib, torch, spec, **kw):
    shape, tau, props, gbody = spec
    lat = gpu_lib.Lattice(shape, tau, stream=torch.cuda.current_stream(), **kw)
    if props is not None:
        lat.set_propellers(props)
    if gbody is not None:
        lat.set_body_force(gbody)
    return lat


@pytest.mark.parametrize("warm", ["zero", "previous"])
def test_graph_replay_is_bitwise_eager(gpu_lib, torch_cuda, warm):
    torch = torch_cuda
    spec = _domains()[0]
    a = _make(gpu_lib, torch, spec, warm=warm)
    b = _make(gpu_lib, torch, spec, warm=warm)
    b.set_graph(True)
    a.step(11, 5)
    b.step(11, 5)  # one eager step, then five replayed pairs
    assert np.array_equal(a.populations(), b.populations())
    sa, sb = a.stats(), b.stats()
    assert sa["step"] == sb["step"] == 11 and sa["mass"] == sb["mass"]
    assert sb["kernel_launches"] == sa["kernel_launches"]
    for lat in (a, b):
        lat.close()


@pytest.mark.parametrize("graph", [False, True])
def test_batch_is_bitwise_per_lattice_stepping(gpu_lib, torch_cuda, graph):
    torch = torch_cuda
    specs = _domains()
    single = [_make(gpu_lib, torch, s, warm="previous") for s in specs]
    batched = [_make(gpu_lib, torch, s, warm="previous") for s in specs]
    for lat in single:
        lat.step(6, 5)
    batch = gpu_lib.Batch(batched)
    batch.set_graph(graph)
    batch.step(6, 5)
    for s, b in zip(single, batched):
        assert np.array_equal(s.populations(), b.populations())
        ss, sb = s.stats(), b.stats()
        assert ss["step"] == sb["step"] == 6
        assert ss["mass"] == sb["mass"] and ss["momentum"] == sb["momentum"]
        if s.np:
            assert np.array_equal(s.points()[2], b.points()[2])
    batch.close()
    for lat in single + batched:
        lat.close()


def test_batch_rejects_mismatched_handles(gpu_lib, torch_cuda):
    torch = torch_cuda
    specs = _domains()
    a = _make(gpu_lib, torch, specs[0])
    b = _make(gpu_lib, torch, specs[1], storage="bf16")
    with pytest.raises(gpu_lib.LbmError):
        gpu_lib.Batch([a, b])
    c = _make(gpu_lib, torch, specs[1], warm="previous")
    batch = gpu_lib.Batch([a, c])
    with pytest.raises(gpu_lib.LbmError):
        batch.step(1, 5)  # warm-start modes differ
    with pytest.raises(gpu_lib.LbmError):
        batch.step(1, 0)  # tolerance mode needs a single lattice
    batch.close()
    for lat in (a, b, c):
        lat.close()
