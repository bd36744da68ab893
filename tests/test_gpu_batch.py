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
    # read-outs after replays (in a replayed pair the second step's pair
    # lists are built beside the first one's collide, into the brick map and
    # positions the read-outs use)
    for x, y in zip(a.points(), b.points()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.fields()[2], b.fields()[2])
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
            for x, y in zip(s.points(), b.points()):
                assert np.array_equal(x, y)
            assert np.array_equal(s.fields()[2], b.fields()[2])
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
    batch.close()
    # tolerance mode: the paper's loop only, one residual target for all
    d = _make(gpu_lib, torch, specs[0], warm="previous", solver="cg")
    e = _make(gpu_lib, torch, specs[1], warm="previous", solver="cg")
    batch = gpu_lib.Batch([d, e])
    with pytest.raises(gpu_lib.LbmError):
        batch.step(1, 0)
    batch.close()
    f = _make(gpu_lib, torch, specs[0], warm="previous", ibm_tol=1e-3)
    g = _make(gpu_lib, torch, specs[1], warm="previous", ibm_tol=2e-3)
    batch = gpu_lib.Batch([f, g])
    with pytest.raises(gpu_lib.LbmError):
        batch.step(1, 0)
    batch.close()
    for lat in (a, b, c, d, e, f, g):
        lat.close()


@pytest.mark.parametrize("warm,tol", [("previous", 2e-3), ("zero", 0.05)])
def test_batch_tolerance_mode_is_bitwise_per_lattice_stepping(gpu_lib, torch_cuda, warm, tol):
    """Every domain of a batch iterates the paper's loop to its own residual
    target (the domains need different counts): the same iteration counts,
    residual histories and bitwise the same states as each lattice stepped
    alone in tolerance mode; an empty domain and the cap warning included."""
    torch = torch_cuda
    specs = _domains()
    kw = dict(warm=warm, ibm_tol=tol, ibm_max_iter=3000)
    single = [_make(gpu_lib, torch, s, **kw) for s in specs]
    batched = [_make(gpu_lib, torch, s, **kw) for s in specs]
    batch = gpu_lib.Batch(batched)
    counts = []
    for _ in range(3):
        for lat in single:
            assert lat.step(1, 0) == gpu_lib.LBM_OK
        assert batch.step(1, 0) == gpu_lib.LBM_OK
        for s, b in zip(single, batched):
            assert s.stats()["last_ibm_iters"] == b.stats()["last_ibm_iters"]
            if s.np:
                assert np.array_equal(s.residuals(), b.residuals())
        counts.append([b.stats()["last_ibm_iters"] for b in batched if b.np])
    for s, b in zip(single, batched):
        assert np.array_equal(s.populations(), b.populations())
        assert s.stats()["mass"] == b.stats()["mass"]
        if s.np:
            assert np.array_equal(s.points()[2], b.points()[2])
    assert any(len(set(c)) > 1 for c in counts), counts  # the domains differ
    # a fixed-count batch step afterwards, and the cap
    assert batch.step(1, 5) == gpu_lib.LBM_OK
    batch.close()
    capped = [_make(gpu_lib, torch, s, warm=warm, ibm_tol=1e-12, ibm_max_iter=9)
              for s in specs]
    batch = gpu_lib.Batch(capped)
    assert batch.step(1, 0) == gpu_lib.LBM_WNOTCONVERGED
    assert [c.stats()["last_ibm_iters"] for c in capped if c.np] == [9, 9]
    batch.close()
    for lat in single + batched + capped:
        lat.close()
