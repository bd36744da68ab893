"""ibm_spread_dev_noalloc: spreading for callers that cannot allocate device
memory (a host application whose pool owns the device, or a time-critical loop
that must not pay cudaMalloc's implicit synchronisation).  It must give the
same field as ibm_spread_dev, call after call, using only the library's static
scratch area.  This file is collected last on purpose."""
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


def _case(torch, shape, n, seed):
    rng = W.SplitMix64(seed)
    x = W.random_points(rng, n, shape)
    v = W.random_array(rng, (n, 3))
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    vd = torch.tensor(v, dtype=torch.float32, device="cuda")
    return xd, vd, np.abs(v).max() * 8


@pytest.mark.parametrize("kernel", ["cosine", "peskin"])
def test_noalloc_spread_matches_allocating_entry_point(gpu_lib, torch_cuda, kernel):
    """Both entry points run the same deterministic kernels on the same inputs
    (pairs sorted by point index, sums in a fixed order), so the fields must
    be bitwise equal; anything left in the shared static scratch by an earlier
    call that leaked into the result would break that.  The device's free
    memory must not change across a call (after the first call on the device,
    which may load the library's kernels)."""
    torch = torch_cuda
    st = torch.cuda.current_stream()
    # two calls in a row on different problems: the second must not see any
    # of the first call's leftovers in the shared static scratch
    for shape, n, seed in (((32, 32, 32), 3000, 51), ((16, 24, 20), 700, 52)):
        xd, vd, scale = _case(torch, shape, n, seed)
        ref = torch.full((3,) + shape, 3.0, dtype=torch.float32, device="cuda")
        scratch = torch.empty(gpu_lib.spread_scratch_bytes(shape, n), dtype=torch.uint8,
                              device="cuda")
        gpu_lib.spread_dev(xd, vd, ref, kernel, scratch, st)
        out = torch.full((3,) + shape, -5.0, dtype=torch.float32, device="cuda")
        gpu_lib.spread_dev_noalloc(xd, vd, out, kernel, st)  # warm: first use
        out.fill_(-5.0)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        gpu_lib.spread_dev_noalloc(xd, vd, out, kernel, st)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.equal(out, ref)
        assert ref.abs().max().item() > 0.1


def test_noalloc_rejects_problems_beyond_its_scratch(gpu_lib, torch_cuda):
    torch = torch_cuda
    shape, n = (128, 128, 128), 20000
    assert gpu_lib.spread_scratch_bytes(shape, n) > gpu_lib.NOALLOC_SCRATCH_BYTES
    xd = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    vd = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    F = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    with pytest.raises(gpu_lib.LbmError) as e:
        gpu_lib.spread_dev_noalloc(xd, vd, F, "cosine", torch.cuda.current_stream())
    assert e.value.code == gpu_lib.LBM_EINVAL
    assert "scratch" in str(e.value)
