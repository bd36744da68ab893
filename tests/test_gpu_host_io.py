"""Mapped host transfers (lbm_set_host_io LBM_HOST_IO_MAPPED): uploads of
moved points read by the next step's kinematics straight from page-locked
host memory, and read-outs of du and the FP64 sums written by kernels into
it.  Every case runs a twin lattice with the default copies on the same
inputs and requires bitwise the same values at every step: an upload read by
the wrong step, or a read-out of the wrong step, changes the results, since
the points move every step."""
import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W

pytestmark = pytest.mark.gpu

SHAPE = (24, 20, 28)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _sheet():
    xs = np.array([(6.3 + 0.7 * i, 9.1, 5.2 + 0.7 * k) for i in range(12) for k in range(14)])
    ut = np.tile([0.02, 0.0, 0.0], (len(xs), 1))
    return xs, ut, np.full(len(xs), 0.49)


def _positions(xs, step):
    """The sheet moved by the caller: along x and, more slowly, along z."""
    return xs + np.array([0.37, 0.0, 0.11]) * step


def _targets(ut, step):
    return (ut * (1.0 + 0.25 * step)).astype(np.float32)


def _pin(torch, shape, dt):
    return torch.zeros(shape, dtype=dt).pin_memory().numpy()


def _pair(gpu_lib, torch):
    xs, ut, area = _sheet()
    out = []
    for _ in range(2):
        lat = gpu_lib.Lattice(SHAPE, 0.7, stream=torch.cuda.current_stream())
        lat.set_points(xs, ut, area)
        out.append(lat)
    out[0].set_host_io("mapped")
    assert out[0].host_io() == "mapped" and out[1].host_io() == "copy"
    return out, xs, ut


def _upload(gpu_lib, lat, X, U=None):
    L = gpu_lib.load()
    gpu_lib._check(L.ibm_update_points(lat.h, len(X), gpu_lib._ptr(X), gpu_lib._ptr(U)), lat.h)


@pytest.mark.parametrize("graph", [False, True])
def test_pipelined_steps_match_copies(gpu_lib, torch_cuda, graph):
    """The pipelined loop of an end-to-end user (upload step k's points and
    targets, enqueue the step and its read-outs, consume step k - 1's results
    while step k runs) against the default copies and blocking read-outs;
    with graphs, two steps per upload (the replayed steps take the upload by
    a copy)."""
    torch = torch_cuda
    (a, b), xs, ut = _pair(gpu_lib, torch)
    chunk = 2 if graph else 1
    if graph:
        a.set_graph(True)
        b.set_graph(True)
    steps = 8
    ref = []
    for k in range(steps):
        b.update_points(_positions(xs, k), _targets(ut, k))
        b.step(chunk, 5)
        s = b.stats()
        ref.append((b.points()[2], np.array([s["mass"]] + list(s["momentum"]))))
    n = a.np
    X = [_pin(torch, (n, 3), torch.float64) for _ in range(2)]
    U = [_pin(torch, (n, 3), torch.float32) for _ in range(2)]
    du = [_pin(torch, (n, 3), torch.float32) for _ in range(2)]
    sums = [_pin(torch, 4, torch.float64) for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    st = torch.cuda.current_stream()
    got = [None] * steps
    for k in range(steps):
        j = k % 2
        X[j][:] = _positions(xs, k)
        U[j][:] = _targets(ut, k)
        _upload(gpu_lib, a, X[j], U[j])
        a.step(chunk, 5)
        a.points_async(du=du[j])
        a.sums_async(sums[j])
        evs[j].record(st)
        if k > 0:
            evs[1 - j].synchronize()
            got[k - 1] = (du[1 - j].copy(), sums[1 - j].copy())
    evs[(steps - 1) % 2].synchronize()
    got[steps - 1] = (du[(steps - 1) % 2].copy(), sums[(steps - 1) % 2].copy())
    for k in range(steps):
        assert np.array_equal(got[k][0], ref[k][0]), k
        assert np.array_equal(got[k][1], ref[k][1]), k
    assert np.abs(ref[-1][0]).max() > 0
    for lat in (a, b):
        lat.close()


def test_upload_is_read_by_the_step(gpu_lib, torch_cuda):
    """The kinematics read a mapped upload when the step runs: a buffer
    changed after ibm_update_points (before lbm_step is called, with the
    device idle) gives the step of the changed values.  (The documented
    contract keeps the buffer unchanged; this checks that the mapped path,
    not a copy, was taken.)"""
    torch = torch_cuda
    (a, b), xs, _ = _pair(gpu_lib, torch)
    X = _pin(torch, (a.np, 3), torch.float64)
    X[:] = _positions(xs, 3)
    _upload(gpu_lib, a, X)
    torch.cuda.synchronize()
    X[:] = _positions(xs, 1)
    a.step(1, 5)
    b.update_points(_positions(xs, 1))
    b.step(1, 5)
    assert np.array_equal(a.points()[2], b.points()[2])
    for lat in (a, b):
        lat.close()


def test_pending_uploads_mode_switches_and_checkpoints(gpu_lib, torch_cuda):
    """Two uploads before a step (the last one counts, a target given only
    by the first still applies), a pageable upload after a mapped one,
    switching back to copies with an upload pending, a checkpoint taken with
    an upload pending, and a batch step with a pending upload."""
    torch = torch_cuda
    (a, b), xs, ut = _pair(gpu_lib, torch)
    n = a.np
    X1, X2 = _pin(torch, (n, 3), torch.float64), _pin(torch, (n, 3), torch.float64)
    U1 = _pin(torch, (n, 3), torch.float32)
    X1[:] = _positions(xs, 7)
    U1[:] = _targets(ut, 2)
    X2[:] = _positions(xs, 1)
    _upload(gpu_lib, a, X1, U1)
    _upload(gpu_lib, a, X2)
    b.update_points(_positions(xs, 1), _targets(ut, 2))
    a.step(1, 5)
    b.step(1, 5)
    assert np.array_equal(a.points()[2], b.points()[2])
    # a mapped upload, then a pageable one: the pageable one counts
    X1[:] = _positions(xs, 9)
    _upload(gpu_lib, a, X1)
    a.update_points(_positions(xs, 2))
    b.update_points(_positions(xs, 2))
    a.step(1, 5)
    b.step(1, 5)
    assert np.array_equal(a.deviations(), b.deviations())
    # switching to copies with an upload pending
    X1[:] = _positions(xs, 3)
    _upload(gpu_lib, a, X1)
    a.set_host_io("copy")
    b.update_points(_positions(xs, 3))
    a.step(1, 5)
    b.step(1, 5)
    assert np.array_equal(a.deviations(), b.deviations())
    # a checkpoint taken with an upload pending holds it
    a.set_host_io("mapped")
    X2[:] = _positions(xs, 4)
    _upload(gpu_lib, a, X2)
    b.update_points(_positions(xs, 4))
    blob = a.save_state()
    c = gpu_lib.Lattice(SHAPE, 0.7, stream=torch.cuda.current_stream())
    c.load_state(blob)
    for lat in (a, b, c):
        lat.step(1, 5)
    assert np.array_equal(a.deviations(), b.deviations())
    assert np.array_equal(c.deviations(), b.deviations())
    # a batch step with an upload pending
    w = W.single_propeller(16)
    other = gpu_lib.Lattice(w.shape, w.tau, stream=torch.cuda.current_stream())
    other.set_propellers(w.props)
    other.step(4, 5)  # (batched lattices share the step parity and warm-start history)
    batch = gpu_lib.Batch([a, other])
    for k in range(5, 8):
        X1[:] = _positions(xs, k)
        _upload(gpu_lib, a, X1)
        b.update_points(_positions(xs, k))
        batch.step(1, 5)
        b.step(1, 5)
        torch.cuda.synchronize()  # (X1 is rewritten next)
    assert np.array_equal(a.points()[2], b.points()[2])
    assert np.array_equal(a.deviations(), b.deviations())
    batch.close()
    for lat in (a, b, c, other):
        lat.close()


def test_read_outs_and_bad_arguments(gpu_lib, torch_cuda):
    """Mapped read-outs of positions, interpolated velocities, du and sums
    equal the blocking read-outs; pageable outputs fall back to copies; an
    unknown mode is refused."""
    torch = torch_cuda
    (a, b), xs, _ = _pair(gpu_lib, torch)
    for lat in (a, b):
        lat.update_points(_positions(xs, 1))
        lat.step(2, 5)
    n = a.np
    x, u, du = (_pin(torch, (n, 3), torch.float64), _pin(torch, (n, 3), torch.float32),
                _pin(torch, (n, 3), torch.float32))
    sums = _pin(torch, 4, torch.float64)
    a.points_async(x, u, du)
    a.sums_async(sums)
    du_pageable = np.zeros((n, 3), np.float32)
    a.points_async(du=du_pageable)
    torch.cuda.synchronize()
    xb, ub, dub = b.points()
    sb = b.stats()
    assert np.array_equal(x, xb) and np.array_equal(u, ub) and np.array_equal(du, dub)
    assert np.array_equal(du_pageable, dub)
    assert sums[0] == sb["mass"] and tuple(sums[1:]) == sb["momentum"]
    L = gpu_lib.load()
    assert L.lbm_set_host_io(a.h, 2) == gpu_lib.LBM_EINVAL
    assert a.host_io() == "mapped"
    assert L.lbm_set_host_io(None, 1) == gpu_lib.LBM_EINVAL
    for lat in (a, b):
        lat.close()
