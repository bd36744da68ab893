"""Parity at the benchmark's full size and launch configuration: the 256^3
array of 64 propellers (89,600 points, 5 iterations per step), two steps from
rest, against the FP64 oracle on the whole lattice."""
import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_dense_array_256_two_steps(gpu_lib, orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.dense_array_256()
    lat = gpu_lib.Lattice(w.shape, w.tau, stream=torch.cuda.current_stream())
    lat.set_propellers(w.props)
    lat.step(2, w.n_iter)
    rho, U, G = lat.fields()
    _, _, du = lat.points()
    s = lat.stats()
    lat.close()
    sim = orc.Simulation(w.shape, w.tau, w.props.as_dict(), n_iter=w.n_iter)
    sim.step(2)
    rho_o, U_o = sim.fields()
    assert rel_l2(U, U_o) < 1e-5
    assert np.abs(rho - rho_o).max() < 5e-7
    assert rel_l2(G, sim.G) < 1e-5
    assert rel_l2(du, sim.du) < 1e-5
    assert abs(s["mass"] - w.cells) / w.cells < 1e-12
