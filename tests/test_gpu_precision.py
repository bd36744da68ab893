"""Reduced-precision population storage (BF16 / FP16 deviations f_i - t_i,
FP32 arithmetic) against the FP64 oracle on the 64^3 downscale of the 384^3
propeller array (216 propellers), and FP32 for reference.

The bound per format is its unit roundoff u (FP16: 2^-11, BF16: 2^-8) on
the relative L2 error of U after STEPS steps.  Each step rounds every stored
deviation once (relative error <= u), which moves U at a cell by at most
about u of its size; the errors do not pile up over the steps (the IBM force
re-imposes the surface velocity every step and the relaxation damps the
rest), and the measured error is about 0.3 u for both formats at 50 steps
(1.5e-4 FP16, 1.2e-3 BF16), so the bound u leaves a margin of ~3.  A lost
deviation form (storing f instead of f - t: the rounding then scales with
t_i, ~20 times the deviations) or a biased rounding that accumulates over
the steps breaks it.
"""
import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W

pytestmark = pytest.mark.gpu

STEPS = 50
# relative L2 bound on U after STEPS steps
BOUND = {"f32": 1e-5, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def oracle_run(orc):
    w = W.dense_array_64()
    sim = orc.Simulation(w.shape, w.tau, w.props.as_dict(), n_iter=w.n_iter)
    sim.step(STEPS)
    return w, sim.fields()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_storage_error_against_oracle(gpu_lib, orc, oracle_run, storage):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w, (rho_o, U_o) = oracle_run
    lat = gpu_lib.Lattice(w.shape, w.tau, storage=storage,
                          stream=torch.cuda.current_stream())
    lat.set_propellers(w.props)
    lat.step(STEPS, w.n_iter)
    rho, U, _ = lat.fields()
    err = rel_l2(U, U_o)
    print("storage %s: rel L2(U) after %d steps = %.3e (bound %.3e), max|rho err| = %.3e"
          % (storage, STEPS, err, BOUND[storage], np.abs(rho - rho_o).max()))
    assert err < BOUND[storage]
    s = lat.stats()
    assert abs(s["mass"] / w.cells - 1.0) < 1e-3
    lat.close()


LONG_STEPS = 200


@pytest.fixture(scope="module")
def oracle_long_run(orc):
    w = W.dense_array_64()
    sim = orc.Simulation(w.shape, w.tau, w.props.as_dict(), n_iter=w.n_iter)
    sim.step(LONG_STEPS)
    return w, sim.fields()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_storage_error_over_a_long_run(gpu_lib, orc, oracle_long_run, storage):
    """The same comparison over 200 steps: the error of the 16-bit forms
    stays within the unit roundoff (it does not accumulate with the steps);
    FP32 stays at its 1e-5 bar."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w, (rho_o, U_o) = oracle_long_run
    lat = gpu_lib.Lattice(w.shape, w.tau, storage=storage,
                          stream=torch.cuda.current_stream())
    lat.set_propellers(w.props)
    lat.step(LONG_STEPS, w.n_iter)
    _, U, _ = lat.fields()
    err = rel_l2(U, U_o)
    print("storage %s: rel L2(U) after %d steps = %.3e (bound %.3e)"
          % (storage, LONG_STEPS, err, BOUND[storage]))
    assert err < BOUND[storage]
    lat.close()


@pytest.mark.parametrize("storage,u", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_roundtrip_rounds_deviations_to_nearest(gpu_lib, orc, storage, u):
    """Stored deviations are f - t rounded to nearest in the 16-bit format:
    the read-back error is at most u |f - t| (plus the smallest subnormal)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    shape = (8, 8, 12)
    rng = W.SplitMix64(61)
    f = orc.init_equilibrium(shape, 1 + 0.02 * W.random_array(rng, shape),
                             0.05 * W.random_array(rng, (3,) + shape))
    t = orc.velocity_set()[1][:, None, None, None]
    lat = gpu_lib.Lattice(shape, 0.8, storage=storage, stream=torch.cuda.current_stream())
    lat.set_populations(f)
    d = lat.deviations().astype(np.float64)
    dev = (f - t).astype(np.float32).astype(np.float64)
    # FP16 subnormal spacing; the FP32 subtraction f - t on the device
    tiny = (6e-8 if storage == "f16" else 0.0) + 2.0 ** -24 * 0.34
    assert np.all(np.abs(d - dev) <= u * np.abs(dev) + tiny)
    lat.close()


@pytest.mark.parametrize("staged", [1, 2])
@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("case", ["single_propeller_32", "propeller_array_64", "box_48x64x80"])
def test_staged_collide_is_bitwise_the_two_cell_kernel(gpu_lib, orc, storage, case, staged):
    """A single lattice with 16-bit storage and the staged collide (1: rows of
    the pulls brought into shared memory by bulk copies) or the four-cell
    collide (2: two packed pairs per thread, 8-byte pulls and stores) chosen,
    against a batch, which keeps the two-cell kernel; all use the same
    per-cell arithmetic and the same partial sums, so populations and FP64
    sums must agree bitwise.  The shapes cover tiles of 16, 8 and 8 rows, the
    y and z seams and a lattice whose rows are not a power of two."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if case == "single_propeller_32":
        w = W.single_propeller(21)
        shape, props = w.shape, w.props
    elif case == "propeller_array_64":
        w = W.dense_array_64()
        shape, props = w.shape, w.props
    else:
        shape = (80, 64, 48)
        props = W.propellers([(20.0, 30.0, 40.0), (30.0, 12.0, 70.0)], 10.0, 3.0, 0.05,
                             [0.4, 2.2])
    st = torch.cuda.current_stream()
    a = gpu_lib.Lattice(shape, 0.7, storage=storage, warm="previous", stream=st)
    a.set_launch_shape(collide_staged=staged)
    b = gpu_lib.Lattice(shape, 0.7, storage=storage, warm="previous", stream=st)
    rng = W.SplitMix64(22)
    f0 = orc.init_equilibrium(shape, 1 + 0.01 * W.random_array(rng, shape),
                              0.02 * W.random_array(rng, (3,) + shape))
    for lat in (a, b):
        lat.set_propellers(props)
        lat.set_populations(f0)
    batch = gpu_lib.Batch([b])
    batch.set_launch_shape(collide_staged=0)
    for _ in range(3):
        a.step(1, 5)
        batch.step(1, 5)
    assert np.array_equal(a.deviations(), b.deviations())
    sa, sb = a.stats(), b.stats()
    assert sa["mass"] == sb["mass"] and sa["momentum"] == sb["momentum"]
    batch.close()
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_four_cell_batch_is_bitwise_single_two_cell_lattices(gpu_lib, orc, storage):
    """A batch of two uneven lattices (one whose cell count leaves the last
    128-cell partial half full) stepped by the four-cell collide against the
    same lattices stepped alone by the two-cell kernel: bitwise populations
    and FP64 sums."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    st = torch.cuda.current_stream()
    w = W.dense_array_64()
    specs = [((64, 64, 64), w.props), ((36, 20, 12), None)]
    rng = W.SplitMix64(23)
    singles, members = [], []
    for shape, props in specs:
        f0 = orc.init_equilibrium(shape, 1 + 0.01 * W.random_array(rng, shape),
                                  0.02 * W.random_array(rng, (3,) + shape))
        for group in (singles, members):
            lat = gpu_lib.Lattice(shape, 0.7, storage=storage, warm="previous", stream=st)
            lat.set_launch_shape(collide_staged=0)
            if props is not None:
                lat.set_propellers(props)
            else:
                lat.set_body_force((1e-5, -2e-5, 3e-5))
            lat.set_populations(f0)
            group.append(lat)
    batch = gpu_lib.Batch(members)
    batch.set_launch_shape(collide_staged=2)
    for _ in range(3):
        for lat in singles:
            lat.step(1, 5)
        batch.step(1, 5)
    for a, b in zip(singles, members):
        assert np.array_equal(a.deviations(), b.deviations())
        sa, sb = a.stats(), b.stats()
        assert sa["mass"] == sb["mass"] and sa["momentum"] == sb["momentum"]
    batch.close()
    for lat in singles + members:
        lat.close()
