"""The C-ABI library builds, loads without a GPU and exports every symbol
that include/lbmibm.h declares; host-side argument checks (no device work)."""
import ctypes

import numpy as np
import pytest

from paper_1904_02108_gb300 import binding


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    return binding.load()


def test_every_declared_function_is_exported(L):
    names = binding.header_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding declares a signature for each
    assert set(names) == set(binding._SIGS), set(names) ^ set(binding._SIGS)


def test_velocity_set_matches_oracle_table(L, orc):
    e, t = binding.velocity_set()
    e2, t2 = orc.velocity_set()
    assert np.array_equal(e, e2) and np.array_equal(t, t2)


def test_stage_names(L):
    assert binding.stage_names() == ["kinematics", "pairs", "brick_init", "point_update",
                                     "brick_spread", "collide_stream", "stats", "residual",
                                     "mlp", "collide_active"]


@pytest.mark.parametrize("dims,tau", [((0, 8, 8), 0.8), ((8, 8, 6), 0.8), ((8, 8, 8), 0.5),
                                      ((8, 8, 8), 0.3), ((8, 8, 8), float("nan")),
                                      ((-4, 8, 8), 0.8)])
def test_create_rejects_bad_arguments_before_touching_the_device(L, dims, tau):
    h = ctypes.c_void_p()
    r = L.lbm_create(dims[0], dims[1], dims[2], tau, ctypes.byref(h))
    assert r == binding.LBM_EINVAL
    assert not h.value
    assert L.lbm_last_error(None)


def test_null_handle_is_einval(L):
    assert L.lbm_step(None, 1, 5) == binding.LBM_EINVAL
    assert L.ibm_set_points(None, 0, None, None, None, None) == binding.LBM_EINVAL
    assert L.lbm_read_stats(None, None) == binding.LBM_EINVAL
    L.lbm_destroy(None)


def test_spread_scratch_size(L):
    assert L.ibm_spread_scratch_bytes(8, 8, 6, 10) == 0  # not a multiple of 4
    a = L.ibm_spread_scratch_bytes(32, 32, 32, 100)
    b = L.ibm_spread_scratch_bytes(32, 32, 32, 1000)
    assert 0 < a < b and a % 256 == 0
