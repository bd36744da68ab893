"""The seeded input generators: propeller geometry and point counts."""
import math

import numpy as np
import pytest

from paper_1904_02108_gb300 import workload as W


def test_splitmix64_is_deterministic_and_bulk_matches_scalar():
    a = W.SplitMix64(99)
    xs = [a.uniform(-1, 1) for _ in range(17)]
    b = W.SplitMix64(99)
    ys = W.random_array(b, (17,))
    assert np.array_equal(np.array(xs), ys)
    assert a.state == b.state
    assert W.SplitMix64(1).next_u64() != W.SplitMix64(2).next_u64()


def test_point_counts_follow_the_blade_geometry():
    assert W.single_propeller().props.n_points == 4 * 18 * 5 == 360
    assert W.dense_array_256().props.n_points == 64 * 4 * 35 * 10 == 89600
    assert W.dense_array_384().props.n_points == 216 * 1400 == 302400


def test_single_propeller_geometry():
    w = W.single_propeller()
    p = w.props
    d = p.xrest - p.centre[0]
    r = np.hypot(d[:, 0], d[:, 1])
    assert abs(r.min() - 1.0) < 1e-12 and abs(r.max() - 13.0) < 1e-12
    assert abs(np.abs(d[:, 2]).max() - 1.5) < 1e-12
    assert np.allclose(p.area, (12 / 17) * (3 / 4))
    assert np.allclose(p.omega * 13.0, 0.05)
    assert 0 <= p.phase[0] < 2 * math.pi
    assert w.shape == (32, 32, 32) and w.tau == 0.8


def test_array_speeds_and_phases_in_range():
    p = W.dense_array_256().props
    vt = p.omega * 25.0
    assert vt.min() >= 0.02 and vt.max() <= 0.06
    assert p.phase.min() >= 0 and p.phase.max() < 2 * math.pi
    assert p.n_bodies == 64


def test_batched_domains_do_not_overlap():
    doms, dropped = W.batched_domains()
    assert len(doms) == 48
    for d in doms:
        n = d.shape[0]
        assert n in (48, 64, 80, 96)
        c = d.props.centre
        assert 1 <= len(c) <= 8
        for i in range(len(c)):
            for j in range(i):
                dxy = math.hypot(*(c[i, :2] - c[j, :2]))
                assert dxy >= 2 * 13 + 4 or abs(c[i, 2] - c[j, 2]) >= 3 + 4
        assert d.props.xrest.min() >= 2 and d.props.xrest.max() <= n - 2


def test_paper_sweep_shape_counts_and_separation():
    """The paper-shaped sweep: 160 x 160 x 320, 3872 points per propeller
    (4 blades of 44 x 22), 18 propellers 69,696 points; no two propellers'
    swept discs plus kernel supports meet, and every point stays inside the box."""
    for n in (1, 2, 3, 4, 5, 6, 18):
        w = W.paper_sweep(n)
        p = w.props
        assert w.shape == (320, 160, 160) and w.cells == 8_192_000
        assert p.n_bodies == n and p.n_points == n * 4 * 44 * 22
        c = p.centre
        for i in range(n):
            for j in range(i):
                dxy = math.hypot(*(c[i, :2] - c[j, :2]))
                assert dxy >= 2 * 31 + 4 or abs(c[i, 2] - c[j, 2]) >= 15 + 4
        lo, hi = p.xrest.min(axis=0), p.xrest.max(axis=0)
        assert np.all(lo >= 2) and np.all(hi <= np.array([160, 160, 320]) - 2)
        vt = p.omega * 31.0
        assert vt.min() >= 0.02 and vt.max() <= 0.06
    assert W.paper_sweep(18).props.n_points == 69696
    with pytest.raises(ValueError):
        W.paper_sweep(21)
