"""Seeded synthetic workloads: rotating four-blade propellers in periodic boxes.

This module only draws inputs; it holds none of the method's arithmetic (no
kinematics, no delta kernel, no lattice update).  Both the CUDA library's tests
and the FP64 oracle consume what it returns.

The paper's propeller is a Blender mesh of 3930 points (Sec. 6) that is not
available, so a synthetic propeller stands in for it: four flat rectangular
blades, each a plate spanned by the radial direction (r in [1, 1 + L]) and the
rotation axis z (|z - z_c| <= W/2), sampled on a regular grid with spacing
close to 0.7 lattice units, edges included.  Blade b of a body lies at angle
b*pi/2 in the rest pose; the body's rotation phi(t) = phase + omega*t about z
through its centre is applied by the solver.  Each point carries the area
s = (L/(n_r-1)) * (W/(n_w-1)) of the plate patch it represents.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014) seeded with
1234 + workload index; uniform doubles take the top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SPACING = 0.7
HUB = 1.0
_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64: state += 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, n: int) -> int:
        return int(self.uniform() * n) % n


@dataclass
class Propellers:
    """Lagrangian points of a set of rigid propellers (rest pose) + bodies."""
    xrest: np.ndarray           # [np, 3] float64, rest pose (angle 0)
    area: np.ndarray            # [np] float64, s(k)
    body: np.ndarray            # [np] int32
    centre: np.ndarray          # [nb, 3] float64
    omega: np.ndarray           # [nb] float64, rad per time step about +z
    phase: np.ndarray           # [nb] float64, angle at t = 0
    blade_length: float = 0.0
    blade_width: float = 0.0

    @property
    def n_points(self) -> int:
        return int(self.xrest.shape[0])

    @property
    def n_bodies(self) -> int:
        return int(self.centre.shape[0])

    def as_dict(self):
        return dict(xrest=self.xrest, area=self.area, body=self.body,
                    centre=self.centre, omega=self.omega, phase=self.phase)


def blade_grid(L: float, W: float):
    n_r = int(round(L / SPACING)) + 1
    n_w = int(round(W / SPACING)) + 1
    return n_r, n_w


def propellers(centres, L, W, v_tip, phase):
    """Rest-pose points of one four-blade propeller per centre."""
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    nb = len(centres)
    v_tip = np.broadcast_to(np.asarray(v_tip, dtype=np.float64), (nb,))
    phase = np.broadcast_to(np.asarray(phase, dtype=np.float64), (nb,))
    n_r, n_w = blade_grid(L, W)
    r = HUB + np.linspace(0.0, L, n_r)
    w = np.linspace(-W / 2.0, W / 2.0, n_w)
    s = (L / (n_r - 1)) * (W / (n_w - 1))
    pts, bod = [], []
    for b in range(nb):
        c = centres[b]
        for blade in range(4):
            a = blade * math.pi / 2.0
            ca, sa = math.cos(a), math.sin(a)
            for ri in r:
                for wi in w:
                    pts.append((c[0] + ri * ca, c[1] + ri * sa, c[2] + wi))
                    bod.append(b)
    R = HUB + L
    xrest = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    return Propellers(
        xrest=xrest,
        area=np.full(len(xrest), s, dtype=np.float64),
        body=np.asarray(bod, dtype=np.int32),
        centre=centres.copy(),
        omega=np.asarray(v_tip / R, dtype=np.float64).copy(),
        phase=np.asarray(phase, dtype=np.float64).copy(),
        blade_length=float(L), blade_width=float(W))


@dataclass
class Workload:
    name: str
    shape: tuple                # (nz, ny, nx)
    tau: float
    props: Propellers
    n_iter: int = 5
    steps: int = 100
    extra: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        nz, ny, nx = self.shape
        return nz * ny * nx


def single_propeller(seed_index: int = 0) -> Workload:
    """32^3 periodic box, tau 0.8, one propeller at the centre: blades 12 x 3,
    tip speed 0.05, seeded initial angle; 5 iterations, 100 steps."""
    rng = SplitMix64(1234 + seed_index)
    phase = rng.uniform(0.0, 2.0 * math.pi)
    p = propellers([(16.0, 16.0, 16.0)], 12.0, 3.0, 0.05, phase)
    return Workload("single_propeller_32", (32, 32, 32), 0.8, p, 5, 100)


def propeller_array(n_side: int, box: int, L: float, W: float, pitch: float,
                    seed: int, tau: float = 0.6):
    rng = SplitMix64(seed)
    centres, vt, ph = [], [], []
    for k in range(n_side):
        for j in range(n_side):
            for i in range(n_side):
                centres.append((pitch / 2 + pitch * i, pitch / 2 + pitch * j,
                                pitch / 2 + pitch * k))
    for _ in centres:
        vt.append(rng.uniform(0.02, 0.06))
        ph.append(rng.uniform(0.0, 2.0 * math.pi))
    return propellers(centres, L, W, np.asarray(vt), np.asarray(ph))


def dense_array_256(seed: int = 1235) -> Workload:
    """256^3, tau 0.6: 4x4x4 propellers (centres 32 + 64 i), blades 24 x 6,
    tip speed U[0.02, 0.06], phase U[0, 2pi); 5 iterations, 1000 steps.
    Other seeds give the same geometry with fresh speeds and phases."""
    p = propeller_array(4, 256, 24.0, 6.0, 64.0, seed)
    return Workload("propeller_array_256", (256, 256, 256), 0.6, p, 5, 1000)


def dense_array_384() -> Workload:
    """384^3, tau 0.6: 6x6x6 propellers of the 256^3 array's geometry."""
    p = propeller_array(6, 384, 24.0, 6.0, 64.0, 1236)
    return Workload("propeller_array_384", (384, 384, 384), 0.6, p, 5, 1000)


def dense_array_64() -> Workload:
    """64^3 downscale of the 384^3 array: 6x6x6 centres at pitch 64/6, blade
    lengths scaled by 1/6 (4 x 1), point spacing kept at 0.7."""
    p = propeller_array(6, 64, 4.0, 1.0, 64.0 / 6.0, 1236)
    return Workload("propeller_array_64", (64, 64, 64), 0.6, p, 5, 100)


# slots of the paper-shaped sweep: z layers from the middle outward, four
# (x, y) positions per layer
_SWEEP_LAYERS = (160.0, 96.0, 224.0, 32.0, 288.0)
_SWEEP_XY = ((40.0, 40.0), (120.0, 120.0), (120.0, 40.0), (40.0, 120.0))


def paper_sweep(n_props: int, seed: int = 1240) -> Workload:
    """The shape of the paper's benchmark (Sec. 6): a 160 x 160 x 320 lattice
    with 1 to 6 or 18 rotating propellers of ~3.9k points each (the paper's
    Blender propeller has 3930; 18 of them 70,740).  Here blades 30 x 15 at the
    0.7 spacing: 3872 points per propeller (69,696 for 18), tip radius 31;
    propeller i in slot i (z layers 64 apart from the middle outward, four
    (x, y) positions 80 apart per layer, no overlapping supports); tip speed
    U[0.02, 0.06], phase U[0, 2pi); tau 0.6, 5 iterations."""
    if not 1 <= n_props <= len(_SWEEP_LAYERS) * len(_SWEEP_XY):
        raise ValueError("1 to 20 propellers")
    rng = SplitMix64(seed)
    centres, vt, ph = [], [], []
    for i in range(n_props):
        x, y = _SWEEP_XY[i % 4]
        centres.append((x, y, _SWEEP_LAYERS[i // 4]))
        vt.append(rng.uniform(0.02, 0.06))
        ph.append(rng.uniform(0.0, 2.0 * math.pi))
    p = propellers(centres, 30.0, 15.0, np.asarray(vt), np.asarray(ph))
    return Workload("paper_sweep_%d" % n_props, (320, 160, 160), 0.6, p, 5, 1000)


def batched_domains(n_domains: int = 48, seed: int = 1238, max_tries: int = 1000):
    """Independent periodic cubes of side U{48,64,80,96}, each with 1-8
    propellers of the 32^3 box's geometry at seeded positions; tip speeds
    U[0.02, 0.06].  Propellers are placed by rejection sampling so that no two
    supports overlap (xy distance >= 2R + 4 or |dz| >= W + 4); one that cannot
    be placed in max_tries draws is dropped (the count is reported)."""
    rng = SplitMix64(seed)
    L, W = 12.0, 3.0
    R = HUB + L
    out, dropped = [], 0
    for d in range(n_domains):
        n = (48, 64, 80, 96)[rng.randint(4)]
        want = 1 + rng.randint(8)
        centres, vt, ph = [], [], []
        for _ in range(want):
            placed = False
            for _t in range(max_tries):
                # the propeller and its support stay inside the box (no wrap)
                c = (rng.uniform(R + 3, n - R - 3), rng.uniform(R + 3, n - R - 3),
                     rng.uniform(W / 2 + 3, n - W / 2 - 3))
                ok = True
                for o in centres:
                    dxy = math.hypot(c[0] - o[0], c[1] - o[1])
                    if dxy < 2 * R + 4 and abs(c[2] - o[2]) < W + 4:
                        ok = False
                        break
                if ok:
                    centres.append(c)
                    vt.append(rng.uniform(0.02, 0.06))
                    ph.append(rng.uniform(0.0, 2.0 * math.pi))
                    placed = True
                    break
            if not placed:
                dropped += 1
        p = propellers(centres, L, W, np.asarray(vt), np.asarray(ph))
        out.append(Workload("batched_%d" % d, (n, n, n), 0.8, p, 5, 500))
    return out, dropped


def random_points(rng: SplitMix64, n: int, shape, margin: float = 0.0):
    """n uniform points inside the periodic box (float64 [n,3], x fastest)."""
    nz, ny, nx = shape
    pts = np.empty((n, 3))
    for k in range(n):
        pts[k] = (rng.uniform(margin, nx - margin), rng.uniform(margin, ny - margin),
                  rng.uniform(margin, nz - margin))
    return pts


def random_array(rng: SplitMix64, shape, lo=-1.0, hi=1.0):
    """Seeded uniform array (float64) of the given shape, C order."""
    n = int(np.prod(shape))
    # draw in bulk: splitmix64 vectorised over a counter (same sequence as
    # repeated next_u64 calls)
    base = np.uint64(rng.state)
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = base + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    rng.state = (int(base) + n * 0x9E3779B97F4A7C15) & _MASK
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return (lo + (hi - lo) * u).reshape(shape)
