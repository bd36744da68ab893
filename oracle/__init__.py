"""FP64 CPU oracle for the coupled D3Q19 BGK + multi-direct-forcing IBM step.

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct definition of the
method (Beny & Latt, arXiv:1904.02108, Sec. 2-3, Alg. 1-2) that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path; the arithmetic lives in ``orc.c`` and this module only marshals
numpy arrays into it.

Layouts: populations ``f[19, nz, ny, nx]``; Eulerian vectors ``U[3, nz, ny, nx]``;
Lagrangian vectors ``v[np, 3]``.  All float64.

Parity: every function here is pinned by the closed-form tests in
``tests/test_oracle_*.py`` (nothing is left unpinned).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

Q = 19


def build(force: bool = False) -> str:
    """Compile ``orc.c`` into ``liborc.so`` with gcc (portable flags only)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
           "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            d, i, l, p = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
            L.orc_velocity_set.argtypes = [p, p]
            L.orc_equilibrium.argtypes = [i, d, p]
            L.orc_equilibrium.restype = d
            L.orc_init_equilibrium.argtypes = [i, i, i, p, p, p]
            L.orc_moments.argtypes = [i, i, i, p, p, p]
            L.orc_collide.argtypes = [i, i, i, d, p, p, p, p]
            L.orc_stream.argtypes = [i, i, i, p, p]
            L.orc_delta.argtypes = [i, d]
            L.orc_delta.restype = d
            L.orc_interpolate.argtypes = [i, i, i, i, p, l, p, p]
            L.orc_spread.argtypes = [i, i, i, i, l, p, p, p]
            L.orc_kinematics.argtypes = [l, p, p, p, p, p, l, p, p]
            L.orc_ibm.argtypes = [i, i, i, i, p, l, p, p, p, i, d, i, i, p, p, p, p, p]
            L.orc_ibm.restype = i
            L.orc_ibm_cg.argtypes = [i, i, i, i, p, l, p, p, p, i, d, i, p, p, p, p, p, p]
            L.orc_ibm_cg.restype = i
            L.orc_sums.argtypes = [i, i, i, p, p]
            L.orc_step.argtypes = [i, i, i, d, i, p, p, l, p, p, p, i, d, i, i,
                                   p, p, p, p, p, p, p, p, i]
            L.orc_step.restype = i
            L.orc_mlp_nparam.restype = i
            L.orc_mlp_forward.argtypes = [l, p, p, p]
            L.orc_mlp_loss_grad.argtypes = [l, p, p, p, p]
            L.orc_mlp_loss_grad.restype = d
            L.orc_mlp_features.argtypes = [i, i, i, i, p, l, p, p, p, p, i, p, p, d, d, p]
            L.orc_learned_init.argtypes = [l, p, p, p, d, p]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


KERNELS = {"cosine": 0, "peskin": 1}


def velocity_set():
    e = np.zeros((Q, 3), dtype=np.int32)
    t = np.zeros(Q, dtype=np.float64)
    lib().orc_velocity_set(_p(e), _p(t))
    return e, t


def equilibrium(i, rho, U):
    U = _f64(U, (3,))
    return lib().orc_equilibrium(int(i), float(rho), _p(U))


def init_equilibrium(shape, rho=None, U=None):
    nz, ny, nx = shape
    f = np.zeros((Q, nz, ny, nx))
    r = None if rho is None else _f64(rho, (nz, ny, nx))
    u = None if U is None else _f64(U, (3, nz, ny, nx))
    lib().orc_init_equilibrium(nx, ny, nz, _p(r), _p(u), _p(f))
    return f


def moments(f):
    f = _f64(f)
    _, nz, ny, nx = f.shape
    rho = np.zeros((nz, ny, nx))
    U = np.zeros((3, nz, ny, nx))
    lib().orc_moments(nx, ny, nz, _p(f), _p(rho), _p(U))
    return rho, U


def collide(f, tau, rho, U, G=None):
    """Returns a collided copy of ``f``."""
    f = _f64(f).copy()
    _, nz, ny, nx = f.shape
    lib().orc_collide(nx, ny, nz, float(tau), _p(f), _p(_f64(rho)), _p(_f64(U)),
                      _p(None if G is None else _f64(G)))
    return f


def stream(f):
    f = _f64(f)
    out = np.empty_like(f)
    _, nz, ny, nx = f.shape
    lib().orc_stream(nx, ny, nz, _p(f), _p(out))
    return out


def delta(r, kernel="cosine"):
    k = KERNELS[kernel]
    L = lib()
    return np.vectorize(lambda a: L.orc_delta(k, float(a)))(np.asarray(r, dtype=np.float64))


def interpolate(U, x, kernel="cosine"):
    U = _f64(U)
    _, nz, ny, nx = U.shape
    x = _f64(x).reshape(-1, 3)
    u = np.zeros_like(x)
    lib().orc_interpolate(nx, ny, nz, KERNELS[kernel], _p(U), len(x), _p(x), _p(u))
    return u


def spread(shape, x, v, kernel="cosine"):
    nz, ny, nx = shape
    x = _f64(x).reshape(-1, 3)
    v = _f64(v).reshape(-1, 3)
    F = np.zeros((3, nz, ny, nx))
    lib().orc_spread(nx, ny, nz, KERNELS[kernel], len(x), _p(x), _p(v), _p(F))
    return F


def kinematics(xrest, body, centre, omega, phase, t):
    xrest = _f64(xrest).reshape(-1, 3)
    body = np.ascontiguousarray(body, dtype=np.int32)
    x = np.zeros_like(xrest)
    ut = np.zeros_like(xrest)
    lib().orc_kinematics(len(xrest), _p(xrest), _p(body), _p(_f64(centre).reshape(-1, 3)),
                         _p(_f64(omega)), _p(_f64(phase)), int(t), _p(x), _p(ut))
    return x, ut


def ibm(U0, x, ut, s, n_iter=5, tol=1e-4, max_iter=500, literal=False,
        du_init=None, kernel="cosine"):
    """Multi-direct forcing (Sec. 3).  Returns (G, du, eps, eps_pt)."""
    U0 = _f64(U0)
    _, nz, ny, nx = U0.shape
    x = _f64(x).reshape(-1, 3)
    ut = _f64(ut).reshape(-1, 3)
    s = _f64(s).reshape(-1)
    n = len(x)
    du = np.zeros((n, 3))
    G = np.zeros_like(U0)
    cap = n_iter if n_iter > 0 else max_iter
    eps = np.zeros(cap)
    eps_pt = np.zeros(cap)
    di = None if du_init is None else _f64(du_init).reshape(-1, 3)
    it = lib().orc_ibm(nx, ny, nz, KERNELS[kernel], _p(U0), n, _p(x), _p(ut), _p(s),
                       int(n_iter), float(tol), int(max_iter), int(bool(literal)),
                       _p(di), _p(du), _p(G), _p(eps), _p(eps_pt))
    return G, du, eps[:it], eps_pt[:it]


def ibm_cg(U0, x, ut, s, n_iter=5, tol=1e-4, max_iter=500, du_init=None,
           kernel="cosine"):
    """Conjugate gradients on the lattice form B G = c of the fixed point of
    Sec. 3 (not in the paper; orc_ibm_cg).  Returns (G, du, eps, eps_pt,
    u_interp)."""
    U0 = _f64(U0)
    _, nz, ny, nx = U0.shape
    x = _f64(x).reshape(-1, 3)
    ut = _f64(ut).reshape(-1, 3)
    s = _f64(s).reshape(-1)
    n = len(x)
    du = np.zeros((n, 3))
    ui = np.zeros((n, 3))
    G = np.zeros_like(U0)
    cap = n_iter if n_iter > 0 else max_iter
    eps = np.zeros(cap)
    eps_pt = np.zeros(cap)
    di = None if du_init is None else _f64(du_init).reshape(-1, 3)
    it = lib().orc_ibm_cg(nx, ny, nz, KERNELS[kernel], _p(U0), n, _p(x), _p(ut), _p(s),
                          int(n_iter), float(tol), int(max_iter), _p(di), _p(du), _p(G),
                          _p(eps), _p(eps_pt), _p(ui))
    return G, du, eps[:it], eps_pt[:it], ui


SOLVERS = {"mdf": 0, "cg": 1}


def sums(f):
    f = _f64(f)
    _, nz, ny, nx = f.shape
    out = np.zeros(4)
    lib().orc_sums(nx, ny, nz, _p(f), _p(out))
    return out


def mlp_nparam():
    return lib().orc_mlp_nparam()


def mlp_forward(P, x):
    """Per-point MLP y = W3 s(W2 s(W1 x + b1) + b2) + b3 (SiLU), FP64."""
    P = _f64(P).reshape(-1)
    x = _f64(x).reshape(-1, 16)
    y = np.zeros((len(x), 3))
    lib().orc_mlp_forward(len(x), _p(P), _p(x), _p(y))
    return y


def mlp_loss_grad(P, x, t):
    """Mean 0.5 |y - t|^2 over the samples and its gradient in P, FP64."""
    P = _f64(P).reshape(-1)
    x = _f64(x).reshape(-1, 16)
    t = _f64(t).reshape(-1, 3)
    g = np.zeros_like(P)
    loss = lib().orc_mlp_loss_grad(len(x), _p(P), _p(x), _p(t), _p(g))
    return loss, g


# Feature scaling of the learned warm start (the values the library's C ABI
# documents for its feature layout): velocities in units of VSCALE, lengths in
# units of LSCALE.
VSCALE = 0.05
LSCALE = 16.0


def mlp_features(U0, x, ut, du_prev=None, body=None, centre=None, omega=None,
                 kernel="cosine", vscale=VSCALE, lscale=LSCALE):
    """The 16 per-point inputs of the learned warm start (orc_mlp_features):
    I[U0 + S[du_prev]], u_k, du_prev, the density of supports on the bricks
    the point's support touches, r and z about the body's axis, |omega| r and
    the slip u_k - I[U0 + S[du_prev]]; velocities / vscale, lengths / lscale.
    Returns [np, 16]."""
    U0 = _f64(U0)
    _, nz, ny, nx = U0.shape
    x = _f64(x).reshape(-1, 3)
    ut = _f64(ut).reshape(-1, 3)
    n = len(x)
    dp = None if du_prev is None else _f64(du_prev).reshape(-1, 3)
    nb = 0 if centre is None else len(_f64(centre).reshape(-1, 3))
    b = None if body is None else np.ascontiguousarray(body, dtype=np.int32)
    c = None if centre is None else _f64(centre).reshape(-1, 3)
    om = None if omega is None else _f64(omega).reshape(-1)
    feat = np.zeros((n, 16))
    lib().orc_mlp_features(nx, ny, nz, KERNELS[kernel], _p(U0), n, _p(x), _p(ut), _p(dp),
                           _p(b), nb, _p(c), _p(om), float(vscale), float(lscale),
                           _p(feat))
    return feat


def learned_init(P, feat, du_prev=None, vscale=VSCALE):
    """du_init = du_prev + vscale * MLP(feat) (orc_learned_init)."""
    P = _f64(P).reshape(-1)
    feat = _f64(feat).reshape(-1, 16)
    n = len(feat)
    dp = None if du_prev is None else _f64(du_prev).reshape(-1, 3)
    out = np.zeros((n, 3))
    lib().orc_learned_init(n, _p(P), _p(feat), _p(dp), float(vscale), _p(out))
    return out


class Simulation:
    """The coupled step of Sec. 2 driven over time on the CPU, in FP64.

    ``points`` (optional) is a dict with ``xrest`` [np,3], ``area`` [np],
    ``body`` [np] and per-body ``centre`` [nb,3], ``omega`` [nb], ``phase`` [nb]
    (rigid rotation about z, Alg. 1), or ``x`` [np,3] and ``ut`` [np,3] for
    fixed points with a prescribed surface velocity.  ``solver`` is "mdf"
    (the multi-direct-forcing loop of Sec. 3) or "cg" (conjugate gradients
    on the same fixed point, ``ibm_cg``).  ``warm`` is the initial guess of
    each step's fixed point: "zero" (the paper), "previous" (the previous
    step's final du) or "mlp" (the learned start du_prev + V MLP(features)
    with the FP64 parameter vector ``mlp``; the features of the last step
    are kept in ``features`` and its initial guess in ``du_init``).
    """

    def __init__(self, shape, tau, points=None, kernel="cosine", n_iter=5,
                 tol=1e-4, max_iter=500, literal=False, warm="zero",
                 gbody=None, solver="mdf", mlp=None):
        self.shape = tuple(shape)
        self.tau = float(tau)
        self.kernel = kernel
        self.n_iter = int(n_iter)
        self.tol = float(tol)
        self.max_iter = int(max_iter)
        self.literal = bool(literal)
        self.warm = warm
        if warm == "mlp" and mlp is None:
            raise ValueError("warm='mlp' needs the MLP parameters")
        self.mlp = None if mlp is None else _f64(mlp).reshape(-1)
        self.features = None
        self.du_init = None
        self.solver = SOLVERS[solver]
        self.gbody = None if gbody is None else _f64(gbody, (3,))
        nz, ny, nx = self.shape
        self.f = init_equilibrium(self.shape)
        self.ftmp = np.empty_like(self.f)
        self.t = 0
        self.points = points
        self.np = 0
        self.area = np.zeros(0)
        if points is not None:
            if "xrest" in points:
                self.np = len(points["xrest"])
            else:
                self.np = len(points["x"])
            self.area = _f64(points.get("area", np.ones(self.np))).reshape(-1)
        self.du = np.zeros((self.np, 3))
        self.rho = np.zeros(self.shape)
        self.U0 = np.zeros((3,) + self.shape)
        self.G = np.zeros((3,) + self.shape)
        self.iters = []
        self.eps = []
        self.eps_pt = []

    def positions(self, t=None):
        t = self.t if t is None else t
        P = self.points
        if "xrest" in P:
            return kinematics(P["xrest"], P["body"], P["centre"], P["omega"], P["phase"], t)
        return _f64(P["x"]).reshape(-1, 3), _f64(P["ut"]).reshape(-1, 3)

    def step(self, n=1):
        L = lib()
        nz, ny, nx = self.shape
        for _ in range(n):
            if self.np:
                x, ut = self.positions()
            else:
                x = ut = np.zeros((0, 3))
            cap = self.n_iter if self.n_iter > 0 else self.max_iter
            eps = np.zeros(max(cap, 1))
            eps_pt = np.zeros(max(cap, 1))
            du_init = None
            if self.warm == "previous" and self.t > 0:
                du_init = self.du.copy()
            elif self.warm == "mlp" and self.np:
                du_prev = self.du.copy() if self.t > 0 else None
                _, U0 = moments(self.f)
                P = self.points
                rigid = "xrest" in P
                self.features = mlp_features(
                    U0, x, ut, du_prev, body=P["body"] if rigid else None,
                    centre=P["centre"] if rigid else None,
                    omega=P["omega"] if rigid else None, kernel=self.kernel)
                du_init = learned_init(self.mlp, self.features, du_prev)
                self.du_init = du_init.copy()
            du = np.zeros((self.np, 3))
            it = L.orc_step(nx, ny, nz, self.tau, KERNELS[self.kernel], _p(self.f),
                            _p(self.ftmp), self.np, _p(_f64(x)), _p(_f64(ut)),
                            _p(self.area), self.n_iter, self.tol, self.max_iter,
                            int(self.literal), _p(du_init), _p(du), _p(self.gbody),
                            _p(self.rho), _p(self.U0), _p(self.G), _p(eps), _p(eps_pt),
                            self.solver)
            self.du = du
            self.iters.append(it)
            self.eps.append(eps[:it].copy())
            self.eps_pt.append(eps_pt[:it].copy())
            self.t += 1
        return self

    def fields(self):
        """rho, U of the current populations (Eq. 1)."""
        return moments(self.f)

    def sums(self):
        return sums(self.f)
