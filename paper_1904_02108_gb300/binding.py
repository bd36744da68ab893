"""Python binding of the C ABI in include/lbmibm.h (argument marshalling only).

Every step of the method runs in the CUDA library ``liblbmibm.so``; this
module converts numpy arrays / torch tensors into pointers and status codes
into exceptions.  There is no CPU fallback: if the library is missing,
``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "liblbmibm.so")
HEADER = os.path.join(ROOT, "include", "lbmibm.h")

LBM_OK = 0
LBM_EINVAL = -1
LBM_ENOMEM = -2
LBM_ECUDA = -3
LBM_ENONFINITE = -4
LBM_ESTATE = -5
LBM_WNOTCONVERGED = 1

STORAGE = {"f32": 0, "bf16": 1, "f16": 2}
DELTA = {"cosine": 0, "peskin": 1}
WARM = {"zero": 0, "previous": 1, "mlp": 2}
HOST_IO = {"copy": 0, "mapped": 1}
MLP_NPARAM = 5443
MLP_VSCALE = 0.05
MLP_LSCALE = 16.0

_c = ctypes
_p = _c.c_void_p
_i = _c.c_int
_d = _c.c_double
_i64 = _c.c_int64


class LbmOpts(_c.Structure):
    _fields_ = [("nx", _i), ("ny", _i), ("nz", _i), ("tau", _d), ("storage", _i),
                ("delta", _i), ("warm_start", _i), ("ibm_tol", _d), ("ibm_max_iter", _i),
                ("stats", _i)]


class LbmStats(_c.Structure):
    _fields_ = [("mass", _d), ("momentum", _d * 3), ("step", _i64), ("last_ibm_iters", _i),
                ("last_residual", _d), ("not_converged", _i64), ("active_bricks", _i64),
                ("kernel_launches", _i64)]


class LaunchShape(_c.Structure):
    _fields_ = [("collide_block", _i), ("brick_blocks", _i), ("point_block", _i),
                ("moments_spb", _i), ("sort_blocks", _i), ("collide_staged", _i),
                ("sort_blocks_ahead", _i)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lbmibm error %d: %s" % (code, msg))
        self.code = code


_lib = None

_SIGS = {
    "lbm_default_opts": (None, [_p]),
    "lbm_create": (_i, [_i, _i, _i, _d, _p]),
    "lbm_create_ex": (_i, [_p, _p]),
    "lbm_destroy": (None, [_p]),
    "lbm_last_error": (_c.c_char_p, [_p]),
    "lbm_set_stream": (_i, [_p, _p]),
    "ibm_set_points": (_i, [_p, _i64, _p, _p, _p, _p]),
    "ibm_set_bodies": (_i, [_p, _i, _p, _p, _p]),
    "lbm_set_body_force": (_i, [_p, _d, _d, _d]),
    "lbm_step": (_i, [_p, _i, _i]),
    "lbm_time": (_i64, [_p]),
    "lbm_set_time": (_i, [_p, _i64]),
    "lbm_read_fields": (_i, [_p, _p, _p, _p]),
    "lbm_read_fields_dev": (_i, [_p, _p, _p, _p]),
    "ibm_read_points": (_i, [_p, _p, _p, _p]),
    "ibm_read_points_async": (_i, [_p, _p, _p, _p]),
    "lbm_read_sums_async": (_i, [_p, _p]),
    "lbm_set_host_io": (_i, [_p, _i]),
    "lbm_get_host_io": (_i, [_p, _p]),
    "ibm_read_points_dev": (_i, [_p, _p, _p, _p]),
    "lbm_read_stats": (_i, [_p, _p]),
    "lbm_read_populations": (_i, [_p, _p]),
    "lbm_write_populations": (_i, [_p, _p]),
    "lbm_read_deviations": (_i, [_p, _p]),
    "lbm_read_residuals": (_i, [_p, _p, _i]),
    "lbm_set_graph": (_i, [_p, _i]),
    "lbm_set_overlap": (_i, [_p, _i]),
    "ibm_set_solver": (_i, [_p, _i]),
    "ibm_get_solver": (_i, [_p]),
    "lbm_set_u0_strategy": (_i, [_p, _i]),
    "lbm_get_u0_strategy": (_i, [_p]),
    "ibm_update_points": (_i, [_p, _i64, _p, _p]),
    "lbm_get_launch_shape": (_i, [_p, _p]),
    "lbm_set_launch_shape": (_i, [_p, _p]),
    "lbm_autotune": (_i, [_p, _i, _i, _p]),
    "lbm_batch_get_launch_shape": (_i, [_p, _p]),
    "lbm_batch_set_launch_shape": (_i, [_p, _p]),
    "lbm_batch_autotune": (_i, [_p, _i, _i, _p]),
    "lbm_batch_create": (_i, [_i, _p, _p]),
    "lbm_batch_step": (_i, [_p, _i, _i]),
    "lbm_batch_set_graph": (_i, [_p, _i]),
    "lbm_batch_destroy": (None, [_p]),
    "lbm_velocity_set": (None, [_p, _p]),
    "lbm_enable_timing": (_i, [_p, _i]),
    "lbm_num_stages": (_i, []),
    "lbm_stage_name": (_c.c_char_p, [_i]),
    "lbm_read_timing": (_i, [_p, _p, _p]),
    "lbm_save_state": (_i, [_p, _p, _p]),
    "lbm_load_state": (_i, [_p, _p, _c.c_size_t]),
    "ibm_interpolate_dev": (_i, [_i, _i, _i, _i, _p, _i64, _p, _p, _p]),
    "ibm_spread_scratch_bytes": (_c.c_size_t, [_i, _i, _i, _i64]),
    "ibm_spread_dev": (_i, [_i, _i, _i, _i, _i64, _p, _p, _p, _p, _p]),
    "ibm_spread_dev_noalloc": (_i, [_i, _i, _i, _i, _i64, _p, _p, _p, _p]),
    "mlp_packed_bytes": (_c.c_size_t, []),
    "mlp_pack_dev": (_i, [_p, _p, _p]),
    "mlp_forward_dev": (_i, [_i64, _p, _p, _p, _p]),
    "mlp_grad_scratch_bytes": (_c.c_size_t, [_i64]),
    "mlp_loss_grad_dev": (_i, [_i64, _p, _p, _p, _p, _p, _p, _p, _p]),
    "mlp_adam_dev": (_i, [_p, _p, _p, _p, _i64, _d, _d, _d, _d, _p, _p]),
    "mlp_set_weights": (_i, [_p, _p]),
    "mlp_set_weights_dev": (_i, [_p, _p]),
    "lbm_set_features": (_i, [_p, _i]),
    "ibm_read_mlp_sample_dev": (_i, [_p, _p, _p]),
}

NOALLOC_SCRATCH_BYTES = 16 << 20


def header_functions():
    """Names of the functions declared in include/lbmibm.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z][a-z0-9_]*)\s*\(", txt)) - {"defined", "sizeof"})


def load(path: str = LIB_PATH):
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblbmibm.so is not built (run __graft_entry__.build()); "
                           "there is no CPU fallback")
    L = _c.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(_p)
    if hasattr(a, "data_ptr"):  # torch tensor
        assert a.is_contiguous()
        return _p(a.data_ptr())
    if isinstance(a, int):
        return _p(a)
    raise TypeError(type(a))


def _check(code, h=None):
    if code < 0:
        msg = load().lbm_last_error(h)
        raise LbmError(code, msg.decode() if msg else "")
    return code


def velocity_set():
    e = np.zeros((19, 3), dtype=np.int32)
    t = np.zeros(19)
    load().lbm_velocity_set(_ptr(e), _ptr(t))
    return e, t


def stage_names():
    L = load()
    return [L.lbm_stage_name(i).decode() for i in range(L.lbm_num_stages())]


class Lattice:
    """Owns one lbm_t handle."""

    def __init__(self, shape, tau, storage="f32", delta="cosine", warm="zero",
                 ibm_tol=1e-4, ibm_max_iter=500, stats=True, stream=None, solver="mdf"):
        L = load()
        nz, ny, nx = shape
        o = LbmOpts()
        L.lbm_default_opts(_c.byref(o))
        o.nx, o.ny, o.nz, o.tau = nx, ny, nz, float(tau)
        o.storage, o.delta, o.warm_start = STORAGE[storage], DELTA[delta], WARM[warm]
        o.ibm_tol, o.ibm_max_iter, o.stats = float(ibm_tol), int(ibm_max_iter), int(stats)
        h = _p()
        _check(L.lbm_create_ex(_c.byref(o), _c.byref(h)))
        self.h = h
        self.shape = (nz, ny, nx)
        self.np = 0
        if stream is not None:
            self.set_stream(stream)
        if solver != "mdf":
            self.set_solver(solver)

    def close(self):
        if getattr(self, "h", None):
            load().lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, code):
        return _check(code, self.h)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._c(load().lbm_set_stream(self.h, _p(raw) if raw else None))

    def set_points(self, X, U_target=None, area=None, body=None):
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
        n = len(X)
        ut = None if U_target is None else np.ascontiguousarray(U_target, np.float32).reshape(-1, 3)
        ar = None if area is None else np.ascontiguousarray(area, np.float32).reshape(-1)
        bd = None if body is None else np.ascontiguousarray(body, np.int32).reshape(-1)
        self._c(load().ibm_set_points(self.h, n, _ptr(X), _ptr(ut), _ptr(ar), _ptr(bd)))
        self.np = n

    def update_points(self, X, U_target=None):
        """Moves the current points (same count) without synchronising; X
        (and U_target) must stay alive until the stream has copied them."""
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
        ut = None if U_target is None else np.ascontiguousarray(U_target, np.float32).reshape(-1, 3)
        self._keep = (X, ut)
        self._c(load().ibm_update_points(self.h, len(X), _ptr(X), _ptr(ut)))

    def set_bodies(self, centre, omega, phase):
        c = np.ascontiguousarray(centre, np.float64).reshape(-1, 3)
        om = np.ascontiguousarray(omega, np.float64).reshape(-1)
        ph = np.ascontiguousarray(phase, np.float64).reshape(-1)
        self._c(load().ibm_set_bodies(self.h, len(c), _ptr(c), _ptr(om), _ptr(ph)))

    def set_propellers(self, props):
        """props: workload.Propellers (rest pose + rigid rotating bodies)."""
        self.set_bodies(props.centre, props.omega, props.phase)
        self.set_points(props.xrest, None, props.area, props.body)

    def set_body_force(self, g):
        self._c(load().lbm_set_body_force(self.h, *[float(v) for v in g]))

    def step(self, n_steps=1, n_ibm_iter=5):
        return self._c(load().lbm_step(self.h, int(n_steps), int(n_ibm_iter)))

    @property
    def time(self):
        return load().lbm_time(self.h)

    def set_time(self, t):
        self._c(load().lbm_set_time(self.h, int(t)))

    def fields(self):
        """rho [nz,ny,nx], U [3,nz,ny,nx], G [3,nz,ny,nx] (float32, host)."""
        rho = np.empty(self.shape, np.float32)
        U = np.empty((3,) + self.shape, np.float32)
        G = np.empty((3,) + self.shape, np.float32)
        self._c(load().lbm_read_fields(self.h, _ptr(rho), _ptr(U), _ptr(G)))
        return rho, U, G

    def fields_dev(self, rho=None, U=None, G=None):
        self._c(load().lbm_read_fields_dev(self.h, _ptr(rho), _ptr(U), _ptr(G)))

    def points(self):
        x = np.empty((self.np, 3), np.float64)
        u = np.empty((self.np, 3), np.float32)
        du = np.empty((self.np, 3), np.float32)
        self._c(load().ibm_read_points(self.h, _ptr(x), _ptr(u), _ptr(du)))
        return x, u, du

    def points_dev(self, x=None, u=None, du=None):
        self._c(load().ibm_read_points_dev(self.h, _ptr(x), _ptr(u), _ptr(du)))

    def points_async(self, x=None, u=None, du=None):
        """Enqueue the read-back of x [n][3] f64, u_interp and du [n][3] f32 into
        the given host arrays (pinned for asynchrony) on the lattice's stream;
        valid once the stream has passed this call."""
        self._c(load().ibm_read_points_async(self.h, _ptr(x), _ptr(u), _ptr(du)))

    def sums_async(self, sums):
        """Enqueue the read-back of the FP64 sums (mass, momentum x, y, z) into
        the host array sums[4]; valid once the stream has passed this call."""
        assert sums.dtype == np.float64 and sums.size >= 4
        self._c(load().lbm_read_sums_async(self.h, _ptr(sums)))

    def set_host_io(self, mode="copy"):
        """"copy" (default) or "mapped": uploads and read-outs of page-locked
        host buffers done by the kernels through their device mapping."""
        self._c(load().lbm_set_host_io(self.h, HOST_IO[mode]))

    def host_io(self):
        v = _c.c_int(0)
        self._c(load().lbm_get_host_io(self.h, _c.byref(v)))
        return {i: k for k, i in HOST_IO.items()}[v.value]

    def stats(self):
        s = LbmStats()
        self._c(load().lbm_read_stats(self.h, _c.byref(s)))
        return dict(mass=s.mass, momentum=tuple(s.momentum), step=s.step,
                    last_ibm_iters=s.last_ibm_iters, last_residual=s.last_residual,
                    not_converged=s.not_converged, active_bricks=s.active_bricks,
                    kernel_launches=s.kernel_launches)

    def populations(self):
        f = np.empty((19,) + self.shape, np.float32)
        self._c(load().lbm_read_populations(self.h, _ptr(f)))
        return f

    def residuals(self, cap=4096):
        """eps of every fixed-point iteration of the last (tolerance-mode) step."""
        eps = np.zeros(cap)
        n = self._c(load().lbm_read_residuals(self.h, _ptr(eps), cap))
        return eps[:min(n, cap)]

    def deviations(self):
        d = np.empty((19,) + self.shape, np.float32)
        self._c(load().lbm_read_deviations(self.h, _ptr(d)))
        return d

    def set_populations(self, f):
        f = np.ascontiguousarray(f, np.float32)
        assert f.shape == (19,) + self.shape
        self._c(load().lbm_write_populations(self.h, _ptr(f)))

    def enable_timing(self, stages=True):
        """stages: True (all), False (off) or an iterable of stage names."""
        if stages is True:
            mask = 0x7FFFFFFF
        elif not stages:
            mask = 0
        else:
            names = stage_names()
            mask = sum(1 << names.index(s) for s in stages)
        self._c(load().lbm_enable_timing(self.h, mask))

    def timing(self):
        L = load()
        n = L.lbm_num_stages()
        ms = np.zeros(n)
        la = np.zeros(n, np.int64)
        self._c(L.lbm_read_timing(self.h, _ptr(ms), _ptr(la)))
        names = stage_names()
        return {names[i]: (float(ms[i]), int(la[i])) for i in range(n)}

    def set_mlp_weights(self, P):
        """P: FP32 parameter vector (numpy on the host or a CUDA tensor)."""
        if hasattr(P, "is_cuda") and P.is_cuda:
            self._c(load().mlp_set_weights_dev(self.h, _ptr(P)))
        else:
            P = np.ascontiguousarray(P, np.float32).reshape(-1)
            assert P.size == MLP_NPARAM
            self._c(load().mlp_set_weights(self.h, _ptr(P)))

    def set_graph(self, on=True):
        """Replay captured pairs of steps (fixed iteration counts)."""
        self._c(load().lbm_set_graph(self.h, int(on)))

    def set_overlap(self, on=True):
        """Collide the cells outside the active bricks while the IBM stages
        run, or (the default) every cell after the IBM loop."""
        self._c(load().lbm_set_overlap(self.h, int(on)))

    SOLVERS = {"mdf": 0, "cg": 1}

    def set_solver(self, solver):
        """The fixed point's iteration: "mdf" (the paper's loop, default) or
        "cg" (conjugate gradients on the same fixed point)."""
        self._c(load().ibm_set_solver(self.h, self.SOLVERS[solver]))

    def solver(self):
        return {v: k for k, v in self.SOLVERS.items()}[load().ibm_get_solver(self.h)]

    U0_STRATEGIES = {"bricks": 0, "box": 1, "kernel": 2}

    def set_u0_strategy(self, strategy):
        """How U0 is pre-computed before the fixed point: "bricks" (the active
        bricks, default), "box" or "kernel" (the paper's two strategies)."""
        self._c(load().lbm_set_u0_strategy(self.h, self.U0_STRATEGIES[strategy]))

    def u0_strategy(self):
        return {v: k for k, v in self.U0_STRATEGIES.items()}[load().lbm_get_u0_strategy(self.h)]

    def launch_shape(self):
        s = LaunchShape()
        self._c(load().lbm_get_launch_shape(self.h, _c.byref(s)))
        return s.as_dict()

    def set_launch_shape(self, **kw):
        """Changes fields of the launch shape (results do not depend on it)."""
        s = LaunchShape(**{**self.launch_shape(), **kw})
        self._c(load().lbm_set_launch_shape(self.h, _c.byref(s)))

    def autotune(self, n_ibm_iter=5, steps_per_trial=4):
        """Times candidate launch shapes on this lattice and keeps the fastest;
        the lattice is left as it was.  Returns the chosen shape."""
        s = LaunchShape()
        self._c(load().lbm_autotune(self.h, int(n_ibm_iter), int(steps_per_trial),
                                    _c.byref(s)))
        return s.as_dict()

    def set_features(self, on=True):
        self._c(load().lbm_set_features(self.h, int(on)))

    def mlp_sample_dev(self, X=None, T=None):
        """Writes the last step's features X[n,16] and targets T[n,3] (CUDA)."""
        self._c(load().ibm_read_mlp_sample_dev(self.h, _ptr(X), _ptr(T)))

    def save_state(self):
        L = load()
        n = _c.c_size_t(0)
        self._c(L.lbm_save_state(self.h, None, _c.byref(n)))
        buf = np.empty(n.value, np.uint8)
        self._c(L.lbm_save_state(self.h, _ptr(buf), _c.byref(n)))
        return buf

    def load_state(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        self._c(load().lbm_load_state(self.h, _ptr(buf), buf.size))


def interpolate_dev(U, x, u, delta="cosine", stream=None):
    """U: cuda float32 [3,nz,ny,nx]; x: cuda float64 [n,3]; u: cuda float32 [n,3]."""
    _, nz, ny, nx = U.shape
    raw = getattr(stream, "cuda_stream", stream)
    _check(load().ibm_interpolate_dev(nx, ny, nz, DELTA[delta], _ptr(U), x.shape[0], _ptr(x),
                                      _ptr(u), _p(raw) if raw else None))


def spread_scratch_bytes(shape, n):
    nz, ny, nx = shape
    return load().ibm_spread_scratch_bytes(nx, ny, nz, int(n))


def spread_dev(x, v, F, delta="cosine", scratch=None, stream=None):
    """x: cuda float64 [n,3]; v: cuda float32 [n,3]; F: cuda float32 [3,nz,ny,nx]."""
    _, nz, ny, nx = F.shape
    raw = getattr(stream, "cuda_stream", stream)
    _check(load().ibm_spread_dev(nx, ny, nz, DELTA[delta], x.shape[0], _ptr(x), _ptr(v),
                                 _ptr(F), _ptr(scratch), _p(raw) if raw else None))


def spread_dev_noalloc(x, v, F, delta="cosine", stream=None):
    """ibm_spread_dev_noalloc: spreading with the library's static scratch
    (no device allocation).  Same arguments as spread_dev without scratch."""
    _, nz, ny, nx = F.shape
    raw = getattr(stream, "cuda_stream", stream)
    _check(load().ibm_spread_dev_noalloc(nx, ny, nz, DELTA[delta], x.shape[0], _ptr(x),
                                         _ptr(v), _ptr(F), _p(raw) if raw else None))


def _raw(stream):
    raw = getattr(stream, "cuda_stream", stream)
    return _p(raw) if raw else None


def mlp_packed_bytes():
    return load().mlp_packed_bytes()


def mlp_pack_dev(P, packed, stream=None):
    _check(load().mlp_pack_dev(_ptr(P), _ptr(packed), _raw(stream)))


def mlp_forward_dev(X, packed, Y, stream=None):
    _check(load().mlp_forward_dev(X.shape[0], _ptr(X), _ptr(packed), _ptr(Y), _raw(stream)))


def mlp_grad_scratch_bytes(n):
    return load().mlp_grad_scratch_bytes(int(n))


def mlp_loss_grad_dev(X, T, P, packed, grad, loss, scratch, stream=None):
    _check(load().mlp_loss_grad_dev(X.shape[0], _ptr(X), _ptr(T), _ptr(P), _ptr(packed),
                                    _ptr(grad), _ptr(loss), _ptr(scratch), _raw(stream)))


def mlp_adam_dev(P, m, v, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, packed=None,
                 stream=None):
    _check(load().mlp_adam_dev(_ptr(P), _ptr(m), _ptr(v), _ptr(grad), int(step), float(lr),
                               float(beta1), float(beta2), float(eps), _ptr(packed),
                               _raw(stream)))


class Batch:
    """Several lattices advanced together, one launch per stage."""

    def __init__(self, lattices):
        self.lattices = list(lattices)
        arr = (_p * len(self.lattices))(*[l.h for l in self.lattices])
        self._arr = arr
        b = _p()
        _check(load().lbm_batch_create(len(self.lattices), arr, _c.byref(b)))
        self.b = b

    def step(self, n_steps=1, n_ibm_iter=5):
        code = load().lbm_batch_step(self.b, int(n_steps), int(n_ibm_iter))
        if code < 0:
            _check(code, self.lattices[0].h)
        return code

    def set_graph(self, on=True):
        _check(load().lbm_batch_set_graph(self.b, int(on)))

    U0_STRATEGIES = {"bricks": 0, "box": 1, "kernel": 2}

    def set_u0_strategy(self, strategy):
        """How U0 is pre-computed before the fixed point: "bricks" (the active
        bricks, default), "box" or "kernel" (the paper's two strategies)."""
        self._c(load().lbm_set_u0_strategy(self.h, self.U0_STRATEGIES[strategy]))

    def u0_strategy(self):
        return {v: k for k, v in self.U0_STRATEGIES.items()}[load().lbm_get_u0_strategy(self.h)]

    def launch_shape(self):
        s = LaunchShape()
        _check(load().lbm_batch_get_launch_shape(self.b, _c.byref(s)))
        return s.as_dict()

    def set_launch_shape(self, **kw):
        s = LaunchShape(**{**self.launch_shape(), **kw})
        _check(load().lbm_batch_set_launch_shape(self.b, _c.byref(s)), self.lattices[0].h)

    def autotune(self, n_ibm_iter=5, steps_per_trial=3):
        s = LaunchShape()
        _check(load().lbm_batch_autotune(self.b, int(n_ibm_iter), int(steps_per_trial),
                                         _c.byref(s)), self.lattices[0].h)
        return s.as_dict()

    def close(self):
        if getattr(self, "b", None):
            load().lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
