"""Python binding of the C ABI in include/lbm_ace.h and include/lbm_ace_surrogate.h
(argument marshalling only).

Every function here forwards to the entry point of the same name in
``liblbm_ace.so``; all lattice Boltzmann arithmetic runs in the library's CUDA
kernels. There is no CPU fallback: if the library cannot be loaded, every call
raises. PyTorch is optional and only used to hand in a CUDA stream or to
receive arrays as tensors.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

from . import build as _build

# status codes
OK, EINVAL, ENOMEM, ECUDA, ENUMERIC, ETIMEOUT, ECALLBACK = 0, -1, -2, -3, -4, -5, -6
# precision
F64, F32, F16DEV, BF16DEV = 0, 1, 2, 3
# model
MODEL_MODIFIED, MODEL_CONSERVATIVE = 0, 1
# velocity
VEL_SINGLE_VORTEX, VEL_UNIFORM, VEL_FIELD, VEL_CALLBACK = 0, 1, 2, 3
# fused step kernel variant
KERNEL_AUTO, KERNEL_DIRECT, KERNEL_BULK, KERNEL_WARP, KERNEL_PAIR = 0, 1, 2, 3, 4
KERNEL_DEV, KERNEL_TWO_STEP, KERNEL_DEV4, KERNEL_QUAD = 5, 6, 7, 8

VELOCITY_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.c_void_p)

# Entry points declared in include/lbm_ace.h (checked by the test suite).
EXPORTS = (
    "lbm_ace_params_default", "lbm_ace_init", "lbm_ace_step", "lbm_ace_get_phi", "lbm_ace_mass",
    "lbm_ace_step_mass", "lbm_ace_get_state", "lbm_ace_set_state", "lbm_ace_steps_done",
    "lbm_ace_launch_shape", "lbm_ace_synchronize", "lbm_ace_last_error", "lbm_ace_status_string",
    "lbm_ace_destroy", "lbm_ace_mass_noalloc",
    "lbm_ace_batch_init", "lbm_ace_batch_step", "lbm_ace_batch_step_sequential", "lbm_ace_batch_autotune",
    "lbm_ace_batch_get_phi", "lbm_ace_batch_mass", "lbm_ace_batch_info", "lbm_ace_batch_steps_done",
    "lbm_ace_batch_synchronize", "lbm_ace_batch_last_error", "lbm_ace_batch_destroy",
    "lbm_ace_batch_step_per_lattice", "lbm_ace_batch_set_ends", "lbm_ace_batch_lattice_steps",
    "lbm_ace_batch_active",
    "lbm_ace_get_phi_device", "lbm_ace_velocity_device", "lbm_ace_reset_device", "lbm_ace_get_stream",
    "lbm_ace_get_params", "lbm_ace_wait_selftest", "lbm_ace_release_cached_memory",
    "lbm_ace_net_create", "lbm_ace_net_set_params", "lbm_ace_net_get_params", "lbm_ace_net_forward",
    "lbm_ace_net_loss_grad", "lbm_ace_net_adam", "lbm_ace_net_gather", "lbm_ace_net_metrics",
    "lbm_ace_net_synchronize", "lbm_ace_net_last_error", "lbm_ace_net_destroy", "lbm_ace_hybrid_advance",
    "lbm_ace_net_launch_shape", "lbm_ace_net_wait_selftest",
)
NET_WIDTH, NET_K, NET_PARAMS = 32, 16, 28929
NOALLOC_CHUNK = 65536
NOALLOC_MAX_PARTIALS = 4096
NOALLOC_MAX_COUNT = NOALLOC_CHUNK * NOALLOC_MAX_PARTIALS


class lbm_ace_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau", ctypes.c_double), ("M", ctypes.c_double), ("eps", ctypes.c_double),
        ("reg_delta", ctypes.c_double),
        ("precision", ctypes.c_int), ("model", ctypes.c_int), ("velocity_kind", ctypes.c_int),
        ("U0", ctypes.c_double), ("T_period", ctypes.c_double), ("vortex_sign", ctypes.c_double),
        ("ux", ctypes.c_double), ("uy", ctypes.c_double),
        ("u_field", ctypes.POINTER(ctypes.c_double)), ("v_field", ctypes.POINTER(ctypes.c_double)),
        ("vel_fn", VELOCITY_FN), ("vel_user", ctypes.c_void_p),
        ("phi0", ctypes.POINTER(ctypes.c_double)),
        ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("R", ctypes.c_double),
        ("device", ctypes.c_int), ("stream", ctypes.c_void_p),
        ("rows_per_cta", ctypes.c_int), ("kernel_variant", ctypes.c_int),
    ]


class lbm_ace_hybrid_stats(ctypes.Structure):
    _fields_ = [("windows", ctypes.c_longlong), ("surrogate_windows", ctypes.c_longlong),
                ("fallback_windows", ctypes.c_longlong), ("mass0", ctypes.c_double), ("width0", ctypes.c_double),
                ("max_mass_drift", ctypes.c_double), ("max_width_dev", ctypes.c_double)]


class LbmAceError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} [status {status}]")
        self.status = status


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_P = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbm_ace.so (compiling it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise LbmAceError(ECUDA, f"CUDA library {path} is missing; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    L.lbm_ace_params_default.argtypes = [ctypes.POINTER(lbm_ace_params)]
    L.lbm_ace_init.argtypes = [ctypes.POINTER(lbm_ace_params), ctypes.POINTER(_P)]
    L.lbm_ace_step.argtypes = [_P, ctypes.c_longlong]
    L.lbm_ace_get_phi.argtypes = [_P, _D, ctypes.c_size_t]
    L.lbm_ace_mass.argtypes = [_P, _D]
    L.lbm_ace_step_mass.argtypes = [_P, _D]
    L.lbm_ace_get_state.argtypes = [_P, _D, _D]
    L.lbm_ace_set_state.argtypes = [_P, _D, _D, ctypes.c_longlong]
    L.lbm_ace_steps_done.argtypes = [_P]
    L.lbm_ace_steps_done.restype = ctypes.c_longlong
    L.lbm_ace_launch_shape.argtypes = [_P] + [ctypes.POINTER(ctypes.c_int)] * 5
    L.lbm_ace_synchronize.argtypes = [_P]
    L.lbm_ace_wait_selftest.argtypes = [_P, ctypes.c_longlong]
    L.lbm_ace_release_cached_memory.argtypes = [ctypes.c_int]
    L.lbm_ace_last_error.argtypes = [_P]
    L.lbm_ace_last_error.restype = ctypes.c_char_p
    L.lbm_ace_status_string.argtypes = [ctypes.c_int]
    L.lbm_ace_status_string.restype = ctypes.c_char_p
    L.lbm_ace_destroy.argtypes = [_P]
    L.lbm_ace_destroy.restype = None
    L.lbm_ace_mass_noalloc.argtypes = [_P, ctypes.c_int, ctypes.c_longlong, _P, _P]
    L.lbm_ace_mass_noalloc.restype = ctypes.c_int
    _I = ctypes.POINTER(ctypes.c_int)
    L.lbm_ace_batch_init.argtypes = [ctypes.POINTER(lbm_ace_params), ctypes.c_int, ctypes.POINTER(_P)]
    L.lbm_ace_batch_step.argtypes = [_P, ctypes.c_longlong]
    L.lbm_ace_batch_step_sequential.argtypes = [_P, ctypes.c_longlong]
    L.lbm_ace_batch_autotune.argtypes = [_P, ctypes.c_int, _I]
    L.lbm_ace_batch_get_phi.argtypes = [_P, ctypes.c_int, _D, ctypes.c_size_t]
    L.lbm_ace_batch_mass.argtypes = [_P, ctypes.c_int, _D]
    L.lbm_ace_batch_info.argtypes = [_P, ctypes.c_int, _I, _I, _I, ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_ace_batch_steps_done.argtypes = [_P]
    L.lbm_ace_batch_steps_done.restype = ctypes.c_longlong
    L.lbm_ace_batch_synchronize.argtypes = [_P]
    L.lbm_ace_batch_last_error.argtypes = [_P]
    L.lbm_ace_batch_last_error.restype = ctypes.c_char_p
    L.lbm_ace_batch_destroy.argtypes = [_P]
    L.lbm_ace_batch_destroy.restype = None
    L.lbm_ace_batch_step_per_lattice.argtypes = [_P, ctypes.c_longlong]
    L.lbm_ace_batch_set_ends.argtypes = [_P, ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_ace_batch_lattice_steps.argtypes = [_P, ctypes.c_int]
    L.lbm_ace_batch_lattice_steps.restype = ctypes.c_longlong
    L.lbm_ace_batch_active.argtypes = [_P, _I, _I]
    for name in ("lbm_ace_batch_init", "lbm_ace_batch_step", "lbm_ace_batch_step_sequential",
                 "lbm_ace_batch_autotune", "lbm_ace_batch_get_phi", "lbm_ace_batch_mass",
                 "lbm_ace_batch_info", "lbm_ace_batch_synchronize", "lbm_ace_batch_step_per_lattice",
                 "lbm_ace_batch_set_ends", "lbm_ace_batch_active"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("lbm_ace_params_default", "lbm_ace_init", "lbm_ace_step", "lbm_ace_get_phi",
                 "lbm_ace_mass", "lbm_ace_step_mass", "lbm_ace_get_state", "lbm_ace_set_state",
                 "lbm_ace_launch_shape", "lbm_ace_synchronize"):
        getattr(L, name).restype = ctypes.c_int
    # device-side access
    L.lbm_ace_get_phi_device.argtypes = [_P, _P]
    L.lbm_ace_velocity_device.argtypes = [_P, ctypes.c_double, _P, _P]
    L.lbm_ace_reset_device.argtypes = [_P, _P, ctypes.c_longlong]
    L.lbm_ace_get_stream.argtypes = [_P]
    L.lbm_ace_get_stream.restype = _P
    L.lbm_ace_get_params.argtypes = [_P, ctypes.POINTER(lbm_ace_params)]
    for name in ("lbm_ace_get_phi_device", "lbm_ace_velocity_device", "lbm_ace_reset_device", "lbm_ace_get_params"):
        getattr(L, name).restype = ctypes.c_int
    # surrogate
    _F = ctypes.POINTER(ctypes.c_float)
    L.lbm_ace_net_create.argtypes = [ctypes.c_int, _P, ctypes.POINTER(_P)]
    L.lbm_ace_net_set_params.argtypes = [_P, _F, ctypes.c_size_t]
    L.lbm_ace_net_get_params.argtypes = [_P, _F, ctypes.c_size_t]
    L.lbm_ace_net_forward.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.lbm_ace_net_loss_grad.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _F,
                                        ctypes.c_size_t]
    L.lbm_ace_net_adam.argtypes = [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    L.lbm_ace_net_gather.argtypes = [_P, _P, _P, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int, ctypes.c_longlong]
    L.lbm_ace_net_metrics.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, _D, _D]
    L.lbm_ace_net_synchronize.argtypes = [_P]
    L.lbm_ace_net_wait_selftest.argtypes = [_P, ctypes.c_longlong]
    L.lbm_ace_net_wait_selftest.restype = ctypes.c_int
    L.lbm_ace_net_launch_shape.argtypes = [_P] + [ctypes.POINTER(ctypes.c_int)] * 5
    L.lbm_ace_net_launch_shape.restype = ctypes.c_int
    L.lbm_ace_net_last_error.argtypes = [_P]
    L.lbm_ace_net_last_error.restype = ctypes.c_char_p
    L.lbm_ace_net_destroy.argtypes = [_P]
    L.lbm_ace_net_destroy.restype = None
    L.lbm_ace_hybrid_advance.argtypes = [_P, _P, ctypes.c_longlong, ctypes.c_double, ctypes.c_double,
                                         ctypes.POINTER(lbm_ace_hybrid_stats)]
    for name in ("lbm_ace_net_create", "lbm_ace_net_set_params", "lbm_ace_net_get_params", "lbm_ace_net_forward",
                 "lbm_ace_net_loss_grad", "lbm_ace_net_adam", "lbm_ace_net_gather", "lbm_ace_net_metrics",
                 "lbm_ace_net_synchronize", "lbm_ace_hybrid_advance"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def params_default() -> lbm_ace_params:
    p = lbm_ace_params()
    load().lbm_ace_params_default(ctypes.byref(p))
    return p


def _check(ctx, rc: int):
    if rc != OK:
        msg = load().lbm_ace_last_error(ctx)
        raise LbmAceError(rc, (msg or b"").decode(errors="replace"))


class Lattice:
    """One lattice owned by the library (wraps lbm_ace_init ... lbm_ace_destroy).

    Keyword arguments set fields of ``lbm_ace_params`` (same names); ``phi0``,
    ``u_field`` and ``v_field`` take float64 arrays of shape [ny, nx];
    ``stream`` takes a CUDA stream handle (int) or a ``torch.cuda.Stream``;
    ``vel_fn`` takes a Python callable ``f(t, nx, ny) -> (u, v)``."""

    def __init__(self, **kw):
        self._lib = load()
        p = params_default()
        self._keep = []
        for k in ("phi0", "u_field", "v_field"):
            a = kw.pop(k, None)
            if a is not None:
                arr = np.ascontiguousarray(a, dtype=np.float64)
                self._keep.append(arr)
                setattr(p, k, _dp(arr))
        stream = kw.pop("stream", None)
        if stream is not None:
            p.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        fn = kw.pop("vel_fn", None)
        if fn is not None:
            def tramp(t, nx, ny, u, v, user, _fn=fn):
                try:
                    uu, vv = _fn(t, nx, ny)
                    n = nx * ny
                    np.ctypeslib.as_array(u, (n,))[:] = np.asarray(uu, dtype=np.float64).ravel()
                    np.ctypeslib.as_array(v, (n,))[:] = np.asarray(vv, dtype=np.float64).ravel()
                    return 0
                except Exception:  # reported to the caller as LBM_ACE_ECALLBACK
                    return 1
            cb = VELOCITY_FN(tramp)
            self._keep.append(cb)
            p.vel_fn = cb
            p.velocity_kind = VEL_CALLBACK
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k!r}")
            setattr(p, k, v)
        self.params = p
        self.nx, self.ny = p.nx, p.ny
        ctx = _P()
        rc = self._lib.lbm_ace_init(ctypes.byref(p), ctypes.byref(ctx))
        if rc != OK:
            raise LbmAceError(rc, (self._lib.lbm_ace_last_error(None) or b"").decode(errors="replace"))
        self.ctx = ctx

    # -- C ABI, one method per entry point --------------------------------------
    def lbm_ace_step(self, n: int = 1) -> "Lattice":
        _check(self.ctx, self._lib.lbm_ace_step(self.ctx, int(n)))
        return self

    step = lbm_ace_step

    def lbm_ace_get_phi(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        """phi(x, t) as float64 [ny, nx], into `out` when given (C-contiguous float64 of
        nx * ny values). A page-locked `out`, such as the numpy view of a pinned torch
        tensor, is written by the library's kernel directly; other memory through a copy."""
        if out is None:
            out = np.empty((self.ny, self.nx), dtype=np.float64)
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == self.nx * self.ny
        _check(self.ctx, self._lib.lbm_ace_get_phi(self.ctx, _dp(out), out.size))
        return out

    phi = lbm_ace_get_phi

    def lbm_ace_mass(self) -> float:
        m = ctypes.c_double()
        _check(self.ctx, self._lib.lbm_ace_mass(self.ctx, ctypes.byref(m)))
        return m.value

    mass = lbm_ace_mass

    def lbm_ace_step_mass(self) -> float:
        m = ctypes.c_double()
        _check(self.ctx, self._lib.lbm_ace_step_mass(self.ctx, ctypes.byref(m)))
        return m.value

    step_mass = lbm_ace_step_mass

    def lbm_ace_get_state(self):
        f = np.empty((9, self.ny, self.nx), dtype=np.float64)
        pp = np.empty((self.ny, self.nx), dtype=np.float64)
        _check(self.ctx, self._lib.lbm_ace_get_state(self.ctx, _dp(f), _dp(pp)))
        return f, pp

    get_state = lbm_ace_get_state

    def lbm_ace_set_state(self, f: np.ndarray, phi_prev: np.ndarray, t: int) -> "Lattice":
        f = np.ascontiguousarray(f, dtype=np.float64)
        pp = np.ascontiguousarray(phi_prev, dtype=np.float64)
        assert f.size == 9 * self.nx * self.ny and pp.size == self.nx * self.ny
        _check(self.ctx, self._lib.lbm_ace_set_state(self.ctx, _dp(f), _dp(pp), int(t)))
        return self

    set_state = lbm_ace_set_state

    def lbm_ace_steps_done(self) -> int:
        return int(self._lib.lbm_ace_steps_done(self.ctx))

    @property
    def t(self) -> int:
        return self.lbm_ace_steps_done()

    def lbm_ace_launch_shape(self):
        v = [ctypes.c_int() for _ in range(5)]
        _check(self.ctx, self._lib.lbm_ace_launch_shape(self.ctx, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    launch_shape = lbm_ace_launch_shape

    def lbm_ace_synchronize(self) -> None:
        _check(self.ctx, self._lib.lbm_ace_synchronize(self.ctx))

    synchronize = lbm_ace_synchronize

    def lbm_ace_wait_selftest(self, limit_cycles: int) -> None:
        """A device wait that nothing completes gives up after `limit_cycles` SM cycles;
        raises LbmAceError with status ETIMEOUT, as a step whose wait gave up would."""
        _check(self.ctx, self._lib.lbm_ace_wait_selftest(self.ctx, int(limit_cycles)))

    # -- device-side access (pointers are device addresses, e.g. tensor.data_ptr()) --
    def lbm_ace_get_phi_device(self, phi_ptr: int) -> None:
        _check(self.ctx, self._lib.lbm_ace_get_phi_device(self.ctx, _P(phi_ptr)))

    def lbm_ace_velocity_device(self, t: float, u_ptr: int, v_ptr: int) -> None:
        _check(self.ctx, self._lib.lbm_ace_velocity_device(self.ctx, float(t), _P(u_ptr), _P(v_ptr)))

    def lbm_ace_reset_device(self, phi_ptr: int, t: int) -> None:
        _check(self.ctx, self._lib.lbm_ace_reset_device(self.ctx, _P(phi_ptr), int(t)))

    def lbm_ace_get_stream(self) -> int:
        return int(self._lib.lbm_ace_get_stream(self.ctx) or 0)

    def lbm_ace_get_params(self) -> lbm_ace_params:
        p = lbm_ace_params()
        _check(self.ctx, self._lib.lbm_ace_get_params(self.ctx, ctypes.byref(p)))
        return p

    def close(self) -> None:
        if getattr(self, "ctx", None):
            self._lib.lbm_ace_destroy(self.ctx)
            self.ctx = None

    lbm_ace_destroy = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many single-vortex lattices advanced together (wraps lbm_ace_batch_*).

    ``lattices`` is a list of dicts of ``lbm_ace_params`` fields (nx, ny, tau, eps, U0,
    T_period, vortex_sign, xc, yc, R, rows_per_cta, ...); precision FP32 and the single
    vortex are set here. ``stream`` as for Lattice."""

    def __init__(self, lattices, stream=None, device=0, model=MODEL_MODIFIED):
        self._lib = load()
        arr = (lbm_ace_params * len(lattices))()
        for k, kw in enumerate(lattices):
            self._lib.lbm_ace_params_default(ctypes.byref(arr[k]))
            arr[k].precision = F32
            arr[k].velocity_kind = VEL_SINGLE_VORTEX
            arr[k].model = model
            arr[k].device = device
            if stream is not None:
                arr[k].stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
            for f, v in kw.items():
                setattr(arr[k], f, v)
        self.shapes = [(int(p.ny), int(p.nx)) for p in arr]
        h = _P()
        rc = self._lib.lbm_ace_batch_init(arr, len(lattices), ctypes.byref(h))
        if rc != OK:
            raise LbmAceError(rc, (self._lib.lbm_ace_batch_last_error(None) or b"").decode(errors="replace"))
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise LbmAceError(rc, (self._lib.lbm_ace_batch_last_error(self.h) or b"").decode(errors="replace"))

    def step(self, n=1):
        self._check(self._lib.lbm_ace_batch_step(self.h, int(n)))
        return self

    def step_sequential(self, n=1):
        self._check(self._lib.lbm_ace_batch_step_sequential(self.h, int(n)))
        return self

    def autotune(self, steps_per_trial=5):
        rows = (ctypes.c_int * len(self.shapes))()
        self._check(self._lib.lbm_ace_batch_autotune(self.h, int(steps_per_trial), rows))
        return list(rows)

    def phi(self, i):
        ny, nx = self.shapes[i]
        out = np.empty((ny, nx))
        self._check(self._lib.lbm_ace_batch_get_phi(self.h, int(i), _dp(out), out.size))
        return out

    def mass(self, i):
        m = ctypes.c_double()
        self._check(self._lib.lbm_ace_batch_mass(self.h, int(i), ctypes.byref(m)))
        return m.value

    def info(self, i=0):
        r, t, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        n = ctypes.c_longlong()
        self._check(self._lib.lbm_ace_batch_info(self.h, int(i), ctypes.byref(r), ctypes.byref(t),
                                                 ctypes.byref(g), ctypes.byref(n)))
        return {"rows": r.value, "tiles": t.value, "grid": g.value, "nodes": n.value}

    @property
    def t(self):
        return int(self._lib.lbm_ace_batch_steps_done(self.h))

    def step_per_lattice(self, n=1):
        self._check(self._lib.lbm_ace_batch_step_per_lattice(self.h, int(n)))
        return self

    def set_ends(self, ends=None):
        """Per-lattice end steps (None: each lattice's T_period rounded; -1: no end)."""
        if ends is None:
            self._check(self._lib.lbm_ace_batch_set_ends(self.h, None))
        else:
            arr = (ctypes.c_longlong * len(self.shapes))(*[int(e) for e in ends])
            self._check(self._lib.lbm_ace_batch_set_ends(self.h, arr))
        return self

    def lattice_steps(self, i):
        return int(self._lib.lbm_ace_batch_lattice_steps(self.h, int(i)))

    def active(self):
        """(lattices, tiles) still advancing at the batch's clock."""
        a, t = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.lbm_ace_batch_active(self.h, ctypes.byref(a), ctypes.byref(t)))
        return a.value, t.value

    def synchronize(self):
        self._check(self._lib.lbm_ace_batch_synchronize(self.h))

    def close(self):
        if getattr(self, "h", None):
            self._lib.lbm_ace_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _ptr(x) -> int:
    """Device address of a torch tensor (data_ptr) or an int."""
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)


class Net:
    """The learned surrogate (wraps lbm_ace_net_create ... lbm_ace_net_destroy). Image
    arguments are device FP32 arrays of [batch, ny, nx] given as torch tensors or
    device addresses; all arithmetic runs in the library's kernels."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = load()
        h = _P()
        s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        rc = self._lib.lbm_ace_net_create(int(device), _P(s), ctypes.byref(h))
        if rc != OK:
            raise LbmAceError(rc, (self._lib.lbm_ace_net_last_error(None) or b"").decode(errors="replace"))
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise LbmAceError(rc, (self._lib.lbm_ace_net_last_error(self.h) or b"").decode(errors="replace"))

    def lbm_ace_net_set_params(self, params) -> None:
        a = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self._lib.lbm_ace_net_set_params(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))

    set_params = lbm_ace_net_set_params

    def lbm_ace_net_get_params(self) -> np.ndarray:
        a = np.empty(NET_PARAMS, dtype=np.float32)
        self._check(self._lib.lbm_ace_net_get_params(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))
        return a

    get_params = lbm_ace_net_get_params

    def lbm_ace_net_forward(self, phi, u, v, phi_out, batch: int, ny: int, nx: int) -> None:
        self._check(self._lib.lbm_ace_net_forward(self.h, _P(_ptr(phi)), _P(_ptr(u)), _P(_ptr(v)),
                                                  _P(_ptr(phi_out)), int(batch), int(ny), int(nx)))

    forward = lbm_ace_net_forward

    def lbm_ace_net_loss_grad(self, phi, u, v, target, batch: int, ny: int, nx: int,
                              want_loss: bool = True, want_grad: bool = False):
        loss = ctypes.c_double(float("nan"))
        g = np.empty(NET_PARAMS, dtype=np.float32) if want_grad else None
        self._check(self._lib.lbm_ace_net_loss_grad(
            self.h, _P(_ptr(phi)), _P(_ptr(u)), _P(_ptr(v)), _P(_ptr(target)), int(batch), int(ny), int(nx),
            ctypes.byref(loss) if want_loss else None,
            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if want_grad else None, NET_PARAMS if want_grad else 0))
        return (loss.value if want_loss else None), g

    loss_grad = lbm_ace_net_loss_grad

    def lbm_ace_net_adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
        self._check(self._lib.lbm_ace_net_adam(self.h, lr, beta1, beta2, eps))

    adam = lbm_ace_net_adam

    def lbm_ace_net_gather(self, dst, src, index, image_elems: int) -> None:
        idx = np.ascontiguousarray(index, dtype=np.int64)
        self._check(self._lib.lbm_ace_net_gather(self.h, _P(_ptr(dst)), _P(_ptr(src)),
                                                 idx.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), idx.size,
                                                 int(image_elems)))

    gather = lbm_ace_net_gather

    def lbm_ace_net_metrics(self, phi, ny: int, nx: int):
        m, w = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.lbm_ace_net_metrics(self.h, _P(_ptr(phi)), int(ny), int(nx), ctypes.byref(m),
                                                  ctypes.byref(w)))
        return m.value, w.value

    metrics = lbm_ace_net_metrics

    def lbm_ace_net_launch_shape(self) -> dict:
        v = [ctypes.c_int() for _ in range(5)]
        self._check(self._lib.lbm_ace_net_launch_shape(self.h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("conv_ctas", "conv_occupancy", "out_ctas", "out_occupancy", "sms"), (x.value for x in v)))

    launch_shape = lbm_ace_net_launch_shape

    def lbm_ace_net_synchronize(self) -> None:
        self._check(self._lib.lbm_ace_net_synchronize(self.h))

    synchronize = lbm_ace_net_synchronize

    def lbm_ace_net_wait_selftest(self, limit_cycles: int) -> None:
        """Run the bounded-wait failure self-test; raises LbmAceError (status ETIMEOUT)
        when the wait gave up, which is the expected outcome."""
        self._check(self._lib.lbm_ace_net_wait_selftest(self.h, int(limit_cycles)))

    wait_selftest = lbm_ace_net_wait_selftest

    def lbm_ace_hybrid_advance(self, lattice: "Lattice", windows: int, mass_tol: float = 1e-6,
                               width_tol: float = 0.1) -> dict:
        st = lbm_ace_hybrid_stats()
        self._check(self._lib.lbm_ace_hybrid_advance(lattice.ctx, self.h, int(windows), float(mass_tol),
                                                     float(width_tol), ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in lbm_ace_hybrid_stats._fields_}

    hybrid_advance = lbm_ace_hybrid_advance

    def close(self) -> None:
        if getattr(self, "h", None):
            self._lib.lbm_ace_net_destroy(self.h)
            self.h = None

    lbm_ace_net_destroy = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def lbm_ace_mass_noalloc(values_ptr: int, precision: int, count: int, out_ptr: int,
                         stream: int = 0) -> int:
    """Allocation-free global mass of `count` device values (FP64 or FP32) into the device
    double at `out_ptr`, asynchronous on `stream`; returns the status code. For callers
    that cannot allocate device memory: the library keeps its partial sums in a fixed
    static device array, so overlapping calls on the GPU race (see include/lbm_ace.h)."""
    return int(load().lbm_ace_mass_noalloc(_P(values_ptr), int(precision), int(count),
                                           _P(out_ptr), _P(int(getattr(stream, "cuda_stream", stream)))))


def release_cached_memory(device: int = 0) -> None:
    """Hand the device memory that destroyed lattices left in the library's pool back to
    the driver (lbm_ace_release_cached_memory); live lattices keep theirs."""
    _check(None, load().lbm_ace_release_cached_memory(int(device)))


def status_string(rc: int) -> str:
    return load().lbm_ace_status_string(rc).decode()


def vortex_lattice(L: int, *, eps: float = 1.0, tau: float = 0.8, U0: float = 0.04,
                   T: float = None, precision: int = F32, R_frac: float = 0.15,
                   xc_frac: float = 0.5, yc_frac: float = 0.75, sign: float = -1.0,
                   **kw) -> Lattice:
    """The single-vortex workload (Section 3, Eq. 14) with the disk built by the library."""
    return Lattice(nx=L, ny=L, tau=tau, eps=eps, U0=U0, T_period=float(T if T else 16 * L),
                   vortex_sign=sign, precision=precision, velocity_kind=VEL_SINGLE_VORTEX,
                   xc=xc_frac * L, yc=yc_frac * L, R=R_frac * L, **kw)


DEFAULT_DELTA = math.exp(-20.0)
