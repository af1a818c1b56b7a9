"""Python binding of the GB300 acoustic propagator library (include/mmod.h).

Argument marshalling only: every step of the propagator runs in the CUDA
kernels of ``libmmod.so``.  The functions keep the C names (``mmod_create``,
``mmod_set_model``, ``mmod_forward`` ...); array arguments may be torch tensors
(device or host), numpy arrays (host) or raw integer addresses, and streams are
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers or ``None`` (the
current torch stream when torch has CUDA, else the legacy default stream).

There is no CPU fallback: without a loadable library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = ["MmodError", "build", "load", "mmod_create", "mmod_destroy", "mmod_set_model",
           "mmod_forward", "mmod_set_state", "mmod_get_state", "mmod_set_kernel",
           "mmod_last_error", "mmod_last_launch_count", "mmod_last_loop_ms", "mmod_cfl_dt",
           "mmod_version", "Propagator", "STATUS", "EXPORTED"]

STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_UNSTABLE", -3: "ERR_OOM", -4: "ERR_CUDA",
          -5: "ERR_TIMEOUT", -6: "ERR_STATE", -7: "ERR_UNSUPPORTED"}
KERNEL_AUTO, KERNEL_SIMPLE, KERNEL_TMA = 0, 1, 2
OPT_PDL = 2
OPT_CKPT_SCHEME = 3
OPT_PERSISTENT = 4
OPT_PERSISTENT_CTAS = 5
OPT_TEST_STALL = 6
OPT_ZLEN = 7
OPT_CPML_PLANES = 8
OPT_CLAIM = 9
OPT_CPML_TILES = 10
BOUNDARY_DAMPING, BOUNDARY_CPML = 0, 1
BATCH_STREAMS, BATCH_FUSED, BATCH_PERSISTENT = 0, 1, 2
SCHEME_SEGMENTS, SCHEME_REVOLVE = 0, 1
REV_ADVANCE, REV_SAVE, REV_RESTORE, REV_REVERSE = 0, 1, 2, 3

# Every symbol include/mmod.h declares (checked against the header by the tests).
EXPORTED = ["mmod_create", "mmod_destroy", "mmod_set_model", "mmod_forward", "mmod_set_state",
            "mmod_get_state", "mmod_set_kernel", "mmod_last_launch_count", "mmod_last_loop_ms",
            "mmod_cfl_dt", "mmod_last_error", "mmod_version", "mmod_check_recip",
            "mmod_tma_variant_count", "mmod_tma_variant_name", "mmod_set_tma_variant", "mmod_get_plan",
            "mmod_forward_noalloc", "mmod_set_option", "mmod_adjoint", "mmod_gradient",
            "mmod_gradient_memory", "mmod_dot", "mmod_batch_create", "mmod_batch_destroy",
            "mmod_batch_forward", "mmod_batch_set_variant", "mmod_batch_last_loop_ms", "mmod_batch_last_error",
            "mmod_autotune", "mmod_batch_autotune", "mmod_revolve_schedule", "mmod_persistent_grid",
            "mmod_tma_variant_info", "mmod_batch_set_mode", "mmod_optimized_coefficients",
            "mmod_set_fd_coefficients", "mmod_vd_create", "mmod_vd_destroy", "mmod_vd_set_model",
            "mmod_vd_set_state", "mmod_vd_forward", "mmod_vd_set_kernel", "mmod_vd_uses_tma", "mmod_vd_set_option",
            "mmod_vd_last_loop_ms", "mmod_vd_last_launch_count", "mmod_vd_last_error", "mmod_vd_get_plan"]
CKPT_FP32, CKPT_BF16, CKPT_FP16, CKPT_BFP16 = 0, 1, 2, 3


class MmodError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
                ("dt", ctypes.c_double), ("nt", ctypes.c_int), ("order", ctypes.c_int),
                ("nbl", ctypes.c_int), ("damp_R", ctypes.c_double),
                ("nsrc", ctypes.c_int), ("src_ijk", ctypes.c_void_p),
                ("nrec", ctypes.c_int), ("rec_ijk", ctypes.c_void_p),
                ("free_surface", ctypes.c_int), ("boundary", ctypes.c_int), ("cpml_f0", ctypes.c_double)]


_lib = None


def build(force: bool = False) -> str:
    """Compile libmmod.so for sm_103a (nvcc) if missing or stale."""
    return _build.build(force=force)


def load():
    """Load libmmod.so (building it first if needed) and declare signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if _build.is_stale():
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "mmod_create": ([ctypes.POINTER(_Config), I, ctypes.POINTER(P)], I),
        "mmod_destroy": ([P], I),
        "mmod_set_model": ([P, P, P], I),
        "mmod_forward": ([P, P, P, P, P], I),
        "mmod_set_state": ([P, P, P, P], I),
        "mmod_get_state": ([P, P, P, P], I),
        "mmod_set_kernel": ([P, I], I),
        "mmod_last_launch_count": ([P], ctypes.c_longlong),
        "mmod_last_loop_ms": ([P], ctypes.c_float),
        "mmod_cfl_dt": ([D, D, D], D),
        "mmod_last_error": ([P], ctypes.c_char_p),
        "mmod_version": ([], ctypes.c_char_p),
        "mmod_check_recip": ([I, ctypes.POINTER(ctypes.c_uint)], I),
        "mmod_tma_variant_count": ([], I),
        "mmod_tma_variant_name": ([I], ctypes.c_char_p),
        "mmod_set_tma_variant": ([P, I], I),
        "mmod_get_plan": ([P, ctypes.POINTER(ctypes.c_int)], I),
        "mmod_forward_noalloc": ([ctypes.POINTER(_Config), I, P, P, P, P, P], I),
        "mmod_set_option": ([P, I, I], I),
        "mmod_adjoint": ([P, P, P, P], I),
        "mmod_gradient": ([P, P, P, P, I, I, P], I),
        "mmod_gradient_memory": ([P, I, I], ctypes.c_longlong),
        "mmod_dot": ([P, P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double), P], I),
        "mmod_batch_create": ([ctypes.POINTER(P), I, ctypes.POINTER(P)], I),
        "mmod_batch_destroy": ([P], I),
        "mmod_batch_forward": ([P, ctypes.POINTER(P), ctypes.POINTER(P), P], I),
        "mmod_batch_set_variant": ([P, I], I),
        "mmod_batch_last_loop_ms": ([P], ctypes.c_float),
        "mmod_batch_last_error": ([P], ctypes.c_char_p),
        "mmod_autotune": ([P, I, P, ctypes.POINTER(I)], I),
        "mmod_batch_autotune": ([P, I, P, ctypes.POINTER(I)], I),
        "mmod_revolve_schedule": ([I, I, P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_longlong)], I),
        "mmod_persistent_grid": ([P], I),
        "mmod_tma_variant_info": ([I, ctypes.POINTER(I)], I),
        "mmod_batch_set_mode": ([P, I], I),
        "mmod_optimized_coefficients": ([D, P], I),
        "mmod_set_fd_coefficients": ([P, P], I),
        "mmod_vd_create": ([ctypes.POINTER(_Config), I, ctypes.POINTER(P)], I),
        "mmod_vd_destroy": ([P], I),
        "mmod_vd_set_model": ([P, P, P, P], I),
        "mmod_vd_set_state": ([P, P, P], I),
        "mmod_vd_forward": ([P, P, P, P, P], I),
        "mmod_vd_set_kernel": ([P, I], I),
        "mmod_vd_uses_tma": ([P], I),
        "mmod_vd_set_option": ([P, I, I], I),
        "mmod_vd_last_loop_ms": ([P], ctypes.c_float),
        "mmod_vd_last_launch_count": ([P], ctypes.c_longlong),
        "mmod_vd_last_error": ([P], ctypes.c_char_p),
        "mmod_vd_get_plan": ([P, ctypes.POINTER(I)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _addr(x):
    """Address of a tensor / array / int (None -> NULL).  Keeps no copies."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(h, st: int):
    if st != 0:
        msg = load().mmod_last_error(h).decode() if h else ""
        raise MmodError(st, msg)


def mmod_cfl_dt(cfl: float, hmin: float, vmax: float) -> float:
    return load().mmod_cfl_dt(cfl, hmin, vmax)


def mmod_version() -> str:
    return load().mmod_version().decode()


def mmod_create(nx, ny, nz, h, dt, nt, *, nbl=0, src_ijk=None, rec_ijk=None, order=8,
                damp_R=1e-3, device=0, free_surface=False, cpml=False, cpml_f0=0.0):
    """Create a handle (ctypes void pointer).  src_ijk / rec_ijk: [n][3] int."""
    src = np.ascontiguousarray(np.zeros((0, 3)) if src_ijk is None else src_ijk, np.int32).reshape(-1, 3)
    rec = np.ascontiguousarray(np.zeros((0, 3)) if rec_ijk is None else rec_ijk, np.int32).reshape(-1, 3)
    cfg = _config(nx, ny, nz, h, dt, nt, nbl, src, rec, order, damp_R, free_surface, cpml, cpml_f0)
    out = ctypes.c_void_p()
    st = load().mmod_create(ctypes.byref(cfg), int(device), ctypes.byref(out))
    if st != 0:
        raise MmodError(st, load().mmod_last_error(None).decode())
    return out


def _config(nx, ny, nz, h, dt, nt, nbl, src, rec, order, damp_R, free_surface=False, cpml=False, cpml_f0=0.0):
    return _Config(int(nx), int(ny), int(nz), float(h[0]), float(h[1]), float(h[2]), float(dt), int(nt),
                   int(order), int(nbl), float(damp_R), len(src), src.ctypes.data if len(src) else None,
                   len(rec), rec.ctypes.data if len(rec) else None, int(bool(free_surface)),
                   BOUNDARY_CPML if cpml else BOUNDARY_DAMPING, float(cpml_f0))


def mmod_forward_noalloc(nx, ny, nz, h, dt, nt, vel, wavelet, traces, final_u=None, *, nbl=0,
                         src_ijk=None, rec_ijk=None, order=8, damp_R=1e-3, device=0, stream=None,
                         free_surface=False):
    """Allocation-free forward run (device pointers only; see include/mmod.h)."""
    src = np.ascontiguousarray(np.zeros((0, 3)) if src_ijk is None else src_ijk, np.int32).reshape(-1, 3)
    rec = np.ascontiguousarray(np.zeros((0, 3)) if rec_ijk is None else rec_ijk, np.int32).reshape(-1, 3)
    cfg = _config(nx, ny, nz, h, dt, nt, nbl, src, rec, order, damp_R, free_surface)
    st = load().mmod_forward_noalloc(ctypes.byref(cfg), int(device), _addr(vel), _addr(wavelet),
                                     _addr(traces), _addr(final_u), _stream(stream))
    if st != 0:
        raise MmodError(st, load().mmod_last_error(None).decode())


def mmod_destroy(h):
    _check(None, load().mmod_destroy(h))


def mmod_set_model(h, vel, stream=None):
    _check(h, load().mmod_set_model(h, _addr(vel), _stream(stream)))


def mmod_forward(h, wavelet, traces, final_u=None, stream=None):
    _check(h, load().mmod_forward(h, _addr(wavelet), _addr(traces), _addr(final_u), _stream(stream)))


def mmod_set_state(h, u_prev, u_cur, stream=None):
    _check(h, load().mmod_set_state(h, _addr(u_prev), _addr(u_cur), _stream(stream)))


def mmod_get_state(h, u_prev, u_cur, stream=None):
    _check(h, load().mmod_get_state(h, _addr(u_prev), _addr(u_cur), _stream(stream)))


def mmod_set_kernel(h, kernel: int):
    _check(h, load().mmod_set_kernel(h, int(kernel)))


def mmod_check_recip(n: int = 1 << 22) -> int:
    """Max ulp difference of the kernels' damping reciprocal vs __frcp_rn."""
    out = ctypes.c_uint(0)
    _check(None, load().mmod_check_recip(int(n), ctypes.byref(out)))
    return int(out.value)


def mmod_tma_variant_count() -> int:
    return int(load().mmod_tma_variant_count())


def mmod_tma_variant_name(v: int) -> str:
    return load().mmod_tma_variant_name(int(v)).decode()


def mmod_set_tma_variant(h, v: int):
    _check(h, load().mmod_set_tma_variant(h, int(v)))


def mmod_adjoint(h, resid, adj_src, stream=None):
    _check(h, load().mmod_adjoint(h, _addr(resid), _addr(adj_src), _stream(stream)))


def mmod_gradient(h, wavelet, resid, grad_v, ckpt_count, ckpt_dtype=0, stream=None):
    _check(h, load().mmod_gradient(h, _addr(wavelet), _addr(resid), _addr(grad_v), int(ckpt_count),
                                   int(ckpt_dtype), _stream(stream)))


def mmod_gradient_memory(h, ckpt_count, ckpt_dtype=0) -> int:
    return int(load().mmod_gradient_memory(h, int(ckpt_count), int(ckpt_dtype)))


def mmod_revolve_schedule(nsteps: int, snaps: int):
    """Binomial checkpointing schedule: (actions int32 [count][3] of
    {kind, a, b} with kind in REV_*, number of advanced steps).  Host only."""
    lib = load()
    count, adv = ctypes.c_longlong(), ctypes.c_longlong()
    st = lib.mmod_revolve_schedule(int(nsteps), int(snaps), None, 0, ctypes.byref(count), ctypes.byref(adv))
    if st != 0:
        raise MmodError(st, "mmod_revolve_schedule: invalid arguments")
    out = np.zeros((max(count.value, 1), 3), np.int32)
    st = lib.mmod_revolve_schedule(int(nsteps), int(snaps), out.ctypes.data, count.value, ctypes.byref(count),
                                   ctypes.byref(adv))
    if st != 0:
        raise MmodError(st, "mmod_revolve_schedule failed")
    return out[: count.value], int(adv.value)


def mmod_tma_variant_info(v: int) -> dict:
    """Threads, shared memory, registers, local bytes and residency of variant v's kernels."""
    out = (ctypes.c_int * 14)()
    st = load().mmod_tma_variant_info(int(v), out)
    if st != 0:
        raise MmodError(st, "mmod_tma_variant_info: variant out of range")
    keys = ("registers", "local_bytes", "static_smem", "ctas_per_sm")
    return {"threads": out[0], "dynamic_smem": out[1],
            **{k: dict(zip(keys, out[2 + 4 * i: 6 + 4 * i])) for i, k in enumerate(("step", "batch", "persistent"))}}


def mmod_optimized_coefficients(kmax: float) -> np.ndarray:
    """c_1..c_4 minimising the relative symbol error over kh in [0, kmax]."""
    out = np.zeros(4, np.float64)
    st = load().mmod_optimized_coefficients(float(kmax), out.ctypes.data)
    if st != 0:
        raise MmodError(st, "mmod_optimized_coefficients: kmax must be in (0, pi]")
    return out


def mmod_dot(a, b, n=None, stream=None) -> float:
    """FP64 dot product of two FP32 device arrays (computed by the library)."""
    out = ctypes.c_double(0.0)
    n = a.numel() if n is None else n
    st = load().mmod_dot(_addr(a), _addr(b), int(n), ctypes.byref(out), _stream(stream))
    if st != 0:
        raise MmodError(st, "mmod_dot failed")
    return float(out.value)


def mmod_set_option(h, option: int, value: int):
    _check(h, load().mmod_set_option(h, int(option), int(value)))


def mmod_get_plan(h) -> dict:
    out = (ctypes.c_int * 8)()
    _check(h, load().mmod_get_plan(h, out))
    keys = ["variant", "tiles_x", "tiles_y", "z_chunks", "planes_per_chunk", "grid", "block", "ctas_per_sm"]
    return dict(zip(keys, list(out)))


def mmod_last_error(h) -> str:
    return load().mmod_last_error(h).decode()


def mmod_last_launch_count(h) -> int:
    return int(load().mmod_last_launch_count(h))


def mmod_last_loop_ms(h) -> float:
    return float(load().mmod_last_loop_ms(h))


def mmod_autotune(h, steps=20, stream=None) -> int:
    v = ctypes.c_int(-1)
    _check(h, load().mmod_autotune(h, int(steps), _stream(stream), ctypes.byref(v)))
    return int(v.value)


class Batch:
    """Several propagators advanced together (one launch per step for all).
    Keeps references to the propagators so they outlive the batch."""

    def __init__(self, props):
        self.props = list(props)
        arr = (ctypes.c_void_p * len(self.props))(*[p.handle.value for p in self.props])
        out = ctypes.c_void_p()
        st = load().mmod_batch_create(arr, len(self.props), ctypes.byref(out))
        if st != 0:
            raise MmodError(st, load().mmod_last_error(None).decode())
        self.handle = out

    def _err(self, st):
        if st != 0:
            raise MmodError(st, load().mmod_batch_last_error(self.handle).decode())

    def forward(self, wavelets, traces, stream=None):
        n = len(self.props)
        w = (ctypes.c_void_p * n)(*[_addr(x) for x in wavelets])
        t = (ctypes.c_void_p * n)(*[_addr(x) for x in traces])
        self._err(load().mmod_batch_forward(self.handle, w, t, _stream(stream)))

    def set_variant(self, v: int):
        self._err(load().mmod_batch_set_variant(self.handle, int(v)))

    def set_mode(self, mode: int):
        """BATCH_STREAMS (default) or BATCH_FUSED."""
        self._err(load().mmod_batch_set_mode(self.handle, int(mode)))

    def autotune(self, steps=20, stream=None) -> int:
        v = ctypes.c_int(-1)
        self._err(load().mmod_batch_autotune(self.handle, int(steps), _stream(stream), ctypes.byref(v)))
        return int(v.value)

    def loop_ms(self) -> float:
        return float(load().mmod_batch_last_loop_ms(self.handle))

    def close(self):
        if self.handle is not None:
            load().mmod_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Propagator:
    """Owning wrapper around one handle for a given problem geometry."""

    def __init__(self, shape, h, dt, nt, *, nbl=0, src_ijk=None, rec_ijk=None, damp_R=1e-3,
                 device=0, order=8, free_surface=False, cpml=False, cpml_f0=0.0):
        nz, ny, nx = shape
        self.shape = tuple(shape)
        self.nt = int(nt)
        self.nsrc = 0 if src_ijk is None else len(np.asarray(src_ijk).reshape(-1, 3))
        self.nrec = 0 if rec_ijk is None else len(np.asarray(rec_ijk).reshape(-1, 3))
        self.device = device
        self.free_surface = bool(free_surface)
        self.handle = mmod_create(nx, ny, nz, h, dt, nt, nbl=nbl, src_ijk=src_ijk, rec_ijk=rec_ijk,
                                  order=order, damp_R=damp_R, device=device, free_surface=free_surface,
                                  cpml=cpml, cpml_f0=cpml_f0)

    @classmethod
    def from_problem(cls, p, device=0):
        return cls(p.vel.shape, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk,
                   damp_R=p.refl, device=device, order=p.order, free_surface=p.free_surface,
                   cpml=p.cpml, cpml_f0=p.cpml_f0)

    def set_model(self, vel, stream=None):
        mmod_set_model(self.handle, vel, stream)

    def set_kernel(self, kernel: int):
        mmod_set_kernel(self.handle, kernel)

    def set_variant(self, v: int):
        mmod_set_tma_variant(self.handle, v)

    def plan(self) -> dict:
        return mmod_get_plan(self.handle)

    def set_fd_coefficients(self, c4=None):
        """Laplacian weights c_1..c_4 (None: the Taylor weights)."""
        arr = None if c4 is None else np.ascontiguousarray(c4, np.float64).reshape(4)
        st = load().mmod_set_fd_coefficients(self.handle, None if arr is None else arr.ctypes.data)
        if st != 0:
            raise MmodError(st, load().mmod_last_error(self.handle).decode())

    def persistent_grid(self) -> int:
        """CTAs of the persistent kernel the next run launches (0: one launch per step)."""
        return int(load().mmod_persistent_grid(self.handle))

    def set_option(self, option: int, value: int):
        mmod_set_option(self.handle, option, value)

    def adjoint(self, resid, adj_src, stream=None):
        mmod_adjoint(self.handle, resid, adj_src, stream)

    def gradient(self, wavelet, resid, grad_v, ckpt_count, ckpt_dtype=0, stream=None):
        mmod_gradient(self.handle, wavelet, resid, grad_v, ckpt_count, ckpt_dtype, stream)

    def gradient_memory(self, ckpt_count, ckpt_dtype=0) -> int:
        return mmod_gradient_memory(self.handle, ckpt_count, ckpt_dtype)

    def autotune(self, steps=20, stream=None) -> int:
        return mmod_autotune(self.handle, steps, stream)

    def forward(self, wavelet, traces, final_u=None, stream=None):
        mmod_forward(self.handle, wavelet, traces, final_u, stream)

    def set_state(self, u_prev, u_cur, stream=None):
        mmod_set_state(self.handle, u_prev, u_cur, stream)

    def get_state(self, u_prev, u_cur, stream=None):
        mmod_get_state(self.handle, u_prev, u_cur, stream)

    @property
    def launches(self) -> int:
        return mmod_last_launch_count(self.handle)

    def loop_ms(self) -> float:
        return mmod_last_loop_ms(self.handle)

    def close(self):
        if self.handle is not None:
            mmod_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class StaggeredPropagator:
    """Owning wrapper around one variable-density (staggered-grid) handle:
    mmod_vd_create / mmod_vd_set_model / mmod_vd_forward.  Device tensors only."""

    def __init__(self, shape, h, dt, nt, *, nbl=0, src_ijk=None, rec_ijk=None, damp_R=1e-3,
                 device=0, cpml=False, cpml_f0=0.0, free_surface=False):
        nz, ny, nx = shape
        self.shape = tuple(shape)
        self.nt = int(nt)
        src = np.zeros((0, 3), np.int32) if src_ijk is None else np.ascontiguousarray(src_ijk, np.int32).reshape(-1, 3)
        rec = np.zeros((0, 3), np.int32) if rec_ijk is None else np.ascontiguousarray(rec_ijk, np.int32).reshape(-1, 3)
        self.nsrc, self.nrec = len(src), len(rec)
        self.device = device
        cfg = _config(nx, ny, nz, h, dt, nt, nbl, src, rec, 8, damp_R, free_surface, cpml, cpml_f0)
        out = ctypes.c_void_p()
        st = load().mmod_vd_create(ctypes.byref(cfg), device, ctypes.byref(out))
        if st != 0:
            raise MmodError(st, load().mmod_vd_last_error(None).decode())
        self.handle = out.value

    @classmethod
    def from_problem(cls, p, device=0):
        return cls(p.vel.shape, p.h, p.dt, p.nt, nbl=p.nbl, src_ijk=p.src_ijk, rec_ijk=p.rec_ijk,
                   damp_R=p.refl, device=device, cpml=p.cpml, cpml_f0=p.cpml_f0, free_surface=p.free_surface)

    def _check(self, st):
        if st != 0:
            raise MmodError(st, load().mmod_vd_last_error(self.handle).decode())

    def set_model(self, vel, rho, stream=None):
        self._check(load().mmod_vd_set_model(self.handle, _addr(vel), _addr(rho), _stream(stream)))

    def set_state(self, state, stream=None):
        """state [4][nz][ny][nx] device FP32: p^0, vx, vy, vz at -1/2 (None: zeros)."""
        self._check(load().mmod_vd_set_state(self.handle, _addr(state), _stream(stream)))

    def forward(self, wavelet, traces, final_state=None, stream=None):
        self._check(load().mmod_vd_forward(self.handle, _addr(wavelet), _addr(traces), _addr(final_state),
                                           _stream(stream)))

    def set_kernel(self, kernel: int):
        self._check(load().mmod_vd_set_kernel(self.handle, kernel))

    def set_option(self, option: int, value: int):
        self._check(load().mmod_vd_set_option(self.handle, option, value))

    @property
    def uses_tma(self) -> bool:
        return load().mmod_vd_uses_tma(self.handle) == 1

    def plan(self) -> dict:
        out = (ctypes.c_int * 6)()
        st = load().mmod_vd_get_plan(self.handle, out)
        if st not in (0, -7):
            self._check(st)
        return dict(zip(["tiles_x", "tiles_y", "z_chunks", "planes_per_chunk", "grid", "block"], list(out)))

    @property
    def launches(self) -> int:
        return int(load().mmod_vd_last_launch_count(self.handle))

    def loop_ms(self) -> float:
        return float(load().mmod_vd_last_loop_ms(self.handle))

    def close(self):
        if getattr(self, "handle", None) is not None:
            load().mmod_vd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
