"""FP64 CPU oracle for the Minimod acoustic isotropic constant-density propagator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it; the product path fails
loudly when its own extension is missing instead of falling back here.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over z); this module
only builds it with gcc and marshals numpy arrays through ctypes.  What each C
function follows in the paper (Eq. 1, Eq. 5, the Sec. 3 Laplacian, Alg. 1 and
Alg. 2) and the readings taken where the paper is silent are stated in the C
file's header.

Parity pins (tests/test_oracle_*.py): Taylor coefficients against the textbook
closed form and the moment identities; Laplacian exact on polynomials of degree
<= 9; the exact discrete standing wave (dispersion relation); discrete energy
conservation (damping off) and decay (damping on); the 3-D homogeneous Green's
function; a dense-matrix stepper on tiny grids; linearity, reciprocity and axis
permutation; for the variable-density staggered system (reading R18) the
staggered weights' closed form, exact staggered differences of polynomials,
the exact discrete standing wave, discrete energy identities, a dense stepper,
the Green's function and the reflection of a density contrast; for the adjoint the dot-product test <F w, r> = <w, F^T r> and a
dense transpose, for the gradient central finite differences of the misfit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no fused multiply-adds, so x86 and Arm hosts round alike.
_CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off"]


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle's C source into a shared library (gcc, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(src)):
            return out
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", *_CFLAGS, src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
        return out


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """ctypes binding of one build of oracle.c (the default one, or a variant)."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I, D = ctypes.c_int, ctypes.c_double
        lib.orc_fd_coeffs.argtypes = [I, P]
        lib.orc_damping_profile.argtypes = [I, I, D, D, D, P]
        lib.orc_laplacian.argtypes = [I, I, I, D, D, D, I, P, P, I, P]
        lib.orc_forward.argtypes = [I, I, I, D, D, D, D, I, I, I, D, P,
                                    I, P, P, I, P, P, P, P, P, P, I, I, P]
        lib.orc_optimized_coeffs.argtypes = [I, D, I, P]
        lib.orc_forward_cpml.argtypes = [I, I, I, D, D, D, D, I, I, D, D, P, I, P, P, I, P, P, P, I, I]
        lib.orc_staggered_coeffs.argtypes = [I, P]
        lib.orc_forward_vd.argtypes = [I, I, I, D, D, D, D, I, I, D, I, D, P, P, I, P, P, I, P, P, P, P, I, I]
        lib.orc_max_threads.argtypes = []
        lib.orc_adjoint.argtypes = [I, I, I, D, D, D, D, I, I, I, D, P, I, P, I, P, P, P, I, I]
        lib.orc_gradient.argtypes = [I, I, I, D, D, D, D, I, I, I, D, P, I, P, P, I, P, P, P, I, I]
        for f in (lib.orc_fd_coeffs, lib.orc_damping_profile, lib.orc_laplacian,
                  lib.orc_forward, lib.orc_max_threads, lib.orc_adjoint, lib.orc_gradient,
                  lib.orc_optimized_coeffs, lib.orc_forward_cpml, lib.orc_staggered_coeffs,
                  lib.orc_forward_vd):
            f.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def max_threads(self) -> int:
        return self.lib.orc_max_threads()

    def fd_coeffs(self, order: int) -> np.ndarray:
        """[c0, c1..cR]: centre weight and Taylor weights of Sec. 3 (unit spacing)."""
        out = np.zeros(max(order // 2, 0) + 1, dtype=np.float64)
        rc = self.lib.orc_fd_coeffs(order, _ptr(out))
        if rc != 0:
            raise ValueError(f"orc_fd_coeffs(order={order}) -> {rc}")
        return out

    def optimized_coeffs(self, order: int, kmax: float, nq: int = 4000) -> np.ndarray:
        """[c0, c1..cR] of reading R16: least-squares weights over kh in [0, kmax]
        with sum m^2 c_m = 1 (unit spacing)."""
        out = np.zeros(order // 2 + 1, dtype=np.float64)
        rc = self.lib.orc_optimized_coeffs(order, float(kmax), int(nq), _ptr(out))
        if rc != 0:
            raise ValueError(f"orc_optimized_coeffs -> {rc}")
        return out

    def damping_profile(self, n: int, nbl: int, h: float, vmax: float, refl: float = 1e-3) -> np.ndarray:
        """eta_a(i), i = 0..n-1, of the damping layers (reading R3)."""
        out = np.zeros(n, dtype=np.float64)
        rc = self.lib.orc_damping_profile(n, nbl, h, vmax, refl, _ptr(out))
        if rc != 0:
            raise ValueError(f"orc_damping_profile -> {rc}")
        return out

    def laplacian(self, u: np.ndarray, h, order: int = 8, free_surface: bool = False, coef=None) -> np.ndarray:
        """Sec. 3 Laplacian of u [nz][ny][nx] with u = 0 outside the grid (with
        free_surface, the odd image of reading R15 above k = 0)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        nz, ny, nx = u.shape
        hx, hy, hz = h
        out = np.empty_like(u)
        cf = None if coef is None else np.ascontiguousarray(coef, np.float64)
        rc = self.lib.orc_laplacian(nx, ny, nz, hx, hy, hz, order, _ptr(u), _ptr(out), int(free_surface),
                                    _ptr(cf))
        if rc != 0:
            raise ValueError(f"orc_laplacian -> {rc}")
        return out

    def forward(self, vel: np.ndarray, h, dt: float, nt: int, *, order: int = 8, nbl: int = 0,
                refl: float = 1e-3, src_ijk=None, wavelet=None, rec_ijk=None,
                u_prev0=None, u_cur0=None, want_state: bool = False, nthreads: int = 0,
                free_surface: bool = False, coef=None):
        """Alg. 1 / Alg. 2 forward run in FP64 (free_surface: reading R15; coef:
        c_1..c_R of the Laplacian instead of the Taylor weights, reading R16).

        vel: [nz][ny][nx] float32 m/s.  src_ijk: [nsrc][3] (i, j, k).  wavelet:
        [nsrc][nt] float32.  rec_ijk: [nrec][3].  Returns traces [nt][nrec]
        (FP64) and, with want_state, also (u^{nt-1}, u^{nt}).
        """
        vel = np.ascontiguousarray(vel, dtype=np.float32)
        nz, ny, nx = vel.shape
        hx, hy, hz = h
        src = (np.zeros((0, 3), np.int32) if src_ijk is None
               else np.ascontiguousarray(src_ijk, np.int32).reshape(-1, 3))
        rec = (np.zeros((0, 3), np.int32) if rec_ijk is None
               else np.ascontiguousarray(rec_ijk, np.int32).reshape(-1, 3))
        nsrc, nrec = src.shape[0], rec.shape[0]
        wav = np.ascontiguousarray(wavelet, np.float32).reshape(nsrc, nt) if nsrc else None
        traces = np.zeros((nt, nrec), dtype=np.float64)
        up0 = None if u_prev0 is None else np.ascontiguousarray(u_prev0, np.float64)
        uc0 = None if u_cur0 is None else np.ascontiguousarray(u_cur0, np.float64)
        upo = np.empty(vel.shape, np.float64) if want_state else None
        uco = np.empty(vel.shape, np.float64) if want_state else None
        rc = self.lib.orc_forward(nx, ny, nz, hx, hy, hz, dt, nt, order, nbl, refl, _ptr(vel),
                                  nsrc, _ptr(src) if nsrc else None, _ptr(wav),
                                  nrec, _ptr(rec) if nrec else None, _ptr(traces) if nrec else None,
                                  _ptr(up0), _ptr(uc0), _ptr(upo), _ptr(uco), nthreads, int(free_surface),
                                  _ptr(None if coef is None else np.ascontiguousarray(coef, np.float64)))
        if rc != 0:
            raise ValueError(f"orc_forward -> {rc}")
        if want_state:
            return traces, upo, uco
        return traces


    def forward_cpml(self, vel, h, dt, nt, *, nbl=0, refl=1e-3, f0=0.0, src_ijk=None, wavelet=None,
                     rec_ijk=None, want_state=False, nthreads=0, free_surface=False):
        """Reading R17: forward run with CPML layers (order 8).  Returns traces
        [nt][nrec] and, with want_state, also u^{nt}."""
        vel = np.ascontiguousarray(vel, dtype=np.float32)
        nz, ny, nx = vel.shape
        src = (np.zeros((0, 3), np.int32) if src_ijk is None
               else np.ascontiguousarray(src_ijk, np.int32).reshape(-1, 3))
        rec = (np.zeros((0, 3), np.int32) if rec_ijk is None
               else np.ascontiguousarray(rec_ijk, np.int32).reshape(-1, 3))
        nsrc, nrec = src.shape[0], rec.shape[0]
        wav = np.ascontiguousarray(wavelet, np.float32).reshape(nsrc, nt) if nsrc else None
        traces = np.zeros((nt, nrec), np.float64)
        uco = np.empty(vel.shape, np.float64) if want_state else None
        rc = self.lib.orc_forward_cpml(nx, ny, nz, h[0], h[1], h[2], dt, nt, nbl, refl, f0, _ptr(vel),
                                       nsrc, _ptr(src) if nsrc else None, _ptr(wav),
                                       nrec, _ptr(rec) if nrec else None, _ptr(traces) if nrec else None,
                                       _ptr(uco), nthreads, int(free_surface))
        if rc != 0:
            raise ValueError(f"orc_forward_cpml -> {rc}")
        return (traces, uco) if want_state else traces

    def staggered_coeffs(self, order: int) -> np.ndarray:
        """[0, a_1..a_R]: staggered first-derivative weights (reading R18, unit spacing)."""
        out = np.zeros(order // 2 + 1, dtype=np.float64)
        rc = self.lib.orc_staggered_coeffs(order, _ptr(out))
        if rc != 0:
            raise ValueError(f"orc_staggered_coeffs(order={order}) -> {rc}")
        return out

    def forward_vd(self, vel, rho, h, dt, nt, *, nbl=0, refl=1e-3, cpml=False, f0=0.0, src_ijk=None,
                   wavelet=None, rec_ijk=None, state0=None, want_state=False, nthreads=0, free_surface=False):
        """Reading R18: variable-density first-order system on the staggered
        grid (order 8), damping layers or (cpml) CPML layers, optionally a
        free surface at k = 0.

        vel, rho: [nz][ny][nx] float32.  state0: optional [4][nz][ny][nx]
        (p^0, vx, vy, vz at -1/2).  Returns traces [nt][nrec] (p^{n+1} at the
        receivers) and, with want_state, the final [4][nz][ny][nx] state
        (p^{nt}, velocities at nt - 1/2).
        """
        vel = np.ascontiguousarray(vel, dtype=np.float32)
        rho = np.ascontiguousarray(rho, dtype=np.float32)
        assert rho.shape == vel.shape
        nz, ny, nx = vel.shape
        src = (np.zeros((0, 3), np.int32) if src_ijk is None
               else np.ascontiguousarray(src_ijk, np.int32).reshape(-1, 3))
        rec = (np.zeros((0, 3), np.int32) if rec_ijk is None
               else np.ascontiguousarray(rec_ijk, np.int32).reshape(-1, 3))
        nsrc, nrec = src.shape[0], rec.shape[0]
        wav = np.ascontiguousarray(wavelet, np.float32).reshape(nsrc, nt) if nsrc else None
        traces = np.zeros((nt, nrec), np.float64)
        s0 = None if state0 is None else np.ascontiguousarray(state0, np.float64).reshape(4, nz, ny, nx)
        so = np.empty((4, nz, ny, nx), np.float64) if want_state else None
        rc = self.lib.orc_forward_vd(nx, ny, nz, h[0], h[1], h[2], dt, nt, nbl, refl, int(bool(cpml)), f0,
                                     _ptr(vel), _ptr(rho), nsrc, _ptr(src) if nsrc else None, _ptr(wav),
                                     nrec, _ptr(rec) if nrec else None, _ptr(traces) if nrec else None,
                                     _ptr(s0), _ptr(so), nthreads, int(bool(free_surface)))
        if rc != 0:
            raise ValueError(f"orc_forward_vd -> {rc}")
        return (traces, so) if want_state else traces

    def adjoint(self, vel, h, dt, nt, *, order=8, nbl=0, refl=1e-3, src_ijk=None, rec_ijk=None,
                resid=None, nthreads=0, free_surface=False):
        """Transpose of the forward map wavelet -> traces: resid [nt][nrec] ->
        adjoint source [nsrc][nt] (FP64)."""
        vel = np.ascontiguousarray(vel, dtype=np.float32)
        nz, ny, nx = vel.shape
        src = np.ascontiguousarray(src_ijk, np.int32).reshape(-1, 3)
        rec = np.ascontiguousarray(rec_ijk, np.int32).reshape(-1, 3)
        r = np.ascontiguousarray(resid, np.float64).reshape(nt, len(rec))
        adj = np.zeros((len(src), nt), np.float64)
        rc = self.lib.orc_adjoint(nx, ny, nz, h[0], h[1], h[2], dt, nt, order, nbl, refl, _ptr(vel),
                                  len(src), _ptr(src), len(rec), _ptr(rec), _ptr(r), _ptr(adj), nthreads,
                                  int(free_surface))
        if rc != 0:
            raise ValueError(f"orc_adjoint -> {rc}")
        return adj

    def gradient(self, vel, h, dt, nt, *, order=8, nbl=0, refl=1e-3, src_ijk=None, wavelet=None,
                 rec_ijk=None, resid=None, nthreads=0, free_surface=False):
        """dJ/dv for J = 1/2 sum |traces - d_obs|^2 given resid = traces - d_obs
        ([nt][nrec]); returns [nz][ny][nx] FP64.  Stores every forward state:
        small grids only."""
        vel = np.ascontiguousarray(vel, dtype=np.float32)
        nz, ny, nx = vel.shape
        src = np.ascontiguousarray(src_ijk, np.int32).reshape(-1, 3)
        rec = np.ascontiguousarray(rec_ijk, np.int32).reshape(-1, 3)
        wav = np.ascontiguousarray(wavelet, np.float32).reshape(len(src), nt)
        r = np.ascontiguousarray(resid, np.float64).reshape(nt, len(rec))
        g = np.zeros(vel.shape, np.float64)
        rc = self.lib.orc_gradient(nx, ny, nz, h[0], h[1], h[2], dt, nt, order, nbl, refl, _ptr(vel),
                                   len(src), _ptr(src), _ptr(wav), len(rec), _ptr(rec), _ptr(r), _ptr(g),
                                   nthreads, int(free_surface))
        if rc != 0:
            raise ValueError(f"orc_gradient -> {rc}")
        return g


def _default() -> Oracle:
    global _lib
    if _lib is None:
        _lib = Oracle(build())
    return _lib


def max_threads() -> int:
    return _default().max_threads()


def fd_coeffs(order: int) -> np.ndarray:
    return _default().fd_coeffs(order)


def damping_profile(n: int, nbl: int, h: float, vmax: float, refl: float = 1e-3) -> np.ndarray:
    return _default().damping_profile(n, nbl, h, vmax, refl)


def forward_cpml(vel, h, dt, nt, **kw):
    return _default().forward_cpml(vel, h, dt, nt, **kw)


def staggered_coeffs(order: int) -> np.ndarray:
    return _default().staggered_coeffs(order)


def forward_vd(vel, rho, h, dt, nt, **kw):
    return _default().forward_vd(vel, rho, h, dt, nt, **kw)


forward_vd.__doc__ = Oracle.forward_vd.__doc__


def optimized_coeffs(order: int, kmax: float, nq: int = 4000) -> np.ndarray:
    return _default().optimized_coeffs(order, kmax, nq)


def laplacian(u: np.ndarray, h, order: int = 8, free_surface: bool = False, coef=None) -> np.ndarray:
    return _default().laplacian(u, h, order, free_surface, coef)


def forward(vel, h, dt, nt, **kw):
    return _default().forward(vel, h, dt, nt, **kw)


forward.__doc__ = Oracle.forward.__doc__


def adjoint(vel, h, dt, nt, **kw):
    return _default().adjoint(vel, h, dt, nt, **kw)


def gradient(vel, h, dt, nt, **kw):
    return _default().gradient(vel, h, dt, nt, **kw)


adjoint.__doc__ = Oracle.adjoint.__doc__
gradient.__doc__ = Oracle.gradient.__doc__
