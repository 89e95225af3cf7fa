"""Nekbone oracle: numpy wrapper around the plain C FP64 reference.

TEST INFRASTRUCTURE ONLY.  The oracle defines what the CUDA library must
compute (arXiv 2005.13425, Sec. III: SEM Poisson on a cubic domain solved by
CG; Listing 1: the element-local tensor-product operator ax_e; Eq. 1-2: the
cost model).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA path and never imports it.

Every function follows the C routine of the same name in
``nekbone_oracle.c``, whose comments cite the passage each one restates.
All pins (the checks that tie each function to the paper and to mathematics
rather than to itself) live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nekbone_oracle.c")
_LIB = os.path.join(_HERE, "libnbo.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libnbo.so`` with gcc (plain C99,
    no FMA contraction, OpenMP only for the independent element loop)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu99", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.nbo_gll.argtypes = [ctypes.c_int, _dp, _dp]
            lib.nbo_dmat.argtypes = [ctypes.c_int, _dp, _dp]
            lib.nbo_box_coords.argtypes = [ctypes.c_int] * 4 + [_dp, ctypes.c_double, _dp, _dp]
            lib.nbo_geom.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            lib.nbo_ax_e.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
            lib.nbo_ax_e.restype = None
            lib.nbo_gid.argtypes = [ctypes.c_int] * 4 + [_i64p]
            lib.nbo_gid.restype = None
            lib.nbo_multiplicity.argtypes = [ctypes.c_int] * 4 + [_i32p]
            lib.nbo_multiplicity.restype = None
            lib.nbo_mask.argtypes = [ctypes.c_int] * 4 + [_u8p]
            lib.nbo_mask.restype = None
            lib.nbo_dssum.argtypes = [ctypes.c_int] * 4 + [_dp]
            lib.nbo_dssum.restype = None
            lib.nbo_apply_mask.argtypes = [ctypes.c_long, _u8p, _dp]
            lib.nbo_apply_mask.restype = None
            lib.nbo_dot_c.argtypes = [ctypes.c_int] * 4 + [_dp, _dp]
            lib.nbo_dot_c.restype = ctypes.c_double
            lib.nbo_apply_A.argtypes = [ctypes.c_int] * 4 + [_dp, _dp, _u8p, _dp, _dp]
            lib.nbo_apply_A.restype = None
            lib.nbo_cg.argtypes = ([ctypes.c_int] * 4 + [_dp, _dp, _u8p, _dp, _dp,
                                   ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int), _dp, _dp])
            lib.nbo_diag_e.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            lib.nbo_diag_e.restype = None
            lib.nbo_jacobi_inverse.argtypes = [ctypes.c_int] * 4 + [_dp, _dp, _u8p, _dp]
            lib.nbo_jacobi_inverse.restype = None
            lib.nbo_pcg.argtypes = ([ctypes.c_int] * 4 + [_dp, _dp, _u8p, _dp, _dp, _dp,
                                    ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int), _dp, _dp])
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- C1, C2
def gll(n: int):
    """GLL nodes xi (ascending, xi_0=-1, xi_N=1) and weights w, n points."""
    xi = np.empty(n)
    w = np.empty(n)
    if _load().nbo_gll(n, _d(xi), _d(w)) != 0:
        raise ValueError("n must be >= 2")
    return xi, w


def dmat(xi) -> np.ndarray:
    """Derivative matrix D[i, l] = dxm1(i, l) = l_l'(xi_i), shape (n, n)."""
    xi = _c(xi)
    n = xi.size
    D = np.empty((n, n))
    _load().nbo_dmat(n, _d(xi), _d(D))
    return D


# ---------------------------------------------------------------- C3
def box_coords(Ex, Ey, Ez, n, amp=0.05, s=(0.0, 0.0, 0.0)):
    """Nodal coordinates xyz[E, 3, n^3] of the perturbed unit-cube box."""
    xi, _ = gll(n)
    E = Ex * Ey * Ez
    xyz = np.empty((E, 3, n ** 3))
    _load().nbo_box_coords(Ex, Ey, Ez, n, _d(xi), float(amp), _d(_c(s)), _d(xyz))
    return xyz


def geom(n, xyz, D=None, w=None):
    """gxyz[E, 6, n^3] (rr, rs, rt, ss, st, tt) and detJ[E, n^3]."""
    xyz = _c(xyz)
    E = xyz.shape[0]
    if D is None or w is None:
        xi, w = gll(n)
        D = dmat(xi)
    gxyz = np.empty((E, 6, n ** 3))
    detJ = np.empty((E, n ** 3))
    rc = _load().nbo_geom(E, n, _d(_c(D)), _d(_c(w)), _d(xyz), _d(gxyz), _d(detJ))
    if rc != 0:
        raise ValueError("non-positive Jacobian in the mesh")
    return gxyz, detJ


# ---------------------------------------------------------------- C4
def ax_e(D, gxyz, u) -> np.ndarray:
    """Element-local Poisson operator of Listing 1; u, w in [E][n^3]."""
    D = _c(D)
    n = D.shape[0]
    gxyz = _c(gxyz)
    E = gxyz.size // (6 * n ** 3)
    u = _c(u).reshape(E, n ** 3)
    w = np.empty_like(u)
    _load().nbo_ax_e(E, n, _d(D), _d(gxyz), _d(u), _d(w))
    return w


# ---------------------------------------------------------------- C5
def gid(Ex, Ey, Ez, n):
    out = np.empty((Ex * Ey * Ez, n ** 3), dtype=np.int64)
    _load().nbo_gid(Ex, Ey, Ez, n, out.ctypes.data_as(_i64p))
    return out


def multiplicity(Ex, Ey, Ez, n):
    out = np.empty((Ex * Ey * Ez, n ** 3), dtype=np.int32)
    _load().nbo_multiplicity(Ex, Ey, Ez, n, out.ctypes.data_as(_i32p))
    return out


def mask(Ex, Ey, Ez, n):
    out = np.empty((Ex * Ey * Ez, n ** 3), dtype=np.uint8)
    _load().nbo_mask(Ex, Ey, Ez, n, out.ctypes.data_as(_u8p))
    return out


def dssum(Ex, Ey, Ez, n, w):
    out = _c(w).copy()
    _load().nbo_dssum(Ex, Ey, Ez, n, _d(out))
    return out


def apply_mask(msk, w):
    out = _c(w).copy()
    _load().nbo_apply_mask(out.size, _c(msk, np.uint8).ctypes.data_as(_u8p), _d(out))
    return out


def dot_c(Ex, Ey, Ez, n, a, b) -> float:
    return float(_load().nbo_dot_c(Ex, Ey, Ez, n, _d(_c(a)), _d(_c(b))))


def apply_A(Ex, Ey, Ez, n, D, gxyz, msk, u):
    """Assembled operator mask(dssum(ax_e(u)))."""
    u = _c(u)
    w = np.empty_like(u)
    _load().nbo_apply_A(Ex, Ey, Ez, n, _d(_c(D)), _d(_c(gxyz)),
                        _c(msk, np.uint8).ctypes.data_as(_u8p), _d(u), _d(w))
    return w


# ---------------------------------------------------------------- C6
def cg(Ex, Ey, Ez, n, D, gxyz, msk, f, x0=None, tol=0.0, maxit=100):
    """Unpreconditioned CG.  Returns (x, iters, relres, rho_hist, status)."""
    f = _c(f)
    x = np.zeros_like(f) if x0 is None else _c(x0).copy()
    hist = np.zeros(maxit + 1)
    iters = ctypes.c_int(0)
    relres = ctypes.c_double(0.0)
    st = _load().nbo_cg(Ex, Ey, Ez, n, _d(_c(D)), _d(_c(gxyz)),
                        _c(msk, np.uint8).ctypes.data_as(_u8p), _d(f), _d(x),
                        float(tol), int(maxit), ctypes.byref(iters),
                        ctypes.byref(relres), _d(hist))
    return x, iters.value, relres.value, hist[: iters.value + 1].copy(), st


def diag_e(D, gxyz):
    """Diagonal of every element matrix of Listing 1, [E][n^3]."""
    D = _c(D)
    n = D.shape[0]
    gxyz = _c(gxyz)
    E = gxyz.size // (6 * n ** 3)
    out = np.empty((E, n ** 3))
    _load().nbo_diag_e(E, n, _d(D), _d(gxyz), _d(out))
    return out


def jacobi_inverse(Ex, Ey, Ez, n, D, gxyz, msk):
    """1 / dssum(diag_e) at unmasked points, 0 at Dirichlet points."""
    E = Ex * Ey * Ez
    out = np.empty((E, n ** 3))
    _load().nbo_jacobi_inverse(Ex, Ey, Ez, n, _d(_c(D)), _d(_c(gxyz)),
                               _c(msk, np.uint8).ctypes.data_as(_u8p), _d(out))
    return out


def pcg(Ex, Ey, Ez, n, D, gxyz, msk, minv, f, x0=None, tol=0.0, maxit=100):
    """Jacobi PCG.  Returns (x, iters, relres, rr_hist, status)."""
    f = _c(f)
    x = np.zeros_like(f) if x0 is None else _c(x0).copy()
    hist = np.zeros(maxit + 1)
    iters = ctypes.c_int(0)
    relres = ctypes.c_double(0.0)
    st = _load().nbo_pcg(Ex, Ey, Ez, n, _d(_c(D)), _d(_c(gxyz)),
                         _c(msk, np.uint8).ctypes.data_as(_u8p), _d(_c(minv)), _d(f), _d(x),
                         float(tol), int(maxit), ctypes.byref(iters), ctypes.byref(relres), _d(hist))
    return x, iters.value, relres.value, hist[: iters.value + 1].copy(), st


# ---------------------------------------------------------------- problems
def box_problem(Ex, Ey, Ez, n, amp=0.05, s=(0.0, 0.0, 0.0)):
    """Everything the Nekbone box problem needs, built by the oracle:
    GLL nodes/weights, D, coordinates, gxyz, detJ, mask, multiplicity, gid."""
    xi, w = gll(n)
    D = dmat(xi)
    xyz = box_coords(Ex, Ey, Ez, n, amp, s)
    gxyz, detJ = geom(n, xyz, D, w)
    return dict(Ex=Ex, Ey=Ey, Ez=Ez, n=n, E=Ex * Ey * Ez, xi=xi, w=w, D=D,
                xyz=xyz, gxyz=gxyz, detJ=detJ, mask=mask(Ex, Ey, Ez, n),
                mult=multiplicity(Ex, Ey, Ez, n), gid=gid(Ex, Ey, Ez, n))


def scatter_unique(Ex, Ey, Ez, n, values_unique):
    """Local copies of a field given per unique global node (u_L = Q u_G)."""
    g = gid(Ex, Ey, Ez, n)
    return _c(values_unique)[g]
