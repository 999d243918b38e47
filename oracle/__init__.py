"""FP64 CPU oracle of the Jacobi-PCG hot path (arxiv 2603.23343, Sec. IV-VII).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain double-precision loops); this
module compiles it with gcc on first use (or via :func:`build`) and wraps it
with numpy-in / numpy-out functions.  Arrays are (nz, ny, nx), x fastest.

Parity status of each function (what pins it, see ``tests/test_oracle.py``):
  apply_poisson   sine eigenpairs, quadratic manufactured solution, 4^3 dense
                  symmetry / Cholesky / full spectrum
  apply_varcoeff  k == c reduces to c * Poisson, energy identity u.Au =
                  sum over faces, dense symmetry / Cholesky
  dot, axpy       integer-valued closed forms, exact rational sums
  pcg             exact termination on m sine modes, manufactured solution,
                  scipy.sparse.linalg.cg on the assembled matrix
  refine          reaches tolerances below the inner tolerance; agrees with a
                  dense direct solve
  csr_apply       the Kronecker-assembled Poisson matrix reproduces the
                  matrix-free operator; a random sparse matrix agrees with a
                  dense product
  csr_pcg         the same iterates as pcg on the assembled Poisson matrix;
                  scipy's CG on a random sparse SPD matrix; exact
                  termination in m steps on a diagonal matrix with m
                  distinct entries
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, NOT_CONVERGED, BREAKDOWN = 0, 3, 4


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.c_double
            I = ctypes.c_int
            L = ctypes.c_int64
            P = ctypes.c_void_p
            lib.orc_dot.restype = D
            lib.orc_dot.argtypes = [L, P, P]
            lib.orc_axpy.restype = None
            lib.orc_axpy.argtypes = [L, D, P, P]
            lib.orc_apply.restype = None
            lib.orc_apply.argtypes = [I, I, I, P, I, I, I, P, P]
            lib.orc_diag.restype = None
            lib.orc_diag.argtypes = [I, I, I, P, I, I, I, P]
            lib.orc_residual.restype = None
            lib.orc_residual.argtypes = [I, I, I, P, I, I, I, P, P, P]
            lib.orc_pcg.restype = I
            lib.orc_pcg.argtypes = [I, I, I, P, I, I, I, P, P, D, I, I, P, P, P]
            lib.orc_true_relres.restype = D
            lib.orc_true_relres.argtypes = [I, I, I, P, I, I, I, P, P]
            lib.orc_csr_apply.restype = None
            lib.orc_csr_apply.argtypes = [L, P, P, P, P, P]
            lib.orc_csr_pcg.restype = I
            lib.orc_csr_pcg.argtypes = [L, P, P, P, P, P, D, I, P, P, P]
            lib.orc_threads.restype = I
            lib.orc_threads.argtypes = []
            lib.orc_refine.restype = I
            lib.orc_refine.argtypes = [I, I, I, P, I, I, I, P, P, D, I, D, I, P, P]
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _kargs(k, kb):
    """(pointer, kbx, kby, kbz, keepalive) for an optional block-coefficient array."""
    if k is None:
        return None, 1, 1, 1, None
    kk = _f64(k)
    if isinstance(kb, int):
        kb = (kb, kb, kb)
    return _ptr(kk), int(kb[0]), int(kb[1]), int(kb[2]), kk


def dot(x, y) -> float:
    x, y = _f64(x).ravel(), _f64(y).ravel()
    assert x.size == y.size
    return float(_load().orc_dot(x.size, _ptr(x), _ptr(y)))


def axpy(alpha: float, x, y) -> np.ndarray:
    """Returns alpha*x + y (new array)."""
    x, out = _f64(x).ravel(), _f64(y).ravel().copy()
    assert x.size == out.size
    _load().orc_axpy(x.size, float(alpha), _ptr(x), _ptr(out))
    return out.reshape(np.shape(y))


def apply(u, k=None, kb=8) -> np.ndarray:
    """A u on the grid of ``u.shape`` = (nz, ny, nx); Poisson when k is None."""
    u = _f64(u)
    nz, ny, nx = u.shape
    out = np.empty_like(u)
    kp, kbx, kby, kbz, _keep = _kargs(k, kb)
    _load().orc_apply(nx, ny, nz, kp, kbx, kby, kbz, _ptr(u), _ptr(out))
    return out


def apply_poisson(u) -> np.ndarray:
    return apply(u)


def apply_varcoeff(u, k, kb=8) -> np.ndarray:
    return apply(u, k, kb)


def diag(shape, k=None, kb=8) -> np.ndarray:
    nz, ny, nx = shape
    out = np.empty(shape, dtype=np.float64)
    kp, kbx, kby, kbz, _keep = _kargs(k, kb)
    _load().orc_diag(nx, ny, nz, kp, kbx, kby, kbz, _ptr(out))
    return out


def residual(b, x, k=None, kb=8) -> np.ndarray:
    b, x = _f64(b), _f64(x)
    nz, ny, nx = b.shape
    out = np.empty_like(b)
    kp, kbx, kby, kbz, _keep = _kargs(k, kb)
    _load().orc_residual(nx, ny, nz, kp, kbx, kby, kbz, _ptr(b), _ptr(x), _ptr(out))
    return out


def true_relres(b, x, k=None, kb=8) -> float:
    b, x = _f64(b), _f64(x)
    nz, ny, nx = b.shape
    kp, kbx, kby, kbz, _keep = _kargs(k, kb)
    return float(_load().orc_true_relres(nx, ny, nz, kp, kbx, kby, kbz, _ptr(b), _ptr(x)))


def _csr(row_ptr, col, val):
    return (np.ascontiguousarray(row_ptr, dtype=np.int64), np.ascontiguousarray(col, dtype=np.int32), _f64(val))


def csr_apply(row_ptr, col, val, x) -> np.ndarray:
    """y = A x for a CSR matrix (row_ptr int64 n+1, col int32, val float64)."""
    rp, cc, vv = _csr(row_ptr, col, val)
    x = _f64(x).ravel()
    y = np.empty_like(x)
    _load().orc_csr_apply(len(rp) - 1, _ptr(rp), _ptr(cc), _ptr(vv), _ptr(x), _ptr(y))
    return y


def csr_pcg(row_ptr, col, val, b, x0=None, tol=1e-6, maxit=2000, history=False):
    """Jacobi-PCG on a CSR matrix (the iteration of pcg with a general operator).
    Returns dict(x, iters, relres, status[, hist])."""
    rp, cc, vv = _csr(row_ptr, col, val)
    b = _f64(b).ravel()
    x = np.zeros_like(b) if x0 is None else _f64(x0).ravel().copy()
    hist = np.zeros(maxit + 1, dtype=np.float64)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _load().orc_csr_pcg(len(rp) - 1, _ptr(rp), _ptr(cc), _ptr(vv), _ptr(b), _ptr(x), float(tol), int(maxit),
                             _ptr(hist), ctypes.byref(it), ctypes.byref(rel))
    out = dict(x=x, iters=it.value, relres=rel.value, status=st)
    if history:
        out["hist"] = hist[: it.value + 1].copy()
    return out


def threads() -> int:
    """Threads the oracle's parallel loops run on."""
    return int(_load().orc_threads())


def pcg(b, x0=None, tol=1e-6, maxit=2000, k=None, kb=8, precond="jacobi", history=False):
    """Jacobi-PCG (or plain CG with precond=None).

    Returns dict(x, iters, relres, status[, hist]).
    """
    b = _f64(b)
    nz, ny, nx = b.shape
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    hist = np.zeros(maxit + 1, dtype=np.float64)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    kp, kbx, kby, kbz, _keep = _kargs(k, kb)
    pc = 0 if precond == "jacobi" else -1
    st = _load().orc_pcg(nx, ny, nz, kp, kbx, kby, kbz, _ptr(b), _ptr(x), float(tol), int(maxit), pc,
                         _ptr(hist), ctypes.byref(it), ctypes.byref(rel))
    out = dict(x=x, iters=it.value, relres=rel.value, status=st)
    if history:
        out["hist"] = hist[: it.value + 1].copy()
    return out


def refine(b, x0=None, tol=1e-8, max_outer=30, inner_tol=1e-2, inner_maxit=1000, k=None, kb=8):
    """FP64 iterative refinement around inner Jacobi-PCG solves."""
    b = _f64(b)
    nz, ny, nx = b.shape
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    rel = ctypes.c_double(0.0)
    tot = ctypes.c_int(0)
    kp, kbx, kby, kbz, _keep = _kargs(k, kb)
    steps = _load().orc_refine(nx, ny, nz, kp, kbx, kby, kbz, _ptr(b), _ptr(x), float(tol),
                               int(max_outer), float(inner_tol), int(inner_maxit),
                               ctypes.byref(rel), ctypes.byref(tot))
    return dict(x=x, steps=steps, relres=rel.value, inner_iters=tot.value)
