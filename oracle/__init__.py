"""CPU FP64 oracle for the domain-wall operator -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. The product library (``paper_2112_01852_gb300``)
never imports, links or executes anything here, and this package imports
nothing from it.

``dw_oracle.cpp`` is a plain C++ implementation written from the operator's
definition (4x4 spin matrices, 3x3 colour matrices, std::complex<double>);
``dense.py`` builds the same operators as explicit dense matrices with numpy
for small lattices; ``eo.py`` writes the even-odd Schur complement and its
solve out of this package's Dhop and K with numpy. All follow the standard
domain-wall operator, which the
paper names (the "Domain Wall kernel", Sec. 4.1; its per-site work and flop
count, Table 3) without writing it down.

All fields are complex128 numpy arrays in the canonical layout:
  fermion (nrhs, V4, Ls, 4, 3), gauge (V4, 4, 3, 3),
  x4 = x + Lx*(y + Ly*(z + Lz*t)), U_mu(x) links x to x + mu.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dw_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

DEFAULT_BC = (1, 1, 1, -1)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ -fopenmp (seconds)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c++17", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            L = ctypes.c_long
            D = ctypes.c_double
            lib.oracle_dhop.argtypes = [P, P, P, P, I, I, P, I, P, L]
            lib.oracle_k.argtypes = [P, P, P, I, I, P, I]
            lib.oracle_dw.argtypes = [P, P, P, P, I, I, P, D, D, D, P, I, P, L]
            lib.oracle_dwdagdw.argtypes = [P, P, P, P, I, I, P, D, D, D, P]
            lib.oracle_cg.argtypes = [P, P, P, P, I, I, P, D, D, D, P, D, I, P, P]
            lib.oracle_num_threads.argtypes = []
            for f in (lib.oracle_dhop, lib.oracle_k, lib.oracle_dw, lib.oracle_dwdagdw,
                      lib.oracle_cg, lib.oracle_num_threads):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    return _load().oracle_num_threads()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _fermion(psi, V4, Ls):
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    if psi.ndim == 4:
        psi = psi[None]
    if psi.shape[1:] != (V4, Ls, 4, 3):
        raise ValueError("fermion shape %s does not match V4=%d Ls=%d" % (psi.shape, V4, Ls))
    return psi


def _common(dims, bc):
    d = np.ascontiguousarray(dims, dtype=np.int32)
    b = np.ascontiguousarray(DEFAULT_BC if bc is None else bc, dtype=np.int32)
    V4 = int(np.prod(d))
    return d, b, V4


def _sites(sites):
    if sites is None:
        return None, 0
    s = np.ascontiguousarray(sites, dtype=np.int64)
    return s, len(s)


def dhop(psi, U, dims, Ls, bc=None, dag=False, sites=None):
    """Bare hopping sum Dhop psi (or Dhop^+ psi); no -1/2, no diagonal term.

    With ``sites`` (array of 4D indices) only those sites are computed and the
    result has shape (nrhs, len(sites), Ls, 4, 3).
    """
    d, b, V4 = _common(dims, bc)
    psi = _fermion(psi, V4, Ls)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    s, ns = _sites(sites)
    nrhs = psi.shape[0]
    out = np.empty((nrhs, ns if s is not None else V4, Ls, 4, 3), np.complex128)
    rc = _load().oracle_dhop(_ptr(out), _ptr(psi), _ptr(U), _ptr(d), Ls, nrhs, _ptr(b),
                             int(bool(dag)), None if s is None else _ptr(s), ns)
    if rc:
        raise ValueError("oracle_dhop failed")
    return out


def kop(psi, dims, Ls, mf, dag=False):
    """The fifth-dimension hop K psi (or K^+ psi), per-RHS masses mf."""
    d, _, V4 = _common(dims, None)
    psi = _fermion(psi, V4, Ls)
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(mf, np.float64), (psi.shape[0],)))
    out = np.empty_like(psi)
    rc = _load().oracle_k(_ptr(out), _ptr(psi), _ptr(d), Ls, psi.shape[0], _ptr(m),
                          int(bool(dag)))
    if rc:
        raise ValueError("oracle_k failed")
    return out


def dw(psi, U, dims, Ls, M5, b, c, mf, bc=None, dag=False, sites=None):
    """Domain-wall operator D psi (or D^+ psi) with per-RHS masses mf."""
    d, bb, V4 = _common(dims, bc)
    psi = _fermion(psi, V4, Ls)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    nrhs = psi.shape[0]
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(mf, np.float64), (nrhs,)))
    s, ns = _sites(sites)
    out = np.empty((nrhs, ns if s is not None else V4, Ls, 4, 3), np.complex128)
    rc = _load().oracle_dw(_ptr(out), _ptr(psi), _ptr(U), _ptr(d), Ls, nrhs, _ptr(bb),
                           float(M5), float(b), float(c), _ptr(m), int(bool(dag)),
                           None if s is None else _ptr(s), ns)
    if rc:
        raise ValueError("oracle_dw failed")
    return out


def dwdagdw(psi, U, dims, Ls, M5, b, c, mf, bc=None):
    """D^+ D psi on full fields."""
    d, bb, V4 = _common(dims, bc)
    psi = _fermion(psi, V4, Ls)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    nrhs = psi.shape[0]
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(mf, np.float64), (nrhs,)))
    out = np.empty_like(psi)
    rc = _load().oracle_dwdagdw(_ptr(out), _ptr(psi), _ptr(U), _ptr(d), Ls, nrhs, _ptr(bb),
                                float(M5), float(b), float(c), _ptr(m))
    if rc:
        raise ValueError("oracle_dwdagdw failed")
    return out


def cg(rhs, U, dims, Ls, M5, b, c, mf, bc=None, tol=1e-10, maxit=10000, x0=None):
    """Textbook CG on D^+D x = rhs per RHS in FP64.

    Returns (x, iters[nrhs], true_resid[nrhs]) where true_resid is the
    recomputed |rhs - D^+D x| / |rhs|.
    """
    d, bb, V4 = _common(dims, bc)
    rhs = _fermion(rhs, V4, Ls)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    nrhs = rhs.shape[0]
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(mf, np.float64), (nrhs,)))
    x = np.zeros_like(rhs) if x0 is None else _fermion(x0, V4, Ls).copy()
    iters = np.zeros(nrhs, np.int32)
    res = np.zeros(nrhs, np.float64)
    rc = _load().oracle_cg(_ptr(x), _ptr(rhs), _ptr(U), _ptr(d), Ls, nrhs, _ptr(bb), float(M5),
                           float(b), float(c), _ptr(m), float(tol), int(maxit), _ptr(iters),
                           _ptr(res))
    if rc < 0:
        raise ValueError("oracle_cg failed")
    return x, iters, res


def inner(x, y):
    """<x, y> = sum conj(x) y over every component."""
    return np.vdot(np.asarray(x).ravel(), np.asarray(y).ravel())


def rel_l2(a, b):
    """|a - b|_2 / |b|_2."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
