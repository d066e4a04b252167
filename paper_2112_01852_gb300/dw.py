"""ctypes binding of libdw_gb300.so with the C ABI's names (include/dw.h).

Argument marshalling only: every function forwards to the C entry point of the
same name, raises DWError on a negative status, and takes device buffers as
integer pointers (``tensor.data_ptr()``) and streams as integer handles
(``torch.cuda.current_stream().cuda_stream``).  There is no fallback: if the
CUDA library has not been built, loading fails loudly.
"""

from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdw_gb300.so")

DW_OK = 0
DW_ERR_ARG = -1
DW_ERR_ALLOC = -2
DW_ERR_CUDA = -3
DW_ERR_STATE = -4
DW_ERR_NOT_CONVERGED = -5
DW_ERR_BREAKDOWN = -6
DW_ERR_TIMEOUT = -7

DW_SHAMIR = 0
DW_MOBIUS = 1
DW_F64 = 0
DW_F32 = 1
DW_F16 = 2

DW_OP_DHOP = 0
DW_OP_DHOP_DAG = 1
DW_OP_D = 2
DW_OP_DDAG = 3
DW_OP_DDAGD = 4

_ERRNAMES = {
    DW_ERR_ARG: "DW_ERR_ARG",
    DW_ERR_ALLOC: "DW_ERR_ALLOC",
    DW_ERR_CUDA: "DW_ERR_CUDA",
    DW_ERR_STATE: "DW_ERR_STATE",
    DW_ERR_NOT_CONVERGED: "DW_ERR_NOT_CONVERGED",
    DW_ERR_BREAKDOWN: "DW_ERR_BREAKDOWN",
    DW_ERR_TIMEOUT: "DW_ERR_TIMEOUT",
}

# Every symbol include/dw.h declares.
SYMBOLS = (
    "dw_create_lattice", "dw_destroy_lattice", "dw_load_gauge", "dw_apply_Dhop",
    "dw_apply_Dhop_dag", "dw_apply_D", "dw_apply_Ddag", "dw_apply_DdagD",
    "dw_apply_DdagD_noalloc", "dw_apply_host",
    "dw_cg_solve", "dw_set_tile", "dw_tune", "dw_device_status", "dw_halo_bytes",
    "dw_halo_pack", "dw_apply_Dhop_halo", "dw_fermion_bytes", "dw_pack_fermion",
    "dw_unpack_fermion", "dw_last_error", "dw_fermion_bytes_eo", "dw_eo_split", "dw_eo_merge",
    "dw_apply_m5_eo", "dw_apply_schur", "dw_solve_eo", "dw_get_tile", "dw_set_wait_polls",
    "dw_set_complex_layout", "dw_halo_pack_op", "dw_apply_op_halo", "dw_field_redot",
    "dw_field_axpby", "dw_set_reliable_delta",
)


class DWError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "?"), code, msg))
        self.code = code


class dw_cg_stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("reliable_updates", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("true_resid", ctypes.c_double),
        ("seconds", ctypes.c_double),
    ]


_lib = None
_lock = threading.Lock()


def load_library():
    """Load the in-tree CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libdw_gb300.so not found at %s: build it first (paper_2112_01852_gb300.build)"
                % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        IP = ctypes.POINTER(ctypes.c_int)
        DP = ctypes.POINTER(ctypes.c_double)
        sig = {
            "dw_create_lattice": (I, [ctypes.POINTER(P), IP, I, I, D, D, D, I, IP]),
            "dw_destroy_lattice": (None, [P]),
            "dw_load_gauge": (I, [P, P, P]),
            "dw_apply_Dhop": (I, [P, P, P, I, P]),
            "dw_apply_Dhop_dag": (I, [P, P, P, I, P]),
            "dw_apply_D": (I, [P, P, P, DP, I, P]),
            "dw_apply_Ddag": (I, [P, P, P, DP, I, P]),
            "dw_apply_DdagD": (I, [P, P, P, DP, I, P]),
            "dw_apply_DdagD_noalloc": (I, [P, P, P, DP, I, P]),
            "dw_apply_host": (I, [P, I, P, P, DP, I, P]),
            "dw_cg_solve": (I, [P, P, P, DP, I, D, I, I, ctypes.POINTER(dw_cg_stats), P]),
            "dw_set_tile": (I, [P, I, I, I, I, I, I, I, I]),
            "dw_tune": (I, [P, I, I, IP, IP, IP, IP, IP, P]),
            "dw_get_tile": (I, [P, I, I, I, IP, IP, IP, IP, IP]),
            "dw_device_status": (I, [P]),
            "dw_set_wait_polls": (I, [P, I]),
            "dw_set_reliable_delta": (I, [P, D]),
            "dw_set_complex_layout": (I, [P, I]),
            "dw_fermion_bytes_eo": (S, [P, I, I]),
            "dw_eo_split": (I, [P, P, P, P, I, I, P]),
            "dw_eo_merge": (I, [P, P, P, P, I, I, P]),
            "dw_apply_m5_eo": (I, [P, P, P, DP, I, I, I, P]),
            "dw_apply_schur": (I, [P, P, P, DP, I, I, P]),
            "dw_solve_eo": (I, [P, P, P, DP, I, D, I, I, ctypes.POINTER(dw_cg_stats), P]),
            "dw_halo_bytes": (S, [P, I, I]),
            "dw_halo_pack": (I, [P, P, P, P, I, I, P]),
            "dw_halo_pack_op": (I, [P, I, P, P, P, DP, I, P]),
            "dw_apply_op_halo": (I, [P, I, P, P, P, P, DP, I, P]),
            "dw_field_redot": (I, [P, I, P, P, I, DP, P]),
            "dw_field_axpby": (I, [P, I, P, DP, P, DP, I, P]),
            "dw_apply_Dhop_halo": (I, [P, P, P, P, P, I, I, P]),
            "dw_fermion_bytes": (S, [P, I, I]),
            "dw_pack_fermion": (I, [P, P, I, P, I, P]),
            "dw_unpack_fermion": (I, [P, P, P, I, I, P]),
            "dw_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc, allow=()):
    if rc < 0 and rc not in allow:
        msg = load_library().dw_last_error().decode(errors="replace")
        raise DWError(rc, msg)
    return rc


def _ints(v, n):
    if v is None:
        return None
    arr = (ctypes.c_int * n)(*[int(x) for x in v])
    return arr


def _doubles(v):
    if v is None:
        return None
    v = [float(x) for x in v]
    return (ctypes.c_double * len(v))(*v)


def dw_last_error() -> str:
    return load_library().dw_last_error().decode(errors="replace")


def dw_create_lattice(dims, Ls, kind, M5, b, c, prec, bc=None):
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.dw_create_lattice(ctypes.byref(h), _ints(dims, 4), int(Ls), int(kind), float(M5),
                                 float(b), float(c), int(prec), _ints(bc, 4)))
    return h.value


def dw_destroy_lattice(lat):
    load_library().dw_destroy_lattice(lat)


def dw_load_gauge(lat, U, stream=0):
    _check(load_library().dw_load_gauge(lat, U, stream))


def dw_apply_Dhop(lat, out, inp, nrhs, stream=0):
    _check(load_library().dw_apply_Dhop(lat, out, inp, int(nrhs), stream))


def dw_apply_Dhop_dag(lat, out, inp, nrhs, stream=0):
    _check(load_library().dw_apply_Dhop_dag(lat, out, inp, int(nrhs), stream))


def dw_apply_D(lat, out, inp, mf, nrhs, stream=0):
    _check(load_library().dw_apply_D(lat, out, inp, _doubles(mf), int(nrhs), stream))


def dw_apply_Ddag(lat, out, inp, mf, nrhs, stream=0):
    _check(load_library().dw_apply_Ddag(lat, out, inp, _doubles(mf), int(nrhs), stream))


def dw_apply_DdagD(lat, out, inp, mf, nrhs, stream=0):
    _check(load_library().dw_apply_DdagD(lat, out, inp, _doubles(mf), int(nrhs), stream))


def dw_apply_DdagD_noalloc(lat, out, inp, mf, nrhs, stream=0):
    _check(load_library().dw_apply_DdagD_noalloc(lat, out, inp, _doubles(mf), int(nrhs), stream))


def dw_apply_host(lat, op, out_host, in_host, mf, nrhs, stream=0):
    _check(load_library().dw_apply_host(lat, int(op), out_host, in_host, _doubles(mf), int(nrhs),
                                        stream))


def dw_cg_solve(lat, x, b, mf, nrhs, tol, maxit, mode, stream=0):
    """Returns (status, [dw_cg_stats]*nrhs); status may be DW_ERR_NOT_CONVERGED."""
    stats = (dw_cg_stats * int(nrhs))()
    rc = _check(load_library().dw_cg_solve(lat, x, b, _doubles(mf), int(nrhs), float(tol),
                                           int(maxit), int(mode), stats, stream),
                allow=(DW_ERR_NOT_CONVERGED,))
    return rc, list(stats)


def dw_solve_eo(lat, x, eta, mf, nrhs, tol, maxit, mode, stream=0):
    """D x = eta with even-odd preconditioning; returns (status, [dw_cg_stats]*nrhs)."""
    stats = (dw_cg_stats * int(nrhs))()
    rc = _check(load_library().dw_solve_eo(lat, x, eta, _doubles(mf), int(nrhs), float(tol),
                                           int(maxit), int(mode), stats, stream),
                allow=(DW_ERR_NOT_CONVERGED,))
    return rc, list(stats)


def dw_set_tile(lat, op, prec, nrhs, spt, tx, variant=0, zblk=0, sgrp=1):
    _check(load_library().dw_set_tile(lat, int(op), int(prec), int(nrhs), int(spt), int(tx),
                                      int(variant), int(zblk), int(sgrp)))


def dw_tune(lat, op, nrhs, stream=0):
    """Returns the chosen (spt, tx, variant, zblk, sgrp)."""
    vals = [ctypes.c_int() for _ in range(5)]
    _check(load_library().dw_tune(lat, int(op), int(nrhs), *[ctypes.byref(v) for v in vals],
                                  stream))
    return tuple(v.value for v in vals)


def dw_device_status(lat):
    """Raises DWError (DW_ERR_TIMEOUT) if a kernel gave up a bounded wait."""
    _check(load_library().dw_device_status(lat))


def dw_set_complex_layout(lat, interleaved):
    _check(load_library().dw_set_complex_layout(lat, int(interleaved)))


def dw_set_wait_polls(lat, polls):
    _check(load_library().dw_set_wait_polls(lat, int(polls)))


def dw_set_reliable_delta(lat, delta):
    _check(load_library().dw_set_reliable_delta(lat, float(delta)))


def dw_fermion_bytes_eo(lat, prec, nrhs):
    return int(load_library().dw_fermion_bytes_eo(lat, int(prec), int(nrhs)))


def dw_eo_split(lat, even, odd, full, prec, nrhs, stream=0):
    _check(load_library().dw_eo_split(lat, even, odd, full, int(prec), int(nrhs), stream))


def dw_eo_merge(lat, full, even, odd, prec, nrhs, stream=0):
    _check(load_library().dw_eo_merge(lat, full, even, odd, int(prec), int(nrhs), stream))


def dw_apply_m5_eo(lat, out, inp, mf, nrhs, inverse, dag, stream=0):
    _check(load_library().dw_apply_m5_eo(lat, out, inp, _doubles(mf), int(nrhs), int(inverse),
                                         int(dag), stream))


def dw_apply_schur(lat, out, inp, mf, nrhs, dag, stream=0):
    _check(load_library().dw_apply_schur(lat, out, inp, _doubles(mf), int(nrhs), int(dag),
                                         stream))


def dw_get_tile(lat, op, prec, nrhs):
    """The (spt, tx, variant, zblk, sgrp) that launches of (op, prec, nrhs) use."""
    vals = [ctypes.c_int() for _ in range(5)]
    _check(load_library().dw_get_tile(lat, int(op), int(prec), int(nrhs),
                                      *[ctypes.byref(v) for v in vals]))
    return tuple(v.value for v in vals)


def dw_halo_bytes(lat, prec, nrhs):
    return int(load_library().dw_halo_bytes(lat, int(prec), int(nrhs)))


def dw_halo_pack(lat, send_dn, send_up, inp, nrhs, dag=0, stream=0):
    _check(load_library().dw_halo_pack(lat, send_dn, send_up, inp, int(nrhs), int(dag), stream))


def dw_apply_Dhop_halo(lat, out, inp, recv_up, recv_dn, nrhs, dag=0, stream=0):
    _check(load_library().dw_apply_Dhop_halo(lat, out, inp, recv_up, recv_dn, int(nrhs),
                                             int(dag), stream))


def dw_halo_pack_op(lat, op, send_dn, send_up, inp, mf, nrhs, stream=0):
    _check(load_library().dw_halo_pack_op(lat, int(op), send_dn, send_up, inp,
                                          None if mf is None else _doubles(mf), int(nrhs),
                                          stream))


def dw_apply_op_halo(lat, op, out, inp, recv_up, recv_dn, mf, nrhs, stream=0):
    _check(load_library().dw_apply_op_halo(lat, int(op), out, inp, recv_up, recv_dn,
                                           None if mf is None else _doubles(mf), int(nrhs),
                                           stream))


def dw_field_redot(lat, prec, a, b, nrhs, stream=0):
    """Re <a_r, b_r> per right-hand side (FP64, host list)."""
    out = (ctypes.c_double * int(nrhs))()
    _check(load_library().dw_field_redot(lat, int(prec), a, b, int(nrhs), out, stream))
    return [float(v) for v in out]


def dw_field_axpby(lat, prec, y, a, x, b, nrhs, stream=0):
    """y_r = a[r] x_r + b[r] y_r."""
    _check(load_library().dw_field_axpby(lat, int(prec), y, _doubles(a), x, _doubles(b),
                                         int(nrhs), stream))


def dw_fermion_bytes(lat, prec, nrhs):
    return int(load_library().dw_fermion_bytes(lat, int(prec), int(nrhs)))


def dw_pack_fermion(lat, dst_internal, prec, src_c128, nrhs, stream=0):
    _check(load_library().dw_pack_fermion(lat, dst_internal, int(prec), src_c128, int(nrhs),
                                          stream))


def dw_unpack_fermion(lat, dst_c128, src_internal, prec, nrhs, stream=0):
    _check(load_library().dw_unpack_fermion(lat, dst_c128, src_internal, int(prec), int(nrhs),
                                            stream))
