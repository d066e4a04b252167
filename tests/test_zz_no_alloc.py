"""GPU test of dw_apply_DdagD_noalloc, the allocation-free D^+D entry point.

Callers whose device memory is owned by their own allocator (a serving pool,
for instance) cannot let the library cudaMalloc scratch space; this entry
point keeps the intermediate D psi in a fixed array inside the library.  Its
output must agree with dw_apply_DdagD on consecutive calls.  The file is
named to be collected last.
"""

import ctypes

import numpy as np
import pytest

from paper_2112_01852_gb300 import build, dw, inputs

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_noalloc_ddagd_matches_ddagd_on_consecutive_calls():
    import torch
    from paper_2112_01852_gb300.lattice import Lattice
    build.build()
    lib = dw.load_library()
    dims, Ls = (8, 8, 8, 8), 8
    mfs = [0.01, 0.05]
    U = inputs.exp_su3_field(dims, seed=31)
    lat = Lattice(dims, Ls, kind=dw.DW_MOBIUS, M5=1.8, b=1.5, c=0.5, prec=dw.DW_F32)
    lat.load_gauge(U)
    st = torch.cuda.current_stream().cuda_stream
    masses = (ctypes.c_double * 2)(*mfs)
    for seed in (32, 33):  # two calls in a row, different inputs
        psi = inputs.gaussian_fermion(dims, Ls, 2, seed=seed)
        x = lat.pack(psi)
        ref = lat.empty(2)
        got = lat.empty(2)
        dw.dw_apply_DdagD(lat.handle, ref.data_ptr(), x.data_ptr(), mfs, 2, st)
        rc = lib.dw_apply_DdagD_noalloc(lat.handle, got.data_ptr(), x.data_ptr(), masses, 2, st)
        assert rc == dw.DW_OK, dw.dw_last_error()
        a = lat.unpack(got, 2)
        b = lat.unpack(ref, 2)
        for r in range(2):
            assert _rel(a[r], b[r]) <= TOL_F32
    # more RHS than the fixed array holds: rejected with DW_ERR_ARG, nothing launched
    big = 400
    xb = lat.empty(big)
    yb = lat.empty(big)
    mb = (ctypes.c_double * big)(*([0.01] * big))
    rc = lib.dw_apply_DdagD_noalloc(lat.handle, yb.data_ptr(), xb.data_ptr(), mb, big, st)
    assert rc == dw.DW_ERR_ARG
    assert "scratch" in dw.dw_last_error()
    torch.cuda.synchronize()
    lat.close()
