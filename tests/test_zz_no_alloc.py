"""GPU test of dw_apply_DdagD_noalloc, the allocation-free D^+D entry point.

Some callers cannot let the library allocate device memory: a serving process
whose device memory is all handed out by its own pool allocator, for
instance, or one that must not make allocation calls while its work is in
flight.  dw_apply_DdagD keeps its intermediate D psi in lattice scratch that it
grows with cudaMalloc; dw_apply_DdagD_noalloc keeps it in a fixed array inside
the library instead.  This file checks, at FP64, FP32 and FP16 storage:

* on a freshly created lattice the call leaves the device's free memory
  unchanged (after one warm-up call on another lattice has loaded the kernels
  and looked the array up), on two calls in a row;
* its output equals dw_apply_DdagD's bit for bit (same kernels, same tiles,
  same order of operations) and the oracle's D^+D within the precision's
  tolerance;
* the largest RHS count that fits the array works, and one more is rejected
  with DW_ERR_ARG before anything runs.

The file is named to be collected last, so that a run that stops at the first
failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

import oracle
from paper_2112_01852_gb300 import build, dw, inputs

pytestmark = pytest.mark.gpu

TOL = {dw.DW_F64: 1e-12, dw.DW_F32: 1e-5, dw.DW_F16: 5e-3}
SCRATCH_BYTES = 32 << 20  # the fixed array's size, as include/dw.h states
M5, B, C = 1.8, 1.5, 0.5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _masses(mfs):
    return (ctypes.c_double * len(mfs))(*mfs)


@pytest.mark.parametrize("prec", [dw.DW_F64, dw.DW_F32, dw.DW_F16], ids=["f64", "f32", "f16"])
def test_noalloc_ddagd(prec):
    import torch
    from paper_2112_01852_gb300.lattice import Lattice
    build.build()
    lib = dw.load_library()
    dims, Ls = (8, 8, 8, 8), 8
    mfs = [0.01, 0.05]
    U = inputs.exp_su3_field(dims, seed=31)
    st = torch.cuda.current_stream().cuda_stream

    def lattice():
        lat = Lattice(dims, Ls, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=prec)
        lat.load_gauge(U)
        return lat

    # warm-up on a lattice of its own: loads the kernels and the array's address
    warm = lattice()
    xw = warm.pack(inputs.gaussian_fermion(dims, Ls, 2, seed=30))
    yw = warm.empty(2)
    assert lib.dw_apply_DdagD_noalloc(warm.handle, yw.data_ptr(), xw.data_ptr(), _masses(mfs),
                                      2, st) == dw.DW_OK, dw.dw_last_error()
    torch.cuda.synchronize()
    del xw, yw
    warm.close()

    lat = lattice()  # fresh: no scratch of its own yet
    for seed in (32, 33):  # two calls in a row, different inputs
        psi = inputs.gaussian_fermion(dims, Ls, 2, seed=seed)
        x = lat.pack(psi)
        got = lat.empty(2)
        ref = lat.empty(2)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = lib.dw_apply_DdagD_noalloc(lat.handle, got.data_ptr(), x.data_ptr(), _masses(mfs),
                                        2, st)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert rc == dw.DW_OK, dw.dw_last_error()
        assert free1 == free0, (free0, free1)
        dw.dw_apply_DdagD(lat.handle, ref.data_ptr(), x.data_ptr(), mfs, 2, st)
        a = lat.unpack(got, 2)
        b = lat.unpack(ref, 2)
        assert np.array_equal(a, b)
        if seed == 32:
            want = oracle.dwdagdw(psi, U, dims, Ls, M5, B, C, mfs)
            for r in range(2):
                assert _rel(a[r], want[r]) <= TOL[prec], (r, _rel(a[r], want[r]))

    # the size limit: the largest RHS count that fits works, one more is refused
    per_rhs = lat.fermion_bytes(1)
    nmax = SCRATCH_BYTES // per_rhs
    assert nmax >= 1
    psi = inputs.gaussian_fermion(dims, Ls, nmax, seed=34)
    x = lat.pack(psi)
    got = lat.empty(nmax)
    ref = lat.empty(nmax)
    big = [0.01 + 0.01 * r for r in range(nmax + 1)]
    rc = lib.dw_apply_DdagD_noalloc(lat.handle, got.data_ptr(), x.data_ptr(),
                                    _masses(big[:nmax]), nmax, st)
    assert rc == dw.DW_OK, dw.dw_last_error()
    dw.dw_apply_DdagD(lat.handle, ref.data_ptr(), x.data_ptr(), big[:nmax], nmax, st)
    assert np.array_equal(lat.unpack(got, nmax), lat.unpack(ref, nmax))
    # rejected on the host before any launch: small dummy buffers are never touched
    dummy_in = torch.empty(64, dtype=torch.uint8, device="cuda")
    dummy_out = torch.empty(64, dtype=torch.uint8, device="cuda")
    rc = lib.dw_apply_DdagD_noalloc(lat.handle, dummy_out.data_ptr(), dummy_in.data_ptr(),
                                    _masses(big), nmax + 1, st)
    assert rc == dw.DW_ERR_ARG
    assert "scratch" in dw.dw_last_error()
    torch.cuda.synchronize()
    lat.close()
