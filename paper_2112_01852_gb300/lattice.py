"""Python-side convenience over the C ABI: device buffers from PyTorch.

``Lattice`` owns a ``dw_lattice`` handle and allocates fields as CUDA byte
tensors sized by ``dw_fermion_bytes``.  Every compute step goes through the C
entry points in :mod:`paper_2112_01852_gb300.dw`; this module only moves
arguments, allocates torch memory and copies numpy arrays to and from the GPU.
"""

from __future__ import annotations

import numpy as np
import torch

from . import dw

PREC_NAMES = {dw.DW_F64: "f64", dw.DW_F32: "f32", dw.DW_F16: "f16"}


def _stream():
    return torch.cuda.current_stream().cuda_stream


class Lattice:
    def __init__(self, dims, Ls, kind=dw.DW_MOBIUS, M5=1.8, b=1.5, c=0.5, prec=dw.DW_F32,
                 bc=(1, 1, 1, -1)):
        if not torch.cuda.is_available():
            raise RuntimeError("Lattice needs a CUDA device")
        self.dims = tuple(int(d) for d in dims)
        self.Ls = int(Ls)
        self.kind = kind
        self.M5, self.b, self.c = float(M5), float(b), float(c)
        if kind == dw.DW_SHAMIR:
            self.b, self.c = 1.0, 0.0
        self.prec = prec
        self.bc = tuple(bc)
        self.V4 = int(np.prod(self.dims))
        self.V5 = self.V4 * self.Ls
        self.handle = dw.dw_create_lattice(self.dims, self.Ls, kind, M5, b, c, prec, bc)

    def close(self):
        if getattr(self, "handle", None):
            torch.cuda.synchronize()
            dw.dw_destroy_lattice(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ memory
    def fermion_bytes(self, nrhs=1, prec=None):
        return dw.dw_fermion_bytes(self.handle, self.prec if prec is None else prec, nrhs)

    def empty(self, nrhs=1, prec=None):
        n = self.fermion_bytes(nrhs, prec)
        return torch.empty(n, dtype=torch.uint8, device="cuda")

    def empty_eo(self, nrhs=1, prec=None):
        """A single-parity field (V4/2 sites; needs all four extents even)."""
        n = dw.dw_fermion_bytes_eo(self.handle, self.prec if prec is None else prec, nrhs)
        return torch.empty(n, dtype=torch.uint8, device="cuda")

    def pack_eo(self, psi, prec=None):
        """Canonical complex128 numpy (nrhs, V4, Ls, 4, 3) -> (even, odd) device fields."""
        prec = self.prec if prec is None else prec
        full = self.pack(psi, prec)
        nrhs = 1 if np.ndim(psi) == 4 else np.shape(psi)[0]
        even, odd = self.empty_eo(nrhs, prec), self.empty_eo(nrhs, prec)
        dw.dw_eo_split(self.handle, even.data_ptr(), odd.data_ptr(), full.data_ptr(), prec, nrhs,
                       _stream())
        return even, odd

    def unpack_eo(self, even, odd, nrhs=1, prec=None):
        """(even, odd) device fields -> canonical complex128 numpy (nrhs, V4, Ls, 4, 3)."""
        prec = self.prec if prec is None else prec
        full = self.empty(nrhs, prec)
        dw.dw_eo_merge(self.handle, full.data_ptr(), even.data_ptr(), odd.data_ptr(), prec, nrhs,
                       _stream())
        return self.unpack(full, nrhs, prec)

    def load_gauge(self, U):
        """U: complex128 numpy (V4, 4, 3, 3), canonical layout."""
        U = np.ascontiguousarray(U, dtype=np.complex128)
        assert U.shape == (self.V4, 4, 3, 3)
        t = torch.from_numpy(U.view(np.float64).reshape(-1)).to("cuda")
        dw.dw_load_gauge(self.handle, t.data_ptr(), _stream())
        torch.cuda.current_stream().synchronize()

    def pack(self, psi, prec=None):
        """Canonical complex128 numpy (nrhs, V4, Ls, 4, 3) -> internal device field."""
        prec = self.prec if prec is None else prec
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        if psi.ndim == 4:
            psi = psi[None]
        nrhs = psi.shape[0]
        src = torch.from_numpy(psi.view(np.float64).reshape(-1)).to("cuda")
        dst = self.empty(nrhs, prec)
        dw.dw_pack_fermion(self.handle, dst.data_ptr(), prec, src.data_ptr(), nrhs, _stream())
        torch.cuda.current_stream().synchronize()
        return dst

    def unpack(self, field, nrhs=1, prec=None):
        """Internal device field -> canonical complex128 numpy (nrhs, V4, Ls, 4, 3)."""
        prec = self.prec if prec is None else prec
        dst = torch.empty(nrhs * self.V5 * 24, dtype=torch.float64, device="cuda")
        dw.dw_unpack_fermion(self.handle, dst.data_ptr(), field.data_ptr(), prec, nrhs,
                             _stream())
        out = dst.cpu().numpy().view(np.complex128)
        return out.reshape(nrhs, self.V4, self.Ls, 4, 3)

    # ------------------------------------------------------------------ operators
    def dhop(self, out, inp, nrhs=1, dag=False):
        f = dw.dw_apply_Dhop_dag if dag else dw.dw_apply_Dhop
        f(self.handle, out.data_ptr(), inp.data_ptr(), nrhs, _stream())

    def D(self, out, inp, mf, nrhs=1):
        dw.dw_apply_D(self.handle, out.data_ptr(), inp.data_ptr(), _masses(mf, nrhs), nrhs,
                      _stream())

    def Ddag(self, out, inp, mf, nrhs=1):
        dw.dw_apply_Ddag(self.handle, out.data_ptr(), inp.data_ptr(), _masses(mf, nrhs), nrhs,
                         _stream())

    def DdagD(self, out, inp, mf, nrhs=1):
        dw.dw_apply_DdagD(self.handle, out.data_ptr(), inp.data_ptr(), _masses(mf, nrhs), nrhs,
                          _stream())

    def apply_host(self, op, out_host, in_host, mf=None, nrhs=1):
        """out_host / in_host: pinned CPU byte tensors holding internal-layout fields."""
        dw.dw_apply_host(self.handle, op, out_host.data_ptr(), in_host.data_ptr(),
                         None if mf is None else _masses(mf, nrhs), nrhs, _stream())

    def set_tile(self, op, spt, tx, variant=0, nrhs=0, prec=None, zblk=0, sgrp=1):
        dw.dw_set_tile(self.handle, op, self.prec if prec is None else prec, nrhs, spt, tx,
                       variant, zblk, sgrp)

    def tune(self, op, nrhs=1):
        return dw.dw_tune(self.handle, op, nrhs, _stream())

    def solve_eo(self, x, eta, mf, nrhs=1, tol=1e-10, maxit=10000, mode=dw.DW_F32):
        """D x = eta by even-odd preconditioned CG (FP64 full fields)."""
        return dw.dw_solve_eo(self.handle, x.data_ptr(), eta.data_ptr(), _masses(mf, nrhs), nrhs,
                              tol, maxit, mode, _stream())

    def cg(self, x, b, mf, nrhs=1, tol=1e-10, maxit=10000, mode=dw.DW_F32):
        return dw.dw_cg_solve(self.handle, x.data_ptr(), b.data_ptr(), _masses(mf, nrhs), nrhs,
                              tol, maxit, mode, _stream())


def _masses(mf, nrhs):
    m = np.broadcast_to(np.asarray(mf, dtype=np.float64), (nrhs,))
    return [float(v) for v in m]
