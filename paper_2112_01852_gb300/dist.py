"""Ranks of a lattice decomposed along t, one process per rank (the paper's
multi-rank runs, Sec. 4.2, where MPI exchanges the faces of the hopping term).

Each rank owns a sub-lattice of Lt / R time slices: the global links of its
t-range, and the global t boundary sign only on the last rank (so that the sign
sits on the one link that crosses the global edge).  One apply of D, D^+ or
their hopping terms has one exchange step: every rank packs the two spin-
projected half-spinor faces of its operator (``dw_halo_pack_op``), sends them
to its t neighbours and applies the operator with the faces it received
(``dw_apply_op_halo``); the stitched result equals the undecomposed kernel bit
for bit.  The conjugate gradient on D^+D completes its inner products across
ranks with one all-reduce of the per-RHS FP64 partial sums.

This module is plumbing around the C ABI: every arithmetic step runs in the
library's kernels (``dw_halo_pack_op``, ``dw_apply_op_halo``,
``dw_field_redot``, ``dw_field_axpby``); torch.distributed moves the faces and
the scalars.  Two backends:

* ``gloo``: the faces go through host memory (device -> host, send / receive,
  host -> device); used by the tests, which run every rank as a process on one
  GPU (or, for the host logic, on the CPU);
* ``nccl``: the faces go device to device with NCCL send / receive and the
  scalars are reduced on the device; for one GPU per rank (not exercised on
  this one-GPU pool).
"""

from __future__ import annotations

import numpy as np

from . import dw


class TComm:
    """Ring of ranks along t over the default torch.distributed group.

    ``exchange`` sends ``send_dn`` to the rank below and ``send_up`` to the rank
    above and fills ``recv_up`` (the rank above's ``send_dn``) and ``recv_dn``
    (the rank below's ``send_up``); with one rank both come from itself (the
    periodic wrap)."""

    TAG_DOWN, TAG_UP = 11, 12

    def __init__(self):
        import torch.distributed as tdist
        self.tdist = tdist
        self.rank = tdist.get_rank() if tdist.is_initialized() else 0
        self.size = tdist.get_world_size() if tdist.is_initialized() else 1
        self.backend = tdist.get_backend() if tdist.is_initialized() else "none"
        self.up = (self.rank + 1) % self.size
        self.dn = (self.rank - 1) % self.size

    def exchange(self, send_dn, send_up, recv_up, recv_dn):
        if self.size == 1:
            recv_up.copy_(send_dn)
            recv_dn.copy_(send_up)
            return
        t = self.tdist
        if self.backend == "nccl":
            ops = [t.P2POp(t.isend, send_dn, self.dn), t.P2POp(t.irecv, recv_up, self.up),
                   t.P2POp(t.isend, send_up, self.up), t.P2POp(t.irecv, recv_dn, self.dn)]
            for r in t.batch_isend_irecv(ops):
                r.wait()
            return
        # gloo: stage through host memory (the device copies synchronise)
        hs_dn, hs_up = send_dn.cpu(), send_up.cpu()
        hr_up, hr_dn = hs_dn.new_empty(hs_dn.shape), hs_up.new_empty(hs_up.shape)
        reqs = [t.isend(hs_dn, self.dn, tag=self.TAG_DOWN),
                t.irecv(hr_up, self.up, tag=self.TAG_DOWN),
                t.isend(hs_up, self.up, tag=self.TAG_UP),
                t.irecv(hr_dn, self.dn, tag=self.TAG_UP)]
        for r in reqs:
            r.wait()
        recv_up.copy_(hr_up)
        recv_dn.copy_(hr_dn)

    def allreduce(self, values):
        """Sum of a list of floats over the ranks (FP64)."""
        if self.size == 1:
            return [float(v) for v in values]
        import torch
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor(list(values), dtype=torch.float64, device=dev)
        self.tdist.all_reduce(t, op=self.tdist.ReduceOp.SUM)
        return [float(v) for v in t.cpu()]

    def allgather_numpy(self, a):
        """This rank's array concatenated in rank order along axis 0 of each
        rank's block (every rank passes an array of the same shape)."""
        if self.size == 1:
            return a
        import torch
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1))
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = t.to(dev)
        parts = [torch.empty_like(t) for _ in range(self.size)]
        self.tdist.all_gather(parts, t)
        return [p.cpu().numpy().view(a.dtype).reshape(a.shape) for p in parts]


class DistLattice:
    """This rank's sub-lattice of a lattice decomposed along t."""

    def __init__(self, comm, dims, Ls, kind=dw.DW_MOBIUS, M5=1.8, b=1.5, c=0.5,
                 prec=dw.DW_F64, bc=(1, 1, 1, -1)):
        from .lattice import Lattice
        Lx, Ly, Lz, Lt = (int(d) for d in dims)
        if Lt % comm.size:
            raise ValueError("Lt = %d is not divisible by %d ranks" % (Lt, comm.size))
        self.comm = comm
        self.dims = (Lx, Ly, Lz, Lt)
        self.Lt_loc = Lt // comm.size
        self.t0 = comm.rank * self.Lt_loc
        self.Vf = Lx * Ly * Lz
        self.Ls = Ls
        self.prec = prec
        bc_loc = (bc[0], bc[1], bc[2], bc[3] if comm.rank == comm.size - 1 else 1)
        self.lat = Lattice((Lx, Ly, Lz, self.Lt_loc), Ls, kind=kind, M5=M5, b=b, c=c,
                           prec=prec, bc=bc_loc)
        self._halo = {}

    # ------------------------------------------------------------------ data
    def sites(self):
        """Global 4D site range of this rank (canonical x4 order, t slowest)."""
        return slice(self.t0 * self.Vf, (self.t0 + self.Lt_loc) * self.Vf)

    def load_gauge(self, U):
        """U: the GLOBAL canonical links (V4, 4, 3, 3); this rank keeps its slab."""
        self.lat.load_gauge(np.ascontiguousarray(U[self.sites()]))

    def pack(self, psi):
        """psi: GLOBAL canonical fermion (nrhs, V4, Ls, 4, 3) -> this rank's field."""
        psi = psi if psi.ndim == 5 else psi[None]
        return self.lat.pack(np.ascontiguousarray(psi[:, self.sites()]))

    def unpack(self, field, nrhs=1):
        """This rank's part, canonical (nrhs, V4_local, Ls, 4, 3)."""
        return self.lat.unpack(field, nrhs)

    def gather(self, field, nrhs=1):
        """The GLOBAL canonical field, assembled on every rank."""
        parts = self.comm.allgather_numpy(self.unpack(field, nrhs))
        if self.comm.size == 1:
            return parts
        return np.concatenate(parts, axis=1)

    def empty(self, nrhs=1):
        return self.lat.empty(nrhs)

    def _buffers(self, nrhs):
        if nrhs not in self._halo:
            import torch
            n = dw.dw_halo_bytes(self.lat.handle, self.prec, nrhs)
            self._halo[nrhs] = [torch.empty(n, dtype=torch.uint8, device="cuda")
                                for _ in range(4)]
        return self._halo[nrhs]

    # ------------------------------------------------------------- operators
    def apply(self, op, out, inp, mf=None, nrhs=1):
        """out = op inp (op: dw.DW_OP_DHOP, DW_OP_DHOP_DAG, DW_OP_D, DW_OP_DDAG) on
        the whole decomposed lattice; this rank's part."""
        import torch
        st = torch.cuda.current_stream().cuda_stream
        send_dn, send_up, recv_up, recv_dn = self._buffers(nrhs)
        m = None if mf is None else list(np.broadcast_to(np.asarray(mf, float), (nrhs,)))
        dw.dw_halo_pack_op(self.lat.handle, op, send_dn.data_ptr(), send_up.data_ptr(),
                           inp.data_ptr(), m, nrhs, st)
        self.comm.exchange(send_dn, send_up, recv_up, recv_dn)
        dw.dw_apply_op_halo(self.lat.handle, op, out.data_ptr(), inp.data_ptr(),
                            recv_up.data_ptr(), recv_dn.data_ptr(), m, nrhs, st)

    def apply_DdagD(self, out, inp, mf, nrhs=1, tmp=None):
        tmp = self.empty(nrhs) if tmp is None else tmp
        self.apply(dw.DW_OP_D, tmp, inp, mf, nrhs)
        self.apply(dw.DW_OP_DDAG, out, tmp, mf, nrhs)

    def dot(self, a, b, nrhs=1):
        """Re <a_r, b_r> over the whole lattice, per RHS."""
        import torch
        st = torch.cuda.current_stream().cuda_stream
        return self.comm.allreduce(dw.dw_field_redot(self.lat.handle, self.prec, a.data_ptr(),
                                                     b.data_ptr(), nrhs, st))

    def axpby(self, y, a, x, b, nrhs=1):
        import torch
        st = torch.cuda.current_stream().cuda_stream
        dw.dw_field_axpby(self.lat.handle, self.prec, y.data_ptr(), list(a), x.data_ptr(),
                          list(b), nrhs, st)

    def cg(self, x, b, mf, nrhs=1, tol=1e-10, maxit=10000):
        """D^+D x = b on the decomposed lattice (CG at this lattice's precision); x
        holds the start vector.  Returns (converged[nrhs], iterations, true
        residual[nrhs])."""
        return cg(_LatticeOps(self, mf, nrhs), x, b, nrhs, tol, maxit)

    def convert(self, other, out, inp, nrhs=1):
        """out (a field of DistLattice `other`: the same sub-lattice at another
        precision) = inp (a field of this one), through the canonical complex128
        layout on the device (dw_unpack_fermion, then dw_pack_fermion)."""
        import torch
        st = torch.cuda.current_stream().cuda_stream
        V5 = self.Vf * self.Lt_loc * self.Ls
        buf = torch.empty(nrhs * V5 * 24, dtype=torch.float64, device="cuda")
        dw.dw_unpack_fermion(self.lat.handle, buf.data_ptr(), inp.data_ptr(), self.prec, nrhs,
                             st)
        dw.dw_pack_fermion(other.lat.handle, out.data_ptr(), other.prec, buf.data_ptr(), nrhs,
                           st)

    def cg_mixed(self, lo, x, b, mf, nrhs=1, tol=1e-10, maxit=10000, inner_tol=1e-5):
        """D^+D x = b with this (high-precision) lattice for the residuals and the
        solution and DistLattice `lo` (same sub-lattice, lower precision) for the
        inner solves: defect correction, see mixed_cg.  Returns (converged[nrhs],
        inner iterations, outer steps, true residual[nrhs])."""
        hi_ops, lo_ops = _LatticeOps(self, mf, nrhs), _LatticeOps(lo, mf, nrhs)
        return mixed_cg(hi_ops, lo_ops, lambda o, i: self.convert(lo, o, i, nrhs),
                        lambda o, i: lo.convert(self, o, i, nrhs), x, b, nrhs, tol, maxit,
                        inner_tol)

    def close(self):
        self._halo.clear()
        self.lat.close()


class _LatticeOps:
    """The vector space of a DistLattice for the generic CG below."""

    def __init__(self, dl, mf, nrhs):
        self.dl, self.mf, self.nrhs = dl, mf, nrhs
        self._tmp = dl.empty(nrhs)

    def new(self):
        v = self.dl.empty(self.nrhs)
        v.zero_()
        return v

    def apply(self, out, inp):
        self.dl.apply_DdagD(out, inp, self.mf, self.nrhs, self._tmp)

    def dot(self, a, b):
        return self.dl.dot(a, b, self.nrhs)

    def axpby(self, y, a, x, b):
        self.dl.axpby(y, a, x, b, self.nrhs)


def cg(ops, x, b, nrhs, tol, maxit, restarts=3):
    """Textbook CG (Hestenes-Stiefel) for nrhs independent systems A x = b over a
    distributed vector space ``ops`` (apply, dot with global sums, axpby, new).
    A converged RHS gets zero step lengths from then on.  The iterated residual
    decides when to stop; the true residual |b - A x| / |b| is then recomputed,
    and if it is above tol the iteration restarts from x (at most `restarts`
    times).  Returns (converged, iterations, true_resid)."""
    r, p, Ap = ops.new(), ops.new(), ops.new()
    bb = ops.dot(b, b)
    tol2 = [tol * tol * v for v in bb]
    iters = 0
    true_res = [0.0] * nrhs
    for _ in range(restarts + 1):
        ops.apply(Ap, x)                        # r = b - A x
        ops.axpby(r, [1.0] * nrhs, b, [0.0] * nrhs)
        ops.axpby(r, [-1.0] * nrhs, Ap, [1.0] * nrhs)
        rr = ops.dot(r, r)
        true_res = [np.sqrt(v / w) if w > 0 else 0.0 for v, w in zip(rr, bb)]
        if all(t <= tol for t in true_res) or iters >= maxit:
            break
        ops.axpby(p, [1.0] * nrhs, r, [0.0] * nrhs)  # p = r
        active = [rr[k] > tol2[k] for k in range(nrhs)]
        while any(active) and iters < maxit:
            ops.apply(Ap, p)
            pAp = ops.dot(p, Ap)
            if any(a and not (v > 0.0 and np.isfinite(v)) for a, v in zip(active, pAp)):
                raise FloatingPointError("CG breakdown: <p, A p> = %r" % (pAp,))
            alpha = [rr[k] / pAp[k] if active[k] else 0.0 for k in range(nrhs)]
            ops.axpby(x, alpha, p, [1.0] * nrhs)
            ops.axpby(r, [-a for a in alpha], Ap, [1.0] * nrhs)
            rr_new = ops.dot(r, r)
            beta = [rr_new[k] / rr[k] if active[k] else 0.0 for k in range(nrhs)]
            ops.axpby(p, [1.0] * nrhs, r, beta)     # p = r + beta p
            rr = [rr_new[k] if active[k] else rr[k] for k in range(nrhs)]
            active = [active[k] and rr[k] > tol2[k] for k in range(nrhs)]
            iters += 1
    converged = [t <= tol for t in true_res]
    return converged, iters, true_res


def mixed_cg(hi, lo, to_lo, to_hi, x, b, nrhs, tol, maxit, inner_tol=1e-5, max_outer=30):
    """Mixed-precision solve of A x = b by defect correction (iterative
    refinement; Wilkinson's scheme, as used for mixed-precision solvers): the
    residual r = b - A x and the solution x stay at the high precision of vector
    space ``hi``; each outer step converts r to the low-precision space ``lo``,
    solves A e = r there with CG (above) to the relative tolerance ``inner_tol``
    and adds the correction e back to x at high precision.  It stops when every
    RHS's high-precision true residual |b - A x| / |b| meets tol (an RHS that
    already meets it gets a zero correction), after ``maxit`` inner iterations
    or after ``max_outer`` outer steps.  ``to_lo(out_lo, in_hi)`` and
    ``to_hi(out_hi, in_lo)`` convert a vector.  Returns (converged, inner
    iterations, outer steps, true_resid)."""
    r, Ax, e_hi = hi.new(), hi.new(), hi.new()
    r_lo, e_lo = lo.new(), lo.new()
    bb = hi.dot(b, b)
    iters = outer = 0
    while True:
        hi.apply(Ax, x)                                  # r = b - A x
        hi.axpby(r, [1.0] * nrhs, b, [0.0] * nrhs)
        hi.axpby(r, [-1.0] * nrhs, Ax, [1.0] * nrhs)
        rr = hi.dot(r, r)
        true_res = [np.sqrt(v / w) if w > 0 else 0.0 for v, w in zip(rr, bb)]
        done = [t <= tol for t in true_res]
        if all(done) or iters >= maxit or outer >= max_outer:
            break
        # the converged RHS solve A e = 0: their correction is zero
        hi.axpby(r, [0.0 if d else 1.0 for d in done], r, [0.0] * nrhs)
        to_lo(r_lo, r)
        lo.axpby(e_lo, [0.0] * nrhs, r_lo, [0.0] * nrhs)  # e = 0
        _, n, _ = cg(lo, e_lo, r_lo, nrhs, inner_tol, maxit - iters, restarts=0)
        iters += n
        outer += 1
        to_hi(e_hi, e_lo)
        hi.axpby(x, [1.0] * nrhs, e_hi, [1.0] * nrhs)
    return done, iters, outer, true_res
