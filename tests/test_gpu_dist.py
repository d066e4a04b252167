"""The multi-rank data plane on the GPU: a lattice decomposed along t into two
ranks, each a separate process with its own CUDA context on the one GPU of
this machine, exchanging half-spinor faces through host memory (gloo).  No
kernel waits on another rank: every exchange happens on the host between
launches.

* The stitched Dhop, Dhop^+, D and D^+ equal the undecomposed kernels (same
  variant-0 tiles) bit for bit, at FP64 and FP32, and match the oracle.
* The distributed FP64 CG on D^+D (global sums over both ranks) reaches an
  oracle-recomputed residual <= 1e-10, and so does the distributed mixed-
  precision solve (FP64 residuals and solution, FP32 inner CG on a second
  decomposed lattice, by defect correction).
"""

import socket

import numpy as np
import pytest

import oracle
from gpu_helpers import BC, TOL, build_library, make_case
from paper_2112_01852_gb300 import dw

pytestmark = pytest.mark.gpu

DIMS, LS, M5, B, C = (4, 4, 4, 8), 4, 1.8, 1.5, 0.5
MF = [0.05, 0.2]
OPS = (dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG, dw.DW_OP_D, dw.DW_OP_DDAG)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, path):
    import torch
    import torch.distributed as tdist
    from paper_2112_01852_gb300 import dist
    tdist.init_process_group("gloo", rank=rank, world_size=world,
                             init_method="tcp://127.0.0.1:%d" % port)
    torch.cuda.set_device(0)
    dw.load_library()
    comm = dist.TComm()
    U, psi = make_case(DIMS, LS, 2, seed=71, links="haar")
    res = {}
    for prec in (dw.DW_F64, dw.DW_F32):
        dl = dist.DistLattice(comm, DIMS, LS, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=prec,
                              bc=BC)
        dl.load_gauge(U)
        x = dl.pack(psi)
        for op in OPS:
            y = dl.empty(2)
            dl.apply(op, y, x, None if op < dw.DW_OP_D else MF, 2)
            res["op_%d_%d" % (prec, op)] = dl.gather(y, 2)
        if prec == dw.DW_F64:
            xs = dl.empty(2)
            xs.zero_()
            conv, iters, true_res = dl.cg(xs, x, MF, 2, tol=1e-10, maxit=4000)
            res["cg_x"] = dl.gather(xs, 2)
            res["cg_conv"] = np.array(conv)
            res["cg_iters"] = np.array(iters)
            res["cg_res"] = np.array(true_res)
        dl.close()
    hi = dist.DistLattice(comm, DIMS, LS, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=dw.DW_F64,
                          bc=BC)
    lo = dist.DistLattice(comm, DIMS, LS, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=dw.DW_F32,
                          bc=BC)
    hi.load_gauge(U)
    lo.load_gauge(U)
    xb = hi.pack(psi)
    xm = hi.empty(2)
    xm.zero_()
    conv, iters, outer, true_res = hi.cg_mixed(lo, xm, xb, MF, 2, tol=1e-10, maxit=8000)
    res["mcg_x"] = hi.gather(xm, 2)
    res["mcg_conv"] = np.array(conv)
    res["mcg_outer"] = np.array(outer)
    res["mcg_res"] = np.array(true_res)
    hi.close()
    lo.close()
    if rank == 0:
        np.savez(path, **res)
    tdist.barrier()
    tdist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks(tmp_path_factory):
    import torch.multiprocessing as mp
    build_library()
    path = str(tmp_path_factory.mktemp("dist") / "ranks.npz")
    mp.start_processes(_worker, args=(2, _free_port(), path), nprocs=2, join=True,
                       start_method="spawn")
    return dict(np.load(path))


def _undecomposed(op, prec, U, psi):
    from paper_2112_01852_gb300.lattice import Lattice
    lat = Lattice(DIMS, LS, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=prec, bc=BC)
    lat.load_gauge(U)  # untuned: the default (variant-0) tile of the halo path
    x = lat.pack(psi)
    y = lat.empty(2)
    if op in (dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG):
        lat.dhop(y, x, 2, dag=op == dw.DW_OP_DHOP_DAG)
    elif op == dw.DW_OP_D:
        lat.D(y, x, MF, 2)
    else:
        lat.Ddag(y, x, MF, 2)
    out = lat.unpack(y, 2)
    lat.close()
    return out


@pytest.mark.parametrize("prec", [dw.DW_F64, dw.DW_F32], ids=["f64", "f32"])
@pytest.mark.parametrize("op", OPS, ids=["Dhop", "Dhop_dag", "D", "Ddag"])
def test_two_process_operators_bitwise(two_ranks, prec, op):
    U, psi = make_case(DIMS, LS, 2, seed=71, links="haar")
    got = two_ranks["op_%d_%d" % (prec, op)]
    assert np.array_equal(got, _undecomposed(op, prec, U, psi))
    if op in (dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG):
        ref = oracle.dhop(psi, U, DIMS, LS, BC, dag=op == dw.DW_OP_DHOP_DAG)
    else:
        ref = oracle.dw(psi, U, DIMS, LS, M5, B, C, MF, BC, dag=op == dw.DW_OP_DDAG)
    for r in range(2):
        assert oracle.rel_l2(got[r], ref[r]) <= TOL[prec]


def test_two_process_cg(two_ranks):
    U, psi = make_case(DIMS, LS, 2, seed=71, links="haar")
    x = two_ranks["cg_x"]
    assert two_ranks["cg_conv"].all()
    Ax = oracle.dwdagdw(x, U, DIMS, LS, M5, B, C, MF, BC)
    for r in range(2):
        rel = np.linalg.norm((psi[r] - Ax[r]).ravel()) / np.linalg.norm(psi[r].ravel())
        assert rel <= 1e-10, (r, rel)
        assert abs(two_ranks["cg_res"][r] - rel) <= 1e-3 * rel + 1e-15


def test_two_process_mixed_cg(two_ranks):
    U, psi = make_case(DIMS, LS, 2, seed=71, links="haar")
    x = two_ranks["mcg_x"]
    assert two_ranks["mcg_conv"].all() and 2 <= int(two_ranks["mcg_outer"]) <= 10
    Ax = oracle.dwdagdw(x, U, DIMS, LS, M5, B, C, MF, BC)
    for r in range(2):
        rel = np.linalg.norm((psi[r] - Ax[r]).ravel()) / np.linalg.norm(psi[r].ravel())
        assert rel <= 1e-10, (r, rel)
        assert abs(two_ranks["mcg_res"][r] - rel) <= 1e-3 * rel + 1e-15
