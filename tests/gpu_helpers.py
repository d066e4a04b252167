"""Shared helpers for the GPU parity tests (CUDA path vs the CPU oracle)."""

import numpy as np

import oracle
from paper_2112_01852_gb300 import dw, inputs

TOL = {dw.DW_F64: 1e-12, dw.DW_F32: 1e-5, dw.DW_F16: 5e-3}
BC = (1, 1, 1, -1)


def build_library():
    from paper_2112_01852_gb300 import build
    build.build()
    dw.load_library()


def make_case(dims, Ls, nrhs, seed, links="exp"):
    if links == "haar":
        U = inputs.haar_su3_field(dims, seed=seed)
    else:
        U = inputs.exp_su3_field(dims, seed=seed)
    psi = inputs.gaussian_fermion(dims, Ls, nrhs, seed=seed)
    return U, psi


def run_gpu(lat, op, psi, mf=None, nrhs=None):
    """Apply `op` (dw.DW_OP_*) through the C ABI to canonical psi; return canonical."""
    nrhs = psi.shape[0] if nrhs is None else nrhs
    x = lat.pack(psi)
    y = lat.empty(nrhs)
    if op == dw.DW_OP_DHOP:
        lat.dhop(y, x, nrhs)
    elif op == dw.DW_OP_DHOP_DAG:
        lat.dhop(y, x, nrhs, dag=True)
    elif op == dw.DW_OP_D:
        lat.D(y, x, mf, nrhs)
    elif op == dw.DW_OP_DDAG:
        lat.Ddag(y, x, mf, nrhs)
    elif op == dw.DW_OP_DDAGD:
        lat.DdagD(y, x, mf, nrhs)
    else:
        raise ValueError(op)
    return lat.unpack(y, nrhs)


def run_oracle(op, psi, U, dims, Ls, M5, b, c, mf, bc=BC):
    if op == dw.DW_OP_DHOP:
        return oracle.dhop(psi, U, dims, Ls, bc)
    if op == dw.DW_OP_DHOP_DAG:
        return oracle.dhop(psi, U, dims, Ls, bc, dag=True)
    if op == dw.DW_OP_D:
        return oracle.dw(psi, U, dims, Ls, M5, b, c, mf, bc)
    if op == dw.DW_OP_DDAG:
        return oracle.dw(psi, U, dims, Ls, M5, b, c, mf, bc, dag=True)
    if op == dw.DW_OP_DDAGD:
        return oracle.dwdagdw(psi, U, dims, Ls, M5, b, c, mf, bc)
    raise ValueError(op)


def rel_err_per_rhs(got, ref):
    return [oracle.rel_l2(got[r], ref[r]) for r in range(ref.shape[0])]


def max_rel(got, ref):
    return max(rel_err_per_rhs(got, ref))


ALL_OPS = (dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG, dw.DW_OP_D, dw.DW_OP_DDAG, dw.DW_OP_DDAGD)
STENCIL_OPS = (dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG, dw.DW_OP_D, dw.DW_OP_DDAG)
OP_NAMES = {dw.DW_OP_DHOP: "Dhop", dw.DW_OP_DHOP_DAG: "Dhop_dag", dw.DW_OP_D: "D",
            dw.DW_OP_DDAG: "Ddag", dw.DW_OP_DDAGD: "DdagD"}


def valid_tiles(Ls, txs=(32, 64, 128)):
    out = []
    for spt in (1, 2, 3, 4):
        if Ls % spt:
            continue
        for tx in txs:
            if tx * (Ls // spt) <= 1024:
                out.append((spt, tx))
    return out


def np_rng(seed):
    return np.random.default_rng(seed)
