"""Parity at the full production size, in the launch configuration the
benchmark times (tuned tiles): Moebius Dhop, D, D^+ and D^+D at 32^3 x 64 x
Ls=12 in FP32 and FP16 storage, links exp(i 0.3 H), seed 5.  The oracle
evaluates a sample of 4D sites (all slices) -- every lattice face and corner
class is included -- and the GPU result is compared there element by element.
For D^+D the oracle first evaluates D psi on the sample and its 4D neighbours
(all that D^+ reads at the sample), then D^+ of that at the sample.
"""

import numpy as np
import pytest

import oracle
from gpu_helpers import BC, TOL, build_library
from paper_2112_01852_gb300 import dw, inputs

pytestmark = pytest.mark.gpu

DIMS, LS, SEED = (32, 32, 32, 64), 12, 5
M5, B, C, MF = 1.8, 1.5, 0.5, 0.01


def _sample_sites(dims, n, seed):
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz, Lt = dims
    V4 = Lx * Ly * Lz * Lt
    sites = set(rng.choice(V4, size=n, replace=False).tolist())
    # every combination of first/last coordinate in each direction
    for mask in range(81):
        c = []
        m = mask
        for L in dims:
            c.append((0, L - 1, L // 2)[m % 3])
            m //= 3
        sites.add(c[0] + Lx * (c[1] + Ly * (c[2] + Lz * c[3])))
    return np.array(sorted(sites), dtype=np.int64)


@pytest.fixture(scope="module")
def fullsize():
    build_library()
    U = inputs.exp_su3_field(DIMS, seed=SEED)
    psi = inputs.gaussian_fermion(DIMS, LS, 1, seed=SEED)
    sites = _sample_sites(DIMS, 2048, seed=99)
    ref = {
        dw.DW_OP_DHOP: oracle.dhop(psi, U, DIMS, LS, BC, sites=sites),
        dw.DW_OP_D: oracle.dw(psi, U, DIMS, LS, M5, B, C, [MF], BC, sites=sites),
        dw.DW_OP_DDAG: oracle.dw(psi, U, DIMS, LS, M5, B, C, [MF], BC, dag=True, sites=sites),
    }
    near = _with_neighbours(DIMS, sites)
    d_near = np.zeros_like(psi)
    d_near[0, near] = oracle.dw(psi, U, DIMS, LS, M5, B, C, [MF], BC, sites=near)[0]
    ref[dw.DW_OP_DDAGD] = oracle.dw(d_near, U, DIMS, LS, M5, B, C, [MF], BC, dag=True,
                                    sites=sites)
    del d_near
    return U, psi, sites, ref


def _with_neighbours(dims, sites):
    """The sites and their eight 4D neighbours (periodic), sorted, unique."""
    Lx, Ly, Lz, Lt = dims
    c = [sites % Lx, sites // Lx % Ly, sites // (Lx * Ly) % Lz, sites // (Lx * Ly * Lz)]
    out = [sites]
    for mu, L in enumerate(dims):
        for step in (1, -1):
            cc = list(c)
            cc[mu] = (c[mu] + step) % L
            out.append(cc[0] + Lx * (cc[1] + Ly * (cc[2] + Lz * cc[3])))
    return np.unique(np.concatenate(out))


@pytest.mark.parametrize("prec", [dw.DW_F32, dw.DW_F16], ids=["f32", "f16"])
def test_fullsize_tuned_operators(fullsize, prec):
    import torch
    from paper_2112_01852_gb300.lattice import Lattice
    U, psi, sites, ref = fullsize
    lat = Lattice(DIMS, LS, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=prec)
    lat.load_gauge(U)
    x = lat.pack(psi)
    y = lat.empty(1)
    for op in (dw.DW_OP_DHOP, dw.DW_OP_D, dw.DW_OP_DDAG, dw.DW_OP_DDAGD):
        if op != dw.DW_OP_DDAGD:
            lat.tune(op, 1)  # the configuration bench.py times (D^+D: the D and D^+ tiles)
        if op == dw.DW_OP_DHOP:
            lat.dhop(y, x)
        elif op == dw.DW_OP_D:
            lat.D(y, x, [MF])
        elif op == dw.DW_OP_DDAG:
            lat.Ddag(y, x, [MF])
        else:
            lat.DdagD(y, x, [MF])
        got = lat.unpack(y)[0][sites]
        err = oracle.rel_l2(got, ref[op][0])
        assert err <= TOL[prec], (op, err)
    del x, y
    torch.cuda.synchronize()
    lat.close()
