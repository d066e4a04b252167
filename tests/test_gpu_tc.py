"""GPU parity of the tensor-core hopping term (stencil variant 8: FP16 storage,
the SU(3) x half-spinor products of Sec. 4.1 / Table 3 as mma.sync m16n8k16
blocks) against the CPU oracle, through the C ABI.

Its links and projected half spinors enter the tensor cores in FP16 and its
sums are FP32, so it is held to the FP16-storage tolerance; it must also agree
with the register kernels at that precision.
"""

import numpy as np
import pytest

from gpu_helpers import TOL, build_library, make_case, max_rel, run_gpu, run_oracle
from paper_2112_01852_gb300 import dw

pytestmark = pytest.mark.gpu

OPS = (dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()


def _lattice(dims, Ls, prec=dw.DW_F16, bc=(1, 1, 1, -1)):
    from paper_2112_01852_gb300.lattice import Lattice
    return Lattice(dims, Ls, kind=dw.DW_MOBIUS, M5=1.8, b=1.5, c=0.5, prec=prec, bc=bc)


@pytest.mark.parametrize("dims,Ls,nrhs", [((4, 4, 4, 8), 8, 2), ((6, 4, 2, 4), 12, 1),
                                          ((2, 6, 4, 2), 4, 3), ((8, 4, 4, 4), 16, 2)],
                         ids=["4x4x4x8_ls8", "6x4x2x4_ls12", "2x6x4x2_ls4", "8x4x4x4_ls16"])
def test_tensor_core_hop(dims, Ls, nrhs):
    bc = (1, -1, 1, -1)
    U, psi = make_case(dims, Ls, nrhs, seed=51, links="haar")
    lat = _lattice(dims, Ls, bc=bc)
    lat.load_gauge(U)
    for op in OPS:
        ref = run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, [0.0] * nrhs, bc)
        lat.set_tile(op, 1, 32, 8)
        got = run_gpu(lat, op, psi)
        assert max_rel(got, ref) <= TOL[dw.DW_F16], (op, max_rel(got, ref))
        lat.set_tile(op, 1, 32, 5)
        reg = run_gpu(lat, op, psi)
        assert max_rel(got, reg) <= TOL[dw.DW_F16]
    lat.close()


def test_tensor_core_hop_limits():
    dims, Ls = (4, 4, 4, 4), 8
    U, _ = make_case(dims, Ls, 1, seed=52)
    for prec in (dw.DW_F64, dw.DW_F32):  # FP16 storage only
        lat = _lattice(dims, Ls, prec=prec)
        with pytest.raises(dw.DWError) as e:
            lat.set_tile(dw.DW_OP_DHOP, 1, 32, 8)
        assert e.value.code == dw.DW_ERR_ARG
        lat.close()
    lat = _lattice(dims, Ls)
    for op, spt, tx in ((dw.DW_OP_D, 1, 32), (dw.DW_OP_DHOP, 2, 32), (dw.DW_OP_DHOP, 1, 64)):
        with pytest.raises(dw.DWError) as e:  # not the hopping term, or not its one tile
            lat.set_tile(op, spt, tx, 8)
        assert e.value.code == dw.DW_ERR_ARG
    lat.close()
    lat = _lattice((4, 4, 4, 4), 6)  # Ls not a multiple of 4
    with pytest.raises(dw.DWError):
        lat.set_tile(dw.DW_OP_DHOP, 1, 32, 8)
    lat.close()
