"""GPU parity of the interleaved-complex layout (the layout ablation of Sec. 4.3,
Table 3: the counterpart of the paper's RIRI layout beside the default
spin-pair, RRII-like one) against the CPU oracle, through the C ABI.

The layout changes how the FP32 quads hold a spin pair ((Re j0, Im j0, Re j1,
Im j1) instead of (Re j0, Re j1, Im j0, Im j1)) and how the stencil pairs its
packed arithmetic; the operator is the same, so both layouts must match the
oracle within the FP32 tolerance, and the layout conversion must round each
real exactly as the default one does.
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


def _lattice(dims, Ls, prec=dw.DW_F32, bc=(1, 1, 1, -1)):
    from paper_2112_01852_gb300.lattice import Lattice
    return Lattice(dims, Ls, kind=dw.DW_MOBIUS, M5=1.8, b=1.5, c=0.5, prec=prec, bc=bc)


def test_complex_layout_roundtrip_rounds_like_the_default():
    dims, Ls = (3, 5, 2, 7), 6
    _, psi = make_case(dims, Ls, 2, seed=41)
    lat = _lattice(dims, Ls)
    dw.dw_set_complex_layout(lat.handle, 1)
    got = lat.unpack(lat.pack(psi), 2)
    want = psi.real.astype(np.float32).astype(np.float64) + \
        1j * psi.imag.astype(np.float32).astype(np.float64)
    assert np.array_equal(got, want)
    lat.close()
    # the same field packed under the two layouts differs in memory order only
    # (a lattice without padding sites, so every byte of the field is written)
    dims, Ls = (8, 4, 2, 2), 4
    _, psi = make_case(dims, Ls, 1, seed=44)
    lat = _lattice(dims, Ls)
    dw.dw_set_complex_layout(lat.handle, 1)
    a = lat.pack(psi).cpu().numpy().view(np.float32)
    dw.dw_set_complex_layout(lat.handle, 0)
    b = lat.pack(psi).cpu().numpy().view(np.float32)
    assert not np.array_equal(a, b)
    # quad k holds (Re j0, Im j0, Re j1, Im j1) against (Re j0, Re j1, Im j0, Im j1)
    assert np.array_equal(a.reshape(-1, 4)[:, [0, 2, 1, 3]], b.reshape(-1, 4))
    lat.close()


@pytest.mark.parametrize("dims", [(32, 4, 2, 6), (3, 5, 2, 7)], ids=["Lx32", "ragged"])
def test_complex_layout_hopping_term(dims):
    Ls = 4
    U, psi = make_case(dims, Ls, 2, seed=42)
    lat = _lattice(dims, Ls)
    lat.load_gauge(U)
    dw.dw_set_complex_layout(lat.handle, 1)
    ran = set()
    for op in OPS:
        ref = run_oracle(op, psi, U, dims, Ls, 1.8, 1.5, 0.5, [0.0, 0.0])
        for var in (4, 5, 6, 7):
            for spt, tx, sgrp in ((1, 32, 1), (2, 64, 2), (2, 128, 1), (4, 32, 1)):
                try:
                    lat.set_tile(op, spt, tx, var, sgrp=sgrp)
                except dw.DWError as e:
                    assert e.code == dw.DW_ERR_ARG  # rows variants need Lx = 32
                    continue
                got = run_gpu(lat, op, psi)
                assert max_rel(got, ref) <= TOL[dw.DW_F32], (op, var, spt, tx, sgrp)
                ran.add(var)
    assert {4, 5} <= ran
    if dims[0] == 32:
        assert {6, 7} <= ran
    dw.dw_device_status(lat.handle)
    # the tuner stays within the variants the layout has
    spt, tx, var, zblk, sgrp = lat.tune(dw.DW_OP_DHOP, 1)
    assert var in (4, 5, 6, 7)
    got = run_gpu(lat, dw.DW_OP_DHOP, psi[:1])
    assert max_rel(got, run_oracle(dw.DW_OP_DHOP, psi[:1], U, dims, Ls, 1.8, 1.5, 0.5,
                                   [0.0])) <= TOL[dw.DW_F32]
    lat.close()


def test_complex_layout_limits():
    dims, Ls = (4, 4, 4, 4), 4
    U, psi = make_case(dims, Ls, 1, seed=43)
    lat64 = _lattice(dims, Ls, prec=dw.DW_F64)
    with pytest.raises(dw.DWError) as e:
        dw.dw_set_complex_layout(lat64.handle, 1)
    assert e.value.code == dw.DW_ERR_ARG
    lat64.close()
    lat = _lattice(dims, Ls)
    lat.load_gauge(U)
    dw.dw_set_complex_layout(lat.handle, 1)
    x = lat.pack(psi)
    y = lat.empty(1)
    for f in (lat.D, lat.Ddag, lat.DdagD):
        with pytest.raises(dw.DWError) as e:
            f(y, x, [0.01])
        assert e.value.code == dw.DW_ERR_STATE
    with pytest.raises(dw.DWError) as e:
        lat.set_tile(dw.DW_OP_DHOP, 1, 32, 0)  # variant 0 is not built for this layout
    assert e.value.code == dw.DW_ERR_ARG
    lat.close()
