"""Even-odd preconditioning on the GPU against the even-odd oracle
(``oracle/eo.py``): parity split and merge, the local part A and its inverse
(and adjoints), the Schur complement Dhat and Dhat^+ at FP64, FP32 and FP16
storage, on lattices with even, unequal extents."""

import numpy as np
import pytest

import oracle
from oracle import eo
from gpu_helpers import TOL, build_library, make_case
from paper_2112_01852_gb300 import dw

pytestmark = pytest.mark.gpu

M5, B, C = 1.8, 1.5, 0.5
CASES = [((2, 2, 2, 2), 4, (1, 1, 1, -1)), ((4, 6, 2, 2), 6, (-1, 1, 1, -1)),
         ((8, 4, 6, 10), 12, (1, 1, 1, -1))]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()


def _lattice(dims, Ls, prec, bc):
    from paper_2112_01852_gb300.lattice import Lattice
    return Lattice(dims, Ls, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=prec, bc=bc)


@pytest.mark.parametrize("prec", [dw.DW_F64, dw.DW_F32, dw.DW_F16], ids=["f64", "f32", "f16"])
def test_split_merge_roundtrip(prec):
    dims, Ls, bc = CASES[1]
    _, psi = make_case(dims, Ls, 2, seed=51)
    lat = _lattice(dims, Ls, prec, bc)
    full = lat.pack(psi)
    even, odd = lat.pack_eo(psi)
    back = lat.empty(2)
    dw.dw_eo_merge(lat.handle, back.data_ptr(), even.data_ptr(), odd.data_ptr(), prec, 2)
    assert np.array_equal(lat.unpack(back, 2), lat.unpack(full, 2))
    # the odd field holds exactly the odd sites
    zero = lat.empty_eo(2)
    zero.zero_()
    only_odd = lat.unpack_eo(zero, odd, 2)
    ref = eo.project(lat.unpack(full, 2), dims, 1)
    assert np.array_equal(only_odd, ref)
    lat.close()


@pytest.mark.parametrize("prec", [dw.DW_F64, dw.DW_F32], ids=["f64", "f32"])
@pytest.mark.parametrize("inverse", [False, True], ids=["A", "Ainv"])
@pytest.mark.parametrize("dag", [False, True], ids=["", "dag"])
def test_local_part(prec, inverse, dag):
    dims, Ls, bc = CASES[1]
    _, psi = make_case(dims, Ls, 2, seed=52)
    mf = [0.03, 0.4]
    lat = _lattice(dims, Ls, prec, bc)
    even, odd = lat.pack_eo(psi)
    out = lat.empty_eo(2)
    dw.dw_apply_m5_eo(lat.handle, out.data_ptr(), even.data_ptr(), mf, 2, int(inverse), int(dag))
    zero = lat.empty_eo(2)
    zero.zero_()
    got = lat.unpack_eo(out, zero, 2)
    x = eo.project(lat.unpack(lat.pack(psi), 2), dims, 0)
    f = eo.m5_inv if inverse else eo.m5
    ref = f(x, dims, Ls, M5, B, C, mf, dag=dag)
    assert oracle.rel_l2(got, ref) <= TOL[prec]
    lat.close()


@pytest.mark.parametrize("prec", [dw.DW_F64, dw.DW_F32, dw.DW_F16], ids=["f64", "f32", "f16"])
@pytest.mark.parametrize("case", range(3))
@pytest.mark.parametrize("dag", [False, True], ids=["Dhat", "Dhat_dag"])
def test_schur_complement(prec, case, dag):
    dims, Ls, bc = CASES[case]
    U, psi = make_case(dims, Ls, 2, seed=53 + case, links="haar")
    mf = [0.02, 0.1]
    lat = _lattice(dims, Ls, prec, bc)
    lat.load_gauge(U)
    _, odd = lat.pack_eo(psi)
    out = lat.empty_eo(2)
    dw.dw_apply_schur(lat.handle, out.data_ptr(), odd.data_ptr(), mf, 2, int(dag))
    zero = lat.empty_eo(2)
    zero.zero_()
    got = lat.unpack_eo(zero, out, 2)
    x = eo.project(lat.unpack(lat.pack(psi), 2), dims, 1)
    f = eo.schur_dag if dag else eo.schur
    for r in range(2):
        ref = f(x[r:r + 1], U, dims, Ls, M5, B, C, [mf[r]], bc)
        assert oracle.rel_l2(got[r:r + 1], ref) <= TOL[prec], r
    lat.close()


def test_eo_needs_even_extents():
    from paper_2112_01852_gb300.lattice import Lattice
    for dims in ((3, 2, 2, 2), (2, 3, 2, 2), (2, 2, 2, 5)):
        lat = Lattice(dims, 4, prec=dw.DW_F64)
        assert dw.dw_fermion_bytes_eo(lat.handle, dw.DW_F64, 1) == 0
        with pytest.raises(dw.DWError) as e:
            dw.dw_apply_schur(lat.handle, 16, 32, [0.1], 1, 0)
        assert e.value.code == dw.DW_ERR_ARG
        lat.close()


@pytest.mark.parametrize("mode", [dw.DW_F64, dw.DW_F32, dw.DW_F16], ids=["f64", "mixed_f32",
                                                                         "mixed_f16"])
def test_solve_eo(mode):
    # D x = eta through the odd-site Schur system, solved to tol on D x = eta
    # itself: the full-lattice residual, recomputed by the oracle, is at most
    # tol, and the preconditioned CG needs fewer iterations than CG on
    # D^+D x = D^+ eta
    dims, Ls, bc = (4, 4, 4, 8), 8, (1, 1, 1, -1)
    U, eta = make_case(dims, Ls, 2, seed=61)
    mf = [0.05, 0.2]
    lat = _lattice(dims, Ls, dw.DW_F64, bc)
    lat.load_gauge(U)
    e = lat.pack(eta)
    x = lat.empty(2)
    x.zero_()
    status, stats = lat.solve_eo(x, e, mf, nrhs=2, tol=1e-10, maxit=5000, mode=mode)
    assert status == dw.DW_OK
    xs = lat.unpack(x, 2)
    for r in range(2):
        assert stats[r].converged == 1
        res = oracle.dw(xs[r:r + 1], U, dims, Ls, M5, B, C, [mf[r]], bc) - eta[r:r + 1]
        rel = np.linalg.norm(res) / np.linalg.norm(eta[r])
        assert rel <= 1e-10, (r, rel)
        assert stats[r].true_resid <= 1e-10
        assert abs(stats[r].true_resid - rel) <= 1e-3 * max(rel, 1e-14) + 1e-15
    # unpreconditioned CG on the normal equations for comparison
    b = lat.pack(oracle.dw(eta, U, dims, Ls, M5, B, C, mf, bc, dag=True))
    y = lat.empty(2)
    y.zero_()
    _, full = lat.cg(y, b, mf, nrhs=2, tol=1e-10, maxit=20000, mode=mode)
    for r in range(2):
        assert stats[r].iters < full[r].iters, (stats[r].iters, full[r].iters)
    lat.close()
