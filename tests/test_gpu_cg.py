"""GPU conjugate gradient on D^+D x = b through the C ABI.

Every solution is judged by the oracle's own FP64 recomputation of the true
residual |b - D^+D x| / |b| (several x are correct to rounding, so the
iterate is checked by its residual), plus a dense solve on a tiny lattice.
"""

import numpy as np
import pytest

import oracle
from gpu_helpers import BC, build_library, make_case
from oracle import dense
from paper_2112_01852_gb300 import dw, inputs

pytestmark = pytest.mark.gpu

M5, B, C = 1.8, 1.5, 0.5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()


def _solve(dims, Ls, U, rhs, mfs, mode, tol=1e-10, maxit=20000, x0=None, kind=dw.DW_MOBIUS):
    from paper_2112_01852_gb300.lattice import Lattice
    lat = Lattice(dims, Ls, kind=kind, M5=M5, b=B, c=C, prec=dw.DW_F64)
    lat.load_gauge(U)
    nrhs = rhs.shape[0]
    b = lat.pack(rhs)
    x = lat.pack(np.zeros_like(rhs) if x0 is None else x0)
    status, stats = lat.cg(x, b, mfs, nrhs=nrhs, tol=tol, maxit=maxit, mode=mode)
    xs = lat.unpack(x, nrhs)
    lat.close()
    return status, stats, xs


def _true_resid(xs, rhs, U, dims, Ls, mfs, b=B, c=C):
    Ax = oracle.dwdagdw(xs, U, dims, Ls, M5, b, c, mfs, BC)
    return [np.linalg.norm((rhs[r] - Ax[r]).ravel()) / np.linalg.norm(rhs[r].ravel())
            for r in range(rhs.shape[0])]


MODES = [(dw.DW_F64, "f64"), (dw.DW_F32, "f32"), (dw.DW_F16, "f16")]


@pytest.mark.parametrize("mode", [m for m, _ in MODES], ids=[n for _, n in MODES])
def test_cg_tiny_matches_dense_solve(mode):
    dims, Ls = (2, 2, 2, 2), 4
    U, rhs = make_case(dims, Ls, 2, seed=21)
    mfs = [0.01, 0.1]
    status, stats, xs = _solve(dims, Ls, U, rhs, mfs, mode)
    assert status == dw.DW_OK
    for r, mf in enumerate(mfs):
        D = dense.dw5(U, dims, Ls, M5, B, C, mf, BC)
        A = D.conj().T @ D
        ref = np.linalg.solve(A, rhs[r].ravel())
        # |x - x*| / |x*| <= cond(A) * |b - A x| / |b|
        assert oracle.rel_l2(xs[r].ravel(), ref) <= np.linalg.cond(A) * 1e-10
        assert stats[r].converged == 1
        assert stats[r].true_resid <= 1e-10
    for res in _true_resid(xs, rhs, U, dims, Ls, mfs):
        assert res <= 1e-10


@pytest.mark.parametrize("mode", [m for m, _ in MODES], ids=[n for _, n in MODES])
def test_cg_8x4_ls8_true_residual(mode):
    dims, Ls = (8, 8, 8, 8), 8
    U, rhs = make_case(dims, Ls, 1, seed=22)
    status, stats, xs = _solve(dims, Ls, U, rhs, [0.01], mode)
    assert status == dw.DW_OK, stats[0].iters
    assert stats[0].converged == 1 and stats[0].iters > 0
    if mode != dw.DW_F64:
        assert stats[0].reliable_updates >= 1
    res = _true_resid(xs, rhs, U, dims, Ls, [0.01])[0]
    assert res <= 1e-10
    # the solver's own FP64 residual agrees with the oracle's
    assert abs(stats[0].true_resid - res) <= 1e-11


def test_cg_batched_uneven_masses_f32():
    dims, Ls = (4, 4, 4, 8), 12
    mfs = [0.005] * 5 + [0.01] * 4 + [0.02] * 2 + [0.05]
    U, rhs = make_case(dims, Ls, len(mfs), seed=4)
    status, stats, xs = _solve(dims, Ls, U, rhs, mfs, dw.DW_F32)
    assert status == dw.DW_OK
    res = _true_resid(xs, rhs, U, dims, Ls, mfs)
    for r in range(len(mfs)):
        assert stats[r].converged == 1
        assert res[r] <= 1e-10
    # lighter masses need more iterations
    assert stats[0].iters >= stats[len(mfs) - 1].iters


def test_cg_shamir_f16():
    dims, Ls = (4, 4, 4, 4), 8
    U, rhs = make_case(dims, Ls, 1, seed=23, links="haar")
    status, stats, xs = _solve(dims, Ls, U, rhs, [0.02], dw.DW_F16, kind=dw.DW_SHAMIR)
    assert status == dw.DW_OK
    Ax = oracle.dwdagdw(xs, U, dims, Ls, M5, 1.0, 0.0, [0.02], BC)
    assert np.linalg.norm((rhs - Ax).ravel()) / np.linalg.norm(rhs.ravel()) <= 1e-10


def test_cg_maxit_reports_not_converged():
    dims, Ls = (4, 4, 4, 4), 8
    U, rhs = make_case(dims, Ls, 1, seed=24)
    status, stats, _ = _solve(dims, Ls, U, rhs, [0.01], dw.DW_F32, maxit=5)
    assert status == dw.DW_ERR_NOT_CONVERGED
    assert stats[0].converged == 0
    assert 5 <= stats[0].iters <= 5 + 8
    assert stats[0].true_resid > 1e-10


def test_cg_resume_from_solution_and_zero_source():
    dims, Ls = (4, 4, 4, 4), 4
    U, rhs = make_case(dims, Ls, 2, seed=25)
    rhs[1] = 0.0
    status, stats, xs = _solve(dims, Ls, U, rhs, [0.01, 0.01], dw.DW_F32)
    assert status == dw.DW_OK
    assert np.all(xs[1] == 0) and stats[1].converged == 1
    # restarting from the solution converges without inner iterations
    status, stats2, xs2 = _solve(dims, Ls, U, rhs[:1], [0.01], dw.DW_F32, x0=xs[:1])
    assert status == dw.DW_OK and stats2[0].iters == 0
    assert np.array_equal(xs2[0], xs[0])


def test_cg_nan_source_is_breakdown():
    dims, Ls = (4, 4, 4, 4), 4
    U, rhs = make_case(dims, Ls, 1, seed=26)
    rhs[0, 3, 1, 2, 1] = np.nan
    with pytest.raises(dw.DWError) as e:
        _solve(dims, Ls, U, rhs, [0.01], dw.DW_F32)
    assert e.value.code == dw.DW_ERR_BREAKDOWN


def test_cg_argument_errors():
    from paper_2112_01852_gb300.lattice import Lattice
    dims, Ls = (4, 4, 4, 4), 4
    U, rhs = make_case(dims, Ls, 1, seed=27)
    lat = Lattice(dims, Ls, prec=dw.DW_F64)
    b = lat.pack(rhs)
    x = lat.empty(1)
    with pytest.raises(dw.DWError) as e:
        lat.cg(x, b, [0.01])  # gauge not loaded
    assert e.value.code == dw.DW_ERR_STATE
    lat.load_gauge(U)
    for kwargs in ({"tol": 0.0}, {"maxit": 0}, {"mode": 9}):
        with pytest.raises(dw.DWError) as e:
            lat.cg(x, b, [0.01], **kwargs)
        assert e.value.code == dw.DW_ERR_ARG
    with pytest.raises(dw.DWError) as e:
        lat.cg(b, b, [0.01])
    assert e.value.code == dw.DW_ERR_ARG
    lat.close()


def test_cg_tunes_its_inner_operator():
    # the solver times tiles for its inner operator; every z-blocking it may
    # choose must divide Lz (24 here: the automatic blocking is 3, which is
    # neither 1, 2 nor 4)
    from paper_2112_01852_gb300.lattice import Lattice
    dims, Ls = (8, 8, 24, 4), 8
    U, b = make_case(dims, Ls, 1, seed=71)
    lat = Lattice(dims, Ls, kind=dw.DW_MOBIUS, M5=1.8, b=1.5, c=0.5, prec=dw.DW_F64)
    lat.load_gauge(U)
    bd = lat.pack(b)
    x = lat.empty(1)
    x.zero_()
    lat.cg(x, bd, [0.1], nrhs=1, tol=1e-8, maxit=50, mode=dw.DW_F32)
    for op in (dw.DW_OP_D, dw.DW_OP_DDAG):
        spt, tx, variant, zblk, sgrp = dw.dw_get_tile(lat.handle, op, dw.DW_F32, 1)
        assert Ls % spt == 0 and tx % 32 == 0 and dims[2] % zblk == 0
        assert (Ls // spt) % sgrp == 0 and (op == dw.DW_OP_D or sgrp <= 8)
    lat.close()


def test_reliable_delta_setting():
    # dw_set_reliable_delta: values outside [0, 1) are refused; a smaller
    # threshold means fewer FP64 reliable updates, and every setting still
    # reaches an oracle-recomputed residual <= 1e-10
    from paper_2112_01852_gb300.lattice import Lattice
    dims, Ls = (8, 8, 8, 8), 8
    U, rhs = make_case(dims, Ls, 1, seed=22)
    lat = Lattice(dims, Ls, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=dw.DW_F64)
    lat.load_gauge(U)
    for bad in (-0.1, 1.0, float("nan")):
        with pytest.raises(dw.DWError) as e:
            dw.dw_set_reliable_delta(lat.handle, bad)
        assert e.value.code == dw.DW_ERR_ARG
    b = lat.pack(rhs)
    updates = {}
    for delta in (0.1, 1e-5, 0.0):  # 0: the default, 1e-3 for FP32 inner fields
        dw.dw_set_reliable_delta(lat.handle, delta)
        x = lat.empty(1)
        x.zero_()
        status, stats = lat.cg(x, b, [0.01], nrhs=1, tol=1e-10, maxit=20000, mode=dw.DW_F32)
        assert status == dw.DW_OK and stats[0].converged == 1
        assert _true_resid(lat.unpack(x, 1), rhs, U, dims, Ls, [0.01])[0] <= 1e-10
        updates[delta] = stats[0].reliable_updates
    assert updates[1e-5] <= updates[0.0] < updates[0.1], updates
    lat.close()
