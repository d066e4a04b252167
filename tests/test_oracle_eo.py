"""Pins for the even-odd oracle (``oracle/eo.py``) against what the mathematics
fixes (no GPU): the Schur complement equals block elimination on the
independent dense-matrix build, the even-even block of that build is the
one-site matrix of the local part, the even-odd solve reproduces D x = eta,
and the adjoints are adjoint."""

import numpy as np
import pytest

import oracle
from oracle import dense, eo
from paper_2112_01852_gb300 import inputs

M5, B, C = 1.8, 1.5, 0.5


def _blocks(dims, Ls):
    """Index sets (canonical vector order) of the even and the odd sites."""
    par = eo.parity(dims)
    per_site = 12 * Ls
    idx = np.arange(len(par) * per_site).reshape(len(par), per_site)
    return idx[par == 0].ravel(), idx[par == 1].ravel()


@pytest.mark.parametrize("bc", [(1, 1, 1, -1), (-1, 1, -1, -1)])
@pytest.mark.parametrize("mf", [0.01, 0.3])
def test_schur_matches_dense_block_elimination(bc, mf):
    dims, Ls = (2, 2, 2, 2), 4
    U = inputs.haar_su3_field(dims, seed=31)
    D = dense.dw5(U, dims, Ls, M5, B, C, mf, bc)
    ie, io = _blocks(dims, Ls)
    Dee, Deo, Doe, Doo = D[np.ix_(ie, ie)], D[np.ix_(ie, io)], D[np.ix_(io, ie)], D[np.ix_(io, io)]
    # the even-even block is the one-site local part on every even site
    A1 = eo.m5_matrix(Ls, M5, B, C, mf)
    nsite = len(ie) // (12 * Ls)
    assert np.allclose(Dee, np.kron(np.eye(nsite), A1), atol=1e-14)
    assert np.allclose(Doo, np.kron(np.eye(nsite), A1), atol=1e-14)
    S = Doo - Doe @ np.linalg.solve(Dee, Deo)
    psi = inputs.gaussian_fermion(dims, Ls, 1, seed=32)
    x_o = eo.project(psi, dims, 1)
    got = eo.schur(x_o, U, dims, Ls, M5, B, C, [mf], bc).ravel()
    ref = np.zeros_like(got)
    ref[io] = S @ x_o.ravel()[io]
    assert oracle.rel_l2(got, ref) < 1e-13
    got_dag = eo.schur_dag(x_o, U, dims, Ls, M5, B, C, [mf], bc).ravel()
    ref_dag = np.zeros_like(got_dag)
    ref_dag[io] = S.conj().T @ x_o.ravel()[io]
    assert oracle.rel_l2(got_dag, ref_dag) < 1e-13
    # even-site parts are zero
    assert np.all(got[ie] == 0) and np.all(got_dag[ie] == 0)


def test_local_inverse_and_adjoint():
    dims, Ls = (2, 2, 2, 4), 6
    psi = inputs.gaussian_fermion(dims, Ls, 2, seed=33)
    mf = [0.02, 0.5]
    for dag in (False, True):
        back = eo.m5_inv(eo.m5(psi, dims, Ls, M5, B, C, mf, dag=dag), dims, Ls, M5, B, C, mf,
                         dag=dag)
        assert oracle.rel_l2(back, psi) < 1e-13
    # A^+ is the conjugate transpose of A on one site
    A = eo.m5_matrix(Ls, M5, B, C, 0.1)
    Ad = eo.m5_matrix(Ls, M5, B, C, 0.1, dag=True)
    assert np.allclose(Ad, A.conj().T, atol=1e-15)


def test_schur_adjointness_on_larger_lattice():
    dims, Ls = (4, 2, 4, 2), 4
    bc = (1, -1, 1, -1)
    U = inputs.exp_su3_field(dims, seed=34)
    x = eo.project(inputs.gaussian_fermion(dims, Ls, 1, seed=35), dims, 1)
    y = eo.project(inputs.gaussian_fermion(dims, Ls, 1, seed=36), dims, 1)
    lhs = oracle.inner(y, eo.schur(x, U, dims, Ls, M5, B, C, [0.05], bc))
    rhs = oracle.inner(eo.schur_dag(y, U, dims, Ls, M5, B, C, [0.05], bc), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_even_odd_solve_solves_full_system():
    dims, Ls = (4, 2, 2, 4), 4
    bc = (-1, 1, 1, -1)
    U = inputs.haar_su3_field(dims, seed=37)
    eta = inputs.gaussian_fermion(dims, Ls, 1, seed=38)
    x = eo.solve(eta, U, dims, Ls, M5, B, C, [0.1], bc, tol=1e-13)
    res = oracle.dw(x, U, dims, Ls, M5, B, C, [0.1], bc) - eta
    assert np.linalg.norm(res) / np.linalg.norm(eta) < 1e-10
