"""Pins for the CPU oracle against what the mathematics fixes (no GPU).

Each test checks the oracle (``oracle/dw_oracle.cpp``) against something other
than itself: the independent dense-matrix build, free-field closed forms in
momentum space, gauge covariance, gamma5-hermiticity / adjointness, textbook
special cases, and the flop count printed in the paper's Table 3.
"""

import os

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2112_01852_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BC = (1, 1, 1, -1)


def _rand_fermion(dims, Ls, nrhs, seed):
    return inputs.gaussian_fermion(dims, Ls, nrhs, seed=seed)


def _vec(f):
    return np.asarray(f).reshape(f.shape[0], -1)


# --------------------------------------------------------------------------
# gamma algebra used by the dense build (the C++ oracle types its own table)


def test_gamma_clifford_algebra():
    g, g5 = dense.gammas()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))
        assert np.allclose(g5 @ g[mu] + g[mu] @ g5, 0)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


# --------------------------------------------------------------------------
# T6: stencil oracle == dense build on 2^4 x Ls=4 (and Ls=1 Wilson, T8)


@pytest.mark.parametrize("Ls", [4, 1])
@pytest.mark.parametrize("dag", [False, True])
def test_dhop_matches_dense(Ls, dag):
    dims = (2, 2, 2, 2)
    U = inputs.haar_su3_field(dims, seed=11)
    psi = _rand_fermion(dims, Ls, 1, seed=12)
    ref = dense.dhop5(U, dims, Ls, BC, dag=dag) @ psi.ravel()
    got = oracle.dhop(psi, U, dims, Ls, BC, dag=dag)
    assert oracle.rel_l2(got.ravel(), ref) < 1e-14


def test_dhop_matches_dense_nonuniform_dims_and_bc():
    dims = (2, 3, 2, 4)
    bc = (-1, 1, -1, -1)
    U = inputs.haar_su3_field(dims, seed=21)
    psi = _rand_fermion(dims, 2, 1, seed=22)
    ref = dense.dhop5(U, dims, 2, bc) @ psi.ravel()
    got = oracle.dhop(psi, U, dims, 2, bc)
    assert oracle.rel_l2(got.ravel(), ref) < 1e-14


@pytest.mark.parametrize("kind", ["shamir", "mobius"])
def test_dw_and_dagger_match_dense(kind):
    dims = (2, 2, 2, 2)
    Ls = 4
    M5 = 1.8
    b, c = (1.0, 0.0) if kind == "shamir" else (1.5, 0.5)
    mfs = [0.01, 0.3]
    U = inputs.haar_su3_field(dims, seed=31)
    psi = _rand_fermion(dims, Ls, 2, seed=32)
    got = oracle.dw(psi, U, dims, Ls, M5, b, c, mfs, BC)
    gotd = oracle.dw(psi, U, dims, Ls, M5, b, c, mfs, BC, dag=True)
    for r, mf in enumerate(mfs):
        D = dense.dw5(U, dims, Ls, M5, b, c, mf, BC)
        assert oracle.rel_l2(got[r].ravel(), D @ psi[r].ravel()) < 1e-14
        assert oracle.rel_l2(gotd[r].ravel(), D.conj().T @ psi[r].ravel()) < 1e-14


def test_k_matches_dense_and_ls1():
    dims = (2, 2, 2, 2)
    for Ls in (1, 2, 5):
        psi = _rand_fermion(dims, Ls, 1, seed=40 + Ls)
        K = dense.k5(16, Ls, 0.07)
        assert oracle.rel_l2(oracle.kop(psi, dims, Ls, 0.07).ravel(), K @ psi.ravel()) < 1e-15
        assert oracle.rel_l2(oracle.kop(psi, dims, Ls, 0.07, dag=True).ravel(),
                             K.conj().T @ psi.ravel()) < 1e-15
    psi = _rand_fermion(dims, 1, 1, seed=49)
    assert np.allclose(oracle.kop(psi, dims, 1, 0.25), -0.25 * psi)


# --------------------------------------------------------------------------
# T1 / T2: free field (U = 1) against closed forms in momentum space


def _plane_wave(dims, p):
    V4 = int(np.prod(dims))
    x4 = np.arange(V4)
    c = []
    r = x4.copy()
    for L in dims:
        c.append(r % L)
        r //= L
    phase = sum(p[mu] * c[mu] for mu in range(4))
    return np.exp(1j * phase)


def _unit_links(dims):
    V4 = int(np.prod(dims))
    return np.broadcast_to(np.eye(3, dtype=complex), (V4, 4, 3, 3)).copy()


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 2, 0, 3), (3, 1, 1, 1)])
def test_free_dhop_plane_wave(n):
    dims = (4, 4, 4, 6)
    p = [2 * np.pi * n[k] / dims[k] for k in range(3)] + [(2 * n[3] + 1) * np.pi / dims[3]]
    Ls = 3
    rng = np.random.default_rng(5)
    chi = rng.standard_normal((Ls, 4, 3)) + 1j * rng.standard_normal((Ls, 4, 3))
    e = _plane_wave(dims, p)
    psi = e[:, None, None, None] * chi[None]
    g, _ = dense.gammas()
    M = 2 * sum(np.cos(pm) for pm in p) * np.eye(4) - 2j * sum(
        np.sin(p[mu]) * g[mu] for mu in range(4))
    expect = e[:, None, None, None] * np.einsum("ab,sbc->sac", M, chi)[None]
    got = oracle.dhop(psi, _unit_links(dims), dims, Ls, BC)[0]
    assert oracle.rel_l2(got, expect) < 1e-13
    # Dhop^+ has the conjugate symbol: 2 sum cos + 2i sum g sin
    Md = 2 * sum(np.cos(pm) for pm in p) * np.eye(4) + 2j * sum(
        np.sin(p[mu]) * g[mu] for mu in range(4))
    expectd = e[:, None, None, None] * np.einsum("ab,sbc->sac", Md, chi)[None]
    gotd = oracle.dhop(psi, _unit_links(dims), dims, Ls, BC, dag=True)[0]
    assert oracle.rel_l2(gotd, expectd) < 1e-13


def test_free_wilson_symbol_closed_form():
    # D_W(p)^+ D_W(p) = [(4 - M5 - sum cos)^2 + sum sin^2] * 1
    for p in ([0.1, 0.7, -1.3, 2.0], [np.pi, 0, 0, np.pi / 4]):
        W = dense.dwilson_p(p, 1.8)
        lam = (4 - 1.8 - sum(np.cos(p))) ** 2 + sum(np.sin(v) ** 2 for v in p)
        assert np.allclose(W.conj().T @ W, lam * np.eye(4), atol=1e-14)


@pytest.mark.parametrize("kind", ["shamir", "mobius"])
@pytest.mark.parametrize("dag", [False, True])
def test_free_dw_momentum_matrix(kind, dag):
    dims = (4, 4, 4, 4)
    Ls, M5, mf = 6, 1.8, 0.05
    b, c = (1.0, 0.0) if kind == "shamir" else (1.5, 0.5)
    p = [2 * np.pi * 1 / 4, 0.0, 2 * np.pi * 3 / 4, 3 * np.pi / 4]
    rng = np.random.default_rng(8)
    chi = rng.standard_normal((Ls * 4, 3)) + 1j * rng.standard_normal((Ls * 4, 3))
    e = _plane_wave(dims, p)
    psi = (e[:, None, None] * chi[None]).reshape(len(e), Ls, 4, 3)
    Dp = dense.dw_p(p, Ls, M5, b, c, mf)
    if dag:
        Dp = Dp.conj().T
    expect = (e[:, None, None] * (Dp @ chi)[None]).reshape(len(e), Ls, 4, 3)
    got = oracle.dw(psi, _unit_links(dims), dims, Ls, M5, b, c, mf, BC, dag=dag)[0]
    assert oracle.rel_l2(got, expect) < 1e-13


# --------------------------------------------------------------------------
# T3: gauge covariance  D[U^g](g psi) = g D[U] psi


def test_gauge_covariance():
    dims = (4, 4, 4, 4)
    Ls, M5, b, c, mf = 4, 1.8, 1.5, 0.5, 0.02
    U = inputs.exp_su3_field(dims, seed=61)
    V4 = 256
    gx = inputs.haar_su3(V4, seed=62, stream=inputs.STREAM_GAUGE_TRANSFORM)
    Ug = np.empty_like(U)
    for x in range(V4):
        c4 = [x % 4, (x // 4) % 4, (x // 16) % 4, x // 64]
        for mu in range(4):
            cf = list(c4)
            cf[mu] = (cf[mu] + 1) % 4
            y = cf[0] + 4 * (cf[1] + 4 * (cf[2] + 4 * cf[3]))
            Ug[x, mu] = gx[x] @ U[x, mu] @ gx[y].conj().T
    psi = _rand_fermion(dims, Ls, 1, seed=63)
    psig = np.einsum("xab,rxsib->rxsia", gx, psi)
    lhs = oracle.dhop(psig, Ug, dims, Ls, BC)
    rhs = np.einsum("xab,rxsib->rxsia", gx, oracle.dhop(psi, U, dims, Ls, BC))
    assert oracle.rel_l2(lhs, rhs) < 1e-14
    lhs = oracle.dw(psig, Ug, dims, Ls, M5, b, c, mf, BC)
    rhs = np.einsum("xab,rxsib->rxsia", gx, oracle.dw(psi, U, dims, Ls, M5, b, c, mf, BC))
    assert oracle.rel_l2(lhs, rhs) < 1e-14


# --------------------------------------------------------------------------
# T4 / T5: gamma5-hermiticity and adjointness


def _g5(f):
    out = f.copy()
    out[..., 2:, :] *= -1
    return out


def test_gamma5_hermiticity_dhop():
    dims = (4, 4, 4, 4)
    U = inputs.exp_su3_field(dims, seed=71)
    psi = _rand_fermion(dims, 3, 1, seed=72)
    lhs = _g5(oracle.dhop(_g5(psi), U, dims, 3, BC))
    rhs = oracle.dhop(psi, U, dims, 3, BC, dag=True)
    assert oracle.rel_l2(lhs, rhs) < 1e-14


def test_r5g5_hermiticity_shamir():
    # D^+ = R5 g5 D g5 R5 for Shamir (b=1, c=0); R5 reflects s -> Ls-1-s
    dims = (4, 4, 4, 4)
    Ls = 6
    U = inputs.exp_su3_field(dims, seed=81)
    psi = _rand_fermion(dims, Ls, 1, seed=82)

    def r5g5(f):
        return _g5(f[:, :, ::-1]).copy()

    lhs = r5g5(oracle.dw(r5g5(psi), U, dims, Ls, 1.8, 1.0, 0.0, 0.03, BC))
    rhs = oracle.dw(psi, U, dims, Ls, 1.8, 1.0, 0.0, 0.03, BC, dag=True)
    assert oracle.rel_l2(lhs, rhs) < 1e-14


@pytest.mark.parametrize("kind", ["shamir", "mobius"])
def test_adjointness(kind):
    dims = (4, 4, 4, 4)
    Ls = 6
    b, c = (1.0, 0.0) if kind == "shamir" else (1.5, 0.5)
    U = inputs.exp_su3_field(dims, seed=91)
    x = _rand_fermion(dims, Ls, 1, seed=92)
    y = _rand_fermion(dims, Ls, 1, seed=93)
    lhs = oracle.inner(x, oracle.dw(y, U, dims, Ls, 1.8, b, c, 0.01, BC))
    rhs = oracle.inner(oracle.dw(x, U, dims, Ls, 1.8, b, c, 0.01, BC, dag=True), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    lhs = oracle.inner(x, oracle.dhop(y, U, dims, Ls, BC))
    rhs = oracle.inner(oracle.dhop(x, U, dims, Ls, BC, dag=True), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_mobius_b1_c0_is_shamir_and_ddagd_hpd():
    dims = (4, 4, 4, 4)
    Ls = 4
    U = inputs.exp_su3_field(dims, seed=101)
    psi = _rand_fermion(dims, Ls, 1, seed=102)
    a = oracle.dw(psi, U, dims, Ls, 1.8, 1.0, 0.0, 0.01, BC)
    # Shamir as the plain expression D_W + 1 - K
    hop = oracle.dhop(psi, U, dims, Ls, BC)
    k = oracle.kop(psi, dims, Ls, 0.01)
    shamir = (4 - 1.8) * psi - 0.5 * hop + psi - k
    assert oracle.rel_l2(a, shamir) < 1e-14
    # D^+ D: Rayleigh quotient real positive and equal to |D psi|^2
    ddd = oracle.dwdagdw(psi, U, dims, Ls, 1.8, 1.5, 0.5, 0.01, BC)
    dpsi = oracle.dw(psi, U, dims, Ls, 1.8, 1.5, 0.5, 0.01, BC)
    q = oracle.inner(psi, ddd)
    assert abs(q.imag) < 1e-12 * abs(q.real)
    assert q.real > 0
    assert abs(q.real - np.vdot(dpsi.ravel(), dpsi.ravel()).real) < 1e-12 * q.real


def test_sampled_sites_equal_full():
    dims = (4, 4, 4, 4)
    Ls = 4
    U = inputs.exp_su3_field(dims, seed=111)
    psi = _rand_fermion(dims, Ls, 2, seed=112)
    sites = np.array([0, 5, 63, 64, 255, 130])
    for dag in (False, True):
        full = oracle.dw(psi, U, dims, Ls, 1.8, 1.5, 0.5, [0.01, 0.05], BC, dag=dag)
        part = oracle.dw(psi, U, dims, Ls, 1.8, 1.5, 0.5, [0.01, 0.05], BC, dag=dag,
                         sites=sites)
        assert np.array_equal(full[:, sites], part)
        fh = oracle.dhop(psi, U, dims, Ls, BC, dag=dag)
        ph = oracle.dhop(psi, U, dims, Ls, BC, dag=dag, sites=sites)
        assert np.array_equal(fh[:, sites], ph)


# --------------------------------------------------------------------------
# T9: CG


def test_cg_matches_dense_solve():
    dims = (2, 2, 2, 2)
    Ls, M5, b, c = 4, 1.8, 1.5, 0.5
    mfs = [0.01, 0.1]
    U = inputs.exp_su3_field(dims, seed=121)
    rhs = _rand_fermion(dims, Ls, 2, seed=122)
    x, iters, res = oracle.cg(rhs, U, dims, Ls, M5, b, c, mfs, BC, tol=1e-12, maxit=5000)
    for r, mf in enumerate(mfs):
        D = dense.dw5(U, dims, Ls, M5, b, c, mf, BC)
        xs = np.linalg.solve(D.conj().T @ D, rhs[r].ravel())
        assert res[r] <= 1e-12
        assert oracle.rel_l2(x[r].ravel(), xs) < 1e-9
        assert iters[r] > 0


def test_cg_reports_not_converged():
    dims = (2, 2, 2, 2)
    U = inputs.exp_su3_field(dims, seed=131)
    rhs = _rand_fermion(dims, 4, 1, seed=132)
    x, iters, res = oracle.cg(rhs, U, dims, 4, 1.8, 1.5, 0.5, 0.01, BC, tol=1e-12, maxit=3)
    assert iters[0] == 3 and res[0] > 1e-12


# --------------------------------------------------------------------------
# Flop convention of the Domain Wall kernel (Table 3)


def _table3():
    vals = {}
    with open(os.path.join(GOLDEN, "table3_flops.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = int(v)
    return vals


def test_flop_count_reproduces_table3():
    cmul, cadd = 6, 2
    project = 6 * cadd                      # 2 spins x 3 colours, one complex add each
    su3_half = 2 * (9 * cmul + 6 * cadd)    # 3x3 complex matrix times two colour vectors
    accumulate = 12 * cadd                  # full spinor add, 7 of the 8 directions
    rrii = 8 * (project + su3_half) + 7 * accumulate
    # RIRI: each of the 6 rows of the SU(3) product starts with 0 + z2*z3 (2 flop more)
    riri = rrii + 8 * 6 * 2
    t3 = _table3()
    assert rrii == t3["RRII"] == 1320
    assert riri == t3["RIRI"] == 1416
