"""What the mathematics fixes, checked on the CUDA path itself (not only through
parity with the oracle): the free-field plane-wave symbols of Dhop and D (T1,
T2), gauge covariance (T3), gamma5-hermiticity of Dhop and R5 gamma5-hermiticity
of Shamir D (T4), adjointness of D / D^+ and hermiticity of D^+D (T5), Mobius
with b = 1, c = 0 being Shamir (T7), and Dhop acting on every slice alike, each
slice being the Ls = 1 Wilson hop (T8).  Each side runs through the C ABI; the
expected values come from closed forms (numpy) or from another call of the GPU
path.  Tolerances: 1e-12 at FP64, 1e-5 at FP32, 5e-3 at FP16 storage.
"""

import numpy as np
import pytest

import oracle
from gpu_helpers import BC, TOL, build_library, run_gpu
from oracle import dense
from paper_2112_01852_gb300 import dw, inputs

pytestmark = pytest.mark.gpu

PRECS = [dw.DW_F64, dw.DW_F32, dw.DW_F16]
PREC_IDS = ["f64", "f32", "f16"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()
    import torch
    assert torch.cuda.is_available()


def _lattice(dims, Ls, prec, kind=dw.DW_MOBIUS, M5=1.8, b=1.5, c=0.5, U=None):
    from paper_2112_01852_gb300.lattice import Lattice
    lat = Lattice(dims, Ls, kind=kind, M5=M5, b=b, c=c, prec=prec, bc=BC)
    if U is not None:
        lat.load_gauge(U)
    return lat


def _plane_wave(dims, p):
    x4 = np.arange(int(np.prod(dims)))
    c, r = [], x4.copy()
    for L in dims:
        c.append(r % L)
        r //= L
    return np.exp(1j * sum(p[mu] * c[mu] for mu in range(4)))


def _unit_links(dims):
    return np.broadcast_to(np.eye(3, dtype=complex), (int(np.prod(dims)), 4, 3, 3)).copy()


def _g5(f):
    out = f.copy()
    out[..., 2:, :] *= -1
    return out


def _fermion(dims, Ls, seed, nrhs=1):
    return inputs.gaussian_fermion(dims, Ls, nrhs, seed=seed)


# T1: free Dhop and Dhop^+ on a plane wave (antiperiodic t momenta)
@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 2, 0, 3), (3, 1, 1, 1)])
def test_free_dhop_plane_wave(prec, n):
    dims, Ls = (4, 4, 4, 6), 3
    p = [2 * np.pi * n[k] / dims[k] for k in range(3)] + [(2 * n[3] + 1) * np.pi / dims[3]]
    rng = np.random.default_rng(11)
    chi = rng.standard_normal((Ls, 4, 3)) + 1j * rng.standard_normal((Ls, 4, 3))
    e = _plane_wave(dims, p)
    psi = (e[:, None, None, None] * chi[None])[None]
    g, _ = dense.gammas()
    cos = 2 * sum(np.cos(v) for v in p) * np.eye(4)
    sin = 2j * sum(np.sin(p[mu]) * g[mu] for mu in range(4))
    lat = _lattice(dims, Ls, prec, U=_unit_links(dims))
    for op, M in ((dw.DW_OP_DHOP, cos - sin), (dw.DW_OP_DHOP_DAG, cos + sin)):
        expect = e[:, None, None, None] * np.einsum("ab,sbc->sac", M, chi)[None]
        got = run_gpu(lat, op, psi)[0]
        assert oracle.rel_l2(got, expect) <= TOL[prec], (op, n)
    lat.close()


# T2: free D and D^+ (Shamir and Mobius) against the 4Ls x 4Ls momentum matrix
@pytest.mark.parametrize("prec", [dw.DW_F64, dw.DW_F32], ids=["f64", "f32"])
@pytest.mark.parametrize("kind", [dw.DW_SHAMIR, dw.DW_MOBIUS], ids=["shamir", "mobius"])
def test_free_dw_momentum_matrix(prec, kind):
    dims, Ls, M5, mf = (4, 4, 4, 4), 6, 1.8, 0.05
    b, c = (1.0, 0.0) if kind == dw.DW_SHAMIR else (1.5, 0.5)
    p = [2 * np.pi / 4, 0.0, 2 * np.pi * 3 / 4, 3 * np.pi / 4]
    rng = np.random.default_rng(12)
    chi = rng.standard_normal((Ls * 4, 3)) + 1j * rng.standard_normal((Ls * 4, 3))
    e = _plane_wave(dims, p)
    psi = (e[:, None, None] * chi[None]).reshape(1, len(e), Ls, 4, 3)
    Dp = dense.dw_p(p, Ls, M5, b, c, mf)
    lat = _lattice(dims, Ls, prec, kind=kind, M5=M5, b=b, c=c, U=_unit_links(dims))
    for op, M in ((dw.DW_OP_D, Dp), (dw.DW_OP_DDAG, Dp.conj().T)):
        expect = (e[:, None, None] * (M @ chi)[None]).reshape(len(e), Ls, 4, 3)
        got = run_gpu(lat, op, psi, mf=[mf])[0]
        assert oracle.rel_l2(got, expect) <= TOL[prec], op
    lat.close()


# T3: D[U^g](g psi) = g D[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x + mu)^+
@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_gauge_covariance(prec):
    dims, Ls, mf = (4, 4, 4, 4), 4, 0.02
    V4 = int(np.prod(dims))
    U = inputs.exp_su3_field(dims, seed=61)
    gx = inputs.haar_su3(V4, seed=62, stream=inputs.STREAM_GAUGE_TRANSFORM)
    Ug = np.empty_like(U)
    for x in range(V4):
        c4 = [x % 4, (x // 4) % 4, (x // 16) % 4, x // 64]
        for mu in range(4):
            cf = list(c4)
            cf[mu] = (cf[mu] + 1) % 4
            y = cf[0] + 4 * (cf[1] + 4 * (cf[2] + 4 * cf[3]))
            Ug[x, mu] = gx[x] @ U[x, mu] @ gx[y].conj().T
    psi = _fermion(dims, Ls, seed=63)
    psig = np.einsum("xab,rxsib->rxsia", gx, psi)
    lat = _lattice(dims, Ls, prec, U=U)
    latg = _lattice(dims, Ls, prec, U=Ug)
    for op in (dw.DW_OP_DHOP, dw.DW_OP_D, dw.DW_OP_DDAG):
        lhs = run_gpu(latg, op, psig, mf=[mf])
        rhs = np.einsum("xab,rxsib->rxsia", gx, run_gpu(lat, op, psi, mf=[mf]))
        assert oracle.rel_l2(lhs, rhs) <= TOL[prec], op
    lat.close()
    latg.close()


# T4: g5 Dhop g5 = Dhop^+; Shamir D^+ = R5 g5 D g5 R5 (R5: s -> Ls-1-s)
@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_gamma5_hermiticity(prec):
    dims, Ls = (4, 4, 4, 4), 6
    U = inputs.exp_su3_field(dims, seed=71)
    psi = _fermion(dims, Ls, seed=72)
    lat = _lattice(dims, Ls, prec, U=U)
    lhs = _g5(run_gpu(lat, dw.DW_OP_DHOP, _g5(psi)))
    rhs = run_gpu(lat, dw.DW_OP_DHOP_DAG, psi)
    assert oracle.rel_l2(lhs, rhs) <= TOL[prec]
    lat.close()

    def r5g5(f):
        return _g5(f[:, :, ::-1]).copy()

    sh = _lattice(dims, Ls, prec, kind=dw.DW_SHAMIR, b=1.0, c=0.0, U=U)
    lhs = r5g5(run_gpu(sh, dw.DW_OP_D, r5g5(psi), mf=[0.03]))
    rhs = run_gpu(sh, dw.DW_OP_DDAG, psi, mf=[0.03])
    assert oracle.rel_l2(lhs, rhs) <= TOL[prec]
    sh.close()


# T5: <x, D y> = <D^+ x, y>, <x, Dhop y> = <Dhop^+ x, y>, D^+D hermitian positive
@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("kind", [dw.DW_SHAMIR, dw.DW_MOBIUS], ids=["shamir", "mobius"])
def test_adjointness(prec, kind):
    dims, Ls, mf = (4, 4, 4, 4), 6, 0.01
    b, c = (1.0, 0.0) if kind == dw.DW_SHAMIR else (1.5, 0.5)
    U = inputs.exp_su3_field(dims, seed=91)
    x = _fermion(dims, Ls, seed=92)
    y = _fermion(dims, Ls, seed=93)
    lat = _lattice(dims, Ls, prec, kind=kind, b=b, c=c, U=U)
    for op, dag in ((dw.DW_OP_D, dw.DW_OP_DDAG), (dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG)):
        lhs = oracle.inner(x, run_gpu(lat, op, y, mf=[mf]))
        rhs = oracle.inner(run_gpu(lat, dag, x, mf=[mf]), y)
        assert abs(lhs - rhs) <= TOL[prec] * abs(lhs), op
    a = oracle.inner(x, run_gpu(lat, dw.DW_OP_DDAGD, y, mf=[mf]))
    bb = oracle.inner(run_gpu(lat, dw.DW_OP_DDAGD, x, mf=[mf]), y)
    assert abs(a - bb) <= TOL[prec] * abs(a)
    q = oracle.inner(x, run_gpu(lat, dw.DW_OP_DDAGD, x, mf=[mf]))
    dx = run_gpu(lat, dw.DW_OP_D, x, mf=[mf])
    assert q.real > 0 and abs(q.imag) <= TOL[prec] * q.real
    assert abs(q.real - np.vdot(dx.ravel(), dx.ravel()).real) <= TOL[prec] * q.real
    lat.close()


# T7: the Mobius lattice with b = 1, c = 0 is the Shamir operator
@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_mobius_b1_c0_is_shamir(prec):
    dims, Ls = (4, 4, 4, 4), 4
    U = inputs.exp_su3_field(dims, seed=101)
    psi = _fermion(dims, Ls, seed=102)
    mo = _lattice(dims, Ls, prec, kind=dw.DW_MOBIUS, b=1.0, c=0.0, U=U)
    sh = _lattice(dims, Ls, prec, kind=dw.DW_SHAMIR, U=U)
    for op in (dw.DW_OP_D, dw.DW_OP_DDAG, dw.DW_OP_DDAGD):
        assert np.array_equal(run_gpu(mo, op, psi, mf=[0.01]), run_gpu(sh, op, psi, mf=[0.01]))
    mo.close()
    sh.close()


# T8: Dhop acts on every slice alike: each slice of an Ls = 5 apply is the
# Ls = 1 (Wilson) hop of that slice
@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_slices_are_wilson_hops(prec):
    dims, Ls = (4, 6, 2, 4), 5
    U = inputs.haar_su3_field(dims, seed=111)
    psi = _fermion(dims, Ls, seed=112)
    lat5 = _lattice(dims, Ls, prec, U=U)
    lat1 = _lattice(dims, 1, prec, U=U)
    for op in (dw.DW_OP_DHOP, dw.DW_OP_DHOP_DAG):
        full = run_gpu(lat5, op, psi)
        for s in range(Ls):
            one = run_gpu(lat1, op, np.ascontiguousarray(psi[:, :, s:s + 1]))
            assert oracle.rel_l2(full[:, :, s:s + 1], one) <= TOL[prec], (op, s)
    lat5.close()
    lat1.close()
