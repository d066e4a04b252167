"""Even-odd (red-black) decomposition of the domain-wall operator -- TEST
INFRASTRUCTURE ONLY (imported by tests/, __graft_entry__.smoke() and bench.py's
CPU legs, never by the product library).

The paper gives no solver and no preconditioner; this is the standard Schur
complement of the 4D even-odd split, written from the operator definition with
the oracle's own Dhop and K (``oracle.dhop``, ``oracle.kop``) and numpy.

Sites are even or odd by (x + y + z + t) mod 2; every extent must be even
(a periodic hop across an odd extent joins sites of equal parity).  The operator
    D = D_W (b + cK) + (1 - K),   D_W = (4 - M5) - Dhop / 2
splits into a part that is local in 4D,
    A = (4 - M5)(b + cK) + (1 - K) = alpha + beta K,
    alpha = b (4 - M5) + 1,  beta = c (4 - M5) - 1,
and the hopping part H = -Dhop (b + cK) / 2, which only couples sites of
opposite parity.  With P_e, P_o the projections on even and odd sites,
    D = [[A, H_eo], [H_oe, A]],  H_eo = P_e H P_o,  H_oe = P_o H P_e,
and the Schur complement on odd sites is
    Dhat = A - H_oe A^-1 H_eo.
D x = eta is solved by Dhat x_o = eta_o - H_oe A^-1 eta_e, then
x_e = A^-1 (eta_e - H_eo x_o).  The adjoints use D^+ = A^+ + H^+ with
A^+ = alpha + beta K^+ and H^+ = -(b + cK^+) Dhop^+ / 2.

All fields here are full-lattice canonical arrays [nrhs][V4][Ls][4][3]; a field
"on odd sites" is zero on the even ones.
"""

from __future__ import annotations

import numpy as np

from . import dhop, kop


def parity(dims) -> np.ndarray:
    """(x + y + z + t) mod 2 per 4D site, x4 = x + Lx (y + Ly (z + Lz t))."""
    Lx, Ly, Lz, Lt = dims
    x4 = np.arange(Lx * Ly * Lz * Lt)
    x = x4 % Lx
    y = (x4 // Lx) % Ly
    z = (x4 // (Lx * Ly)) % Lz
    t = x4 // (Lx * Ly * Lz)
    return (x + y + z + t) & 1


def project(psi, dims, p):
    """Zero the sites whose parity is not p."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    out[:, parity(dims) != p] = 0
    return out


def coeffs(M5, b, c):
    """alpha, beta of the local part A = alpha + beta K."""
    return b * (4.0 - M5) + 1.0, c * (4.0 - M5) - 1.0


def m5(psi, dims, Ls, M5, b, c, mf, dag=False):
    """A psi (A^+ psi): alpha psi + beta K psi, site by site."""
    al, be = coeffs(M5, b, c)
    return al * psi + be * kop(psi, dims, Ls, mf, dag=dag)


def m5_matrix(Ls, M5, b, c, mf, dag=False):
    """The 12 Ls x 12 Ls matrix of A (A^+) on one 4D site, index (s, spin, colour)."""
    n = 12 * Ls
    basis = np.eye(n, dtype=np.complex128).reshape(n, 1, Ls, 4, 3)
    cols = m5(basis, (1, 1, 1, 1), Ls, M5, b, c, [mf] * n, dag=dag)
    return cols.reshape(n, n).T


def m5_inv(psi, dims, Ls, M5, b, c, mf, dag=False):
    """A^-1 psi (A^-+ psi) with the inverse of the one-site matrix (numpy)."""
    psi = np.asarray(psi, dtype=np.complex128)
    nrhs, V4 = psi.shape[0], psi.shape[1]
    mfs = np.broadcast_to(np.asarray(mf, np.float64), (nrhs,))
    out = np.empty_like(psi)
    for r in range(nrhs):
        inv = np.linalg.inv(m5_matrix(Ls, M5, b, c, mfs[r], dag=dag))
        out[r] = (psi[r].reshape(V4, 12 * Ls) @ inv.T).reshape(V4, Ls, 4, 3)
    return out


def hop(psi, U, dims, Ls, b, c, mf, bc=None, dag=False):
    """H psi = -Dhop (b + cK) psi / 2, or H^+ psi = -(b + cK^+) Dhop^+ psi / 2."""
    if not dag:
        phi = b * psi + c * kop(psi, dims, Ls, mf)
        return -0.5 * dhop(phi, U, dims, Ls, bc)
    h = dhop(psi, U, dims, Ls, bc, dag=True)
    return -0.5 * (b * h + c * kop(h, dims, Ls, mf, dag=True))


def schur(x_o, U, dims, Ls, M5, b, c, mf, bc=None):
    """Dhat x_o = A x_o - H_oe A^-1 H_eo x_o on odd sites."""
    x_o = project(x_o, dims, 1)
    t = project(hop(x_o, U, dims, Ls, b, c, mf, bc), dims, 0)
    t = m5_inv(t, dims, Ls, M5, b, c, mf)
    u = project(hop(t, U, dims, Ls, b, c, mf, bc), dims, 1)
    return m5(x_o, dims, Ls, M5, b, c, mf) - u


def schur_dag(y_o, U, dims, Ls, M5, b, c, mf, bc=None):
    """Dhat^+ y_o = A^+ y_o - H_eo^+ A^-+ H_oe^+ y_o on odd sites."""
    y_o = project(y_o, dims, 1)
    t = project(hop(y_o, U, dims, Ls, b, c, mf, bc, dag=True), dims, 0)
    t = m5_inv(t, dims, Ls, M5, b, c, mf, dag=True)
    u = project(hop(t, U, dims, Ls, b, c, mf, bc, dag=True), dims, 1)
    return m5(y_o, dims, Ls, M5, b, c, mf, dag=True) - u


def schur_rhs(eta, U, dims, Ls, M5, b, c, mf, bc=None):
    """eta_o - H_oe A^-1 eta_e: the right-hand side of the odd-site system."""
    t = m5_inv(project(eta, dims, 0), dims, Ls, M5, b, c, mf)
    return project(eta, dims, 1) - project(hop(t, U, dims, Ls, b, c, mf, bc), dims, 1)


def reconstruct(x_o, eta, U, dims, Ls, M5, b, c, mf, bc=None):
    """The full solution: x_e = A^-1 (eta_e - H_eo x_o), with x_o on odd sites."""
    x_o = project(x_o, dims, 1)
    r = project(eta, dims, 0) - project(hop(x_o, U, dims, Ls, b, c, mf, bc), dims, 0)
    return x_o + m5_inv(r, dims, Ls, M5, b, c, mf)


def solve(eta, U, dims, Ls, M5, b, c, mf, bc=None, tol=1e-12, maxit=20000):
    """D x = eta by CG on Dhat^+ Dhat x_o = Dhat^+ etahat_o (plain numpy CG,
    FP64; small lattices), then the even sites by reconstruct."""
    rhs = schur_dag(schur_rhs(eta, U, dims, Ls, M5, b, c, mf, bc), U, dims, Ls, M5, b, c, mf, bc)
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    rr = np.vdot(r.ravel(), r.ravel()).real
    bb = rr
    for _ in range(maxit):
        if rr <= tol * tol * bb:
            break
        Ap = schur_dag(schur(p, U, dims, Ls, M5, b, c, mf, bc), U, dims, Ls, M5, b, c, mf, bc)
        a = rr / np.vdot(p.ravel(), Ap.ravel()).real
        x += a * p
        r -= a * Ap
        rr_new = np.vdot(r.ravel(), r.ravel()).real
        p = r + (rr_new / rr) * p
        rr = rr_new
    return reconstruct(x, eta, U, dims, Ls, M5, b, c, mf, bc)
