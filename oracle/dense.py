"""Dense-matrix build of the domain-wall operator -- TEST INFRASTRUCTURE ONLY.

A second, independent statement of the operator for tiny lattices (2^4 x Ls=4
gives 768 x 768 matrices). It shares nothing with ``dw_oracle.cpp``: the gamma
matrices are assembled from the Pauli matrices with ``np.block``, every hop is
placed as a Kronecker product (spin (x) colour) at its (x, y) block, and the
adjoint is taken numerically as the conjugate transpose.

Vector index of a 5D spinor component: ((x4 * Ls + s) * 4 + spin) * 3 + colour,
identical to the canonical fermion layout, x4 = x + Lx*(y + Ly*(z + Lz*t)).

The operator is the standard domain-wall one (the paper names its hopping part
the "Domain Wall kernel", Sec. 4.1, without writing it down):
  Dhop = sum_mu [(1 - g_mu) U_mu(x) delta_{y,x+mu} + (1 + g_mu) U_mu(x-mu)^+ delta_{y,x-mu}],
  D_W = (4 - M5) - Dhop/2,  D = D_W (b + cK) + (1 - K).
"""

from __future__ import annotations

import numpy as np

_S1 = np.array([[0, 1], [1, 0]], dtype=complex)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
_S3 = np.array([[1, 0], [0, -1]], dtype=complex)
_I2 = np.eye(2, dtype=complex)
_Z2 = np.zeros((2, 2), dtype=complex)


def gammas():
    """Chiral-basis Euclidean gammas (g_x, g_y, g_z, g_t) and g5 = diag(1,1,-1,-1)."""
    g = [np.block([[_Z2, 1j * s], [-1j * s, _Z2]]) for s in (_S1, _S2, _S3)]
    g.append(np.block([[_Z2, _I2], [_I2, _Z2]]))
    g5 = -(g[0] @ g[1] @ g[2] @ g[3])
    return g, g5


def _coords(x4, dims):
    c = []
    for L in dims:
        c.append(x4 % L)
        x4 //= L
    return c


def _index(c, dims):
    Lx, Ly, Lz, _ = dims
    return c[0] + Lx * (c[1] + Ly * (c[2] + Lz * c[3]))


def hop4(U, dims, bc=(1, 1, 1, -1), dag=False):
    """4D hopping matrix on (x4, spin, colour): shape (12 V4, 12 V4)."""
    g, _ = gammas()
    V4 = int(np.prod(dims))
    H = np.zeros((V4 * 12, V4 * 12), dtype=complex)
    sgn = -1.0 if dag else 1.0
    one = np.eye(4, dtype=complex)
    for x in range(V4):
        c = _coords(x, dims)
        for mu in range(4):
            cf = list(c)
            cf[mu] += 1
            ph_f = 1.0
            if cf[mu] == dims[mu]:
                cf[mu] = 0
                ph_f = bc[mu]
            cb = list(c)
            cb[mu] -= 1
            ph_b = 1.0
            if cb[mu] < 0:
                cb[mu] = dims[mu] - 1
                ph_b = bc[mu]
            yf = _index(cf, dims)
            yb = _index(cb, dims)
            H[x * 12:(x + 1) * 12, yf * 12:(yf + 1) * 12] += ph_f * np.kron(
                one - sgn * g[mu], U[x, mu])
            H[x * 12:(x + 1) * 12, yb * 12:(yb + 1) * 12] += ph_b * np.kron(
                one + sgn * g[mu], U[yb, mu].conj().T)
    return H


def fifth_dim_hop(Ls, mf):
    """K on (s, spin): shape (4 Ls, 4 Ls)."""
    _, g5 = gammas()
    Pp = 0.5 * (np.eye(4) + g5)
    Pm = 0.5 * (np.eye(4) - g5)
    K = np.zeros((4 * Ls, 4 * Ls), dtype=complex)
    for s in range(Ls):
        # P- from s+1 (wall: -mf P- psi_0), P+ from s-1 (wall: -mf P+ psi_{Ls-1})
        n = s + 1
        fn = 1.0
        if n == Ls:
            n, fn = 0, -mf
        p = s - 1
        fp = 1.0
        if p < 0:
            p, fp = Ls - 1, -mf
        K[s * 4:(s + 1) * 4, n * 4:(n + 1) * 4] += fn * Pm
        K[s * 4:(s + 1) * 4, p * 4:(p + 1) * 4] += fp * Pp
    return K


def dhop5(U, dims, Ls, bc=(1, 1, 1, -1), dag=False):
    """5D hopping matrix (identity in s): shape (12 V4 Ls, 12 V4 Ls)."""
    H = hop4(U, dims, bc, dag)
    V4 = int(np.prod(dims))
    H = H.reshape(V4, 12, V4, 12)
    out = np.einsum("xayb,st->xsaytb", H, np.eye(Ls))
    return out.reshape(V4 * Ls * 12, V4 * Ls * 12)


def k5(V4, Ls, mf):
    """K on the full 5D space (identity in x4 and colour)."""
    K = fifth_dim_hop(Ls, mf)
    return np.kron(np.eye(V4), np.kron(K, np.eye(3)))


def dw5(U, dims, Ls, M5, b, c, mf, bc=(1, 1, 1, -1)):
    """Dense D = D_W (b + cK) + (1 - K)."""
    V4 = int(np.prod(dims))
    n = V4 * Ls * 12
    one = np.eye(n)
    DW = (4.0 - M5) * one - 0.5 * dhop5(U, dims, Ls, bc)
    K = k5(V4, Ls, mf)
    return DW @ (b * one + c * K) + (one - K)


def dwilson_p(p, M5):
    """Free Wilson operator in momentum space: (4 - M5 - sum cos p) + i sum g_mu sin p."""
    g, _ = gammas()
    m = (4.0 - M5 - sum(np.cos(pm) for pm in p)) * np.eye(4, dtype=complex)
    for mu in range(4):
        m = m + 1j * np.sin(p[mu]) * g[mu]
    return m


def dw_p(p, Ls, M5, b, c, mf):
    """Free domain-wall operator at momentum p on (s, spin): (4 Ls, 4 Ls)."""
    Wp = np.kron(np.eye(Ls), dwilson_p(p, M5))
    K = fifth_dim_hop(Ls, mf)
    one = np.eye(4 * Ls)
    return Wp @ (b * one + c * K) + (one - K)
