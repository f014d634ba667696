"""Operators A for the oracle (test infrastructure only).

CSROperator: y = A x for a complex CSR matrix (scipy.sparse as the library
primitive).  Used for the bidiagonal test matrix of Example 1 (Sec. 3) and the
convection-diffusion batch.

WilsonOperator: the Wilson-Dirac-style matrix of Example 7 (Sec. 4) written
as A = a I - H with the hopping term

    (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                        + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu) ]

on a periodic 4-d lattice.  Gamma matrices in the chiral basis:
gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] for k = 1, 2, 3 (mu = 0, 1, 2 =
x, y, z) and gamma_4 = [[0, I], [I, 0]] (mu = 3 = t).  The oracle applies the
full 4x4 gamma matrices with numpy.roll shifts: no spin projection trick, no
blocking.  The system (1/kappa) I - H is A - sigma I with a = 0 and
sigma = -1/kappa.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_PAULI = np.array([
    [[0, 1], [1, 0]],
    [[0, -1j], [1j, 0]],
    [[1, 0], [0, -1]],
], dtype=np.complex128)


def gamma_matrices() -> np.ndarray:
    """gamma_mu, mu = 0..3 (x, y, z, t), chiral basis, 4x4 Hermitian."""
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    z = np.zeros((2, 2), dtype=np.complex128)
    for k in range(3):
        g[k] = np.block([[z, -1j * _PAULI[k]], [1j * _PAULI[k], z]])
    g[3] = np.block([[z, np.eye(2)], [np.eye(2), z]])
    return g


def gamma5() -> np.ndarray:
    """gamma_5 = gamma_x gamma_y gamma_z gamma_t."""
    g = gamma_matrices()
    return g[0] @ g[1] @ g[2] @ g[3]


class CSROperator:
    """A given as CSR (int32 rowptr/col, complex128 vals)."""

    def __init__(self, rowptr, col, vals):
        self.n = len(rowptr) - 1
        self.A = sp.csr_matrix((np.asarray(vals, np.complex128), np.asarray(col), np.asarray(rowptr)),
                               shape=(self.n, self.n))

    def matvec(self, x):
        return self.A @ x

    def dense(self):
        return self.A.toarray()


class WilsonOperator:
    """A = a I - H on a periodic lattice ``dims`` = (Lx, Ly, Lz, Lt).

    ``links`` is complex128 [4, V, 3, 3] with V = Lx*Ly*Lz*Lt and site index
    ((t*Lz + z)*Ly + y)*Lx + x; vectors are length 12*V with component index
    site*12 + spin*3 + color."""

    def __init__(self, dims, links, diag_a=0.0):
        self.dims = tuple(int(d) for d in dims)
        Lx, Ly, Lz, Lt = self.dims
        self.V = Lx * Ly * Lz * Lt
        self.n = 12 * self.V
        self.a = complex(diag_a)
        # field arrays are indexed [t, z, y, x, ...]
        self.U = np.asarray(links, np.complex128).reshape(4, Lt, Lz, Ly, Lx, 3, 3)
        self.g = gamma_matrices()
        self.one = np.eye(4, dtype=np.complex128)

    # numpy axis of each direction mu in a [t, z, y, x, spin, color] field
    _AXIS = (3, 2, 1, 0)

    def _field(self, v):
        Lx, Ly, Lz, Lt = self.dims
        return v.reshape(Lt, Lz, Ly, Lx, 4, 3)

    def hop(self, v):
        """H v."""
        psi = self._field(np.asarray(v, np.complex128))
        out = np.zeros_like(psi)
        for mu in range(4):
            ax = self._AXIS[mu]
            U = self.U[mu]
            # forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
            fwd = np.roll(psi, -1, axis=ax)                    # fwd[x] = psi[x + mu]
            fwd = np.einsum("...ab,...sb->...sa", U, fwd)      # color
            out += np.einsum("st,...tc->...sc", self.one - self.g[mu], fwd)
            # backward: (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu)
            Ub = np.roll(U, 1, axis=ax)                        # Ub[x] = U_mu[x - mu]
            bwd = np.roll(psi, 1, axis=ax)                     # bwd[x] = psi[x - mu]
            bwd = np.einsum("...ba,...sb->...sa", Ub.conj(), bwd)
            out += np.einsum("st,...tc->...sc", self.one + self.g[mu], bwd)
        return out.reshape(-1)

    def matvec(self, v):
        """A v = a v - H v."""
        return self.a * np.asarray(v, np.complex128) - self.hop(v)

    def gamma5_apply(self, v):
        psi = self._field(np.asarray(v, np.complex128))
        return np.einsum("st,...tc->...sc", gamma5(), psi).reshape(-1)

    def dense(self):
        """Dense A (tiny lattices only)."""
        n = self.n
        M = np.zeros((n, n), dtype=np.complex128)
        e = np.zeros(n, dtype=np.complex128)
        for j in range(n):
            e[j] = 1.0
            M[:, j] = self.matvec(e)
            e[j] = 0.0
        return M
