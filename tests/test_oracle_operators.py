"""Pins for the oracle's operators (Example 7's Wilson-Dirac matrix, Sec. 4;
the CSR matrices of Example 1, Sec. 3) and for the input generators."""
import numpy as np
import pytest

import workloads as W
from oracle import CSROperator, WilsonOperator, gamma_matrices, gamma5


def test_gamma_algebra():
    g = gamma_matrices()
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2 * np.eye(4) * (a == b))
    # chiral basis: gamma_5 is diagonal +-1 and anticommutes with every gamma_mu
    g5 = gamma5()
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))
    for a in range(4):
        assert np.allclose(g5 @ g[a] + g[a] @ g5, 0)


def test_su3_links_unitary_det1():
    U = W.su3_links((3, 2, 2, 2), 0.5, W.rng(7, 0))
    eye = np.einsum("mvij,mvkj->mvik", U, U.conj())
    assert np.abs(eye - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13
    # eps = 0 gives the free field
    assert np.allclose(W.su3_links((2, 2, 2, 2), 0.0, W.rng(7, 0)), np.eye(3))


def _free_spectrum(dims):
    """Closed form: lambda(H) = sum_mu 2 cos p_mu +- 2i sqrt(sum_mu sin^2 p_mu),
    p_mu = 2 pi n_mu / L_mu, each with multiplicity 6 (2 spins x 3 colours)."""
    out = []
    for idx in np.ndindex(*dims):
        p = 2 * np.pi * np.array(idx) / np.array(dims)
        re = 2 * np.cos(p).sum()
        im = 2 * np.sqrt((np.sin(p) ** 2).sum())
        out += [re + 1j * im] * 6 + [re - 1j * im] * 6
    return np.array(out)


def _match_multiset(a, b, tol):
    a = list(a)
    for z in b:
        i = int(np.argmin(np.abs(np.array(a) - z)))
        assert abs(a[i] - z) < tol, (z, a[i])
        a.pop(i)


def test_wilson_free_field_spectrum():
    dims = (4, 3, 3, 2)
    op = WilsonOperator(dims, W.su3_links(dims, 0.0, W.rng(9, 0)))
    ev = np.linalg.eigvals(-op.dense())          # A = -H with a = 0
    _match_multiset(ev, _free_spectrum(dims), 1e-9)


def test_wilson_gamma5_hermiticity_and_adjoint():
    dims = (3, 2, 4, 2)
    op = WilsonOperator(dims, W.su3_links(dims, 0.4, W.rng(9, 0)))
    H = -op.dense()
    G5 = np.kron(np.eye(op.V), np.kron(gamma5(), np.eye(3)))
    assert np.abs(G5 @ H @ G5 - H.conj().T).max() < 1e-12


def test_wilson_gauge_covariance():
    """U'_mu(x) = g(x) U_mu(x) g(x+mu)^H  =>  H' (G psi) = G (H psi), so the
    spectrum is gauge invariant; a misplaced or untransposed backward link
    breaks this."""
    dims = (3, 2, 2, 4)
    Lx, Ly, Lz, Lt = dims
    U = W.su3_links(dims, 0.5, W.rng(3, 0))
    g = W.su3_links(dims, 1.0, W.rng(4, 0))[0]            # one SU(3) matrix per site
    Uf = U.reshape(4, Lt, Lz, Ly, Lx, 3, 3)
    gf = g.reshape(Lt, Lz, Ly, Lx, 3, 3)
    axis = (3, 2, 1, 0)
    Up = np.empty_like(Uf)
    for mu in range(4):
        gnext = np.roll(gf, -1, axis=axis[mu])
        Up[mu] = gf @ Uf[mu] @ gnext.conj().swapaxes(-1, -2)
    op = WilsonOperator(dims, U)
    opp = WilsonOperator(dims, Up.reshape(4, -1, 3, 3))
    psi = np.random.default_rng(0).standard_normal(op.n) + 1j * np.random.default_rng(1).standard_normal(op.n)

    def gauge(v):
        f = v.reshape(Lt, Lz, Ly, Lx, 4, 3)
        return np.einsum("...ab,...sb->...sa", gf, f).reshape(-1)

    assert np.abs(opp.hop(gauge(psi)) - gauge(op.hop(psi))).max() < 1e-12


def test_wilson_diag_term():
    dims = (2, 2, 2, 2)
    op = WilsonOperator(dims, W.su3_links(dims, 0.3, W.rng(1, 0)), diag_a=0.7 - 0.2j)
    op0 = WilsonOperator(dims, W.su3_links(dims, 0.3, W.rng(1, 0)))
    v = np.arange(op.n) * (1 + 0.5j)
    assert np.allclose(op.matvec(v), (0.7 - 0.2j) * v + op0.matvec(v))


def test_csr_bidiag_and_convdiff():
    rowptr, col, vals = W.bidiag_csr(np.arange(1, 6, dtype=float), 1.0)
    A = CSROperator(rowptr, col, vals).dense()
    assert np.allclose(A, np.diag(np.arange(1, 6)) + np.diag(np.ones(4), 1))
    # convection-diffusion: row sums vanish in the interior (consistency of the stencil
    # for constants), Dirichlet boundary rows keep the missing neighbours out
    s = 6
    rowptr, col, vals = W.convdiff_csr(s, 3.0, -2.0, 0.25)
    A = CSROperator(rowptr, col, vals).dense()
    h = 1 / (s + 1)
    inner = [iy * s + ix for iy in range(1, s - 1) for ix in range(1, s - 1)]
    assert np.allclose(A[inner].sum(axis=1), 0.25j)
    # the convective part is antisymmetric, the diffusive part symmetric
    D = (A + A.T) / 2 - np.diag(np.diag(A))
    C = (A - A.T) / 2
    x = np.linspace(h, 1 - h, s)
    u = np.tile(x, s)                       # u = x: grad u = (1, 0), Laplace u = 0
    assert np.allclose((C @ u)[inner], 3.0)
    assert np.allclose(((D + np.diag(np.diag(A).real)) @ u)[inner], 0, atol=1e-8)


def test_generators_deterministic():
    a = W.z2_noise(W.rng(3, 1), 100, 2)
    b = W.z2_noise(W.rng(3, 1), 100, 2)
    assert np.array_equal(a, b)
    assert np.allclose(np.abs(a), 1.0)
    assert set(np.round(a.real * np.sqrt(2)).astype(int).ravel()) == {-1, 1}
    k = W.kappa_list(0.2, 6)
    assert k[0] == pytest.approx(0.196) and k[-1] == pytest.approx(0.115)
