"""Pins of the oracle's FOM-Sh and FOM-DR-Sh (Sec. 3, Examples 2 and 3), the Galerkin
counterparts of GMRES-Sh and GMRES-DR-Sh (comparison methods in the paper).

* Cycle 1 of FOM(m)-Sh is the Galerkin solution: every shifted residual is orthogonal
  to the Krylov space K_m (brute force over explicit Krylov vectors) and all residuals
  are parallel to v_{m+1}; the collinearity factors and shortcut norms match the true
  residuals after restarted cycles; FOM-DR keeps the recurrence A V_k = V_{k+1} Hbar_k.
* Example 2 (Example 1 matrix, m = 40, shifts 0.4 (base), 0, -1): GMRES-Sh is better for
  the base shift, FOM-Sh for the shift 0, and FOM-Sh reaches 1e-8 for the shift -1
  within 400 matvecs while GMRES-Sh does not.
* Example 3 (m = 80, shifts 0 (base), 1.4): FOM-Sh fails on the shift 1.4 where GMRES-Sh
  converges far further, and FOM-DR-Sh(80,2) reaches 1e-8 on it."""
import numpy as np

import workloads as W
from oracle import CSROperator, fom_sh_dense_step, gmres_dr_sh, ritz
from tests.test_oracle_gmres_dr import tiny_matrix

SIG = np.array([0.0, -0.4, -1.5], dtype=np.complex128)


def test_fom_cycle1_is_galerkin():
    A, b = tiny_matrix(seed=4)
    m = 6
    r = gmres_dr_sh(lambda v: A @ v, b, SIG, m, 0, 1e-14, max_cycles=1, method="fom")
    K = np.empty((A.shape[0], m + 1), dtype=complex)
    K[:, 0] = b
    for j in range(m):
        K[:, j + 1] = A @ K[:, j]
    Q = np.linalg.qr(K)[0]
    Km, v_next = Q[:, :m], Q[:, m]
    res = [b - (A @ r["x"][:, i] - s * r["x"][:, i]) for i, s in enumerate(SIG)]
    for i in range(len(SIG)):
        assert np.linalg.norm(Km.conj().T @ res[i]) < 1e-10 * np.linalg.norm(b)
        # parallel to v_{m+1}
        assert np.linalg.norm(res[i] - np.vdot(v_next, res[i]) * v_next) < 1e-10 * np.linalg.norm(b)
        # x_i in K_m
        x = r["x"][:, i]
        assert np.linalg.norm(x - Km @ (Km.conj().T @ x)) < 1e-10 * np.linalg.norm(x)


def test_fom_restarts_keep_collinear_residuals():
    A, b = tiny_matrix(seed=5)
    for k in (0, 3):
        r = gmres_dr_sh(lambda v: A @ v, b, SIG, 8, k, 1e-14, max_cycles=4, method="fom", record=True)
        for h in r["history"]:
            r1 = b - (A @ h["x"][:, 0] - SIG[0] * h["x"][:, 0])
            for i, s in enumerate(SIG):
                ri = b - (A @ h["x"][:, i] - s * h["x"][:, i])
                assert np.linalg.norm(ri - h["beta"][i] * r1) < 1e-9 * np.linalg.norm(b), (k, i)
                assert abs(np.linalg.norm(ri) - h["norms"][i]) < 1e-9 * np.linalg.norm(b), (k, i)
        if k:
            Vk1, Hk = r["Vk1"], r["Hk"]
            assert np.linalg.norm(A @ Vk1[:, :k] - Vk1 @ Hk) < 1e-10 * np.linalg.norm(Hk)


def test_fom_step_and_ritz_definitions():
    g = np.random.default_rng(6)
    m = 7
    Hbar = np.triu(g.standard_normal((m + 1, m)) + 1j * g.standard_normal((m + 1, m)), -1)
    c = np.zeros(m + 1, complex)
    c[0] = 2.0
    beta = np.array([1.0, 0.5 + 0.5j, -1.0])
    D, s, bn, nrm = fom_sh_dense_step(Hbar, c, SIG, beta, np.ones(3, bool))
    Ib = np.eye(m + 1, m)
    for i, sg in enumerate(SIG):
        ri = beta[i] * c - (Hbar - sg * Ib) @ D[:, i]
        assert np.linalg.norm(ri[:m]) < 1e-12 * np.linalg.norm(c)        # Galerkin
        assert abs(ri[m] - bn[i] * s[m]) < 1e-12 * abs(s[m])              # parallel to the base
    theta, idx, G = ritz(Hbar - SIG[0] * Ib, 3)
    for q, i in enumerate(idx):
        assert np.linalg.norm(Hbar[:m] @ G[:, q] - (theta[i] + SIG[0]) * G[:, q]) < 1e-10


def _first(r, i, nb, tol=1e-8):
    for h in r["history"]:
        if h["norms"][i] <= tol * nb:
            return h["mvps"]
    return None


def test_example2_gmres_vs_fom():
    rowptr, col, vals = W.paper_example1_matrix()
    A = CSROperator(rowptr, col, vals)
    b = np.random.default_rng([41, 0]).standard_normal(1000).astype(complex)
    nb = np.linalg.norm(b)
    sig = np.array([0.4, 0.0, -1.0], complex)
    gm = gmres_dr_sh(A.matvec, b, sig, 40, 0, 1e-8, max_mvps=800, record=True)
    fo = gmres_dr_sh(A.matvec, b, sig, 40, 0, 1e-8, max_mvps=800, record=True, method="fom")
    assert gm["norms"][0] < fo["norms"][0]                 # base 0.4: GMRES better
    assert fo["norms"][1] < 0.1 * gm["norms"][1]           # shift 0: FOM better
    f1 = _first(fo, 2, nb)
    g1 = _first(gm, 2, nb)
    assert f1 is not None and f1 <= 400, f1                # shift -1: FOM under 1e-8 within 400
    assert g1 is None or g1 > 400, g1


def test_example3_fom_dr_fixes_the_shift():
    rowptr, col, vals = W.paper_example1_matrix()
    A = CSROperator(rowptr, col, vals)
    b = np.random.default_rng([41, 0]).standard_normal(1000).astype(complex)
    nb = np.linalg.norm(b)
    sig = np.array([0.0, 1.4], complex)
    gm = gmres_dr_sh(A.matvec, b, sig, 80, 0, 1e-8, max_mvps=1200, record=True)
    fo = gmres_dr_sh(A.matvec, b, sig, 80, 0, 1e-8, max_mvps=1200, record=True, method="fom")
    fd = gmres_dr_sh(A.matvec, b, sig, 80, 2, 1e-8, max_mvps=1200, record=True, method="fom")
    assert fo["norms"][1] > 1e-2 * nb                      # FOM-Sh(80) fails on 1.4
    assert gm["norms"][1] < 1e-4 * nb                      # GMRES-Sh(80) far better
    fd1 = _first(fd, 1, nb)
    assert fd1 is not None and fd1 <= 600, fd1             # FOM-DR-Sh(80,2) fixes it
