"""Pins for the oracle's Minres projection (Sec. 2.3), GMRES-Proj-Sh with the
extra right-hand side and correction phase (Sec. 4), and related
right-hand sides (Sec. 5)."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import (CSROperator, correct_solutions, eigvec_projection, extra_rhs_solve, gmres_dr_sh, gmres_proj_sh,
                    kept_eigenpairs,
                    minres_projection, related_rhs_projection, solve_all_rhs)

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
SIG1 = np.array([0.0, -0.4, -2.0], dtype=np.complex128)     # Example 1 shifts


@pytest.fixture(scope="module")
def ex1():
    """Example 1 matrix, RHS 1 solved by GMRES-DR(25,10)-Sh to 1e-10."""
    rowptr, col, vals = W.paper_example1_matrix()
    A = CSROperator(rowptr, col, vals)
    g = np.random.default_rng([41, 0])
    B = g.standard_normal((1000, 3)).astype(complex)
    r1 = gmres_dr_sh(A.matvec, B[:, 0], SIG1, 25, 10, 1e-10)
    return A, A.dense(), B, r1


def test_minres_projection_is_minimiser(ex1):
    A, Ad, B, r1 = ex1
    Vk1, Hk = r1["Vk1"], r1["Hk"]
    k = Hk.shape[1]
    r0 = B[:, 1]
    for sig in (0.0, -2.0):
        d, dx, r = minres_projection(Vk1, Hk, sig, r0)
        M = (Ad - sig * np.eye(1000)) @ Vk1[:, :k]           # explicit (A - sig I) V_k
        y = np.linalg.lstsq(M, r0, rcond=None)[0]
        assert np.linalg.norm(d - y) < 1e-8 * np.linalg.norm(y)
        assert np.linalg.norm(r - (r0 - M @ y)) < 1e-10 * np.linalg.norm(r0)
        # the projected residual is orthogonal to (A - sig I) V_k
        assert np.linalg.norm(M.conj().T @ r) < 1e-9 * np.linalg.norm(M) * np.linalg.norm(r0)


def test_theorem1_exact_eigenvectors_keep_residuals_parallel():
    """Theorem 1 (Sec. 4): over exact eigenvectors the projection keeps
    r_i = beta_i r_1 (gamma_i = 0), with the non-base update of step 4."""
    g = np.random.default_rng(5)
    n, k = 30, 4
    A = np.diag(np.concatenate([[0.1, 0.3, 0.5, 0.7], np.linspace(2, 5, n - 4)])) + 0.3 * np.triu(
        g.standard_normal((n, n)), 1)
    A = A.astype(complex)
    lam, Z = np.linalg.eig(A)
    sel = np.argsort(np.abs(lam))[:k]
    Vk = np.linalg.qr(Z[:, sel])[0]                 # invariant: A V_k = V_k (V_k^H A V_k)
    v = g.standard_normal(n) + 0j
    v -= Vk @ (Vk.conj().T @ v)
    v /= np.linalg.norm(v)
    Vk1 = np.hstack([Vk, v[:, None]])
    Hk = np.vstack([Vk.conj().T @ A @ Vk, np.zeros((1, k))])
    sig = np.array([0.0, -0.5, -1.2])
    beta = np.array([1.0, 0.7 - 0.2j, 1.3j])
    r0 = g.standard_normal(n) + 1j * g.standard_normal(n)
    d1, dx1, r1 = minres_projection(Vk1, Hk, sig[0], r0)
    for i in (1, 2):
        di = np.linalg.solve(Hk[:k] - sig[i] * np.eye(k), beta[i] * (Hk[:k] @ d1 - sig[0] * d1))
        ri = beta[i] * r0 - (A - sig[i] * np.eye(n)) @ (Vk @ di)
        assert np.linalg.norm(ri - beta[i] * r1) < 1e-12 * np.linalg.norm(ri)


def test_proj_sh_residuals_parallel_except_vk1(ex1):
    """Eq. keyder1: after every projection + GMRES-Sh cycle the non-base
    residuals are beta_i r + g_i v_{k+1}; g_i is the accumulated gamma."""
    A, Ad, B, r1 = ex1
    Vk1, Hk = r1["Vk1"], r1["Hk"]
    v = Vk1[:, -1]
    b = B[:, 1]
    res = gmres_proj_sh(A.matvec, Vk1, Hk, b, SIG1, 15, 1e-10, record=True)
    for h in res["history"]:
        rb = b - Ad @ h["x"][:, 0] + SIG1[0] * h["x"][:, 0]
        assert np.linalg.norm(rb - h["r"]) < 1e-9 * np.linalg.norm(b)
        for i in (1, 2):
            ri = b - Ad @ h["x"][:, i] + SIG1[i] * h["x"][:, i]
            e = ri - h["beta"][i] * rb
            assert np.linalg.norm(e - v * np.vdot(v, e)) < 1e-9 * np.linalg.norm(b)
            assert abs(np.vdot(v, e) - h["gamma"][i]) < 1e-9 * np.linalg.norm(b)


def test_proj_beats_plain_gmres_sh(ex1):
    """Example 7's point on the Example 1 matrix: projecting over the
    eigenvectors from RHS 1 cuts the mvps of GMRES(m)-Sh several-fold."""
    A, Ad, B, r1 = ex1
    pr = gmres_proj_sh(A.matvec, r1["Vk1"], r1["Hk"], B[:, 1], SIG1[:1], 15, 1e-8)
    assert pr["converged"].all()
    gm = gmres_proj_sh(A.matvec, None, None, B[:, 1], SIG1[:1], 15, 1e-8, max_mvps=3 * pr["mvps"],
                       project=False)
    assert not gm["converged"].any(), (gm["mvps"], pr["mvps"])


def test_correction_and_dense_lu(ex1):
    """Full pipeline of Sec. 4 (Example 5 order): every shift of every RHS
    matches dense LU after the correction; before it the non-base shifts
    plateau (Example 5)."""
    A, Ad, B, r1 = ex1
    out = solve_all_rhs(A.matvec, B, SIG1, 25, 10, 15, 1e-10, 1e-6)
    for j in range(3):
        for i, s in enumerate(SIG1):
            M = Ad - s * np.eye(1000)
            xe = np.linalg.solve(M, B[:, j])
            rel_res = np.linalg.norm(B[:, j] - M @ out["X"][:, i, j]) / np.linalg.norm(B[:, j])
            assert rel_res < 3e-10, (i, j, rel_res)
            assert np.linalg.norm(out["X"][:, i, j] - xe) < 1e-7 * np.linalg.norm(xe)


def test_example5_plateau_and_table42_trend(ex1):
    """Example 5: without the correction the sigma=-2 residual levels off
    orders of magnitude above rtol (paper: 4e-3 at rtol 1e-6).  Table 4.2:
    with rtol 1e-8 an extra RHS solved to 1e-5 restores ~rtol accuracy,
    and a loose 1e-1 leaves a much larger residual (paper: 2.4e-8 vs
    9.9e-5 absolute)."""
    A, Ad, B, _ = ex1
    tab = GOLDEN["table4_2"]
    rtol = tab["rtol"]
    r1 = gmres_dr_sh(A.matvec, B[:, 0], SIG1, 25, 10, rtol)
    Vk1, Hk = r1["Vk1"], r1["Hk"]
    v = Vk1[:, -1]
    b = B[:, 1]
    pr = gmres_proj_sh(A.matvec, Vk1, Hk, b, SIG1, 15, rtol)
    M2 = Ad + 2 * np.eye(1000)
    before = np.linalg.norm(b - M2 @ pr["x"][:, 2])
    assert before > 100 * rtol * np.linalg.norm(b)                     # plateau well above rtol
    after = {}
    for et in (1e-5, 1e-1):
        ex = extra_rhs_solve(A.matvec, Vk1, Hk, SIG1, 15, et)
        X, gam = correct_solutions(A.matvec, v, ex["S"], SIG1, b, pr["x"])
        after[et] = np.linalg.norm(b - M2 @ X[:, 2])
    paper_good = tab["after_correction"][tab["extra_tols"].index(1e-5)]
    paper_bad = tab["after_correction"][tab["extra_tols"].index(1e-1)]
    assert after[1e-5] < 30 * paper_good
    assert after[1e-5] < before / 100
    assert after[1e-1] > 10 * after[1e-5]
    assert after[1e-1] < 30 * paper_bad


def test_related_rhs_projection():
    """Sec. 5: B^H B d = B^H b^j is shift independent; all shifted residuals
    equal b^j - B d; a b^j in span(B) is solved exactly for every shift."""
    g = np.random.default_rng(8)
    n = 50
    A = np.diag(np.linspace(1, 4, n)) + 0.2 * np.triu(g.standard_normal((n, n)), 1) + 0j
    sig = np.array([0.0, -0.5, -1.0])
    Bp = g.standard_normal((n, 3)) + 0j
    Xp = np.stack([np.linalg.solve(A - s * np.eye(n), Bp) for s in sig], axis=1)   # n x ns x 3
    bj = Bp @ np.array([0.3, -1.0, 2.0]) + 0j
    x0, r, d = related_rhs_projection(Bp, Xp, bj)
    assert np.linalg.norm(r) < 1e-13 * np.linalg.norm(bj)
    for i, s in enumerate(sig):
        assert np.linalg.norm(x0[:, i] - np.linalg.solve(A - s * np.eye(n), bj)) < 1e-12 * np.linalg.norm(x0)
    bj2 = bj + 1e-4 * g.standard_normal(n)
    x0, r, d = related_rhs_projection(Bp, Xp, bj2)
    for i, s in enumerate(sig):
        ri = bj2 - (A - s * np.eye(n)) @ x0[:, i]
        assert np.linalg.norm(ri - r) < 1e-12 * np.linalg.norm(bj2)
    assert np.linalg.norm(Bp.conj().T @ r) < 1e-12 * np.linalg.norm(bj2)


def test_theorem1_exact_eigenvectors():
    """Theorem 1 (Sec. 4): projecting shifted systems with parallel residuals over
    exact eigenvectors keeps the residuals parallel.  An exactly invariant kept pair
    (V_k spans k eigenvectors, last row of Hbar_k zero): kept_eigenpairs returns the
    exact eigenvalues with zero residuals, and after eigvec_projection every true
    shifted residual is beta_i times the new base residual, which is orthogonal to
    the eigenvectors."""
    g = np.random.default_rng(12)
    n, k = 40, 5
    X = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    lam = np.concatenate([np.array([0.3, 0.7 + 0.2j, 1.1, 1.5 - 0.1j, 2.0]), 4 + g.standard_normal(n - k)])
    A = X @ np.diag(lam) @ np.linalg.inv(X)
    Q = np.linalg.qr(np.hstack([X[:, :k], g.standard_normal((n, 1))]))[0]   # V_{k+1}
    Hk = Q.conj().T @ A @ Q[:, :k]
    assert np.linalg.norm(Hk[k]) < 1e-11 * np.linalg.norm(Hk)
    sig = np.array([0.0, -0.5, -2.0 + 0.3j])
    th, G, res = kept_eigenpairs(Hk, sig[0], k)
    assert np.allclose(np.sort_complex(th), np.sort_complex(lam[:k]), atol=1e-10)
    assert res.max() < 1e-10
    beta = np.array([1.0, 0.7 - 0.2j, 1.3j])
    r0 = g.standard_normal(n) + 1j * g.standard_normal(n)
    r1, dx = eigvec_projection(Q, Hk, th, G, sig, beta, np.ones(3, bool), r0)
    Z = Q[:, :k] @ G
    assert np.linalg.norm(Z.conj().T @ r1) < 1e-11 * np.linalg.norm(r0)
    for i, s in enumerate(sig):
        ri = beta[i] * r0 - (A @ dx[:, i] - s * dx[:, i])
        assert np.linalg.norm(ri - beta[i] * r1) < 1e-11 * np.linalg.norm(r0), i


def test_example4_table4_1():
    """Example 4 / Table 4.1 (Sec. 4) on the Example 1 matrix, shifts 0, -0.4, -2: the
    first right-hand side by GMRES-DR(25,10) to 1e-10, the second by GMRES(15)-Proj-Sh
    over the first k approximate eigenvectors (k = 10, 8, 6, 4, 2).  The paper's RHS is
    unseeded, so over two seeds: the eigen-residual of the k-th vector grows with k and
    stays within a factor 100 of the printed column, the base system's matvec count is
    within one cycle (15) of the printed one, and the worst non-base shift is far less
    accurate with all ten vectors than with the four most accurate."""
    gold = GOLDEN["table4_1"]
    rowptr, col, vals = W.paper_example1_matrix()
    A = CSROperator(rowptr, col, vals)
    sig = np.array([0, -0.4, -2], complex)
    for seed in range(2):
        g = np.random.default_rng([40, seed])
        b1 = g.standard_normal(1000).astype(complex)
        b2 = g.standard_normal(1000).astype(complex)
        r1 = gmres_dr_sh(A.matvec, b1, sig, 25, 10, 1e-10)
        th, G, res = kept_eigenpairs(r1["Hk"], sig[0], 10)
        worst = {}
        for kk, er, mv in zip(gold["k"], gold["eig_res"], gold["mvps"]):
            assert er / 100 <= res[kk - 1] <= er * 100, (seed, kk, res[kk - 1])
            pr = gmres_proj_sh(A.matvec, r1["Vk1"], r1["Hk"], b2, sig, 15, 1e-10, max_mvps=3000,
                               eig=(th[:kk], G[:, :kk]))
            assert abs(pr["mvps"] - mv) <= 15, (seed, kk, pr["mvps"])
            x = pr["x"]
            assert np.linalg.norm(b2 - A.matvec(x[:, 0])) <= 1e-10 * np.linalg.norm(b2)
            worst[kk] = max(np.linalg.norm(b2 - (A.matvec(x[:, i]) - sig[i] * x[:, i])) / np.linalg.norm(b2)
                            for i in (1, 2))
        assert all(res[a - 1] < res[b - 1] for a, b in ((2, 4), (4, 6), (6, 8), (8, 10)))
        assert worst[10] > 30 * worst[4] and worst[10] > 1e-5 and worst[4] < 1e-7, worst
