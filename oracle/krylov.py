"""Deflated multi-shift GMRES, written out plainly in complex128.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows the paper: A is n x n, sigma_1 is the base shift, the Arnoldi
/ GMRES-DR recurrence is A V_m = V_{m+1} Hbar_m (eq. recurAr / recur0), Ibar
is the (m+1) x m identity, c holds the coordinates of the current residual in
V_{m+1} (r_0 = V_{m+1} c), beta_i are the collinearity factors
r_{0,i} = beta_i r_{0,1} (Sec. 2.1).  Indices in code are 0-based: v_j in the
code is v_{j+1} in the paper.

Readings of the paper used here:
  * orthogonalisation is classical Gram-Schmidt with one full
    reorthogonalisation (CGS2); v_{k+1} is reorthogonalised after a restart;
  * harmonic Ritz vectors (Sec. 2.2 cites GMRES-DR for the formula) are taken
    with respect to the base-shifted matrix Hhat = Hbar - sigma_1 Ibar:
    M = H + f hrow with H = Hhat[:m], hrow = Hhat[m], f = H^{-H} hrow^H,
    i.e. the pencil Hhat^H Hhat g = theta H^H g; the k of smallest |theta|
    are kept, ties (relative 1e-9) broken by larger Im(theta), then larger
    Re(theta);
  * convergence is the relative 2-norm ||r_i|| / ||b|| <= tol tested at the
    end of each cycle with the shortcut norms of eq. (gsh3); converged
    non-base shifts are frozen;
  * the Proj phase keeps the v_{k+1} component aside (Sec. 4) and the
    correction uses gamma_i = v_{k+1}^H r_i with the true residual r_i
    (eq. keyder4b);
  * lucky breakdown: when h_{j+1,j} <= 1e-12 ||A v_j|| the space is invariant
    and every shifted system is solved exactly from the square system.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

BREAKDOWN_RTOL = 1e-12
TIE_RTOL = 1e-9


def _ibar(rows, cols):
    return np.eye(rows, cols, dtype=np.complex128)


# --------------------------------------------------------------------------
# Arnoldi (eq. recurAr), classical Gram-Schmidt twice
# --------------------------------------------------------------------------

def arnoldi_cgs2_step(matvec, V, Hbar, j):
    """Add column j of A V = V Hbar: w = A v_j, orthogonalise w against
    v_0..v_j twice (classical Gram-Schmidt), h_{j+1,j} = ||w||,
    v_{j+1} = w / h_{j+1,j}.  Returns (h_{j+1,j}, ||A v_j||)."""
    w = matvec(V[:, j])
    w0 = np.linalg.norm(w)
    Vj = V[:, : j + 1]
    h1 = Vj.conj().T @ w
    w = w - Vj @ h1
    h2 = Vj.conj().T @ w
    w = w - Vj @ h2
    Hbar[: j + 1, j] = h1 + h2
    hn = np.linalg.norm(w)
    Hbar[j + 1, j] = hn
    if hn > BREAKDOWN_RTOL * w0:
        V[:, j + 1] = w / hn
    return hn, w0


# --------------------------------------------------------------------------
# GMRES-Sh small problem (Sec. 2.1, eqs. gsh1-gsh3; GMRES-DR-Sh steps 3-5)
# --------------------------------------------------------------------------

def gmres_sh_dense_step(Hbar, c, sigma, beta, active):
    """One GMRES-Sh reduced solve.

    Base system: d_1 = argmin ||c - (Hbar - sigma_1 Ibar) d||,
    s = c - (Hbar - sigma_1 Ibar) d_1.  Other shifts: QR factorisation
    Hbar - sigma_i Ibar = Q R, then R d_i = beta_i Q^H c - beta_i^new Q^H s
    where the last row (zero on the left) gives beta_i^new and the first m
    rows give d_i.  Shortcut norms (eq. gsh3): ||r_1|| = ||s||,
    ||r_i|| = |beta_i^new| ||s||.

    Returns D (m x ns; inactive columns zero), s, beta_new, norms."""
    m = Hbar.shape[1]
    ns = len(sigma)
    Ib = _ibar(m + 1, m)
    Hs1 = Hbar - sigma[0] * Ib
    d1 = sla.lstsq(Hs1, c)[0]
    s = c - Hs1 @ d1
    snorm = np.linalg.norm(s)
    D = np.zeros((m, ns), dtype=np.complex128)
    D[:, 0] = d1
    beta_new = np.array(beta, dtype=np.complex128)
    for i in range(1, ns):
        if not active[i]:
            continue
        Q, R = sla.qr(Hbar - sigma[i] * Ib)           # Q: (m+1)x(m+1), R: (m+1)xm
        qc = Q.conj().T @ c
        qs = Q.conj().T @ s
        beta_new[i] = beta[i] * qc[m] / qs[m]
        D[:, i] = sla.solve_triangular(R[:m, :m], beta[i] * qc[:m] - beta_new[i] * qs[:m])
    norms = np.abs(beta_new) * snorm
    norms[0] = snorm
    return D, s, beta_new, norms


def fom_sh_dense_step(Hbar, c, sigma, beta, active):
    """One FOM-Sh reduced solve (Sec. 3, Examples 2-3: the Galerkin counterpart of
    GMRES-Sh).  Every shift solves the square system (H_m - sigma_i I) d_i = beta_i c[:m];
    each residual beta_i c - (Hbar - sigma_i Ibar) d_i is then a multiple of e_{m+1}
    (the residuals are parallel without any constraint), so with the base residual
    s = c - (Hbar - sigma_1 Ibar) d_1: beta_i^new = (beta_i c - (Hbar - sigma_i Ibar) d_i)[m] / s[m].
    Returns D, s, beta_new, norms as gmres_sh_dense_step."""
    m = Hbar.shape[1]
    ns = len(sigma)
    Ib = _ibar(m + 1, m)
    Hs1 = Hbar - sigma[0] * Ib
    d1 = np.linalg.solve(Hs1[:m], c[:m])
    s = c - Hs1 @ d1
    snorm = np.linalg.norm(s)
    D = np.zeros((m, ns), dtype=np.complex128)
    D[:, 0] = d1
    beta_new = np.array(beta, dtype=np.complex128)
    for i in range(1, ns):
        if not active[i]:
            continue
        Hsi = Hbar - sigma[i] * Ib
        di = np.linalg.solve(Hsi[:m], beta[i] * c[:m])
        beta_new[i] = (beta[i] * c - Hsi @ di)[m] / s[m]
        D[:, i] = di
    norms = np.abs(beta_new) * snorm
    norms[0] = snorm
    return D, s, beta_new, norms


def ritz(Hs, k):
    """Regular Ritz pairs of the shifted recurrence matrix Hs = Hbar - sigma_1 Ibar:
    eigenpairs of its square part Hs[:m] (the restart of FOM-DR).  Returns
    (theta_all, chosen indices, G_chosen (m x k)) like harmonic_ritz."""
    m = Hs.shape[1]
    theta, G = sla.eig(Hs[:m, :])
    idx = select_smallest(theta, k)
    return theta, idx, G[:, idx]


# --------------------------------------------------------------------------
# harmonic Ritz vectors (Sec. 2.2; formula from the cited GMRES-DR paper)
# --------------------------------------------------------------------------

def _before(a, b):
    """Selection order for 'smallest' harmonic Ritz values."""
    ma, mb = abs(a), abs(b)
    scale = max(ma, mb)
    if abs(ma - mb) > TIE_RTOL * scale:
        return ma < mb
    if abs(a.imag - b.imag) > TIE_RTOL * scale:
        return a.imag > b.imag
    return a.real > b.real


def select_smallest(theta, k):
    """Indices of the k 'smallest' values under ``_before`` (selection sort,
    scanning in index order)."""
    remaining = list(range(len(theta)))
    chosen = []
    for _ in range(k):
        best = remaining[0]
        for i in remaining[1:]:
            if _before(theta[i], theta[best]):
                best = i
        chosen.append(best)
        remaining.remove(best)
    return chosen


def harmonic_ritz(Hs, k):
    """Harmonic Ritz pairs of the shifted recurrence matrix Hs = Hbar - sigma_1
    Ibar ((m+1) x m).  Solves (H + f hrow) g = theta g with H = Hs[:m],
    hrow = Hs[m] and H^H f = hrow^H.  Returns (theta_all, chosen indices,
    G_chosen (m x k))."""
    m = Hs.shape[1]
    H = Hs[:m, :]
    hrow = Hs[m, :]
    f = np.linalg.solve(H.conj().T, hrow.conj())
    M = H + np.outer(f, hrow)
    theta, G = sla.eig(M)
    idx = select_smallest(theta, k)
    return theta, idx, G[:, idx]


# --------------------------------------------------------------------------
# GMRES-DR(m,k)-Sh (Sec. 3, algorithm "GMRES-DR-Sh")
# --------------------------------------------------------------------------

def _restart_matrices(Hbar, s, G):
    """GMRES-DR restart: orthonormal P_k from [G; 0], p_{k+1} from s, then
    the new leading block Hbar_k = P_{k+1}^H Hbar P_k and c = P_{k+1}^H s."""
    m = Hbar.shape[1]
    k = G.shape[1]
    Gpad = np.vstack([G, np.zeros((1, k), dtype=np.complex128)])
    Pk = np.linalg.qr(Gpad)[0]
    p = s - Pk @ (Pk.conj().T @ s)
    p = p - Pk @ (Pk.conj().T @ p)
    p = p / np.linalg.norm(p)
    P = np.hstack([Pk, p[:, None]])
    Hk = P.conj().T @ Hbar @ Pk[:m, :]
    ck = P.conj().T @ s
    return P, Hk, ck


def _reorth_last(V, k):
    """Classical Gram-Schmidt twice of v_k against v_0..v_{k-1}, normalise."""
    v = V[:, k]
    Vk = V[:, :k]
    for _ in range(2):
        v = v - Vk @ (Vk.conj().T @ v)
    V[:, k] = v / np.linalg.norm(v)


def _solve_invariant(Hbar, c, j1, sigma, beta, active):
    """Lucky breakdown after j1 Arnoldi columns: span(V[:, :j1]) is invariant,
    every shifted system is solved by the square j1 x j1 system."""
    Hsq = Hbar[:j1, :j1]
    ns = len(sigma)
    D = np.zeros((j1, ns), dtype=np.complex128)
    for i in range(ns):
        if i == 0 or active[i]:
            D[:, i] = np.linalg.solve(Hsq - sigma[i] * np.eye(j1), beta[i] * c[:j1])
    return D


def gmres_dr_sh(matvec, b, sigma, m, k, tol, max_mvps=100000, max_cycles=None, record=False, method="gmres"):
    """GMRES-DR(m,k)-Sh for (A - sigma_i I) x_i = b, zero initial guess.

    Returns a dict with
      x      : n x ns solutions,
      mvps   : matrix-vector products with A (m in the first cycle, m - k after),
      cycles, converged (per shift), norms (shortcut, last cycle),
      Vk1, Hk: the kept deflation pair A V_k = V_{k+1} Hbar_k (eq. recur1),
               from a restart computed on the final cycle,
      history: per-cycle records when ``record`` (mvps, norms, beta, x copy,
               theta, Vm, Hbar, c, G).
    """
    b = np.asarray(b, np.complex128)
    sigma = np.asarray(sigma, np.complex128)
    n, ns = b.shape[0], len(sigma)
    x = np.zeros((n, ns), dtype=np.complex128)
    beta = np.ones(ns, dtype=np.complex128)
    active = np.ones(ns, dtype=bool)
    bnorm = np.linalg.norm(b)
    V = np.zeros((n, m + 1), dtype=np.complex128)
    Hbar = np.zeros((m + 1, m), dtype=np.complex128)
    c = np.zeros(m + 1, dtype=np.complex128)
    V[:, 0] = b / bnorm
    c[0] = bnorm
    j0 = 0
    mvps = 0
    cycles = 0
    history = []
    Vk1 = Hk = None
    norms = np.full(ns, bnorm)
    while True:
        # step 2: extend the recurrence A V_m = V_{m+1} Hbar_m
        broke = None
        for j in range(j0, m):
            hn, w0 = arnoldi_cgs2_step(matvec, V, Hbar, j)
            mvps += 1
            if hn <= BREAKDOWN_RTOL * w0:
                broke = j + 1
                break
        cycles += 1
        if broke is not None:
            D = _solve_invariant(Hbar, c, broke, sigma, beta, active)
            x += V[:, :broke] @ D
            norms = np.zeros(ns)
            active[:] = False
            converged = np.ones(ns, dtype=bool)
            break
        # steps 3-5: base least squares, shifted solves, solution updates
        # (method "fom": FOM-Sh / FOM-DR-Sh, Sec. 3 Examples 2-3: Galerkin solves, Ritz restart)
        step = fom_sh_dense_step if method == "fom" else gmres_sh_dense_step
        D, s, beta_new, nrm = step(Hbar, c, sigma, beta, active)
        x += V[:, :m] @ D
        upd = active.copy()
        upd[0] = True
        beta = np.where(upd, beta_new, beta)
        norms = np.where(upd, nrm, norms)      # a frozen shift keeps its residual
        Hs1 = Hbar - sigma[0] * _ibar(m + 1, m)
        theta, idx, G = (ritz if method == "fom" else harmonic_ritz)(Hs1, k)
        if record:
            history.append(dict(mvps=mvps, norms=norms.copy(), beta=beta.copy(), x=x.copy(),
                                theta=theta, idx=idx, G=G, Vm=V.copy(), Hbar=Hbar.copy(), c=c.copy(),
                                s=s.copy()))
        # step 6: convergence test; frozen shifts stop updating
        conv = norms <= tol * bnorm
        active &= ~conv
        active[0] = True
        converged = conv
        P, Hk_new, ck = _restart_matrices(Hbar, s, G)
        V[:, : k + 1] = V @ P
        _reorth_last(V, k)
        if conv.all() or mvps >= max_mvps or (max_cycles is not None and cycles >= max_cycles):
            Vk1 = V[:, : k + 1].copy()
            Hk = Hk_new.copy()
            break
        Hbar[:] = 0
        Hbar[: k + 1, :k] = Hk_new
        c[:] = 0
        c[: k + 1] = ck
        j0 = k
    return dict(x=x, mvps=mvps, cycles=cycles, converged=converged, norms=norms, beta=beta,
                Vk1=Vk1, Hk=Hk, history=history)


# --------------------------------------------------------------------------
# Minres projection over V_k (Sec. 2.3) and GMRES-Proj-Sh (Sec. 4)
# --------------------------------------------------------------------------

def minres_projection(Vk1, Hk, sigma1, r0):
    """Minres Projection for V_k applied to A - sigma1 I:
    c = V_{k+1}^H r_0, d = argmin ||c - (Hbar_k - sigma1 Ibar) d||,
    dx = V_k d, r = r_0 - V_{k+1} (Hbar_k - sigma1 Ibar) d."""
    k = Hk.shape[1]
    Hs = Hk - sigma1 * _ibar(k + 1, k)
    c = Vk1.conj().T @ r0
    d = sla.lstsq(Hs, c)[0]
    dx = Vk1[:, :k] @ d
    r = r0 - Vk1 @ (Hs @ d)
    return d, dx, r


def kept_eigenpairs(Hk, sigma1, k_sel):
    """Approximate eigenpairs carried by the kept pair A V_k = V_{k+1} Hbar_k (eq. recur1):
    the harmonic Ritz pairs of span(V_k) with respect to the base shift (the same
    formula as the restart, on Hbar_k - sigma1 Ibar), the k_sel 'smallest' ones (Sec. 4,
    Example 4 keeps "the first k").  Returns (theta (k_sel): eigenvalue approximations
    of A, G (k x k_sel): z_l = V_k g_l with ||g_l|| = 1, res (k_sel): eigen-residual
    norms ||A z_l - theta_l z_l|| = ||(Hbar_k - theta_l Ibar) g_l||)."""
    k = Hk.shape[1]
    theta, idx, G = harmonic_ritz(Hk - sigma1 * _ibar(k + 1, k), k_sel)
    G = G / np.linalg.norm(G, axis=0)
    th = theta[idx] + sigma1
    res = np.array([np.linalg.norm(Hk @ G[:, l] - th[l] * _ibar(k + 1, k) @ G[:, l]) for l in range(k_sel)])
    return th, G, res


def eigvec_projection(Vk1, Hk, th, G, sigma, beta, active, r):
    """Projection of every shifted system over approximate eigenvectors Z = V_k G with
    eigenvalues th, as in the proof of Theorem 1 (Sec. 4): d_i = beta_i (Theta - sigma_i)^{-1}
    (Z^H Z)^{-1} Z^H r, x_i += Z d_i.  Returns (the new base residual r - (A - sigma_1 I) Z d_1,
    computed through the recurrence, and the n x ns solution increments).  With exact
    eigenvectors every shifted residual is beta_i times the new base residual; with
    approximate ones the algorithm assumes it."""
    k = Hk.shape[1]
    Z = Vk1[:, :k] @ G
    w = np.linalg.solve(Z.conj().T @ Z, Z.conj().T @ r)
    dx = np.zeros((r.shape[0], len(sigma)), dtype=np.complex128)
    for i in range(len(sigma)):
        if i == 0 or active[i]:
            dx[:, i] = Z @ (beta[i] * w / (th - sigma[i]))
    d1 = w / (th - sigma[0])
    rnew = r - Vk1 @ ((Hk - sigma[0] * _ibar(k + 1, k)) @ (G @ d1))
    return rnew, dx


def gmres_proj_sh(matvec, Vk1, Hk, b, sigma, m_p, tol, max_mvps=100000, record=False, project=True, eig=None):
    """GMRES(m_p)-Proj(k)-Sh for one right-hand side (Sec. 4, algorithm
    "GMRES-Proj-Sh for the second and subsequent right-hand sides", steps
    2-6).  Zero initial guess.  The non-base residuals are
    beta_i r + g_i v_{k+1}; the v_{k+1} part is ignored by the test and
    removed later by the correction.  ``project=False`` gives plain
    GMRES(m_p)-Sh (no deflation).  ``eig=(theta, G)`` replaces the Minres
    projection over V_k by the projection over the selected approximate
    eigenvectors V_k G (``eigvec_projection``; Sec. 4, Theorem 1 and Example 4):
    no v_{k+1} component is tracked and no correction applies.

    Returns dict(x, mvps, cycles, converged, norms, beta, gamma_acc, history)."""
    b = np.asarray(b, np.complex128)
    sigma = np.asarray(sigma, np.complex128)
    n, ns = b.shape[0], len(sigma)
    k = Hk.shape[1] if Hk is not None else 0
    x = np.zeros((n, ns), dtype=np.complex128)
    beta = np.ones(ns, dtype=np.complex128)
    gamma = np.zeros(ns, dtype=np.complex128)
    active = np.ones(ns, dtype=bool)
    bnorm = np.linalg.norm(b)
    r = b.copy()
    mvps = 0
    cycles = 0
    history = []
    norms = np.full(ns, bnorm)
    converged = np.zeros(ns, dtype=bool)
    while True:
        if project and k > 0 and eig is not None:
            r, dx = eigvec_projection(Vk1, Hk, eig[0], eig[1], sigma, beta, active, r)
            x += dx
        elif project and k > 0:
            # step 3: Minres projection for V_k on the base shift
            d1, dx1, r = minres_projection(Vk1, Hk, sigma[0], r)
            x[:, 0] += dx1
            # step 4: (H_k - sigma_i I) d_i = beta_i (H_k - sigma_1 I) d_1
            Hsq = Hk[:k, :k]
            t = Hk @ d1 - sigma[0] * np.concatenate([d1, [0]])
            for i in range(1, ns):
                if not active[i]:
                    continue
                di = np.linalg.solve(Hsq - sigma[i] * np.eye(k), beta[i] * (Hsq @ d1 - sigma[0] * d1))
                x[:, i] += Vk1[:, :k] @ di
                # eq. keyder2: (Hbar_k - sigma_i Ibar) d_i = t_i - gamma_i e_{k+1}
                lhs = Hk @ di - sigma[i] * np.concatenate([di, [0]])
                gamma[i] += (beta[i] * t - lhs)[k]
        # step 5: one cycle of GMRES(m_p)-Sh on r
        rn = np.linalg.norm(r)
        W = np.zeros((n, m_p + 1), dtype=np.complex128)
        Hb = np.zeros((m_p + 1, m_p), dtype=np.complex128)
        cw = np.zeros(m_p + 1, dtype=np.complex128)
        W[:, 0] = r / rn
        cw[0] = rn
        broke = None
        for j in range(m_p):
            hn, w0 = arnoldi_cgs2_step(matvec, W, Hb, j)
            mvps += 1
            if hn <= BREAKDOWN_RTOL * w0:
                broke = j + 1
                break
        cycles += 1
        if broke is not None:
            D = _solve_invariant(Hb, cw, broke, sigma, beta, active)
            x += W[:, :broke] @ D
            r = np.zeros_like(r)
            norms = np.zeros(ns)
            converged = np.ones(ns, dtype=bool)
            break
        D, s, beta_new, nrm = gmres_sh_dense_step(Hb, cw, sigma, beta, active)
        x += W[:, :m_p] @ D
        r = W @ s
        upd = active.copy()
        upd[0] = True
        beta = np.where(upd, beta_new, beta)
        norms = np.where(upd, nrm, norms)      # a frozen shift keeps its residual
        if record:
            history.append(dict(mvps=mvps, norms=norms.copy(), x=x.copy(), r=r.copy(), beta=beta.copy(),
                                gamma=gamma.copy()))
        # step 6: test, ignoring the v_{k+1} component of non-base residuals
        conv = norms <= tol * bnorm
        active &= ~conv
        active[0] = True
        converged = conv
        if conv.all() or mvps >= max_mvps:
            break
    return dict(x=x, mvps=mvps, cycles=cycles, converged=converged, norms=norms, beta=beta,
                gamma_acc=gamma, history=history)


def extra_rhs_solve(matvec, Vk1, Hk, sigma, m_p, extra_tol, max_mvps=100000):
    """Shifted systems with the extra right-hand side v_{k+1} (eq. keyder3),
    solved by GMRES-Proj-Sh and then corrected (Sec. 4, algorithm "GMRES-Proj-Sh
    for the extra right-hand side", step 7): s_i = s~_i / (1 - gamma_i),
    gamma_i = v_{k+1}^H r_i with r_i = v_{k+1} - (A - sigma_i I) s~_i."""
    sigma = np.asarray(sigma, np.complex128)
    k = Hk.shape[1]
    v = Vk1[:, k]
    res = gmres_proj_sh(matvec, Vk1, Hk, v, sigma, m_p, extra_tol, max_mvps)
    S = res["x"].copy()
    gam = np.zeros(len(sigma), dtype=np.complex128)
    for i in range(1, len(sigma)):
        ri = v - (matvec(S[:, i]) - sigma[i] * S[:, i])
        gam[i] = np.vdot(v, ri)
        S[:, i] = S[:, i] / (1.0 - gam[i])
    res["S"] = S
    res["gamma"] = gam
    return res


def correct_solutions(matvec, v, S, sigma, b, X):
    """Correction phase (Sec. 4, step 7; eqs. keyder4, keyder4b):
    x_i += (v_{k+1}^H r_i) s_i for the non-base shifts, r_i the true residual."""
    X = X.copy()
    gam = np.zeros(len(sigma), dtype=np.complex128)
    for i in range(1, len(sigma)):
        ri = b - (matvec(X[:, i]) - sigma[i] * X[:, i])
        gam[i] = np.vdot(v, ri)
        X[:, i] += gam[i] * S[:, i]
    return X, gam


# --------------------------------------------------------------------------
# related right-hand sides (Sec. 5, eqs. relrhs1, relrhs2)
# --------------------------------------------------------------------------

def related_rhs_projection(Bprev, Xprev, b):
    """Minres projection over the previous solutions: B^H B d = B^H b^j
    (independent of the shift), x_i = X_i d, common residual b^j - B d.
    ``Xprev`` is n x ns x (j-1).  Returns (x0 n x ns, r, d)."""
    d = sla.lstsq(Bprev, b)[0]
    x0 = np.einsum("nsj,j->ns", Xprev, d)
    r = b - Bprev @ d
    return x0, r, d


# --------------------------------------------------------------------------
# the whole multi-RHS, multi-shift pipeline (Sec. 4, Example 5 order)
# --------------------------------------------------------------------------

def solve_all_rhs(matvec, B, sigma, m, k, m_p, tol, extra_tol, max_mvps=100000):
    """RHS 1 by GMRES-DR(m,k)-Sh; the extra right-hand side v_{k+1} by
    GMRES(m_p)-Proj(k)-Sh + its correction; RHS 2.. by GMRES(m_p)-Proj(k)-Sh
    followed by the correction x_i += (v_{k+1}^H r_i) s_i.

    Returns dict(X: n x ns x nrhs, mvps per stage, Vk1, Hk, S)."""
    B = np.asarray(B, np.complex128)
    if B.ndim == 1:
        B = B[:, None]
    sigma = np.asarray(sigma, np.complex128)
    n, nrhs = B.shape
    ns = len(sigma)
    X = np.zeros((n, ns, nrhs), dtype=np.complex128)
    r1 = gmres_dr_sh(matvec, B[:, 0], sigma, m, k, tol, max_mvps)
    X[:, :, 0] = r1["x"]
    out = dict(mvps_rhs1=r1["mvps"], cycles_rhs1=r1["cycles"], Vk1=r1["Vk1"], Hk=r1["Hk"],
               mvps_extra=0, mvps_proj=[])
    if nrhs > 1:
        ex = extra_rhs_solve(matvec, r1["Vk1"], r1["Hk"], sigma, m_p, extra_tol, max_mvps)
        out["mvps_extra"] = ex["mvps"]
        out["S"] = ex["S"]
        v = r1["Vk1"][:, k]
        for j in range(1, nrhs):
            pr = gmres_proj_sh(matvec, r1["Vk1"], r1["Hk"], B[:, j], sigma, m_p, tol, max_mvps)
            X[:, :, j], _ = correct_solutions(matvec, v, ex["S"], sigma, B[:, j], pr["x"])
            out["mvps_proj"].append(pr["mvps"])
    out["X"] = X
    return out
