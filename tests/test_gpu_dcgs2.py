"""Arnoldi cycles of the complex64 stages against the oracle (runs on a GB300; -m gpu).

The complex64 stages build the recurrence A V_m = V_{m+1} Hbar_m (eq. recurAr)
by Gram-Schmidt with delayed reorthogonalisation (each step's second pass
merged into the next step's projection), the FP64 stages by classical
Gram-Schmidt twice, as the oracle does.  The complex64 result is not the
oracle's to rounding level in every column (rounding in a Krylov recurrence
grows with the step), so it is checked by the properties that define it, at
any size:

* V_{m+1} orthonormal, ||V^H V - I||_max <= 1e-5;
* the Arnoldi relation with the oracle's complex128 operator,
  ||A V_m - V_{m+1} Hbar_m|| / ||Hbar_m|| <= 1e-5 (complex64 rounding of
  O(1e3) terms, u = 6e-8);
* Hbar_m upper Hessenberg with a real positive subdiagonal after a start from
  one vector, and equal to the oracle's first columns to 1e-5;
* after a restart from a kept pair (j0 = k, the Schur-vector restart that
  keeps A V_k = V_{k+1} Hbar_k), the same relation over all m columns; the
  FP64 cycle equals the oracle's continuation to 1e-10;
* a lucky breakdown (an exactly invariant start vector) stops at m_eff = 1.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import CSROperator, WilsonOperator, arnoldi_cgs2_step
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_0707_0502_gb300 as g  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = g.gdr_create(0)
    yield c
    g.gdr_destroy(c)


def make_case(ctx, case):
    if case.startswith("wilson"):
        dims = tuple(int(x) for x in case.split("_")[1].split("x"))
        links = W.su3_links(dims, 0.4, W.rng(33, 0))
        A = WilsonOperator(dims, links, diag_a=0.0)
        op = g.gdr_op_wilson(ctx, dims, dev(links), 0.0, g.GDR_LINK_C64)
        return A.matvec, A.n, op
    if case == "bidiag":
        rowptr, col, vals = W.config(1).op[1:]
    else:
        rowptr, col, vals = W.convdiff_csr(36, 12.0, -7.0, 0.3)  # n = 1296
    A = CSROperator(rowptr, col, vals)
    op = g.gdr_op_csr(ctx, dev(rowptr), dev(col), dev(vals))
    return A.matvec, A.n, op


def oracle_arnoldi(matvec, v0, m, V=None, H=None, j0=0):
    n = v0.shape[0]
    if V is None:
        V = np.zeros((n, m + 1), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        V[:, 0] = v0 / np.linalg.norm(v0)
    for j in range(j0, m):
        arnoldi_cgs2_step(matvec, V, H, j)
    return V, H


def run_cycle(ctx, op, prec, V0, H0, j0, m, flags=0):
    """V0: n x (j0+1) start columns, H0: (m+1) x m with the kept columns; returns V, Hbar, m_eff."""
    n = V0.shape[0]
    dt = torch.complex128 if prec == g.GDR_PREC_FP64 else torch.complex64
    V = torch.zeros((m + 1, n), dtype=dt, device="cuda")
    V[: j0 + 1] = dev(V0.T, dt)
    H = dev(np.ascontiguousarray(H0.T))  # column-major (m+1) x m
    me = g.gdr_arnoldi_cycle(ctx, op, prec, V, j0, m, H, flags)
    return host(V).T.astype(np.complex128), host(H).T.copy(), me


def check_relation(matvec, V, H, m, tol):
    orth = np.abs(V.conj().T @ V - np.eye(m + 1)).max()
    AV = np.stack([matvec(V[:, j]) for j in range(m)], axis=1)
    relres = np.linalg.norm(AV - V @ H) / np.linalg.norm(H)
    assert orth <= tol, orth
    assert relres <= tol, relres


CASES = ["wilson_4x4x4x6", "wilson_8x8x8x8", "bidiag", "convdiff"]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("flags", [0, g.GDR_FLAG_CGS2], ids=["dcgs2", "cgs2"])
def test_c64_cycle_from_start(ctx, case, flags):
    matvec, n, op = make_case(ctx, case)
    m = 30
    v0 = np.random.default_rng(5).standard_normal(n) + 1j * np.random.default_rng(6).standard_normal(n)
    v0 /= np.linalg.norm(v0)
    H0 = np.zeros((m + 1, m), dtype=np.complex128)
    V, H, me = run_cycle(ctx, op, g.GDR_PREC_MIXED, v0[:, None], H0, 0, m, flags)
    assert me == m
    check_relation(matvec, V, H, m, 1e-5)
    # Hessenberg, real positive subdiagonal
    assert np.abs(np.tril(H, -2)).max() == 0.0
    sub = np.diag(H, -1)
    assert np.all(sub.real > 0) and np.abs(sub.imag).max() <= 1e-6 * np.abs(sub).max()
    # the first columns equal the oracle's (rounding has not grown yet)
    _, Hr = oracle_arnoldi(matvec, v0, m)
    j5 = 5
    assert np.linalg.norm(H[:, :j5] - Hr[:, :j5]) <= 1e-5 * np.linalg.norm(Hr[:, :j5])
    g.gdr_op_destroy(op)


def kept_pair(matvec, v0, m, k):
    """A GMRES-DR-style kept pair from an m-step oracle Arnoldi: P_k = Schur vectors
    of H_m for k of its eigenvalues (an invariant subspace of H_m), p_{k+1} = e_{m+1};
    V_{k+1} = V_{m+1} P and Hbar_k = P^H Hbar_m P_k satisfy A V_k = V_{k+1} Hbar_k."""
    V, H = oracle_arnoldi(matvec, v0, m)
    T, Q = sla.schur(H[:m, :m], output="complex")
    Pk = np.vstack([Q[:, :k], np.zeros((1, k))])
    P = np.hstack([Pk, np.eye(m + 1)[:, m:]])
    Vk1 = V @ P
    Hk = P.conj().T @ H @ Pk[:m]
    return Vk1, Hk


@pytest.mark.parametrize("case", ["wilson_8x8x8x8", "convdiff"])
@pytest.mark.parametrize("prec", [g.GDR_PREC_MIXED, g.GDR_PREC_FP64], ids=["c64", "fp64"])
def test_cycle_after_restart(ctx, case, prec):
    matvec, n, op = make_case(ctx, case)
    m, k = 30, 12
    v0 = np.random.default_rng(7).standard_normal(n) + 0.5j
    Vk1, Hk = kept_pair(matvec, v0, m, k)
    assert np.linalg.norm(np.stack([matvec(Vk1[:, j]) for j in range(k)], 1) - Vk1 @ Hk) <= 1e-12 * np.linalg.norm(Hk)
    H0 = np.zeros((m + 1, m), dtype=np.complex128)
    H0[: k + 1, :k] = Hk
    V, H, me = run_cycle(ctx, op, prec, Vk1, H0, k, m)
    assert me == m
    check_relation(matvec, V, H, m, 1e-5 if prec == g.GDR_PREC_MIXED else 1e-12)
    assert np.abs(np.tril(H[:, k:], -(k + 2))).max() == 0.0  # rows below j+1 stay zero
    if prec == g.GDR_PREC_FP64:  # the oracle's CGS2 continuation, to rounding
        Vr = np.zeros((n, m + 1), dtype=np.complex128)
        Vr[:, : k + 1] = Vk1
        Hr = H0.copy()
        Vr, Hr = oracle_arnoldi(matvec, Vk1[:, 0], m, Vr, Hr, k)
        assert np.linalg.norm(H - Hr) <= 1e-10 * np.linalg.norm(Hr)
        assert np.linalg.norm(V - Vr) <= 1e-10 * np.linalg.norm(Vr)
    g.gdr_op_destroy(op)


@pytest.mark.parametrize("flags", [0, g.GDR_FLAG_CGS2], ids=["dcgs2", "cgs2"])
def test_c64_lucky_breakdown(ctx, flags):
    """A diagonal matrix and v_0 = e_0: A v_0 = a_0 v_0 exactly, so the first
    orthogonalised vector is exactly zero and the cycle stops with m_eff = 1."""
    n = 64
    a = np.arange(1, n + 1, dtype=np.float64) * (1.0 + 0.5j)
    rowptr = np.arange(n + 1, dtype=np.int32)
    col = np.arange(n, dtype=np.int32)
    op = g.gdr_op_csr(ctx, dev(rowptr), dev(col), dev(a.astype(np.complex128)))
    m = 8
    v0 = np.zeros(n, dtype=np.complex128)
    v0[0] = 1.0
    V, H, me = run_cycle(ctx, op, g.GDR_PREC_MIXED, v0[:, None], np.zeros((m + 1, m), complex), 0, m, flags)
    assert me == 1
    assert abs(H[0, 0] - a[0]) <= 1e-6 * abs(a[0])
    assert abs(H[1, 0]) <= 1e-6
    assert np.all(V[:, 1:] == 0)  # no vector after the breakdown
    g.gdr_op_destroy(op)
