"""Parity of each CUDA step with the oracle (runs on a GB300; -m gpu).

Tolerances: FP64 paths agree with the complex128 oracle to ~1e2 unit
roundoffs of the quantity; complex64 paths to ~1e-6 relative (FP32 has
u = 6e-8, the sums here have <= 1e3 terms); bfloat16 links to ~1e-2
(u = 4e-3)."""
import numpy as np
import pytest

import workloads as W
from oracle import CSROperator, WilsonOperator, arnoldi_cgs2_step, gmres_dr_sh, gmres_sh_dense_step
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


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


# ---------------------------------------------------------------- matvec a1/a2

# small lattices run the direction-split kernel (ragged last block of 32 sites
# for 2^4 and 3x4x2x6); 16x16x8x8 with 3 columns the thread-per-site kernel
WILSON_DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (3, 4, 2, 6), (8, 4, 4, 2), (16, 16, 8, 8)]


@pytest.mark.parametrize("dims", WILSON_DIMS)
@pytest.mark.parametrize("store", [g.GDR_LINK_C64, g.GDR_LINK_BF16])
def test_wilson_matvec(ctx, dims, store):
    links = W.su3_links(dims, 0.4, W.rng(31, 0))
    op_o = WilsonOperator(dims, links, diag_a=0.25)
    op = g.gdr_op_wilson(ctx, dims, dev(links), 0.25, store)
    rng = np.random.default_rng(3)
    ncol = 3
    X = rng.standard_normal((ncol, op_o.n)) + 1j * rng.standard_normal((ncol, op_o.n))
    sig = np.array([0.0, -7.5 + 0.1j, 2.0])
    ref = np.stack([op_o.matvec(X[c]) - sig[c] * X[c] for c in range(ncol)])
    Y = torch.zeros((ncol, op_o.n), dtype=torch.complex128, device="cuda")
    g.gdr_op_apply(ctx, op, g.GDR_PREC_FP64, sig, dev(X), Y)
    torch.cuda.synchronize()
    assert rel(host(Y), ref) < 1e-14
    Y32 = torch.zeros((ncol, op_o.n), dtype=torch.complex64, device="cuda")
    g.gdr_op_apply(ctx, op, g.GDR_PREC_MIXED, sig, dev(X, torch.complex64), Y32)
    torch.cuda.synchronize()
    assert rel(host(Y32), ref) < (1e-6 if store == g.GDR_LINK_C64 else 1e-2)
    g.gdr_op_destroy(op)


@pytest.mark.parametrize("which", ["bidiag", "convdiff"])
def test_csr_matvec(ctx, which):
    if which == "bidiag":
        rowptr, col, vals = W.config(1).op[1:]
    else:
        rowptr, col, vals = W.convdiff_csr(37, 12.0, -7.0, 0.3)     # odd n = 1369
    A = CSROperator(rowptr, col, vals)
    op = g.gdr_op_csr(ctx, dev(rowptr), dev(col), dev(vals))
    rng = np.random.default_rng(4)
    X = rng.standard_normal((2, A.n)) + 1j * rng.standard_normal((2, A.n))
    sig = np.array([0.5, -1.0 + 2j])
    ref = np.stack([A.matvec(X[c]) - sig[c] * X[c] for c in range(2)])
    Y = torch.zeros((2, A.n), dtype=torch.complex128, device="cuda")
    g.gdr_op_apply(ctx, op, g.GDR_PREC_FP64, sig, dev(X), Y)
    torch.cuda.synchronize()
    assert rel(host(Y), ref) < 1e-14
    g.gdr_op_destroy(op)


# -------------------------------------------------------------- Arnoldi step a3

def _oracle_basis(matvec, n, J, seed):
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    V = np.zeros((n, J + 2), dtype=complex)
    H = np.zeros((J + 2, J + 1), dtype=complex)
    V[:, 0] = b / np.linalg.norm(b)
    for j in range(J):
        arnoldi_cgs2_step(matvec, V, H, j)
    return V


@pytest.mark.parametrize("prob", ["wilson", "bidiag"])
@pytest.mark.parametrize("j", [0, 7, 29])
def test_arnoldi_step(ctx, prob, j):
    if prob == "wilson":
        dims = (4, 4, 4, 4)
        links = W.su3_links(dims, 0.3, W.rng(32, 0))
        A = WilsonOperator(dims, links)
        op = g.gdr_op_wilson(ctx, dims, dev(links), 0.0, g.GDR_LINK_C64)
    else:
        rowptr, col, vals = W.config(1).op[1:]
        A = CSROperator(rowptr, col, vals)
        op = g.gdr_op_csr(ctx, dev(rowptr), dev(col), dev(vals))
    V = _oracle_basis(A.matvec, A.n, j, 5)
    Vo = V.copy()
    Ho = np.zeros((j + 2, j + 1), dtype=complex)
    arnoldi_cgs2_step(A.matvec, Vo, Ho, j)
    # FP64 on the device
    Vt = dev(V[:, : j + 2].T.copy())
    h = torch.zeros(j + 2, dtype=torch.complex128, device="cuda")
    g.gdr_arnoldi_step(ctx, op, g.GDR_PREC_FP64, Vt, j, h)
    torch.cuda.synchronize()
    assert rel(host(h), Ho[:, j]) < 1e-12
    assert rel(host(Vt)[j + 1], Vo[:, j + 1]) < 1e-12
    # complex64: the oracle step on the rounded basis
    V32 = V[:, : j + 2].astype(np.complex64)
    Vr = V32.astype(np.complex128).copy()
    Hr = np.zeros((j + 2, j + 1), dtype=complex)
    arnoldi_cgs2_step(A.matvec, Vr, Hr, j)
    Vt32 = dev(V32.T.copy())
    h32 = torch.zeros(j + 2, dtype=torch.complex128, device="cuda")
    g.gdr_arnoldi_step(ctx, op, g.GDR_PREC_MIXED, Vt32, j, h32)
    torch.cuda.synchronize()
    assert rel(host(h32), Hr[:, j]) < 2e-6
    assert rel(host(Vt32)[j + 1], Vr[:, j + 1]) < 5e-5
    g.gdr_op_destroy(op)


# ------------------------------------------------------------ dense steps a4

def _oracle_cycle(m=25, k=10, cycles=2):
    p = W.config(1)
    A = CSROperator(*p.op[1:])
    res = gmres_dr_sh(A.matvec, p.B[:, 0], p.sigma, m, k, 1e-14, max_cycles=cycles, record=True)
    return p, res["history"]


@pytest.mark.parametrize("cycle", [0, 1])
def test_dense_gmres_sh(ctx, cycle):
    p, hist = _oracle_cycle()
    h = hist[cycle]
    Hbar, c = h["Hbar"], h["c"]
    m = Hbar.shape[1]
    ns = len(p.sigma)
    beta = np.array([1.0, 0.8 - 0.3j, 1.7j, -0.4])
    D, s, bn, nr = gmres_sh_dense_step(Hbar, c, p.sigma, beta, np.ones(ns, bool))
    Dt = torch.zeros((ns, m), dtype=torch.complex128, device="cuda")
    st = torch.zeros(m + 1, dtype=torch.complex128, device="cuda")
    bt = torch.zeros(ns, dtype=torch.complex128, device="cuda")
    nt = torch.zeros(ns, dtype=torch.float64, device="cuda")
    g.gdr_dense_gmres_sh(ctx, m, p.sigma, dev(Hbar.T.copy()), dev(c), dev(beta), Dt, st, bt, nt)
    torch.cuda.synchronize()
    assert rel(host(Dt).T, D) < 1e-10
    assert rel(host(st), s) < 1e-9
    assert rel(host(bt)[1:], bn[1:]) < 1e-10
    assert rel(host(nt), nr) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("cycle", [0, 1])
def test_dense_restart(ctx, cycle, prec):
    """FP64: the oracle's restart to rounding.  Mixed (the FP32 eigensolve used
    with a complex64 basis): the same selection and subspace to FP32 accuracy."""
    p, hist = _oracle_cycle()
    h = hist[cycle]
    Hbar, s = h["Hbar"], h["s"]
    m = Hbar.shape[1]
    k = 10
    fp64 = prec == "fp64"
    tol_th, tol_orth, tol_sub = (1e-9, 1e-12, 1e-9) if fp64 else (1e-5, 1e-6, 1e-4)
    # oracle restart products
    from oracle.krylov import _restart_matrices
    P, Hk, ck = _restart_matrices(Hbar, s, h["G"])
    theta = torch.zeros(m, dtype=torch.complex128, device="cuda")
    Pt = torch.zeros((k + 1, m + 1), dtype=torch.complex128, device="cuda")
    Hkt = torch.zeros((k, k + 1), dtype=torch.complex128, device="cuda")
    ckt = torch.zeros(k + 1, dtype=torch.complex128, device="cuda")
    g.gdr_dense_restart(ctx, g.GDR_PREC_FP64 if fp64 else g.GDR_PREC_MIXED, m, k, p.sigma[0],
                        dev(Hbar.T.copy()), dev(s), theta, Pt, Hkt, ckt)
    torch.cuda.synchronize()
    th = host(theta)
    ref = h["theta"]
    # same spectrum (as multisets)
    for z in ref:
        assert np.min(np.abs(th - z)) < tol_th * np.abs(ref).max()
    Pg, Hg, cg = host(Pt).T, host(Hkt).T, host(ckt)
    assert np.linalg.norm(Pg.conj().T @ Pg - np.eye(k + 1)) < tol_orth
    # basis-independent products: projector, projected recurrence, residual
    assert np.linalg.norm(Pg[:, :k] @ Pg[:, :k].conj().T - P[:, :k] @ P[:, :k].conj().T) < tol_sub
    assert np.linalg.norm(Pg @ Hg @ Pg[:m, :k].conj().T - P @ Hk @ P[:m, :k].conj().T) < tol_sub * np.linalg.norm(Hk)
    assert rel(Pg @ cg, s) < (1e-10 if fp64 else 1e-6)  # mixed: P_k orthonormal to FP32 accuracy
    # the restart keeps an Arnoldi-like recurrence: Hbar P_k lies in span(P_{k+1})
    Hhat = Hbar.copy()
    Hhat[:m] -= p.sigma[0] * np.eye(m)
    HP = Hhat @ Pg[:m, :k]
    assert np.linalg.norm(HP - Pg @ (Pg.conj().T @ HP)) < (1e-12 if fp64 else 1e-5) * np.linalg.norm(Hhat)


def test_basis_update(ctx):
    rng = np.random.default_rng(6)
    n, nv, nout, nx = 1001, 26, 11, 4
    V = rng.standard_normal((n, nv)) + 1j * rng.standard_normal((n, nv))
    C = rng.standard_normal((nv, nout + nx)) + 1j * rng.standard_normal((nv, nout + nx))
    X0 = rng.standard_normal((n, nx)) + 1j * rng.standard_normal((n, nx))
    Vt, Xt = dev(V.T.copy()), dev(X0.T.copy())
    g.gdr_basis_update(ctx, g.GDR_PREC_FP64, n, nv, Vt, dev(C.T.copy()), nout, nx, Xt)
    torch.cuda.synchronize()
    assert rel(host(Vt).T[:, :nout], V @ C[:, :nout]) < 1e-14
    assert rel(host(Vt).T[:, nout:], V[:, nout:]) == 0
    assert rel(host(Xt).T, X0 + V @ C[:, nout:]) < 1e-14
    # complex64 basis, FP64 solutions
    n2 = 1000
    V32 = V[:n2].astype(np.complex64)
    Vt = dev(V32.T.copy())
    Xt = dev(X0[:n2].T.copy())
    g.gdr_basis_update(ctx, g.GDR_PREC_MIXED, n2, nv, Vt, dev(C.T.copy()), nout, nx, Xt)
    torch.cuda.synchronize()
    Vr = V32.astype(complex)
    assert rel(host(Vt).T[:, :nout], Vr @ C[:, :nout]) < 1e-6
    assert rel(host(Xt).T, X0[:n2] + Vr @ C[:, nout:]) < 1e-6


# ------------------------------------------------------------ base least squares (a4)

def hessenberg_with_condition(m, kappa, seed):
    """An (m+1) x m upper Hessenberg matrix whose singular values spread from 1 to about
    1/kappa: a unitarily similar Hessenberg form of U diag(s) W^H, last column dropped."""
    rng = np.random.default_rng(seed)

    def unitary(k):
        q, _ = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
        return q
    s = np.logspace(0, -np.log10(kappa), m + 1)
    M = unitary(m + 1) @ np.diag(s) @ unitary(m + 1).conj().T
    import scipy.linalg as sla
    return sla.hessenberg(M)[:, :m]


@pytest.mark.parametrize("kappa", [1e1, 1e3, 1e6])
@pytest.mark.parametrize("prec", [g.GDR_PREC_FP64, g.GDR_PREC_MIXED], ids=["fp64", "mixed"])
def test_dense_ls(ctx, kappa, prec):
    """The base least squares of a GMRES cycle against numpy's least-squares solution.  The
    complex64-basis form (FP32 QR + one FP64-residual refinement step, random c: a large
    least-squares residual) leaves y accurate to about its correction's size -- ~3e-6 at
    kappa 1e3, ~5e-4 at kappa 1e6 (numpy emulation of the same arithmetic) -- and the
    residual norm within ~1e-9 of the minimum.  At kappa 1e6 the correction exceeds
    1e-4 ||y||, so the FP64 form must take over: the 1e-7 bar there holds only through
    that fallback.  s = c - Hhat y is formed from y in FP64, so its error is bounded by
    ||Hhat|| ||dy||."""
    m = 30
    Hh = hessenberg_with_condition(m, kappa, 11)
    sigma1 = 0.25 - 0.5j
    H = Hh + sigma1 * np.eye(m + 1, m)  # Hbar with Hbar - sigma1 Ibar = Hh
    rng = np.random.default_rng(12)
    c = rng.standard_normal(m + 1) + 1j * rng.standard_normal(m + 1)
    y_ref = np.linalg.lstsq(Hh, c, rcond=None)[0]
    s_ref = c - Hh @ y_ref
    y = torch.zeros(m, dtype=torch.complex128, device="cuda")
    s = torch.zeros(m + 1, dtype=torch.complex128, device="cuda")
    g.gdr_dense_ls(ctx, prec, m, sigma1, dev(np.ascontiguousarray(H.T)), dev(c), y, s)
    tol = 1e-8 if prec == g.GDR_PREC_FP64 else (1e-7 if kappa > 1e5 else 3e-5)
    assert rel(host(y), y_ref) <= tol, rel(host(y), y_ref)
    assert np.linalg.norm(host(s)) <= (1 + 1e-8) * np.linalg.norm(s_ref)
    bound = tol * np.linalg.norm(Hh, 2) * np.linalg.norm(y_ref) + 1e-12 * np.linalg.norm(c)
    assert np.linalg.norm(host(s) - s_ref) <= bound, (np.linalg.norm(host(s) - s_ref), bound)
