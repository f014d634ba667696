"""End-to-end parity of the CUDA solves with the oracle (-m gpu).

Bars (from the solver's target): every (shift, rhs) pair reaches a true FP64
relative residual <= 1e-8 (computed here by the ORACLE's operator on the
returned X); solutions agree with the oracle's to <= 1e-6 relative (MIXED)
and the all-FP64 path agrees with the oracle at a matched cycle count to
<= 1e-10."""
import numpy as np
import pytest

import workloads as W
from oracle import CSROperator, gmres_dr_sh, solve_all_rhs
from tests.gpu_util import dev, host, small_wilson

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


def solve(ctx, op, sigma, B, prec, m, k, tol=1e-8, nrhs=None, **kw):
    B = np.atleast_2d(B.T).copy() if B.ndim == 2 else B[None, :].copy()
    nr = B.shape[0]
    X = torch.zeros((nr, len(sigma), B.shape[1]), dtype=torch.complex128, device="cuda")
    prm = g.gdr_params_default(m=m, k=k, tol=tol, prec=prec, **kw)
    st, rep, _ = g.gdr_solve_multishift(ctx, op, sigma, dev(B), X, prm)
    return st, rep, host(X)


def relres(matvec, b, s, x):
    return np.linalg.norm(b - (matvec(x) - s * x)) / np.linalg.norm(b)


@pytest.mark.parametrize("sweep", [True, False])
def test_config1_matched_cycles_fp64(ctx, sweep):
    """All-FP64 GPU path = oracle to 1e-10 after the same number of cycles, with the
    persistent Arnoldi sweep and with one launch per Arnoldi phase."""
    p = W.config(1)
    A = CSROperator(*p.op[1:])
    op = g.make_operator(ctx, p)
    extra = 0 if sweep else g.GDR_FLAG_NO_SWEEP
    for cycles in (1, 2, 5):
        ref = gmres_dr_sh(A.matvec, p.B[:, 0], p.sigma, p.m, p.k, 1e-30, max_cycles=cycles)
        st, rep, X = solve(ctx, op, p.sigma, p.B, g.GDR_PREC_FP64, p.m, p.k, tol=1e-30, max_cycles=cycles,
                           flags=g.GDR_FLAG_NO_PROJ | g.GDR_FLAG_NO_REFINE | extra)
        assert rep["cycles_rhs1"] == cycles and rep["mvps_rhs1"] == ref["mvps"]
        for i in range(len(p.sigma)):
            e = np.linalg.norm(X[0, i] - ref["x"][:, i]) / np.linalg.norm(ref["x"][:, i])
            assert e < 1e-10, (cycles, i, e)
    g.gdr_op_destroy(op)


@pytest.mark.parametrize("prec", [g.GDR_PREC_FP64, g.GDR_PREC_MIXED])
def test_config1_converged(ctx, prec):
    p = W.config(1)
    A = CSROperator(*p.op[1:])
    op = g.make_operator(ctx, p)
    ref = gmres_dr_sh(A.matvec, p.B[:, 0], p.sigma, p.m, p.k, 1e-12)
    st, rep, X = solve(ctx, op, p.sigma, p.B, prec, p.m, p.k)
    assert st == g.GDR_OK, rep
    for i, s in enumerate(p.sigma):
        assert relres(A.matvec, p.B[:, 0], s, X[0, i]) <= 1e-8
        assert np.linalg.norm(X[0, i] - ref["x"][:, i]) <= 1e-6 * np.linalg.norm(ref["x"][:, i])
    if prec == g.GDR_PREC_FP64:
        assert rep["mvps_rhs1"] == gmres_dr_sh(A.matvec, p.B[:, 0], p.sigma, p.m, p.k, 1e-8)["mvps"]
    g.gdr_op_destroy(op)


def test_graph_and_direct_launch_identical(ctx):
    p = W.config(1)
    op = g.make_operator(ctx, p)
    _, _, X1 = solve(ctx, op, p.sigma, p.B, g.GDR_PREC_FP64, p.m, p.k)
    _, _, X2 = solve(ctx, op, p.sigma, p.B, g.GDR_PREC_FP64, p.m, p.k, flags=g.GDR_FLAG_NO_GRAPH)
    assert np.array_equal(X1, X2)
    g.gdr_op_destroy(op)


def test_lucky_breakdown(ctx):
    p = W.config(1)
    op = g.make_operator(ctx, p)
    b = np.zeros((p.n, 1), dtype=complex)
    b[0] = 1
    st, rep, X = solve(ctx, op, p.sigma, b, g.GDR_PREC_FP64, p.m, p.k)
    assert st == g.GDR_OK and rep["mvps_rhs1"] == 1
    for i, s in enumerate(p.sigma):
        assert np.allclose(X[0, i], b[:, 0] / (1 - s), atol=1e-14)
    g.gdr_op_destroy(op)


@pytest.fixture(scope="module")
def wil():
    return small_wilson((4, 4, 4, 4), 0.3, cid=21, nshift=4, nrhs=3)


@pytest.mark.parametrize("prec", [g.GDR_PREC_FP64, g.GDR_PREC_MIXED])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_wilson_multishift_multirhs(ctx, wil, prec, nrhs):
    p, A = wil
    B = p.B[:, :nrhs]
    op = g.make_operator(ctx, p)
    ref = solve_all_rhs(A.matvec, B, p.sigma, p.m, p.k, p.m_proj, 1e-12, 1e-6)
    st, rep, X = solve(ctx, op, p.sigma, B, prec, p.m, p.k, m_proj=p.m_proj)
    assert st == g.GDR_OK, rep
    for j in range(nrhs):
        for i, s in enumerate(p.sigma):
            assert relres(A.matvec, B[:, j], s, X[j, i]) <= 1e-8, (i, j)
            xr = ref["X"][:, i, j]
            assert np.linalg.norm(X[j, i] - xr) <= 1e-6 * np.linalg.norm(xr), (i, j)
    g.gdr_op_destroy(op)


@pytest.mark.parametrize("prec", [g.GDR_PREC_FP64, g.GDR_PREC_MIXED])
def test_wilson16_long_vectors(ctx, prec):
    """16^4 lattice (786,432 unknowns): long vectors, so the Arnoldi step runs its
    separate update / dot passes once the basis outgrows L2.  2 shifts, GMRES-DR(30,10);
    true residuals by the oracle's operator."""
    from oracle import WilsonOperator
    dims = (16, 16, 16, 16)
    links = W.su3_links(dims, 0.4, W.rng(3, 0))
    A = WilsonOperator(dims, links, diag_a=0.0)
    kc = W.load_kappa_c()["cfg3:16x16x16x16:eps0.4"]
    sigma = np.array([-1.0 / (0.9 * kc), -1.0 / 0.12], complex)
    b = W.gaussian_complex(W.rng(3, 7), A.n, 1)[:, 0]
    op = g.gdr_op_wilson(ctx, dims, torch.as_tensor(links).cuda(), 0.0, g.GDR_LINK_C64)
    st, rep, X = solve(ctx, op, sigma, b, prec, 30, 10)
    assert st == g.GDR_OK, rep
    for i, s in enumerate(sigma):
        assert relres(A.matvec, b, s, X[0, i]) <= 1e-8, (i, rep)
    g.gdr_op_destroy(op)


def test_deflation_saves_matvecs_example7_shape(ctx):
    """The comparison of Example 7 (Sec. 4) on the synthetic 8^4 Wilson operator and its
    six kappa shifts: the second right-hand side by GMRES(20)-Proj(20)-Sh over the kept
    eigenvectors needs fewer matvecs than plain GMRES(20)-Sh, and the first by
    GMRES-DR(40,20)-Sh fewer than GMRES(40)-Sh; all pairs still reach 1e-8 (FP64).  The
    near-unit synthetic links give a spectrum without the few isolated small eigenvalues
    of the paper's QCD matrix, so the saving is far below its 2680 -> 280 (measured
    here: 240 -> 220)."""
    p = W.config(2)
    B = np.concatenate([p.B, W.gaussian_complex(W.rng(2, 9), p.n, 1)], axis=1)
    op = g.make_operator(ctx, p)
    common = dict(m_proj=20, flags=g.GDR_FLAG_SEQUENTIAL)
    st, dr, _ = solve(ctx, op, p.sigma, B, g.GDR_PREC_FP64, 40, 20, **common)
    assert st == g.GDR_OK and dr["max_relres"] <= 1e-8
    common["flags"] |= g.GDR_FLAG_NO_PROJ
    st, plain, _ = solve(ctx, op, p.sigma, B, g.GDR_PREC_FP64, 40, 20, **common)
    assert st == g.GDR_OK and plain["max_relres"] <= 1e-8
    st, g40, _ = solve(ctx, op, p.sigma, B[:, :1], g.GDR_PREC_FP64, 40, 0, flags=g.GDR_FLAG_SEQUENTIAL)
    assert st == g.GDR_OK and g40["max_relres"] <= 1e-8
    # right-hand side 2: deflated projection vs none (paper: 280 vs 2680 mvps on its QCD matrix)
    assert dr["mvps_proj"] < plain["mvps_proj"], (dr["mvps_proj"], plain["mvps_proj"])
    # right-hand side 1: deflated restarting vs plain restarting
    assert dr["mvps_rhs1"] < g40["mvps_rhs1"], (dr["mvps_rhs1"], g40["mvps_rhs1"])
    g.gdr_op_destroy(op)


@pytest.mark.parametrize("prec", [g.GDR_PREC_FP64, g.GDR_PREC_MIXED])
def test_projection_large_k(ctx, prec):
    """A kept pair of k = 76 (m = 84, near the largest pair the dense kernels take): the
    projection operators of GMRES-Proj-Sh come from Gauss-Jordan on a 76 x 153 system in
    shared memory.  Every (shift, rhs) pair reaches 1e-8 and matches the oracle's
    GMRES-DR-Sh + GMRES-Proj-Sh solution."""
    rowptr, col, vals = W.paper_example1_matrix()
    A = CSROperator(rowptr, col, vals)
    op = g.gdr_op_csr(ctx, dev(rowptr), dev(col), dev(vals))
    sig = np.array([0, -0.4, -2], complex)
    gen = np.random.default_rng([41, 0])
    B = gen.standard_normal((1000, 3)).astype(complex)
    st, rep, X = solve(ctx, op, sig, B, prec, 84, 76, tol=1e-8, m_proj=8)
    assert st == g.GDR_OK, rep
    assert rep["mvps_rhs1"] > 84 and rep["mvps_proj"] > 0  # restarted: the kept pair exists
    ref = solve_all_rhs(A.matvec, B, sig, 84, 76, 8, 1e-12, 1e-6)
    for j in range(3):
        for i, s in enumerate(sig):
            assert relres(A.matvec, B[:, j], s, X[j, i]) <= 1e-8, (i, j)
            xr = ref["X"][:, i, j]
            assert np.linalg.norm(X[j, i] - xr) <= 1e-6 * np.linalg.norm(xr), (i, j)
    g.gdr_op_destroy(op)
