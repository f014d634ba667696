"""Related right-hand sides (Sec. 5, Example 8) on the GPU (-m gpu).

Right-hand sides b^j = b^1 + 1e-4 u^j (Example 8's recipe, complex Gaussian u^j)
on a small Wilson lattice with four kappa shifts.  With GDR_FLAG_RELATED_RHS each
right-hand side after the first starts from the Minres projection over the
previous solutions (B^H B d = B^H b^j, x_i = X_i d, common residual b^j - B d):
the size of that residual matches the oracle's least-squares projection, every
(shift, rhs) pair reaches the FP64 residual 1e-8 and the oracle pipeline's
solution, and the later right-hand sides need fewer matvecs than without the
projection (the paper reports about half)."""
import numpy as np
import pytest

import workloads as W
from oracle import related_rhs_projection, solve_all_rhs
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


@pytest.fixture(scope="module")
def related():
    p, A = small_wilson((4, 4, 4, 4), 0.3, cid=21, nshift=4, nrhs=1)
    U = W.gaussian_complex(W.rng(21, 8), p.n, 4)
    B = np.concatenate([p.B, p.B + 1e-4 * U], axis=1)  # 5 right-hand sides
    ref = solve_all_rhs(A.matvec, B, p.sigma, p.m, p.k, p.m_proj, 1e-12, 1e-6)
    # the oracle's projected residual of every b^j over b^1..b^{j-1}
    rel = 0.0
    for j in range(1, B.shape[1]):
        _, r, _ = related_rhs_projection(B[:, :j], np.zeros((p.n, len(p.sigma), j), complex), B[:, j])
        rel = max(rel, np.linalg.norm(r) / np.linalg.norm(B[:, j]))
    return p, A, B, ref, rel


def run(ctx, op, p, B, prec, flags):
    X = torch.zeros((B.shape[1], len(p.sigma), p.n), dtype=torch.complex128, device="cuda")
    prm = g.gdr_params_default(m=p.m, k=p.k, m_proj=p.m_proj, tol=1e-8, prec=prec, flags=flags)
    st, rep, _ = g.gdr_solve_multishift(ctx, op, p.sigma, dev(B.T.copy()), X, prm)
    return st, rep, host(X)


@pytest.mark.parametrize("prec", [g.GDR_PREC_FP64, g.GDR_PREC_MIXED])
def test_related_rhs_example8_shape(ctx, related, prec):
    p, A, B, ref, rel_oracle = related
    op = g.make_operator(ctx, p)
    st, rep, X = run(ctx, op, p, B, prec, g.GDR_FLAG_RELATED_RHS)
    assert st == g.GDR_OK, rep
    for j in range(B.shape[1]):
        for i, s in enumerate(p.sigma):
            b = B[:, j]
            assert np.linalg.norm(b - (A.matvec(X[j, i]) - s * X[j, i])) <= 1e-8 * np.linalg.norm(b), (i, j)
            xr = ref["X"][:, i, j]
            assert np.linalg.norm(X[j, i] - xr) <= 1e-6 * np.linalg.norm(xr), (i, j)
    # the projection's residual (FP64 normal equations) against the oracle's least squares
    assert rel_oracle < 1e-3
    assert abs(rep["related_resid"] - rel_oracle) <= 1e-6 * rel_oracle, (rep["related_resid"], rel_oracle)
    # fewer matvecs for right-hand sides 2.. than the same pipeline without the projection
    st0, base, _ = run(ctx, op, p, B, prec, g.GDR_FLAG_SEQUENTIAL)
    assert st0 == g.GDR_OK
    later = rep["mvps_proj"] + rep["mvps_refine"]
    later0 = base["mvps_proj"] + base["mvps_refine"]
    assert later < later0, (rep, base)
    assert rep["mvps_rhs1"] == base["mvps_rhs1"]
    g.gdr_op_destroy(op)


def test_related_rhs_identical_rhs(ctx, related):
    """b^2 = b^1: the projection solves the second right-hand side exactly (common
    residual zero up to rounding), so no Proj stage runs for it."""
    p, A, _, _, _ = related
    B = np.concatenate([p.B, p.B], axis=1)
    op = g.make_operator(ctx, p)
    st, rep, X = run(ctx, op, p, B, g.GDR_PREC_FP64, g.GDR_FLAG_RELATED_RHS)
    assert st == g.GDR_OK, rep
    assert rep["related_resid"] < 1e-12
    assert rep["mvps_proj"] == 0
    assert np.allclose(X[1], X[0], rtol=0, atol=1e-12 * np.abs(X[0]).max())
    g.gdr_op_destroy(op)
