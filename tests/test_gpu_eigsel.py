"""Projection over selected approximate eigenvectors (Sec. 4, Theorem 1, Example 4)
on the GPU (-m gpu), GDR_FLAG_EIG_SELECT.

Example 4's setting: the Example 1 matrix, shifts 0, -0.4, -2, the first right-hand
side by GMRES-DR(25,10)-Sh to 1e-10 and the second by GMRES(15)-Proj-Sh over the
first k approximate eigenvectors (no refinement, so the shifted systems show the
accuracy the eigenvectors allow).  The GPU's matvec count equals the oracle's on the
same inputs and lies within one cycle of Table 4.1; its largest eigen-residual
matches the oracle's; the non-base accuracy is far worse with all ten vectors than
with the four most accurate.  Then the full mixed-precision pipeline with the flag on
a Wilson problem: every pair reaches 1e-8 and the oracle's solution."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import CSROperator, gmres_dr_sh, gmres_proj_sh, kept_eigenpairs, solve_all_rhs
from tests.gpu_util import dev, host, small_wilson

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_0707_0502_gb300 as g  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))["table4_1"]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = g.gdr_create(0)
    yield c
    g.gdr_destroy(c)


def solve(ctx, op, sigma, B, prec, **kw):
    X = torch.zeros((B.shape[1], len(sigma), B.shape[0]), dtype=torch.complex128, device="cuda")
    prm = g.gdr_params_default(prec=prec, **kw)
    st, rep, _ = g.gdr_solve_multishift(ctx, op, sigma, dev(np.ascontiguousarray(B.T)), X, prm)
    return st, rep, host(X)


@pytest.mark.parametrize("ks", [10, 4])
def test_example4_on_gpu(ctx, ks):
    rowptr, col, vals = W.paper_example1_matrix()
    A = CSROperator(rowptr, col, vals)
    op = g.gdr_op_csr(ctx, dev(rowptr), dev(col), dev(vals))
    sig = np.array([0, -0.4, -2], complex)
    gen = np.random.default_rng([40, 0])
    b1 = gen.standard_normal(1000).astype(complex)
    b2 = gen.standard_normal(1000).astype(complex)
    B = np.stack([b1, b2], axis=1)
    st, rep, X = solve(ctx, op, sig, B, g.GDR_PREC_FP64, m=25, k=10, m_proj=15, tol=1e-10, k_select=ks,
                       flags=g.GDR_FLAG_EIG_SELECT | g.GDR_FLAG_NO_REFINE | g.GDR_FLAG_SEQUENTIAL)
    assert st in (g.GDR_OK, g.GDR_ENOCONV), rep
    # the oracle on the same inputs
    r1 = gmres_dr_sh(A.matvec, b1, sig, 25, 10, 1e-10)
    th, G, res = kept_eigenpairs(r1["Hk"], sig[0], ks)
    pr = gmres_proj_sh(A.matvec, r1["Vk1"], r1["Hk"], b2, sig, 15, 1e-10, max_mvps=3000, eig=(th, G))
    assert rep["mvps_rhs1"] == r1["mvps"] == 250
    assert rep["mvps_proj"] == pr["mvps"], (rep["mvps_proj"], pr["mvps"])
    mv = GOLD["mvps"][GOLD["k"].index(ks)]
    assert abs(rep["mvps_proj"] - mv) <= 15
    assert rep["mvps_extra"] == 0
    assert abs(rep["eig_resid_max"] - res.max()) <= 1e-4 * res.max(), (rep["eig_resid_max"], res.max())
    nb = np.linalg.norm(b2)
    rel = [np.linalg.norm(b2 - (A.matvec(X[1, i]) - s * X[1, i])) / nb for i, s in enumerate(sig)]
    assert rel[0] <= 1e-10
    worst = max(rel[1:])
    ref = max(np.linalg.norm(b2 - (A.matvec(pr["x"][:, i]) - s * pr["x"][:, i])) / nb for i, s in enumerate(sig)
              if i > 0)
    if ks == 10:
        assert worst > 1e-5 and ref > 1e-5, (worst, ref)     # limited by the inaccurate eigenvectors
    else:
        assert worst < 1e-7 and ref < 1e-7, (worst, ref)
    g.gdr_op_destroy(op)


@pytest.mark.parametrize("prec", [g.GDR_PREC_FP64, g.GDR_PREC_MIXED])
def test_eigsel_pipeline_wilson(ctx, prec):
    p, A = small_wilson((4, 4, 4, 4), 0.3, cid=21, nshift=4, nrhs=3)
    op = g.make_operator(ctx, p)
    st, rep, X = solve(ctx, op, p.sigma, p.B, prec, m=p.m, k=p.k, m_proj=p.m_proj, tol=1e-8,
                       flags=g.GDR_FLAG_EIG_SELECT)
    assert st == g.GDR_OK, rep
    assert rep["mvps_extra"] == 0 and rep["eig_resid_max"] > 0
    ref = solve_all_rhs(A.matvec, p.B, p.sigma, p.m, p.k, p.m_proj, 1e-12, 1e-6)
    for j in range(p.B.shape[1]):
        b = p.B[:, j]
        for i, s in enumerate(p.sigma):
            x = X[j, i]
            assert np.linalg.norm(b - (A.matvec(x) - s * x)) <= 1e-8 * np.linalg.norm(b), (i, j)
            xr = ref["X"][:, i, j]
            assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr), (i, j)
    g.gdr_op_destroy(op)
