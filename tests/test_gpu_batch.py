"""Batch of independent shifted problems (-m gpu): every problem of a ragged
CSR batch is solved as one column of a batched GMRES-DR(m,k)-Sh cycle.

Bars: each (problem, shift) pair reaches a true FP64 relative residual
<= 1e-8 computed by the oracle's operator; on the small batch the solutions
agree with the oracle's per-problem GMRES-DR-Sh to <= 1e-6 relative."""
import numpy as np
import pytest

import workloads as W
from oracle import CSROperator, gmres_dr_sh

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


def _small_batch():
    gen = np.random.default_rng([55, 2])
    probs = []
    for s in (7, 9, 13, 20, 33):                      # n = 49 .. 1089, odd and even
        cx, cy = gen.uniform(-20, 20, 2)
        rowptr, col, vals = W.convdiff_csr(s, cx, cy, gen.uniform(0, 0.5))
        b = W.gaussian_complex(gen, s * s, 1)
        probs.append(W.Problem(name=f"cd{s}", op=("csr", rowptr, col, vals), n=s * s,
                               sigma=np.array([1.0, 0.0, 0.1, 0.5], complex), B=b, m=20, k=6, m_proj=14))
    return probs


def _solve(ctx, probs, prec):
    op = g.make_batch_operator(ctx, probs)
    ns = len(probs[0].sigma)
    sig = np.stack([p.sigma for p in probs])
    B = torch.as_tensor(np.concatenate([p.B[:, 0] for p in probs])).cuda()
    X = torch.zeros(sum(p.n for p in probs) * ns, dtype=torch.complex128, device="cuda")
    prm = g.gdr_params_default(m=probs[0].m, k=probs[0].k, m_proj=probs[0].m_proj, tol=1e-8, prec=prec)
    st, rep, per = g.gdr_solve_batch(ctx, op, sig, B, X, prm)
    g.gdr_op_destroy(op)
    Xh = X.cpu().numpy()
    out, off = [], 0
    for p in probs:
        out.append(Xh[off * ns:(off + p.n) * ns].reshape(ns, p.n))
        off += p.n
    return st, rep, per, out


@pytest.mark.parametrize("prec", [g.GDR_PREC_FP64, g.GDR_PREC_MIXED])
def test_small_ragged_batch(ctx, prec):
    probs = _small_batch()
    st, rep, per, X = _solve(ctx, probs, prec)
    assert st == g.GDR_OK and (per == 0).all(), (rep, per)
    for p, x in zip(probs, X):
        A = CSROperator(*p.op[1:])
        ref = gmres_dr_sh(A.matvec, p.B[:, 0], p.sigma, p.m, p.k, 1e-12)
        for i, s in enumerate(p.sigma):
            r = p.B[:, 0] - (A.matvec(x[i]) - s * x[i])
            assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(p.B[:, 0]), (p.name, i)
            assert np.linalg.norm(x[i] - ref["x"][:, i]) <= 1e-6 * np.linalg.norm(ref["x"][:, i]), (p.name, i)


def test_config5_full_batch(ctx):
    """64 convection-diffusion problems, sides 32..256 (1K-65K unknowns), 4 shifts,
    GMRES-DR(30,10), complex64 with FP64 refinement, one batch."""
    probs = W.config(5)
    st, rep, per, X = _solve(ctx, probs, g.GDR_PREC_MIXED)
    assert st == g.GDR_OK and (per == 0).all(), (rep, per)
    worst = 0.0
    for p, x in zip(probs, X):
        A = CSROperator(*p.op[1:])
        for i, s in enumerate(p.sigma):
            r = p.B[:, 0] - (A.matvec(x[i]) - s * x[i])
            worst = max(worst, np.linalg.norm(r) / np.linalg.norm(p.B[:, 0]))
    assert worst <= 1e-8, worst
