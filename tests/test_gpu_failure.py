"""Failure detection without a GPU fault (-m gpu): every failure is made on the
host side or by a bounded wait, and the library reports it as a status with the
context still usable afterwards."""
import time

import numpy as np
import pytest

import workloads as W

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


def _small_solve(ctx, p, prm, B=None):
    op = g.make_operator(ctx, p)
    Bt = torch.as_tensor(np.ascontiguousarray((p.B if B is None else B).T)).cuda()
    X = torch.zeros((p.B.shape[1], len(p.sigma), p.n), dtype=torch.complex128, device="cuda")
    try:
        return g.gdr_solve_multishift(ctx, op, p.sigma, Bt, X, prm)
    finally:
        g.gdr_op_destroy(op)


def test_grid_barrier_completes(ctx):
    assert g.gdr_barrier_selftest(ctx, 2000, 0) == g.GDR_OK


def test_grid_barrier_times_out_and_context_survives(ctx):
    """A barrier that waits for a block that does not exist ends by its spin
    bound: GDR_ETIMEOUT after about a second, then the context still solves."""
    t0 = time.perf_counter()
    st = g.gdr_barrier_selftest(ctx, 3, 1)
    dt = time.perf_counter() - t0
    assert st == g.GDR_ETIMEOUT
    assert 0.05 < dt < 30.0, dt
    p = W.config(1)
    prm = g.gdr_params_default(m=p.m, k=p.k, tol=1e-8, prec=g.GDR_PREC_FP64)
    st, rep, _ = _small_solve(ctx, p, prm)
    assert st == g.GDR_OK and rep["max_relres"] <= 1e-8


def test_nan_rhs_reports_enan(ctx):
    p = W.config(1)
    B = p.B.copy()
    B[17, 0] = np.nan
    prm = g.gdr_params_default(m=p.m, k=p.k, tol=1e-8, prec=g.GDR_PREC_MIXED)
    with pytest.raises(g.GdrError) as e:
        _small_solve(ctx, p, prm, B)
    assert e.value.status == g.GDR_ENAN
    st, rep, _ = _small_solve(ctx, p, prm)  # the context is still usable
    assert st == g.GDR_OK


def test_cycle_cap_reports_enoconv(ctx):
    """One GMRES-DR cycle, no refinement: the bidiagonal problem needs ~10, so the
    solve stops with GDR_ENOCONV and reports the residual it reached."""
    p = W.config(1)
    prm = g.gdr_params_default(m=p.m, k=p.k, tol=1e-8, prec=g.GDR_PREC_FP64, max_cycles=1,
                               flags=g.GDR_FLAG_NO_REFINE)
    st, rep, _ = _small_solve(ctx, p, prm)
    assert st == g.GDR_ENOCONV
    assert rep["cycles_rhs1"] == 1 and rep["max_relres"] > 1e-8


def test_invalid_arguments_are_einval(ctx):
    p = W.config(1)
    prm = g.gdr_params_default(m=0, k=0, tol=1e-8, prec=g.GDR_PREC_FP64)
    with pytest.raises(g.GdrError) as e:
        _small_solve(ctx, p, prm)
    assert e.value.status == g.GDR_EINVAL
    prm = g.gdr_params_default(m=p.m, k=p.k, tol=1e-8, prec=g.GDR_PREC_FP64, m_refine=g.GDR_MAX_M + 1)
    with pytest.raises(g.GdrError) as e:
        _small_solve(ctx, p, prm)
    assert e.value.status == g.GDR_EINVAL
    assert g.gdr_barrier_selftest(ctx, 0, 0) == g.GDR_EINVAL
