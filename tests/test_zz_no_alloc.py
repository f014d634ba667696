"""The allocation-free GMRES-Sh reduced solve gives the same results as the
allocating entry point (-m gpu).

gdr_dense_gmres_sh_noalloc serves callers that cannot let the library
allocate device memory; it keeps its workspace in one fixed device array.
Two calls in a row with different inputs check that nothing left over from
the previous call leaks into the next one.  This file sorts last so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import workloads as W
from oracle import CSROperator, gmres_dr_sh

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_0707_0502_gb300 as g  # noqa: E402


def _inputs():
    p = W.config(1)
    A = CSROperator(*p.op[1:])
    hist = gmres_dr_sh(A.matvec, p.B[:, 0], p.sigma, p.m, p.k, 1e-14, max_cycles=2, record=True)["history"]
    return p, hist


def _run(fn, ctx, m, sigma, Hbar, c, beta):
    ns = len(sigma)
    D = torch.zeros((ns, m), dtype=torch.complex128, device="cuda")
    s = torch.zeros(m + 1, dtype=torch.complex128, device="cuda")
    bn = torch.zeros(ns, dtype=torch.complex128, device="cuda")
    nr = torch.zeros(ns, dtype=torch.float64, device="cuda")
    fn(ctx, m, sigma, torch.as_tensor(Hbar.T.copy()).cuda(), torch.as_tensor(c).cuda(),
       torch.as_tensor(beta).cuda(), D, s, bn, nr)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (D, s, bn, nr)]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_noalloc_matches_allocating_entry_point():
    import __graft_entry__
    __graft_entry__.build()
    ctx = g.gdr_create(0)
    try:
        p, hist = _inputs()
        calls = [(hist[1], p.sigma, np.array([1.0, 0.8 - 0.3j, 1.7j, -0.4])),
                 (hist[0], p.sigma[:3], np.array([1.0, -2.0 + 0.5j, 0.3j]))]
        for h, sig, beta in calls:            # two calls in a row, different sizes and inputs
            Hbar, c = h["Hbar"], h["c"]
            m = Hbar.shape[1]
            ref = _run(g.gdr_dense_gmres_sh, ctx, m, sig, Hbar, c, beta)
            out = _run(g.gdr_dense_gmres_sh_noalloc, ctx, m, sig, Hbar, c, beta)
            for a, b in zip(out, ref):
                assert rel(a, b) < 1e-10
        with pytest.raises(g.GdrError) as e:
            h = hist[0]
            _run(g.gdr_dense_gmres_sh_noalloc, ctx, h["Hbar"].shape[1], np.zeros(17), h["Hbar"], h["c"],
                 np.ones(17, complex))
        assert e.value.status == g.GDR_EINVAL and "GDR_NOALLOC_MAX_NS" in str(e.value)
    finally:
        g.gdr_destroy(ctx)
