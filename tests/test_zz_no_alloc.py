"""The allocation-free GMRES-Sh reduced solve against the oracle's reduced
solve and against the allocating entry point (-m gpu).

gdr_dense_gmres_sh_noalloc serves callers that cannot let the library
allocate device memory; it keeps its workspace in one fixed device array.
Its outputs (D, s, beta_new, norms) are compared with the oracle's
gmres_sh_dense_step on the same recorded Hbar and c, to 1e-10 (FP64), and
with gdr_dense_gmres_sh.  Two calls in a row with different inputs check that
nothing left over from the previous call leaks into the next one; one call at
the documented limits (m = 96, ns = 16) and one past them (GDR_EINVAL).  This
file sorts last so that a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest

import workloads as W
from oracle import CSROperator, arnoldi_cgs2_step, gmres_dr_sh, gmres_sh_dense_step

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
        # a recurrence at the documented limits: 96 Arnoldi steps on the bidiagonal
        # matrix, 16 shifts
        A = CSROperator(*p.op[1:])
        m96 = g.GDR_NOALLOC_MAX_M
        V = np.zeros((p.n, m96 + 1), dtype=np.complex128)
        H96 = np.zeros((m96 + 1, m96), dtype=np.complex128)
        V[:, 0] = p.B[:, 0] / np.linalg.norm(p.B[:, 0])
        for j in range(m96):
            arnoldi_cgs2_step(A.matvec, V, H96, j)
        c96 = np.zeros(m96 + 1, dtype=np.complex128)
        c96[0] = np.linalg.norm(p.B[:, 0])
        sig16 = np.concatenate([p.sigma, -np.linspace(0.1, 30.0, 12) + 0.05j])
        beta16 = np.exp(0.3j * np.arange(16)) * np.linspace(1.0, 0.2, 16)
        calls.append(({"Hbar": H96, "c": c96}, sig16, beta16))
        for h, sig, beta in calls:            # calls in a row, different sizes and inputs
            Hbar, c = h["Hbar"], h["c"]
            m = Hbar.shape[1]
            out = _run(g.gdr_dense_gmres_sh_noalloc, ctx, m, sig, Hbar, c, beta)
            # the oracle's reduced solve on the same Hbar, c; s = c - Hhat d_1 is small
            # near convergence, so it is compared on the scale of c
            D, s, bn, nr = gmres_sh_dense_step(Hbar, c, np.asarray(sig), beta, np.ones(len(sig), bool))
            assert rel(out[0], D.T) < 1e-10, rel(out[0], D.T)
            assert np.linalg.norm(out[1] - s) < 1e-10 * np.linalg.norm(c)
            assert rel(out[2], bn) < 1e-10 and rel(out[3], nr) < 1e-10
            # and the allocating entry point
            ref = _run(g.gdr_dense_gmres_sh, ctx, m, sig, Hbar, c, beta)
            for a, b in zip(out, ref):
                assert rel(a, b) < 1e-10
        with pytest.raises(g.GdrError) as e:
            h = hist[0]
            _run(g.gdr_dense_gmres_sh_noalloc, ctx, h["Hbar"].shape[1], np.zeros(g.GDR_NOALLOC_MAX_NS + 1),
                 h["Hbar"], h["c"], np.ones(g.GDR_NOALLOC_MAX_NS + 1, complex))
        assert e.value.status == g.GDR_EINVAL and "GDR_NOALLOC_MAX_NS" in str(e.value)
    finally:
        g.gdr_destroy(ctx)
