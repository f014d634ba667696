"""Helpers shared by the GPU tests (marshalling between numpy and torch)."""
import numpy as np

import workloads as W
from oracle import WilsonOperator


def dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def small_wilson(dims=(4, 4, 4, 4), eps=0.3, cid=21, nshift=4, nrhs=1, seed_rhs=None):
    """A Wilson problem with kappa_c measured by the oracle (dense on tiny lattices)."""
    import scipy.sparse.linalg as spla
    links = W.su3_links(dims, eps, W.rng(cid, 0))
    op = WilsonOperator(dims, links)
    H = spla.LinearOperator((op.n, op.n), matvec=op.hop, dtype=np.complex128)
    lam = spla.eigs(H, k=4, which="LR", ncv=60, tol=1e-8, v0=np.ones(op.n, complex), return_eigenvectors=False)
    kc = 1.0 / lam.real.max()
    p = W.wilson_problem(cid, dims=dims, eps=eps, nshift=nshift, nrhs=nrhs, kappa_c=kc, m=30, k=12, m_proj=18)
    return p, op
