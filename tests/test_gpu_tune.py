"""Launch shapes and the autotuner (runs on a GB300; -m gpu).

Every matvec launch shape the autotuner may choose is forced in turn through
gdr_op_set_shape and compared with the oracle's operator, so that whichever
shape a tuned solve runs with is covered by parity: the shapes only move the
same arithmetic around (the FP64 results agree with the oracle to rounding,
whatever the order of a CSR row's or the four directions' partial sums).
The column-pair form (packed FP32x2 arithmetic, complex64 only) is checked
the same way, against the oracle and, with bf16 links, against the one-column
form on the same operator.  Then gdr_autotune on a lattice where the persistent
sweep applies, a full solve with GDR_FLAG_AUTOTUNE checked by the oracle's
operator, and one with the pair form forced for every column count."""
import numpy as np
import pytest

import workloads as W
from oracle import CSROperator, WilsonOperator
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


# col_inner 2 / 3: column groups (ragged last group for 5 columns or 3 pairs)
WILSON_SHAPES = [(0, t, ci) for t in (64, 128, 256) for ci in (0, 1)] + [(1, 128, 0), (1, 128, 1),
                                                                         (0, 128, 2), (0, 64, 3), (1, 128, 2)]
PAIR_SHAPES = [(2, t, ci) for t in (64, 128) for ci in (0, 1, 2)]
CSR_SHAPES = [(tpr, t, ci) for tpr in (1, 2, 4, 8) for t in (128, 256) for ci in (0, 1)] + [(2, 128, 2)]


# 3x4x2x6: 144 sites, ragged last tile for every block size; 8x8x4x4 several tiles
@pytest.mark.parametrize("dims", [(3, 4, 2, 6), (8, 8, 4, 4)])
@pytest.mark.parametrize("ncol", [1, 5])
def test_wilson_every_shape(ctx, dims, ncol):
    links = W.su3_links(dims, 0.4, W.rng(41, 0))
    op_o = WilsonOperator(dims, links, diag_a=0.5)
    op = g.gdr_op_wilson(ctx, dims, dev(links), 0.5, g.GDR_LINK_C64)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((ncol, op_o.n)) + 1j * rng.standard_normal((ncol, op_o.n))
    sig = -1.0 / np.linspace(0.12, 0.13, ncol) + 0.01j
    ref = np.stack([op_o.matvec(X[c]) - sig[c] * X[c] for c in range(ncol)])
    X128, X64 = dev(X), dev(X, torch.complex64)
    for form, threads, ci in WILSON_SHAPES:
        for prec in (g.GDR_PREC_FP64, g.GDR_PREC_MIXED):
            g.gdr_op_set_shape(op, prec, ncol, form, threads, ci)
            assert g.gdr_op_get_shape(op, prec, ncol) == {"form": form, "threads": threads, "col_inner": ci}
        Y = torch.zeros((ncol, op_o.n), dtype=torch.complex128, device="cuda")
        g.gdr_op_apply(ctx, op, g.GDR_PREC_FP64, sig, X128, Y)
        Y32 = torch.zeros((ncol, op_o.n), dtype=torch.complex64, device="cuda")
        g.gdr_op_apply(ctx, op, g.GDR_PREC_MIXED, sig, X64, Y32)
        torch.cuda.synchronize()
        assert rel(host(Y), ref) < 1e-14, (form, threads, ci)
        assert rel(host(Y32), ref) < 1e-6, (form, threads, ci)
    g.gdr_op_destroy(op)


# ncol 1: a column paired with itself; 5: an odd last pair; 6: pairs only
@pytest.mark.parametrize("dims", [(3, 4, 2, 6), (8, 8, 4, 4)])
@pytest.mark.parametrize("ncol", [1, 5, 6])
def test_wilson_pair_shapes(ctx, dims, ncol):
    links = W.su3_links(dims, 0.4, W.rng(43, 0))
    op_o = WilsonOperator(dims, links, diag_a=0.5)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((ncol, op_o.n)) + 1j * rng.standard_normal((ncol, op_o.n))
    sig = -1.0 / np.linspace(0.12, 0.13, ncol) + 0.01j * np.arange(1, ncol + 1)
    ref = np.stack([op_o.matvec(X[c]) - sig[c] * X[c] for c in range(ncol)])
    X64 = dev(X, torch.complex64)
    for store in (g.GDR_LINK_C64, g.GDR_LINK_BF16):
        op = g.gdr_op_wilson(ctx, dims, dev(links), 0.5, store)
        g.gdr_op_set_shape(op, g.GDR_PREC_MIXED, ncol, 0, 128, 0)
        Y1 = torch.zeros((ncol, op_o.n), dtype=torch.complex64, device="cuda")
        g.gdr_op_apply(ctx, op, g.GDR_PREC_MIXED, sig, X64, Y1)      # one column per thread
        for form, threads, ci in PAIR_SHAPES:
            g.gdr_op_set_shape(op, g.GDR_PREC_MIXED, ncol, form, threads, ci)
            assert g.gdr_op_get_shape(op, g.GDR_PREC_MIXED, ncol) == {"form": form, "threads": threads,
                                                                      "col_inner": ci}
            Y = torch.full((ncol, op_o.n), 7.0 + 7.0j, dtype=torch.complex64, device="cuda")  # all entries written
            g.gdr_op_apply(ctx, op, g.GDR_PREC_MIXED, sig, X64, Y)
            torch.cuda.synchronize()
            if store == g.GDR_LINK_C64:
                assert rel(host(Y), ref) < 1e-6, (form, threads, ci)
            assert rel(host(Y), host(Y1)) < 1e-6, (store, form, threads, ci)
        g.gdr_op_destroy(op)


def test_solve_with_pair_forms(ctx):
    """Every complex64 matvec of a mixed solve in a pair form (forced for each column
    count the solve uses: the nearest set count within 2x applies), including the
    stages that scale or subtract from a right-hand side."""
    p = W.wilson_problem(2, dims=(8, 8, 8, 8), eps=0.3, nshift=4, nrhs=3, m=24, k=10, m_proj=14,
                         kappa_c=0.1325)
    dims, diag_a, links = p.op[1], p.op[2], p.op[3]
    op_o = WilsonOperator(dims, links, diag_a=diag_a)
    for form in (2,):
        op = g.gdr_op_wilson(ctx, dims, dev(links), diag_a, g.GDR_LINK_BF16)
        for nc in (1, 2, 4, 8, 16, 32, 64, 128):
            g.gdr_op_set_shape(op, g.GDR_PREC_MIXED, nc, form, 128, nc % 2)
        params = g.gdr_params_default(m=p.m, k=p.k, m_proj=p.m_proj, tol=1e-8, prec=g.GDR_PREC_MIXED,
                                      flags=g.GDR_FLAG_NO_SWEEP)
        nrhs = p.B.shape[1]
        X = torch.zeros((nrhs, len(p.sigma), p.n), dtype=torch.complex128, device="cuda")
        st, rep, _ = g.gdr_solve_multishift(ctx, op, p.sigma, dev(np.ascontiguousarray(p.B.T)), X, params)
        assert st == g.GDR_OK, rep
        Xh = host(X)
        for j in range(nrhs):
            b = p.B[:, j]
            for i, s in enumerate(p.sigma):
                x = Xh[j, i]
                assert np.linalg.norm(b - (op_o.matvec(x) - s * x)) / np.linalg.norm(b) <= 1.05e-8, (form, j, i)
        g.gdr_op_destroy(op)


@pytest.mark.parametrize("ncol", [1, 3])
def test_csr_every_shape(ctx, ncol):
    # 5-point rows (and the bidiagonal's 1-2 entries): rows shorter than TPR
    for rowptr, col, vals in (W.convdiff_csr(37, 12.0, -7.0, 0.3), W.config(1).op[1:]):
        A = CSROperator(rowptr, col, vals)
        op = g.gdr_op_csr(ctx, dev(rowptr), dev(col), dev(vals))
        rng = np.random.default_rng(6)
        X = rng.standard_normal((ncol, A.n)) + 1j * rng.standard_normal((ncol, A.n))
        sig = np.linspace(0.5, -1.0, ncol) + 0.25j
        ref = np.stack([A.matvec(X[c]) - sig[c] * X[c] for c in range(ncol)])
        X128, X64 = dev(X), dev(X, torch.complex64)
        for tpr, threads, ci in CSR_SHAPES:
            for prec in (g.GDR_PREC_FP64, g.GDR_PREC_MIXED):
                g.gdr_op_set_shape(op, prec, ncol, tpr, threads, ci)
            Y = torch.zeros((ncol, A.n), dtype=torch.complex128, device="cuda")
            g.gdr_op_apply(ctx, op, g.GDR_PREC_FP64, sig, X128, Y)
            Y32 = torch.zeros((ncol, A.n), dtype=torch.complex64, device="cuda")
            g.gdr_op_apply(ctx, op, g.GDR_PREC_MIXED, sig, X64, Y32)
            torch.cuda.synchronize()
            assert rel(host(Y), ref) < 1e-14, (tpr, threads, ci)
            assert rel(host(Y32), ref) < 1e-6, (tpr, threads, ci)
        g.gdr_op_destroy(op)


def test_csr_batch_every_shape(ctx):
    probs = [W.config(5)[i] for i in (0, 1, 2)]  # uneven sizes
    op = g.make_batch_operator(ctx, probs)
    nmax = max(p.n for p in probs)
    rng = np.random.default_rng(7)
    X = np.zeros((3, nmax), dtype=complex)
    for c, p in enumerate(probs):
        X[c, :p.n] = rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)
    sig = np.array([1.0, 0.1, 0.5])
    refs = [CSROperator(*p.op[1:]).matvec(X[c, :p.n]) - sig[c] * X[c, :p.n] for c, p in enumerate(probs)]
    for tpr, threads, ci in CSR_SHAPES:
        g.gdr_op_set_shape(op, g.GDR_PREC_FP64, 3, tpr, threads, ci)
        Y = torch.zeros((3, nmax), dtype=torch.complex128, device="cuda")
        g.gdr_op_apply(ctx, op, g.GDR_PREC_FP64, sig, dev(X), Y)
        torch.cuda.synchronize()
        Yh = host(Y)
        for c, p in enumerate(probs):
            assert rel(Yh[c, :p.n], refs[c]) < 1e-14, (tpr, threads, ci, c)
    g.gdr_op_destroy(op)


def test_set_shape_rejects_bad_shapes(ctx):
    links = W.su3_links((2, 2, 2, 2), 0.3, W.rng(42, 0))
    op = g.gdr_op_wilson(ctx, (2, 2, 2, 2), dev(links), 0.0, g.GDR_LINK_C64)
    for form, threads in ((1, 256), (2, 128), (0, 96), (3, 128)):
        with pytest.raises(g.GdrError):
            g.gdr_op_set_shape(op, g.GDR_PREC_FP64, 1, form, threads, 0)
    for form, threads in ((2, 256), (3, 64)):   # pairs: complex64, 64 or 128 threads
        with pytest.raises(g.GdrError):
            g.gdr_op_set_shape(op, g.GDR_PREC_MIXED, 2, form, threads, 0)
    g.gdr_op_set_shape(op, g.GDR_PREC_FP64, 4, 0, 256, 1)
    assert g.gdr_op_get_shape(op, g.GDR_PREC_FP64, 8)["threads"] == 256   # nearest count within 2x
    assert g.gdr_op_get_shape(op, g.GDR_PREC_FP64, 9)["form"] == 1        # beyond: default (tiny lattice)
    g.gdr_op_set_shape(op, g.GDR_PREC_FP64, 0)                            # forget all
    assert g.gdr_op_get_shape(op, g.GDR_PREC_FP64, 1)["col_inner"] == 0   # defaults: one column
    assert g.gdr_op_get_shape(op, g.GDR_PREC_FP64, 4)["col_inner"] == 1   # several: column-inner order
    with pytest.raises(g.GdrError):
        g.gdr_op_set_shape(op, g.GDR_PREC_FP64, 4, 0, 128, -1)             # no negative column order
    with pytest.raises(g.GdrError):
        g.gdr_autotune(ctx, op, g.GDR_PREC_FP64, 0)
    g.gdr_op_destroy(op)


def test_autotune_wilson_and_tuned_solve(ctx):
    p = W.wilson_problem(2, dims=(8, 8, 8, 8), eps=0.3, nshift=4, nrhs=1, m=24, k=10, m_proj=14,
                         rhs="gaussian", kappa_c=0.1325)
    dims, diag_a, links = p.op[1], p.op[2], p.op[3]
    op = g.gdr_op_wilson(ctx, dims, dev(links), diag_a, g.GDR_LINK_C64)
    r = g.gdr_autotune(ctx, op, g.GDR_PREC_MIXED, 1, p.m)
    assert r["candidates"] == 4 and r["mv_ms"] > 0 and r["mv_ms"] <= r["mv_ms_default"] * 1.0001
    assert r["sweep"] in (0, 1) and r["cycle_ms_sweep"] > 0 and r["cycle_ms_launch"] > 0
    best = g.gdr_op_get_shape(op, g.GDR_PREC_MIXED, 1)
    assert best == r["best"]
    r6 = g.gdr_autotune(ctx, op, g.GDR_PREC_FP64, 6, 0)
    assert r6["candidates"] == 8 and r6["sweep"] == -1
    # a solve with whatever was chosen (and the flag, which tunes what is still missing),
    # checked by the oracle's operator and against a solve with the default shapes
    op_o = WilsonOperator(dims, links, diag_a=diag_a)

    def solve(flags):
        params = g.gdr_params_default(m=p.m, k=p.k, m_proj=p.m_proj, tol=1e-8, prec=g.GDR_PREC_MIXED, flags=flags)
        X = torch.zeros((1, len(p.sigma), p.n), dtype=torch.complex128, device="cuda")
        st, rep, _ = g.gdr_solve_multishift(ctx, op, p.sigma, dev(p.B.T.copy()), X, params)
        assert st == g.GDR_OK
        return host(X)[0]

    Xt = solve(g.GDR_FLAG_AUTOTUNE)
    b = p.B[:, 0]
    for i, s in enumerate(p.sigma):
        assert np.linalg.norm(b - (op_o.matvec(Xt[i]) - s * Xt[i])) / np.linalg.norm(b) <= 1.05e-8
    g.gdr_op_set_shape(op, g.GDR_PREC_FP64, 0)   # forget every tuned choice
    Xd = solve(0)
    assert rel(Xt, Xd) < 1e-6
    g.gdr_op_destroy(op)


def test_autotune_batch(ctx):
    probs = [W.config(5)[i] for i in range(4)]
    op = g.make_batch_operator(ctx, probs)
    r = g.gdr_autotune(ctx, op, g.GDR_PREC_MIXED, 4, 30)
    assert r["candidates"] == 16 and r["sweep"] in (0, 1)
    r = g.gdr_autotune(ctx, op, g.GDR_PREC_FP64, 16, 0)   # 4 columns per problem
    assert r["candidates"] == 16
    with pytest.raises(g.GdrError):
        g.gdr_autotune(ctx, op, g.GDR_PREC_FP64, 6, 0)    # not a multiple of the problem count
    g.gdr_op_destroy(op)
