"""The projection dot C = V^H R on the tensor cores (runs on a GB300; -m gpu).

gdr_basis_dot forms c = V_{k+1}^H r of GMRES-Proj-Sh step 4 (Sec. 2.3) for many
columns at once.  For complex64 inputs with 8 or more columns it runs on the
tensor cores: TF32 inputs (10 fraction bits) and FP32 accumulation.  Each dot
is then bounded, element by element, by

    |C - C_exact| <= (2^-9 + 2n 2^-24) * sum_k |v_k| |r_k|

(two input roundings of at most 2^-10 relative each, and a worst-case FP32
accumulation over the 2n real products; the sum is over the real interleaved
components, the same for the real and the imaginary part).  The CUDA-core
form (FP32 products, FP64 sums) is held to 2^-22 of the same sum.  C_exact is
numpy's FP64 product of the same complex64 inputs.

Cases span ragged K stages (2n not a multiple of 32), one and two column tiles
(ncol up to 200: 128 columns per tile), basis sizes from 1 to 97 (the MMA has
128 rows, zero-filled above nv), a padded column stride, and the fallbacks (odd
n, fewer than 8 columns, the flag) that must give the CUDA-core result.  The
residual update (second half of the file) is checked the same way.  The kernel that ran is
read from the library's profiler."""
import numpy as np
import pytest

from tests.gpu_util import dev

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


def c64(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def run_dot(ctx, n, nv, ncol, ldr, seed, flags=0):
    rng = np.random.default_rng(seed)
    V = c64(rng, nv, n)             # row i = basis vector v_i (column-major n x nv)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    Rm = c64(rng, ncol, ldr)        # row c = column r_c, stride ldr
    Rm[:, :n] *= np.exp(rng.uniform(-3, 3, size=(ncol, 1))).astype(np.float32)  # column scales over ~6 decades
    Cd = torch.zeros((ncol, nv), dtype=torch.complex128, device="cuda")
    g.gdr_profile(ctx, True)
    g.gdr_basis_dot(ctx, g.GDR_PREC_MIXED, n, nv, dev(V), ncol, dev(Rm), ldr, Cd, flags)
    prof = g.gdr_profile_report(ctx)
    g.gdr_profile(ctx, False)
    R = Rm[:, :n]
    exact = np.conj(V.astype(np.complex128)) @ R.astype(np.complex128).T        # nv x ncol
    Vf = np.abs(V.view(np.float32)).astype(np.float64)                            # nv x 2n
    Rf = np.abs(R.view(np.float32)).astype(np.float64)                            # ncol x 2n
    S = Vf @ Rf.T
    return Cd.cpu().numpy().T, exact, S, prof


def tc_ran(prof):
    return prof.get("tc_proj_dot_c64", {}).get("launches", 0) > 0


@pytest.mark.parametrize("n,nv,ncol,ldr", [
    (3000, 21, 8, 3000),       # 2n = 6000: a ragged last K stage; fewest columns
    (5000, 21, 40, 5006),      # padded column stride
    (2048, 64, 130, 2048),     # two column tiles (65 + 65)
    (4000, 97, 120, 4000),     # the largest basis (m + 1 = 97 of the MMA's 128 rows)
    (1000, 1, 200, 1000),      # one basis vector, two tiles of 100
    (262144, 21, 120, 262144), # a long vector split over many CTAs
    (2000, 64, 300, 2002),     # three column tiles (112 wide), padded stride
])
def test_tensor_core_dot(ctx, n, nv, ncol, ldr):
    C, exact, S, prof = run_dot(ctx, n, nv, ncol, ldr, seed=n + nv + ncol)
    assert tc_ran(prof), prof
    bound = (2.0 ** -9 + 2 * n * 2.0 ** -24) * S
    assert np.all(np.abs(C.real - exact.real) <= bound)
    assert np.all(np.abs(C.imag - exact.imag) <= bound)
    # and the rounding is TF32's, not lost terms: typical errors far below the bound
    assert np.median(np.abs(C - exact) / S) < 2.0 ** -10


@pytest.mark.parametrize("n,nv,ncol,ldr,flags", [
    (3001, 21, 40, 3001, 0),                            # odd n: rows not on 16-byte boundaries
    (3000, 21, 7, 3000, 0),                             # too few columns
    (3000, 21, 40, 3000, 8192),                         # GDR_FLAG_NO_TENSOR_CORES
])
def test_cuda_core_fallback(ctx, n, nv, ncol, ldr, flags):
    assert flags in (0, g.GDR_FLAG_NO_TENSOR_CORES)
    C, exact, S, prof = run_dot(ctx, n, nv, ncol, ldr, seed=7 * n + nv, flags=flags)
    assert not tc_ran(prof), prof
    bound = 2.0 ** -22 * S
    assert np.all(np.abs(C.real - exact.real) <= bound)
    assert np.all(np.abs(C.imag - exact.imag) <= bound)


def test_fp64_dot(ctx):
    rng = np.random.default_rng(3)
    n, nv, ncol = 4000, 30, 24
    V = rng.standard_normal((nv, n)) + 1j * rng.standard_normal((nv, n))
    R = rng.standard_normal((ncol, n)) + 1j * rng.standard_normal((ncol, n))
    Cd = torch.zeros((ncol, nv), dtype=torch.complex128, device="cuda")
    g.gdr_basis_dot(ctx, g.GDR_PREC_FP64, n, nv, dev(V), ncol, dev(R), n, Cd)
    exact = np.conj(V) @ R.T
    S = np.abs(V) @ np.abs(R).T
    assert np.all(np.abs(Cd.cpu().numpy().T - exact) <= 1e-13 * S)


# ------------------------------------------------------------------ residual update
#
# gdr_basis_residual_update: R[:, c] += V T[:, c] (the projection's residual update).
# On the tensor cores V and T are split into two TF32 parts each and three products
# are accumulated in FP32, so the result carries FP32-level errors, element by element
#
#     |R_out - R_exact| <= 2^-16 * S + 2^-22 * (|R_in| + |R_exact|),
#
# S = sum_k |A_mk| |B_kc| over the real form (K = 2 nv terms; 2^-16 covers the worst-case
# FP32 accumulation of up to 96 terms and the dropped lo*lo product), the second term
# the final FP32 addition.  A single TF32 product would leave errors near 2^-11 S: the
# median is held far below that.  The CUDA-core form is held to the same bound.

def run_update(ctx, n, nv, ncol, ldr, seed, flags=0):
    rng = np.random.default_rng(seed)
    V = c64(rng, nv, n)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    T = rng.standard_normal((ncol, nv)) + 1j * rng.standard_normal((ncol, nv))
    T *= np.exp(rng.uniform(-4, 2, size=(ncol, 1)))           # column scales over ~6 decades
    Rm = c64(rng, ncol, ldr)
    R0 = Rm.copy()
    Rd = dev(Rm)
    g.gdr_profile(ctx, True)
    g.gdr_basis_residual_update(ctx, g.GDR_PREC_MIXED, n, nv, dev(V), ncol, dev(T), Rd, ldr, flags)
    prof = g.gdr_profile_report(ctx)
    g.gdr_profile(ctx, False)
    out = Rd.cpu().numpy()
    Vd = V.astype(np.complex128)
    exact = R0[:, :n].astype(np.complex128) + T @ Vd            # row c: r_c + V T[:, c]
    # S over the real form: |Re v||Re t| + |Im v||Im t| (real row), |Im v||Re t| + |Re v||Im t| (imag row)
    Sre = np.abs(T.real) @ np.abs(Vd.real) + np.abs(T.imag) @ np.abs(Vd.imag)
    Sim = np.abs(T.real) @ np.abs(Vd.imag) + np.abs(T.imag) @ np.abs(Vd.real)
    return out, R0, exact, Sre, Sim, prof


def check_update(out, R0, exact, Sre, Sim, n):
    got = out[:, :n].astype(np.complex128)
    r0 = R0[:, :n].astype(np.complex128)
    bre = 2.0 ** -16 * Sre + 2.0 ** -22 * (np.abs(r0.real) + np.abs(exact.real))
    bim = 2.0 ** -16 * Sim + 2.0 ** -22 * (np.abs(r0.imag) + np.abs(exact.imag))
    assert np.all(np.abs(got.real - exact.real) <= bre)
    assert np.all(np.abs(got.imag - exact.imag) <= bim)
    assert np.array_equal(out[:, n:], R0[:, n:])                 # padding of the column stride untouched


def tcu_ran(prof):
    return prof.get("tc_proj_update_c64", {}).get("launches", 0) > 0


@pytest.mark.parametrize("n,nv,ncol,ldr", [
    (3000, 21, 8, 3000),        # ragged last row tile (3000 = 46 x 64 + 56); fewest columns
    (5000, 41, 120, 5006),      # the 24^3x32 Proj shape (k = 40), padded stride
    (4096, 48, 130, 4096),      # largest basis of this form, two column tiles of 96
    (1000, 1, 40, 1000),        # one basis vector
    (262144, 31, 96, 262144),   # a long vector: many row tiles per CTA
    (2000, 41, 300, 2002),      # three column tiles (128 wide), padded stride
])
def test_tensor_core_residual_update(ctx, n, nv, ncol, ldr):
    out, R0, exact, Sre, Sim, prof = run_update(ctx, n, nv, ncol, ldr, seed=n + 3 * nv + ncol)
    assert tcu_ran(prof), prof
    check_update(out, R0, exact, Sre, Sim, n)
    # split TF32: errors at the FP32 level, far below a single TF32 product's ~2^-11 S
    got = out[:, :n].astype(np.complex128)
    rel = np.abs(got.real - exact.real) / (Sre + np.abs(exact.real))
    assert np.median(rel) < 2.0 ** -20


@pytest.mark.parametrize("n,nv,ncol,flags", [
    (3000, 21, 7, 0),                         # too few columns
    (3000, 49, 40, 0),                        # more basis vectors than this form takes
    (3000, 21, 40, 8192),                     # GDR_FLAG_NO_TENSOR_CORES
])
def test_residual_update_cuda_cores(ctx, n, nv, ncol, flags):
    assert flags in (0, g.GDR_FLAG_NO_TENSOR_CORES)
    out, R0, exact, Sre, Sim, prof = run_update(ctx, n, nv, ncol, n, seed=11 * n + nv, flags=flags)
    assert not tcu_ran(prof), prof
    check_update(out, R0, exact, Sre, Sim, n)


def test_fp64_residual_update(ctx):
    rng = np.random.default_rng(5)
    n, nv, ncol = 3000, 30, 20
    V = rng.standard_normal((nv, n)) + 1j * rng.standard_normal((nv, n))
    T = rng.standard_normal((ncol, nv)) + 1j * rng.standard_normal((ncol, nv))
    R0 = rng.standard_normal((ncol, n)) + 1j * rng.standard_normal((ncol, n))
    Rd = dev(R0)
    g.gdr_basis_residual_update(ctx, g.GDR_PREC_FP64, n, nv, dev(V), ncol, dev(T), Rd, n)
    exact = R0 + T @ V
    S = np.abs(T) @ np.abs(V) + np.abs(R0)
    assert np.all(np.abs(Rd.cpu().numpy() - exact) <= 1e-13 * S)


# ------------------------------------------------------------------ whole solves

def test_solve_with_and_without_tensor_cores(ctx):
    """A mixed solve whose refinement batch (3 right-hand sides x 4 shifts = 12 pair
    columns over the kept basis) takes the tensor-core projection, against the same
    solve with GDR_FLAG_NO_TENSOR_CORES: both reach the FP64 true residual 1e-8 with the
    oracle's operator, their solutions agree to 1e-6, and the tensor-core kernels ran in
    the first only."""
    import workloads as W
    from oracle import WilsonOperator
    p = W.wilson_problem(2, dims=(8, 8, 8, 8), eps=0.3, nshift=4, nrhs=3, m=24, k=10, m_proj=14,
                         kappa_c=0.1325)
    dims, diag_a, links = p.op[1], p.op[2], p.op[3]
    op_o = WilsonOperator(dims, links, diag_a=diag_a)
    op = g.gdr_op_wilson(ctx, dims, dev(links), diag_a, g.GDR_LINK_C64)
    out = {}
    for flags in (0, g.GDR_FLAG_NO_TENSOR_CORES):
        prm = g.gdr_params_default(m=p.m, k=p.k, m_proj=p.m_proj, tol=1e-8, prec=g.GDR_PREC_MIXED, flags=flags)
        X = torch.zeros((p.B.shape[1], len(p.sigma), p.n), dtype=torch.complex128, device="cuda")
        g.gdr_profile(ctx, True)
        st, rep, _ = g.gdr_solve_multishift(ctx, op, p.sigma, dev(np.ascontiguousarray(p.B.T)), X, prm)
        prof = g.gdr_profile_report(ctx)
        g.gdr_profile(ctx, False)
        assert st == g.GDR_OK, rep
        ran = tc_ran(prof) or tcu_ran(prof)
        assert ran == (flags == 0), (flags, sorted(prof))
        Xh = X.cpu().numpy()
        for j in range(p.B.shape[1]):
            b = p.B[:, j]
            for i, s in enumerate(p.sigma):
                x = Xh[j, i]
                assert np.linalg.norm(b - (op_o.matvec(x) - s * x)) <= 1.05e-8 * np.linalg.norm(b), (flags, j, i)
        out[flags] = Xh
    a, b = out[0], out[g.GDR_FLAG_NO_TENSOR_CORES]
    assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)
    g.gdr_op_destroy(op)
