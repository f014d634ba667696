"""Seeded synthetic inputs for the deflated multi-shift GMRES solver.

This module only *makes inputs*: matrices, gauge links, right-hand sides and
shift lists.  It holds none of the solver's arithmetic, so both the CPU oracle
(``oracle/``) and the CUDA library are fed from here without sharing any code
with each other.

Problem statement (Sec. 1, eq. (1)): (A - sigma_i I) x_i^j = b^j for shifts
i = 1..ns and right-hand sides j = 1..nrhs; sigma_1 is the base shift.

Every generator draws from ``numpy.random.default_rng([config_id, purpose])``
with purpose 0 = gauge links, 1 = right-hand sides, 2 = matrix parameters.
numpy's Generator streams are platform independent, so the x86 development
host and the aarch64 GPU host build identical arrays (up to the last-bit
rounding of the matrix exponential used for gauge links).

Layouts (all complex128, C order):
  * spinor fields: component index ``site*12 + spin*3 + color`` with
    ``site = ((t*Lz + z)*Ly + y)*Lx + x``;
  * gauge links: ``links[mu, site, a, b]`` = U_mu(x)_{ab}, the link from x to
    x + mu-hat, mu = 0..3 for x, y, z, t;
  * CSR: int32 ``rowptr`` (n+1), int32 ``col`` (nnz), complex128 ``vals``.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
KAPPA_C_FILE = os.path.join(_HERE, "kappa_c.json")


def rng(config_id: int, purpose: int) -> np.random.Generator:
    """The seeded stream for (config, purpose)."""
    return np.random.default_rng([int(config_id), int(purpose)])


# --------------------------------------------------------------------------
# CSR matrices
# --------------------------------------------------------------------------

def bidiag_csr(diag, sup=1.0):
    """Upper bidiagonal matrix with the given diagonal and a constant
    superdiagonal, as CSR (the test matrix of Example 1, Sec. 3)."""
    diag = np.asarray(diag, dtype=np.complex128)
    n = diag.shape[0]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        cols.append(i)
        vals.append(diag[i])
        if i + 1 < n:
            cols.append(i + 1)
            vals.append(sup)
        rowptr[i + 1] = len(cols)
    return rowptr, np.asarray(cols, dtype=np.int32), np.asarray(vals, dtype=np.complex128)


def convdiff_csr(s: int, cx: float, cy: float, delta: float):
    """5-point centred discretisation of -Laplace(u) + c.grad(u) on the unit
    square with Dirichlet boundaries, h = 1/(s+1), unscaled (1/h^2), plus an
    imaginary diagonal shift i*delta.  Lexicographic ordering row = iy*s + ix."""
    h = 1.0 / (s + 1)
    n = s * s
    centre = 4.0 / h**2 + 1j * delta
    east = -1.0 / h**2 + cx / (2 * h)
    west = -1.0 / h**2 - cx / (2 * h)
    north = -1.0 / h**2 + cy / (2 * h)
    south = -1.0 / h**2 - cy / (2 * h)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cols = np.empty(5 * n, dtype=np.int32)
    vals = np.empty(5 * n, dtype=np.complex128)
    p = 0
    for iy in range(s):
        for ix in range(s):
            r = iy * s + ix
            for (dx, dy, v) in ((0, -1, south), (-1, 0, west), (0, 0, centre), (1, 0, east), (0, 1, north)):
                jx, jy = ix + dx, iy + dy
                if 0 <= jx < s and 0 <= jy < s:
                    cols[p] = jy * s + jx
                    vals[p] = v
                    p += 1
            rowptr[r + 1] = p
    return rowptr, cols[:p].copy(), vals[:p].copy()


# --------------------------------------------------------------------------
# SU(3) gauge links
# --------------------------------------------------------------------------

def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_1..lambda_8 (3x3, Hermitian, traceless)."""
    L = np.zeros((8, 3, 3), dtype=np.complex128)
    L[0][0, 1] = L[0][1, 0] = 1
    L[1][0, 1] = -1j; L[1][1, 0] = 1j
    L[2][0, 0] = 1; L[2][1, 1] = -1
    L[3][0, 2] = L[3][2, 0] = 1
    L[4][0, 2] = -1j; L[4][2, 0] = 1j
    L[5][1, 2] = L[5][2, 1] = 1
    L[6][1, 2] = -1j; L[6][2, 1] = 1j
    L[7][0, 0] = L[7][1, 1] = 1 / np.sqrt(3); L[7][2, 2] = -2 / np.sqrt(3)
    return L


def su3_links(dims, eps: float, gen: np.random.Generator) -> np.ndarray:
    """Links U = exp(i eps X), X = sum_a omega_a lambda_a / 2, omega_a ~ N(0,1).

    The exponential uses the Hermitian eigendecomposition of X, then the result
    is re-unitarised (polar factor) and its determinant phase removed so that
    each link is in SU(3) to rounding.  Returns complex128 [4, V, 3, 3]."""
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    V = Lx * Ly * Lz * Lt
    omega = gen.standard_normal((4, V, 8))
    X = np.einsum("mva,aij->mvij", omega, gell_mann()) / 2.0
    w, Q = np.linalg.eigh(X)
    U = np.einsum("mvij,mvj,mvkj->mvik", Q, np.exp(1j * eps * w), Q.conj())
    # polar re-unitarisation, then fix det = 1
    u, _, vh = np.linalg.svd(U)
    U = u @ vh
    det = np.linalg.det(U)
    U = U / (det ** (1.0 / 3.0))[..., None, None]
    return np.ascontiguousarray(U)


# --------------------------------------------------------------------------
# right-hand sides
# --------------------------------------------------------------------------

def gaussian_real(gen, n, ncol=None):
    shape = (n,) if ncol is None else (n, ncol)
    return gen.standard_normal(shape).astype(np.complex128)


def gaussian_complex(gen, n, ncol=None):
    shape = (n,) if ncol is None else (n, ncol)
    return (gen.standard_normal(shape) + 1j * gen.standard_normal(shape)) / np.sqrt(2.0)


def z2_noise(gen, n, ncol=None):
    """Entries (+-1 +- i)/sqrt(2) with independent signs."""
    shape = (n,) if ncol is None else (n, ncol)
    re = gen.integers(0, 2, size=shape) * 2 - 1
    im = gen.integers(0, 2, size=shape) * 2 - 1
    return (re + 1j * im).astype(np.complex128) / np.sqrt(2.0)


# --------------------------------------------------------------------------
# shift lists
# --------------------------------------------------------------------------

def load_kappa_c():
    """Critical kappa per Wilson lattice, written by ``make_kappa_c.py``."""
    with open(KAPPA_C_FILE) as f:
        return json.load(f)


def kappa_list(kappa_c: float, count: int, lo: float = 0.115, frac: float = 0.98):
    """``count`` kappa values evenly spaced from ``lo`` to ``frac*kappa_c``
    inclusive, returned largest first (the largest kappa is closest to
    critical, so it converges slowest and is the base system)."""
    hi = frac * kappa_c
    assert lo < hi, (lo, hi)
    return np.linspace(lo, hi, count)[::-1].copy()


def wilson_shifts(kappas):
    """Systems (1/kappa) I - H are written A - sigma I with A = -H and
    sigma = -1/kappa."""
    return (-1.0 / np.asarray(kappas, dtype=np.float64)).astype(np.complex128)


# --------------------------------------------------------------------------
# the five benchmark configurations
# --------------------------------------------------------------------------

WILSON_LATTICES = {
    2: ((8, 8, 8, 8), 0.3),
    3: ((16, 16, 16, 16), 0.4),
    4: ((24, 24, 24, 32), 0.5),
}


@dataclass
class Problem:
    """One synthetic problem: operator description + shifts + RHS + solver
    parameters.  ``op`` is ``("csr", rowptr, col, vals)`` or
    ``("wilson", dims, diag_a, links)``."""
    name: str
    op: tuple
    n: int
    sigma: np.ndarray            # complex128 [ns], sigma[0] is the base shift
    B: np.ndarray                # complex128 [n, nrhs]
    m: int
    k: int
    m_proj: int
    tol: float = 1e-8
    extra_tol: float = 1e-5
    prec: str = "fp64"
    extra: dict = field(default_factory=dict)


def wilson_problem(cid: int, dims=None, eps=None, nshift=None, nrhs=None, kappa_c=None,
                   m=None, k=None, m_proj=None, rhs="z2"):
    """Wilson-Dirac-style problem of configuration ``cid`` (2, 3 or 4), or a
    reduced lattice of the same recipe when ``dims`` is given (tests)."""
    d0, e0 = WILSON_LATTICES.get(cid, ((4, 4, 4, 4), 0.3))
    dims = tuple(dims or d0)
    eps = e0 if eps is None else eps
    links = su3_links(dims, eps, rng(cid, 0))
    V = int(np.prod(dims))
    n = 12 * V
    if kappa_c is None:
        kappa_c = load_kappa_c()[lattice_key(dims, eps, cid)]
    kap = kappa_list(kappa_c, nshift)
    sigma = wilson_shifts(kap)
    g = rng(cid, 1)
    if rhs == "gaussian":
        B = gaussian_complex(g, n, nrhs)
    else:
        B = z2_noise(g, n, nrhs)
    return Problem(name=f"wilson{'x'.join(map(str, dims))}", op=("wilson", dims, 0.0, links), n=n,
                   sigma=sigma, B=B, m=m, k=k, m_proj=m_proj,
                   extra={"kappa": kap, "kappa_c": kappa_c, "eps": eps, "dims": dims})


def lattice_key(dims, eps, cid):
    return f"cfg{cid}:{'x'.join(map(str, dims))}:eps{eps:g}"


def config(cid: int) -> list[Problem] | Problem:
    """The benchmark configurations 1..5 (config 5 returns a list of 64)."""
    if cid == 1:
        rowptr, col, vals = bidiag_csr(np.arange(1, 1001, dtype=np.float64), 1.0)
        B = gaussian_real(rng(1, 1), 1000, 1)
        return Problem(name="bidiag1000", op=("csr", rowptr, col, vals), n=1000,
                       sigma=np.array([0, -0.5, -2, -10], dtype=np.complex128), B=B,
                       m=25, k=10, m_proj=15, prec="fp64")
    if cid == 2:
        p = wilson_problem(2, nshift=6, nrhs=1, m=40, k=20, m_proj=20, rhs="gaussian")
        p.prec = "mixed"
        return p
    if cid == 3:
        p = wilson_problem(3, nshift=8, nrhs=8, m=60, k=30, m_proj=30)
        p.prec = "mixed"
        return p
    if cid == 4:
        # m_p = 20 as in the paper's Example 7 (GMRES(20)-Proj); measured faster than m - k = 40
        p = wilson_problem(4, nshift=10, nrhs=12, m=80, k=40, m_proj=20)
        p.prec = "mixed"
        p.extra["links"] = "bf16"
        return p
    if cid == 5:
        g = rng(5, 2)
        sides = g.integers(32, 257, size=64)
        cxy = g.uniform(-20, 20, size=(64, 2))
        delta = g.uniform(0, 0.5, size=64)
        gr = rng(5, 1)
        probs = []
        for p in range(64):
            s = int(sides[p])
            rowptr, col, vals = convdiff_csr(s, cxy[p, 0], cxy[p, 1], delta[p])
            n = s * s
            B = gaussian_complex(gr, n, 1)
            probs.append(Problem(name=f"convdiff{s}", op=("csr", rowptr, col, vals), n=n,
                                 sigma=np.array([1.0, 0.0, 0.1, 0.5], dtype=np.complex128), B=B,
                                 m=30, k=10, m_proj=20, prec="mixed",
                                 extra={"side": s, "c": tuple(cxy[p]), "delta": float(delta[p])}))
        return probs
    raise ValueError(cid)


def paper_example1_matrix(n: int = 1000):
    """Example 1 (Sec. 3): bidiagonal, diagonal 0.1, 1, 2, ..., n-1, ones on
    the superdiagonal."""
    diag = np.concatenate([[0.1], np.arange(1, n, dtype=np.float64)])
    return bidiag_csr(diag, 1.0)
