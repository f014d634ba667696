"""Python binding of libgdr.so (include/gdr.h): deflated multi-shift GMRES on GB300.

Argument marshalling only: every step of the solver runs in the CUDA library.
The functions carry the C names (``gdr_create``, ``gdr_solve_multishift``,
...) and take torch tensors (device memory) or numpy arrays (host shift lists,
host buffers with GDR_FLAG_HOST_PTRS) in place of raw pointers.  There is no
CPU fallback: importing works without a GPU, but ``gdr_create`` raises when no
CUDA device can be used, and every call raises when libgdr.so is missing.

Layouts: the C side is column-major, so an n x ncol matrix is a contiguous
torch tensor of shape (ncol, n); solutions X (n x ns x nrhs) are a tensor of
shape (nrhs, ns, n).  Complex numbers are complex128 (complex64 for the MIXED
step-level calls).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgdr.so")

GDR_OK, GDR_EINVAL, GDR_ENOMEM, GDR_ECUDA, GDR_ENOCONV, GDR_EBREAKDOWN, GDR_ENAN, GDR_ETIMEOUT, GDR_ENOTIMPL = range(9)
GDR_PREC_FP64, GDR_PREC_MIXED = 0, 1
GDR_LINK_C128, GDR_LINK_C64, GDR_LINK_BF16 = 0, 1, 2
GDR_MAX_M = 96
GDR_NOALLOC_MAX_M, GDR_NOALLOC_MAX_NS = 96, 16
(GDR_FLAG_HOST_PTRS, GDR_FLAG_NO_GRAPH, GDR_FLAG_SEQUENTIAL, GDR_FLAG_NO_PROJ, GDR_FLAG_NO_REFINE, GDR_FLAG_NO_SWEEP,
 GDR_FLAG_FP64_EIG, GDR_FLAG_AUTOTUNE, GDR_FLAG_RELATED_RHS, GDR_FLAG_EIG_SELECT,
 GDR_FLAG_FOM, GDR_FLAG_CGS2, GDR_FLAG_FP64_DENSE, GDR_FLAG_NO_TENSOR_CORES) = (
    1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192)


class gdr_params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("k", ctypes.c_int), ("m_proj", ctypes.c_int),
                ("tol", ctypes.c_double), ("extra_tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("refine_tol", ctypes.c_double), ("max_mvps", ctypes.c_long), ("max_cycles", ctypes.c_int), ("refine_max", ctypes.c_int),
                ("prec", ctypes.c_int), ("flags", ctypes.c_uint), ("k_select", ctypes.c_int),
                ("m_refine", ctypes.c_int), ("refine_rank_tol", ctypes.c_double)]


class gdr_report(ctypes.Structure):
    _fields_ = [("mvps_rhs1", ctypes.c_long), ("cycles_rhs1", ctypes.c_long), ("mvps_extra", ctypes.c_long),
                ("mvps_proj", ctypes.c_long), ("mvps_refine", ctypes.c_long), ("resid_cols", ctypes.c_long),
                ("refine_passes", ctypes.c_int), ("pairs_cleaned", ctypes.c_int),
                ("max_relres", ctypes.c_double), ("t_total_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_long), ("t_rhs1_ms", ctypes.c_double),
                ("t_proj_ms", ctypes.c_double), ("t_refine_ms", ctypes.c_double), ("host_syncs", ctypes.c_long),
                ("related_resid", ctypes.c_double), ("eig_resid_max", ctypes.c_double),
                ("shared_cols", ctypes.c_long), ("shared_pairs", ctypes.c_long), ("mvps_shared", ctypes.c_long)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class gdr_shape(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("threads", ctypes.c_int), ("col_inner", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class gdr_tune_result(ctypes.Structure):
    _fields_ = [("best", gdr_shape), ("mv_ms", ctypes.c_double), ("mv_ms_default", ctypes.c_double),
                ("candidates", ctypes.c_int), ("sweep", ctypes.c_int), ("cycle_ms_sweep", ctypes.c_double),
                ("cycle_ms_launch", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["best"] = self.best.as_dict()
        return d


class GdrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "GDR_OK", 1: "GDR_EINVAL", 2: "GDR_ENOMEM", 3: "GDR_ECUDA", 4: "GDR_ENOCONV",
           5: "GDR_EBREAKDOWN", 6: "GDR_ENAN", 7: "GDR_ETIMEOUT", 8: "GDR_ENOTIMPL"}

# exported symbols and their signatures (argument marshalling only)
_P = ctypes.c_void_p
_SIGS = {
    "gdr_params_default": (None, [ctypes.POINTER(gdr_params)]),
    "gdr_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P]),
    "gdr_destroy": (None, [_P]),
    "gdr_last_error": (ctypes.c_char_p, [_P]),
    "gdr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gdr_op_csr": (ctypes.c_int, [_P, ctypes.c_long, ctypes.c_long, _P, _P, _P, ctypes.POINTER(_P)]),
    "gdr_op_wilson": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.c_double, _P, ctypes.c_int,
                                     ctypes.POINTER(_P)]),
    "gdr_op_csr_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "gdr_solve_batch": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P, ctypes.POINTER(gdr_params),
                                       ctypes.POINTER(gdr_report), _P]),
    "gdr_op_destroy": (None, [_P]),
    "gdr_op_n": (ctypes.c_long, [_P]),
    "gdr_op_apply": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "gdr_autotune": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(gdr_tune_result)]),
    "gdr_op_set_shape": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(gdr_shape)]),
    "gdr_op_get_shape": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(gdr_shape)]),
    "gdr_solve_multishift": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, _P, _P,
                                            ctypes.POINTER(gdr_params), ctypes.POINTER(_P),
                                            ctypes.POINTER(gdr_report)]),
    "gdr_solve_proj": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, ctypes.c_int, _P, _P,
                                      ctypes.POINTER(gdr_params), ctypes.POINTER(gdr_report)]),
    "gdr_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "gdr_profile_report": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_long]),
    "gdr_defl_export": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_int)]),
    "gdr_defl_destroy": (None, [_P]),
    "gdr_arnoldi_step": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, _P]),
    "gdr_arnoldi_cycle": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_uint,
                                         ctypes.POINTER(ctypes.c_int)]),
    "gdr_dense_gmres_sh": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gdr_dense_gmres_sh_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P,
                                                  _P]),
    "gdr_barrier_selftest": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "gdr_dense_ls": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]),
    "gdr_dense_restart": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "gdr_basis_update": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_long, ctypes.c_int, _P, _P, ctypes.c_int,
                                        ctypes.c_int, _P]),
    "gdr_basis_dot": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_long, ctypes.c_int, _P, ctypes.c_int, _P,
                                     ctypes.c_long, _P, ctypes.c_uint]),
    "gdr_basis_residual_update": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_long, ctypes.c_int, _P, ctypes.c_int, _P,
                                                 _P, ctypes.c_long, ctypes.c_uint]),
}

_lib = None


def lib():
    """The loaded libgdr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgdr.so not built ({LIB_PATH}); run __graft_entry__.build() "
                               "or python -m paper_0707_0502_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st, ctx=None):
    if st != GDR_OK:
        msg = lib().gdr_last_error(ctx)
        raise GdrError(st, msg.decode() if msg else "")


def _ptr(t):
    """Raw pointer of a torch tensor (device) or numpy array (host)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous(), "tensors must be contiguous"
    return t.data_ptr()


def _c128_host(vals):
    a = np.ascontiguousarray(np.asarray(vals, dtype=np.complex128).ravel())
    return a


# ------------------------------------------------------------------ context

def gdr_params_default(**overrides):
    p = gdr_params()
    lib().gdr_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def gdr_create(device=0, stream=None):
    """Context on ``device`` using ``stream`` (a torch.cuda.Stream, a raw
    cudaStream_t int, or None for the current torch stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = _P()
    _check(lib().gdr_create(ctypes.byref(h), int(device), _P(int(stream)) if stream else None))
    return h


def gdr_destroy(ctx):
    lib().gdr_destroy(ctx)


def gdr_last_error(ctx):
    return lib().gdr_last_error(ctx).decode()


# ---------------------------------------------------------------- operators

def gdr_op_csr(ctx, rowptr, col, vals):
    """rowptr/col: int32 device tensors, vals: complex128 device tensor."""
    h = _P()
    n = rowptr.numel() - 1
    _check(lib().gdr_op_csr(ctx, n, vals.numel(), _ptr(rowptr), _ptr(col), _ptr(vals), ctypes.byref(h)), ctx)
    return h


def gdr_op_wilson(ctx, dims, links, diag_a=0.0, store=GDR_LINK_C64):
    """links: complex128 device tensor [4, V, 3, 3]."""
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    h = _P()
    _check(lib().gdr_op_wilson(ctx, d, float(diag_a), _ptr(links), int(store), ctypes.byref(h)), ctx)
    return h


def gdr_op_csr_batch(ctx, n, nnz, rowptr, col, vals):
    """n, nnz: per-problem sizes (host); rowptr/col (int32) and vals (complex128):
    the problems' CSR arrays concatenated, on the device."""
    nn = np.ascontiguousarray(np.asarray(n, dtype=np.int64))
    nz = np.ascontiguousarray(np.asarray(nnz, dtype=np.int64))
    h = _P()
    _check(lib().gdr_op_csr_batch(ctx, len(nn), nn.ctypes.data, nz.ctypes.data, _ptr(rowptr), _ptr(col), _ptr(vals),
                                  ctypes.byref(h)), ctx)
    return h


def gdr_solve_batch(ctx, op, sigma, B, X, params):
    """sigma: (nprob, ns); B: concatenated right-hand sides; X: concatenated n_p x ns
    blocks (column-major per problem).  Returns (status, report, per-problem status)."""
    s = _c128_host(sigma)
    sg = np.asarray(sigma)
    nprob, ns = sg.shape
    rep = gdr_report()
    per = np.zeros(nprob, dtype=np.int32)
    st = lib().gdr_solve_batch(ctx, op, int(ns), s.ctypes.data, _ptr(B), _ptr(X), ctypes.byref(params),
                               ctypes.byref(rep), per.ctypes.data)
    if st not in (GDR_OK, GDR_ENOCONV):
        _check(st, ctx)
    return st, rep.as_dict(), per


def make_batch_operator(ctx, problems, device="cuda"):
    """Batch operator from a list of ``workloads.Problem`` with CSR operators."""
    import torch
    rp = np.concatenate([p.op[1] for p in problems]).astype(np.int32)
    cl = np.concatenate([p.op[2] for p in problems]).astype(np.int32)
    vl = np.concatenate([p.op[3] for p in problems]).astype(np.complex128)
    return gdr_op_csr_batch(ctx, [p.n for p in problems], [len(p.op[2]) for p in problems],
                            torch.as_tensor(rp, device=device), torch.as_tensor(cl, device=device),
                            torch.as_tensor(vl, device=device))


def gdr_op_destroy(op):
    lib().gdr_op_destroy(op)


def gdr_op_n(op):
    return lib().gdr_op_n(op)


def gdr_op_apply(ctx, op, prec, sigma, X, Y):
    """Y[c] = (A - sigma_c I) X[c]; X, Y: (ncol, n) complex128 (FP64) or complex64 (MIXED)."""
    s = _c128_host(sigma)
    _check(lib().gdr_op_apply(ctx, op, int(prec), len(s), s.ctypes.data, _ptr(X), _ptr(Y)), ctx)


def gdr_autotune(ctx, op, prec, ncol, m=0):
    """Time the matvec shapes (and, m > 0, the Arnoldi forms) for ncol columns; returns the result dict."""
    r = gdr_tune_result()
    _check(lib().gdr_autotune(ctx, op, int(prec), int(ncol), int(m), ctypes.byref(r)), ctx)
    return r.as_dict()


def gdr_op_set_shape(op, prec, ncol, form=None, threads=None, col_inner=0):
    """Set the matvec shape of op for (prec, ncol); form=None forgets it (ncol <= 0: all)."""
    if form is None:
        st = lib().gdr_op_set_shape(op, int(prec), int(ncol), None)
    else:
        sh = gdr_shape(int(form), int(threads), int(col_inner))
        st = lib().gdr_op_set_shape(op, int(prec), int(ncol), ctypes.byref(sh))
    if st != GDR_OK:
        raise GdrError(st, "bad shape")


def gdr_op_get_shape(op, prec, ncol):
    sh = gdr_shape()
    st = lib().gdr_op_get_shape(op, int(prec), int(ncol), ctypes.byref(sh))
    if st != GDR_OK:
        raise GdrError(st, "bad arguments")
    return sh.as_dict()


# ------------------------------------------------------------------- solves

def gdr_solve_multishift(ctx, op, sigma, B, X, params, want_defl=False):
    """B: (nrhs, n) complex128, X: (nrhs, ns, n) complex128, written.  Device
    tensors, or numpy arrays when params.flags has GDR_FLAG_HOST_PTRS.
    Returns (status, report dict, deflation handle or None).  Raises on
    errors other than GDR_ENOCONV."""
    s = _c128_host(sigma)
    rep = gdr_report()
    dh = _P()
    nrhs = B.shape[0] if B.ndim == 2 else 1
    st = lib().gdr_solve_multishift(ctx, op, len(s), s.ctypes.data, nrhs, _ptr(B), _ptr(X), ctypes.byref(params),
                                    ctypes.byref(dh) if want_defl else None, ctypes.byref(rep))
    if st not in (GDR_OK, GDR_ENOCONV):
        _check(st, ctx)
    return st, rep.as_dict(), (dh if want_defl and dh.value else None)


def gdr_solve_proj(ctx, op, defl, sigma, B, X, params):
    s = _c128_host(sigma)
    rep = gdr_report()
    nrhs = B.shape[0] if B.ndim == 2 else 1
    st = lib().gdr_solve_proj(ctx, op, defl, len(s), s.ctypes.data, nrhs, _ptr(B), _ptr(X), ctypes.byref(params),
                              ctypes.byref(rep))
    if st not in (GDR_OK, GDR_ENOCONV):
        _check(st, ctx)
    return st, rep.as_dict()


def gdr_profile(ctx, enable):
    _check(lib().gdr_profile(ctx, 1 if enable else 0), ctx)


def gdr_profile_report(ctx):
    """{kernel: {"launches", "ms", "bytes"}} accumulated since gdr_profile(ctx, True)."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().gdr_profile_report(ctx, buf, len(buf)), ctx)
    return json.loads(buf.value.decode())


def gdr_defl_export(ctx, defl, V=None, n_k=None):
    """Returns (k, Hbar_k as numpy (k+1) x k); fills V ((k+1, n) device tensor) if given."""
    k = ctypes.c_int()
    _check(lib().gdr_defl_export(ctx, defl, None, None, ctypes.byref(k)), ctx)
    H = np.zeros((k.value, k.value + 1), dtype=np.complex128)  # column-major (k+1) x k
    _check(lib().gdr_defl_export(ctx, defl, _ptr(V), H.ctypes.data, ctypes.byref(k)), ctx)
    return k.value, H.T.copy()


def gdr_defl_destroy(defl):
    lib().gdr_defl_destroy(defl)


# --------------------------------------------------------------- step level

def gdr_arnoldi_step(ctx, op, prec, V, j, hcol):
    """V: (j+2, n) device tensor (rows are basis vectors), hcol: (j+2,) complex128 device."""
    _check(lib().gdr_arnoldi_step(ctx, op, int(prec), _ptr(V), int(j), _ptr(hcol)), ctx)


def gdr_arnoldi_cycle(ctx, op, prec, V, j0, m, Hbar, flags=0):
    """V: (m+1, n) device tensor (rows are basis vectors; rows 0..j0 given), Hbar:
    (m, m+1) complex128 device tensor (column-major (m+1) x m; columns < j0 given).
    Returns m_eff (m, or the length after a lucky breakdown)."""
    me = ctypes.c_int(0)
    _check(lib().gdr_arnoldi_cycle(ctx, op, int(prec), _ptr(V), int(j0), int(m), _ptr(Hbar), int(flags),
                                   ctypes.byref(me)), ctx)
    return me.value


def gdr_dense_gmres_sh(ctx, m, sigma, Hbar, c, beta, D, s, beta_new, norms):
    """Hbar: (m, m+1) complex128 device (column-major (m+1) x m), c: (m+1,), beta: (ns,);
    out D: (ns, m), s: (m+1,), beta_new: (ns,), norms: (ns,) float64."""
    sg = _c128_host(sigma)
    _check(lib().gdr_dense_gmres_sh(ctx, int(m), len(sg), _ptr(Hbar), _ptr(c), sg.ctypes.data, _ptr(beta), _ptr(D),
                                    _ptr(s), _ptr(beta_new), _ptr(norms)), ctx)


def gdr_dense_gmres_sh_noalloc(ctx, m, sigma, Hbar, c, beta, D, s, beta_new, norms):
    """Same as gdr_dense_gmres_sh, with no device allocation inside the library
    (fixed workspace; m <= 96, ns <= 16; calls must not overlap on the GPU)."""
    sg = _c128_host(sigma)
    _check(lib().gdr_dense_gmres_sh_noalloc(ctx, int(m), len(sg), _ptr(Hbar), _ptr(c), sg.ctypes.data, _ptr(beta),
                                            _ptr(D), _ptr(s), _ptr(beta_new), _ptr(norms)), ctx)


def gdr_dense_ls(ctx, prec, m, sigma1, Hbar, c, y, s):
    """Hbar: (m, m+1) complex128 device (column-major (m+1) x m, Hessenberg), c: (m+1,);
    out y: (m,), s: (m+1,) complex128 device."""
    sg = _c128_host([sigma1])
    _check(lib().gdr_dense_ls(ctx, int(prec), int(m), sg.ctypes.data, _ptr(Hbar), _ptr(c), _ptr(y), _ptr(s)), ctx)


def gdr_dense_restart(ctx, prec, m, k, sigma1, Hbar, s, theta, P, Hk, ck):
    sg = _c128_host([sigma1])
    _check(lib().gdr_dense_restart(ctx, int(prec), int(m), int(k), sg.ctypes.data, _ptr(Hbar), _ptr(s), _ptr(theta),
                                   _ptr(P), _ptr(Hk), _ptr(ck)), ctx)


def gdr_barrier_selftest(ctx, rounds, phantom):
    """Status of the grid-barrier self-test (GDR_OK, or GDR_ETIMEOUT with phantom);
    does not raise for GDR_ETIMEOUT."""
    return lib().gdr_barrier_selftest(ctx, int(rounds), int(phantom))


def gdr_basis_update(ctx, prec, n, nv, V, C, nout, nx, X):
    _check(lib().gdr_basis_update(ctx, int(prec), int(n), int(nv), _ptr(V), _ptr(C), int(nout), int(nx), _ptr(X)),
           ctx)


def gdr_basis_dot(ctx, prec, n, nv, V, ncol, R, ldr, C, flags=0):
    _check(lib().gdr_basis_dot(ctx, int(prec), int(n), int(nv), _ptr(V), int(ncol), _ptr(R), int(ldr), _ptr(C),
                               int(flags)), ctx)


def gdr_basis_residual_update(ctx, prec, n, nv, V, ncol, T, R, ldr, flags=0):
    _check(lib().gdr_basis_residual_update(ctx, int(prec), int(n), int(nv), _ptr(V), int(ncol), _ptr(T), _ptr(R),
                                           int(ldr), int(flags)), ctx)


# ------------------------------------------------------------- convenience

def make_operator(ctx, problem, store=GDR_LINK_C64, device="cuda"):
    """Operator handle from a ``workloads.Problem``-style ``op`` tuple."""
    import torch
    kind = problem.op[0]
    if kind == "csr":
        _, rowptr, col, vals = problem.op
        return gdr_op_csr(ctx, torch.as_tensor(rowptr, dtype=torch.int32, device=device),
                          torch.as_tensor(col, dtype=torch.int32, device=device),
                          torch.as_tensor(vals, dtype=torch.complex128, device=device))
    _, dims, diag_a, links = problem.op
    return gdr_op_wilson(ctx, dims, torch.as_tensor(links, dtype=torch.complex128, device=device), diag_a, store)
