// extern "C" entry points of include/gdr.h: argument checks, buffer staging
// and error translation around the solver drivers.  No C++ exception crosses
// this boundary.
#include <array>
#include <chrono>
#include <cstring>
#include <type_traits>

#include "kernels.cuh"
#include "solver.cuh"

namespace {

thread_local std::string g_err;  // message of the last failure without a context

template <typename F>
gdr_status guarded(gdr_ctx* ctx, F&& f) {
  try {
    f();
    return GDR_OK;
  } catch (const gdr_error& e) {
    if (ctx) ctx->err = e.what();
    g_err = e.what();
    return e.st;
  } catch (const std::exception& e) {
    if (ctx) ctx->err = e.what();
    g_err = e.what();
    return GDR_ECUDA;
  }
}

// a tensor-core wait that gave up during the call (the kernel then returned without
// its result): report it as GDR_ETIMEOUT and clear the flag for the next call
void tc_check(gdr_ctx* ctx) {
  if (!ctx->tc_err) return;
  int e = 0;
  GDR_CUDA(cudaMemcpy(&e, ctx->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    GDR_CUDA(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), ctx->stream));
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    throw gdr_error(GDR_ETIMEOUT, "tensor-core projection: a wait gave up");
  }
}

void check_params(gdr_ctx* ctx, const gdr_params& p) {
  ctx->tc_proj = !(p.flags & GDR_FLAG_NO_TENSOR_CORES);
  GDR_REQUIRE(p.m >= 2 && p.m <= GDR_MAX_M, "m must be in [2, GDR_MAX_M]");
  GDR_REQUIRE(p.k >= 0 && p.k < p.m, "k must satisfy 0 <= k < m");
  GDR_REQUIRE(p.m_proj >= 0 && p.m_proj <= GDR_MAX_M, "m_proj must be in [0, GDR_MAX_M]");
  GDR_REQUIRE(p.m_refine <= GDR_MAX_M, "m_refine must be at most GDR_MAX_M");
  GDR_REQUIRE(p.tol > 0 && p.extra_tol > 0, "tolerances must be positive");
  GDR_REQUIRE(p.max_mvps > 0, "max_mvps must be positive");
  GDR_REQUIRE(p.prec == GDR_PREC_FP64 || p.prec == GDR_PREC_MIXED, "unknown precision");
}

// inner_tol <= 0: loose complex64 stages when the basis is L2-resident (there the
// FP64 dense steps of each GMRES-DR cycle dominate); otherwise as tight as the
// operator's precision makes worthwhile, since each (shift, rhs) pair is refined on
// its own while the stage serves all shifts at once (measured on GB300: 16^4 with
// complex64 links 537 -> 480 ms at 3e-7; the 64-problem CSR batch 641 -> 611 ms at
// 1e-6; bf16 links limit what a complex64 stage and a refinement pass reach, so a
// tighter stage there only adds work: 24^3x32 11.2 s at 1e-5, 12.0 s at 1e-6).
gdr_params resolve_inner_tol(const gdr_ctx* ctx, const gdr_op* A, long n, const gdr_params& p) {
  gdr_params r = p;
  const double basis = (double)(p.m + 1) * (double)n * sizeof(c64);
  const bool long_vectors = basis > 0.5 * (double)ctx->l2_bytes;
  const bool bf16 = A->kind == OP_WILSON && A->store == GDR_LINK_BF16;
  if (!(r.inner_tol > 0)) {
    if (!long_vectors) r.inner_tol = 1e-3;
    // bf16 links: the links' rounding holds the stages' true residuals near 1e-3 whatever
    // the inner tolerance; measured at 24^3x32: 1e-4 2.71 s, 1e-5 2.94 s, 3e-4 and 1e-3 a
    // third refinement pass (2.78 / 2.86 s)
    else if (bf16) r.inner_tol = 1e-4;
    else if (A->kind == OP_CSR_BATCH) r.inner_tol = 1e-6;
    else r.inner_tol = 3e-7;
  }
  // a complex64 refinement pass reliably reduces its residual by 1e-4: one pass then
  // usually finishes a pair that the stage left at ~1e-4.  With bf16 links on long vectors
  // a pass gains only ~1e-3 against the true operator whatever it asks: 2e-4 (24^3x32:
  // 2.53 s with refinement cycles of 6, against 2.61 s at 1e-4 and 8)
  if (!(r.refine_tol > 0)) r.refine_tol = (bf16 && long_vectors) ? 2e-4 : std::min(r.inner_tol, 1e-4);
  return r;
}

std::vector<c128> host_c128(const double* p, int count) {
  std::vector<c128> v(count);
  for (int i = 0; i < count; ++i) v[i] = {p[2 * i], p[2 * i + 1]};
  return v;
}

}  // namespace

extern "C" {

void gdr_params_default(gdr_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->m = 40;
  p->k = 20;
  p->m_proj = 0;
  p->tol = 1e-8;
  p->extra_tol = 1e-5;
  p->inner_tol = 0.0;  // automatic
  p->refine_tol = 0.0;  // automatic
  p->max_mvps = 100000;
  p->max_cycles = 0;
  p->refine_max = 3;
  p->prec = GDR_PREC_FP64;
  p->flags = 0;
}

const char* gdr_status_string(gdr_status s) {
  switch (s) {
    case GDR_OK: return "GDR_OK";
    case GDR_EINVAL: return "GDR_EINVAL";
    case GDR_ENOMEM: return "GDR_ENOMEM";
    case GDR_ECUDA: return "GDR_ECUDA";
    case GDR_ENOCONV: return "GDR_ENOCONV";
    case GDR_EBREAKDOWN: return "GDR_EBREAKDOWN";
    case GDR_ENAN: return "GDR_ENAN";
    case GDR_ETIMEOUT: return "GDR_ETIMEOUT";
    case GDR_ENOTIMPL: return "GDR_ENOTIMPL";
  }
  return "GDR_?";
}

gdr_status gdr_create(gdr_ctx** out, int device, void* cuda_stream) {
  if (!out) return GDR_EINVAL;
  *out = nullptr;
  gdr_ctx* ctx = new gdr_ctx();
  gdr_status st = guarded(nullptr, [&] {
    int count = 0;
    GDR_CUDA(cudaGetDeviceCount(&count));
    GDR_REQUIRE(device >= 0 && device < count, "no such CUDA device");
    GDR_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    GDR_CUDA(cudaGetDeviceProperties(&prop, device));
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    ctx->max_smem_optin = prop.sharedMemPerBlockOptin;
    ctx->l2_bytes = prop.l2CacheSize;
    if (cuda_stream) {
      ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      // a blocking stream orders with the legacy default stream and can be captured
      GDR_CUDA(cudaStreamCreate(&ctx->stream));
      ctx->own_stream = true;
    }
    dense_init(ctx);
    krylov_init(ctx);
    sweep_init(ctx);
    tc_proj_init(ctx);
  });
  if (st != GDR_OK) {
    delete ctx;
    return st;
  }
  *out = ctx;
  return GDR_OK;
}

void gdr_destroy(gdr_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->ws)
    if (kv.second.p) cudaFree(kv.second.p);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* gdr_last_error(const gdr_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

gdr_status gdr_op_csr(gdr_ctx* ctx, long n, long nnz, const int* rowptr, const int* col, const double* vals,
                      gdr_op** out) {
  if (!ctx || !out) return GDR_EINVAL;
  *out = nullptr;
  gdr_op* op = new gdr_op();
  gdr_status st = guarded(ctx, [&] {
    GDR_REQUIRE(n > 0 && nnz >= 0, "bad CSR sizes");
    GDR_REQUIRE(rowptr && (nnz == 0 || (col && vals)), "null CSR array");
    GDR_CUDA(cudaSetDevice(ctx->device));
    op->ctx = ctx;
    op->kind = OP_CSR;
    op->n = n;
    op->nnz = nnz;
    op_build_csr(ctx, op, rowptr, col, vals);
  });
  if (st != GDR_OK) {
    gdr_op_destroy(op);
    return st;
  }
  *out = op;
  return GDR_OK;
}

gdr_status gdr_op_wilson(gdr_ctx* ctx, const int dims[4], double diag_a, const double* links, gdr_link_fmt store,
                         gdr_op** out) {
  if (!ctx || !out || !dims) return GDR_EINVAL;
  *out = nullptr;
  gdr_op* op = new gdr_op();
  gdr_status st = guarded(ctx, [&] {
    for (int i = 0; i < 4; ++i) GDR_REQUIRE(dims[i] >= 2, "each lattice extent must be >= 2");
    GDR_REQUIRE(links != nullptr, "null links");
    GDR_REQUIRE(store == GDR_LINK_C128 || store == GDR_LINK_C64 || store == GDR_LINK_BF16, "bad link format");
    GDR_CUDA(cudaSetDevice(ctx->device));
    op->ctx = ctx;
    op->kind = OP_WILSON;
    for (int i = 0; i < 4; ++i) op->dims[i] = dims[i];
    op->V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    op->n = 12 * op->V;
    op->diag_a = diag_a;
    op->store = store;
    op_build_wilson(ctx, op, links);
  });
  if (st != GDR_OK) {
    gdr_op_destroy(op);
    return st;
  }
  *out = op;
  return GDR_OK;
}

gdr_status gdr_op_csr_batch(gdr_ctx* ctx, int nprob, const long* n, const long* nnz, const int* rowptr,
                            const int* col, const double* vals, gdr_op** out) {
  if (!ctx || !out) return GDR_EINVAL;
  *out = nullptr;
  gdr_op* op = new gdr_op();
  gdr_status st = guarded(ctx, [&] {
    GDR_REQUIRE(nprob >= 1 && n && nnz && rowptr, "bad CSR batch arguments");
    for (int p = 0; p < nprob; ++p) GDR_REQUIRE(n[p] > 0 && nnz[p] >= 0, "bad CSR batch sizes");
    GDR_CUDA(cudaSetDevice(ctx->device));
    op->ctx = ctx;
    op->kind = OP_CSR_BATCH;
    op->nprob = nprob;
    op_build_csr_batch(ctx, op, n, nnz, rowptr, col, vals);
  });
  if (st != GDR_OK) {
    gdr_op_destroy(op);
    return st;
  }
  *out = op;
  return GDR_OK;
}

void gdr_op_destroy(gdr_op* op) {
  if (!op) return;
  cudaFree(op->rp_off);
  cudaFree(op->nz_off);
  cudaFree(op->nrow);
  cudaFree(op->rowptr);
  cudaFree(op->col);
  cudaFree(op->vals128);
  cudaFree(op->vals64);
  cudaFree(op->links128);
  cudaFree(op->links64);
  cudaFree(op->links16);
  delete op;
}

long gdr_op_n(const gdr_op* op) { return op ? op->n : 0; }

gdr_status gdr_op_apply(gdr_ctx* ctx, const gdr_op* A, gdr_prec prec, int ncol, const double* sigma, const void* X,
                        void* Y) {
  if (!ctx || !A) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_REQUIRE(ncol >= 0 && (ncol == 0 || (sigma && X && Y)), "bad gdr_op_apply arguments");
    if (ncol == 0) return;
    c128* sd = ctx->get<c128>("apply.sigma", (size_t)ncol);
    GDR_CUDA(cudaMemcpyAsync(sd, sigma, sizeof(c128) * ncol, cudaMemcpyHostToDevice, ctx->stream));
    auto run = [&](auto tag) {
      using R = decltype(tag);
      const cx<R>* x = static_cast<const cx<R>*>(X);
      cx<R>* y = static_cast<cx<R>*>(Y);
      if (A->kind != OP_WILSON) {
        op_apply<R>(ctx, A, ncol, sd, x, A->n, y, A->n, nullptr, 0);
        return;
      }
      // interface (site-major) order <-> the library's pair-major order
      cx<R>* xl = ctx->get<cx<R>>("apply.x", (size_t)A->n * ncol);
      cx<R>* yl = ctx->get<cx<R>>("apply.y", (size_t)A->n * ncol);
      op_order<cx<R>>(ctx, A, ncol, x, A->n, xl, A->n, true);
      op_apply<R>(ctx, A, ncol, sd, xl, A->n, yl, A->n, nullptr, 0);
      op_order<cx<R>>(ctx, A, ncol, yl, A->n, y, A->n, false);
    };
    if (prec == GDR_PREC_FP64)
      run(double{});
    else
      run(float{});
  });
}

// Staging of right-hand sides and solutions between the interface order (leading
// dimension n, host or device memory) and the library order (device, leading dimension
// ld); Wilson vectors are reordered through a scratch buffer of at most ~256 MB.
static int stage_chunk(const gdr_op* A, long ld, int cols) {
  return (int)std::max<long>(1, std::min<long>(cols, (256L << 20) / (ld * (long)sizeof(c128))));
}
static void stage_in(gdr_ctx* ctx, const gdr_op* A, int cols, const double* src, c128* dst, long ld,
                     cudaMemcpyKind kind) {
  const long n = A->n;
  if (A->kind != OP_WILSON) {
    GDR_CUDA(cudaMemcpy2DAsync(dst, ld * sizeof(c128), src, n * sizeof(c128), n * sizeof(c128), cols, kind,
                               ctx->stream));
    return;
  }
  const int ch = stage_chunk(A, ld, cols);
  c128* tmp = ctx->get<c128>("api.order", (size_t)ld * ch);
  for (int c0 = 0; c0 < cols; c0 += ch) {
    const int nc = std::min(ch, cols - c0);
    GDR_CUDA(cudaMemcpy2DAsync(tmp, ld * sizeof(c128), src + 2 * (long)c0 * n, n * sizeof(c128), n * sizeof(c128),
                               nc, kind, ctx->stream));
    op_order<c128>(ctx, A, nc, tmp, ld, dst + (long)c0 * ld, ld, true);
  }
}
static void stage_out(gdr_ctx* ctx, const gdr_op* A, int cols, const c128* src, long ld, double* dst,
                      cudaMemcpyKind kind) {
  const long n = A->n;
  if (A->kind != OP_WILSON) {
    GDR_CUDA(cudaMemcpy2DAsync(dst, n * sizeof(c128), src, ld * sizeof(c128), n * sizeof(c128), cols, kind,
                               ctx->stream));
    return;
  }
  const int ch = stage_chunk(A, ld, cols);
  c128* tmp = ctx->get<c128>("api.order", (size_t)ld * ch);
  for (int c0 = 0; c0 < cols; c0 += ch) {
    const int nc = std::min(ch, cols - c0);
    op_order<c128>(ctx, A, nc, src + (long)c0 * ld, ld, tmp, ld, false);
    GDR_CUDA(cudaMemcpy2DAsync(dst + 2 * (long)c0 * n, n * sizeof(c128), tmp, ld * sizeof(c128), n * sizeof(c128),
                               nc, kind, ctx->stream));
  }
}

gdr_status gdr_autotune(gdr_ctx* ctx, gdr_op* A, gdr_prec prec, int ncol, int m, gdr_tune_result* out) {
  if (!ctx || !A) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_REQUIRE(prec == GDR_PREC_FP64 || prec == GDR_PREC_MIXED, "bad precision");
    GDR_REQUIRE(ncol >= 1 && ncol <= 65535, "ncol must be in [1, 65535]");
    GDR_REQUIRE(m >= 0 && m <= GDR_MAX_M, "m must be in [0, GDR_MAX_M]");
    GDR_REQUIRE(A->kind != OP_CSR_BATCH || ncol % A->nprob == 0,
                "for a CSR batch ncol must be a multiple of the problem count");
    GDR_CUDA(cudaSetDevice(ctx->device));
    gdr_tune_result r{};
    tune_op(ctx, A, prec, ncol, m, r);
    if (out) *out = r;
  });
}

gdr_status gdr_op_set_shape(gdr_op* A, gdr_prec prec, int ncol, const gdr_shape* shape) {
  if (!A) return GDR_EINVAL;
  const int fk = prec == GDR_PREC_FP64 ? 1 : 0;
  if (!shape) {
    if (ncol <= 0) {
      A->mv_tuned.clear();
      A->sweep_tuned.clear();
    } else {
      A->mv_tuned.erase({fk, ncol});
    }
    return GDR_OK;
  }
  if (ncol < 1) return GDR_EINVAL;
  if (shape->col_inner < 0 || shape->col_inner > 65535) return GDR_EINVAL;
  MvShape s{shape->form, shape->threads, shape->col_inner};
  if (A->kind == OP_WILSON) {
    if (s.form == 1 && s.threads != 128) return GDR_EINVAL;
    if (s.form < 0 || s.form > 2) return GDR_EINVAL;
    if (s.form >= 2 && (fk == 1 || s.threads == 256)) return GDR_EINVAL;  // pairs: complex64, 64 or 128 threads
    if (s.threads != 64 && s.threads != 128 && s.threads != 256) return GDR_EINVAL;
  } else {
    if (s.form != 1 && s.form != 2 && s.form != 4 && s.form != 8) return GDR_EINVAL;
    if (s.threads != 128 && s.threads != 256) return GDR_EINVAL;
  }
  A->mv_tuned[{fk, ncol}] = s;
  return GDR_OK;
}

gdr_status gdr_op_get_shape(const gdr_op* A, gdr_prec prec, int ncol, gdr_shape* out) {
  if (!A || !out || ncol < 1) return GDR_EINVAL;
  const MvShape s = mv_shape(A->ctx, A, prec == GDR_PREC_FP64, ncol);
  *out = gdr_shape{s.form, s.threads, s.col_inner};
  return GDR_OK;
}

// GDR_FLAG_AUTOTUNE: tune every (precision, columns, m) a solve's stages launch
// with that the operator has no shape for yet
static void autotune_stages(gdr_ctx* ctx, const gdr_op* A, const gdr_params& p,
                            const std::vector<std::array<int, 3>>& keys) {
  if (!(p.flags & GDR_FLAG_AUTOTUNE)) return;
  gdr_op* Am = const_cast<gdr_op*>(A);  // the tuned shapes are a cache on the handle
  for (const auto& k : keys) {
    if (k[1] < 1 || k[1] > 65535) continue;
    if (A->mv_tuned.count({k[0], k[1]})) continue;
    gdr_tune_result r{};
    tune_op(ctx, Am, k[0] ? GDR_PREC_FP64 : GDR_PREC_MIXED, k[1], k[2], r);
  }
}

gdr_status gdr_solve_multishift(gdr_ctx* ctx, const gdr_op* A, int ns, const double* sigma, int nrhs, const double* B,
                                double* X, const gdr_params* params, gdr_defl** defl_out, gdr_report* report) {
  if (!ctx || !A) return GDR_EINVAL;
  if (defl_out) *defl_out = nullptr;
  gdr_report rep{};
  gdr_status result = GDR_OK;
  gdr_status st = guarded(ctx, [&] {
    GDR_REQUIRE(params && sigma && B && X, "null argument");
    GDR_REQUIRE(ns >= 1 && nrhs >= 1, "ns and nrhs must be >= 1");
    const gdr_params& p = *params;
    check_params(ctx, p);
    GDR_CUDA(cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    const long launches0 = ctx->launches;
    const long n = A->n, ld = pad_ld(n);
    std::vector<c128> sig = host_c128(sigma, ns);
    c128* Bi = ctx->get<c128>("api.B", (size_t)ld * nrhs);
    c128* Xi = ctx->get<c128>("api.X", (size_t)ld * ns * nrhs);
    const cudaMemcpyKind kin = (p.flags & GDR_FLAG_HOST_PTRS) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kout = (p.flags & GDR_FLAG_HOST_PTRS) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    stage_in(ctx, A, nrhs, B, Bi, ld, kin);
    const gdr_params pr = resolve_inner_tol(ctx, A, A->n, p);
    {
      const int fi = p.prec == GDR_PREC_FP64 ? 1 : 0, mp = pr.m_proj > 0 ? pr.m_proj : pr.m - pr.k;
      std::vector<std::array<int, 3>> keys{{fi, 1, pr.m}};
      if (nrhs > 1) keys.push_back({fi, nrhs - 1, mp});
      if (!fi && !(p.flags & GDR_FLAG_NO_REFINE)) keys.push_back({0, ns * nrhs, mp});
      keys.push_back({1, ns * nrhs, 0});
      autotune_stages(ctx, A, p, keys);
    }
    if (p.prec == GDR_PREC_MIXED)
      result = solve_pipeline<float>(ctx, A, sig, nrhs, Bi, ld, Xi, ld, pr, defl_out, rep);
    else
      result = solve_pipeline<double>(ctx, A, sig, nrhs, Bi, ld, Xi, ld, pr, defl_out, rep);
    stage_out(ctx, A, ns * nrhs, Xi, ld, X, kout);
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    tc_check(ctx);
    rep.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    rep.kernel_launches = ctx->launches - launches0;
  });
  if (report) *report = rep;
  return st != GDR_OK ? st : result;
}

gdr_status gdr_solve_batch(gdr_ctx* ctx, const gdr_op* A, int ns, const double* sigma, const double* B, double* X,
                           const gdr_params* params, gdr_report* report, int* status) {
  if (!ctx || !A) return GDR_EINVAL;
  gdr_report rep{};
  gdr_status result = GDR_OK;
  gdr_status st = guarded(ctx, [&] {
    GDR_REQUIRE(A->kind == OP_CSR_BATCH, "gdr_solve_batch needs an operator from gdr_op_csr_batch");
    GDR_REQUIRE(params && sigma && B && X && ns >= 1, "bad gdr_solve_batch arguments");
    const gdr_params& p = *params;
    check_params(ctx, p);
    GDR_CUDA(cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    const long launches0 = ctx->launches;
    const int np = A->nprob;
    const long ld = pad_ld(A->n);
    std::vector<c128> sig = host_c128(sigma, np * ns);
    c128* Bi = ctx->get<c128>("api.B", (size_t)ld * np);
    c128* Xi = ctx->get<c128>("api.X", (size_t)ld * ns * np);
    const bool host = (p.flags & GDR_FLAG_HOST_PTRS) != 0;
    const cudaMemcpyKind kin = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kout = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    GDR_CUDA(cudaMemsetAsync(Bi, 0, sizeof(c128) * ld * np, ctx->stream));
    long off = 0;
    for (int q = 0; q < np; ++q) {
      const long nq = A->nrow_host[q];
      GDR_CUDA(cudaMemcpyAsync(Bi + (long)q * ld, B + 2 * off, sizeof(c128) * nq, kin, ctx->stream));
      off += nq;
    }
    const gdr_params pr = resolve_inner_tol(ctx, A, A->n * (long)A->nprob, p);
    {
      const int fi = p.prec == GDR_PREC_FP64 ? 1 : 0, mp = pr.m_proj > 0 ? pr.m_proj : pr.m - pr.k;
      std::vector<std::array<int, 3>> keys{{fi, A->nprob, pr.m}};
      if (!fi && !(p.flags & GDR_FLAG_NO_REFINE)) keys.push_back({0, A->nprob * ns, mp});
      keys.push_back({1, A->nprob * ns, 0});
      autotune_stages(ctx, A, p, keys);
    }
    if (p.prec == GDR_PREC_MIXED)
      result = solve_batch_pipeline<float>(ctx, A, ns, sig, Bi, Xi, pr, rep, status);
    else
      result = solve_batch_pipeline<double>(ctx, A, ns, sig, Bi, Xi, pr, rep, status);
    off = 0;
    for (int q = 0; q < np; ++q) {
      const long nq = A->nrow_host[q];
      GDR_CUDA(cudaMemcpy2DAsync(X + 2 * off * ns, nq * sizeof(c128), Xi + (long)q * ns * ld, ld * sizeof(c128),
                                 nq * sizeof(c128), ns, kout, ctx->stream));
      off += nq;
    }
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    tc_check(ctx);
    rep.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    rep.kernel_launches = ctx->launches - launches0;
  });
  if (report) *report = rep;
  return st != GDR_OK ? st : result;
}

gdr_status gdr_solve_proj(gdr_ctx* ctx, const gdr_op* A, const gdr_defl* defl, int ns, const double* sigma, int nrhs,
                          const double* B, double* X, const gdr_params* params, gdr_report* report) {
  if (!ctx || !A || !defl) return GDR_EINVAL;
  gdr_report rep{};
  gdr_status result = GDR_OK;
  gdr_status st = guarded(ctx, [&] {
    GDR_REQUIRE(params && sigma && B && X, "null argument");
    GDR_REQUIRE(ns >= 1 && nrhs >= 1, "ns and nrhs must be >= 1");
    GDR_REQUIRE(defl->n == A->n, "deflation space size differs from the operator");
    GDR_REQUIRE(defl->wilson_V == (A->kind == OP_WILSON ? A->V : 0), "deflation space from another operator kind");
    const gdr_params& p = *params;
    check_params(ctx, p);
    GDR_CUDA(cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    const long launches0 = ctx->launches;
    const long n = A->n, ld = pad_ld(n);
    const int mp = p.m_proj > 0 ? p.m_proj : p.m - p.k;
    autotune_stages(ctx, A, p, {{p.prec == GDR_PREC_FP64 ? 1 : 0, nrhs, mp}});
    std::vector<c128> sig = host_c128(sigma, ns);
    c128* Bi = ctx->get<c128>("api.B", (size_t)ld * nrhs);
    c128* Xi = ctx->get<c128>("api.X", (size_t)ld * ns * nrhs);
    const cudaMemcpyKind kin = (p.flags & GDR_FLAG_HOST_PTRS) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind kout = (p.flags & GDR_FLAG_HOST_PTRS) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    stage_in(ctx, A, nrhs, B, Bi, ld, kin);
    GDR_CUDA(cudaMemsetAsync(Xi, 0, sizeof(c128) * ld * ns * nrhs, ctx->stream));
    auto run = [&](auto tag) {
      using R = decltype(tag);
      cx<R>* rin = ctx->get<cx<R>>("api.rin", (size_t)ld * nrhs);
      cx<R>* vd = ctx->get<cx<R>>("api.vd", (size_t)ld * (defl->k + 1));
      if (std::is_same<R, double>::value) {
        copy128(ctx, n, nrhs, Bi, ld, reinterpret_cast<c128*>(rin), ld);
        copy128(ctx, n, defl->k + 1, defl->V128, defl->ldv, reinterpret_cast<c128*>(vd), ld);
      } else {
        cvt_128_to_64(ctx, n, nrhs, Bi, ld, reinterpret_cast<c64*>(rin), ld);
        cvt_128_to_64(ctx, n, defl->k + 1, defl->V128, defl->ldv, reinterpret_cast<c64*>(vd), ld);
      }
      ProjJob<R> job;
      job.ncol = nrhs;
      job.ns = ns;
      job.m_p = mp;
      job.k = defl->k;
      job.project = !(p.flags & GDR_FLAG_NO_PROJ);
      job.Vd = vd;
      job.ldvd = ld;
      job.Hk = defl->Hk;
      job.rhs = rin;
      job.ldrhs = ld;
      job.sigma.resize((size_t)nrhs * ns);
      for (int c = 0; c < nrhs; ++c)
        for (int i = 0; i < ns; ++i) job.sigma[(size_t)c * ns + i] = sig[i];
      job.tol.assign(nrhs, p.tol);
      job.X = Xi;
      job.ldx = ld;
      job.xcs = (long)ns * ld;
      job.max_mvps = p.max_mvps;
      EigSel es;  // Sec. 4, Theorem 1: over the first k_select approximate eigenvectors instead
      if (job.project && (p.flags & GDR_FLAG_EIG_SELECT)) {
        const int ks = (p.k_select > 0 && p.k_select < defl->k) ? p.k_select : defl->k;
        std::vector<double> eres(ks);
        eigsel_setup(ctx, defl->Hk, defl->k, ks, sig[0], es, eres.data());
        for (double v : eres) rep.eig_resid_max = std::max(rep.eig_resid_max, v);
        job.eigsel = &es;
      }
      ProjResult pr = proj_batch<R>(ctx, A, job, !(p.flags & GDR_FLAG_NO_GRAPH));
      for (long v : pr.mvps) rep.mvps_proj += v;
      result = pr.status;
    };
    if (p.prec == GDR_PREC_MIXED)
      run(float{});
    else
      run(double{});
    stage_out(ctx, A, ns * nrhs, Xi, ld, X, kout);
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    tc_check(ctx);
    rep.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    rep.kernel_launches = ctx->launches - launches0;
  });
  if (report) *report = rep;
  return st != GDR_OK ? st : result;
}

gdr_status gdr_profile(gdr_ctx* ctx, int enable) {
  if (!ctx) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    for (auto& r : ctx->prof_pending) {
      ctx->ev_pool.push_back(r.a);
      ctx->ev_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    ctx->prof.clear();
    ctx->profile = enable != 0;
  });
}

gdr_status gdr_profile_report(gdr_ctx* ctx, char* buf, long len) {
  if (!ctx || !buf || len <= 0) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    for (auto& r : ctx->prof_pending) {
      float ms = 0;
      GDR_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      auto& g = ctx->prof[r.name];
      g.launches++;
      g.ms += ms;
      g.bytes += r.bytes;
      ctx->ev_pool.push_back(r.a);
      ctx->ev_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    std::string s = "{";
    bool first = true;
    for (auto& kv : ctx->prof) {
      char line[256];
      std::snprintf(line, sizeof(line), "%s\"%s\": {\"launches\": %ld, \"ms\": %.6f, \"bytes\": %.0f}",
                    first ? "" : ", ", kv.first.c_str(), kv.second.launches, kv.second.ms, kv.second.bytes);
      s += line;
      first = false;
    }
    s += "}";
    GDR_REQUIRE((long)s.size() < len, "profile report buffer too small");
    std::memcpy(buf, s.c_str(), s.size() + 1);
  });
}

gdr_status gdr_defl_export(gdr_ctx* ctx, const gdr_defl* defl, double* V, double* Hbar, int* k_out) {
  if (!ctx || !defl) return GDR_EINVAL;
  return guarded(ctx, [&] {
    if (k_out) *k_out = defl->k;
    if (V && defl->wilson_V)
      wilson_order<c128>(ctx, defl->wilson_V, defl->k + 1, defl->V128, defl->ldv, reinterpret_cast<c128*>(V),
                         defl->n, false);
    else if (V)
      GDR_CUDA(cudaMemcpy2DAsync(V, defl->n * sizeof(c128), defl->V128, defl->ldv * sizeof(c128),
                                 defl->n * sizeof(c128), defl->k + 1, cudaMemcpyDeviceToDevice, ctx->stream));
    if (Hbar) std::memcpy(Hbar, defl->Hk_host.data(), sizeof(c128) * defl->Hk_host.size());
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

void gdr_defl_destroy(gdr_defl* defl) {
  if (!defl) return;
  cudaFree(defl->V);
  cudaFree(defl->V128);
  cudaFree(defl->Hk);
  delete defl;
}

// ------------------------------------------------------------ step level

gdr_status gdr_arnoldi_step(gdr_ctx* ctx, const gdr_op* A, gdr_prec prec, void* V, int j, double* hcol) {
  if (!ctx || !A || !V || !hcol) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_REQUIRE(j >= 0 && j + 1 <= GDR_MAX_M, "j out of range");
    const long n = A->n;
    GDR_REQUIRE(prec == GDR_PREC_FP64 || n % 2 == 0, "complex64 step-level calls need an even n");
    auto run = [&](auto tag) {
      using R = decltype(tag);
      Batch<R> b;
      b.ncol = 1;
      b.n = n;
      b.m = j + 1;
      b.ns = 1;
      // Wilson: the basis in the library's pair-major order for the step, v_{j+1} back
      cx<R>* Vu = static_cast<cx<R>*>(V);
      cx<R>* Vl = Vu;
      if (A->kind == OP_WILSON) {
        Vl = ctx->get<cx<R>>("step.Vl", (size_t)n * (j + 2));
        op_order<cx<R>>(ctx, A, j + 1, Vu, n, Vl, n, true);
      }
      b.V = Vl;
      b.ldv = n;
      b.vcs = 0;
      b.W = ctx->get<cx<R>>("step.W", (size_t)pad_ld(n));
      b.W2 = ctx->get<cx<R>>("step.W2", (size_t)pad_ld(n));
      b.wcs = 0;
      b.H = ctx->get<c128>("step.H", (size_t)(j + 2) * (j + 1));
      b.cvec = nullptr;
      b.h1 = ctx->get<c128>("step.h1", (size_t)(j + 3));
      b.h2 = ctx->get<c128>("step.h2", (size_t)(j + 3));
      const long units = (n * (long)sizeof(cx<R>) + 15) / 16;
      b.nblk = (int)std::max<long>(1, std::min<long>((units + 255) / 256, 3L * ctx->num_sms));
      b.pstride = (long)(b.nblk + 64) * (j + 3);
      b.part = ctx->get<c128>("step.part", (size_t)b.pstride + 64);
      b.cnt = ctx->get<unsigned>("step.cnt", 4);
      b.gcnt = ctx->get<unsigned>("step.gcnt", 64);
      GDR_CUDA(cudaMemsetAsync(b.gcnt, 0, 64 * sizeof(unsigned), ctx->stream));
      b.st = ctx->get<ColState>("step.st", 1);
      b.sigma = nullptr;
      ColState s = {};
      s.run = 1;
      s.active = 1;
      s.m_eff = j + 1;
      GDR_CUDA(cudaMemsetAsync(b.cnt, 0, 4 * sizeof(unsigned), ctx->stream));
      GDR_CUDA(cudaMemcpyAsync(b.st, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->stream));
      GDR_CUDA(cudaStreamSynchronize(ctx->stream));
      cx<R>* wl = nullptr;
      arnoldi_step<R>(ctx, A, b, j, j, j, wl);
      if (Vl != Vu) op_order<cx<R>>(ctx, A, 1, Vl + (long)(j + 1) * n, n, Vu + (long)(j + 1) * n, n, false);
      GDR_CUDA(cudaMemcpyAsync(hcol, b.H + (long)j * (j + 2), sizeof(c128) * (j + 2), cudaMemcpyDeviceToDevice,
                               ctx->stream));
    };
    if (prec == GDR_PREC_FP64)
      run(double{});
    else
      run(float{});
  });
}

gdr_status gdr_arnoldi_cycle(gdr_ctx* ctx, const gdr_op* A, gdr_prec prec, void* V, int j0, int m, double* Hbar,
                             unsigned flags, int* m_eff) {
  if (!ctx || !A || !V || !Hbar) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_REQUIRE(m >= 1 && m <= GDR_MAX_M && j0 >= 0 && j0 < m, "bad j0 / m");
    const long n = A->n;
    GDR_REQUIRE(prec == GDR_PREC_FP64 || n % 2 == 0, "complex64 step-level calls need an even n");
    auto run = [&](auto tag) {
      using R = decltype(tag);
      Batch<R> b;
      b.ncol = 1;
      b.n = n;
      b.m = m;
      b.ns = 1;
      b.ldv = pad_ld(n);
      b.vcs = b.ldv * (m + 1);
      b.V = ctx->get<cx<R>>("cyc.V", (size_t)b.vcs);
      GDR_CUDA(cudaMemsetAsync(b.V, 0, sizeof(cx<R>) * b.vcs, ctx->stream));  // columns a breakdown leaves: 0
      // the given columns, in the library's vector order
      if (A->kind == OP_WILSON)
        op_order<cx<R>>(ctx, A, j0 + 1, static_cast<const cx<R>*>(V), n, b.V, b.ldv, true);
      else
        GDR_CUDA(cudaMemcpy2DAsync(b.V, b.ldv * sizeof(cx<R>), V, n * sizeof(cx<R>), n * sizeof(cx<R>), j0 + 1,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
      b.wcs = b.ldv;
      b.W = ctx->get<cx<R>>("cyc.W", (size_t)b.ldv);
      b.W2 = ctx->get<cx<R>>("cyc.W2", (size_t)b.ldv);
      b.H = ctx->get<c128>("cyc.H", (size_t)(m + 1) * m);
      GDR_CUDA(cudaMemsetAsync(b.H, 0, sizeof(c128) * (m + 1) * m, ctx->stream));
      if (j0 > 0)
        GDR_CUDA(cudaMemcpyAsync(b.H, Hbar, sizeof(c128) * (m + 1) * j0, cudaMemcpyDeviceToDevice, ctx->stream));
      b.cvec = nullptr;
      b.h1 = ctx->get<c128>("cyc.h1", (size_t)(m + 2));
      b.h2 = ctx->get<c128>("cyc.h2", (size_t)(m + 2));
      b.hd = ctx->get<c128>("cyc.hd", (size_t)(2 * m + 8));
      b.dc = ctx->get<c128>("cyc.dc", (size_t)(2 * m + 8));
      b.Hf = ctx->get<c64>("cyc.Hf", (size_t)(m + 1) * m);
      const long units = (n * (long)sizeof(cx<R>) + 15) / 16;
      b.nblk = (int)std::max<long>(1, std::min<long>((units + 255) / 256, 3L * ctx->num_sms));
      b.pstride = (long)(b.nblk + 64) * (2 * m + 8);
      b.part = ctx->get<c128>("cyc.part", (size_t)b.pstride + 64);
      b.cnt = ctx->get<unsigned>("cyc.cnt", 4);
      b.gcnt = ctx->get<unsigned>("cyc.gcnt", 64);
      GDR_CUDA(cudaMemsetAsync(b.gcnt, 0, 64 * sizeof(unsigned), ctx->stream));
      GDR_CUDA(cudaMemsetAsync(b.cnt, 0, 4 * sizeof(unsigned), ctx->stream));
      b.st = ctx->get<ColState>("cyc.st", 1);
      b.sigma = nullptr;
      ColState s = {};
      s.run = 1;
      s.active = 1;
      s.m_eff = m;
      GDR_CUDA(cudaMemcpyAsync(b.st, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->stream));
      if (std::is_same<R, float>::value && !(flags & GDR_FLAG_CGS2)) {
        arnoldi_dcgs2<R>(ctx, A, b, j0, m);
      } else {
        cx<R>* wl = nullptr;
        for (int j = j0; j < m; ++j) arnoldi_step<R>(ctx, A, b, j, j0, m - 1, wl);
      }
      if (A->kind == OP_WILSON)
        op_order<cx<R>>(ctx, A, m - j0, b.V + (long)(j0 + 1) * b.ldv, b.ldv,
                        static_cast<cx<R>*>(V) + (long)(j0 + 1) * n, n, false);
      else
        GDR_CUDA(cudaMemcpy2DAsync(static_cast<cx<R>*>(V) + (long)(j0 + 1) * n, n * sizeof(cx<R>),
                                   b.V + (long)(j0 + 1) * b.ldv, b.ldv * sizeof(cx<R>), n * sizeof(cx<R>), m - j0,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
      GDR_CUDA(cudaMemcpyAsync(Hbar + 2 * (long)(m + 1) * j0, b.H + (long)(m + 1) * j0,
                               sizeof(c128) * (m + 1) * (m - j0), cudaMemcpyDeviceToDevice, ctx->stream));
      ColState out;
      GDR_CUDA(cudaMemcpyAsync(&out, b.st, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
      GDR_CUDA(cudaStreamSynchronize(ctx->stream));
      if (m_eff) *m_eff = out.broke ? out.m_eff : m;
      if (out.nan) throw gdr_error(GDR_ENAN, "NaN/Inf in the Arnoldi recurrence");
    };
    if (prec == GDR_PREC_FP64)
      run(double{});
    else
      run(float{});
  });
}

gdr_status gdr_dense_gmres_sh(gdr_ctx* ctx, int m, int ns, const double* Hbar, const double* c, const double* sigma,
                              const double* beta, double* D, double* s, double* beta_new, double* norms) {
  if (!ctx) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_REQUIRE(m >= 1 && m <= GDR_MAX_M && ns >= 1, "bad sizes");
    GDR_REQUIRE(Hbar && c && sigma && beta && D && s && beta_new && norms, "null argument");
    DenseCycle d{};
    d.ncol = 1; d.m = m; d.k = 0; d.ns = ns; d.kfull = m + 1;  // general Hbar
    c128* H = ctx->get<c128>("dstep.H", (size_t)(m + 1) * m);
    c128* cv = ctx->get<c128>("dstep.c", (size_t)(m + 1));
    c128* sg = ctx->get<c128>("dstep.sigma", (size_t)ns);
    GDR_CUDA(cudaMemcpyAsync(H, Hbar, sizeof(c128) * (m + 1) * m, cudaMemcpyDeviceToDevice, ctx->stream));
    GDR_CUDA(cudaMemcpyAsync(cv, c, sizeof(c128) * (m + 1), cudaMemcpyDeviceToDevice, ctx->stream));
    GDR_CUDA(cudaMemcpyAsync(sg, sigma, sizeof(c128) * ns, cudaMemcpyHostToDevice, ctx->stream));
    d.H = H; d.cvec = cv; d.sigma = sg;
    d.beta = reinterpret_cast<c128*>(beta_new);
    GDR_CUDA(cudaMemcpyAsync(d.beta, beta, sizeof(c128) * ns, cudaMemcpyDeviceToDevice, ctx->stream));
    d.norms = norms;
    d.sact = ctx->get<int>("dstep.sact", (size_t)ns);
    std::vector<int> ones(ns, 1);
    GDR_CUDA(cudaMemcpyAsync(d.sact, ones.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, ctx->stream));
    d.ldc = m + 1;
    d.ccs = (long)(m + 1) * (ns + 1);
    d.Cf = ctx->get<c128>("dstep.Cf", (size_t)d.ccs);
    d.s = reinterpret_cast<c128*>(s);
    d.st = ctx->get<ColState>("dstep.st", 1);
    ColState st = {};
    st.active = 1;
    st.m_eff = m;
    GDR_CUDA(cudaMemcpyAsync(d.st, &st, sizeof(st), cudaMemcpyHostToDevice, ctx->stream));
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    dense_cycle(ctx, d);
    GDR_CUDA(cudaMemcpy2DAsync(D, m * sizeof(c128), d.Cf, (m + 1) * sizeof(c128), m * sizeof(c128), ns,
                               cudaMemcpyDeviceToDevice, ctx->stream));
    ColState out;
    GDR_CUDA(cudaMemcpyAsync(&out, d.st, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    if (out.err) throw gdr_error((gdr_status)out.err, "singular reduced system");
  });
}

gdr_status gdr_dense_ls(gdr_ctx* ctx, gdr_prec prec, int m, const double* sigma1, const double* Hbar, const double* c,
                        double* y, double* s) {
  if (!ctx) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_REQUIRE(m >= 1 && m <= GDR_MAX_M, "bad sizes");
    GDR_REQUIRE(prec == GDR_PREC_FP64 || prec == GDR_PREC_MIXED, "prec must be GDR_PREC_FP64 or GDR_PREC_MIXED");
    GDR_REQUIRE(sigma1 && Hbar && c && y && s, "null argument");
    DenseCycle d{};
    d.ncol = 1; d.m = m; d.k = 0; d.ns = 1; d.kfull = 0;  // Hessenberg recurrence
    d.ls32 = (prec == GDR_PREC_MIXED) ? 1 : 0;
    c128* sg = ctx->get<c128>("lstep.sigma", 1);
    GDR_CUDA(cudaMemcpyAsync(sg, sigma1, sizeof(c128), cudaMemcpyHostToDevice, ctx->stream));
    d.H = reinterpret_cast<const c128*>(Hbar);
    d.cvec = reinterpret_cast<const c128*>(c);
    d.sigma = sg;
    d.beta = ctx->get<c128>("lstep.beta", 1);
    d.norms = ctx->get<double>("lstep.norms", 1);
    d.sact = ctx->get<int>("lstep.sact", 1);
    const c128 one = {1.0, 0.0};
    const int on = 1;
    GDR_CUDA(cudaMemcpyAsync(d.beta, &one, sizeof(one), cudaMemcpyHostToDevice, ctx->stream));
    GDR_CUDA(cudaMemcpyAsync(d.sact, &on, sizeof(on), cudaMemcpyHostToDevice, ctx->stream));
    d.ldc = m + 1;
    d.ccs = (long)(m + 1) * 2;
    d.Cf = ctx->get<c128>("lstep.Cf", (size_t)d.ccs);
    d.s = reinterpret_cast<c128*>(s);
    d.st = ctx->get<ColState>("lstep.st", 1);
    ColState st = {};
    st.active = 1;
    st.m_eff = m;
    GDR_CUDA(cudaMemcpyAsync(d.st, &st, sizeof(st), cudaMemcpyHostToDevice, ctx->stream));
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    dense_cycle(ctx, d);
    GDR_CUDA(cudaMemcpyAsync(y, d.Cf, m * sizeof(c128), cudaMemcpyDeviceToDevice, ctx->stream));
    ColState out;
    GDR_CUDA(cudaMemcpyAsync(&out, d.st, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    if (out.err) throw gdr_error((gdr_status)out.err, "singular reduced system");
  });
}

gdr_status gdr_dense_restart(gdr_ctx* ctx, gdr_prec prec, int m, int k, const double* sigma1, const double* Hbar,
                             const double* s, double* theta, double* P, double* Hk, double* ck) {
  if (!ctx) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_REQUIRE(m >= 2 && m <= GDR_MAX_M && k >= 1 && k < m, "bad sizes");
    GDR_REQUIRE(prec == GDR_PREC_FP64 || prec == GDR_PREC_MIXED, "prec must be GDR_PREC_FP64 or GDR_PREC_MIXED");
    GDR_REQUIRE(sigma1 && Hbar && s && theta && P && Hk && ck, "null argument");
    DenseCycle d{};
    d.ncol = 1; d.m = m; d.k = k; d.ns = 1; d.kfull = m + 1;  // general Hbar
    d.hr32 = (prec == GDR_PREC_MIXED) ? 1 : 0;
    c128* sg = ctx->get<c128>("rstep.sigma", 1);
    GDR_CUDA(cudaMemcpyAsync(sg, sigma1, sizeof(c128), cudaMemcpyHostToDevice, ctx->stream));
    d.H = reinterpret_cast<const c128*>(Hbar);
    d.sigma = sg;
    d.s = const_cast<c128*>(reinterpret_cast<const c128*>(s));
    d.ldc = m + 1;
    d.ccs = (long)(m + 1) * (k + 1);
    d.Cf = reinterpret_cast<c128*>(P);
    d.Pk = ctx->get<c128>("rstep.Pk", (size_t)(m + 1) * k);
    d.Hk = reinterpret_cast<c128*>(Hk);
    d.ck = reinterpret_cast<c128*>(ck);
    d.theta = reinterpret_cast<c128*>(theta);
    d.scratch_per_col = (long)2 * ((long)m * m + 2L * m * k + 64);
    d.scratch = ctx->get<double>("rstep.scratch", (size_t)d.scratch_per_col);
    d.st = ctx->get<ColState>("rstep.st", 1);
    ColState st = {};
    st.active = 1;
    st.m_eff = m;
    GDR_CUDA(cudaMemcpyAsync(d.st, &st, sizeof(st), cudaMemcpyHostToDevice, ctx->stream));
    dense_restart(ctx, d);
    ColState out;
    GDR_CUDA(cudaMemcpyAsync(&out, d.st, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    if (out.err) throw gdr_error((gdr_status)out.err, "harmonic Ritz restart failed");
  });
}

gdr_status gdr_barrier_selftest(gdr_ctx* ctx, int rounds, int phantom) {
  if (!ctx) return GDR_EINVAL;
  gdr_status r = GDR_OK;
  const gdr_status g = guarded(ctx, [&] {
    GDR_REQUIRE(rounds >= 1 && rounds <= 1000000, "rounds must be in [1, 1e6]");
    r = barrier_selftest(ctx, rounds, phantom ? 1 : 0);
    if (r != GDR_OK) ctx->err = "grid barrier gave up (spin bound reached)";
  });
  return g != GDR_OK ? g : r;
}

gdr_status gdr_basis_update(gdr_ctx* ctx, gdr_prec prec, long n, int nv, void* V, const double* C, int nout, int nx,
                            double* X) {
  if (!ctx) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_REQUIRE(n > 0 && nv >= 1 && nout >= 0 && nout <= nv && nx >= 0, "bad sizes");
    GDR_REQUIRE(V && C && (nx == 0 || X), "null argument");
    if (prec == GDR_PREC_FP64)
      combine<double>(ctx, n, 1, static_cast<c128*>(V), n, 0, nv, reinterpret_cast<const c128*>(C), nv, 0, nout, nx,
                      0, reinterpret_cast<c128*>(X), n, 0, nullptr, 0, nullptr);
    else
      combine<float>(ctx, n, 1, static_cast<c64*>(V), n, 0, nv, reinterpret_cast<const c128*>(C), nv, 0, nout, nx, 0,
                     reinterpret_cast<c128*>(X), n, 0, nullptr, 0, nullptr);
  });
}

gdr_status gdr_basis_dot(gdr_ctx* ctx, gdr_prec prec, long n, int nv, const void* V, int ncol, const void* R, long ldr,
                         double* C, unsigned flags) {
  if (!ctx) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_REQUIRE(n > 0 && nv >= 1 && nv <= GDR_MAX_M + 1 && ncol >= 1 && ldr >= n, "bad sizes");
    GDR_REQUIRE(V && R && C, "null argument");
    GDR_CUDA(cudaSetDevice(ctx->device));
    ctx->tc_proj = !(flags & GDR_FLAG_NO_TENSOR_CORES);
    auto run = [&](auto zero) {
      using R_ = decltype(zero);
      Batch<R_> b;
      b.ncol = ncol;
      b.n = n;
      b.m = nv;
      b.V = static_cast<cx<R_>*>(const_cast<void*>(V));
      b.ldv = n;
      b.vcs = 0;
      const long units = (n * (long)sizeof(cx<R_>) + 15) / 16;
      b.nblk = (int)std::max<long>(1, std::min<long>((units + 255) / 256, 3L * ctx->num_sms));
      b.pstride = (long)(b.nblk + 64) * (nv + 3);
      b.part = ctx->get<c128>("bdot.part", (size_t)b.pstride * ncol + 64);
      b.cnt = ctx->get<unsigned>("bdot.cnt", (size_t)4 * ncol);
      b.gcnt = ctx->get<unsigned>("bdot.gcnt", (size_t)64 * ncol);
      GDR_CUDA(cudaMemsetAsync(b.cnt, 0, 4 * sizeof(unsigned) * ncol, ctx->stream));
      GDR_CUDA(cudaMemsetAsync(b.gcnt, 0, 64 * sizeof(unsigned) * ncol, ctx->stream));
      b.st = ctx->get<ColState>("bdot.st", (size_t)ncol);
      ColState s0 = {};
      s0.run = 1;
      s0.active = 1;
      s0.m_eff = nv;
      std::vector<ColState> sv(ncol, s0);
      GDR_CUDA(cudaMemcpyAsync(b.st, sv.data(), sizeof(ColState) * ncol, cudaMemcpyHostToDevice, ctx->stream));
      c128* h = ctx->get<c128>("bdot.h", (size_t)(nv + 2) * ncol);
      gs_dot_shared_reserve(ctx, n, ncol, nv);
      gs_dot<R_>(ctx, b, nv, static_cast<const cx<R_>*>(R), ldr, h, false, nullptr);
      GDR_CUDA(cudaMemcpy2DAsync(C, sizeof(c128) * nv, h, sizeof(c128) * (nv + 2), sizeof(c128) * nv, ncol,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
      GDR_CUDA(cudaStreamSynchronize(ctx->stream));
      tc_check(ctx);
    };
    if (prec == GDR_PREC_FP64)
      run(double{});
    else
      run(float{});
  });
}

gdr_status gdr_basis_residual_update(gdr_ctx* ctx, gdr_prec prec, long n, int nv, const void* V, int ncol,
                                     const double* T, void* R, long ldr, unsigned flags) {
  if (!ctx) return GDR_EINVAL;
  return guarded(ctx, [&] {
    GDR_REQUIRE(n > 0 && nv >= 1 && nv <= GDR_MAX_M + 1 && ncol >= 1 && ldr >= n, "bad sizes");
    GDR_REQUIRE(V && T && R, "null argument");
    GDR_CUDA(cudaSetDevice(ctx->device));
    ctx->tc_proj = !(flags & GDR_FLAG_NO_TENSOR_CORES);
    ColState* st = ctx->get<ColState>("bres.st", (size_t)ncol);
    ColState s0 = {};
    s0.run = 1;
    s0.active = 1;
    std::vector<ColState> sv(ncol, s0);
    GDR_CUDA(cudaMemcpyAsync(st, sv.data(), sizeof(ColState) * ncol, cudaMemcpyHostToDevice, ctx->stream));
    gs_dot_shared_reserve(ctx, n, ncol, nv);
    const c128* Tc = reinterpret_cast<const c128*>(T);
    if (prec == GDR_PREC_FP64)
      combine<double>(ctx, n, ncol, static_cast<c128*>(const_cast<void*>(V)), n, 0, nv, Tc, nv, nv, 0, 0, 2, nullptr,
                      0, 0, static_cast<c128*>(R), ldr, st);
    else
      combine<float>(ctx, n, ncol, static_cast<c64*>(const_cast<void*>(V)), n, 0, nv, Tc, nv, nv, 0, 0, 2, nullptr, 0,
                     0, static_cast<c64*>(R), ldr, st);
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    tc_check(ctx);
  });
}

}  // extern "C"
