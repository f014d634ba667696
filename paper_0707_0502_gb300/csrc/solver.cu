// Solver drivers (host code + small kernels).
//
//  dr_sh      GMRES-DR(m,k)-Sh for one right-hand side (Sec. 3, algorithm
//             "GMRES-DR-Sh"): each cycle extends the recurrence, solves the
//             reduced problems of every shift, restarts with k harmonic Ritz
//             vectors and updates all solutions in one pass over the basis.
//  proj_batch GMRES(m_p)-Proj(k)-Sh (Sec. 4) on a batch of columns in lockstep:
//             Minres projection over the kept V_k, then one GMRES(m_p)-Sh
//             cycle per column; every column has its own Krylov basis but the
//             matvec is one multi-column launch.
//  solve      Sec. 4 pipeline (Example 5 order) + correction phase, FP64 true
//             residuals, and (MIXED) iterative refinement of every (shift, rhs)
//             pair by batched single-shift Proj solves, with an FP64 cleanup.
//
// One cycle is a fixed sequence of kernels on the context stream; it is
// captured once into a CUDA graph and replayed.  The host reads one small
// status block per cycle.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <limits>
#include <functional>
#include <type_traits>

#include "kernels.cuh"
#include "solver.cuh"

namespace {

__global__ void init_cols_kernel(ColState* st, int ncol, const double* bn2, const double* tolv, const int* mask,
                                 int ns, int* sact, c128* beta, c128* gamma, double* norms) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  const double bn = sqrt(bn2[c]);
  ColState s = {};
  s.run = 0;
  s.active = (mask ? mask[c] : 1) && bn > 0 && isfinite(bn);
  s.bnorm = bn;
  s.tol = tolv[c];
  s.rnorm = bn;
  s.conv = s.active ? 0 : 1;
  st[c] = s;
  for (int i = 0; i < ns; ++i) {
    sact[(long)c * ns + i] = 1;
    beta[(long)c * ns + i] = {1, 0};
    if (gamma) gamma[(long)c * ns + i] = {0, 0};
    norms[(long)c * ns + i] = bn;
  }
}

__global__ void set_run_kernel(ColState* st, int ncol) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncol) st[c].run = st[c].active;
}

// normalise V[:, j] of every column with ||.||^2 in nrm2[c]
template <typename R>
__global__ void normalize_kernel(cx<R>* V, long ldv, long vcs, int j, long n, const double* nrm2, const ColState* st,
                                 const int* nvec) {
  const int c = blockIdx.y;
  if (st && !st[c].active) return;
  if (nvec) n = nvec[c];
  const double nn = nrm2[c];
  if (!(nn > 0)) return;
  const R s = (R)(1.0 / sqrt(nn));
  cx<R>* v = V + c * vcs + (long)j * ldv;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) v[i] = s * v[i];
}

// s_i <- s_i / (1 - gamma_i) for i >= 1 (extra right-hand side correction)
__global__ void extra_scale_kernel(long n, int ns, const c128* gam, c128* S, long lds) {
  const int i = blockIdx.y + 1;
  const c128 g = gam[i];
  const c128 one_minus = {1.0 - g.x, -g.y};
  const double d = one_minus.x * one_minus.x + one_minus.y * one_minus.y;
  const c128 f = {one_minus.x / d, -one_minus.y / d};
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x)
    S[(long)i * lds + r] = f * S[(long)i * lds + r];
}

// X[:, j*ns + i] += gam[j*ns + i] * S[:, i] for i >= 1, every rhs j of the batch
__global__ void correct_kernel(long n, int ns, const c128* gam, const c128* S, long lds, c128* X, long ldx) {
  const int p = blockIdx.y;  // pair index j*ns + i
  const int i = p % ns;
  if (i == 0) return;
  const c128 g = gam[p];
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x)
    X[(long)p * ldx + r] += g * S[(long)i * lds + r];
}

// Residuals after the correction, without a matvec: with s_i = s~_i / (1 - gs_i) and
// r^s_i = v - (A - sigma_i) s~_i, (A - sigma_i) s_i = (v - r^s_i) / (1 - gs_i), so
// x_i += g_i s_i turns r_i into r_i - g_i / (1 - gs_i) (v - r^s_i) (i >= 1; i = 0 is not
// corrected).  Pairs p = j*ns + i of the right-hand sides j of the batch; Rs = the extra
// system's residuals r^s_i, gs = its gamma_i; Rin / Rout at stride ld per pair.
__global__ void corrected_resid_kernel(long n, int ns, const c128* gam, const c128* gs, const c128* v, const c128* Rs,
                                       const c128* Rin, c128* Rout, long ld) {
  const int p = blockIdx.y, i = p % ns;
  c128 f = {0, 0};
  if (i > 0) {
    const c128 om = {1.0 - gs[i].x, -gs[i].y};
    const double d = om.x * om.x + om.y * om.y;
    f = gam[p] * c128{om.x / d, -om.y / d};
  }
  const c128* ri = Rin + (long)p * ld;
  c128* ro = Rout + (long)p * ld;
  const c128* rs = Rs + (long)i * ld;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x)
    ro[r] = i > 0 ? ri[r] - f * (v[r] - rs[r]) : ri[r];
}

// Related right-hand sides (Sec. 5, eqs. relrhs1-relrhs2).  M is the j x (j+1)
// augmented system [B^H B | B^H b_j] (row-major, FP64, overwritten); d solves it by
// Gaussian elimination with partial pivoting, one warp (lanes stride the rows).  A
// column with no usable pivot (linearly dependent right-hand sides) gets d = 0.
__global__ void related_solve_kernel(int j, c128* M, c128* d) {
  const int lane = threadIdx.x;
  const int w = j + 1;
  for (int p = 0; p < j; ++p) {
    double best = -1.0;
    int piv = p;
    for (int r = p + lane; r < j; r += 32) {
      const double a = norm2(M[r * w + p]);
      if (a > best) {
        best = a;
        piv = r;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, piv, o);
      if (ob > best || (ob == best && op < piv)) {
        best = ob;
        piv = op;
      }
    }
    if (piv != p)
      for (int c = p + lane; c < w; c += 32) {
        const c128 t = M[p * w + c];
        M[p * w + c] = M[piv * w + c];
        M[piv * w + c] = t;
      }
    __syncwarp();
    const c128 pv = M[p * w + p];
    const double pn = norm2(pv);
    if (pn > 0.0) {
      const c128 inv = {pv.x / pn, -pv.y / pn};
      for (int r = p + 1 + lane; r < j; r += 32) {
        const c128 f = M[r * w + p] * inv;
        for (int c = p; c < w; ++c) M[r * w + c] -= f * M[p * w + c];
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    for (int p = j - 1; p >= 0; --p) {
      c128 acc = M[p * w + j];
      for (int c = p + 1; c < j; ++c) acc -= M[p * w + c] * d[c];
      const c128 pv = M[p * w + p];
      const double pn = norm2(pv);
      d[p] = pn > 0.0 ? acc * c128{pv.x / pn, -pv.y / pn} : c128{0.0, 0.0};
    }
  }
}

// guesses X_j[:, i] = sum_r d_r X_r[:, i] for every shift i (blockIdx.y < ns) and the
// common residual res = b_j - sum_r d_r b_r (blockIdx.y == ns); X_r[:, i] at X + (r ns + i) ldx
__global__ void related_guess_kernel(long n, int ns, int j, const c128* __restrict__ d, c128* X, long ldx,
                                     const c128* __restrict__ B, long ldb, c128* __restrict__ res) {
  const int i = blockIdx.y;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    c128 acc = {0.0, 0.0};
    if (i < ns) {
      for (int r = 0; r < j; ++r) acc += d[r] * X[((long)r * ns + i) * ldx + e];
      X[((long)j * ns + i) * ldx + e] = acc;
    } else {
      for (int r = 0; r < j; ++r) acc += d[r] * B[(long)r * ldb + e];
      res[e] = B[(long)j * ldb + e] - acc;
    }
  }
}

// D_c += Cp_c[:, 0:ns] ((k+1) x ns per column, leading dimension k+1) for the active columns:
// the projection's solution coefficients summed over the cycles of a Proj batch, so that
// x_i += V_k d_i is applied once at the end instead of every cycle
// X[c][i] += E[c][i] (FP64 += complex64): the summed corrections of a Proj batch
template <typename R>
__global__ void add_correction_kernel(long n, int ns, const cx<R>* __restrict__ E, long ldx, long xcs, c128* X,
                                      const int* nvec) {
  const int c = blockIdx.y / ns, i = blockIdx.y % ns;
  const long nc = nvec ? nvec[c] : n;
  const cx<R>* e = E + c * xcs + (long)i * ldx;
  c128* x = X + c * xcs + (long)i * ldx;
  for (long r = blockIdx.x * 256L + threadIdx.x; r < nc; r += (long)gridDim.x * 256) x[r] = x[r] + up(e[r]);
}

__global__ void dacc_kernel(int k1, int ns, const c128* __restrict__ Cp, long ccs, c128* D, const ColState* st) {
  const int c = blockIdx.y;
  if (!st[c].active) return;
  for (int t = threadIdx.x; t < k1 * ns; t += blockDim.x) D[(long)c * k1 * ns + t] += Cp[c * ccs + t];
}

// X[:, q] += Y[:, q], q < cols
__global__ void add_cols_kernel(long n, const c128* __restrict__ Y, long ldy, c128* X, long ldx) {
  const int q = blockIdx.y;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    X[(long)q * ldx + e] += Y[(long)q * ldy + e];
}

unsigned grid1(gdr_ctx* ctx, long n) {
  long g = (n + 255) / 256;
  long cap = (long)ctx->num_sms * 8;
  return (unsigned)std::max(1L, std::min(g, cap));
}

struct Graph {
  cudaGraphExec_t exec = nullptr;
  long nodes = 0;
  ~Graph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

void run_cycle(gdr_ctx* ctx, bool use_graph, Graph& g, const std::function<void()>& enqueue) {
  if (!use_graph || ctx->profile) {  // per-kernel events need direct launches
    enqueue();
    return;
  }
  if (!g.exec) {
    const long before = ctx->launches;
    GDR_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue();
    } catch (...) {
      cudaGraph_t gg;
      cudaStreamEndCapture(ctx->stream, &gg);
      if (gg) cudaGraphDestroy(gg);
      throw;
    }
    cudaGraph_t gg;
    GDR_CUDA(cudaStreamEndCapture(ctx->stream, &gg));
    GDR_CUDA(cudaGraphInstantiate(&g.exec, gg, 0));
    GDR_CUDA(cudaGraphDestroy(gg));
    g.nodes = ctx->launches - before;
    ctx->launches = before;
  }
  GDR_CUDA(cudaGraphLaunch(g.exec, ctx->stream));
  ctx->launches += g.nodes;
}

// host wait on the context stream (counted in the report)
void stream_sync(gdr_ctx* ctx) {
  GDR_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->syncs++;
}

// Grid of the Gram-Schmidt reduction kernels: enough 256-thread blocks for one
// 16-byte unit per thread, at most 3 per SM (all resident in one wave at the
// register use of the dot kernel).
template <typename R>
int nblk_for(gdr_ctx* ctx, long n) {
  const long units = (n * (long)sizeof(cx<R>) + 15) / 16;
  long g = (units + 255) / 256;
  g = std::min<long>(g, 3L * ctx->num_sms);
  return (int)std::max<long>(g, 1);
}

// Allocate a batch of `ncol` Krylov spaces of size m (workspace names prefixed by tag).
template <typename R>
Batch<R> make_batch(gdr_ctx* ctx, const std::string& tag, long n, int ncol, int m, int ns, int hmin = 0) {
  Batch<R> b;
  b.ncol = ncol;
  b.n = n;
  b.m = m;
  b.ns = ns;
  b.ldv = pad_ld(n);
  b.vcs = b.ldv * (m + 1);
  b.V = ctx->get<cx<R>>(tag + ".V", (size_t)b.vcs * ncol);
  b.wcs = b.ldv;
  b.W = ctx->get<cx<R>>(tag + ".W", (size_t)b.wcs * ncol);
  b.W2 = ctx->get<cx<R>>(tag + ".W2", (size_t)b.wcs * ncol);
  b.H = ctx->get<c128>(tag + ".H", (size_t)(m + 1) * m * ncol);
  b.cvec = ctx->get<c128>(tag + ".c", (size_t)(m + 1) * ncol);
  b.h1 = ctx->get<c128>(tag + ".h1", (size_t)(m + 2) * ncol);
  b.h2 = ctx->get<c128>(tag + ".h2", (size_t)(m + 2) * ncol);
  b.hd = ctx->get<c128>(tag + ".hd", (size_t)(2 * m + 8) * ncol);
  b.dc = ctx->get<c128>(tag + ".dc", (size_t)(2 * m + 8) * ncol);
  b.Hf = ctx->get<c64>(tag + ".Hf", (size_t)(m + 1) * m * ncol);
  b.nblk = nblk_for<R>(ctx, n);
  // block partials, then slot-group partials (DCGS2 dot pass: 2m + 8 values per slot)
  b.pstride = (long)(b.nblk + 64) * std::max(2 * m + 8, hmin);
  b.part = ctx->get<c128>(tag + ".part", (size_t)b.pstride * ncol + 64);
  b.cnt = ctx->get<unsigned>(tag + ".cnt", (size_t)4 * ncol);
  b.gcnt = ctx->get<unsigned>(tag + ".gcnt", (size_t)64 * ncol);
  GDR_CUDA(cudaMemsetAsync(b.gcnt, 0, sizeof(unsigned) * 64 * ncol, ctx->stream));
  GDR_CUDA(cudaMemsetAsync(b.cnt, 0, sizeof(unsigned) * 4 * ncol, ctx->stream));
  b.st = ctx->get<ColState>(tag + ".st", (size_t)ncol);
  b.sigma = ctx->get<c128>(tag + ".sigma", (size_t)ns * ncol);
  ctx->get<double>("start_rn2", (size_t)ncol + 4);  // used inside captured cycles: allocate now
  return b;
}

struct Shifted {  // per-column shift bookkeeping
  int* sact;
  c128* beta;
  c128* gamma;
  double* norms;
};

// vector length of column c (a CSR batch: the rows of problem c / cpp), and the sum over
// every `every`-th of ncol columns (host side: the profiler's algorithmic byte counts)
double len_of(const gdr_op* A, int c, int cpp) {
  return A->kind == OP_CSR_BATCH ? (double)A->nrow_host[c / cpp] : (double)A->n;
}
double len_sum(const gdr_op* A, int ncol, int cpp, int every = 1) {
  double t = 0;
  for (int c = 0; c < ncol; c += every) t += len_of(A, c, cpp);
  return t;
}

Shifted make_shifted(gdr_ctx* ctx, const std::string& tag, int ncol, int ns) {
  Shifted s;
  s.sact = ctx->get<int>(tag + ".sact", (size_t)ncol * ns);
  s.beta = ctx->get<c128>(tag + ".beta", (size_t)ncol * ns);
  s.gamma = ctx->get<c128>(tag + ".gamma", (size_t)ncol * ns);
  s.norms = ctx->get<double>(tag + ".norms", (size_t)ncol * ns);
  return s;
}

template <typename R>
void reorth_column(gdr_ctx* ctx, const Batch<R>& b, int j, double* nrm2) {
  // classical Gram-Schmidt twice of v_j against v_0..v_{j-1}, then normalise
  cx<R>* vj = b.V + (long)j * b.ldv;
  gs_dot<R>(ctx, b, j, vj, b.vcs, b.h1, false);
  gs_update<R>(ctx, b, j, vj, b.vcs, b.h1, false);
  gs_dot<R>(ctx, b, j, vj, b.vcs, b.h1, false);
  gs_update<R>(ctx, b, j, vj, b.vcs, b.h1, false);
  norms2<cx<R>>(ctx, b.n, b.ncol, vj, b.vcs, nrm2, b.part, b.nblk, b.cnt, b.nvec);
  dim3 g(grid1(ctx, b.n), (unsigned)b.ncol);
  normalize_kernel<R><<<g, 256, 0, ctx->stream>>>(b.V, b.ldv, b.vcs, j, b.n, nrm2, b.st, b.nvec);
  GDR_LAUNCHED(ctx);
}

// ---- shift-shared refinement helpers (not in the paper)

// Pivoted Cholesky of a Hermitian positive semidefinite Gram matrix G (nc x nc,
// column-major): G ~= L L^H with L (nc x p, column-major), column t of L belonging to
// pivot piv[t] (L[piv[s], t] = 0 for t > s).  Pivots are taken greedily (largest
// remaining diagonal) until the trace of the remaining Schur complement is <= thr2
// or p == pmax.  Returns p.
int pivoted_cholesky(const std::vector<c128>& G, int nc, double thr2, int pmax, std::vector<c128>& L,
                     std::vector<int>& piv) {
  std::vector<double> d(nc);
  std::vector<char> used(nc, 0);
  for (int i = 0; i < nc; ++i) d[i] = G[i + (long)i * nc].x;
  L.assign((size_t)nc * std::max(pmax, 1), c128{0, 0});
  piv.clear();
  int p = 0;
  while (p < pmax) {
    double tr = 0, best = 0;
    int pv = -1;
    for (int i = 0; i < nc; ++i)
      if (!used[i]) {
        tr += std::max(d[i], 0.0);
        if (d[i] > best) {
          best = d[i];
          pv = i;
        }
      }
    if (pv < 0 || tr <= thr2) break;
    const double lpp = std::sqrt(best);
    for (int i = 0; i < nc; ++i) {
      if (used[i]) continue;
      c128 v = G[i + (long)pv * nc];
      for (int t = 0; t < p; ++t) v -= L[i + (long)t * nc] * conj(L[pv + (long)t * nc]);
      L[i + (long)p * nc] = (1.0 / lpp) * v;
    }
    L[pv + (long)p * nc] = {lpp, 0.0};
    for (int i = 0; i < nc; ++i)
      if (!used[i] && i != pv) d[i] -= norm2(L[i + (long)p * nc]);
    used[pv] = 1;
    piv.push_back(pv);
    ++p;
  }
  return p;
}

// Y = R W with orthonormal columns for the pivoted Cholesky factor L of R^H R:
// Y = R_piv L_piv^{-H}, so W[piv[s], t] = (L_piv^{-H})[s, t] (upper triangular,
// column-major nc x p), zero in the other rows.
std::vector<c128> orth_weights(const std::vector<c128>& L, const std::vector<int>& piv, int nc) {
  const int p = (int)piv.size();
  // M = L_piv^{-1} (lower triangular, p x p) by forward substitution, then W = M^H
  std::vector<c128> M((size_t)p * p, c128{0, 0});
  for (int t = 0; t < p; ++t) {  // column t of L_piv^{-1}: solve L_piv x = e_t
    for (int s = 0; s < p; ++s) {
      c128 v = {s == t ? 1.0 : 0.0, 0.0};
      for (int u = 0; u < s; ++u) v -= L[piv[s] + (long)u * nc] * M[u + (long)t * p];
      const c128 dg = L[piv[s] + (long)s * nc];
      const double dn = norm2(dg);
      M[s + (long)t * p] = (1.0 / dn) * (conj(dg) * v);
    }
  }
  std::vector<c128> W((size_t)nc * p, c128{0, 0});
  for (int s = 0; s < p; ++s)
    for (int t = 0; t < p; ++t) W[piv[s] + (long)t * nc] = conj(M[t + (long)s * p]);
  return W;
}

// X[:, i] += sum_t C[t, i] Z[:, t*ns + i] for the shifts i of one right-hand side whose
// flag act[i] is set (C: p x ns column-major, device; Z: FP64 columns at stride ldz)
__global__ void shared_apply_kernel(long n, int ns, int p, const c128* __restrict__ C, const int* __restrict__ act,
                                    const c128* __restrict__ Z, long ldz, c128* X, long ldx) {
  const int i = blockIdx.y;
  if (!act[i]) return;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    c128 acc = {0, 0};
    for (int t = 0; t < p; ++t) acc += C[t + (long)i * p] * Z[((long)t * ns + i) * ldz + e];
    X[(long)i * ldx + e] += acc;
  }
}

std::vector<ColState> read_states(gdr_ctx* ctx, const ColState* st, int ncol) {
  ColState* h = static_cast<ColState*>(ctx->host_status(sizeof(ColState) * ncol));
  GDR_CUDA(cudaMemcpyAsync(h, st, sizeof(ColState) * ncol, cudaMemcpyDeviceToHost, ctx->stream));
  stream_sync(ctx);
  return std::vector<ColState>(h, h + ncol);
}

}  // namespace

// ------------------------------------------------------------- GMRES-DR-Sh

template <typename R>
DrResult dr_sh(gdr_ctx* ctx, const gdr_op* A, const DrJob<R>& job, bool use_graph) {
  const long n = A->n;
  const int ncol = job.ncol, ns = job.ns, m = job.m, k = job.k;
  Batch<R> b = make_batch<R>(ctx, "dr", n, ncol, m, ns);
  b.nvec = job.nvec;
  b.cpp = job.cpp;
  b.ntot = len_sum(A, ncol, job.cpp);
  Shifted sh = make_shifted(ctx, "dr", ncol, ns);
  GDR_CUDA(cudaMemcpyAsync(b.sigma, job.sigma.data(), sizeof(c128) * ns * ncol, cudaMemcpyHostToDevice,
                           ctx->stream));
  const int ldc = m + 1;
  const int ncf = k + 1 + ns + 1;
  DenseCycle d{};
  d.ncol = ncol; d.m = m; d.k = k; d.ns = ns; d.kfull = k;
  d.H = b.H; d.cvec = b.cvec; d.sigma = b.sigma;
  d.beta = sh.beta; d.norms = sh.norms; d.sact = sh.sact;
  d.ccs = (long)ldc * ncf; d.ldc = ldc;
  d.Cf = ctx->get<c128>("dr.Cf", (size_t)d.ccs * ncol);
  d.s = ctx->get<c128>("dr.s", (size_t)(m + 1) * ncol);
  d.Pk = ctx->get<c128>("dr.Pk", (size_t)(m + 1) * std::max(k, 1) * ncol);
  d.Hk = ctx->get<c128>("dr.Hk", (size_t)(k + 1) * std::max(k, 1) * ncol);
  d.ck = ctx->get<c128>("dr.ck", (size_t)(k + 1) * ncol);
  d.theta = ctx->get<c128>("dr.theta", (size_t)m * ncol);
  d.scratch_per_col = (long)2 * ((long)m * m + 2L * m * std::max(k, 1) + 64);
  d.scratch = ctx->get<double>("dr.scratch", (size_t)d.scratch_per_col * ncol);
  d.st = b.st;
  d.want_r = (k == 0);  // GMRES(m): restart from the residual vector r = V_{m+1} s
  d.hr32 = (std::is_same<R, float>::value && job.eig32) ? 1 : 0;  // complex64 basis: FP32 eigensolve in the restart
  d.fom = job.fom ? 1 : 0;
  cx<R>* rres = ctx->get<cx<R>>("dr.r", (size_t)b.ldv * ncol);
  double* bn2 = ctx->get<double>("dr.bn2", (size_t)ncol + 4);
  double* nrm2 = ctx->get<double>("dr.nrm2", (size_t)ncol + 4);
  double* tolv = ctx->get<double>("dr.tol", (size_t)ncol + 4);
  GDR_CUDA(cudaMemcpyAsync(tolv, job.tol.data(), sizeof(double) * ncol, cudaMemcpyHostToDevice, ctx->stream));
  norms2<cx<R>>(ctx, n, ncol, job.rhs, job.ldrhs, bn2, b.part, b.nblk, b.cnt, b.nvec);
  init_cols_kernel<<<(ncol + 31) / 32, 32, 0, ctx->stream>>>(b.st, ncol, bn2, tolv, nullptr, ns, sh.sact, sh.beta,
                                                              sh.gamma, sh.norms);
  GDR_LAUNCHED(ctx);
  start_cycle<R>(ctx, b, job.rhs, job.ldrhs);

  const bool sweep = job.sweep && sweep_fits<R>(ctx, A, b) &&
                    sweep_choice(A, std::is_same<R, double>::value, ncol, m) != 0;
  if (sweep) sweep_reserve<R>(ctx, b);
  Graph g_first, g_next;
  DrResult res;
  res.k_eff = k;
  res.col_mvps.assign(ncol, 0);
  res.col_conv.assign(ncol, 0);
  std::vector<int> done(ncol, 0);
  int j0 = 0;
  for (;;) {
    const int jstart = j0;
    auto enqueue = [&]() {
      set_run_kernel<<<(ncol + 31) / 32, 32, 0, ctx->stream>>>(b.st, ncol);
      GDR_LAUNCHED(ctx);
      if (sweep) {
        arnoldi_sweep<R>(ctx, A, b, jstart, m);
        scale_into<R>(ctx, b, m, b.W2, b.wcs);
      } else if (std::is_same<R, float>::value && job.dcgs2) {
        arnoldi_dcgs2<R>(ctx, A, b, jstart, m);
      } else {
        cx<R>* wl = nullptr;
        for (int j = jstart; j < m; ++j) arnoldi_step<R>(ctx, A, b, j, jstart, m - 1, wl);
      }
      dense_cycle(ctx, d);
      // restart (V_{k+1} <- V_{m+1} P_{k+1}) fused with x_i += V_m d_i
      combine<R>(ctx, n, ncol, b.V, b.ldv, b.vcs, m + 1, d.Cf, ldc, d.ccs, k > 0 ? k + 1 : 0, ns, k > 0 ? 0 : 1,
                 job.X, job.ldx, job.xcs, rres, b.ldv, b.st, b.nvec, 1, col_len(b));
      if (k > 0) reorth_column<R>(ctx, b, k, nrm2);
      cycle_finish(ctx, d, b.H, b.cvec);
    };
    run_cycle(ctx, use_graph, jstart == 0 ? g_first : g_next, enqueue);
    const std::vector<ColState> st = read_states(ctx, b.st, ncol);
    res.cycles++;
    bool any_active = false;
    long mx = 0;
    for (int c = 0; c < ncol; ++c) {
      if (done[c]) continue;
      res.col_mvps[c] += st[c].broke ? (st[c].m_eff - jstart) : (m - jstart);
      mx = std::max(mx, res.col_mvps[c]);
      if (st[c].nan) res.status = GDR_ENAN;
      else if (st[c].err && res.status == GDR_OK) res.status = (gdr_status)st[c].err;
      if (st[c].conv) res.col_conv[c] = 1;
      if (st[c].broke && c == 0) res.broke = true;
      if (st[c].broke) res.any_broke = true;
      if (st[c].active) any_active = true;
      else done[c] = 1;
    }
    res.mvps = std::max(res.mvps, mx);
    if (!any_active) break;
    if (mx >= job.max_mvps || (job.max_cycles > 0 && res.cycles >= job.max_cycles)) {
      if (res.status == GDR_OK) res.status = GDR_ENOCONV;
      break;
    }
    j0 = k;
    if (k == 0) start_cycle<R>(ctx, b, rres, b.ldv);
  }
  res.V = b.V;
  res.ldv = b.ldv;
  res.vcs = b.vcs;
  res.Hk = d.Hk;
  res.valid_defl = (k > 0) && !res.broke && res.status != GDR_ENAN && res.status != GDR_EBREAKDOWN;
  std::vector<double> nr((size_t)ns * ncol);
  GDR_CUDA(cudaMemcpyAsync(nr.data(), sh.norms, sizeof(double) * ns * ncol, cudaMemcpyDeviceToHost, ctx->stream));
  stream_sync(ctx);
  res.norms = nr;
  return res;
}

template <typename R>
void tune_arnoldi(gdr_ctx* ctx, const gdr_op* A, int ncol, int m, double& t_sweep, double& t_launch, int& choice) {
  t_sweep = t_launch = 0;
  choice = -1;
  Batch<R> probe;  // sizes only: no workspace unless the sweep applies
  probe.n = A->n;
  probe.ncol = ncol;
  probe.m = m;
  if (!sweep_fits<R>(ctx, A, probe)) return;
  Batch<R> b = make_batch<R>(ctx, "tune", A->n, ncol, m, 1);
  if (A->kind == OP_CSR_BATCH) {  // column c: problem c / cpp, its own length
    b.cpp = ncol / A->nprob;
    std::vector<int> nv(ncol);
    for (int c = 0; c < ncol; ++c) nv[c] = (int)A->nrow_host[c / b.cpp];
    int* nvd = ctx->get<int>("tune.nvec", (size_t)ncol);
    GDR_CUDA(cudaMemcpyAsync(nvd, nv.data(), sizeof(int) * ncol, cudaMemcpyHostToDevice, ctx->stream));
    b.nvec = nvd;
  }
  b.ntot = len_sum(A, ncol, b.cpp);
  if (!sweep_fits<R>(ctx, A, b)) return;
  sweep_reserve<R>(ctx, b);
  Shifted sh = make_shifted(ctx, "tune", ncol, 1);
  cx<R>* r = ctx->get<cx<R>>("tune.r", (size_t)b.ldv * ncol);
  double* bn2 = ctx->get<double>("tune.bn2", (size_t)ncol + 4);
  double* tolv = ctx->get<double>("tune.tol", (size_t)ncol + 4);
  GDR_CUDA(cudaMemsetAsync(tolv, 0, sizeof(double) * ncol, ctx->stream));
  GDR_CUDA(cudaMemsetAsync(r, 0, sizeof(cx<R>) * b.ldv * ncol, ctx->stream));
  fill_uniform<R>(ctx, b.n, ncol, b.ldv, r, 0x7a11ull);
  norms2<cx<R>>(ctx, b.n, ncol, r, b.ldv, bn2, b.part, b.nblk, b.cnt, b.nvec);
  init_cols_kernel<<<(ncol + 31) / 32, 32, 0, ctx->stream>>>(b.st, ncol, bn2, tolv, nullptr, 1, sh.sact, sh.beta,
                                                              sh.gamma, sh.norms);
  GDR_LAUNCHED(ctx);
  start_cycle<R>(ctx, b, r, b.ldv);
  // one pass j = 0..m-1 in either form, from the same v_0 each time (the launch form as
  // the solves run it by default: delayed reorthogonalisation on a complex64 basis)
  constexpr bool dcgs2 = true;
  auto pass = [&](bool sw) {
    set_run_kernel<<<(ncol + 31) / 32, 32, 0, ctx->stream>>>(b.st, ncol);
    GDR_LAUNCHED(ctx);
    if (sw) {
      arnoldi_sweep<R>(ctx, A, b, 0, m);
      scale_into<R>(ctx, b, m, b.W2, b.wcs);
    } else if (std::is_same<R, float>::value && dcgs2) {
      arnoldi_dcgs2<R>(ctx, A, b, 0, m);
    } else {
      cx<R>* wl = nullptr;
      for (int j = 0; j < m; ++j) arnoldi_step<R>(ctx, A, b, j, 0, m - 1, wl);
    }
  };
  Graph gs, gl;
  auto timed = [&](bool sw) {
    Graph& g = sw ? gs : gl;
    run_cycle(ctx, true, g, [&] { pass(sw); });  // capture + warm-up
    cudaEvent_t e0, e1;
    GDR_CUDA(cudaEventCreate(&e0));
    GDR_CUDA(cudaEventCreate(&e1));
    const int reps = 5;
    GDR_CUDA(cudaEventRecord(e0, ctx->stream));
    for (int q = 0; q < reps; ++q) run_cycle(ctx, true, g, [&] { pass(sw); });
    GDR_CUDA(cudaEventRecord(e1, ctx->stream));
    GDR_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    GDR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (double)ms / reps;
  };
  t_sweep = timed(true);
  t_launch = timed(false);
  const std::vector<ColState> st = read_states(ctx, b.st, ncol);
  for (int c = 0; c < ncol; ++c)
    if (st[c].nan || st[c].err) throw gdr_error(GDR_ECUDA, "autotune: Arnoldi pass on random vectors failed");
  choice = t_sweep <= t_launch ? 1 : 0;
}
template void tune_arnoldi<float>(gdr_ctx*, const gdr_op*, int, int, double&, double&, int&);
template void tune_arnoldi<double>(gdr_ctx*, const gdr_op*, int, int, double&, double&, int&);

// ------------------------------------------------- GMRES(m_p)-Proj(k)-Sh

template <typename R>
ProjResult proj_batch(gdr_ctx* ctx, const gdr_op* A, const ProjJob<R>& job, bool use_graph) {
  const long n = A->n;
  const int ncol = job.ncol, ns = job.ns, mp = job.m_p, k = job.k;
  Batch<R> b = make_batch<R>(ctx, "pj", n, ncol, mp, ns, k + 2);
  b.nvec = job.nvec;
  b.cpp = job.cpp;
  b.ntot = len_sum(A, ncol, job.cpp);
  Shifted sh = make_shifted(ctx, "pj", ncol, ns);
  GDR_CUDA(cudaMemcpyAsync(b.sigma, job.sigma.data(), sizeof(c128) * ns * ncol, cudaMemcpyHostToDevice,
                           ctx->stream));
  // residual vectors r_c (the batch's own copy of the right-hand sides)
  const long ldr = pad_ld(n);
  cx<R>* r = ctx->get<cx<R>>("pj.r", (size_t)ldr * ncol);
  GDR_CUDA(cudaMemcpy2DAsync(r, ldr * sizeof(cx<R>), job.rhs, job.ldrhs * sizeof(cx<R>), n * sizeof(cx<R>), ncol,
                             cudaMemcpyDeviceToDevice, ctx->stream));
  double* bn2 = ctx->get<double>("pj.bn2", (size_t)ncol + 4);
  double* tolv = ctx->get<double>("pj.tol", (size_t)ncol);
  int* mask = ctx->get<int>("pj.mask", (size_t)ncol);
  double* nrm2 = ctx->get<double>("pj.nrm2", (size_t)ncol);
  GDR_CUDA(cudaMemcpyAsync(tolv, job.tol.data(), sizeof(double) * ncol, cudaMemcpyHostToDevice, ctx->stream));
  std::vector<int> mk(ncol, 1);
  if (!job.mask.empty()) mk = job.mask;
  GDR_CUDA(cudaMemcpyAsync(mask, mk.data(), sizeof(int) * ncol, cudaMemcpyHostToDevice, ctx->stream));
  norms2<cx<R>>(ctx, n, ncol, r, ldr, bn2, b.part, b.nblk, b.cnt, b.nvec);
  init_cols_kernel<<<(ncol + 31) / 32, 32, 0, ctx->stream>>>(b.st, ncol, bn2, tolv, mask, ns, sh.sact, sh.beta,
                                                              sh.gamma, sh.norms);
  GDR_LAUNCHED(ctx);
  // projection: shared deflation basis (vcs = 0)
  Batch<R> bd = b;
  bd.V = const_cast<cx<R>*>(job.Vd);
  bd.ldv = job.ldvd;
  bd.vcs = job.vdcs;
  bd.vpp = job.dpp;
  bd.vtot = job.vdcs == 0 ? (double)len_of(A, 0, job.cpp) : len_sum(A, ncol, job.cpp, job.dpp);
  bd.m = k;
  c128* cproj = ctx->get<c128>("pj.cproj", (size_t)(k + 2) * ncol);
  c128* Cp = ctx->get<c128>("pj.Cp", (size_t)(k + 1) * (ns + 1) * ncol);
  if (k > 0 && job.project && job.vdcs == 0) gs_dot_shared_reserve(ctx, n, ncol, k + 1);
  // complex64 vectors: the cycles' solution updates V_m y_i are summed in complex64 (the
  // precision the correction is computed in) and added to the FP64 solutions once, at
  // the end, instead of FP64 arithmetic per element and cycle
  cx<R>* Ef = nullptr;
  if (std::is_same<R, float>::value) {
    const size_t ne = (size_t)ncol * job.xcs;
    Ef = ctx->get<cx<R>>("pj.E", ne);
    GDR_CUDA(cudaMemsetAsync(Ef, 0, sizeof(cx<R>) * ne, ctx->stream));
  }
  // the projection's solution coefficients, summed over the cycles (applied to X at the end)
  c128* Dacc = nullptr;
  if (k > 0 && job.project) {
    Dacc = ctx->get<c128>("pj.Dacc", (size_t)(k + 1) * ns * ncol);
    GDR_CUDA(cudaMemsetAsync(Dacc, 0, sizeof(c128) * (k + 1) * ns * ncol, ctx->stream));
  }
  c128* pops = nullptr;  // the projection's solution operators, formed once for all cycles
  if (k > 0 && job.project && !job.eigsel) {
    pops = ctx->get<c128>("pj.ops", (size_t)(k + 1) * (k + 1) * (ns + 1) * ncol);
    proj_setup(ctx, ncol, k, ns, job.Hk, b.sigma, b.st, pops, job.hkcs, job.dpp);
  }
  // GMRES-Sh dense step
  const int ldc = mp + 1;
  DenseCycle d{};
  d.ncol = ncol; d.m = mp; d.k = 0; d.ns = ns; d.kfull = 0;
  d.H = b.H; d.cvec = b.cvec; d.sigma = b.sigma;
  d.beta = sh.beta; d.norms = sh.norms; d.sact = sh.sact;
  d.Cf = ctx->get<c128>("pj.Cf", (size_t)ldc * (ns + 1) * ncol); d.ldc = ldc; d.ccs = (long)ldc * (ns + 1);
  d.s = ctx->get<c128>("pj.s", (size_t)(mp + 1) * ncol);
  d.Pk = d.Hk = d.ck = nullptr;
  d.theta = nullptr;
  d.scratch = nullptr;
  d.scratch_per_col = 0;
  d.st = b.st;
  d.want_r = true;
  d.ls32 = std::is_same<R, float>::value && job.ls32;  // GMRES(m_p) cycles on a complex64 basis

  const bool sweep = job.sweep && sweep_fits<R>(ctx, A, b) &&
                    sweep_choice(A, std::is_same<R, double>::value, ncol, mp) != 0;
  if (sweep) sweep_reserve<R>(ctx, b);
  Graph gr;
  ProjResult res;
  res.mvps.assign(ncol, 0);
  res.converged.assign(ncol, 0);
  std::vector<int> done(ncol, 0);
  auto enqueue = [&]() {
    set_run_kernel<<<(ncol + 31) / 32, 32, 0, ctx->stream>>>(b.st, ncol);
    GDR_LAUNCHED(ctx);
    if (k > 0 && job.project) {
      // steps 3-4: Minres projection over V_k (or over selected eigenvectors); c = V_{k+1}^H r
      gs_dot<R>(ctx, bd, k + 1, r, ldr, cproj, false);
      dense_projection(ctx, ncol, k, ns, job.Hk, cproj, b.sigma, sh.beta, sh.sact, sh.gamma, Cp, (long)(k + 1) * (ns + 1),
                       pops, b.st, job.hkcs, job.dpp, job.eigsel);
      // r -= V_{k+1} (Hbar_k - sigma_1 Ibar) d_1 now; x_i += V_k d_i summed over the cycles
      const long pcs = (long)(k + 1) * (ns + 1);
      dacc_kernel<<<dim3(1, (unsigned)ncol), 128, 0, ctx->stream>>>(k + 1, ns, Cp, pcs, Dacc, b.st);
      GDR_LAUNCHED(ctx);
      combine<R>(ctx, n, ncol, bd.V, bd.ldv, job.vdcs, k + 1, Cp + (long)ns * (k + 1), k + 1, pcs, 0, 0, 2,
                 nullptr, 0, 0, r, ldr, b.st, b.nvec, job.dpp, col_len(b), basis_len(bd));
    }
    // step 5: one GMRES(m_p)-Sh cycle on r
    start_cycle<R>(ctx, b, r, ldr);
    if (sweep) {
      arnoldi_sweep<R>(ctx, A, b, 0, mp);
      scale_into<R>(ctx, b, mp, b.W2, b.wcs);
    } else if (std::is_same<R, float>::value && job.dcgs2) {
      arnoldi_dcgs2<R>(ctx, A, b, 0, mp);
    } else {
      cx<R>* wl = nullptr;
      for (int j = 0; j < mp; ++j) arnoldi_step<R>(ctx, A, b, j, 0, mp - 1, wl);
    }
    dense_cycle(ctx, d);
    combine<R>(ctx, n, ncol, b.V, b.ldv, b.vcs, mp + 1, d.Cf, ldc, d.ccs, 0, ns, 1, job.X, job.ldx, job.xcs, r, ldr,
               b.st, b.nvec, 1, col_len(b), 0, Ef);
    cycle_finish(ctx, d, b.H, b.cvec);
  };
  for (;;) {
    run_cycle(ctx, use_graph, gr, enqueue);
    std::vector<ColState> st = read_states(ctx, b.st, ncol);
    res.cycles++;
    bool any_active = false;
    bool cap = false;
    for (int c = 0; c < ncol; ++c) {
      if (done[c] || !mk[c]) continue;
      res.mvps[c] += st[c].broke ? st[c].m_eff : mp;
      if (st[c].nan) res.status = GDR_ENAN;
      else if (st[c].err && res.status == GDR_OK) res.status = (gdr_status)st[c].err;
      if (st[c].conv) res.converged[c] = 1;
      if (st[c].active) any_active = true;
      else done[c] = 1;
      if (res.mvps[c] >= job.max_mvps) cap = true;
    }
    if (!any_active) break;
    if (cap) {
      if (res.status == GDR_OK) res.status = GDR_ENOCONV;
      break;
    }
  }
  if (Dacc) {  // x_i += V_k (sum of the cycles' d_i), every column (zero where it never ran)
    if (Ef && job.vdcs == 0 && job.xcs == (long)ns * job.ldx && b.nvec == nullptr && job.dpp == 1) {
      // into the complex64 corrections, as ncol * ns columns e_p += V_k Dacc_p (the
      // shared-basis update, on the tensor cores where it applies), added to X below
      combine<R>(ctx, n, ncol * ns, bd.V, bd.ldv, 0, k + 1, Dacc, k + 1, k + 1, 0, 0, 2, nullptr, 0, 0, Ef, job.ldx,
                 nullptr, nullptr, 1, col_len(b) * ns, basis_len(bd));
    } else {
      combine<R>(ctx, n, ncol, bd.V, bd.ldv, job.vdcs, k + 1, Dacc, k + 1, (long)(k + 1) * ns, 0, ns, 0, job.X,
                 job.ldx, job.xcs, nullptr, 0, nullptr, b.nvec, job.dpp, col_len(b), basis_len(bd));
    }
  }
  if (Ef) {  // x_i += e_i, the cycles' corrections, once in FP64
    dim3 ge(grid1(ctx, n), (unsigned)(ncol * ns));
    add_correction_kernel<R><<<ge, 256, 0, ctx->stream>>>(n, ns, Ef, job.ldx, job.xcs, job.X, b.nvec);
    GDR_LAUNCHED(ctx);
  }
  res.gamma.resize((size_t)ncol * ns);
  GDR_CUDA(cudaMemcpyAsync(res.gamma.data(), sh.gamma, sizeof(c128) * ncol * ns, cudaMemcpyDeviceToHost, ctx->stream));
  stream_sync(ctx);
  return res;
}

// --------------------------------------------------------- FP64 residuals

// R[:, j*ns + i] = B[:, j] - (A - sigma_i I) X[:, j*ns + i]; relres[p] = ||R_p|| / ||b_j||.
// With `only`, the pairs p with only[p] == 0 keep the residual R already holds (their X
// has not changed since it was formed) and only the others are recomputed.
void true_residuals(gdr_ctx* ctx, const gdr_op* A, int ns, const c128* sigma_dev, int nrhs, const c128* B, long ldb,
                    const c128* X, long ldx, c128* R, long ldr, std::vector<double>& relres,
                    const std::vector<double>& bnorm, const std::vector<int>* only) {
  const long n = A->n;
  const int np = ns * nrhs;
  int* run = nullptr;
  if (only) {
    GDR_REQUIRE((int)only->size() == np, "true_residuals: mask size");
    run = ctx->get<int>("res.run", (size_t)np);
    GDR_CUDA(cudaMemcpyAsync(run, only->data(), sizeof(int) * np, cudaMemcpyHostToDevice, ctx->stream));
  }
  for (int j = 0; j < nrhs; ++j) {
    if (only) {
      bool any = false;
      for (int i = 0; i < ns; ++i) any = any || (*only)[(long)j * ns + i];
      if (!any) continue;
    }
    op_apply_skip(ctx, A, ns, sigma_dev, X + (long)j * ns * ldx, ldx, R + (long)j * ns * ldr, ldr, B + j * ldb, 0,
                  run ? run + (long)j * ns : nullptr, 1);
  }
  const int nblk = (int)std::min<long>((n + 255) / 256, 2L * ctx->num_sms);
  c128* part = ctx->get<c128>("res.part", (size_t)nblk * np + 64);
  unsigned* cnt = ctx->get<unsigned>("res.cnt", (size_t)4 * np);
  double* out = ctx->get<double>("res.out", (size_t)np);
  GDR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * 4 * np, ctx->stream));
  norms2<c128>(ctx, n, np, R, ldr, out, part, nblk, cnt);
  std::vector<double> h(np);
  GDR_CUDA(cudaMemcpyAsync(h.data(), out, sizeof(double) * np, cudaMemcpyDeviceToHost, ctx->stream));
  stream_sync(ctx);
  relres.resize(np);
  for (int p = 0; p < np; ++p) relres[p] = std::sqrt(h[p]) / (bnorm[p / ns] > 0 ? bnorm[p / ns] : 1.0);
}

// ------------------------------------------------------------ the pipeline

template <typename R>
static void to_inner(gdr_ctx* ctx, long n, int cols, const c128* in, long ldi, cx<R>* out, long ldo) {
  if (std::is_same<R, double>::value)
    copy128(ctx, n, cols, in, ldi, reinterpret_cast<c128*>(out), ldo);
  else
    cvt_128_to_64(ctx, n, cols, in, ldi, reinterpret_cast<c64*>(out), ldo);
}

template <typename R>
gdr_status solve_pipeline(gdr_ctx* ctx, const gdr_op* A, const std::vector<c128>& sigma, int nrhs, const c128* B,
                          long ldb, c128* X, long ldx, const gdr_params& p, gdr_defl** defl_out, gdr_report& rep) {
  const long n = A->n;
  const int ns = (int)sigma.size();
  const bool mixed = std::is_same<R, float>::value;
  const bool use_graph = !(p.flags & GDR_FLAG_NO_GRAPH);
  const int m = p.m, k = p.k, mp = p.m_proj > 0 ? p.m_proj : p.m - p.k;
  // refinement cycles: on short vectors (latency-bound steps) longer than the Proj stage's,
  // fewer restarts of the per-pair solves (measured: 8^4 14.0 -> 13.4 ms, the CSR batch
  // 611 -> 592 ms); on long vectors the Gram-Schmidt bytes of a step grow with its index
  // while the deflated projection keeps restarts cheap, so short cycles (measured on
  // GB300: 24^3x32 refinement 7.0 s at 40, 4.4 s at 20, 3.9 s at 12, 2.2 s at 8 and 6
  // with the current kernels; 16^4 189 ms at 30, 133 ms at 12, 88 ms at 8; with bf16 links,
  // whose passes ask less of the inner solve, 6: 24^3x32 2.53 s against 2.58 s at 8)
  const int mr = p.m_refine > 0 ? p.m_refine
                                : (A->n <= (1L << 17) ? std::min(m, mp + (m - mp) / 2)
                                                      : std::min(mp, (A->kind == OP_WILSON && A->store == GDR_LINK_BF16) ? 6 : 8));
  const long ld = pad_ld(n);
  gdr_status status = GDR_OK;
  auto worst = [&](gdr_status s) {
    if (s != GDR_OK && (status == GDR_OK || status == GDR_ENOCONV)) status = s;
  };
  // phase wall times, taken where the stream has just been synchronised
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
  const long syncs0 = ctx->syncs;
  auto tp = clk::now();
  GDR_CUDA(cudaMemsetAsync(X, 0, sizeof(c128) * ldx * ns * nrhs, ctx->stream));
  c128* sig_dev = ctx->get<c128>("pl.sigma", (size_t)ns);
  GDR_CUDA(cudaMemcpyAsync(sig_dev, sigma.data(), sizeof(c128) * ns, cudaMemcpyHostToDevice, ctx->stream));
  // ||b_j||
  std::vector<double> bnorm(nrhs);
  {
    const int nblk = (int)std::min<long>((n + 255) / 256, 2L * ctx->num_sms);
    c128* part = ctx->get<c128>("pl.part", (size_t)nblk * nrhs + 64);
    unsigned* cnt = ctx->get<unsigned>("pl.cnt", (size_t)4 * nrhs);
    double* out = ctx->get<double>("pl.bn", (size_t)nrhs);
    GDR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * 4 * nrhs, ctx->stream));
    norms2<c128>(ctx, n, nrhs, B, ldb, out, part, nblk, cnt);
    GDR_CUDA(cudaMemcpyAsync(bnorm.data(), out, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    stream_sync(ctx);
    for (auto& v : bnorm) v = std::sqrt(v);
  }
  for (double v : bnorm) {
    if (!std::isfinite(v)) {  // NaN or Inf in a right-hand side: X stays zero
      rep.max_relres = v;
      rep.host_syncs = ctx->syncs - syncs0;
      return GDR_ENAN;
    }
  }
  // ---- RHS 1: GMRES-DR(m,k)-Sh
  cx<R>* bin = ctx->get<cx<R>>("pl.bin", (size_t)ld);
  to_inner<R>(ctx, n, 1, B, ldb, bin, ld);
  const double tol1 = mixed ? std::max(p.tol, p.inner_tol) : p.tol;
  DrJob<R> dj;
  dj.ncol = 1;
  dj.ns = ns;
  dj.m = m;
  dj.k = k;
  dj.rhs = bin;
  dj.ldrhs = ld;
  dj.sigma = sigma;
  dj.tol.assign(1, tol1);
  dj.X = X;
  dj.ldx = ldx;
  dj.xcs = (long)ns * ldx;
  dj.max_mvps = p.max_mvps;
  dj.max_cycles = p.max_cycles;
  dj.sweep = !(p.flags & GDR_FLAG_NO_SWEEP);
  dj.dcgs2 = !(p.flags & GDR_FLAG_CGS2);
  dj.eig32 = !(p.flags & (GDR_FLAG_FP64_EIG | GDR_FLAG_FP64_DENSE));
  dj.fom = (p.flags & GDR_FLAG_FOM) != 0;
  DrResult dr = dr_sh<R>(ctx, A, dj, use_graph);
  rep.t_rhs1_ms = ms_since(tp);
  tp = clk::now();
  rep.mvps_rhs1 = dr.mvps;
  rep.cycles_rhs1 = dr.cycles;
  if (dr.status == GDR_ENOCONV && p.max_cycles > 0) {
    worst(GDR_ENOCONV);
  } else {
    worst(dr.status);
  }
  const int kd = dr.valid_defl ? k : 0;
  // the kept pair, FP64 copy of V_{k+1}
  c128* V128 = nullptr;
  if (kd > 0) {
    V128 = ctx->get<c128>("pl.V128", (size_t)ld * (kd + 1));
    if (mixed)
      cvt_64_to_128(ctx, n, kd + 1, reinterpret_cast<const c64*>(dr.V), dr.ldv, V128, ld);
    else
      copy128(ctx, n, kd + 1, reinterpret_cast<const c128*>(dr.V), dr.ldv, V128, ld);
  }
  if (defl_out && kd > 0) {
    gdr_defl* df = new gdr_defl();
    df->ctx = ctx;
    df->n = n;
    df->ldv = ld;
    df->k = kd;
    df->prec = mixed ? GDR_PREC_MIXED : GDR_PREC_FP64;
    df->wilson_V = A->kind == OP_WILSON ? A->V : 0;
    GDR_CUDA(cudaMalloc(&df->V128, sizeof(c128) * ld * (kd + 1)));
    GDR_CUDA(cudaMalloc(&df->V, sizeof(cx<R>) * ld * (kd + 1)));
    GDR_CUDA(cudaMalloc(&df->Hk, sizeof(c128) * (kd + 1) * kd));
    GDR_CUDA(cudaMemcpyAsync(df->V128, V128, sizeof(c128) * ld * (kd + 1), cudaMemcpyDeviceToDevice, ctx->stream));
    GDR_CUDA(cudaMemcpy2DAsync(df->V, ld * sizeof(cx<R>), dr.V, dr.ldv * sizeof(cx<R>), n * sizeof(cx<R>), kd + 1,
                               cudaMemcpyDeviceToDevice, ctx->stream));
    GDR_CUDA(cudaMemcpyAsync(df->Hk, dr.Hk, sizeof(c128) * (kd + 1) * kd, cudaMemcpyDeviceToDevice, ctx->stream));
    df->Hk_host.resize((size_t)(kd + 1) * kd);
    GDR_CUDA(cudaMemcpyAsync(df->Hk_host.data(), dr.Hk, sizeof(c128) * (kd + 1) * kd, cudaMemcpyDeviceToHost,
                             ctx->stream));
    stream_sync(ctx);
    *defl_out = df;
  }
  // keep the deflation pair in a buffer the later stages do not overwrite
  cx<R>* Vd = nullptr;
  c128* Hkd = nullptr;
  if (kd > 0) {
    Vd = ctx->get<cx<R>>("pl.Vd", (size_t)ld * (kd + 1));
    Hkd = ctx->get<c128>("pl.Hkd", (size_t)(kd + 1) * kd);
    GDR_CUDA(cudaMemcpy2DAsync(Vd, ld * sizeof(cx<R>), dr.V, dr.ldv * sizeof(cx<R>), n * sizeof(cx<R>), kd + 1,
                               cudaMemcpyDeviceToDevice, ctx->stream));
    GDR_CUDA(cudaMemcpyAsync(Hkd, dr.Hk, sizeof(c128) * (kd + 1) * kd, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  const bool project = kd > 0 && !(p.flags & GDR_FLAG_NO_PROJ);
  const bool related = (p.flags & GDR_FLAG_RELATED_RHS) != 0 && nrhs > 1;
  // Sec. 4, Example 4: right-hand sides 2.. projected over the first k_select approximate
  // eigenvectors of the kept pair (Theorem 1), no extra right-hand side, no correction
  EigSel es;
  const bool eigsel = project && nrhs > 1 && (p.flags & GDR_FLAG_EIG_SELECT) != 0;
  if (eigsel) {
    const int ks = (p.k_select > 0 && p.k_select < kd) ? p.k_select : kd;
    std::vector<double> eres(ks);
    eigsel_setup(ctx, Hkd, kd, ks, sigma[0], es, eres.data());
    for (double v : eres) rep.eig_resid_max = std::max(rep.eig_resid_max, v);
  }
  const int np = ns * nrhs;
  c128* Rres = ctx->get<c128>("pl.Rres", (size_t)ld * np);
  std::vector<double> relres(np, std::numeric_limits<double>::infinity());
  // the extra right-hand side's FP64 solutions s_i ((A - sigma_i) s_i ~ v_{k+1}) and
  // v_{k+1}, once the Proj stage has formed them: the shift-shared refinement's correction
  const c128* S_extra = nullptr;
  const c128* v_extra = nullptr;

  // ---- FP64 true residuals, refinement (MIXED) and cleanup of the (shift, rhs) pairs of
  //      right-hand sides [r0, r1); relres of those pairs updated
  std::vector<int> resid_ready;  // per pair: its FP64 residual is already in Rres
  auto refine_rhs = [&](int r0, int r1) {
    const int qg = r0 * ns, nq = (r1 - r0) * ns;
    const c128* Bq = B + (long)r0 * ldb;
    c128* Xq = X + (long)qg * ldx;
    c128* Rq = Rres + (long)qg * ld;
    std::vector<double> bnq(bnorm.begin() + r0, bnorm.begin() + r1);
    std::vector<double> rr;
    // the first evaluation skips the pairs whose residuals the correction phase left in Rres
    const bool pre = !resid_ready.empty() && r0 == 0 && r1 == nrhs;
    auto residuals = [&](const std::vector<int>* only = nullptr) {
      true_residuals(ctx, A, ns, sig_dev, r1 - r0, Bq, ldb, Xq, ldx, Rq, ld, rr, bnq, only);
      if (only) {
        for (int v : *only) rep.resid_cols += v ? 1 : 0;
      } else {
        rep.resid_cols += nq;
      }
      for (int q = 0; q < nq; ++q) relres[qg + q] = rr[q];
    };
    if (pre) {
      std::vector<int> todo(nq);
      for (int q = 0; q < nq; ++q) todo[q] = resid_ready[q] ? 0 : 1;
      resid_ready.clear();
      residuals(&todo);
    } else {
      residuals();
    }
    // Shift-shared pass (not in the paper; complex64 only): per right-hand side j, the
    // active residuals R_j = [r_i^j] are written as Y_j C_j + E_j with Y_j orthonormal
    // (pivoted Cholesky of R_j^H R_j, ||E_j||_F <= refine_rank_tol ||R_j||_2 roughly);
    // each column of Y_j is solved for all shifts at once by GMRES(m_r)-Proj(k)-Sh
    // (one Krylov space per column, as for the later right-hand sides of Sec. 4), then
    // x_i^j += sum_t C_j[t, i] z_{t,i}, and the v_{k+1} components of the new true
    // residuals are removed with the extra right-hand side's solutions (eq. keyder4b:
    // x_i += (v_{k+1}^H r_i) s_i).  With bf16 links the stage's residuals are close to
    // low rank across the shifts (their differences come from the link rounding acting
    // on solutions that vary smoothly with the shift), so this needs far fewer columns
    // than one per pair.  Returns false (nothing done) when it would not.
    auto shared_pass = [&](const std::vector<int>& mask) -> bool {
      if (!mixed || !(p.refine_rank_tol > 0) || kd <= 0 || !project || !S_extra || ns < 2) return false;
      if (!std::is_same<R, float>::value) return false;
      const int nr = r1 - r0;
      // Gram matrices of the active residuals of each right-hand side (FP64 dots)
      c128* gram = ctx->get<c128>("sh.gram", (size_t)nr * ns * ns);
      const int gnb = (int)std::min<long>((n + 255) / 256, 2L * ctx->num_sms);
      c128* gpart = ctx->get<c128>("sh.part", (size_t)gnb * ns + 64);
      unsigned* gcnt = ctx->get<unsigned>("sh.cnt", (size_t)4 * ns);
      GDR_CUDA(cudaMemsetAsync(gcnt, 0, sizeof(unsigned) * 4 * ns, ctx->stream));
      for (int j = 0; j < nr; ++j)
        for (int a = 0; a < ns; ++a) {
          if (!mask[j * ns + a]) continue;
          const c128* ra = Rq + (long)(j * ns + a) * ld;
          // r_a^H r_b for b >= a (columns of R_j from a on)
          dots128(ctx, n, ns - a, ra, 0, Rq + (long)(j * ns + a) * ld, ld, gram + ((long)j * ns + a) * ns + a,
                  gpart, gnb, gcnt);
        }
      std::vector<c128> Gh((size_t)nr * ns * ns);
      GDR_CUDA(cudaMemcpyAsync(Gh.data(), gram, sizeof(c128) * Gh.size(), cudaMemcpyDeviceToHost, ctx->stream));
      stream_sync(ctx);
      struct Rhs {
        int j, nc, p;
        std::vector<int> act;  // shifts of this rhs in the pass (indices into 0..ns-1)
        std::vector<c128> W, C;
        std::vector<double> tol;
      };
      std::vector<Rhs> rs;
      int cols = 0, pairs = 0;
      for (int j = 0; j < nr; ++j) {
        Rhs e;
        e.j = j;
        for (int i = 0; i < ns; ++i)
          if (mask[j * ns + i]) e.act.push_back(i);
        e.nc = (int)e.act.size();
        if (e.nc == 0) continue;
        // Gram of the active columns, G[x, y] = r_{act x}^H r_{act y}, from the stored
        // gram[(j*ns + a)*ns + b] = r_a^H r_b (b >= a)
        std::vector<c128> G((size_t)e.nc * e.nc);
        double gmax = 0;
        for (int x = 0; x < e.nc; ++x)
          for (int y = 0; y < e.nc; ++y) {
            const int a = std::min(e.act[x], e.act[y]), b = std::max(e.act[x], e.act[y]);
            c128 v = Gh[((size_t)j * ns + a) * ns + b];
            if (e.act[x] > e.act[y]) v = conj(v);
            G[x + (size_t)y * e.nc] = v;
            gmax = std::max(gmax, G[x + (size_t)x * e.nc].x);
          }
        std::vector<c128> L;
        std::vector<int> piv;
        const double thr = p.refine_rank_tol * std::sqrt(gmax);
        e.p = pivoted_cholesky(G, e.nc, thr * thr, e.nc, L, piv);
        if (e.p == 0) continue;
        e.W = orth_weights(L, piv, e.nc);
        e.C.assign((size_t)e.p * ns, c128{0, 0});
        std::vector<double> cmax(e.p, 0.0);
        for (int t = 0; t < e.p; ++t)
          for (int x = 0; x < e.nc; ++x) {
            e.C[t + (size_t)e.act[x] * e.p] = conj(L[x + (size_t)t * e.nc]);
            cmax[t] = std::max(cmax[t], std::sqrt(norm2(L[x + (size_t)t * e.nc])));
          }
        // column t is refined until its error, weighted by its largest coefficient, is
        // below the target 0.3 tol ||b_j||, but not beyond refine_tol
        e.tol.resize(e.p);
        for (int t = 0; t < e.p; ++t)
          e.tol[t] = std::min(0.5, std::max(0.3 * p.tol * bnq[j] / std::max(cmax[t], 1e-300), p.refine_tol));
        cols += e.p;
        pairs += e.nc;
        rs.push_back(std::move(e));
      }
      if (cols == 0 || cols > 0.7 * pairs) return false;
      rep.shared_cols += cols;
      rep.shared_pairs += pairs;
      // memory: per column a complex64 Krylov basis of m_r + 1 vectors (+ work), its FP64
      // right-hand side and the FP64 solutions of all shifts
      size_t freeb = 0, totb = 0;
      GDR_CUDA(cudaMemGetInfo(&freeb, &totb));
      const size_t per_col = (size_t)ld * (sizeof(cx<R>) * (mr + 6) + sizeof(c128) * (ns + 1)) + 65536;
      const int chunk = (int)std::max<size_t>(1, (freeb / 2) / per_col);
      size_t e0 = 0;
      while (e0 < rs.size()) {  // groups of right-hand sides whose columns fit
        size_t e1 = e0;
        int cn = 0;
        while (e1 < rs.size() && (cn == 0 || cn + rs[e1].p <= chunk)) cn += rs[e1++].p;
        c128* Y128 = ctx->get<c128>("sh.Y128", (size_t)ld * cn);
        cx<R>* Y = ctx->get<cx<R>>("sh.Y", (size_t)ld * cn);
        c128* Z = ctx->get<c128>("sh.Z", (size_t)ld * ns * cn);
        c128* Wd = ctx->get<c128>("sh.W", (size_t)ns * ns * (e1 - e0));
        c128* Cd = ctx->get<c128>("sh.C", (size_t)ns * ns * (e1 - e0));
        int* actd = ctx->get<int>("sh.act", (size_t)ns * (e1 - e0));
        GDR_CUDA(cudaMemsetAsync(Y128, 0, sizeof(c128) * ld * cn, ctx->stream));
        GDR_CUDA(cudaMemsetAsync(Z, 0, sizeof(c128) * ld * ns * cn, ctx->stream));
        ProjJob<R> job;
        job.ncol = cn;
        job.ns = ns;
        job.m_p = mr;
        job.k = kd;
        job.project = true;
        job.Vd = Vd;
        job.ldvd = ld;
        job.Hk = Hkd;
        job.rhs = Y;
        job.ldrhs = ld;
        job.sigma.resize((size_t)cn * ns);
        job.tol.clear();
        job.X = Z;
        job.ldx = ld;
        job.xcs = (long)ns * ld;
        job.max_mvps = p.max_mvps;
        job.sweep = !(p.flags & GDR_FLAG_NO_SWEEP);
        job.dcgs2 = !(p.flags & GDR_FLAG_CGS2);
        job.ls32 = !(p.flags & GDR_FLAG_FP64_DENSE);
        int c0 = 0;
        for (size_t e = e0; e < e1; ++e) {
          const Rhs& r = rs[e];
          const long slot = (long)(e - e0);
          // W padded to ns x ns (rows = all shifts of the rhs, inactive rows zero), C as p x ns
          std::vector<c128> Wf((size_t)ns * r.p, c128{0, 0});
          for (int x = 0; x < r.nc; ++x)
            for (int t = 0; t < r.p; ++t) Wf[r.act[x] + (size_t)t * ns] = r.W[x + (size_t)t * r.nc];
          std::vector<int> af(ns, 0);
          for (int i : r.act) af[i] = 1;
          GDR_CUDA(cudaMemcpyAsync(Wd + slot * ns * ns, Wf.data(), sizeof(c128) * Wf.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
          GDR_CUDA(cudaMemcpyAsync(Cd + slot * ns * ns, r.C.data(), sizeof(c128) * r.C.size(),
                                   cudaMemcpyHostToDevice, ctx->stream));
          GDR_CUDA(cudaMemcpyAsync(actd + slot * ns, af.data(), sizeof(int) * ns, cudaMemcpyHostToDevice,
                                   ctx->stream));
          // Y_j = R_j W (FP64), then its complex64 copy as the right-hand sides
          combine<double>(ctx, n, 1, const_cast<c128*>(Rq + (long)r.j * ns * ld), ld, 0, ns, Wd + slot * ns * ns,
                          ns, 0, 0, r.p, 0, Y128 + (long)c0 * ld, ld, 0, nullptr, 0, nullptr);
          for (int t = 0; t < r.p; ++t) {
            for (int i = 0; i < ns; ++i) job.sigma[(size_t)(c0 + t) * ns + i] = sigma[i];
            job.tol.push_back(r.tol[t]);
          }
          c0 += r.p;
        }
        to_inner<R>(ctx, n, cn, Y128, ld, Y, ld);
        ProjResult pr = proj_batch<R>(ctx, A, job, use_graph);
        for (int c = 0; c < cn; ++c) {
          rep.mvps_refine += pr.mvps[c];
          rep.mvps_shared += pr.mvps[c];
        }
        if (pr.status == GDR_ENAN || pr.status == GDR_ECUDA) worst(pr.status);
        // x_i^j += sum_t C_j[t, i] z_{t,i}
        c0 = 0;
        for (size_t e = e0; e < e1; ++e) {
          const Rhs& r = rs[e];
          const long slot = (long)(e - e0);
          dim3 ga(grid1(ctx, n), (unsigned)ns);
          shared_apply_kernel<<<ga, 256, 0, ctx->stream>>>(n, ns, r.p, Cd + slot * ns * ns, actd + slot * ns,
                                                          Z + (long)c0 * ns * ld, ld, Xq + (long)r.j * ns * ldx, ldx);
          GDR_LAUNCHED(ctx);
          c0 += r.p;
        }
        e0 = e1;
      }
      // remove the v_{k+1} components of the new true residuals (shifts i >= 1)
      residuals();
      c128* gam = ctx->get<c128>("sh.gam", (size_t)nq);
      const int dnb = (int)std::min<long>((n + 255) / 256, 2L * ctx->num_sms);
      c128* dpart = ctx->get<c128>("sh.dpart", (size_t)dnb * nq + 64);
      unsigned* dcnt = ctx->get<unsigned>("sh.dcnt", (size_t)4 * nq);
      GDR_CUDA(cudaMemsetAsync(dcnt, 0, sizeof(unsigned) * 4 * nq, ctx->stream));
      dots128(ctx, n, nq, v_extra, 0, Rq, ld, gam, dpart, dnb, dcnt);
      dim3 gc(grid1(ctx, n), (unsigned)nq);
      correct_kernel<<<gc, 256, 0, ctx->stream>>>(n, ns, gam, S_extra, ld, Xq, ldx);
      GDR_LAUNCHED(ctx);
      return true;
    };
    const int max_pass = (p.flags & GDR_FLAG_NO_REFINE) ? -1 : std::max(0, p.refine_max);
    for (int pass = 0; pass <= max_pass; ++pass) {
      std::vector<int> mask(nq, 0);
      int nact = 0;
      for (int q = 0; q < nq; ++q)
        if (!(rr[q] <= p.tol)) {
          mask[q] = 1;
          ++nact;
        }
      if (nact == 0) break;
      const bool cleanup = (pass == max_pass) || !mixed;
      rep.refine_passes++;
      if (cleanup) rep.pairs_cleaned += nact;
      if (!cleanup && shared_pass(mask)) {
        residuals();
        continue;
      }
      // chunk the pairs by memory
      size_t freeb = 0, totb = 0;
      GDR_CUDA(cudaMemGetInfo(&freeb, &totb));
      const size_t elem = cleanup ? sizeof(c128) : sizeof(cx<R>);
      const size_t per_col = elem * (size_t)ld * (mr + 5) + 4096;  // basis, work vectors, correction
      int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)nq, (freeb / 2) / per_col));
      for (int q0 = 0; q0 < nq; q0 += chunk) {
        const int cn = std::min(chunk, nq - q0);
        bool any = false;
        for (int q = q0; q < q0 + cn; ++q) any = any || mask[q];
        if (!any) continue;
        std::vector<double> tolc(cn);
        std::vector<int> mk(mask.begin() + q0, mask.begin() + q0 + cn);
        for (int c = 0; c < cn; ++c) {
          const int q = q0 + c;
          // relative to the residual column: reach tol * ||b|| with margin
          tolc[c] = std::max(0.3 * p.tol / std::max(rr[q], 1e-300), cleanup ? 0.0 : p.refine_tol);
          tolc[c] = std::min(tolc[c], 0.5);
        }
        auto run_refine = [&](auto tag) {
          using RR = decltype(tag);
          cx<RR>* rin = ctx->get<cx<RR>>("rf.rin", (size_t)ld * cn);
          to_inner<RR>(ctx, n, cn, Rq + (long)q0 * ld, ld, rin, ld);
          ProjJob<RR> job;
          job.ncol = cn;
          job.ns = 1;
          job.m_p = mr;
          job.k = kd;
          job.project = project;
          cx<RR>* vd = nullptr;
          if (kd > 0) {
            if (std::is_same<RR, R>::value) {
              vd = reinterpret_cast<cx<RR>*>(Vd);
            } else {  // FP64 cleanup after a complex64 solve: FP64 copy of the kept basis
              vd = reinterpret_cast<cx<RR>*>(V128);
            }
          }
          job.Vd = vd;
          job.ldvd = ld;
          job.Hk = Hkd;
          job.rhs = rin;
          job.ldrhs = ld;
          job.sigma.resize(cn);
          for (int c = 0; c < cn; ++c) job.sigma[c] = sigma[(q0 + c) % ns];
          job.tol = tolc;
          job.mask = mk;
          job.X = Xq + (long)q0 * ldx;
          job.ldx = ldx;
          job.xcs = ldx;
          job.max_mvps = p.max_mvps;
          job.sweep = !(p.flags & GDR_FLAG_NO_SWEEP);
          job.dcgs2 = !(p.flags & GDR_FLAG_CGS2);
          job.ls32 = !(p.flags & GDR_FLAG_FP64_DENSE);
          ProjResult pr = proj_batch<RR>(ctx, A, job, use_graph);
          for (int c = 0; c < cn; ++c) rep.mvps_refine += pr.mvps[c];
          if (pr.status == GDR_ENAN || pr.status == GDR_ECUDA) worst(pr.status);
        };
        if (cleanup)
          run_refine(double{});
        else
          run_refine(R{});
      }
      residuals(&mask);  // only the pairs this pass refined have a new X
    }
  };

  // ---- extra right-hand side v_{k+1} and RHS 2..nrhs: GMRES(m_p)-Proj(k)-Sh
  if (nrhs > 1) {
    const int ncol = nrhs;  // column 0: v_{k+1} (if deflating), columns 1..: b^2..b^nrhs
    cx<R>* rhs = ctx->get<cx<R>>("pl.rhs", (size_t)ld * ncol);
    c128* XP = ctx->get<c128>("pl.XP", (size_t)ld * ns * ncol);  // slot 0: S (extra), slot j: X for rhs j+1
    GDR_CUDA(cudaMemsetAsync(XP, 0, sizeof(c128) * ld * ns * ncol, ctx->stream));
    if (project && !eigsel)
      GDR_CUDA(cudaMemcpyAsync(rhs, Vd + (long)kd * ld, sizeof(cx<R>) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    if (!related) to_inner<R>(ctx, n, nrhs - 1, B + ldb, ldb, rhs + ld, ld);
    std::vector<int> mask(ncol, 1);
    if (!project || eigsel) mask[0] = 0;
    std::vector<double> tol_scale(ncol, 1.0);  // stage tolerance of a column relative to ||b_j|| / ||its rhs||
    const bool seq = (p.flags & GDR_FLAG_SEQUENTIAL) != 0 || related;
    const int first = (project && !eigsel) ? 0 : 1;
    auto run_cols = [&](int c0, int cn) {
      ProjJob<R> job;
      job.ncol = cn;
      job.ns = ns;
      job.m_p = mp;
      job.k = kd;
      job.project = project;
      job.Vd = Vd;
      job.ldvd = ld;
      job.Hk = Hkd;
      job.rhs = rhs + (long)c0 * ld;
      job.ldrhs = ld;
      job.sigma.resize((size_t)cn * ns);
      for (int c = 0; c < cn; ++c)
        for (int i = 0; i < ns; ++i) job.sigma[(size_t)c * ns + i] = sigma[i];
      job.tol.resize(cn);
      for (int c = 0; c < cn; ++c)
        job.tol[c] = std::min(0.5, tol_scale[c0 + c] * ((c0 + c == 0) ? p.extra_tol
                                                                      : (mixed ? std::max(p.tol, p.inner_tol) : p.tol)));
      job.mask.assign(mask.begin() + c0, mask.begin() + c0 + cn);
      job.X = XP + (long)c0 * ns * ld;
      job.ldx = ld;
      job.xcs = (long)ns * ld;
      job.max_mvps = p.max_mvps;
      job.sweep = !(p.flags & GDR_FLAG_NO_SWEEP);
      job.dcgs2 = !(p.flags & GDR_FLAG_CGS2);
      job.ls32 = !(p.flags & GDR_FLAG_FP64_DENSE);
      if (eigsel) job.eigsel = &es;
      ProjResult pr = proj_batch<R>(ctx, A, job, use_graph && !seq);
      for (int c = 0; c < cn; ++c) {
        if (c0 + c == 0) rep.mvps_extra += pr.mvps[c];
        else rep.mvps_proj += pr.mvps[c];
      }
      worst(pr.status);
    };
    // correction phase (FP64): extra solutions s_i = s~_i / (1 - gamma_i), then x_i^j += gamma_i^j s_i
    c128* RP = ctx->get<c128>("pl.RP", (size_t)ld * ns * ncol);
    const bool correct = project && ns > 1 && !eigsel;
    const c128* v128 = correct ? V128 + (long)kd * ld : nullptr;
    c128* gam = ctx->get<c128>("pl.gam", (size_t)ns * ncol);
    const int dnblk = (int)std::min<long>((n + 255) / 256, 2L * ctx->num_sms);
    c128* dpart = ctx->get<c128>("pl.dpart", (size_t)dnblk * ns * ncol + 64);
    unsigned* dcnt = ctx->get<unsigned>("pl.dcnt", (size_t)4 * ns * ncol);
    GDR_CUDA(cudaMemsetAsync(dcnt, 0, sizeof(unsigned) * 4 * ns * ncol, ctx->stream));
    auto scale_extra = [&]() {  // extra system residuals v - (A - sigma_i) s~_i, gamma_i, s_i
      std::vector<double> rr;
      std::vector<double> one(1, 1.0);
      true_residuals(ctx, A, ns, sig_dev, 1, v128, ld, XP, ld, RP, ld, rr, one);
      dots128(ctx, n, ns, v128, 0, RP, ld, gam, dpart, dnblk, dcnt);
      dim3 ge(grid1(ctx, n), (unsigned)(ns - 1));
      extra_scale_kernel<<<ge, 256, 0, ctx->stream>>>(n, ns, gam, XP, ld);
      GDR_LAUNCHED(ctx);
    };
    // slots [j0, j0 + nr) solved for right-hand sides Bc (FP64, ld ldbc): residuals, gamma_i^j, corrections
    auto correct_slots = [&](int j0, int nr, const c128* Bc, long ldbc, const std::vector<double>& bn) {
      std::vector<double> rr;
      true_residuals(ctx, A, ns, sig_dev, nr, Bc, ldbc, XP + (long)j0 * ns * ld, ld, RP + (long)j0 * ns * ld, ld, rr,
                     bn);
      dots128(ctx, n, ns * nr, v128, 0, RP + (long)j0 * ns * ld, ld, gam + (long)j0 * ns, dpart, dnblk, dcnt);
      dim3 gc(grid1(ctx, n), (unsigned)(ns * nr));
      correct_kernel<<<gc, 256, 0, ctx->stream>>>(n, ns, gam + (long)j0 * ns, XP, ld, XP + (long)j0 * ns * ld, ld);
      GDR_LAUNCHED(ctx);
    };
    if (!related) {
      if (seq) {
        for (int c = first; c < ncol; ++c) run_cols(c, 1);
      } else {
        run_cols(first, ncol - first);
      }
      if (correct) {
        scale_extra();
        std::vector<double> bn2(bnorm.begin() + 1, bnorm.end());
        correct_slots(1, nrhs - 1, B + ldb, ldb, bn2);
        S_extra = XP;  // slot 0: s_i = s~_i / (1 - gamma_i)
        v_extra = v128;
        if (nrhs > 1) {  // the corrected residuals of RHS 2.. (pairs ns..), for the refinement
          dim3 gr(grid1(ctx, n), (unsigned)(ns * (nrhs - 1)));
          corrected_resid_kernel<<<gr, 256, 0, ctx->stream>>>(n, ns, gam + ns, gam, v128, RP, RP + (long)ns * ld,
                                                              Rres + (long)ns * ld, ld);
          GDR_LAUNCHED(ctx);
          resid_ready.assign((size_t)nrhs * ns, 1);
          for (int i = 0; i < ns; ++i) resid_ready[i] = 0;
        }
      }
      // results of RHS 2.. into X
      for (int j = 1; j < nrhs; ++j)
        copy128(ctx, n, ns, XP + (long)j * ns * ld, ld, X + (long)j * ns * ldx, ldx);
      rep.t_proj_ms = ms_since(tp);
      tp = clk::now();
      refine_rhs(0, nrhs);
    } else {
      // Sec. 5: right-hand sides one at a time, each started from the Minres projection over the
      // converged solutions of the previous ones (B^H B d = B^H b_j, x_i = X_i d, common residual
      // b_j - B d), then Proj-Sh and the correction on that residual, then refined to tol
      if (project && !eigsel) run_cols(0, 1);
      if (correct) scale_extra();
      refine_rhs(0, 1);
      c128* M = ctx->get<c128>("rel.M", (size_t)nrhs * (nrhs + 1));
      c128* dvec = ctx->get<c128>("rel.d", (size_t)nrhs);
      c128* res = ctx->get<c128>("rel.r", (size_t)ld);
      double* rn2 = ctx->get<double>("rel.rn", 4);
      c128* ypart = ctx->get<c128>("rel.part", (size_t)dnblk * (nrhs + 1) + 64);
      unsigned* ycnt = ctx->get<unsigned>("rel.cnt", (size_t)4 * (nrhs + 1));
      for (int j = 1; j < nrhs; ++j) {
        // [B^H B | B^H b_j], row a = b_a^H [b_0 .. b_j]
        GDR_CUDA(cudaMemsetAsync(ycnt, 0, sizeof(unsigned) * 4 * (nrhs + 1), ctx->stream));
        for (int a = 0; a < j; ++a)
          dots128(ctx, n, j + 1, B + (long)a * ldb, 0, B, ldb, M + (long)a * (j + 1), ypart, dnblk, ycnt);
        related_solve_kernel<<<1, 32, 0, ctx->stream>>>(j, M, dvec);
        GDR_LAUNCHED(ctx);
        dim3 gg(grid1(ctx, n), (unsigned)(ns + 1));
        related_guess_kernel<<<gg, 256, 0, ctx->stream>>>(n, ns, j, dvec, X, ldx, B, ldb, res);
        GDR_LAUNCHED(ctx);
        norms2<c128>(ctx, n, 1, res, ld, rn2, ypart, dnblk, ycnt);
        double rn = 0;
        GDR_CUDA(cudaMemcpyAsync(&rn, rn2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        stream_sync(ctx);
        rn = std::sqrt(rn);
        rep.related_resid = std::max(rep.related_resid, rn / std::max(bnorm[j], 1e-300));
        // the Proj stage only where the projected residual misses the stage tolerance
        // (refinement finishes the pairs either way)
        if (rn > (mixed ? std::max(p.tol, p.inner_tol) : p.tol) * bnorm[j]) {
          to_inner<R>(ctx, n, 1, res, ld, rhs + (long)j * ld, ld);
          tol_scale[j] = bnorm[j] / rn;
          run_cols(j, 1);
          if (correct) {
            std::vector<double> bnr(1, rn);
            correct_slots(j, 1, res, ld, bnr);
          }
          dim3 ga(grid1(ctx, n), (unsigned)ns);
          add_cols_kernel<<<ga, 256, 0, ctx->stream>>>(n, XP + (long)j * ns * ld, ld, X + (long)j * ns * ldx, ldx);
          GDR_LAUNCHED(ctx);
        }
        refine_rhs(j, j + 1);
      }
      rep.t_proj_ms = ms_since(tp);
      tp = clk::now();
    }
  } else {
    rep.t_proj_ms = ms_since(tp);
    tp = clk::now();
    refine_rhs(0, 1);
  }
  double mx = 0;
  for (double v : relres) mx = std::max(mx, v);
  rep.max_relres = mx;
  rep.t_refine_ms = ms_since(tp);
  rep.host_syncs = ctx->syncs - syncs0;
  if (!(mx <= p.tol)) {
    if (status == GDR_OK) status = GDR_ENOCONV;
  } else if (status == GDR_ENOCONV && p.max_cycles <= 0) {
    status = GDR_OK;  // a stage stopped at its cap but refinement reached tol
  }
  return status;
}

// ------------------------------------------------- batch of independent problems

template <typename R>
gdr_status solve_batch_pipeline(gdr_ctx* ctx, const gdr_op* A, int ns, const std::vector<c128>& sigma,
                                const c128* B, c128* X, const gdr_params& p, gdr_report& rep, int* prob_status) {
  const int np = A->nprob;
  const long n = A->n, ld = pad_ld(n);
  const bool mixed = std::is_same<R, float>::value;
  const bool use_graph = !(p.flags & GDR_FLAG_NO_GRAPH);
  const int m = p.m, k = p.k, mp = p.m_proj > 0 ? p.m_proj : p.m - p.k;
  // refinement cycles: on short vectors (latency-bound steps) longer than the Proj stage's,
  // fewer restarts of the per-pair solves (measured: 8^4 14.0 -> 13.4 ms, the CSR batch
  // 611 -> 592 ms); on long vectors the Gram-Schmidt bytes of a step grow with its index
  // while the deflated projection keeps restarts cheap, so short cycles (measured on
  // GB300: 24^3x32 refinement 7.0 s at 40, 4.4 s at 20, 3.9 s at 12, 2.2 s at 8 and 6
  // with the current kernels; 16^4 189 ms at 30, 133 ms at 12, 88 ms at 8; with bf16 links,
  // whose passes ask less of the inner solve, 6: 24^3x32 2.53 s against 2.58 s at 8)
  const int mr = p.m_refine > 0 ? p.m_refine
                                : (A->n <= (1L << 17) ? std::min(m, mp + (m - mp) / 2)
                                                      : std::min(mp, (A->kind == OP_WILSON && A->store == GDR_LINK_BF16) ? 6 : 8));
  const int npair = np * ns;
  GDR_CUDA(cudaMemsetAsync(X, 0, sizeof(c128) * ld * npair, ctx->stream));
  // per-pair lengths (pair q = problem q / ns, shift q % ns)
  std::vector<int> nvp_h(npair);
  for (int q = 0; q < npair; ++q) nvp_h[q] = (int)A->nrow_host[q / ns];
  int* nvp = ctx->get<int>("bt.nvp", (size_t)npair);
  GDR_CUDA(cudaMemcpyAsync(nvp, nvp_h.data(), sizeof(int) * npair, cudaMemcpyHostToDevice, ctx->stream));
  c128* sig_dev = ctx->get<c128>("bt.sigma", (size_t)npair);
  GDR_CUDA(cudaMemcpyAsync(sig_dev, sigma.data(), sizeof(c128) * npair, cudaMemcpyHostToDevice, ctx->stream));
  const int nblk = (int)std::min<long>((n + 255) / 256, 2L * ctx->num_sms);
  c128* part = ctx->get<c128>("bt.part", (size_t)nblk * npair + 64);
  unsigned* cnt = ctx->get<unsigned>("bt.cnt", (size_t)4 * npair);
  double* out = ctx->get<double>("bt.out", (size_t)npair);
  GDR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * 4 * npair, ctx->stream));
  std::vector<double> bnorm(np);
  norms2<c128>(ctx, n, np, B, ld, out, part, nblk, cnt, A->nrow);
  GDR_CUDA(cudaMemcpyAsync(bnorm.data(), out, sizeof(double) * np, cudaMemcpyDeviceToHost, ctx->stream));
  stream_sync(ctx);
  for (auto& v : bnorm) v = std::sqrt(v);
  {
    bool bad = false;
    for (int q = 0; q < np; ++q) {
      if (!std::isfinite(bnorm[q])) {  // NaN or Inf in problem q's right-hand side
        bad = true;
        if (prob_status) prob_status[q] = GDR_ENAN;
      }
    }
    if (bad) {
      rep.max_relres = std::numeric_limits<double>::quiet_NaN();
      return GDR_ENAN;
    }
  }
  // ---- every problem's GMRES-DR(m,k)-Sh, the problems as columns of one batch
  cx<R>* bin = ctx->get<cx<R>>("bt.bin", (size_t)ld * np);
  to_inner<R>(ctx, ld, np, B, ld, bin, ld);
  DrJob<R> dj;
  dj.ncol = np;
  dj.ns = ns;
  dj.m = m;
  dj.k = k;
  dj.rhs = bin;
  dj.ldrhs = ld;
  dj.sigma = sigma;
  dj.tol.assign(np, mixed ? std::max(p.tol, p.inner_tol) : p.tol);
  dj.nvec = A->nrow;
  dj.cpp = 1;
  dj.X = X;
  dj.ldx = ld;
  dj.xcs = (long)ns * ld;
  dj.max_mvps = p.max_mvps;
  dj.max_cycles = p.max_cycles;
  dj.sweep = !(p.flags & GDR_FLAG_NO_SWEEP);
  dj.dcgs2 = !(p.flags & GDR_FLAG_CGS2);
  dj.eig32 = !(p.flags & (GDR_FLAG_FP64_EIG | GDR_FLAG_FP64_DENSE));
  dj.fom = (p.flags & GDR_FLAG_FOM) != 0;
  DrResult dr = dr_sh<R>(ctx, A, dj, use_graph);
  for (long v : dr.col_mvps) rep.mvps_rhs1 += v;
  rep.cycles_rhs1 = dr.cycles;
  gdr_status status = (dr.status == GDR_ENOCONV) ? GDR_OK : dr.status;
  // ---- FP64 true residuals per (problem, shift), refinement / cleanup by batched GMRES(m_p)
  c128* Rres = ctx->get<c128>("bt.Rres", (size_t)ld * npair);
  auto residuals = [&](std::vector<double>& rr) {
    GDR_CUDA(cudaMemsetAsync(Rres, 0, sizeof(c128) * ld * npair, ctx->stream));
    op_apply<double>(ctx, A, npair, sig_dev, X, ld, Rres, ld, B, ld, ns);
    norms2<c128>(ctx, n, npair, Rres, ld, out, part, nblk, cnt, nvp);
    std::vector<double> h(npair);
    GDR_CUDA(cudaMemcpyAsync(h.data(), out, sizeof(double) * npair, cudaMemcpyDeviceToHost, ctx->stream));
    stream_sync(ctx);
    rr.resize(npair);
    for (int q = 0; q < npair; ++q) rr[q] = std::sqrt(h[q]) / (bnorm[q / ns] > 0 ? bnorm[q / ns] : 1.0);
    rep.resid_cols += npair;
  };
  std::vector<double> relres;
  residuals(relres);
  const int max_pass = (p.flags & GDR_FLAG_NO_REFINE) ? -1 : std::max(0, p.refine_max);
  for (int pass = 0; pass <= max_pass; ++pass) {
    std::vector<int> mask(npair, 0);
    int nact = 0;
    for (int q = 0; q < npair; ++q)
      if (!(relres[q] <= p.tol)) {
        mask[q] = 1;
        ++nact;
      }
    if (nact == 0) break;
    const bool cleanup = (pass == max_pass) || !mixed;
    rep.refine_passes++;
    if (cleanup) rep.pairs_cleaned += nact;
    std::vector<double> tolc(npair);
    for (int q = 0; q < npair; ++q)
      tolc[q] = std::min(0.5, std::max(0.3 * p.tol / std::max(relres[q], 1e-300), cleanup ? 0.0 : p.refine_tol));
    auto run = [&](auto tag) {
      using RR = decltype(tag);
      cx<RR>* rin = ctx->get<cx<RR>>("bt.rin", (size_t)ld * npair);
      to_inner<RR>(ctx, ld, npair, Rres, ld, rin, ld);
      ProjJob<RR> job;
      job.ncol = npair;
      job.ns = 1;
      job.m_p = mr;
      job.k = 0;
      job.project = false;
      // every pair projects over its own problem's kept pair of the GMRES-DR stage
      // (in the precision of that stage's basis)
      if (std::is_same<RR, R>::value && dr.valid_defl && !dr.any_broke && k > 0) {
        job.k = k;
        job.project = true;
        job.Vd = reinterpret_cast<const cx<RR>*>(dr.V);
        job.ldvd = dr.ldv;
        job.vdcs = dr.vcs;
        job.Hk = dr.Hk;
        job.hkcs = (long)(k + 1) * k;
        job.dpp = ns;
      }
      job.rhs = rin;
      job.ldrhs = ld;
      job.sigma = sigma;
      job.tol = tolc;
      job.mask = mask;
      job.nvec = nvp;
      job.cpp = ns;
      job.X = X;
      job.ldx = ld;
      job.xcs = ld;
      job.max_mvps = p.max_mvps;
      job.sweep = !(p.flags & GDR_FLAG_NO_SWEEP);
      job.dcgs2 = !(p.flags & GDR_FLAG_CGS2);
      job.ls32 = !(p.flags & GDR_FLAG_FP64_DENSE);
      ProjResult pr = proj_batch<RR>(ctx, A, job, use_graph);
      for (long v : pr.mvps) rep.mvps_refine += v;
      if (pr.status == GDR_ENAN) status = GDR_ENAN;
    };
    if (cleanup)
      run(double{});
    else
      run(R{});
    residuals(relres);
  }
  double mx = 0;
  for (int q = 0; q < npair; ++q) mx = std::max(mx, relres[q]);
  rep.max_relres = mx;
  if (prob_status)
    for (int pb = 0; pb < np; ++pb) {
      bool ok = true;
      for (int i = 0; i < ns; ++i) ok = ok && relres[pb * ns + i] <= p.tol;
      prob_status[pb] = ok ? GDR_OK : GDR_ENOCONV;
    }
  if (status == GDR_OK && !(mx <= p.tol)) status = GDR_ENOCONV;
  return status;
}

// ------------------------------------------------------------ instances

template DrResult dr_sh<float>(gdr_ctx*, const gdr_op*, const DrJob<float>&, bool);
template DrResult dr_sh<double>(gdr_ctx*, const gdr_op*, const DrJob<double>&, bool);
template ProjResult proj_batch<float>(gdr_ctx*, const gdr_op*, const ProjJob<float>&, bool);
template ProjResult proj_batch<double>(gdr_ctx*, const gdr_op*, const ProjJob<double>&, bool);
template gdr_status solve_pipeline<float>(gdr_ctx*, const gdr_op*, const std::vector<c128>&, int, const c128*, long,
                                          c128*, long, const gdr_params&, gdr_defl**, gdr_report&);
template gdr_status solve_pipeline<double>(gdr_ctx*, const gdr_op*, const std::vector<c128>&, int, const c128*, long,
                                           c128*, long, const gdr_params&, gdr_defl**, gdr_report&);
template gdr_status solve_batch_pipeline<float>(gdr_ctx*, const gdr_op*, int, const std::vector<c128>&, const c128*,
                                                c128*, const gdr_params&, gdr_report&, int*);
template gdr_status solve_batch_pipeline<double>(gdr_ctx*, const gdr_op*, int, const std::vector<c128>&, const c128*,
                                                 c128*, const gdr_params&, gdr_report&, int*);
