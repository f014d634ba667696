// Operator kernels: y = (A - sigma_c I) x_c for ncol columns, optionally as the
// residual y = b - (A - sigma_c I) x_c.
//
//  * CSR matvec (the matrices of Examples 1-6, Sec. 3-4; convection-diffusion).
//  * Wilson-Dirac-style stencil A = a I - H (Example 7, Sec. 4):
//      (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu)
//    evaluated with the spin projection of the chiral basis: writing
//    gamma_mu = [[0, B_mu], [B_mu^H, 0]] with B_mu unitary 2x2,
//      (1 -+ gamma_mu) psi = [h ; -+ B_mu^H h],   h = u -+ B_mu d,   psi = [u ; d],
//    so each hop multiplies one link into a 2-spin half spinor only.
//
// Vectors are site-major (site*12 + spin*3 + colour).  Links are stored
// structure-of-arrays [mu][e][V] (e = a*3 + b) so that a warp's loads of one
// link element are contiguous.
#include <type_traits>

#include "common.cuh"
#include "wilson.cuh"

namespace {

// ------------------------------------------------------------- CSR kernel

template <typename R, typename VT>
__global__ void csr_kernel(long n, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const VT* __restrict__ vals, const c128* __restrict__ sigma,
                           const cx<R>* __restrict__ X, long ldx, cx<R>* __restrict__ Y, long ldy,
                           const cx<R>* __restrict__ B, long ldb, const int* __restrict__ run, int run_stride,
                           int cpp, const double* __restrict__ xs, int xs_stride) {
  const long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (r >= n) return;
  if (run && !run[(long)c * run_stride]) return;
  const cx<R>* x = X + c * ldx;
  cx<R> acc = {0, 0};
  const int p0 = rowptr[r], p1 = rowptr[r + 1];
  for (int p = p0; p < p1; ++p) {
    VT v = vals[p];
    cx<R> a = {(R)v.x, (R)v.y};
    acc += a * x[col[p]];
  }
  if (sigma) acc -= cvt<R>(sigma[c]) * x[r];
  if (xs) acc = (R)xs[(long)c * xs_stride] * acc;
  if (B) acc = B[(c / cpp) * ldb + r] - acc;
  Y[c * ldy + r] = acc;
}

// CSR batch: column c uses problem c / cpp (its own rows, local column indices)
template <typename R, typename VT>
__global__ void csr_batch_kernel(const long* __restrict__ rp_off, const long* __restrict__ nz_off,
                                 const int* __restrict__ nrow, const int* __restrict__ rowptr,
                                 const int* __restrict__ col, const VT* __restrict__ vals,
                                 const c128* __restrict__ sigma, const cx<R>* __restrict__ X, long ldx,
                                 cx<R>* __restrict__ Y, long ldy, const cx<R>* __restrict__ B, long ldb,
                                 const int* __restrict__ run, int run_stride, int cpp,
                                 const double* __restrict__ xs, int xs_stride) {
  const long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  const int p = c / cpp;
  if (r >= nrow[p]) return;
  if (run && !run[(long)c * run_stride]) return;
  const int* rp = rowptr + rp_off[p];
  const int* cl = col + nz_off[p];
  const VT* vl = vals + nz_off[p];
  const cx<R>* x = X + c * ldx;
  cx<R> acc = {0, 0};
  const int p0 = rp[r], p1 = rp[r + 1];
  for (int q = p0; q < p1; ++q) {
    const VT v = vl[q];
    acc += cx<R>{(R)v.x, (R)v.y} * x[cl[q]];
  }
  if (sigma) acc -= cvt<R>(sigma[c]) * x[r];
  if (xs) acc = (R)xs[(long)c * xs_stride] * acc;
  if (B) acc = B[(long)p * ldb + r] - acc;
  Y[c * ldy + r] = acc;
}

// ---------------------------------------------------------- Wilson kernel

template <typename R, typename LT>
__global__ void __launch_bounds__(128) wilson_kernel(const LT* __restrict__ links, int Lx, int Ly, int Lz, int Lt,
                                                    double diag_a, const c128* __restrict__ sigma,
                                                    const cx<R>* __restrict__ X, long ldx, cx<R>* __restrict__ Y,
                                                    long ldy, const cx<R>* __restrict__ B, long ldb,
                                                    const int* __restrict__ run, int run_stride, int cpp,
                                                    const double* __restrict__ xs, int xs_stride) {
  const long V = (long)Lx * Ly * Lz * Lt;
  const long site = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (site >= V) return;
  if (run && !run[(long)c * run_stride]) return;
  const cx<R>* x = X + c * ldx;
  long q = site;
  const int ix = (int)(q % Lx); q /= Lx;
  const int iy = (int)(q % Ly); q /= Ly;
  const int iz = (int)(q % Lz);
  const int it = (int)(q / Lz);
  Spinor<R> acc;
#pragma unroll
  for (int i = 0; i < 12; ++i) acc.s[i] = {0, 0};
  hop_mu<0, R, LT>(links, x, V, site, ix, Lx, 1, acc);
  hop_mu<1, R, LT>(links, x, V, site, iy, Ly, (long)Lx, acc);
  hop_mu<2, R, LT>(links, x, V, site, iz, Lz, (long)Lx * Ly, acc);
  hop_mu<3, R, LT>(links, x, V, site, it, Lt, (long)Lx * Ly * Lz, acc);
  // y = (a - sigma_c) x - H x   [ or b - that ]
  Spinor<R> p;
  load_spinor<R>(x, site, p);
  const c128 sg = sigma ? sigma[c] : c128{0.0, 0.0};
  const cx<R> dg = {(R)(diag_a - sg.x), (R)(-sg.y)};
  cx<R>* y = Y + c * ldy + site * 12;
  const cx<R>* b = B ? B + (c / cpp) * ldb + site * 12 : nullptr;
  const R sc = xs ? (R)xs[(long)c * xs_stride] : R(1);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    cx<R> v = sc * (dg * p.s[i] - acc.s[i]);
    if (b) v = b[i] - v;
    y[i] = v;
  }
}

// Small lattices: a block takes 32 sites and warp w computes the two hops in
// direction w for them (warp-uniform direction, a quarter of the per-thread
// dependency chain), the four partial spinors are summed through shared memory
// and the output, with the diagonal term, is written one component per thread
// (coalesced).  Used when one thread per site cannot fill the GPU.
template <typename R, typename LT>
__global__ void __launch_bounds__(128) wilson_split_kernel(const LT* __restrict__ links, int Lx, int Ly, int Lz,
                                                          int Lt, double diag_a, const c128* __restrict__ sigma,
                                                          const cx<R>* __restrict__ X, long ldx,
                                                          cx<R>* __restrict__ Y, long ldy,
                                                          const cx<R>* __restrict__ B, long ldb,
                                                          const int* __restrict__ run, int run_stride, int cpp,
                                                          const double* __restrict__ xs, int xs_stride) {
  __shared__ cx<R> part[4][32][13];  // odd row length: conflict-free in both phases
  const long V = (long)Lx * Ly * Lz * Lt;
  const int c = blockIdx.y;
  if (run && !run[(long)c * run_stride]) return;
  const int mu = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long site0 = blockIdx.x * 32L, site = site0 + lane;
  const cx<R>* x = X + c * ldx;
  Spinor<R> acc;
#pragma unroll
  for (int i = 0; i < 12; ++i) acc.s[i] = {0, 0};
  if (site < V) {
    long q = site;
    const int ix = (int)(q % Lx); q /= Lx;
    const int iy = (int)(q % Ly); q /= Ly;
    const int iz = (int)(q % Lz);
    const int it = (int)(q / Lz);
    switch (mu) {  // uniform in the warp
      case 0: hop_mu<0, R, LT>(links, x, V, site, ix, Lx, 1, acc); break;
      case 1: hop_mu<1, R, LT>(links, x, V, site, iy, Ly, (long)Lx, acc); break;
      case 2: hop_mu<2, R, LT>(links, x, V, site, iz, Lz, (long)Lx * Ly, acc); break;
      default: hop_mu<3, R, LT>(links, x, V, site, it, Lt, (long)Lx * Ly * Lz, acc); break;
    }
  }
#pragma unroll
  for (int i = 0; i < 12; ++i) part[mu][lane][i] = acc.s[i];
  __syncthreads();
  const c128 sg = sigma ? sigma[c] : c128{0.0, 0.0};
  const cx<R> dg = {(R)(diag_a - sg.x), (R)(-sg.y)};
  cx<R>* y = Y + c * ldy;
  const cx<R>* b = B ? B + (c / cpp) * ldb : nullptr;
  const long nout = min(32L, V - site0) * 12;
  const R sc = xs ? (R)xs[(long)c * xs_stride] : R(1);
  for (int q = threadIdx.x; q < nout; q += 128) {
    const int sl = q / 12, comp = q % 12;
    const cx<R> h = part[0][sl][comp] + part[1][sl][comp] + part[2][sl][comp] + part[3][sl][comp];
    const long e = site0 * 12 + q;
    cx<R> v = sc * (dg * x[e] - h);
    if (b) v = b[e] - v;
    y[e] = v;
  }
}

}  // namespace

template <typename R>
static void op_apply_launch(gdr_ctx* ctx, const gdr_op* A, int ncol, const c128* sigma, const cx<R>* X, long ldx,
                            cx<R>* Y, long ldy, const cx<R>* B, long ldb, const int* run, int run_stride, int cpp,
                            const double* xs, int xs_stride);

template <typename R>
static void op_apply_impl(gdr_ctx* ctx, const gdr_op* A, int ncol, const c128* sigma, const cx<R>* X, long ldx,
                          cx<R>* Y, long ldy, const cx<R>* B, long ldb, const int* run, int run_stride, int cpp,
                          const double* xs, int xs_stride) {
  if (ncol <= 0) return;
  constexpr bool F64 = std::is_same<R, double>::value;
  const double sv = sizeof(cx<R>);
  if (A->kind == OP_CSR || A->kind == OP_CSR_BATCH) {
    // row pointers, column indices, values, x read, y written (+ b read)
    const double bytes = (double)A->n * 4 + (double)A->nnz * (4 + (F64 ? 16 : 8)) +
                         (double)ncol * A->n * sv * (B ? 3 : 2);
    KProf kp(ctx, F64 ? "csr_matvec_c128" : "csr_matvec_c64", bytes);
    op_apply_launch<R>(ctx, A, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride);
  } else {
    // per site: 4 links of 18 reals, 24 reals of x read and of y written (+ b read)
    const double sl = F64 ? 8 : (A->store == GDR_LINK_BF16 ? 2 : 4);
    const double bytes = (double)A->V * (4 * 18 * sl + (double)ncol * 12 * sv * (B ? 3 : 2));
    KProf kp(ctx, F64 ? "wilson_matvec_c128" : (A->store == GDR_LINK_BF16 ? "wilson_matvec_c64_bf16links"
                                                                        : "wilson_matvec_c64"), bytes);
    op_apply_launch<R>(ctx, A, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride);
  }
}

template <typename R>
static void op_apply_launch(gdr_ctx* ctx, const gdr_op* A, int ncol, const c128* sigma, const cx<R>* X, long ldx,
                            cx<R>* Y, long ldy, const cx<R>* B, long ldb, const int* run, int run_stride, int cpp,
                          const double* xs, int xs_stride) {
  constexpr bool F64 = std::is_same<R, double>::value;
  if (A->kind == OP_CSR) {
    dim3 grid((unsigned)((A->n + 255) / 256), (unsigned)ncol);
    if (F64) {
      csr_kernel<double, c128><<<grid, 256, 0, ctx->stream>>>(
          A->n, A->rowptr, A->col, A->vals128, sigma, (const c128*)X, ldx, (c128*)Y, ldy, (const c128*)B, ldb, run,
          run_stride, cpp, xs, xs_stride);
    } else {
      csr_kernel<float, c64><<<grid, 256, 0, ctx->stream>>>(A->n, A->rowptr, A->col, A->vals64, sigma,
                                                             (const c64*)X, ldx, (c64*)Y, ldy, (const c64*)B, ldb,
                                                             run, run_stride, cpp, xs, xs_stride);
    }
    GDR_LAUNCHED(ctx);
  } else if (A->kind == OP_CSR_BATCH) {
    dim3 grid((unsigned)((A->n + 255) / 256), (unsigned)ncol);  // A->n = largest problem
    if (F64) {
      csr_batch_kernel<double, c128><<<grid, 256, 0, ctx->stream>>>(
          A->rp_off, A->nz_off, A->nrow, A->rowptr, A->col, A->vals128, sigma, (const c128*)X, ldx, (c128*)Y, ldy,
          (const c128*)B, ldb, run, run_stride, cpp, xs, xs_stride);
    } else {
      csr_batch_kernel<float, c64><<<grid, 256, 0, ctx->stream>>>(
          A->rp_off, A->nz_off, A->nrow, A->rowptr, A->col, A->vals64, sigma, (const c64*)X, ldx, (c64*)Y, ldy,
          (const c64*)B, ldb, run, run_stride, cpp, xs, xs_stride);
    }
    GDR_LAUNCHED(ctx);
  } else if ((A->V + 127) / 128 * ncol < 2L * ctx->num_sms) {
    // too few sites for one thread per site: direction-split form
    dim3 grid((unsigned)((A->V + 31) / 32), (unsigned)ncol);
    const int* d = A->dims;
    if (F64) {
      wilson_split_kernel<double, c128><<<grid, 128, 0, ctx->stream>>>(
          A->links128, d[0], d[1], d[2], d[3], A->diag_a, sigma, (const c128*)X, ldx, (c128*)Y, ldy, (const c128*)B,
          ldb, run, run_stride, cpp, xs, xs_stride);
    } else if (A->store == GDR_LINK_BF16) {
      wilson_split_kernel<float, __nv_bfloat162><<<grid, 128, 0, ctx->stream>>>(
          A->links16, d[0], d[1], d[2], d[3], A->diag_a, sigma, (const c64*)X, ldx, (c64*)Y, ldy, (const c64*)B, ldb,
          run, run_stride, cpp, xs, xs_stride);
    } else {
      wilson_split_kernel<float, c64><<<grid, 128, 0, ctx->stream>>>(
          A->links64, d[0], d[1], d[2], d[3], A->diag_a, sigma, (const c64*)X, ldx, (c64*)Y, ldy, (const c64*)B, ldb,
          run, run_stride, cpp, xs, xs_stride);
    }
    GDR_LAUNCHED(ctx);
  } else {
    dim3 grid((unsigned)((A->V + 127) / 128), (unsigned)ncol);
    const int* d = A->dims;
    if (F64) {
      wilson_kernel<double, c128><<<grid, 128, 0, ctx->stream>>>(A->links128, d[0], d[1], d[2], d[3], A->diag_a,
                                                                 sigma, (const c128*)X, ldx, (c128*)Y, ldy,
                                                                 (const c128*)B, ldb, run, run_stride, cpp, xs, xs_stride);
    } else if (A->store == GDR_LINK_BF16) {
      wilson_kernel<float, __nv_bfloat162><<<grid, 128, 0, ctx->stream>>>(
          A->links16, d[0], d[1], d[2], d[3], A->diag_a, sigma, (const c64*)X, ldx, (c64*)Y, ldy, (const c64*)B, ldb,
          run, run_stride, cpp, xs, xs_stride);
    } else {
      wilson_kernel<float, c64><<<grid, 128, 0, ctx->stream>>>(A->links64, d[0], d[1], d[2], d[3], A->diag_a, sigma,
                                                               (const c64*)X, ldx, (c64*)Y, ldy, (const c64*)B, ldb,
                                                               run, run_stride, cpp, xs, xs_stride);
    }
    GDR_LAUNCHED(ctx);
  }
}

void op_apply_skip(gdr_ctx* ctx, const gdr_op* A, int ncol, const c128* sigma, const c128* X, long ldx, c128* Y,
                   long ldy, const c128* B, long ldb, const int* run, int run_stride, int cpp, const double* xs,
                   int xs_stride) {
  op_apply_impl<double>(ctx, A, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride);
}
void op_apply_skip(gdr_ctx* ctx, const gdr_op* A, int ncol, const c128* sigma, const c64* X, long ldx, c64* Y,
                   long ldy, const c64* B, long ldb, const int* run, int run_stride, int cpp, const double* xs,
                   int xs_stride) {
  op_apply_impl<float>(ctx, A, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride);
}

template <typename R>
void op_apply(gdr_ctx* ctx, const gdr_op* A, int ncol, const c128* sigma, const cx<R>* X, long ldx, cx<R>* Y,
              long ldy, const cx<R>* B, long ldb, int cpp) {
  op_apply_skip(ctx, A, ncol, sigma, X, ldx, Y, ldy, B, ldb, nullptr, 0, cpp, nullptr, 0);
}
template void op_apply<double>(gdr_ctx*, const gdr_op*, int, const c128*, const c128*, long, c128*, long, const c128*,
                               long, int);
template void op_apply<float>(gdr_ctx*, const gdr_op*, int, const c128*, const c64*, long, c64*, long, const c64*,
                              long, int);

// ------------------------------------------------------ operator creation

namespace {
__global__ void links_soa_kernel(const c128* __restrict__ in, long V, c128* o128, c64* o64, __nv_bfloat162* o16) {
  // in: [mu][V][9] (AoS, API layout) -> out [mu][e][V]
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= 4 * V * 9) return;
  const long mu = t / (V * 9);
  const long rem = t % (V * 9);
  const long site = rem / 9;
  const int e = (int)(rem % 9);
  const c128 u = in[t];
  const long o = (mu * 9 + e) * V + site;
  o128[o] = u;
  if (o64) o64[o] = to64(u);
  if (o16) o16[o] = __floats2bfloat162_rn((float)u.x, (float)u.y);
}
__global__ void vals_to64_kernel(const c128* __restrict__ in, long n, c64* out) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t < n) out[t] = to64(in[t]);
}
}  // namespace

void op_build_csr(gdr_ctx* ctx, gdr_op* op, const int* rowptr, const int* col, const double* vals) {
  GDR_CUDA(cudaMalloc(&op->rowptr, (op->n + 1) * sizeof(int)));
  GDR_CUDA(cudaMalloc(&op->col, std::max<long>(op->nnz, 1) * sizeof(int)));
  GDR_CUDA(cudaMalloc(&op->vals128, std::max<long>(op->nnz, 1) * sizeof(c128)));
  GDR_CUDA(cudaMalloc(&op->vals64, std::max<long>(op->nnz, 1) * sizeof(c64)));
  GDR_CUDA(cudaMemcpyAsync(op->rowptr, rowptr, (op->n + 1) * sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
  if (op->nnz > 0) {
    GDR_CUDA(cudaMemcpyAsync(op->col, col, op->nnz * sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
    GDR_CUDA(cudaMemcpyAsync(op->vals128, vals, op->nnz * sizeof(c128), cudaMemcpyDeviceToDevice, ctx->stream));
    vals_to64_kernel<<<(unsigned)((op->nnz + 255) / 256), 256, 0, ctx->stream>>>(op->vals128, op->nnz, op->vals64);
    GDR_LAUNCHED(ctx);
  }
  GDR_CUDA(cudaStreamSynchronize(ctx->stream));
}

void op_build_wilson(gdr_ctx* ctx, gdr_op* op, const double* links) {
  const long nl = 4 * op->V * 9;
  GDR_CUDA(cudaMalloc(&op->links128, nl * sizeof(c128)));
  if (op->store == GDR_LINK_BF16) {
    GDR_CUDA(cudaMalloc(&op->links16, nl * sizeof(__nv_bfloat162)));
  } else {
    GDR_CUDA(cudaMalloc(&op->links64, nl * sizeof(c64)));
  }
  links_soa_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, ctx->stream>>>((const c128*)links, op->V, op->links128,
                                                                          op->links64, op->links16);
  GDR_LAUNCHED(ctx);
  GDR_CUDA(cudaStreamSynchronize(ctx->stream));
}

void op_build_csr_batch(gdr_ctx* ctx, gdr_op* op, const long* n, const long* nnz, const int* rowptr, const int* col,
                        const double* vals) {
  std::vector<long> rp(op->nprob), nz(op->nprob);
  std::vector<int> nr(op->nprob);
  long rtot = 0, ztot = 0, nmax = 0;
  for (int p = 0; p < op->nprob; ++p) {
    rp[p] = rtot;
    nz[p] = ztot;
    nr[p] = (int)n[p];
    rtot += n[p] + 1;
    ztot += nnz[p];
    nmax = std::max(nmax, n[p]);
  }
  op->n = nmax;
  op->nnz = ztot;
  op->nrow_host.assign(n, n + op->nprob);
  GDR_CUDA(cudaMalloc(&op->rowptr, rtot * sizeof(int)));
  GDR_CUDA(cudaMalloc(&op->col, std::max<long>(ztot, 1) * sizeof(int)));
  GDR_CUDA(cudaMalloc(&op->vals128, std::max<long>(ztot, 1) * sizeof(c128)));
  GDR_CUDA(cudaMalloc(&op->vals64, std::max<long>(ztot, 1) * sizeof(c64)));
  GDR_CUDA(cudaMalloc(&op->rp_off, op->nprob * sizeof(long)));
  GDR_CUDA(cudaMalloc(&op->nz_off, op->nprob * sizeof(long)));
  GDR_CUDA(cudaMalloc(&op->nrow, op->nprob * sizeof(int)));
  GDR_CUDA(cudaMemcpyAsync(op->rowptr, rowptr, rtot * sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
  if (ztot > 0) {
    GDR_CUDA(cudaMemcpyAsync(op->col, col, ztot * sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
    GDR_CUDA(cudaMemcpyAsync(op->vals128, vals, ztot * sizeof(c128), cudaMemcpyDeviceToDevice, ctx->stream));
    vals_to64_kernel<<<(unsigned)((ztot + 255) / 256), 256, 0, ctx->stream>>>(op->vals128, ztot, op->vals64);
    GDR_LAUNCHED(ctx);
  }
  GDR_CUDA(cudaMemcpyAsync(op->rp_off, rp.data(), op->nprob * sizeof(long), cudaMemcpyHostToDevice, ctx->stream));
  GDR_CUDA(cudaMemcpyAsync(op->nz_off, nz.data(), op->nprob * sizeof(long), cudaMemcpyHostToDevice, ctx->stream));
  GDR_CUDA(cudaMemcpyAsync(op->nrow, nr.data(), op->nprob * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  GDR_CUDA(cudaStreamSynchronize(ctx->stream));
}
