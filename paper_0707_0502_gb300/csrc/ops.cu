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
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "wilson.cuh"

double run_share(gdr_ctx* ctx, int ncol, const int* run, int run_stride, const int* nvec);

namespace {

// ------------------------------------------------------------- CSR kernel

// Block -> (tile, column).  col_inner: consecutive blocks take one tile for
// consecutive columns, so the tile's links or matrix rows are fetched from HBM
// once and served from L2 to the other columns' blocks running beside it.  With
// col_inner = g >= 2 that order holds within groups of g columns and the groups
// follow one another (the last may be narrower): the links are fetched once per
// group, and a neighbour read a few planes of sites later still finds the
// group's vectors in L2, which all columns at once would have pushed out.
DEV void tile_col(int ncol, int col_inner, long& tile, int& c) {
  if (col_inner) {
    const unsigned G = (col_inner == 1 || col_inner > ncol) ? (unsigned)ncol : (unsigned)col_inner;
    const unsigned span = gridDim.x / (unsigned)ncol * G;  // blocks of one full group
    const unsigned grp = blockIdx.x / span, r = blockIdx.x - grp * span;
    const unsigned gw = min(G, (unsigned)ncol - grp * G);  // this group's width
    tile = r / gw;
    c = (int)(grp * G + r % gw);
  } else {
    tile = blockIdx.x;
    c = blockIdx.y;
  }
}

// sum over the TPR lanes of a row (TPR consecutive lanes of one warp)
template <int TPR, typename R>
DEV cx<R> row_sum(cx<R> acc) {
  if constexpr (TPR > 1) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned mask = ((1u << TPR) - 1u) << (lane & ~(unsigned)(TPR - 1));
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(mask, acc.x, o, TPR);
      acc.y += __shfl_xor_sync(mask, acc.y, o, TPR);
    }
  }
  return acc;
}

// y_r = (A x)_r with TPR threads per row (blockDim.x / TPR rows per block)
template <typename R, typename VT, int TPR>
__global__ void csr_kernel(long n, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const VT* __restrict__ vals, const c128* __restrict__ sigma,
                           const cx<R>* __restrict__ X, long ldx, cx<R>* __restrict__ Y, long ldy,
                           const cx<R>* __restrict__ B, long ldb, const int* __restrict__ run, int run_stride,
                           int cpp, const double* __restrict__ xs, int xs_stride, int ncol, int col_inner) {
  long tile;
  int c;
  tile_col(ncol, col_inner, tile, c);
  const long r = tile * (blockDim.x / TPR) + threadIdx.x / TPR;
  if (r >= n) return;  // uniform over the row's lanes
  if (run && !run[(long)c * run_stride]) return;
  const cx<R>* x = X + c * ldx;
  cx<R> acc = {0, 0};
  const int p0 = rowptr[r], p1 = rowptr[r + 1];
  for (int p = p0 + (int)(threadIdx.x % TPR); p < p1; p += TPR) {
    VT v = vals[p];
    cx<R> a = {(R)v.x, (R)v.y};
    acc += a * x[col[p]];
  }
  acc = row_sum<TPR>(acc);
  if (TPR > 1 && threadIdx.x % TPR) return;
  if (sigma) acc -= cvt<R>(sigma[c]) * x[r];
  if (xs) acc = (R)xs[(long)c * xs_stride] * acc;
  if (B) acc = B[(c / cpp) * ldb + r] - acc;
  Y[c * ldy + r] = acc;
}

// CSR batch: column c uses problem c / cpp (its own rows, local column indices)
template <typename R, typename VT, int TPR>
__global__ void csr_batch_kernel(const long* __restrict__ rp_off, const long* __restrict__ nz_off,
                                 const int* __restrict__ nrow, const int* __restrict__ rowptr,
                                 const int* __restrict__ col, const VT* __restrict__ vals,
                                 const c128* __restrict__ sigma, const cx<R>* __restrict__ X, long ldx,
                                 cx<R>* __restrict__ Y, long ldy, const cx<R>* __restrict__ B, long ldb,
                                 const int* __restrict__ run, int run_stride, int cpp,
                                 const double* __restrict__ xs, int xs_stride, int ncol, int col_inner) {
  long tile;
  int c;
  tile_col(ncol, col_inner, tile, c);
  const long r = tile * (blockDim.x / TPR) + threadIdx.x / TPR;
  const int p = c / cpp;
  if (r >= nrow[p]) return;
  if (run && !run[(long)c * run_stride]) return;
  const int* rp = rowptr + rp_off[p];
  const int* cl = col + nz_off[p];
  const VT* vl = vals + nz_off[p];
  const cx<R>* x = X + c * ldx;
  cx<R> acc = {0, 0};
  const int p0 = rp[r], p1 = rp[r + 1];
  for (int q = p0 + (int)(threadIdx.x % TPR); q < p1; q += TPR) {
    const VT v = vl[q];
    acc += cx<R>{(R)v.x, (R)v.y} * x[cl[q]];
  }
  acc = row_sum<TPR>(acc);
  if (TPR > 1 && threadIdx.x % TPR) return;
  if (sigma) acc -= cvt<R>(sigma[c]) * x[r];
  if (xs) acc = (R)xs[(long)c * xs_stride] * acc;
  if (B) acc = B[(long)p * ldb + r] - acc;
  Y[c * ldy + r] = acc;
}

// ---------------------------------------------------------- Wilson kernel

// Resident warps: the matvec is bound by the latency of its neighbour gathers, so
// the registers are capped for 24 resident warps per SM (complex64: 80 registers)
// or 16 (complex128: 128 registers) instead of the compiler's choice (16 warps).
template <typename R>
constexpr int wilson_min_blocks(int nt) {
  return (sizeof(R) == 4 ? 768 : 512) / nt;
}

template <typename R, typename LT, int NT>
__global__ void __launch_bounds__(NT, wilson_min_blocks<R>(NT)) wilson_kernel(const LT* __restrict__ links, int Lx, int Ly, int Lz, int Lt,
                                                   double diag_a, const c128* __restrict__ sigma,
                                                   const cx<R>* __restrict__ X, long ldx, cx<R>* __restrict__ Y,
                                                   long ldy, const cx<R>* __restrict__ B, long ldb,
                                                   const int* __restrict__ run, int run_stride, int cpp,
                                                   const double* __restrict__ xs, int xs_stride, int ncol,
                                                   int col_inner) {
  const long V = (long)Lx * Ly * Lz * Lt;
  long tile;
  int c;
  tile_col(ncol, col_inner, tile, c);
  const long site = tile * NT + threadIdx.x;
  if (site >= V) return;
  if (run && !run[(long)c * run_stride]) return;
  const cx<R>* x = X + c * ldx;
  int ix, iy, iz, it;
  site_coords(site, Lx, Ly, Lz, ix, iy, iz, it);
  Spinor<R> acc;
#pragma unroll
  for (int i = 0; i < 12; ++i) acc.s[i] = {0, 0};
  hop_mu<0, R, LT>(links, x, V, site, ix, Lx, 1, acc);
  hop_mu<1, R, LT>(links, x, V, site, iy, Ly, (long)Lx, acc);
  hop_mu<2, R, LT>(links, x, V, site, iz, Lz, (long)Lx * Ly, acc);
  hop_mu<3, R, LT>(links, x, V, site, it, Lt, (long)Lx * Ly * Lz, acc);
  // y = (a - sigma_c) x - H x   [ or b - that ]
  Spinor<R> p;
  load_spinor<R>(x, V, site, p);
  const c128 sg = sigma ? sigma[c] : c128{0.0, 0.0};
  const cx<R> dg = {(R)(diag_a - sg.x), (R)(-sg.y)};
  cx<R>* y = Y + c * ldy;
  const R sc = xs ? (R)xs[(long)c * xs_stride] : R(1);
  const cx<R>* b = B ? B + (c / cpp) * ldb : nullptr;
  // (a - sigma) x - H x or b + H x - (a - sigma) x as FMA chains (two FMAs and at most one
  // add per real component; the unscaled forms skip the multiplication by s_c = 1)
  auto out = [&](cx<R> xv, cx<R> av, cx<R> bv, bool hasb) -> cx<R> {
    if (hasb) {
      const R ur = bv.x + av.x, ui = bv.y + av.y;
      return {fma(dg.y, xv.y, fma(-dg.x, xv.x, ur)), fma(-dg.y, xv.x, fma(-dg.x, xv.y, ui))};
    }
    return {fma(-dg.y, xv.y, fma(dg.x, xv.x, -av.x)), fma(dg.y, xv.x, fma(dg.x, xv.y, -av.y))};
  };
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    cx<R> v0, v1;
    if (xs) {
      v0 = sc * (dg * p.s[2 * i] - acc.s[2 * i]);
      v1 = sc * (dg * p.s[2 * i + 1] - acc.s[2 * i + 1]);
      if (b) {
        cx<R> b0, b1;
        load_pair<R>(b, V, site, i, b0, b1);
        v0 = b0 - v0;
        v1 = b1 - v1;
      }
    } else if (b) {
      cx<R> b0, b1;
      load_pair<R>(b, V, site, i, b0, b1);
      v0 = out(p.s[2 * i], acc.s[2 * i], b0, true);
      v1 = out(p.s[2 * i + 1], acc.s[2 * i + 1], b1, true);
    } else {
      v0 = out(p.s[2 * i], acc.s[2 * i], {0, 0}, false);
      v1 = out(p.s[2 * i + 1], acc.s[2 * i + 1], {0, 0}, false);
    }
    store_pair<R>(y, V, site, i, v0, v1);
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
                                                          const double* __restrict__ xs, int xs_stride, int ncol,
                                                          int col_inner) {
  __shared__ cx<R> part[4][32][13];  // odd row length: conflict-free in both phases
  const long V = (long)Lx * Ly * Lz * Lt;
  long tile;
  int c;
  tile_col(ncol, col_inner, tile, c);
  if (run && !run[(long)c * run_stride]) return;
  const int mu = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long site0 = tile * 32L, site = site0 + lane;
  const cx<R>* x = X + c * ldx;
  Spinor<R> acc;
#pragma unroll
  for (int i = 0; i < 12; ++i) acc.s[i] = {0, 0};
  if (site < V) {
    int ix, iy, iz, it;
    site_coords(site, Lx, Ly, Lz, ix, iy, iz, it);
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
  const R sc = xs ? (R)xs[(long)c * xs_stride] : R(1);
  // output element q: pair q / 64, site q % 64 / 2, half q % 2 (64 consecutive elements of a pair)
  for (int q = threadIdx.x; q < 6 * 64; q += 128) {
    const int pr = q >> 6, sl = (q & 63) >> 1, comp = 2 * pr + (q & 1);
    if (site0 + sl >= V) continue;
    const cx<R> h = part[0][sl][comp] + part[1][sl][comp] + part[2][sl][comp] + part[3][sl][comp];
    const long e = 2 * ((long)pr * V + site0) + (q & 63);
    cx<R> v = sc * (dg * x[e] - h);
    if (b) v = b[e] - v;
    y[e] = v;
  }
}

// Column pairs (complex64 vectors): a thread takes one site for columns 2p and 2p + 1
// and computes both with packed FP32x2 arithmetic (hop2); an odd last column is paired
// with itself and stored once.  Same operator and output as wilson_kernel.
// Registers are capped for 16 resident warps per SM (128 registers): with 12 warps and no
// cap (168 registers) the same kernel was 17% slower at 24^3x32, 12 columns.
template <typename LT, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) wilson_pair_kernel(
    const LT* __restrict__ links, int Lx, int Ly, int Lz, int Lt, double diag_a, const c128* __restrict__ sigma,
    const c64* __restrict__ X, long ldx, c64* __restrict__ Y, long ldy, const c64* __restrict__ B, long ldb,
    const int* __restrict__ run, int run_stride, int cpp, const double* __restrict__ xs, int xs_stride, int ncol,
    int col_inner) {
  const long V = (long)Lx * Ly * Lz * Lt;
  const int npair = (ncol + 1) / 2;
  long tile;
  int cp;
  tile_col(npair, col_inner, tile, cp);
  const long site = tile * NT + threadIdx.x;
  if (site >= V) return;
  const int c0 = 2 * cp, c1 = min(2 * cp + 1, ncol - 1);
  const bool st0 = !run || run[(long)c0 * run_stride];
  const bool st1 = c1 != c0 && (!run || run[(long)c1 * run_stride]);
  if (!st0 && !st1) return;
  const c64* x0 = X + c0 * ldx;
  const c64* x1 = X + c1 * ldx;
  int ix, iy, iz, it;
  site_coords(site, Lx, Ly, Lz, ix, iy, iz, it);
  Spinor2 acc;
#pragma unroll
  for (int i = 0; i < 12; ++i) acc.s[i] = {0ull, 0ull};
  hop_mu2<0, LT>(links, x0, x1, V, site, ix, Lx, 1, acc);
  hop_mu2<1, LT>(links, x0, x1, V, site, iy, Ly, (long)Lx, acc);
  hop_mu2<2, LT>(links, x0, x1, V, site, iz, Lz, (long)Lx * Ly, acc);
  hop_mu2<3, LT>(links, x0, x1, V, site, it, Lt, (long)Lx * Ly * Lz, acc);
  // y = (a - sigma_c) x - H x   [ or b - that ]
  Spinor2 p;
  load_spinor2(x0, x1, V, site, p);
  const c128 s0 = sigma ? sigma[c0] : c128{0.0, 0.0}, s1 = sigma ? sigma[c1] : c128{0.0, 0.0};
  const f2 dr = f2_pack((float)(diag_a - s0.x), (float)(diag_a - s1.x));
  const f2 di = f2_pack((float)(-s0.y), (float)(-s1.y)), ndi = f2_pack((float)s0.y, (float)s1.y);
  const f2 sc = f2_pack(xs ? (float)xs[(long)c0 * xs_stride] : 1.f, xs ? (float)xs[(long)c1 * xs_stride] : 1.f);
  const c64* b0 = B ? B + (c0 / cpp) * ldb : nullptr;
  const c64* b1 = B ? B + (c1 / cpp) * ldb : nullptr;
  float4* y0 = reinterpret_cast<float4*>(Y + c0 * ldy) + site;
  float4* y1 = reinterpret_cast<float4*>(Y + c1 * ldy) + site;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    cx2 v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const cx2 xv = p.s[2 * i + h], av = acc.s[2 * i + h];
      const f2 tr = f2_fma(ndi, xv.im, f2_sub(f2_mul(dr, xv.re), av.re));
      const f2 ti = f2_fma(di, xv.re, f2_sub(f2_mul(dr, xv.im), av.im));
      v[h] = {f2_mul(sc, tr), f2_mul(sc, ti)};
    }
    if (b0) {
      const float4 u0 = __ldg(reinterpret_cast<const float4*>(b0) + i * V + site);
      const float4 u1 = __ldg(reinterpret_cast<const float4*>(b1) + i * V + site);
      v[0] = {f2_sub(f2_pack(u0.x, u1.x), v[0].re), f2_sub(f2_pack(u0.y, u1.y), v[0].im)};
      v[1] = {f2_sub(f2_pack(u0.z, u1.z), v[1].re), f2_sub(f2_pack(u0.w, u1.w), v[1].im)};
    }
    float a0r, a1r, a0i, a1i, b0r, b1r, b0i, b1i;
    f2_unpack(v[0].re, a0r, a1r);
    f2_unpack(v[0].im, a0i, a1i);
    f2_unpack(v[1].re, b0r, b1r);
    f2_unpack(v[1].im, b0i, b1i);
    if (st0) y0[i * V] = make_float4(a0r, a0i, b0r, b0i);
    if (st1) y1[i * V] = make_float4(a1r, a1i, b1r, b1i);
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
  const double act = run_share(ctx, ncol, run, run_stride, nullptr);  // profiler: columns still running
  if (A->kind == OP_CSR || A->kind == OP_CSR_BATCH) {
    // row pointers, column indices, values, x read, y written (+ b read)
    const double bytes = (double)A->n * 4 + (double)A->nnz * (4 + (F64 ? 16 : 8)) +
                         act * (double)ncol * A->n * sv * (B ? 3 : 2);
    KProf kp(ctx, F64 ? "csr_matvec_c128" : "csr_matvec_c64", bytes);
    op_apply_launch<R>(ctx, A, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride);
  } else {
    // per site: 4 links of 18 reals, 24 reals of x read and of y written (+ b read)
    const double sl = F64 ? 8 : (A->store == GDR_LINK_BF16 ? 2 : 4);
    const double bytes = (double)A->V * (4 * 18 * sl + act * (double)ncol * 12 * sv * (B ? 3 : 2));
    KProf kp(ctx, F64 ? "wilson_matvec_c128" : (A->store == GDR_LINK_BF16 ? "wilson_matvec_c64_bf16links"
                                                                        : "wilson_matvec_c64"), bytes);
    op_apply_launch<R>(ctx, A, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride);
  }
}

MvShape mv_default(const gdr_ctx* ctx, const gdr_op* A, int ncol);

MvShape mv_shape(const gdr_ctx* ctx, const gdr_op* A, bool f64, int ncol) {
  const int fk = f64 ? 1 : 0;
  auto it = A->mv_tuned.find({fk, ncol});
  if (it != A->mv_tuned.end()) return it->second;
  const MvShape* near = nullptr;
  double best = std::log(2.0) + 1e-9;
  for (const auto& kv : A->mv_tuned) {
    if (kv.first.first != fk) continue;
    const double r = std::fabs(std::log((double)kv.first.second / (double)ncol));
    if (r <= best) {
      best = r;
      near = &kv.second;
    }
  }
  if (near) return *near;
  return mv_default(ctx, A, ncol);
}

MvShape mv_default(const gdr_ctx* ctx, const gdr_op* A, int ncol) {
  MvShape s;
  if (A->kind == OP_WILSON) {
    // too few sites for one thread per site: direction-split form
    s.form = ((A->V + 127) / 128 * ncol < 2L * ctx->num_sms) ? 1 : 0;
    s.threads = 128;
  } else {
    s.form = 1;
    s.threads = 256;
  }
  // several columns sharing one operator: consecutive blocks take one tile for all
  // columns, so its links / rows are read from HBM once (column by column, each
  // column's pass evicts them from L2 on large problems)
  s.col_inner = (ncol > 1 && A->kind != OP_CSR_BATCH) ? 1 : 0;
  return s;
}

// grid of `tiles` tiles for ncol columns in the shape's column order
static dim3 tile_grid(long tiles, int ncol, int col_inner) {
  return col_inner ? dim3((unsigned)(tiles * ncol), 1) : dim3((unsigned)tiles, (unsigned)ncol);
}

template <typename R, typename VT, int TPR>
static void csr_launch(gdr_ctx* ctx, const gdr_op* A, const VT* vals, const MvShape& s, int ncol, const c128* sigma,
                       const cx<R>* X, long ldx, cx<R>* Y, long ldy, const cx<R>* B, long ldb, const int* run,
                       int run_stride, int cpp, const double* xs, int xs_stride) {
  const long rows = s.threads / TPR;
  const dim3 grid = tile_grid((A->n + rows - 1) / rows, ncol, s.col_inner);  // A->n: largest problem of a batch
  if (A->kind == OP_CSR)
    csr_kernel<R, VT, TPR><<<grid, s.threads, 0, ctx->stream>>>(A->n, A->rowptr, A->col, vals, sigma, X, ldx, Y, ldy,
                                                                 B, ldb, run, run_stride, cpp, xs, xs_stride, ncol,
                                                                 s.col_inner);
  else
    csr_batch_kernel<R, VT, TPR><<<grid, s.threads, 0, ctx->stream>>>(
        A->rp_off, A->nz_off, A->nrow, A->rowptr, A->col, vals, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp,
        xs, xs_stride, ncol, s.col_inner);
  GDR_LAUNCHED(ctx);
}

template <typename R, typename LT>
static void wilson_launch(gdr_ctx* ctx, const gdr_op* A, const LT* links, const MvShape& s, int ncol,
                          const c128* sigma, const cx<R>* X, long ldx, cx<R>* Y, long ldy, const cx<R>* B, long ldb,
                          const int* run, int run_stride, int cpp, const double* xs, int xs_stride) {
  const int* d = A->dims;
  if constexpr (std::is_same<R, float>::value) {
    if (s.form == 2) {  // column pairs, packed FP32x2
      const int npair = (ncol + 1) / 2;
#define GDR_WILSON_PAIR(NT)                                                                                          \
  wilson_pair_kernel<LT, NT><<<tile_grid((A->V + NT - 1) / NT, npair, s.col_inner), NT, 0, ctx->stream>>>(         \
      links, d[0], d[1], d[2], d[3], A->diag_a, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride, \
      ncol, s.col_inner)
      if (s.threads == 64) GDR_WILSON_PAIR(64);
      else GDR_WILSON_PAIR(128);
#undef GDR_WILSON_PAIR
      GDR_LAUNCHED(ctx);
      return;
    }
  }
  if (s.form == 1) {
    wilson_split_kernel<R, LT><<<tile_grid((A->V + 31) / 32, ncol, s.col_inner), 128, 0, ctx->stream>>>(
        links, d[0], d[1], d[2], d[3], A->diag_a, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride,
        ncol, s.col_inner);
  } else {
#define GDR_WILSON_SITE(NT)                                                                                         \
  wilson_kernel<R, LT, NT><<<tile_grid((A->V + NT - 1) / NT, ncol, s.col_inner), NT, 0, ctx->stream>>>(             \
      links, d[0], d[1], d[2], d[3], A->diag_a, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride, \
      ncol, s.col_inner)
    if (s.threads == 64) GDR_WILSON_SITE(64);
    else if (s.threads == 256) GDR_WILSON_SITE(256);
    else GDR_WILSON_SITE(128);
#undef GDR_WILSON_SITE
  }
  GDR_LAUNCHED(ctx);
}

template <typename R>
static void op_apply_launch(gdr_ctx* ctx, const gdr_op* A, int ncol, const c128* sigma, const cx<R>* X, long ldx,
                            cx<R>* Y, long ldy, const cx<R>* B, long ldb, const int* run, int run_stride, int cpp,
                            const double* xs, int xs_stride) {
  constexpr bool F64 = std::is_same<R, double>::value;
  const MvShape s = mv_shape(ctx, A, F64, ncol);
  if (A->kind == OP_CSR || A->kind == OP_CSR_BATCH) {
    using VT = typename std::conditional<F64, c128, c64>::type;
    const VT* vals;
    if constexpr (F64) vals = A->vals128;
    else vals = A->vals64;
    switch (s.form) {
      case 2: csr_launch<R, VT, 2>(ctx, A, vals, s, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride); break;
      case 4: csr_launch<R, VT, 4>(ctx, A, vals, s, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride); break;
      case 8: csr_launch<R, VT, 8>(ctx, A, vals, s, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride); break;
      default: csr_launch<R, VT, 1>(ctx, A, vals, s, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs, xs_stride); break;
    }
  } else if constexpr (F64) {
    wilson_launch<R, c128>(ctx, A, A->links128, s, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs,
                           xs_stride);
  } else if (A->store == GDR_LINK_BF16) {
    wilson_launch<R, __nv_bfloat162>(ctx, A, A->links16, s, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp,
                                     xs, xs_stride);
  } else {
    wilson_launch<R, c64>(ctx, A, A->links64, s, ncol, sigma, X, ldx, Y, ldy, B, ldb, run, run_stride, cpp, xs,
                          xs_stride);
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

// ------------------------------------------ vector order at the C interface

namespace {
// site-major (s*12 + q) <-> pair-major (2 ((q/2) V + s) + q%2) Wilson vectors; the
// pair-major side is walked contiguously
template <typename T>
__global__ void wilson_order_kernel(long V, const T* __restrict__ in, long ldi, T* __restrict__ out, long ldo,
                                    int to_lib) {
  const int c = blockIdx.y;
  const long n = 12 * V;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long pv = i >> 1;
    const long p = pv / V, site = pv - p * V;
    const long u = site * 12 + 2 * p + (i & 1);
    if (to_lib) out[c * ldo + i] = in[c * ldi + u];
    else out[c * ldo + u] = in[c * ldi + i];
  }
}
}  // namespace

template <typename T>
void wilson_order(gdr_ctx* ctx, long V, int cols, const T* in, long ldi, T* out, long ldo, bool to_lib) {
  if (cols <= 0) return;
  GDR_REQUIRE(in != out, "vector reordering needs distinct buffers");
  dim3 grid((unsigned)std::min<long>((12 * V + 255) / 256, 8L * ctx->num_sms), (unsigned)cols);
  wilson_order_kernel<T><<<grid, 256, 0, ctx->stream>>>(V, in, ldi, out, ldo, to_lib ? 1 : 0);
  GDR_LAUNCHED(ctx);
}
template void wilson_order<c128>(gdr_ctx*, long, int, const c128*, long, c128*, long, bool);

template <typename T>
void op_order(gdr_ctx* ctx, const gdr_op* A, int cols, const T* in, long ldi, T* out, long ldo, bool to_lib) {
  if (cols <= 0) return;
  if (A->kind == OP_WILSON) {
    wilson_order<T>(ctx, A->V, cols, in, ldi, out, ldo, to_lib);
  } else if (in != out) {
    GDR_CUDA(cudaMemcpy2DAsync(out, ldo * sizeof(T), in, ldi * sizeof(T), A->n * sizeof(T), cols,
                               cudaMemcpyDeviceToDevice, ctx->stream));
  }
}
template void op_order<c128>(gdr_ctx*, const gdr_op*, int, const c128*, long, c128*, long, bool);
template void op_order<c64>(gdr_ctx*, const gdr_op*, int, const c64*, long, c64*, long, bool);

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

