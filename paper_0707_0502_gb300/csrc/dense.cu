// Small dense FP64 steps of the cycle, one CTA per (column, task), matrices in
// shared memory.
//
//  * GMRES-Sh reduced solves (Sec. 2.1, eqs. gsh1-gsh3; GMRES-DR-Sh steps 3-5):
//      base  d_1 = argmin ||c - (Hbar - sigma_1 Ibar) d||,  s = c - (Hbar - sigma_1 Ibar) d_1
//      shift i: QR of Hbar - sigma_i Ibar, R d_i = beta_i Q^H c - beta_new Q^H s, the
//      zero last row of R giving beta_new.
//  * GMRES-DR restart (Sec. 2.2; formula of the cited GMRES-DR paper): harmonic
//    Ritz pairs of Hhat = Hbar - sigma_1 Ibar from M = H + f hrow with H^H f = hrow^H,
//    M reduced to Hessenberg form, complex single-shift QR with Schur vectors,
//    eigenvectors of the triangular factor by back substitution, the k of smallest
//    |theta| orthonormalised into P_k; then p_{k+1} from s, Hbar_k = P^H Hbar P_k,
//    c_k = P^H s.
//  * Minres projection over V_k (Sec. 2.3) and the non-base update of
//    GMRES-Proj-Sh step 4: (H_k - sigma_i I) d_i = beta_i (H_k - sigma_1 I) d_1.
//
// All arithmetic is FP64.  Householder reflectors follow the usual complex
// convention: H = I - tau v v^H, v_0 = 1, H^H [alpha; x] = [beta; 0], beta real.
#include "kernels.cuh"

// Phase marks for timing studies; empty in the library build.
#ifndef GDR_DENSE_MARK
#define GDR_DENSE_MARK(i, v)
#endif

namespace {

constexpr int DT = 128;  // threads per dense CTA
constexpr unsigned FULL = 0xffffffffu;
// precision-dependent limits of the dense steps
template <typename R> struct Lim;
template <> struct Lim<double> {
  static constexpr double eps = 2.220446049250313e-16;
  static constexpr double tie = 1e-9;  // relative width of a tie in the selection order
  static constexpr double tiny = 1e-300;
};
template <> struct Lim<float> {
  static constexpr float eps = 1.1920929e-7f;
  static constexpr float tie = 2e-5f;
  static constexpr float tiny = 1e-30f;
};

DEV double sqrt_(double a) { return sqrt(a); }
DEV float sqrt_(float a) { return sqrtf(a); }
DEV double fabs_(double a) { return fabs(a); }
DEV float fabs_(float a) { return fabsf(a); }
DEV double fmax_(double a, double b) { return fmax(a, b); }
DEV float fmax_(float a, float b) { return fmaxf(a, b); }
DEV double copysign_(double a, double b) { return copysign(a, b); }
DEV float copysign_(float a, float b) { return copysignf(a, b); }
DEV double hypot_(double a, double b) { return hypot(a, b); }
DEV float hypot_(float a, float b) { return hypotf(a, b); }

template <typename R> DEV cx<R> cdiv(cx<R> a, cx<R> b) {
  const R d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
template <typename R> DEV R cabs_(cx<R> a) { return hypot_(a.x, a.y); }
template <typename R> DEV cx<R> csqrt_(cx<R> z) {
  const R r = cabs_(z);
  if (r == R(0)) return {0, 0};
  const R re = sqrt_(R(0.5) * (r + fabs_(z.x)));
  if (z.x >= R(0)) return {re, z.y / (2 * re)};
  return {fabs_(z.y) / (2 * re), copysign_(re, z.y)};
}
template <typename R> DEV cx<R> shfl_xor_c(cx<R> v, int m) {
  return {__shfl_xor_sync(FULL, v.x, m), __shfl_xor_sync(FULL, v.y, m)};
}
template <typename R> DEV cx<R> warp_sum_c(cx<R> v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += shfl_xor_c(v, m);
  return v;
}
template <typename R> DEV R warp_sum_r(R v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(FULL, v, m);
  return v;
}

template <typename R>
struct ShT {  // small shared scratch of a dense CTA
  R red[DT / 32];
  cx<R> bc[4];
  cx<R> nx[4];  // QR sweep: entries (kk+1, kk), (kk+1, kk+1), (kk+2, kk), (kk+2, kk+1) after the left update
  int ibc[4];
};
using Sh = ShT<double>;

template <typename R> DEV R block_sum(R v, ShT<R>& sh) {
  v = warp_sum_r(v);
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = v;
  __syncthreads();
  R t = 0;
#pragma unroll
  for (int w = 0; w < DT / 32; ++w) t += sh.red[w];
  __syncthreads();
  return t;
}

// 1/sqrt(a) for a > 0.  FP64: single-precision estimate, then two Newton steps
// y <- y (3 - a y^2) / 2 (quadratic convergence: ~1e-7 -> 1e-14 -> 1e-16); a
// normal-range float must hold a, otherwise the FP64 expression is used.
// FP32: the hardware estimate and one Newton step.
DEV double rsqrt_nr(double a) {
  if (!(a > 1e-36 && a < 1e36)) return 1.0 / sqrt(a);
  double y = (double)rsqrtf((float)a);
  y = y * (1.5 - 0.5 * a * y * y);
  y = y * (1.5 - 0.5 * a * y * y);
  return y;
}
DEV float rsqrt_nr(float a) {
  const float y = rsqrtf(a);
  return y * (1.5f - 0.5f * a * y * y);
}

// Givens rotation U = [[cs, sn], [-conj(sn), cs]] with U [x; y] = [r; 0]; rot = {cs, Re sn, Im sn}
template <typename R> DEV void givens(cx<R> x, cx<R> y, R* rot) {
  const R ax2 = norm2(x), ay2 = norm2(y);
  if (ay2 == R(0)) {
    rot[0] = 1; rot[1] = 0; rot[2] = 0;
  } else if (ax2 == R(0)) {
    const R inv = rsqrt_nr(ay2);
    rot[0] = 0; rot[1] = y.x * inv; rot[2] = -y.y * inv;
  } else {
    const R inv_r = rsqrt_nr(ax2 + ay2);
    const R inv_ax = rsqrt_nr(ax2);
    rot[0] = ax2 * inv_ax * inv_r;  // |x| / r
    // sn = (x / |x|) conj(y) / r
    const R f = inv_ax * inv_r;
    rot[1] = (x.x * y.x + x.y * y.y) * f;
    rot[2] = (x.y * y.x - x.x * y.y) * f;
  }
}

// Householder QR of the first `cols` columns of A (rows x ntot, column-major,
// lda), reflectors applied to all ntot columns.  R in the upper triangle, v
// below the diagonal, tau[j].  Column j of the factored part is known to be
// zero below row max(j+1, kfull) (the GMRES-DR recurrence matrix is upper
// Hessenberg except for a full leading block; kfull >= rows means dense), so
// reflector j spans rows j..last(j) only.
DEV int qr_last(int j, int rows, int kfull) { return min(rows - 1, max(j + 1, kfull)); }

template <typename R>
DEV void cta_qr(cx<R>* A, int lda, int rows, int cols, int ntot, cx<R>* tau, ShT<R>& sh, int kfull) {
  using C = cx<R>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = 0; j < cols && j < rows; ++j) {
    const int last = qr_last(j, rows, kfull);
    R s = 0;
    for (int i = j + 1 + threadIdx.x; i <= last; i += DT) s += norm2(A[i + (long)j * lda]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      const C alpha = A[j + (long)j * lda];
      if (s == R(0) && alpha.y == R(0)) {
        tau[j] = {0, 0};
      } else {
        const R beta = -copysign_(sqrt_(norm2(alpha) + s), alpha.x);
        tau[j] = {(beta - alpha.x) / beta, -alpha.y / beta};
        sh.bc[0] = cdiv(C{1, 0}, alpha - C{beta, 0});
        A[j + (long)j * lda] = {beta, 0};
      }
    }
    __syncthreads();
    const C tj = tau[j];
    if (tj.x == R(0) && tj.y == R(0)) continue;  // uniform across the CTA
    const C scal = sh.bc[0];
    for (int i = j + 1 + threadIdx.x; i <= last; i += DT) A[i + (long)j * lda] = A[i + (long)j * lda] * scal;
    __syncthreads();
    const C ct = conj(tj);
    if (last - j < 32) {
      // short reflector: one thread per column
      for (int cc = j + 1 + threadIdx.x; cc < ntot; cc += DT) {
        C* col = A + (long)cc * lda;
        C w = col[j];
        for (int i = j + 1; i <= last; ++i) w += cmulc(A[i + (long)j * lda], col[i]);
        const C f = ct * w;
        col[j] -= f;
        for (int i = j + 1; i <= last; ++i) col[i] -= A[i + (long)j * lda] * f;
      }
    } else {
      for (int cc = j + 1 + warp; cc < ntot; cc += DT / 32) {
        C* col = A + (long)cc * lda;
        C w = {0, 0};
        for (int i = j + lane; i <= last; i += 32) {
          const C vi = (i == j) ? C{1, 0} : A[i + (long)j * lda];
          w += cmulc(vi, col[i]);
        }
        w = warp_sum_c(w);
        const C f = ct * w;
        for (int i = j + lane; i <= last; i += 32) {
          const C vi = (i == j) ? C{1, 0} : A[i + (long)j * lda];
          col[i] -= vi * f;
        }
      }
    }
    __syncthreads();
  }
}

// Givens QR of the columns j0..cols-1 of an upper Hessenberg block (column j is
// zero below row j+1), applied to all ntot columns, by warp 0 alone: every lane
// forms the rotation of column j from its two entries, then rotates its own
// columns; no block barriers, one FP64 dependency chain per rotation.  R is left
// in the upper triangle (the eliminated entries hold rounding residue only).
DEV void warp_givens_qr(c128* A, int lda, int rows, int j0, int cols, int ntot) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  for (int j = j0; j < cols && j + 1 < rows; ++j) {
    double rot[3];
    givens(A[j + (long)j * lda], A[j + 1 + (long)j * lda], rot);
    const double cs = rot[0];
    const c128 sn = {rot[1], rot[2]};
    for (int cc = j + lane; cc < ntot; cc += 32) {
      const c128 a = A[j + (long)cc * lda], b = A[j + 1 + (long)cc * lda];
      A[j + (long)cc * lda] = cs * a + sn * b;
      A[j + 1 + (long)cc * lda] = cs * b - conj(sn) * a;
    }
    __syncwarp();
  }
}

// QR of the GMRES recurrence matrix: Householder reflectors for its dense leading
// block (columns < kfull - 1), Givens rotations for the Hessenberg columns after it.
DEV void hess_qr(c128* A, int lda, int rows, int cols, int ntot, c128* tau, Sh& sh, int kfull) {
  const int jd = max(0, min(cols, kfull - 1));
  cta_qr(A, lda, rows, jd, ntot, tau, sh, kfull);
  warp_givens_qr(A, lda, rows, jd, cols, ntot);
  __syncthreads();
}

// Solve R y = y in place (R: upper nsz x nsz of A): reciprocals of the diagonal by
// all threads, then warp 0 substitutes (warp barriers only).  False on a zero pivot.
DEV bool fast_backsolve(const c128* A, int lda, int nsz, c128* y, c128* rinv, Sh& sh) {
  if (threadIdx.x == 0) sh.ibc[0] = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < nsz; j += DT) {
    const c128 p = A[j + (long)j * lda];
    if (p.x == 0.0 && p.y == 0.0) {
      sh.ibc[0] = 1;
      rinv[j] = {0, 0};
    } else {
      rinv[j] = cdiv(c128{1, 0}, p);
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int j = nsz - 1; j >= 0; --j) {
      const c128 xj = y[j] * rinv[j];
      __syncwarp();
      if (threadIdx.x == 0) y[j] = xj;
      for (int i = threadIdx.x; i < j; i += 32) y[i] -= A[i + (long)j * lda] * xj;
      __syncwarp();
    }
  }
  __syncthreads();
  return sh.ibc[0] == 0;
}

// load (Hbar - sig Ibar)[0:rows, 0:cols] into A (lda), rounded to the precision of A
template <typename R>
DEV void load_shifted(cx<R>* A, int lda, const c128* H, int ldh, int rows, int cols, c128 sig) {
  for (int t = threadIdx.x; t < rows * cols; t += DT) {
    const int i = t % rows, j = t / rows;
    c128 v = H[i + (long)j * ldh];
    if (i == j) v -= sig;
    A[i + (long)j * lda] = cvt<R>(v);
  }
}

// odd leading dimension: row-wise accesses of 16-byte elements hit distinct banks
HD int odd_ld(int rows) { return rows | 1; }

DEV void set_err(ColState* st, int code) {
  if (threadIdx.x == 0) atomicCAS(&st->err, 0, code);
}

// Back substitution R x = b in place (R: upper n x n of A, FP32), by one warp; false on a
// zero pivot (that x_j := 0).
DEV bool warp_backsolve32(const c64* A, int la, int n, c64* b) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int j = n - 1; j >= 0; --j) {
    const c64 p = A[j + (long)j * la];
    c64 xj = {0, 0};
    if (p.x == 0.f && p.y == 0.f) ok = false;
    else xj = cdiv(b[j], p);
    __syncwarp();
    if (lane == 0) b[j] = xj;
    for (int i = lane; i < j; i += 32) b[i] -= A[i + (long)j * la] * xj;
    __syncwarp();
  }
  return ok;
}

// min || c - Hhat y || for a Hessenberg recurrence (zero below the subdiagonal) built on a
// complex64 basis, in FP32 with one step of refinement: warp 0 reduces [Hhat | c], rounded
// to FP32, to triangular form by Givens rotations (kept) and back-substitutes; the FP64
// residual r = c - Hhat y of the FP64 copy of y is rotated and solved the same way and the
// correction added.  The correction measures the FP32 solve's error; when the least-squares
// residual is large the step removes only part of it, so y is accurate to about the
// correction's size, while ||c - Hhat y|| stays within ~1e-9 (relative) of the minimum --
// what a GMRES cycle needs, since the caller forms s = c - Hhat y from this y in FP64 and
// the residual update stays consistent with the solution update.  When the correction
// exceeds 1e-4 ||y|| (kappa(Hhat) beyond ~1e5) or a pivot is zero, the result is not
// trusted and the function returns false, for the caller's FP64 solve.
// smem: the FP32 matrix and the rotations; r: rows FP64 entries of scratch; y: me FP64
// entries.
DEV bool ls32_solve(const c128* H, int ldh, const c128* cv, c128 sig, int rows, int me, unsigned char* smem,
                    c128* r, c128* y, Sh& sh) {
  const int lane = threadIdx.x & 31;
  const int la = odd_ld(rows);
  c64* A = reinterpret_cast<c64*>(smem);                          // rows x (me + 1)
  float* rot = reinterpret_cast<float*>(A + (long)la * (me + 1));  // 3 per column
  c64* b = A + (long)me * la;                                      // right-hand column
  load_shifted(A, la, H, ldh, rows, me, sig);
  for (int i = threadIdx.x; i < rows; i += DT) b[i] = cvt<float>(cv[i]);
  if (threadIdx.x == 0) sh.ibc[0] = 0;
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int j = 0; j < me && j + 1 < rows; ++j) {
      float g[3];
      givens(A[j + (long)j * la], A[j + 1 + (long)j * la], g);
      __syncwarp();  // every lane has read the pair before column j is rotated
      if (lane == 0) {
        rot[3 * j] = g[0];
        rot[3 * j + 1] = g[1];
        rot[3 * j + 2] = g[2];
      }
      const float cs = g[0];
      const c64 sn = {g[1], g[2]};
      for (int cc = j + lane; cc <= me; cc += 32) {
        const c64 a = A[j + (long)cc * la], bb = A[j + 1 + (long)cc * la];
        A[j + (long)cc * la] = cs * a + sn * bb;
        A[j + 1 + (long)cc * la] = cs * bb - conj(sn) * a;
      }
      __syncwarp();
    }
    if (!warp_backsolve32(A, la, me, b) && lane == 0) sh.ibc[0] = 1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < me; i += DT) y[i] = up(b[i]);
  __syncthreads();
  for (int i = threadIdx.x; i < rows; i += DT) {
    c128 v = cv[i];
    for (int j = max(0, i - 1); j < me; ++j) {  // row i of a Hessenberg matrix starts at column i-1
      c128 h = H[i + (long)j * ldh];
      if (i == j) h -= sig;
      v -= h * y[j];
    }
    r[i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int i = lane; i < rows; i += 32) b[i] = cvt<float>(r[i]);
    __syncwarp();
    if (lane == 0) {
      for (int j = 0; j < me && j + 1 < rows; ++j) {
        const float cs = rot[3 * j];
        const c64 sn = {rot[3 * j + 1], rot[3 * j + 2]};
        const c64 a = b[j], bb = b[j + 1];
        b[j] = cs * a + sn * bb;
        b[j + 1] = cs * bb - conj(sn) * a;
      }
    }
    __syncwarp();
    if (!warp_backsolve32(A, la, me, b) && lane == 0) sh.ibc[0] = 1;
    // size of the refinement step: ||correction||^2 <= 1e-8 ||y||^2
    double cn = 0, yn = 0;
    for (int i = lane; i < me; i += 32) {
      cn += (double)norm2(b[i]);
      yn += norm2(y[i]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      cn += __shfl_xor_sync(0xffffffffu, cn, off);
      yn += __shfl_xor_sync(0xffffffffu, yn, off);
    }
    if (lane == 0 && !(cn <= 1e-8 * yn)) sh.ibc[0] = 2;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < me; i += DT) y[i] += up(b[i]);
  __syncthreads();
  return sh.ibc[0] == 0;
}

// ------------------------------------------------- reduced solves (D1/D2)

// base least squares: d_1 into Cf column k+1 (+ s into Cf column k+1+ns if want_r)
DEV void base_ls(const DenseCycle& d, int c, c128* A, Sh& sh) {
  ColState* st = d.st + c;
  const int m = d.m, me = st->m_eff, k = d.k;
  const bool broke = st->broke;
  const c128* H = d.H + (long)c * (m + 1) * m;
  const c128* cv = d.cvec + (long)c * (m + 1);
  const c128 sig = d.sigma[(long)c * d.ns];
  // GMRES: least squares on the (m+1) x m recurrence; FOM (and a lucky breakdown): the
  // square m x m Galerkin system
  const int rows = (broke || d.fom) ? me : me + 1;
  const int lda = odd_ld(rows);
  c128* tau = A + (long)lda * (me + 1);
  c128* y = tau + (me + 1);
  c128* rinv = y + (me + 1);
  // complex64 basis, Hessenberg recurrence: FP32 least squares + refinement (tau as
  // scratch), the FP64 form below when that is not trusted
  const bool done32 = d.ls32 && d.kfull <= 1 && !d.fom &&
                      ls32_solve(H, m + 1, cv, sig, rows, me, reinterpret_cast<unsigned char*>(A), tau, y, sh);
  if (!done32) {
    load_shifted(A, lda, H, m + 1, rows, me, sig);
    for (int i = threadIdx.x; i < rows; i += DT) A[i + (long)me * lda] = cv[i];
    if (threadIdx.x == 0) sh.ibc[0] = 0;
    __syncthreads();
    hess_qr(A, lda, rows, me, me + 1, tau, sh, d.kfull);
    for (int i = threadIdx.x; i < me; i += DT) y[i] = A[i + (long)me * lda];
    __syncthreads();
    if (!fast_backsolve(A, lda, me, y, rinv, sh)) set_err(st, GDR_EBREAKDOWN);
  }
  // d_1 -> Cf, s = c - Hhat d_1 from the original Hbar
  c128* Cf = d.Cf + (long)c * d.ccs;
  const int xc = (k > 0 ? k + 1 : 0);
  for (int i = threadIdx.x; i <= m; i += DT) Cf[i + (long)xc * d.ldc] = (i < me) ? y[i] : c128{0, 0};
  c128* s = d.s + (long)c * (m + 1);
  double sn = 0;
  for (int i = threadIdx.x; i <= m; i += DT) {
    c128 v = {0, 0};
    if (!broke && i <= me) {
      v = cv[i];
      for (int j = 0; j < me; ++j) {
        c128 hij = H[i + (long)j * (m + 1)];
        if (i == j) hij -= sig;
        v -= hij * y[j];
      }
    }
    s[i] = v;
    sn += norm2(v);
    if (d.want_r) Cf[i + (long)(xc + d.ns) * d.ldc] = v;
  }
  sn = block_sum(sn, sh);
  if (threadIdx.x == 0) {
    d.norms[(long)c * d.ns] = sqrt(sn);
    st->rnorm = sqrt(sn);
    if (!isfinite(sn)) st->nan = 1;
  }
}

// shift i >= 1: [(Hbar - sigma_i Ibar) | c | s] -> QR, beta_new, d_i into Cf column k+1+i
DEV void shift_solve(const DenseCycle& d, int c, int i, c128* A, Sh& sh) {
  ColState* st = d.st + c;
  const int m = d.m, me = st->m_eff, k = d.k;
  const bool broke = st->broke;
  c128* Cf = d.Cf + (long)c * d.ccs;
  const int col = (k > 0 ? k + 1 : 0) + i;
  int* sact = d.sact + (long)c * d.ns;
  if (!sact[i]) {  // frozen shift: no update
    for (int r = threadIdx.x; r <= m; r += DT) Cf[r + (long)col * d.ldc] = {0, 0};
    return;
  }
  const c128* H = d.H + (long)c * (m + 1) * m;
  const c128* cv = d.cvec + (long)c * (m + 1);
  const c128* s = d.s + (long)c * (m + 1);
  const c128 sig = d.sigma[(long)c * d.ns + i];
  const c128 beta = d.beta[(long)c * d.ns + i];
  if (d.fom) {
    // FOM: (H_m - sigma_i I) d_i = beta_i c[0:m] (Galerkin); the residual
    // beta_i c - (Hbar - sigma_i Ibar) d_i is a multiple of e_{m+1}: beta_new relates
    // its last component to that of the base residual s
    const int lda = odd_ld(me);
    load_shifted(A, lda, H, m + 1, me, me, sig);
    for (int r = threadIdx.x; r < me; r += DT) A[r + (long)me * lda] = cv[r];
    c128* tau = A + (long)lda * (me + 1);
    c128* y = tau + (me + 1);
    c128* rinv = y + (me + 1);
    if (threadIdx.x == 0) sh.ibc[0] = 0;
    __syncthreads();
    hess_qr(A, lda, me, me, me + 1, tau, sh, d.kfull);
    for (int r = threadIdx.x; r < me; r += DT) y[r] = beta * A[r + (long)me * lda];
    __syncthreads();
    if (!fast_backsolve(A, lda, me, y, rinv, sh)) set_err(st, GDR_EBREAKDOWN);
    __syncthreads();
    for (int r = threadIdx.x; r <= m; r += DT) Cf[r + (long)col * d.ldc] = (r < me) ? y[r] : c128{0, 0};
    if (threadIdx.x == 0) {
      c128 bnew = {0, 0};
      if (!broke) {
        c128 t = beta * cv[me];
        for (int j = 0; j < me; ++j) t -= H[me + (long)j * (m + 1)] * y[j];
        const c128 sl = s[me];
        if (sl.x == 0.0 && sl.y == 0.0) set_err(st, GDR_EBREAKDOWN);
        else bnew = cdiv(t, sl);
      }
      d.beta[(long)c * d.ns + i] = bnew;
      d.norms[(long)c * d.ns + i] = cabs_(bnew) * st->rnorm;
    }
    return;
  }
  const int rows = broke ? me : me + 1;
  const int lda = odd_ld(rows);
  load_shifted(A, lda, H, m + 1, rows, me, sig);
  for (int r = threadIdx.x; r < rows; r += DT) {
    A[r + (long)me * lda] = cv[r];
    A[r + (long)(me + 1) * lda] = s[r];
  }
  c128* tau = A + (long)lda * (me + 2);
  c128* y = tau + (me + 1);
  c128* rinv = y + (me + 1);
  if (threadIdx.x == 0) sh.ibc[0] = 0;
  __syncthreads();
  hess_qr(A, lda, rows, me, me + 2, tau, sh, d.kfull);
  c128 bnew = {0, 0};
  if (!broke) {
    const c128 qc = A[me + (long)me * lda], qs = A[me + (long)(me + 1) * lda];
    if (qs.x == 0.0 && qs.y == 0.0) {
      set_err(st, GDR_EBREAKDOWN);
    } else {
      bnew = beta * cdiv(qc, qs);
    }
  }
  for (int r = threadIdx.x; r < me; r += DT)
    y[r] = beta * A[r + (long)me * lda] - bnew * A[r + (long)(me + 1) * lda];
  __syncthreads();
  if (!fast_backsolve(A, lda, me, y, rinv, sh)) set_err(st, GDR_EBREAKDOWN);
  for (int r = threadIdx.x; r <= m; r += DT) Cf[r + (long)col * d.ldc] = (r < me) ? y[r] : c128{0, 0};
  if (threadIdx.x == 0) {
    d.beta[(long)c * d.ns + i] = bnew;
    d.norms[(long)c * d.ns + i] = cabs_(bnew) * st->rnorm;
  }
}

// --------------------------------------------------- harmonic Ritz (D1)

// selection order of the "smallest" harmonic Ritz values, magnitudes precomputed:
// |theta| ascending; within a relative tie, larger Im, then larger Re
template <typename R> DEV bool before_m(cx<R> a, R ma, cx<R> b, R mb) {
  const R scale = fmax_(ma, mb);
  if (fabs_(ma - mb) > Lim<R>::tie * scale) return ma < mb;
  if (fabs_(a.y - b.y) > Lim<R>::tie * scale) return a.y > b.y;
  return a.x > b.x;
}

// v <- Hhat^{-H} v for Hhat = Q R as cta_qr leaves it (R in T, reflectors below it, tau),
// by one warp: forward substitution with R^H, right-looking (every lane forms z_j, the
// lanes update the entries below it), then v <- Q z with the reflectors in reverse order
// (warp-reduced dots).  A zero diagonal entry of R sets *zero_pivot (z_j := 0).
template <typename R>
DEV void solve_rh_warp(const cx<R>* T, int lda, int m, const cx<R>* tau, cx<R>* v, int kfull, int* zero_pivot) {
  using C = cx<R>;
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < m; ++j) {
    const C rjj = T[j + (long)j * lda];
    C z = {0, 0};
    if (rjj.x == R(0) && rjj.y == R(0)) {
      if (lane == 0) *zero_pivot = 1;
    } else {
      z = cdiv(v[j], conj(rjj));
    }
    __syncwarp();
    if (lane == 0) v[j] = z;
    for (int i = j + 1 + lane; i < m; i += 32) v[i] -= cmulc(T[j + (long)i * lda], z);
    __syncwarp();
  }
  for (int j = m - 1; j >= 0; --j) {
    const C tj = tau[j];
    if (tj.x == R(0) && tj.y == R(0)) continue;
    const int last = qr_last(j, m, kfull);
    C w = {0, 0};
    for (int i = j + 1 + lane; i <= last; i += 32) w += cmulc(T[i + (long)j * lda], v[i]);
    w = warp_sum_c(w);
    w += v[j];
    const C f = tj * w;
    __syncwarp();
    if (lane == 0) v[j] -= f;
    for (int i = j + 1 + lane; i <= last; i += 32) v[i] -= T[i + (long)j * lda] * f;
    __syncwarp();
  }
}

// Shared-memory layout of the FP32 harmonic Ritz path (byte offsets, 16-byte
// aligned): T (m x (m+2), odd ld), Z (m rows of odd stride), Y (eigenvectors of
// T, m x k, odd ld), then f in FP64, the FP64 refinement residual, tau, theta
// and the selection.
struct Hr32Layout {
  long T, Z, Y, fd, rr, tau, theta, sel, total;
};
HD long al16(long x) { return (x + 15) & ~15L; }
HD int odd_ld2(int rows) { return rows | 1; }
HD Hr32Layout hr32_layout(int m, int k) {
  const long ld = odd_ld2(m);
  Hr32Layout L{};
  long o = 0;
  L.T = o; o = al16(o + 8 * ld * (m + 2));
  L.Z = o; o = al16(o + 8 * ld * m);
  L.Y = o; o = al16(o + 8 * ld * k);
  L.fd = o; o = al16(o + 16L * m);
  L.rr = o; o = al16(o + 8L * m);
  L.tau = o; o = al16(o + 8L * m);
  L.theta = o; o = al16(o + 8L * m);
  L.sel = o; o = al16(o + 4L * k);
  L.total = o;
  return L;
}

// Harmonic Ritz step of the restart in precision R: f = Hhat^{-H} hrow^H, M = Hhat +
// f hrow, Hessenberg reduction of M with the reflectors accumulated into Z,
// complex single-shift QR to the Schur form T = Z^H M Z, eigenvectors of T for the
// k smallest |theta| by back substitution, G = Z Y orthonormalised into P_k
// ((m+1) x k, last row 0); all m values into theta.
//
// R = double: everything in FP64, Z and Y in the per-column global scratch; a
// failure sets the column's error and returns false.
// R = float (complex64 basis): T, Z, Y in shared memory (hr32_layout); f is
// refined to FP64 accuracy by two steps of iterative refinement (FP64
// residual, FP32 factors).  Returns false, touching no state, when FP32 is not
// enough (non-finite values, no convergence of the QR iteration, a selected
// eigenvector nearly dependent on the others); the caller then runs the FP64 form.
template <typename R>
DEV bool harmonic_ritz(const DenseCycle& d, int c, unsigned char* smem, ShT<R>& sh) {
  using C = cx<R>;
  constexpr bool F32 = sizeof(R) == 4;
  ColState* st = d.st + c;
  const int m = d.m, k = d.k;
  const c128* H = d.H + (long)c * (m + 1) * m;
  const c128 sig = d.sigma[(long)c * d.ns];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lda = odd_ld(m);
  C *T, *Z, *Y, *f, *tau, *theta;
  int* sel;
  c128* fd = nullptr;  // FP32 path: f in FP64
  int ldz, ldy;
  if constexpr (F32) {
    const Hr32Layout L = hr32_layout(m, k);
    T = reinterpret_cast<C*>(smem + L.T);
    Z = reinterpret_cast<C*>(smem + L.Z);
    Y = reinterpret_cast<C*>(smem + L.Y);
    fd = reinterpret_cast<c128*>(smem + L.fd);
    f = reinterpret_cast<C*>(smem + L.rr);
    tau = reinterpret_cast<C*>(smem + L.tau);
    theta = reinterpret_cast<C*>(smem + L.theta);
    sel = reinterpret_cast<int*>(smem + L.sel);
    ldz = lda;
    ldy = lda;
  } else {
    T = reinterpret_cast<C*>(smem);
    double* scr = d.scratch + (long)c * d.scratch_per_col;
    Z = reinterpret_cast<C*>(scr);                // m x m, row-major, row t owned by thread DT-1-t
    Y = Z + (long)m * m;                          // eigenvectors of T, ld = odd_ld(m)
    f = T + (long)lda * (m + 2);                  // m
    tau = f + m;                                  // m
    theta = tau + m;                              // m
    sel = reinterpret_cast<int*>(theta + m);      // k
    ldz = m;
    ldy = lda;
  }
  auto fail = [&]() {
    if constexpr (!F32) set_err(st, GDR_EBREAKDOWN);
    return false;
  };
  GDR_DENSE_MARK(0, 0);
  if (!d.fom) {  // regular Ritz values (FOM-DR restart): M = Hhat, no f
  // 1) f = Hhat^{-H} hrow^H with Hhat = (Hbar - sigma_1 Ibar)[0:m, 0:m] = Q R:
  //    R^H z = hrow^H, f = Q z (thread 0 solves; the factors stay in T)
  load_shifted(T, lda, H, m + 1, m, m, sig);
  if (threadIdx.x == 0) sh.ibc[0] = 0;
  __syncthreads();
  cta_qr(T, lda, m, m, m, tau, sh, d.kfull);
  GDR_DENSE_MARK(10, 0);
  auto solve_rh = [&](C* v) {  // v <- Hhat^{-H} v, warp 0
    if (warp == 0) solve_rh_warp(T, lda, m, tau, v, d.kfull, &sh.ibc[0]);
  };
  for (int i = threadIdx.x; i < m; i += DT) f[i] = cvt<R>(conj(H[m + (long)i * (m + 1)]));
  __syncthreads();
  solve_rh(f);
  __syncthreads();
  if (sh.ibc[0]) return fail();
  GDR_DENSE_MARK(11, 0);
  if constexpr (F32) {
    for (int i = threadIdx.x; i < m; i += DT) fd[i] = up(f[i]);
    for (int it = 0; it < 2; ++it) {
      __syncthreads();
      // residual hrow^H - Hhat^H f in FP64 (thread i: row i of Hhat^H = column i of Hhat)
      for (int i = threadIdx.x; i < m; i += DT) {
        const c128* hc = H + (long)i * (m + 1);
        c128 acc = conj(H[m + (long)i * (m + 1)]);
        for (int j = 0; j < m; ++j) {
          c128 h = hc[j];
          if (j == i) h -= sig;
          acc -= cmulc(h, fd[j]);
        }
        f[i] = cvt<R>(acc);
      }
      __syncthreads();
      solve_rh(f);
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += DT) fd[i] += up(f[i]);
    }
    __syncthreads();
  } else {
    fd = reinterpret_cast<c128*>(f);
  }
  }  // !d.fom
  GDR_DENSE_MARK(1, 0);
  // 2) M = Hhat + f hrow (formed in FP64; M = Hhat for regular Ritz values)
  for (int t = threadIdx.x; t < m * m; t += DT) {
    const int i = t % m, j = t / m;
    c128 v = H[i + (long)j * (m + 1)];
    if (i == j) v -= sig;
    if (!d.fom) v += fd[i] * H[m + (long)j * (m + 1)];
    T[i + (long)j * lda] = cvt<R>(v);
  }
  __syncthreads();
  GDR_DENSE_MARK(2, 0);
  const int zrow = DT - 1 - threadIdx.x;  // FP64 form: row of Z owned by this thread in the sweep
  if constexpr (F32) {
    // 3+4) Hessenberg reduction M = Z Hh Z^H with Z accumulated in the same pass.
    // Per column j: warp 0 forms the reflector (v into vh, tau), then one thread
    // per column applies it from the left, one thread per row from the right to M
    // and to Z (no warp reductions; three block barriers per column).
    C* vh = f;  // f is free once M is formed
    for (int r = warp; r < m; r += DT / 32) {
      C* zr = Z + (long)r * ldz;
      for (int i = lane; i < m; i += 32) zr[i] = {R(r == i ? 1 : 0), R(0)};
    }
    for (int j = 0; j + 2 < m; ++j) {
      if (warp == 0) {
        R s = 0;
        for (int i = j + 2 + lane; i < m; i += 32) s += norm2(T[i + (long)j * lda]);
        s = warp_sum_r(s);
        const C alpha = T[j + 1 + (long)j * lda];
        const bool triv = (s == R(0) && alpha.y == R(0));
        C tj = {0, 0}, scal = {0, 0};
        R beta = 0;
        if (!triv) {
          beta = -copysign_(sqrt_(norm2(alpha) + s), alpha.x);
          tj = {(beta - alpha.x) / beta, -alpha.y / beta};
          scal = cdiv(C{1, 0}, alpha - C{beta, 0});
        }
        for (int i = j + 2 + lane; i < m; i += 32) {
          vh[i] = triv ? C{0, 0} : T[i + (long)j * lda] * scal;
          T[i + (long)j * lda] = {0, 0};
        }
        if (lane == 0) {
          vh[j + 1] = {1, 0};
          tau[j] = tj;
          if (!triv) T[j + 1 + (long)j * lda] = {beta, 0};
        }
      }
      __syncthreads();
      const C tj = tau[j];
      if (tj.x == R(0) && tj.y == R(0)) continue;  // uniform across the CTA
      // left: rows j+1.., columns j+1..m-1 : (I - conj(tau) v v^H)
      const C ct = conj(tj);
      for (int cc = j + 1 + threadIdx.x; cc < m; cc += DT) {
        C* colp = T + (long)cc * lda;
        C w = {0, 0};
        for (int i = j + 1; i < m; ++i) w += cmulc(vh[i], colp[i]);
        const C fct = ct * w;
        for (int i = j + 1; i < m; ++i) colp[i] -= vh[i] * fct;
      }
      __syncthreads();
      // right: all rows of M and of Z : X (I - tau v v^H)
      for (int r = threadIdx.x; r < 2 * m; r += DT) {
        C w = {0, 0};
        if (r < m) {
          for (int i = j + 1; i < m; ++i) w += T[r + (long)i * lda] * vh[i];
          const C fct = tj * w;
          for (int i = j + 1; i < m; ++i) T[r + (long)i * lda] -= fct * conj(vh[i]);
        } else {
          C* zr = Z + (long)(r - m) * ldz;
          for (int i = j + 1; i < m; ++i) w += zr[i] * vh[i];
          const C fct = tj * w;
          for (int i = j + 1; i < m; ++i) zr[i] -= fct * conj(vh[i]);
        }
      }
      __syncthreads();
    }
    GDR_DENSE_MARK(3, 0);
    GDR_DENSE_MARK(4, 0);
  } else {
    // 3) Hessenberg reduction M = Q Hh Q^H, reflectors kept below the subdiagonal
    for (int j = 0; j + 2 < m; ++j) {
      R s = 0;
      for (int i = j + 2 + threadIdx.x; i < m; i += DT) s += norm2(T[i + (long)j * lda]);
      s = block_sum(s, sh);
      if (threadIdx.x == 0) {
        const C alpha = T[j + 1 + (long)j * lda];
        if (s == R(0) && alpha.y == R(0)) {
          tau[j] = {0, 0};
        } else {
          const R beta = -copysign_(sqrt_(norm2(alpha) + s), alpha.x);
          tau[j] = {(beta - alpha.x) / beta, -alpha.y / beta};
          sh.bc[0] = cdiv(C{1, 0}, alpha - C{beta, 0});
          T[j + 1 + (long)j * lda] = {beta, 0};
        }
      }
      __syncthreads();
      const C tj = tau[j];
      if (tj.x == R(0) && tj.y == R(0)) continue;
      const C scal = sh.bc[0];
      for (int i = j + 2 + threadIdx.x; i < m; i += DT) T[i + (long)j * lda] = T[i + (long)j * lda] * scal;
      __syncthreads();
      // left: rows j+1.., columns j+1..m-1 : (I - conj(tau) v v^H)
      const C ct = conj(tj);
      for (int cc = j + 1 + warp; cc < m; cc += DT / 32) {
        C* colp = T + (long)cc * lda;
        C w = {0, 0};
        for (int i = j + 1 + lane; i < m; i += 32) {
          const C vi = (i == j + 1) ? C{1, 0} : T[i + (long)j * lda];
          w += cmulc(vi, colp[i]);
        }
        w = warp_sum_c(w);
        const C fct = ct * w;
        for (int i = j + 1 + lane; i < m; i += 32) {
          const C vi = (i == j + 1) ? C{1, 0} : T[i + (long)j * lda];
          colp[i] -= vi * fct;
        }
      }
      __syncthreads();
      // right: all rows, columns j+1..m-1 : M (I - tau v v^H)
      for (int r = warp; r < m; r += DT / 32) {
        C w = {0, 0};
        for (int i = j + 1 + lane; i < m; i += 32) {
          const C vi = (i == j + 1) ? C{1, 0} : T[i + (long)j * lda];
          w += T[r + (long)i * lda] * vi;
        }
        w = warp_sum_c(w);
        const C fct = tj * w;
        for (int i = j + 1 + lane; i < m; i += 32) {
          const C vi = (i == j + 1) ? C{1, 0} : T[i + (long)j * lda];
          T[r + (long)i * lda] -= fct * conj(vi);
        }
      }
      __syncthreads();
    }
    GDR_DENSE_MARK(3, 0);
    // 4) Z = Q = H_0 H_1 ... : Z <- Z H_j for j = 0.., one warp per row of Z
    //    (I - tau v v^H applied from the right), then clear below the subdiagonal.
    //    During the QR sweep row t of Z belongs to thread DT-1-t.
    for (int r = warp; r < m; r += DT / 32) {
      C* zr = Z + (long)r * ldz;
      for (int i = lane; i < m; i += 32) zr[i] = {R(r == i ? 1 : 0), R(0)};
    }
    __syncthreads();
    for (int j = 0; j + 2 < m; ++j) {
      const C tj = tau[j];
      if (tj.x == R(0) && tj.y == R(0)) continue;
      for (int r = warp; r < m; r += DT / 32) {
        C* zr = Z + (long)r * ldz;
        C w = {0, 0};
        for (int i = j + 1 + lane; i < m; i += 32) {
          const C vi = (i == j + 1) ? C{1, 0} : T[i + (long)j * lda];
          w += zr[i] * vi;
        }
        w = warp_sum_c(w);
        const C fct = tj * w;
        for (int i = j + 1 + lane; i < m; i += 32) {
          const C vi = (i == j + 1) ? C{1, 0} : T[i + (long)j * lda];
          zr[i] -= fct * conj(vi);
        }
      }
      __syncwarp();
    }
    __syncthreads();
    for (int q = threadIdx.x; q < m * m; q += DT) {
      const int i = q % m, j = q / m;
      if (i > j + 1) T[i + (long)j * lda] = {0, 0};
    }
    __syncthreads();
    GDR_DENSE_MARK(4, 0);
  }
  // 5) complex single-shift QR to Schur form T = Z^H M Z
  R hnorm = 0;
  for (int q = threadIdx.x; q < m * m; q += DT) hnorm = fmax_(hnorm, cabs_(T[(q % m) + (long)(q / m) * lda]));
  {
    // max over the CTA (NaN propagates as a failure below)
    R v = hnorm;
#pragma unroll
    for (int mm = 16; mm > 0; mm >>= 1) v = fmax_(v, __shfl_xor_sync(FULL, v, mm));
    if (lane == 0) sh.red[warp] = v;
    __syncthreads();
    hnorm = fmax_(fmax_(sh.red[0], sh.red[1]), fmax_(sh.red[2], sh.red[3]));
    __syncthreads();
  }
  if constexpr (F32) {
    if (!(hnorm < 1e30f)) return false;  // overflowed or non-finite in FP32
  }
  const R smallnum = fmax_(hnorm * Lim<R>::eps, Lim<R>::tiny);
  const R eps2 = Lim<R>::eps * Lim<R>::eps;
  R* rot = reinterpret_cast<R*>(&sh.bc[1]);  // rot[0] = cs, (rot[1], rot[2]) = sn
  int hi = m - 1, its = 0, total = 0;
  bool failed = false;
  while (hi >= 0) {
    if (warp == 0) {
      // deflation: the largest l in (0, hi] with |h_{l,l-1}|^2 <= eps^2 (|h_{l-1,l-1}|^2 + |h_{l,l}|^2),
      // tested 32 subdiagonals at a time from the bottom (uniform result in the warp)
      int l = 0;
      for (int top = hi; top > 0; top -= 32) {
        const int cand = top - lane;
        bool neg = false;
        if (cand > 0) {
          const R sub = norm2(T[cand + (long)(cand - 1) * lda]);
          R ref = norm2(T[cand - 1 + (long)(cand - 1) * lda]) + norm2(T[cand + (long)cand * lda]);
          if (ref == R(0)) ref = hnorm * hnorm;
          neg = (sub <= eps2 * ref || sub <= smallnum * smallnum * R(1e-6));
        }
        const unsigned bal = __ballot_sync(FULL, neg);
        if (bal) {
          l = top - (__ffs(bal) - 1);  // lowest lane = largest candidate
          break;
        }
      }
      if (lane == 0) {
        if (l > 0) T[l + (long)(l - 1) * lda] = {0, 0};
        sh.ibc[1] = l;
        if (l < hi) {
          // Wilkinson shift of the trailing 2x2 block (exceptional shift every 10th sweep),
          // then the first rotation of the sweep
          ++its;
          C mu;
          const C a = T[hi - 1 + (long)(hi - 1) * lda], b = T[hi - 1 + (long)hi * lda];
          const C cc = T[hi + (long)(hi - 1) * lda], dd = T[hi + (long)hi * lda];
          if (its % 10 == 0) {
            mu = dd + C{fabs_(cc.x) + fabs_(cc.y), 0};
          } else {
            const C half = R(0.5) * (a - dd);
            const C disc = csqrt_(half * half + b * cc);
            const C l1 = dd + half + disc, l2 = dd + half - disc;
            mu = (norm2(l1 - dd) <= norm2(l2 - dd)) ? l1 : l2;
          }
          givens(T[l + (long)l * lda] - mu, T[l + 1 + (long)l * lda], rot);
        } else {
          its = 0;
        }
      }
    }
    __syncthreads();
    const int lo = sh.ibc[1];
    if (lo == hi) {
      --hi;
      continue;
    }
    ++total;
    if (total > 40 * m) {
      failed = true;
      break;
    }
    for (int kk = lo; kk < hi; ++kk) {
      const R cs = rot[0];
      const C sn = {rot[1], rot[2]};
      // left: rows kk, kk+1, columns max(kk-1,0)..m-1
      for (int cc = max(kk - 1, 0) + threadIdx.x; cc < m; cc += DT) {
        const C a = T[kk + (long)cc * lda], b = T[kk + 1 + (long)cc * lda];
        const C b_new = (cc == kk - 1 && kk > lo) ? C{0, 0} : cs * b - conj(sn) * a;
        T[kk + (long)cc * lda] = cs * a + sn * b;
        T[kk + 1 + (long)cc * lda] = b_new;
        if ((cc == kk || cc == kk + 1) && kk + 2 <= hi) {  // inputs of the next rotation
          sh.nx[cc - kk] = b_new;
          sh.nx[2 + cc - kk] = T[kk + 2 + (long)cc * lda];
        }
      }
      __syncthreads();
      // right: columns kk, kk+1, rows 0..min(kk+2, hi).  The owner, a thread with
      // no row of Z, forms the next rotation from the entries of rows kk+1, kk+2
      // saved by the left update.
      const int rlast = min(kk + 2, hi);
      C x_next = {0, 0}, y_next = {0, 0};
      const bool own = (threadIdx.x == DT - 1 - m) && (kk + 2 <= hi);
      if (own) {
        x_next = cs * sh.nx[0] + sh.nx[1] * conj(sn);
        y_next = cs * sh.nx[2] + sh.nx[3] * conj(sn);
      }
      for (int r = threadIdx.x; r <= rlast; r += DT) {
        const C a = T[r + (long)kk * lda], b = T[r + (long)(kk + 1) * lda];
        T[r + (long)kk * lda] = cs * a + b * conj(sn);
        T[r + (long)(kk + 1) * lda] = cs * b - a * sn;
      }
      if (own) givens(x_next, y_next, rot);
      if (zrow >= 0 && zrow < m) {
        C* zr = Z + (long)zrow * ldz;
        const C a = zr[kk], b = zr[kk + 1];
        zr[kk] = cs * a + b * conj(sn);
        zr[kk + 1] = cs * b - a * sn;
      }
      __syncthreads();
    }
  }
  if (failed) return fail();
  __syncthreads();
  GDR_DENSE_MARK(5, 0);
  // 6) eigenvalues and selection of the k smallest
  c128* th = d.theta + (long)c * m;
  for (int i = threadIdx.x; i < m; i += DT) {
    theta[i] = T[i + (long)i * lda];
    th[i] = up(theta[i]);
  }
  __syncthreads();
  // k rounds of a warp argmin under `before_m` (ties: lower index), which picks what
  // the index-order selection sort picks for a consistent order; |theta| computed once
  if (warp == 0) {
    R mag[3];
    unsigned used = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int i = lane + 32 * q;
      mag[q] = (i < m) ? sqrt_(norm2(theta[i])) : R(0);
    }
    for (int q = 0; q < k; ++q) {
      int bi = -1;
      R bm = 0;
      C bt = {0, 0};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int i = lane + 32 * r;
        if (i >= m || (used >> r & 1u)) continue;
        if (bi < 0 || before_m(theta[i], mag[r], bt, bm)) { bi = i; bm = mag[r]; bt = theta[i]; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const int oi = __shfl_xor_sync(FULL, bi, off);
        const R om = __shfl_xor_sync(FULL, bm, off);
        const C ot = shfl_xor_c(bt, off);
        bool take = false;
        if (oi >= 0) {
          if (bi < 0) take = true;
          else if (before_m(ot, om, bt, bm)) take = true;
          else if (!before_m(bt, bm, ot, om) && oi < bi) take = true;
        }
        if (take) { bi = oi; bm = om; bt = ot; }
      }
      if (lane == 0) sel[q] = bi;
      if ((bi & 31) == lane) used |= 1u << (bi >> 5);
    }
  }
  __syncthreads();
  GDR_DENSE_MARK(6, 0);
  // 7) eigenvectors of T (back substitution, one thread per selected value), Y = m x k
  for (int q = threadIdx.x; q < k; q += DT) {
    const int p = sel[q];
    const C lam = theta[p];
    C* y = Y + (long)q * ldy;
    for (int i = p + 1; i < m; ++i) y[i] = {0, 0};
    y[p] = {1, 0};
    for (int i = p - 1; i >= 0; --i) {
      C sacc = {0, 0};
      for (int j = i + 1; j <= p; ++j) sacc += T[i + (long)j * lda] * y[j];
      C den = T[i + (long)i * lda] - lam;
      if (cabs_(den) < smallnum) den = {smallnum, 0};
      y[i] = -cdiv(sacc, den);
    }
    // normalise (avoid overflow in later products)
    R nn = 0;
    for (int i = 0; i <= p; ++i) nn = fmax_(nn, cabs_(y[i]));
    for (int i = 0; i <= p; ++i) y[i] = (R(1) / nn) * y[i];
  }
  __syncthreads();
  GDR_DENSE_MARK(7, 0);
  // 8) G = Z Y into T (ld m+1, last row 0): thread t computes row t of G
  const int ldp = m + 1;
  const int t = threadIdx.x;
  if (t < m) {
    const C* zr = Z + (long)t * ldz;
    for (int q = 0; q < k; ++q) {
      const C* y = Y + (long)q * ldy;
      const int p = sel[q];
      C acc = {0, 0};
      for (int j = 0; j <= p; ++j) acc += zr[j] * y[j];
      T[t + (long)q * ldp] = acc;
    }
  } else if (t == m) {
    for (int q = 0; q < k; ++q) T[m + (long)q * ldp] = {0, 0};
  }
  __syncthreads();
  GDR_DENSE_MARK(8, 0);
  if (d.graw) {  // the raw eigenvectors G and their values (selection order), no P_k
    c128* gout = d.graw + (long)c * ldp * k;
    for (int q = threadIdx.x; q < ldp * k; q += DT) gout[q] = up(T[q]);
    for (int q = threadIdx.x; q < k; q += DT) d.gtheta[(long)c * k + q] = up(theta[sel[q]]);
    __syncthreads();
    return true;
  }
  // 9) P_k = orth([G; 0]) by classical Gram-Schmidt twice, in T (ld m+1)
  C* coef = theta;  // reuse (size >= k)
  for (int q = 0; q < k; ++q) {
    C* pq = T + (long)q * ldp;
    R n0 = 0;
    if constexpr (F32) {
      for (int i = threadIdx.x; i < m; i += DT) n0 += norm2(pq[i]);
      n0 = block_sum(n0, sh);
    }
    for (int pass = 0; pass < 2; ++pass) {
      for (int l = warp; l < q; l += DT / 32) {
        const C* pl = T + (long)l * ldp;
        C w = {0, 0};
        for (int i = lane; i < m; i += 32) w += cmulc(pl[i], pq[i]);
        w = warp_sum_c(w);
        if (lane == 0) coef[l] = w;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += DT) {
        C v = pq[i];
        for (int l = 0; l < q; ++l) v -= T[i + (long)l * ldp] * coef[l];
        pq[i] = v;
      }
      __syncthreads();
    }
    R nn = 0;
    for (int i = threadIdx.x; i < m; i += DT) nn += norm2(pq[i]);
    nn = block_sum(nn, sh);
    if constexpr (F32) {
      // nearly dependent on the vectors before it: FP32 orthogonalisation would lose it
      if (!(nn > R(1e-6) * n0) || !(nn < 1e30f)) return false;
    } else {
      if (!(nn > 0) || !isfinite(nn)) set_err(st, GDR_EBREAKDOWN);
    }
    const R inv = R(1) / sqrt_(nn);
    for (int i = threadIdx.x; i < m; i += DT) pq[i] = inv * pq[i];
    __syncthreads();
  }
  c128* Pk = d.Pk + (long)c * ldp * k;
  for (int q = threadIdx.x; q < ldp * k; q += DT) Pk[q] = up(T[q]);
  GDR_DENSE_MARK(9, total);
  return true;
}

// restart completion (D2): p_{k+1} from s, P into Cf, Hbar_k, c_k.  The products are split
// over nslice CTAs by columns of P_k (slice s: columns [k s / nslice, k (s+1) / nslice) of
// T1 = Hbar P_k, Hbar_k and Cf); every slice forms p_{k+1} itself (it enters row k of
// Hbar_k), slice 0 also writes c_k and p_{k+1} into Cf.
DEV void restart_finish(const DenseCycle& d, int c, c128* A, Sh& sh, int slice = 0, int nslice = 1) {
  const int m = d.m, k = d.k, ldp = m + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ColState* st = d.st + c;
  const c128* Pk = d.Pk + (long)c * ldp * k;
  const c128* H = d.H + (long)c * (m + 1) * m;
  const c128* s = d.s + (long)c * (m + 1);
  c128* P = A;                        // (m+1) x (k+1)
  c128* T1 = P + (long)ldp * (k + 1);  // (m+1) x k  = Hbar P_k[0:m]
  c128* coef = T1 + (long)ldp * k;     // k+1
  for (int q = threadIdx.x; q < ldp * k; q += DT) P[q] = Pk[q];
  c128* p = P + (long)ldp * k;
  for (int i = threadIdx.x; i < ldp; i += DT) p[i] = s[i];
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int l = warp; l < k; l += DT / 32) {
      const c128* pl = P + (long)l * ldp;
      c128 w = {0, 0};
      for (int i = lane; i < ldp; i += 32) w += cmulc(pl[i], p[i]);
      w = warp_sum_c(w);
      if (lane == 0) coef[l] = w;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ldp; i += DT) {
      c128 v = p[i];
      for (int l = 0; l < k; ++l) v -= P[i + (long)l * ldp] * coef[l];
      p[i] = v;
    }
    __syncthreads();
  }
  double nn = 0;
  for (int i = threadIdx.x; i < ldp; i += DT) nn += norm2(p[i]);
  nn = block_sum(nn, sh);
  if (!(nn > 0) || !isfinite(nn)) set_err(st, GDR_EBREAKDOWN);
  const double inv = 1.0 / sqrt(nn);
  for (int i = threadIdx.x; i < ldp; i += DT) p[i] = inv * p[i];
  __syncthreads();
  const int j0 = (int)((long)k * slice / nslice), nj = (int)((long)k * (slice + 1) / nslice) - j0;
  // T1[:, 0:nj] = Hbar (m+1 x m) * P_k[0:m, j0:j0+nj]
  for (int q = threadIdx.x; q < ldp * nj; q += DT) {
    const int i = q % ldp, j = j0 + q / ldp;
    c128 acc = {0, 0};
    for (int l = 0; l < m; ++l) acc += H[i + (long)l * (m + 1)] * P[l + (long)j * ldp];
    T1[q] = acc;
  }
  __syncthreads();
  // Hbar_k[:, j0:j0+nj] = P^H T1  ((k+1) rows), c_k = P^H s
  c128* Hk = d.Hk + (long)c * (k + 1) * k;
  for (int q = threadIdx.x; q < (k + 1) * nj; q += DT) {
    const int i = q % (k + 1), jj = q / (k + 1);
    c128 acc = {0, 0};
    for (int l = 0; l < ldp; ++l) acc += cmulc(P[l + (long)i * ldp], T1[l + (long)jj * ldp]);
    Hk[i + (long)(j0 + jj) * (k + 1)] = acc;
  }
  // P into the coefficient matrix (restart part of `combine`)
  c128* Cf = d.Cf + (long)c * d.ccs;
  for (int q = threadIdx.x; q < ldp * nj; q += DT) {
    const int i = q % ldp, j = j0 + q / ldp;
    Cf[i + (long)j * d.ldc] = P[i + (long)j * ldp];
  }
  if (slice != 0) return;
  c128* ck = d.ck + (long)c * (k + 1);
  for (int i = threadIdx.x; i <= k; i += DT) {
    c128 acc = {0, 0};
    for (int l = 0; l < ldp; ++l) acc += cmulc(P[l + (long)i * ldp], s[l]);
    ck[i] = acc;
  }
  for (int i = threadIdx.x; i < ldp; i += DT) Cf[i + (long)k * d.ldc] = p[i];
}

__global__ void __launch_bounds__(DT) dense_d1_kernel(DenseCycle d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Sh sh;
  c128* A = reinterpret_cast<c128*>(smem_raw);
  const int c = blockIdx.y;
  ColState* st = d.st + c;
  if (!st->active) return;
  if (blockIdx.x == 0) {
    base_ls(d, c, A, sh);
  } else {
    if (st->broke || st->m_eff < d.m || d.k == 0) return;
    if (d.hr32) {
      __shared__ ShT<float> shf;
      if (harmonic_ritz<float>(d, c, smem_raw, shf)) return;
    }
    harmonic_ritz<double>(d, c, smem_raw, sh);
  }
}

__global__ void __launch_bounds__(DT) dense_d2_kernel(DenseCycle d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Sh sh;
  c128* A = reinterpret_cast<c128*>(smem_raw);
  const int c = blockIdx.y;
  ColState* st = d.st + c;
  if (!st->active) return;
  // blocks 1..ns-1: shift solves; block 0 and blocks ns.. : slices of the restart products
  if (blockIdx.x == 0 || (int)blockIdx.x >= d.ns) {
    const int slice = blockIdx.x == 0 ? 0 : (int)blockIdx.x - d.ns + 1;
    if (d.k > 0 && !st->broke && st->m_eff == d.m && st->err == 0) restart_finish(d, c, A, sh, slice, d.rslices);
  } else {
    shift_solve(d, c, blockIdx.x, A, sh);
  }
}

// restart products alone (harmonic Ritz, then P_{k+1}, Hbar_k, c_k), for a given s
__global__ void __launch_bounds__(DT) restart_only_kernel(DenseCycle d, int phase) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Sh sh;
  c128* A = reinterpret_cast<c128*>(smem_raw);
  const int c = blockIdx.y;
  if (phase == 0) {
    if (d.hr32) {
      __shared__ ShT<float> shf;
      if (harmonic_ritz<float>(d, c, smem_raw, shf)) return;
    }
    harmonic_ritz<double>(d, c, smem_raw, sh);
  } else if (d.st[c].err == 0)
    restart_finish(d, c, A, sh);
}

__global__ void cycle_finish_kernel(DenseCycle d, c128* Hn, c128* cn) {
  const int c = blockIdx.x;
  ColState* st = d.st + c;
  if (!st->active) return;
  const int m = d.m, k = d.k, ns = d.ns;
  __shared__ int allconv;
  if (threadIdx.x == 0) {
    const double thr = st->tol * st->bnorm;
    int* sact = d.sact + (long)c * ns;
    const double* nr = d.norms + (long)c * ns;
    int ac = 1;
    for (int i = 0; i < ns; ++i) {
      const bool ci = st->broke || nr[i] <= thr;
      if (i > 0 && sact[i] && ci) sact[i] = 0;  // freeze
      if (!ci) ac = 0;
      if (!isfinite(nr[i])) st->nan = 1;
    }
    if (st->broke) ac = 1;
    st->conv = ac;
    allconv = ac;
  }
  __syncthreads();
  // next cycle's recurrence: Hbar = [Hbar_k 0; 0 0], c = [c_k; 0]
  if (k > 0 && !allconv && !st->broke && st->err == 0) {
    c128* H = Hn + (long)c * (m + 1) * m;
    const c128* Hk = d.Hk + (long)c * (k + 1) * k;
    for (long q = threadIdx.x; q < (long)(m + 1) * m; q += blockDim.x) {
      const int i = (int)(q % (m + 1)), j = (int)(q / (m + 1));
      H[q] = (i <= k && j < k) ? Hk[i + (long)j * (k + 1)] : c128{0, 0};
    }
    c128* cv = cn + (long)c * (m + 1);
    for (int i = threadIdx.x; i <= m; i += blockDim.x) cv[i] = (i <= k) ? d.ck[(long)c * (k + 1) + i] : c128{0, 0};
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->run = 0;
    if (allconv || st->err || st->nan) st->active = 0;
  }
}

// ------------------------------------------------------------ projection

// The projection's solution operators depend only on Hbar_k and the shifts, which stay
// fixed for every cycle of a batch: they are formed once (one setup launch) and each
// cycle applies them to c = V_{k+1}^H r with short dot products.  Per column c, (ns + 1)
// blocks of (k+1) x (k+1), column-major with leading dimension k+1, at ops + c (ns+1)(k+1)^2:
//   block 0  : P_1 = (Hbar_k - sigma_1 Ibar)^+ (least-squares solution operator) in rows
//              0..k-1, row k zero
//   block ns : T_1 = (Hbar_k - sigma_1 Ibar) P_1
//   block i  : S_i = (H_k - sigma_i I)^{-1} T_1[0:k, :] in rows 0..k-1 and, in row k,
//              g_i = T_1[k, :] - h_{k+1} S_i (h_{k+1}: the last row of Hbar_k)
// so that d_1 = P_1 c, (Hbar_k - sigma_1 Ibar) d_1 = T_1 c, d_i = beta_i S_i c solves
// (H_k - sigma_i I) d_i = beta_i (H_k - sigma_1 I) d_1 and the v_{k+1} component of the
// shifted residual grows by beta_i g_i c (the last row of Ibar is zero).

struct ProjArgs {
  int k, ns;
  const c128* Hk; const c128* cproj; const c128* sigma; const c128* beta; const int* sact;
  c128* gamma; c128* Cf; long ccs; ColState* st;
  long hkcs; int hpp;  // column c uses Hk + (c / hpp) * hkcs
};

// Gauss-Jordan elimination with partial pivoting on the k x w matrix W (column-major,
// leading dimension k) whose first k columns hold a square system: on return columns
// k..w-1 hold the system's inverse times the block they held.  Warp 0 finds the pivot
// (largest |W[i, j]|, i >= j, the smaller row index on a tie); all threads swap and scale the
// pivot row, then eliminate column j from the other rows in the columns after j.
// False (uniform over the CTA) on a zero pivot.
constexpr int GT = 256;  // threads of the Gauss-Jordan projection setup
DEV bool cta_gauss_jordan(c128* W, int k, int w, int* piv_s, c128* inv_s) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = j;
      for (int i = j + lane; i < k; i += 32) {
        const double v = norm2(W[i + (long)j * k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_xor_sync(FULL, best, off);
        const int oi = __shfl_xor_sync(FULL, bi, off);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        *piv_s = (best > 0.0 && isfinite(best)) ? bi : -1;
        if (best > 0.0) *inv_s = cdiv(c128{1, 0}, W[bi + (long)j * k]);
      }
    }
    __syncthreads();
    const int p = *piv_s;
    if (p < 0) return false;
    const c128 inv = *inv_s;
    for (int cc = j + threadIdx.x; cc < w; cc += GT) {
      const c128 top = W[j + (long)cc * k], pr = W[p + (long)cc * k];
      if (p != j) W[p + (long)cc * k] = top;
      W[j + (long)cc * k] = pr * inv;
    }
    __syncthreads();
    const int nc = w - j - 1;
    for (int t = threadIdx.x; t < k * nc; t += GT) {
      const int i = t % k, cc = j + 1 + t / k;
      if (i != j) W[i + (long)cc * k] -= W[i + (long)j * k] * W[j + (long)cc * k];
    }
    __syncthreads();
  }
  return true;
}

HD size_t proj_gj_smem(int k) { return sizeof(c128) * ((size_t)k * (2 * k + 1) + (size_t)(k + 1)); }

// The projection operators by Gauss-Jordan (one CTA per column and shift, GT threads):
// P_1 from the normal equations (Hbar_k - sigma_1 Ibar)^H (Hbar_k - sigma_1 Ibar) P_1 =
// (Hbar_k - sigma_1 Ibar)^H and one Newton-Schulz step, T_1 = (Hbar_k - sigma_1 Ibar) P_1
// formed from that P_1 (so T_1 c is the image of P_1 c to FP64 rounding whatever P_1's
// accuracy: the residual update stays consistent with the solution update), then for shift
// i >= 1 S_i from [H_k - sigma_i I | T_1[0:k, :]] and g_i.  CTA 0 writes blocks 0 and ns;
// CTA i forms its own T_1 in block i and overwrites it with [S_i; g_i].
__global__ void __launch_bounds__(GT) proj_gj_setup_kernel(ProjArgs a, c128* ops) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int piv_s;
  __shared__ c128 inv_s;
  const int c = blockIdx.y, i = blockIdx.x;
  ColState* st = a.st + c;
  if (!st->active) return;
  const int k = a.k, ld = k + 1, w = 2 * k + 1;
  const long bs = (long)ld * ld;
  const c128* Hk = a.Hk + (long)(c / a.hpp) * a.hkcs;
  const c128 s1 = a.sigma[(long)c * a.ns];
  c128* W = reinterpret_cast<c128*>(smem_raw);  // k x w
  c128* trow = W + (long)k * w;                 // row k of T_1
  c128* ob = ops + (long)c * (a.ns + 1) * bs;
  auto A1 = [&](int r, int l) {
    c128 h = Hk[r + (long)l * (k + 1)];
    if (r == l) h -= s1;
    return h;
  };
  for (int t = threadIdx.x; t < k * w; t += GT) {
    const int p = t % k, q = t / k;
    if (q < k) {
      c128 v0 = {0, 0}, v1 = {0, 0};
      int r = 0;
      for (; r + 1 <= k; r += 2) {
        v0 += cmulc(A1(r, p), A1(r, q));
        v1 += cmulc(A1(r + 1, p), A1(r + 1, q));
      }
      if (r <= k) v0 += cmulc(A1(r, p), A1(r, q));
      W[t] = v0 + v1;
    } else {
      W[t] = conj(A1(q - k, p));
    }
  }
  __syncthreads();
  bool ok = cta_gauss_jordan(W, k, w, &piv_s, &inv_s);
  c128* P = W + (long)k * k;  // P_1, k x (k+1), leading dimension k
  c128* Tb = ob + (long)(i == 0 ? a.ns : i) * bs;
  auto form_t1 = [&]() {  // Tb = (Hbar_k - sigma_1 Ibar) P_1
    for (int t = threadIdx.x; t < ld * ld; t += GT) {
      const int r = t % ld, j = t / ld;
      c128 v0 = {0, 0}, v1 = {0, 0};
      int l = 0;
      for (; l + 1 < k; l += 2) {
        v0 += A1(r, l) * P[l + (long)j * k];
        v1 += A1(r, l + 1) * P[l + 1 + (long)j * k];
      }
      if (l < k) v0 += A1(r, l) * P[l + (long)j * k];
      Tb[t] = v0 + v1;
    }
  };
  form_t1();
  __syncthreads();
  // one Newton-Schulz step P_1 <- P_1 (2 I - T_1) towards the pseudo-inverse: the normal
  // equations square the condition number, the step squares P_1's relative error again
  // (QR accuracy up to kappa ~ 1e7); the new P_1 goes to W's free left block (columns
  // 0..k-1) and to trow (column k), then back
  for (int t = threadIdx.x; t < k * ld; t += GT) {
    const int l = t % k, j = t / k;
    c128 v0 = P[l + (long)j * k] + P[l + (long)j * k], v1 = {0, 0};
    int r = 0;
    for (; r + 1 <= k; r += 2) {
      v0 -= P[l + (long)r * k] * Tb[r + (long)j * ld];
      v1 -= P[l + (long)(r + 1) * k] * Tb[r + 1 + (long)j * ld];
    }
    if (r <= k) v0 -= P[l + (long)r * k] * Tb[r + (long)j * ld];
    if (j < k) W[l + (long)j * k] = v0 + v1;
    else trow[l] = v0 + v1;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * ld; t += GT) {
    const int l = t % k, j = t / k;
    P[l + (long)j * k] = (j < k) ? W[l + (long)j * k] : trow[l];
  }
  __syncthreads();
  form_t1();
  if (i == 0) {
    for (int t = threadIdx.x; t < ld * ld; t += GT) {
      const int r = t % ld, j = t / ld;
      ob[t] = (r < k) ? P[r + (long)j * k] : c128{0, 0};
    }
    if (__syncthreads_or(!ok)) set_err(st, GDR_EBREAKDOWN);
    return;
  }
  __syncthreads();  // this CTA's T_1 is complete
  const c128 si = a.sigma[(long)c * a.ns + i];
  for (int t = threadIdx.x; t < k * w; t += GT) {
    const int p = t % k, q = t / k;
    if (q < k) {
      c128 h = Hk[p + (long)q * (k + 1)];
      if (p == q) h -= si;
      W[t] = h;
    } else {
      W[t] = Tb[p + (long)(q - k) * ld];
    }
  }
  for (int j = threadIdx.x; j < ld; j += GT) trow[j] = Tb[k + (long)j * ld];
  __syncthreads();
  ok = cta_gauss_jordan(W, k, w, &piv_s, &inv_s) && ok;
  for (int t = threadIdx.x; t < ld * ld; t += GT) {
    const int r = t % ld, j = t / ld;
    if (r < k) {
      Tb[t] = P[r + (long)j * k];  // S_i (W's right block)
    } else {
      c128 g = trow[j];
      for (int l = 0; l < k; ++l) g -= Hk[k + (long)l * (k + 1)] * P[l + (long)j * k];
      Tb[t] = g;
    }
  }
  if (__syncthreads_or(!ok)) set_err(st, GDR_EBREAKDOWN);
}

// one cycle's projection (one CTA per column and shift): the operators applied to c
__global__ void __launch_bounds__(DT) dense_proj_kernel(ProjArgs a, const c128* ops) {
  __shared__ c128 cs[GDR_MAX_M + 2];
  const int c = blockIdx.y, i = blockIdx.x;
  ColState* st = a.st + c;
  if (!st->active) return;
  const int k = a.k, ld = k + 1, ldc = k + 1;
  const long bs = (long)ld * ld;
  c128* Cf = a.Cf + (long)c * a.ccs;
  if (i > 0 && !a.sact[(long)c * a.ns + i]) {
    for (int r = threadIdx.x; r <= k; r += DT) Cf[r + (long)i * ldc] = {0, 0};
    return;
  }
  for (int r = threadIdx.x; r <= k; r += DT) cs[r] = a.cproj[(long)c * (k + 2) + r];
  __syncthreads();
  const c128* ob = ops + (long)c * (a.ns + 1) * bs;
  const c128 bi = (i > 0) ? a.beta[(long)c * a.ns + i] : c128{1, 0};
  const int nrow = (i == 0) ? 2 * ld : ld;
  for (int r = threadIdx.x; r < nrow; r += DT) {
    const bool tpart = r >= ld;  // base CTA: rows of T_1 after those of P_1
    const int q = tpart ? r - ld : r;
    const c128* M = ob + (long)(tpart ? a.ns : i) * bs + q;
    c128 acc0 = {0, 0}, acc1 = {0, 0};
    int j = 0;
    for (; j + 1 <= k; j += 2) {
      acc0 += M[(long)j * ld] * cs[j];
      acc1 += M[(long)(j + 1) * ld] * cs[j + 1];
    }
    if (j <= k) acc0 += M[(long)j * ld] * cs[j];
    const c128 v = acc0 + acc1;
    if (i == 0) {
      if (tpart) Cf[q + (long)a.ns * ldc] = -v;
      else Cf[q] = (q < k) ? v : c128{0, 0};
    } else if (q < k) {
      Cf[q + (long)i * ldc] = bi * v;
    } else {
      Cf[k + (long)i * ldc] = {0, 0};
      a.gamma[(long)c * a.ns + i] += bi * v;
    }
  }
}

// Selected approximate eigenvectors of a kept pair (Sec. 4, Theorem 1, Example 4).
// d: the kept pair as a cycle of size m = k (dense leading block), d.k = ks, graw /
// gtheta set.  After the harmonic Ritz step: unit columns of G, theta of A (+ sigma_1),
// eigen-residuals, and M = (G^H G)^{-1} G^H by Gaussian elimination with partial
// pivoting on [G^H G | G^H] in the column's FP64 scratch (row-major, width ks + k).
__global__ void __launch_bounds__(DT) eigsel_setup_kernel(DenseCycle d, c128* M, double* res) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Sh sh;
  __shared__ int piv_s;
  if (!harmonic_ritz<double>(d, 0, smem_raw, sh)) return;
  const int k = d.m, ks = d.k, ldg = k + 1, w = ks + k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  c128* G = d.graw;
  c128* th = d.gtheta;
  const c128 s1 = d.sigma[0];
  const c128* H = d.H;  // (k+1) x k
  for (int q = warp; q < ks; q += DT / 32) {  // unit columns, eigen-residuals
    c128* g = G + (long)q * ldg;
    double nn = 0;
    for (int i = lane; i < k; i += 32) nn += norm2(g[i]);
    nn = warp_sum_r(nn);
    const double inv = 1.0 / sqrt(nn);
    for (int i = lane; i < k; i += 32) g[i] = inv * g[i];
    __syncwarp();
    const c128 lam = th[q] + s1;
    double rr = 0;
    for (int r = lane; r <= k; r += 32) {
      c128 acc = (r < k) ? -(lam * g[r]) : c128{0, 0};
      for (int j = 0; j < k; ++j) acc += H[r + (long)j * (k + 1)] * g[j];
      rr += norm2(acc);
    }
    rr = warp_sum_r(rr);
    if (lane == 0) {
      th[q] = lam;
      res[q] = sqrt(rr);
    }
  }
  __syncthreads();
  c128* Aug = reinterpret_cast<c128*>(d.scratch);  // ks x (ks + k)
  for (int q = threadIdx.x; q < ks * w; q += DT) {
    const int r = q / w, cc = q % w;
    c128 v = {0, 0};
    if (cc < ks) {
      for (int i = 0; i < k; ++i) v += cmulc(G[i + (long)r * ldg], G[i + (long)cc * ldg]);
    } else {
      v = conj(G[(cc - ks) + (long)r * ldg]);
    }
    Aug[q] = v;
  }
  __syncthreads();
  for (int p = 0; p < ks; ++p) {
    if (warp == 0) {
      double best = -1.0;
      int pv = p;
      for (int r = p + lane; r < ks; r += 32) {
        const double a = norm2(Aug[(long)r * w + p]);
        if (a > best) {
          best = a;
          pv = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, pv, o);
        if (ob > best || (ob == best && op < pv)) {
          best = ob;
          pv = op;
        }
      }
      if (lane == 0) piv_s = pv;
    }
    __syncthreads();
    const int pv = piv_s;
    if (pv != p)
      for (int cc = p + threadIdx.x; cc < w; cc += DT) {
        const c128 t = Aug[(long)p * w + cc];
        Aug[(long)p * w + cc] = Aug[(long)pv * w + cc];
        Aug[(long)pv * w + cc] = t;
      }
    __syncthreads();
    const c128 pval = Aug[(long)p * w + p];
    const double pn = norm2(pval);
    if (pn > 0.0) {
      const c128 inv = {pval.x / pn, -pval.y / pn};
      const int rows = ks - p - 1, cols = w - p;
      for (int q = threadIdx.x; q < rows * cols; q += DT) {
        const int r = p + 1 + q / cols, cc = p + q % cols;
        const c128 f = Aug[(long)r * w + p] * inv;
        if (cc > p) Aug[(long)r * w + cc] -= f * Aug[(long)p * w + cc];
      }
      __syncthreads();
      for (int r = p + 1 + threadIdx.x; r < ks; r += DT) Aug[(long)r * w + p] = {0, 0};
    } else if (threadIdx.x == 0) {
      set_err(d.st, GDR_EBREAKDOWN);  // dependent eigenvectors
    }
    __syncthreads();
  }
  // back substitution, one thread per column of G^H: M[l][j], row-major ks x k
  for (int j = threadIdx.x; j < k; j += DT) {
    for (int l = ks - 1; l >= 0; --l) {
      c128 acc = Aug[(long)l * w + ks + j];
      for (int q = l + 1; q < ks; ++q) acc -= Aug[(long)l * w + q] * M[(long)q * k + j];
      const c128 pval = Aug[(long)l * w + l];
      const double pn = norm2(pval);
      M[(long)l * k + j] = pn > 0.0 ? acc * c128{pval.x / pn, -pval.y / pn} : c128{0, 0};
    }
  }
}

struct EigSelArgs {
  const c128* G; const c128* M; const c128* theta; int ks;
};

// Theorem 1 projection for column c (grid.y) and shift i (grid.x)
__global__ void __launch_bounds__(DT) eigsel_proj_kernel(ProjArgs a, EigSelArgs e) {
  __shared__ c128 dv[GDR_MAX_M], ev[GDR_MAX_M + 1];
  const int c = blockIdx.y, i = blockIdx.x;
  ColState* st = a.st + c;
  if (!st->active) return;
  const int k = a.k, ldc = k + 1, ks = e.ks, ldg = k + 1;
  const c128* Hk = a.Hk + (long)(c / a.hpp) * a.hkcs;
  c128* Cf = a.Cf + (long)c * a.ccs;
  const int* sact = a.sact + (long)c * a.ns;
  if (i > 0 && !sact[i]) {
    for (int r = threadIdx.x; r <= k; r += DT) Cf[r + (long)i * ldc] = {0, 0};
    return;
  }
  const c128* cp = a.cproj + (long)c * (k + 2);
  const c128 si = a.sigma[(long)c * a.ns + i];
  const c128 bi = i == 0 ? c128{1, 0} : a.beta[(long)c * a.ns + i];
  for (int l = threadIdx.x; l < ks; l += DT) {
    c128 acc = {0, 0};
    for (int j = 0; j < k; ++j) acc += e.M[(long)l * k + j] * cp[j];
    const c128 den = e.theta[l] - si;
    const double dn = norm2(den);
    dv[l] = (bi * acc) * c128{den.x / dn, -den.y / dn};
  }
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += DT) {
    c128 acc = {0, 0};
    for (int l = 0; l < ks; ++l) acc += e.G[r + (long)l * ldg] * dv[l];
    ev[r] = acc;
    Cf[r + (long)i * ldc] = acc;
  }
  if (threadIdx.x == 0) Cf[k + (long)i * ldc] = {0, 0};
  __syncthreads();
  if (i == 0) {  // residual column -(Hbar_k - sigma_1 Ibar) e_1
    for (int r = threadIdx.x; r <= k; r += DT) {
      c128 acc = (r < k) ? -(si * ev[r]) : c128{0, 0};
      for (int j = 0; j < k; ++j) acc += Hk[r + (long)j * (k + 1)] * ev[j];
      Cf[r + (long)a.ns * ldc] = -acc;
    }
  }
}

}  // namespace

size_t dense_smem_bytes(int m, int k) {
  // largest of: shift solve (m+1) x (m+3) + vectors; harmonic Ritz m x (m+2) + 4m;
  // restart completion P ((m+1) x (k+1)), T1 ((m+1) x k), coefficients
  const size_t a = (size_t)(m + 2) * (m + 3) + 2 * (m + 2);
  const size_t b = (size_t)(m + 1) * (m + 2) + 4 * (size_t)m + 8;
  const size_t r = (size_t)(m + 1) * (2 * k + 1) + k + 2;
  return sizeof(c128) * std::max(a, std::max(b, r));
}

void dense_init(gdr_ctx* ctx) {
  size_t lim = set_max_dyn_smem(ctx, dense_d1_kernel);
  lim = std::min(lim, set_max_dyn_smem(ctx, dense_d2_kernel));
  lim = std::min(lim, set_max_dyn_smem(ctx, proj_gj_setup_kernel));
  lim = std::min(lim, set_max_dyn_smem(ctx, eigsel_setup_kernel));
  lim = std::min(lim, set_max_dyn_smem(ctx, restart_only_kernel));
  ctx->dense_smem_limit = lim;
}

// dynamic shared memory of the cycle kernels; drops the FP32 harmonic Ritz form
// (hr32) when its layout does not fit
static size_t cycle_smem(gdr_ctx* ctx, DenseCycle& d) {
  size_t smem = dense_smem_bytes(d.m, d.k);
  GDR_REQUIRE(smem <= ctx->dense_smem_limit, "basis size m too large for the dense FP64 kernels");
  if (d.hr32 && d.k > 0) {
    const size_t s32 = (size_t)hr32_layout(d.m, d.k).total;
    if (s32 <= ctx->dense_smem_limit)
      smem = std::max(smem, s32);
    else
      d.hr32 = 0;
  }
  return smem;
}

void dense_restart(gdr_ctx* ctx, const DenseCycle& dc) {
  DenseCycle d = dc;
  const size_t smem = cycle_smem(ctx, d);
  dim3 g(1, (unsigned)d.ncol);
  restart_only_kernel<<<g, DT, smem, ctx->stream>>>(d, 0);
  GDR_LAUNCHED(ctx);
  restart_only_kernel<<<g, DT, smem, ctx->stream>>>(d, 1);
  GDR_LAUNCHED(ctx);
}

void dense_cycle(gdr_ctx* ctx, const DenseCycle& dc) {
  DenseCycle d = dc;
  const size_t smem = cycle_smem(ctx, d);
  dim3 g1(d.k > 0 ? 2 : 1, (unsigned)d.ncol);
  {
    KProf kp(ctx, d.k > 0 ? "dense_ls_harmonic_ritz" : "dense_ls", 0.0);
    dense_d1_kernel<<<g1, DT, smem, ctx->stream>>>(d);
    GDR_LAUNCHED(ctx);
  }
  // restart products over up to 8 CTAs per column, about 4 columns of P_k each
  d.rslices = d.k > 0 ? std::max(1, std::min(8, d.k / 4)) : 1;
  dim3 g2((unsigned)(d.ns + d.rslices - 1), (unsigned)d.ncol);
  {
    KProf kp(ctx, "dense_shifts_restart", 0.0);
    dense_d2_kernel<<<g2, DT, smem, ctx->stream>>>(d);
    GDR_LAUNCHED(ctx);
  }
}

void cycle_finish(gdr_ctx* ctx, const DenseCycle& d, c128* H, c128* cvec) {
  cycle_finish_kernel<<<d.ncol, 128, 0, ctx->stream>>>(d, H, cvec);
  GDR_LAUNCHED(ctx);
}

void proj_setup(gdr_ctx* ctx, int ncol, int k, int ns, const c128* Hk, const c128* sigma, ColState* st, c128* ops,
                long hkcs, int hpp) {
  GDR_REQUIRE(k >= 1 && k <= GDR_MAX_M, "bad projection size");
  ProjArgs a{k, ns, Hk, nullptr, sigma, nullptr, nullptr, nullptr, nullptr, 0, st, hkcs, hpp};
  const size_t smem = proj_gj_smem(k);
  GDR_REQUIRE(smem <= ctx->dense_smem_limit, "k too large for the projection setup");
  KProf kp(ctx, "dense_projection_setup", 0.0);
  dim3 g((unsigned)ns, (unsigned)ncol);
  proj_gj_setup_kernel<<<g, GT, smem, ctx->stream>>>(a, ops);
  GDR_LAUNCHED(ctx);
}

void dense_projection(gdr_ctx* ctx, int ncol, int k, int ns, const c128* Hk, const c128* cproj, const c128* sigma,
                      const c128* beta, const int* sact, c128* gamma, c128* Cf, long ccs, const c128* ops,
                      ColState* st, long hkcs, int hpp, const EigSel* es) {
  ProjArgs a{k, ns, Hk, cproj, sigma, beta, sact, gamma, Cf, ccs, st, hkcs, hpp};
  if (es) {
    GDR_REQUIRE(es->ks >= 1 && es->ks <= k && k <= GDR_MAX_M, "bad eigenvector selection");
    dim3 g((unsigned)ns, (unsigned)ncol);
    KProf kp(ctx, "dense_projection_eigsel", 0.0);
    eigsel_proj_kernel<<<g, DT, 0, ctx->stream>>>(a, EigSelArgs{es->G, es->M, es->theta, es->ks});
    GDR_LAUNCHED(ctx);
    return;
  }
  GDR_REQUIRE(ops != nullptr && k <= GDR_MAX_M, "projection operators not formed");
  dim3 g((unsigned)ns, (unsigned)ncol);
  KProf kp(ctx, "dense_projection", 0.0);
  dense_proj_kernel<<<g, DT, 0, ctx->stream>>>(a, ops);
  GDR_LAUNCHED(ctx);
}

void eigsel_setup(gdr_ctx* ctx, const c128* Hk, int k, int ks, c128 sigma1, EigSel& out, double* res_host) {
  GDR_REQUIRE(k >= 1 && k <= GDR_MAX_M && ks >= 1 && ks <= k, "bad eigenvector selection size");
  DenseCycle d{};
  d.ncol = 1;
  d.m = k;
  d.k = ks;
  d.ns = 1;
  d.kfull = k + 1;  // the kept Hbar_k is dense
  d.H = Hk;
  c128* sig = ctx->get<c128>("es.sigma", 1);
  GDR_CUDA(cudaMemcpyAsync(sig, &sigma1, sizeof(c128), cudaMemcpyHostToDevice, ctx->stream));
  d.sigma = sig;
  d.theta = ctx->get<c128>("es.theta_all", (size_t)k);
  d.scratch_per_col = std::max<long>(2L * ((long)k * k + 2L * k * ks + 64), 2L * (long)ks * (ks + k) + 64);
  d.scratch = ctx->get<double>("es.scratch", (size_t)d.scratch_per_col);
  d.Pk = ctx->get<c128>("es.Pk", (size_t)(k + 1) * ks);
  d.graw = ctx->get<c128>("es.G", (size_t)(k + 1) * ks);
  d.gtheta = ctx->get<c128>("es.theta", (size_t)ks);
  d.st = ctx->get<ColState>("es.st", 1);
  ColState s0 = {};
  s0.active = 1;
  s0.m_eff = k;
  GDR_CUDA(cudaMemcpyAsync(d.st, &s0, sizeof(s0), cudaMemcpyHostToDevice, ctx->stream));
  c128* M = ctx->get<c128>("es.M", (size_t)ks * k);
  double* res = ctx->get<double>("es.res", (size_t)ks);
  const size_t smem = dense_smem_bytes(k, ks);
  GDR_REQUIRE(smem <= ctx->dense_smem_limit, "k too large for the eigenvector selection");
  KProf kp(ctx, "eigsel_setup", 0.0);
  eigsel_setup_kernel<<<1, DT, smem, ctx->stream>>>(d, M, res);
  GDR_LAUNCHED(ctx);
  ColState s1;
  GDR_CUDA(cudaMemcpyAsync(&s1, d.st, sizeof(s1), cudaMemcpyDeviceToHost, ctx->stream));
  if (res_host) GDR_CUDA(cudaMemcpyAsync(res_host, res, sizeof(double) * ks, cudaMemcpyDeviceToHost, ctx->stream));
  GDR_CUDA(cudaStreamSynchronize(ctx->stream));
  if (s1.err) throw gdr_error((gdr_status)s1.err, "eigenvector selection: harmonic Ritz step failed");
  out.G = d.graw;
  out.M = M;
  out.theta = d.gtheta;
  out.ks = ks;
}
