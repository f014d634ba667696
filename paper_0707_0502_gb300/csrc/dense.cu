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
constexpr double EPS = 2.220446049250313e-16;

DEV c128 cdiv(c128 a, c128 b) {
  const double d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
DEV double cabs_(c128 a) { return hypot(a.x, a.y); }
DEV c128 csqrt_(c128 z) {
  const double r = cabs_(z);
  if (r == 0.0) return {0, 0};
  const double re = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0) return {re, z.y / (2 * re)};
  return {fabs(z.y) / (2 * re), copysign(re, z.y)};
}
DEV c128 shfl_xor_c(c128 v, int m) {
  return {__shfl_xor_sync(FULL, v.x, m), __shfl_xor_sync(FULL, v.y, m)};
}
DEV c128 warp_sum_c(c128 v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += shfl_xor_c(v, m);
  return v;
}
DEV double warp_sum_d(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(FULL, v, m);
  return v;
}

struct Sh {  // small shared scratch of a dense CTA
  double red[DT / 32];
  c128 bc[4];
  c128 nx[4];  // QR sweep: entries (kk+1, kk), (kk+1, kk+1), (kk+2, kk), (kk+2, kk+1) after the left update
  int ibc[4];
};

DEV double block_sum(double v, Sh& sh) {
  v = warp_sum_d(v);
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
#pragma unroll
  for (int w = 0; w < DT / 32; ++w) t += sh.red[w];
  __syncthreads();
  return t;
}

// Householder QR of the first `cols` columns of A (rows x ntot, column-major,
// lda), reflectors applied to all ntot columns.  R in the upper triangle, v
// below the diagonal, tau[j].  Column j of the factored part is known to be
// zero below row max(j+1, kfull) (the GMRES-DR recurrence matrix is upper
// Hessenberg except for a full leading block; kfull >= rows means dense), so
// reflector j spans rows j..last(j) only.
DEV int qr_last(int j, int rows, int kfull) { return min(rows - 1, max(j + 1, kfull)); }

DEV void cta_qr(c128* A, int lda, int rows, int cols, int ntot, c128* tau, Sh& sh, int kfull) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = 0; j < cols && j < rows; ++j) {
    const int last = qr_last(j, rows, kfull);
    double s = 0;
    for (int i = j + 1 + threadIdx.x; i <= last; i += DT) s += norm2(A[i + (long)j * lda]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      const c128 alpha = A[j + (long)j * lda];
      if (s == 0.0 && alpha.y == 0.0) {
        tau[j] = {0, 0};
      } else {
        const double beta = -copysign(sqrt(norm2(alpha) + s), alpha.x);
        tau[j] = {(beta - alpha.x) / beta, -alpha.y / beta};
        sh.bc[0] = cdiv(c128{1, 0}, alpha - c128{beta, 0});
        A[j + (long)j * lda] = {beta, 0};
      }
    }
    __syncthreads();
    const c128 tj = tau[j];
    if (tj.x == 0.0 && tj.y == 0.0) continue;  // uniform across the CTA
    const c128 scal = sh.bc[0];
    for (int i = j + 1 + threadIdx.x; i <= last; i += DT) A[i + (long)j * lda] = A[i + (long)j * lda] * scal;
    __syncthreads();
    const c128 ct = conj(tj);
    if (last - j < 32) {
      // short reflector: one thread per column
      for (int cc = j + 1 + threadIdx.x; cc < ntot; cc += DT) {
        c128* col = A + (long)cc * lda;
        c128 w = col[j];
        for (int i = j + 1; i <= last; ++i) w += cmulc(A[i + (long)j * lda], col[i]);
        const c128 f = ct * w;
        col[j] -= f;
        for (int i = j + 1; i <= last; ++i) col[i] -= A[i + (long)j * lda] * f;
      }
    } else {
      for (int cc = j + 1 + warp; cc < ntot; cc += DT / 32) {
        c128* col = A + (long)cc * lda;
        c128 w = {0, 0};
        for (int i = j + lane; i <= last; i += 32) {
          const c128 vi = (i == j) ? c128{1, 0} : A[i + (long)j * lda];
          w += cmulc(vi, col[i]);
        }
        w = warp_sum_c(w);
        const c128 f = ct * w;
        for (int i = j + lane; i <= last; i += 32) {
          const c128 vi = (i == j) ? c128{1, 0} : A[i + (long)j * lda];
          col[i] -= vi * f;
        }
      }
    }
    __syncthreads();
  }
}

// y <- Q y for the reflectors of cta_qr (applied in reverse order), one thread.
DEV void apply_q_serial(const c128* A, int lda, int rows, int cols, const c128* tau, c128* y, int kfull) {
  for (int j = min(cols, rows) - 1; j >= 0; --j) {
    const c128 tj = tau[j];
    if (tj.x == 0.0 && tj.y == 0.0) continue;
    const int last = qr_last(j, rows, kfull);
    c128 w = y[j];
    for (int i = j + 1; i <= last; ++i) w += cmulc(A[i + (long)j * lda], y[i]);
    const c128 f = tj * w;
    y[j] -= f;
    for (int i = j + 1; i <= last; ++i) y[i] -= A[i + (long)j * lda] * f;
  }
}

// Solve R y = y (R: upper nsz x nsz of A) in place.  Returns false on a zero pivot.
DEV bool cta_backsolve(const c128* A, int lda, int nsz, c128* y, Sh& sh) {
  bool ok = true;
  for (int j = nsz - 1; j >= 0; --j) {
    if (threadIdx.x == 0) {
      const c128 p = A[j + (long)j * lda];
      if (p.x == 0.0 && p.y == 0.0) {
        sh.ibc[0] = 1;
        y[j] = {0, 0};
      } else {
        y[j] = cdiv(y[j], p);
      }
    }
    __syncthreads();
    const c128 xj = y[j];
    for (int i = threadIdx.x; i < j; i += DT) y[i] -= A[i + (long)j * lda] * xj;
    __syncthreads();
  }
  if (sh.ibc[0]) ok = false;
  return ok;
}

// load (Hbar - sig Ibar)[0:rows, 0:cols] into A (lda)
DEV void load_shifted(c128* A, int lda, const c128* H, int ldh, int rows, int cols, c128 sig) {
  for (int t = threadIdx.x; t < rows * cols; t += DT) {
    const int i = t % rows, j = t / rows;
    c128 v = H[i + (long)j * ldh];
    if (i == j) v -= sig;
    A[i + (long)j * lda] = v;
  }
}

// odd leading dimension: row-wise accesses of 16-byte elements hit distinct banks
HD int odd_ld(int rows) { return rows | 1; }

DEV void set_err(ColState* st, int code) {
  if (threadIdx.x == 0) atomicCAS(&st->err, 0, code);
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
  const int rows = broke ? me : me + 1;
  const int lda = odd_ld(rows);
  load_shifted(A, lda, H, m + 1, rows, me, sig);
  for (int i = threadIdx.x; i < rows; i += DT) A[i + (long)me * lda] = cv[i];
  c128* tau = A + (long)lda * (me + 1);
  c128* y = tau + (me + 1);
  if (threadIdx.x == 0) sh.ibc[0] = 0;
  __syncthreads();
  cta_qr(A, lda, rows, me, me + 1, tau, sh, d.kfull);
  for (int i = threadIdx.x; i < me; i += DT) y[i] = A[i + (long)me * lda];
  __syncthreads();
  if (!cta_backsolve(A, lda, me, y, sh)) set_err(st, GDR_EBREAKDOWN);
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
  const int rows = broke ? me : me + 1;
  const int lda = odd_ld(rows);
  load_shifted(A, lda, H, m + 1, rows, me, sig);
  for (int r = threadIdx.x; r < rows; r += DT) {
    A[r + (long)me * lda] = cv[r];
    A[r + (long)(me + 1) * lda] = s[r];
  }
  c128* tau = A + (long)lda * (me + 2);
  c128* y = tau + (me + 1);
  if (threadIdx.x == 0) sh.ibc[0] = 0;
  __syncthreads();
  cta_qr(A, lda, rows, me, me + 2, tau, sh, d.kfull);
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
  if (!cta_backsolve(A, lda, me, y, sh)) set_err(st, GDR_EBREAKDOWN);
  for (int r = threadIdx.x; r <= m; r += DT) Cf[r + (long)col * d.ldc] = (r < me) ? y[r] : c128{0, 0};
  if (threadIdx.x == 0) {
    d.beta[(long)c * d.ns + i] = bnew;
    d.norms[(long)c * d.ns + i] = cabs_(bnew) * st->rnorm;
  }
}

// --------------------------------------------------- harmonic Ritz (D1)

// 1/sqrt(a) for a > 0: single-precision estimate, then two Newton steps
// y <- y (3 - a y^2) / 2 in FP64 (quadratic convergence: ~1e-7 -> 1e-14 -> 1e-16).
// A normal-range float must hold a; otherwise fall back to the FP64 expression.
DEV double rsqrt_nr(double a) {
  if (!(a > 1e-36 && a < 1e36)) return 1.0 / sqrt(a);
  double y = (double)rsqrtf((float)a);
  y = y * (1.5 - 0.5 * a * y * y);
  y = y * (1.5 - 0.5 * a * y * y);
  return y;
}

// Givens rotation U = [[cs, sn], [-conj(sn), cs]] with U [x; y] = [r; 0]; rot = {cs, Re sn, Im sn}
DEV void givens(c128 x, c128 y, double* rot) {
  const double ax2 = norm2(x), ay2 = norm2(y);
  if (ay2 == 0.0) {
    rot[0] = 1.0; rot[1] = 0.0; rot[2] = 0.0;
  } else if (ax2 == 0.0) {
    const double inv = rsqrt_nr(ay2);
    rot[0] = 0.0; rot[1] = y.x * inv; rot[2] = -y.y * inv;
  } else {
    const double inv_r = rsqrt_nr(ax2 + ay2);
    const double inv_ax = rsqrt_nr(ax2);
    rot[0] = ax2 * inv_ax * inv_r;  // |x| / r
    // sn = (x / |x|) conj(y) / r
    const double f = inv_ax * inv_r;
    rot[1] = (x.x * y.x + x.y * y.y) * f;
    rot[2] = (x.y * y.x - x.x * y.y) * f;
  }
}

// selection order with precomputed magnitudes
DEV bool before_m(c128 a, double ma, c128 b, double mb) {
  const double scale = fmax(ma, mb);
  if (fabs(ma - mb) > 1e-9 * scale) return ma < mb;
  if (fabs(a.y - b.y) > 1e-9 * scale) return a.y > b.y;
  return a.x > b.x;
}

// selection order of the "smallest" harmonic Ritz values
DEV bool before(c128 a, c128 b) {
  const double ma = cabs_(a), mb = cabs_(b);
  const double scale = fmax(ma, mb);
  if (fabs(ma - mb) > 1e-9 * scale) return ma < mb;
  if (fabs(a.y - b.y) > 1e-9 * scale) return a.y > b.y;
  return a.x > b.x;
}

// Hessenberg reduction + shifted QR with Schur vectors + eigenvectors of the
// k smallest; writes P_k ((m+1) x k, orthonormal, last row 0) and theta.
DEV void harmonic_ritz(const DenseCycle& d, int c, c128* T, Sh& sh) {
  ColState* st = d.st + c;
  const int m = d.m, k = d.k;
  const c128* H = d.H + (long)c * (m + 1) * m;
  const c128 sig = d.sigma[(long)c * d.ns];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* scr = d.scratch + (long)c * d.scratch_per_col;
  c128* Z = reinterpret_cast<c128*>(scr);        // m x m, row-major, row t owned by thread t
  c128* Y = Z + (long)m * m;                     // m x k   eigenvectors of T
  c128* G = Y + (long)m * k;                     // m x k   eigenvectors of M
  const int lda = odd_ld(m);
  c128* f = T + (long)lda * (m + 2);             // m
  c128* tau = f + m;                             // m
  c128* theta = tau + m;                         // m
  int* sel = reinterpret_cast<int*>(theta + m);  // k
  GDR_DENSE_MARK(0, 0);
  // 1) f = H^{-H} hrow^H with H = Hhat[0:m, 0:m] = Q R:  R^H z = hrow^H, f = Q z
  load_shifted(T, lda, H, m + 1, m, m, sig);
  if (threadIdx.x == 0) sh.ibc[0] = 0;
  __syncthreads();
  cta_qr(T, lda, m, m, m, tau, sh, d.kfull);
  if (threadIdx.x == 0) {
    for (int j = 0; j < m; ++j) {  // forward substitution with R^H
      c128 v = conj(H[m + (long)j * (m + 1)]);
      for (int i = 0; i < j; ++i) v -= cmulc(T[i + (long)j * lda], f[i]);
      const c128 rjj = T[j + (long)j * lda];
      if (rjj.x == 0.0 && rjj.y == 0.0) {
        sh.ibc[0] = 1;
        f[j] = {0, 0};
      } else {
        f[j] = cdiv(v, conj(rjj));
      }
    }
    apply_q_serial(T, lda, m, m, tau, f, d.kfull);
  }
  __syncthreads();
  if (sh.ibc[0]) set_err(st, GDR_EBREAKDOWN);
  GDR_DENSE_MARK(1, 0);
  // 2) M = H + f hrow
  for (int t = threadIdx.x; t < m * m; t += DT) {
    const int i = t % m, j = t / m;
    c128 v = H[i + (long)j * (m + 1)];
    if (i == j) v -= sig;
    T[i + (long)j * lda] = v + f[i] * H[m + (long)j * (m + 1)];
  }
  __syncthreads();
  GDR_DENSE_MARK(2, 0);
  // 3) Hessenberg reduction M = Q Hh Q^H, reflectors kept below the subdiagonal
  for (int j = 0; j + 2 < m; ++j) {
    double s = 0;
    for (int i = j + 2 + threadIdx.x; i < m; i += DT) s += norm2(T[i + (long)j * lda]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      const c128 alpha = T[j + 1 + (long)j * lda];
      if (s == 0.0 && alpha.y == 0.0) {
        tau[j] = {0, 0};
      } else {
        const double beta = -copysign(sqrt(norm2(alpha) + s), alpha.x);
        tau[j] = {(beta - alpha.x) / beta, -alpha.y / beta};
        sh.bc[0] = cdiv(c128{1, 0}, alpha - c128{beta, 0});
        T[j + 1 + (long)j * lda] = {beta, 0};
      }
    }
    __syncthreads();
    const c128 tj = tau[j];
    if (tj.x == 0.0 && tj.y == 0.0) continue;
    const c128 scal = sh.bc[0];
    for (int i = j + 2 + threadIdx.x; i < m; i += DT) T[i + (long)j * lda] = T[i + (long)j * lda] * scal;
    __syncthreads();
    // left: rows j+1.., columns j+1..m-1 : (I - conj(tau) v v^H)
    const c128 ct = conj(tj);
    for (int cc = j + 1 + warp; cc < m; cc += DT / 32) {
      c128* colp = T + (long)cc * lda;
      c128 w = {0, 0};
      for (int i = j + 1 + lane; i < m; i += 32) {
        const c128 vi = (i == j + 1) ? c128{1, 0} : T[i + (long)j * lda];
        w += cmulc(vi, colp[i]);
      }
      w = warp_sum_c(w);
      const c128 fct = ct * w;
      for (int i = j + 1 + lane; i < m; i += 32) {
        const c128 vi = (i == j + 1) ? c128{1, 0} : T[i + (long)j * lda];
        colp[i] -= vi * fct;
      }
    }
    __syncthreads();
    // right: all rows, columns j+1..m-1 : M (I - tau v v^H)
    for (int r = warp; r < m; r += DT / 32) {
      c128 w = {0, 0};
      for (int i = j + 1 + lane; i < m; i += 32) {
        const c128 vi = (i == j + 1) ? c128{1, 0} : T[i + (long)j * lda];
        w += T[r + (long)i * lda] * vi;
      }
      w = warp_sum_c(w);
      const c128 fct = tj * w;
      for (int i = j + 1 + lane; i < m; i += 32) {
        const c128 vi = (i == j + 1) ? c128{1, 0} : T[i + (long)j * lda];
        T[r + (long)i * lda] -= fct * conj(vi);
      }
    }
    __syncthreads();
  }
  GDR_DENSE_MARK(3, 0);
  // 4) Z = Q = H_0 H_1 ... : Z <- Z H_j for j = 0.., one warp per row of Z
  //    (I - tau v v^H applied from the right), then clear below the subdiagonal.
  //    During the QR sweep row t of Z belongs to thread DT-1-t.
  const int zrow = DT - 1 - threadIdx.x;  // row of Z owned by this thread in the sweep
  for (int r = warp; r < m; r += DT / 32) {
    c128* zr = Z + (long)r * m;
    for (int i = lane; i < m; i += 32) zr[i] = {r == i ? 1.0 : 0.0, 0.0};
  }
  __syncthreads();
  for (int j = 0; j + 2 < m; ++j) {
    const c128 tj = tau[j];
    if (tj.x == 0.0 && tj.y == 0.0) continue;
    for (int r = warp; r < m; r += DT / 32) {
      c128* zr = Z + (long)r * m;
      c128 w = {0, 0};
      for (int i = j + 1 + lane; i < m; i += 32) {
        const c128 vi = (i == j + 1) ? c128{1, 0} : T[i + (long)j * lda];
        w += zr[i] * vi;
      }
      w = warp_sum_c(w);
      const c128 fct = tj * w;
      for (int i = j + 1 + lane; i < m; i += 32) {
        const c128 vi = (i == j + 1) ? c128{1, 0} : T[i + (long)j * lda];
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
  // 5) complex single-shift QR to Schur form T = Z^H M Z
  double hnorm = 0;
  for (int q = threadIdx.x; q < m * m; q += DT) hnorm = fmax(hnorm, cabs_(T[q]));
  {
    // max over the CTA
    double v = hnorm;
#pragma unroll
    for (int mm = 16; mm > 0; mm >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, mm));
    if (lane == 0) sh.red[warp] = v;
    __syncthreads();
    hnorm = fmax(fmax(sh.red[0], sh.red[1]), fmax(sh.red[2], sh.red[3]));
    __syncthreads();
  }
  const double smallnum = fmax(hnorm * EPS, 1e-300);
  const double eps2 = EPS * EPS;
  double* rot = reinterpret_cast<double*>(&sh.bc[1]);  // rot[0] = cs, (rot[1], rot[2]) = sn
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
          const double sub = norm2(T[cand + (long)(cand - 1) * lda]);
          double ref = norm2(T[cand - 1 + (long)(cand - 1) * lda]) + norm2(T[cand + (long)cand * lda]);
          if (ref == 0.0) ref = hnorm * hnorm;
          neg = (sub <= eps2 * ref || sub <= smallnum * smallnum * 1e-6);
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
        c128 mu;
        const c128 a = T[hi - 1 + (long)(hi - 1) * lda], b = T[hi - 1 + (long)hi * lda];
        const c128 cc = T[hi + (long)(hi - 1) * lda], dd = T[hi + (long)hi * lda];
        if (its % 10 == 0) {
          mu = dd + c128{fabs(cc.x) + fabs(cc.y), 0};
        } else {
          const c128 half = 0.5 * (a - dd);
          const c128 disc = csqrt_(half * half + b * cc);
          const c128 l1 = dd + half + disc, l2 = dd + half - disc;
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
      const double cs = rot[0];
      const c128 sn = {rot[1], rot[2]};
      // left: rows kk, kk+1, columns max(kk-1,0)..m-1
      for (int cc = max(kk - 1, 0) + threadIdx.x; cc < m; cc += DT) {
        const c128 a = T[kk + (long)cc * lda], b = T[kk + 1 + (long)cc * lda];
        const c128 b_new = (cc == kk - 1 && kk > lo) ? c128{0, 0} : cs * b - conj(sn) * a;
        T[kk + (long)cc * lda] = cs * a + sn * b;
        T[kk + 1 + (long)cc * lda] = b_new;
        if ((cc == kk || cc == kk + 1) && kk + 2 <= hi) {  // inputs of the next rotation
          sh.nx[cc - kk] = b_new;
          sh.nx[2 + cc - kk] = T[kk + 2 + (long)cc * lda];
        }
      }
      __syncthreads();
      // right: columns kk, kk+1, rows 0..min(kk+2, hi); the thread of row kk+2 (or kk+1
      // at the end of the sweep) also does row kk+1 and forms the next rotation
      const int rlast = min(kk + 2, hi);
      // (the owner, a thread with no row of this update, forms the next rotation from
      //  the entries of rows kk+1, kk+2 saved by the left update)
      c128 x_next = {0, 0}, y_next = {0, 0};
      const bool own = (threadIdx.x == DT - 1 - m) && (kk + 2 <= hi);
      if (own) {
        x_next = cs * sh.nx[0] + sh.nx[1] * conj(sn);
        y_next = cs * sh.nx[2] + sh.nx[3] * conj(sn);
      }
      for (int r = threadIdx.x; r <= rlast; r += DT) {
        const c128 a = T[r + (long)kk * lda], b = T[r + (long)(kk + 1) * lda];
        T[r + (long)kk * lda] = cs * a + b * conj(sn);
        T[r + (long)(kk + 1) * lda] = cs * b - a * sn;
      }
      if (own) givens(x_next, y_next, rot);
      if (zrow >= 0 && zrow < m) {
        c128* zr = Z + (long)zrow * m;
        const c128 a = zr[kk], b = zr[kk + 1];
        zr[kk] = cs * a + b * conj(sn);
        zr[kk + 1] = cs * b - a * sn;
      }
      __syncthreads();
    }
  }
  if (failed) {
    set_err(st, GDR_EBREAKDOWN);
    return;
  }
  __syncthreads();
  GDR_DENSE_MARK(5, 0);
  // 6) eigenvalues and selection of the k smallest
  c128* th = d.theta + (long)c * m;
  for (int i = threadIdx.x; i < m; i += DT) {
    theta[i] = T[i + (long)i * lda];
    th[i] = theta[i];
  }
  __syncthreads();
  // k rounds of a warp argmin under `before` (ties: lower index), which picks what
  // the index-order selection sort picks for a consistent order; |theta| computed once
  if (warp == 0) {
    double mag[3];
    unsigned used = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int i = lane + 32 * q;
      mag[q] = (i < m) ? sqrt(norm2(theta[i])) : 0.0;
    }
    for (int q = 0; q < k; ++q) {
      int bi = -1;
      double bm = 0.0;
      c128 bt = {0, 0};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int i = lane + 32 * r;
        if (i >= m || (used >> r & 1u)) continue;
        if (bi < 0 || before_m(theta[i], mag[r], bt, bm)) { bi = i; bm = mag[r]; bt = theta[i]; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const int oi = __shfl_xor_sync(FULL, bi, off);
        const double om = __shfl_xor_sync(FULL, bm, off);
        const c128 ot = shfl_xor_c(bt, off);
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
    const c128 lam = theta[p];
    c128* y = Y + (long)q * m;
    for (int i = p + 1; i < m; ++i) y[i] = {0, 0};
    y[p] = {1, 0};
    for (int i = p - 1; i >= 0; --i) {
      c128 sacc = {0, 0};
      for (int j = i + 1; j <= p; ++j) sacc += T[i + (long)j * lda] * y[j];
      c128 den = T[i + (long)i * lda] - lam;
      if (cabs_(den) < smallnum) den = {smallnum, 0};
      y[i] = -cdiv(sacc, den);
    }
    // normalise (avoid overflow in later products)
    double nn = 0;
    for (int i = 0; i <= p; ++i) nn = fmax(nn, cabs_(y[i]));
    for (int i = 0; i <= p; ++i) y[i] = (1.0 / nn) * y[i];
  }
  __syncthreads();
  GDR_DENSE_MARK(7, 0);
  // 8) G = Z Y : thread t computes row t of G (Z is complete after the barrier)
  const int t = threadIdx.x;
  if (t < m) {
    const c128* zr = Z + (long)t * m;
    for (int q = 0; q < k; ++q) {
      const c128* y = Y + (long)q * m;
      const int p = sel[q];
      c128 acc = {0, 0};
      for (int j = 0; j <= p; ++j) acc += zr[j] * y[j];
      G[t + (long)q * m] = acc;
    }
  }
  __syncthreads();
  GDR_DENSE_MARK(8, 0);
  // 9) P_k = orth([G; 0]) by classical Gram-Schmidt twice, in T (ld m+1)
  const int ldp = m + 1;
  for (int q = threadIdx.x; q < ldp * k; q += DT) {
    const int i = q % ldp, j = q / ldp;
    T[q] = (i < m) ? G[i + (long)j * m] : c128{0, 0};
  }
  __syncthreads();
  c128* coef = theta;  // reuse (size >= k)
  for (int q = 0; q < k; ++q) {
    c128* pq = T + (long)q * ldp;
    for (int pass = 0; pass < 2; ++pass) {
      for (int l = warp; l < q; l += DT / 32) {
        const c128* pl = T + (long)l * ldp;
        c128 w = {0, 0};
        for (int i = lane; i < m; i += 32) w += cmulc(pl[i], pq[i]);
        w = warp_sum_c(w);
        if (lane == 0) coef[l] = w;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += DT) {
        c128 v = pq[i];
        for (int l = 0; l < q; ++l) v -= T[i + (long)l * ldp] * coef[l];
        pq[i] = v;
      }
      __syncthreads();
    }
    double nn = 0;
    for (int i = threadIdx.x; i < m; i += DT) nn += norm2(pq[i]);
    nn = block_sum(nn, sh);
    if (!(nn > 0) || !isfinite(nn)) set_err(st, GDR_EBREAKDOWN);
    const double inv = 1.0 / sqrt(nn);
    for (int i = threadIdx.x; i < m; i += DT) pq[i] = inv * pq[i];
    __syncthreads();
  }
  c128* Pk = d.Pk + (long)c * ldp * k;
  for (int q = threadIdx.x; q < ldp * k; q += DT) Pk[q] = T[q];
  GDR_DENSE_MARK(9, total);
}

// restart completion (D2 block 0): p_{k+1} from s, P into Cf, Hbar_k, c_k
DEV void restart_finish(const DenseCycle& d, int c, c128* A, Sh& sh) {
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
  // T1 = Hbar (m+1 x m) * P_k[0:m, :]
  for (int q = threadIdx.x; q < ldp * k; q += DT) {
    const int i = q % ldp, j = q / ldp;
    c128 acc = {0, 0};
    for (int l = 0; l < m; ++l) acc += H[i + (long)l * (m + 1)] * P[l + (long)j * ldp];
    T1[q] = acc;
  }
  __syncthreads();
  // Hbar_k = P^H T1  ((k+1) x k), c_k = P^H s
  c128* Hk = d.Hk + (long)c * (k + 1) * k;
  for (int q = threadIdx.x; q < (k + 1) * k; q += DT) {
    const int i = q % (k + 1), j = q / (k + 1);
    c128 acc = {0, 0};
    for (int l = 0; l < ldp; ++l) acc += cmulc(P[l + (long)i * ldp], T1[l + (long)j * ldp]);
    Hk[q] = acc;
  }
  c128* ck = d.ck + (long)c * (k + 1);
  for (int i = threadIdx.x; i <= k; i += DT) {
    c128 acc = {0, 0};
    for (int l = 0; l < ldp; ++l) acc += cmulc(P[l + (long)i * ldp], s[l]);
    ck[i] = acc;
  }
  // P into the coefficient matrix (restart part of `combine`)
  c128* Cf = d.Cf + (long)c * d.ccs;
  for (int q = threadIdx.x; q < ldp * (k + 1); q += DT) {
    const int i = q % ldp, j = q / ldp;
    Cf[i + (long)j * d.ldc] = P[q];
  }
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
    harmonic_ritz(d, c, A, sh);
  }
}

__global__ void __launch_bounds__(DT) dense_d2_kernel(DenseCycle d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Sh sh;
  c128* A = reinterpret_cast<c128*>(smem_raw);
  const int c = blockIdx.y;
  ColState* st = d.st + c;
  if (!st->active) return;
  if (blockIdx.x == 0) {
    if (d.k > 0 && !st->broke && st->m_eff == d.m && st->err == 0) restart_finish(d, c, A, sh);
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
  if (phase == 0)
    harmonic_ritz(d, c, A, sh);
  else if (d.st[c].err == 0)
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

struct ProjArgs {
  int k, ns;
  const c128* Hk; const c128* cproj; const c128* sigma; const c128* beta; const int* sact;
  c128* gamma; c128* Cf; long ccs; ColState* st;
};

__global__ void __launch_bounds__(DT) dense_proj_kernel(ProjArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Sh sh;
  const int c = blockIdx.y, i = blockIdx.x;
  ColState* st = a.st + c;
  if (!st->active) return;
  const int k = a.k, ldc = k + 1;
  c128* Cf = a.Cf + (long)c * a.ccs;
  const int* sact = a.sact + (long)c * a.ns;
  if (i > 0 && !sact[i]) {
    for (int r = threadIdx.x; r <= k; r += DT) Cf[r + (long)i * ldc] = {0, 0};
    return;
  }
  c128* A = reinterpret_cast<c128*>(smem_raw);  // (k+1) x (k+1), odd leading dimension
  const int la = odd_ld(k + 1);
  c128* tau = A + (long)la * (k + 1);
  c128* d1 = tau + (k + 1);
  c128* t = d1 + (k + 1);   // (Hbar_k - sigma_1 Ibar) d_1, length k+1
  c128* y = t + (k + 1);
  const c128 s1 = a.sigma[(long)c * a.ns];
  // base: min || c - (Hbar_k - s1 Ibar) d ||
  load_shifted(A, la, a.Hk, k + 1, k + 1, k, s1);
  for (int r = threadIdx.x; r <= k; r += DT) A[r + (long)k * la] = a.cproj[(long)c * (k + 2) + r];
  if (threadIdx.x == 0) sh.ibc[0] = 0;
  __syncthreads();
  cta_qr(A, la, k + 1, k, k + 1, tau, sh, k + 1);
  for (int r = threadIdx.x; r < k; r += DT) d1[r] = A[r + (long)k * la];
  __syncthreads();
  if (!cta_backsolve(A, la, k, d1, sh)) set_err(st, GDR_EBREAKDOWN);
  for (int r = threadIdx.x; r <= k; r += DT) {
    c128 acc = {0, 0};
    for (int j = 0; j < k; ++j) {
      c128 h = a.Hk[r + (long)j * (k + 1)];
      if (r == j) h -= s1;
      acc += h * d1[j];
    }
    t[r] = acc;
  }
  __syncthreads();
  if (i == 0) {
    for (int r = threadIdx.x; r <= k; r += DT) {
      Cf[r + (long)0 * ldc] = (r < k) ? d1[r] : c128{0, 0};
      Cf[r + (long)a.ns * ldc] = -t[r];
    }
    return;
  }
  // shift i: (H_k - s_i I) d_i = beta_i (H_k - s1 I) d_1 = beta_i t[0:k]
  const c128 si = a.sigma[(long)c * a.ns + i];
  const c128 bi = a.beta[(long)c * a.ns + i];
  const int lb = odd_ld(k);
  load_shifted(A, lb, a.Hk, k + 1, k, k, si);
  for (int r = threadIdx.x; r < k; r += DT) A[r + (long)k * lb] = bi * t[r];
  if (threadIdx.x == 0) sh.ibc[0] = 0;
  __syncthreads();
  cta_qr(A, lb, k, k, k + 1, tau, sh, k);
  for (int r = threadIdx.x; r < k; r += DT) y[r] = A[r + (long)k * lb];
  __syncthreads();
  if (!cta_backsolve(A, lb, k, y, sh)) set_err(st, GDR_EBREAKDOWN);
  for (int r = threadIdx.x; r <= k; r += DT) Cf[r + (long)i * ldc] = (r < k) ? y[r] : c128{0, 0};
  // gamma_i += [beta_i t - (Hbar_k - s_i Ibar) d_i]_{k+1}  (last row of Ibar is zero)
  if (threadIdx.x == 0) {
    c128 acc = {0, 0};
    for (int j = 0; j < k; ++j) acc += a.Hk[k + (long)j * (k + 1)] * y[j];
    a.gamma[(long)c * a.ns + i] += bi * t[k] - acc;
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
  lim = std::min(lim, set_max_dyn_smem(ctx, dense_proj_kernel));
  lim = std::min(lim, set_max_dyn_smem(ctx, restart_only_kernel));
  ctx->dense_smem_limit = lim;
}

void dense_restart(gdr_ctx* ctx, const DenseCycle& d) {
  const size_t smem = dense_smem_bytes(d.m, d.k);
  GDR_REQUIRE(smem <= ctx->dense_smem_limit, "basis size m too large for the dense FP64 kernels");
  dim3 g(1, (unsigned)d.ncol);
  restart_only_kernel<<<g, DT, smem, ctx->stream>>>(d, 0);
  GDR_LAUNCHED(ctx);
  restart_only_kernel<<<g, DT, smem, ctx->stream>>>(d, 1);
  GDR_LAUNCHED(ctx);
}

void dense_cycle(gdr_ctx* ctx, const DenseCycle& d) {
  const size_t smem = dense_smem_bytes(d.m, d.k);
  GDR_REQUIRE(smem <= ctx->dense_smem_limit, "basis size m too large for the dense FP64 kernels");
  dim3 g1(d.k > 0 ? 2 : 1, (unsigned)d.ncol);
  {
    KProf kp(ctx, d.k > 0 ? "dense_ls_harmonic_ritz" : "dense_ls", 0.0);
    dense_d1_kernel<<<g1, DT, smem, ctx->stream>>>(d);
    GDR_LAUNCHED(ctx);
  }
  dim3 g2((unsigned)d.ns, (unsigned)d.ncol);
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

void dense_projection(gdr_ctx* ctx, int ncol, int k, int ns, const c128* Hk, const c128* cproj, const c128* sigma,
                      const c128* beta, const int* sact, c128* gamma, c128* Cf, long ccs, double*, long,
                      ColState* st) {
  ProjArgs a{k, ns, Hk, cproj, sigma, beta, sact, gamma, Cf, ccs, st};
  const size_t smem = sizeof(c128) * ((size_t)(k + 2) * (k + 1) + 5 * (size_t)(k + 2));
  GDR_REQUIRE(smem <= ctx->dense_smem_limit, "k too large for the projection kernel");
  dim3 g((unsigned)ns, (unsigned)ncol);
  KProf kp(ctx, "dense_projection", 0.0);
  dense_proj_kernel<<<g, DT, smem, ctx->stream>>>(a);
  GDR_LAUNCHED(ctx);
}
