// Launchers shared between the kernel files and the solver driver.
#pragma once
#include "common.cuh"

// Per-column device state of a (possibly column-batched) Arnoldi cycle.
struct ColState {
  int run;          // 1 while this cycle's vector kernels should work on the column
  int active;       // column still iterating; 0 makes every kernel skip it
  int broke;        // lucky breakdown in this cycle
  int m_eff;        // Arnoldi length of this cycle (m unless breakdown)
  int nan;          // NaN/Inf seen
  int err;          // gdr_status from a reduced solve (0 = ok)
  int conv;         // every shift of the column converged after this cycle
  int j;            // current Arnoldi column (diagnostic)
  double inv_norm;  // 1 / h_{j+1,j}, read by the scale kernel
  double bnorm;     // ||b|| of the column (relative tolerance)
  double tol;       // relative tolerance of the column
  double rnorm;     // base residual norm after this cycle (||s||)
  double wnorm0;    // ||A v_j|| of the last step (breakdown test)
  double pad2;
};

// Layout of one batched Arnoldi problem set (all device pointers).
template <typename R>
struct Batch {
  int ncol = 1;          // columns (independent Krylov spaces)
  long n = 0;
  int m = 0;             // basis size
  int ns = 1;            // shifts per column
  cx<R>* V = nullptr;    // basis, column c at V + c*vcs, vectors at stride ldv
  long ldv = 0, vcs = 0;
  cx<R>* W = nullptr;    // work vectors per column (stride wcs): W receives A v_j,
  cx<R>* W2 = nullptr;   // W2 the orthogonalised w (next step's unnormalised input)
  long wcs = 0;
  c128* H = nullptr;     // (m+1) x m per column, stride (m+1)*m
  c128* cvec = nullptr;  // m+1 per column
  c128* h1 = nullptr;    // (m+2) per column: GS dots (+ ||w||^2 in slot m+1)
  c128* h2 = nullptr;
  c128* hd = nullptr;    // DCGS2 dot values per column (2m + 8), see arnoldi_dcgs2
  c128* dc = nullptr;    // DCGS2 update coefficients per column (2m + 8)
  c64* Hf = nullptr;     // DCGS2: FP32 copy of H (same layout), for the small H s correction
  c128* part = nullptr;  // block partials, per column pstride
  long pstride = 0;
  unsigned* cnt = nullptr;  // last-block counters, per column (4 slots)
  unsigned* gcnt = nullptr; // slot-group counters of the two-level reductions, per column (64)
  ColState* st = nullptr;
  c128* sigma = nullptr;    // ns per column
  int nblk = 0;             // grid size of the reduction kernels
  const int* nvec = nullptr;  // per-column vector length (device); nullptr: all columns have length n
  int cpp = 1;                // operator problem of column c is c / cpp (CSR batch)
  int vpp = 1;                // gs_dot only: column c works on basis c / vpp (shared deflation bases)
  // host-side sums for the algorithmic byte counts of the profiler (0: n per column / per basis)
  double ntot = 0;            // the columns' vector lengths
  double vtot = 0;            // the lengths of the distinct bases gs_dot reads (vpp > 1)
};

// profiler only (gdr_profile on, graphs off): the share of the elements of `ncol` columns
// whose run flag (device, stride run_stride ints) is set, weighted by the per-column lengths
// nvec (device, may be null: equal lengths); kernels skip the other columns.  1 when the
// profiler is off.  Synchronises the stream.
double run_share(gdr_ctx* ctx, int ncol, const int* run, int run_stride, const int* nvec);
template <typename R> inline double run_share(gdr_ctx* ctx, const Batch<R>& b) {
  return run_share(ctx, b.ncol, &b.st[0].run, (int)(sizeof(ColState) / sizeof(int)), b.nvec);
}

// algorithmic element counts of a batch: all its columns, and the bases gs_dot reads
template <typename R> inline double col_len(const Batch<R>& b) { return b.ntot > 0 ? b.ntot : (double)b.n * b.ncol; }
template <typename R> inline double basis_len(const Batch<R>& b) {
  if (b.vtot > 0) return b.vtot;
  return b.vpp > 1 ? (double)b.n * ((b.ncol + b.vpp - 1) / b.vpp) : col_len(b);
}

// krylov.cu --------------------------------------------------------------
// h_out[c][0..nv-1] = V_c[:, 0:nv]^H w_c  (+ ||w_c||^2 in h_out[c][nv] if wnorm).  With wprev,
// v_{nv-1} is taken as wprev_c * inv_norm_c and stored into V on the way.
template <typename R>
void gs_dot(gdr_ctx* ctx, const Batch<R>& b, int nv, const cx<R>* w, long wcs, c128* h_out, bool wnorm,
            const cx<R>* wprev = nullptr);
// workspace of gs_dot for ncol columns sharing one basis of nv <= 48 vectors (vcs = 0), to be
// reserved before a CUDA graph capture that contains such a gs_dot
void gs_dot_shared_reserve(gdr_ctx* ctx, long n, int ncol, int nv);
// wout_c = w_c - V_c[:, 0:nv] h_c and h_out[c][0..nv-1] = V_c[:, 0:nv]^H wout_c in one pass
template <typename R>
void gs_update_dot(gdr_ctx* ctx, const Batch<R>& b, int nv, const cx<R>* w, cx<R>* wout, long wcs, const c128* h,
                   c128* h_out);
// w_c -= V_c[:, 0:nv] h_c ; if final: Arnoldi step j = nv-1 is completed (Hbar column, norm, breakdown)
template <typename R>
void gs_update(gdr_ctx* ctx, const Batch<R>& b, int nv, cx<R>* w, long wcs, const c128* h, bool final_step);
// V_c[:, j] = w_c * inv_norm_c   (skips broken / inactive columns)
template <typename R>
void scale_into(gdr_ctx* ctx, const Batch<R>& b, int j, const cx<R>* w, long wcs);
// one CGS2 Arnoldi step on every column (Hbar column j, h_{j+1,j}).  Steps after
// the first of a sweep (j > jstart) take v_j from wlast (the previous step's
// orthogonalised vector, W or W2) scaled by 1/h_{j,j-1} and store it into V in
// their first dot pass; wlast is updated to this step's vector; the last step
// (j == jlast) writes v_{j+1} into V.  Launches: matvec, dot, update+dot, update
// while the basis fits in L2, else matvec, dot, update, dot, update (+ scale at jlast).
template <typename R>
void arnoldi_step(gdr_ctx* ctx, const gdr_op* A, const Batch<R>& b, int j, int jstart, int jlast, cx<R>*& wlast);
// Arnoldi steps jstart..jend-1 of every column by classical Gram-Schmidt with delayed
// reorthogonalisation (DCGS2: per step one matvec, one dot pass and one update pass
// over the basis), then a finalising pass that writes v_jend; v_jstart must be final
// (normalised and orthogonal to v_0..v_{jstart-1}).  Needs the batch's hd / dc buffers
// and partials of (2m + 8) values per slot.
template <typename R>
void arnoldi_dcgs2(gdr_ctx* ctx, const gdr_op* A, const Batch<R>& b, int jstart, int jend);
// persistent Arnoldi sweep (sweep.cu): steps jstart..jend-1 of every column in one
// cooperative launch; v_jend is left unnormalised in W2 (scale_into writes it).
// sweep_fits: short vectors, where the sweep replaces the per-phase launches.
// sweep_reserve: its workspace, allocated before any stream capture.
template <typename R>
bool sweep_fits(gdr_ctx* ctx, const gdr_op* A, const Batch<R>& b);
template <typename R>
void sweep_reserve(gdr_ctx* ctx, const Batch<R>& b);
template <typename R>
void arnoldi_sweep(gdr_ctx* ctx, const gdr_op* A, const Batch<R>& b, int jstart, int jend);
void sweep_init(gdr_ctx* ctx);
// grid-barrier self-test (gdr_barrier_selftest)
gdr_status barrier_selftest(gdr_ctx* ctx, int rounds, int phantom);
// start a cycle from r_c: V_c[:,0] = r_c/||r_c||, cvec_c = ||r_c|| e_1, H_c = 0, state reset
template <typename R>
void start_cycle(gdr_ctx* ctx, const Batch<R>& b, const cx<R>* r, long rcs);
// out[c] = ||x_c||^2 (FP64 accumulation), x c128 or cx<R>, `cols` columns of length n at stride xcs
template <typename T>
void norms2(gdr_ctx* ctx, long n, int cols, const T* x, long xcs, double* out, c128* part, int nblk, unsigned* cnt,
            const int* nvec = nullptr);
// dots[c] = u_c^H x_c (FP64)   (ucs = 0 shares u)
void dots128(gdr_ctx* ctx, long n, int cols, const c128* u, long ucs, const c128* x, long xcs, c128* out,
             c128* part, int nblk, unsigned* cnt);

// Basis combination (restart + multi-shift update, Proj updates):
//   V_c[:, 0:nout] <- V_c[:, 0:nv] C_c[:, 0:nout]            (in place)
//   X_c[:, i]      += V_c[:, 0:nv] C_c[:, nout+i], i < nx    (X is FP64; with Xf, Xf_c[:, i]
//                     is updated instead, in the vectors' precision, same strides; nout = 0)
//   rmode 1: Rv_c = V_c C_c[:, nout+nx];  rmode 2: Rv_c += V_c C_c[:, nout+nx]
// C_c is c128 nv x (nout+nx+(rmode?1:0)), column-major with leading dim ldc, column stride ccs.
// vcs = 0 shares one basis between all columns.
template <typename R>
// lenh / vlenh: host sums of the columns' lengths / of the distinct bases' lengths for the
// profiler's byte count (0: n per column; one basis when vcs = 0)
void combine(gdr_ctx* ctx, long n, int ncol, cx<R>* V, long ldv, long vcs, int nv, const c128* C, int ldc, long ccs,
             int nout, int nx, int rmode, c128* X, long ldx, long xcs, cx<R>* Rv, long rcs, const ColState* st,
             const int* nvec = nullptr, int vpp = 1, double lenh = 0, double vlenh = 0, cx<R>* Xf = nullptr);

void krylov_init(gdr_ctx* ctx);

// tc_proj.cu: the projection dot C = V^H R over a basis shared by many complex64 columns on
// the tensor cores (TF32 inputs, FP32 accumulation): partials per (K range, column, vector)
// into part; nsplit receives the number of K ranges; prof_bytes is the algorithmic byte count
// the profiler records for the launch.  False (nothing launched) when it does not apply
// (nv > 128, no tensor-map encoder, V or R not on 16-byte boundaries or an odd stride).
void tc_proj_init(gdr_ctx* ctx);
int tc_proj_splits(gdr_ctx* ctx, long n, int ncol);
bool tc_proj_dot(gdr_ctx* ctx, long n, const c64* V, long ldv, int nv, const c64* R, long ldr, int ncol, c128* part,
                 int* err, int& nsplit, double prof_bytes);
// R += V T (rmode 2) or R = V T (rmode 1) for ncol complex64 columns over one basis V
// (nv <= 48 vectors), T's column c at C + c * ccs, on the tensor cores with split TF32
// (FP32-level accuracy); columns whose state is not active are left alone.  False
// (nothing launched) when it does not apply.
bool tc_proj_update(gdr_ctx* ctx, long n, const c64* V, long ldv, int nv, const c128* C, long ccs, int rmode, c64* R,
                    long ldr, int ncol, const ColState* st, int* err, double prof_bytes);

// conversions / small vector ops (FP64 <-> complex64)
void cvt_128_to_64(gdr_ctx* ctx, long n, int cols, const c128* in, long ics, c64* out, long ocs);
void cvt_64_to_128(gdr_ctx* ctx, long n, int cols, const c64* in, long ics, c128* out, long ocs);
void copy128(gdr_ctx* ctx, long n, int cols, const c128* in, long ics, c128* out, long ocs);
// X[:, c] += a_c * S[:, c]   (a: device c128 per column; ssc = 0 shares S)
void axpy_cols(gdr_ctx* ctx, long n, int cols, const c128* a, const c128* S, long ssc, c128* X, long xcs);
// X[:, c] *= a_c
void scal_cols(gdr_ctx* ctx, long n, int cols, const c128* a, c128* X, long xcs);

// ops.cu -----------------------------------------------------------------
// y_c = xs_c (A - sigma_c) x_c  [or b - that], skipping columns whose run flag is 0;
// xs (optional, stride xs_stride doubles) scales each column's result: the
// Arnoldi step passes 1/h_{j+1,j} and the unnormalised vector
void op_apply_skip(gdr_ctx* ctx, const gdr_op* A, int ncol, const c128* sigma, const c128* X, long ldx, c128* Y,
                   long ldy, const c128* B, long ldb, const int* run, int run_stride, int cpp = 1,
                   const double* xs = nullptr, int xs_stride = 0);
void op_apply_skip(gdr_ctx* ctx, const gdr_op* A, int ncol, const c128* sigma, const c64* X, long ldx, c64* Y,
                   long ldy, const c64* B, long ldb, const int* run, int run_stride, int cpp = 1,
                   const double* xs = nullptr, int xs_stride = 0);
// launch shape of the operator kernels for ncol columns (FP64 or complex64 vectors): the
// shape set for this column count, else the one set for the nearest count within a
// factor 2, else the defaults (Wilson: direction-split while one thread per site cannot
// fill the GPU; CSR: one thread per row; several columns of one operator in column-inner
// block order)
MvShape mv_shape(const gdr_ctx* ctx, const gdr_op* A, bool f64, int ncol);
MvShape mv_default(const gdr_ctx* ctx, const gdr_op* A, int ncol);
// Vector order: the C interface passes Wilson vectors site-major, the library keeps
// them pair-major (see wilson.cuh).  to_lib: interface -> library order, else back.
// Other operators: a plain copy (none when in == out).  in and out must differ.
template <typename T>
void op_order(gdr_ctx* ctx, const gdr_op* A, int cols, const T* in, long ldi, T* out, long ldo, bool to_lib);
// the same for Wilson vectors of V sites (c128)
template <typename T>
void wilson_order(gdr_ctx* ctx, long V, int cols, const T* in, long ldi, T* out, long ldo, bool to_lib);

// tune.cu ----------------------------------------------------------------
// x[:, c] (cols columns of n at stride ld) = counter-based uniform [-1, 1) values (timing inputs)
template <typename R>
void fill_uniform(gdr_ctx* ctx, long n, int cols, long ld, cx<R>* x, unsigned long long seed);
// gdr_autotune: the fastest matvec shape for (prec, ncol), kept on A; with m > 0 the
// Arnoldi form (sweep / per-phase launches) for (prec, ncol, m)
gdr_status tune_op(gdr_ctx* ctx, gdr_op* A, gdr_prec prec, int ncol, int m, gdr_tune_result& out);
// the tuned Arnoldi form: 1 sweep, 0 per-phase launches, -1 not tuned
int sweep_choice(const gdr_op* A, bool f64, int ncol, int m);
void op_build_csr_batch(gdr_ctx* ctx, gdr_op* op, const long* n, const long* nnz, const int* rowptr, const int* col,
                        const double* vals);
void op_build_csr(gdr_ctx* ctx, gdr_op* op, const int* rowptr, const int* col, const double* vals);
void op_build_wilson(gdr_ctx* ctx, gdr_op* op, const double* links);

// dense.cu ---------------------------------------------------------------
// Reduced solves of one cycle.  Per column c (grid.y) with m_eff from the state:
//  base: d_1 = argmin ||c - (Hbar - sigma_1 Ibar) d||, s = c - (...) d_1
//  shifts i >= 1 (active): [(Hbar - sigma_i Ibar) | s] [d_i ; beta_new] = beta_i c  via QR
//  restart (k > 0): harmonic Ritz of Hbar - sigma_1 Ibar, P_{k+1}, Hbar_k, c_k
// Coefficients for `combine` go to Cf (ldc = m+1, per column ccs): columns
//  [0, k+1) = P_{k+1} (when k > 0), [k+1, k+1+ns) = [d_i ; 0],
//  and when want_r: column k+1+ns = s (the new residual r = V_{m+1} s).
struct DenseCycle {
  int ncol, m, k, ns;
  int kfull;  // Hbar is zero below row max(j+1, kfull) in column j (k for GMRES-DR, 0 Hessenberg, m+1 dense)
  const c128* H; const c128* cvec; const c128* sigma;
  c128* beta; double* norms; int* sact;     // per column: ns each
  c128* Cf; int ldc; long ccs;              // coefficient matrices
  c128* s;                                  // (m+1) per column
  c128* Pk; c128* Hk; c128* ck;             // restart products (k>0)
  c128* theta;                              // m per column (harmonic Ritz values)
  double* scratch;                          // per column dense scratch
  long scratch_per_col;
  ColState* st;
  bool want_r;
  int hr32;  // harmonic Ritz eigensolve in FP32 (complex64 basis); FP64 when it cannot be trusted
  int fom = 0;             // FOM-Sh / FOM-DR-Sh (Sec. 3): square Galerkin solves, regular Ritz restart
  c128* graw = nullptr;    // if set: harmonic Ritz stops after the eigenvectors, G ((m+1) x k per column,
  c128* gtheta = nullptr;  // last row 0) into graw and their values (selection order) into gtheta
  int rslices = 1;         // CTAs per column that share the restart products (by columns of P_k)
  int ls32 = 0;            // complex64 basis: base least squares of a Hessenberg recurrence in FP32 + refinement
};

// Projection over selected approximate eigenvectors of a kept pair (Sec. 4, Theorem 1,
// Example 4): z_l = V_k g_l (||g_l|| = 1), eigenvalues theta_l of A, M = (G^H G)^{-1} G^H.
struct EigSel {
  const c128* G = nullptr;      // k x ks, leading dimension k + 1
  const c128* M = nullptr;      // ks x k, row-major
  const c128* theta = nullptr;  // ks
  int ks = 0;
};
// The ks 'smallest' harmonic Ritz pairs of the kept pair (Hk: device (k+1) x k, base
// shift sigma1) and M; buffers from the context workspace; res_host (ks values, may be
// null) receives the eigen-residual norms ||(Hbar_k - theta_l Ibar) g_l||.  Synchronises.
void eigsel_setup(gdr_ctx* ctx, const c128* Hk, int k, int ks, c128 sigma1, EigSel& out, double* res_host);
void dense_cycle(gdr_ctx* ctx, const DenseCycle& d);
// cycle bookkeeping after the reduced solves: convergence test, beta/active update,
// the next cycle's Hbar/c (from Hk/ck when k > 0)
void cycle_finish(gdr_ctx* ctx, const DenseCycle& d, c128* H, c128* cvec);

// Minres projection over V_k for every column (Sec. 2.3; Proj-Sh steps 3-4):
// c = V_{k+1}^H r given in cproj (stride k+2 per column), base LS on Hbar_k - sigma_1 Ibar,
// shifts: (H_k - sigma_i I) d_i = beta_i (H_k - sigma_1 I) d_1; gamma_i accumulated.
// Writes Cf (ldc = k+1): columns [0, ns) = [d_i ; 0], column ns = -(Hbar_k - sigma_1 Ibar) d_1.
// Hk: column c uses Hk + (c / hpp) * hkcs (hkcs = 0: one Hbar_k shared by all columns).
// With es (selected eigenvectors): the Theorem 1 projection instead (every column, every
// shift: d_i = beta_i (Theta - sigma_i)^{-1} M c[0:k], Cf[:, i] = [G d_i ; 0], residual
// column -(Hbar_k - sigma_1 Ibar) G d_1; gamma untouched).
// ops: the operators proj_setup formed for the same Hk, shifts and columns (unused with es).
void dense_projection(gdr_ctx* ctx, int ncol, int k, int ns, const c128* Hk, const c128* cproj, const c128* sigma,
                      const c128* beta, const int* sact, c128* gamma, c128* Cf, long ccs, const c128* ops,
                      ColState* st, long hkcs = 0, int hpp = 1, const EigSel* es = nullptr);
// The projection's solution operators for every active column (ops: ncol (ns + 1) (k+1)^2
// entries): P_1 = (Hbar_k - sigma_1 Ibar)^+, T_1 = (Hbar_k - sigma_1 Ibar) P_1 and, per
// shift i >= 1, S_i = (H_k - sigma_i I)^{-1} T_1[0:k, :] with the row g_i = T_1[k, :] -
// h_{k+1} S_i; formed once for a batch whose Hbar_k and shifts stay fixed.
void proj_setup(gdr_ctx* ctx, int ncol, int k, int ns, const c128* Hk, const c128* sigma, ColState* st, c128* ops,
                long hkcs = 0, int hpp = 1);

size_t dense_smem_bytes(int m, int k);
// harmonic Ritz restart products alone, for the s already in d.s
void dense_restart(gdr_ctx* ctx, const DenseCycle& d);
void dense_init(gdr_ctx* ctx);
