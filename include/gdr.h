/*
 * gdr.h -- C ABI of a GB300 (sm_103a) implementation of deflated multi-shift
 * GMRES: GMRES-DR(m,k)-Sh for the first right-hand side and GMRES(m_p)-Proj(k)-Sh
 * with the extra right-hand side v_{k+1} and the correction phase for the
 * others, after Darnell, Morgan and Wilcox, "Deflated GMRES for Systems with
 * Multiple Shifts and Multiple Right-Hand Sides".
 *
 * Problem (Sec. 1, eq. (1)):  (A - sigma_i I) x_i^j = b^j,  i = 1..ns, j = 1..nrhs,
 * sigma_1 (sigma[0] here) is the base shift, no preconditioning.
 *
 * Conventions for every entry point
 *  - Complex numbers are interleaved (re, im) doubles: a "c128 array of length L"
 *    is 2*L doubles.  Matrices are column-major.
 *  - Pointers are DEVICE pointers on the context's device unless the entry point
 *    says "host".  The caller owns every buffer it passes; the library owns its
 *    workspace (allocated on first use, grown on demand, freed by gdr_destroy).
 *  - Work is queued on the context's stream.  Solves synchronise that stream
 *    before returning (they read convergence words between cycles); the
 *    step-level entry points do not.
 *  - Every entry point returns a gdr_status; on error gdr_last_error() holds a
 *    one-line message.  No C++ exception crosses the ABI.  The library never
 *    falls back to host computation: without a usable CUDA device gdr_create
 *    fails with GDR_ECUDA.
 *  - Vectors of a Wilson operator use the site-major layout
 *    index = site*12 + spin*3 + color, site = ((t*Lz + z)*Ly + y)*Lx + x.
 */
#ifndef GDR_H
#define GDR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GDR_OK = 0,
  GDR_EINVAL = 1,      /* bad argument (sizes, null pointers, m > GDR_MAX_M, k >= m, ...) */
  GDR_ENOMEM = 2,      /* device allocation failed */
  GDR_ECUDA = 3,       /* a CUDA call failed; the context is unusable */
  GDR_ENOCONV = 4,     /* max_mvps / max_cycles reached before tol; X holds the last iterate */
  GDR_EBREAKDOWN = 5,  /* a singular reduced system (shift at an eigenvalue of the recurrence) */
  GDR_ENAN = 6,        /* NaN/Inf appeared in the recurrence */
  GDR_ETIMEOUT = 7,    /* a bounded device wait ran out */
  GDR_ENOTIMPL = 8
} gdr_status;

/* Arithmetic of the bulk vectors.  FP64: complex128 everywhere.  MIXED: matvec,
 * Gram-Schmidt and basis updates in complex64 (FP32 accumulation), small dense
 * steps, solutions and true residuals in FP64, with iterative refinement. */
typedef enum { GDR_PREC_FP64 = 0, GDR_PREC_MIXED = 1 } gdr_prec;

/* Storage of Wilson gauge links used by the complex64 matvec (the FP64
 * residuals always use the complex128 links given at creation). */
typedef enum { GDR_LINK_C128 = 0, GDR_LINK_C64 = 1, GDR_LINK_BF16 = 2 } gdr_link_fmt;

#define GDR_MAX_M 96            /* largest basis size m (and m_proj) */

/* gdr_params.flags */
#define GDR_FLAG_HOST_PTRS    1u  /* B and X of a solve are HOST pointers; copies are made inside */
#define GDR_FLAG_NO_GRAPH     2u  /* launch every kernel directly instead of replaying CUDA graphs */
#define GDR_FLAG_SEQUENTIAL   4u  /* right-hand sides 2.. one at a time (no column batching) */
#define GDR_FLAG_NO_PROJ      8u  /* later right-hand sides by plain GMRES(m_p)-Sh (no deflation) */
#define GDR_FLAG_NO_REFINE   16u  /* no refinement / cleanup after the stages (residuals still reported) */
#define GDR_FLAG_NO_SWEEP    32u  /* short vectors: one launch per Arnoldi phase instead of the persistent
                                     per-cycle sweep kernel */
#define GDR_FLAG_FP64_EIG    64u  /* MIXED: harmonic-Ritz eigensolve in FP64 instead of FP32 */
#define GDR_FLAG_RELATED_RHS 256u /* related right-hand sides (Sec. 5, Example 8): RHS 2.. one at a time,
                                     each started from the Minres projection over the converged solutions
                                     of the previous ones (B^H B d = B^H b_j, x_i = X_i d, common residual
                                     b_j - B d), then GMRES(m_p)-Proj(k)-Sh + correction on that residual
                                     and refinement to tol before the next */
#define GDR_FLAG_EIG_SELECT  512u /* right-hand sides 2.. by GMRES(m_p)-Proj-Sh projecting over the first
                                     k_select approximate eigenvectors of the kept pair (harmonic Ritz
                                     vectors of smallest |theta - sigma_1|) as in Theorem 1 (Sec. 4,
                                     Example 4), instead of the Minres projection over V_k with the extra
                                     right-hand side and the correction phase */
#define GDR_FLAG_FOM        1024u /* right-hand side 1 (and every problem of a batch) by FOM(m)-Sh (k = 0)
                                     or FOM-DR(m,k)-Sh (Sec. 3, Examples 2-3): square Galerkin solves for
                                     every shift (residuals parallel by construction) and a restart with
                                     regular Ritz vectors; later stages unchanged */
#define GDR_FLAG_CGS2      2048u /* MIXED: Arnoldi steps of the complex64 stages (outside the persistent
                                     sweep) by classical Gram-Schmidt twice, four passes over the basis
                                     per step, instead of the default delayed reorthogonalisation (DCGS2:
                                     the second pass of step j merged into the projection of step j+1,
                                     two passes per step); the FP64 stages always use the former */
#define GDR_FLAG_FP64_DENSE 4096u /* MIXED: every small dense step in FP64 -- the harmonic-Ritz eigensolve
                                     (as GDR_FLAG_FP64_EIG) and the reduced least squares of the GMRES(m_p)
                                     cycles of the Proj and refinement stages (default: FP32 Givens QR with
                                     one FP64-residual refinement step, the FP64 form when that step's
                                     correction exceeds 1e-4 of the solution) */
#define GDR_FLAG_NO_TENSOR_CORES 8192u /* MIXED: the projection dot of the Proj and refinement batches over
                                     the shared kept basis on the CUDA cores (FP32) instead of the tensor
                                     cores (TF32, tcgen05) */
#define GDR_FLAG_AUTOTUNE   128u  /* before the first cycle, run gdr_autotune for the matvec and Arnoldi
                                     form of each stage whose (precision, columns, m) the operator has
                                     no tuned shape for yet (the tuning time is part of the solve) */

typedef struct gdr_ctx gdr_ctx;
typedef struct gdr_op gdr_op;
typedef struct gdr_defl gdr_defl;

typedef struct {
  int m;              /* GMRES-DR basis size (first right-hand side) */
  int k;              /* harmonic Ritz vectors kept across restarts, 0 < k < m */
  int m_proj;         /* GMRES cycle length in the Proj phase (0: m - k) */
  double tol;         /* relative residual target ||b - (A - sigma_i I) x|| / ||b|| */
  double extra_tol;   /* relative tolerance for the extra right-hand side v_{k+1} */
  double inner_tol;   /* MIXED: relative residual of the complex64 GMRES-DR / Proj stages before FP64
                         refinement; <= 0 chooses it: 1e-3 when the complex64 basis fits in half of
                         the L2 cache (cycles limited by the FP64 dense steps), else 1e-4 with bf16
                         Wilson links, 1e-6 for a CSR batch, 3e-7 otherwise */
  double refine_tol;  /* MIXED: floor of the relative reduction asked of one complex64 refinement pass
                         (its target is max(0.3 tol ||b|| / ||r||, refine_tol)); <= 0 chooses
                         2e-4 with bf16 Wilson links when the basis does not fit in half of L2,
                         else min(inner_tol, 1e-4) */
  long max_mvps;      /* cap on Arnoldi matvecs per solve stage (per column) */
  int max_cycles;     /* 0: unlimited; else stop RHS 1 after this many cycles */
  int refine_max;     /* MIXED: refinement passes before the FP64 cleanup */
  gdr_prec prec;
  unsigned flags;
  int k_select;       /* GDR_FLAG_EIG_SELECT: approximate eigenvectors projected over (1..k; <= 0: k) */
  int m_refine;       /* cycle length of the refinement / cleanup solves (not in the paper); <= 0:
                         min(m, m_p + (m - m_p) / 2) for vectors of at most 2^17 elements, else
                         min(m_p, 6) with bf16 Wilson links, min(m_p, 8) otherwise */
  double refine_rank_tol; /* MIXED, shift-shared refinement (not in the paper; off when <= 0, the
                         default): a complex64 refinement pass may refine the residuals of one
                         right-hand side's shifts over a few orthonormal directions of their span
                         (pivoted Cholesky of their Gram matrix, directions kept while the rest
                         exceeds refine_rank_tol times the largest residual), each direction one
                         multi-shift GMRES(m_refine)-Proj(k)-Sh column for all shifts, followed by the
                         extra-right-hand-side correction; used when that needs at most 0.7 times the
                         columns of per-pair refinement and the Proj stage's extra solutions exist
                         (nrhs > 1).  Off by default: on the bf16-link 24^3x32 workload it took more
                         matvecs than per-pair refinement (its non-base shifts converge slowly in
                         short restarted cycles) */
} gdr_params;

typedef struct {
  long mvps_rhs1;       /* Arnoldi matvecs, first right-hand side (m + (cycles-1)(m-k)) */
  long cycles_rhs1;
  long mvps_extra;      /* matvecs spent on the extra right-hand side v_{k+1} */
  long mvps_proj;       /* matvecs of the Proj phase, summed over right-hand sides 2.. */
  long mvps_refine;     /* matvecs of refinement / cleanup solves, summed over columns */
  long resid_cols;      /* FP64 true-residual matvec columns */
  int refine_passes;
  int pairs_cleaned;    /* (shift, rhs) pairs finished by the FP64 cleanup */
  double max_relres;    /* max over (shift, rhs) of the final FP64 true relative residual */
  double t_total_ms;    /* wall time of the solve */
  long kernel_launches; /* kernels of this library launched by the solve (graph nodes counted) */
  double t_rhs1_ms;     /* wall time of the GMRES-DR(m,k)-Sh stage (right-hand side 1) */
  double t_proj_ms;     /* extra right-hand side, Proj stage and corrections (GDR_FLAG_RELATED_RHS:
                           everything after right-hand side 1, its refinement included) */
  double t_refine_ms;   /* FP64 true residuals, refinement passes and FP64 cleanup */
  long host_syncs;      /* host waits on the stream (one per cycle for the convergence test, ...) */
  double related_resid; /* GDR_FLAG_RELATED_RHS: largest ||b_j - B d|| / ||b_j|| over j >= 2 (else 0) */
  double eig_resid_max; /* GDR_FLAG_EIG_SELECT: largest eigen-residual ||A z - theta z|| (||z|| = 1)
                           of the selected approximate eigenvectors (else 0) */
  long shared_cols;     /* multi-shift columns of the shift-shared refinement passes (summed) */
  long shared_pairs;    /* (shift, rhs) pairs those passes refined (summed); per-pair passes would
                           have used one column each */
  long mvps_shared;     /* matvecs of the shift-shared passes (part of mvps_refine) */
} gdr_report;

/* ---------------------------------------------------------------- context */

void gdr_params_default(gdr_params *p);

/* Create a context on `device`; `cuda_stream` is a cudaStream_t (NULL: the
 * legacy default stream).  Fails with GDR_ECUDA when no device is usable. */
gdr_status gdr_create(gdr_ctx **ctx, int device, void *cuda_stream);
void gdr_destroy(gdr_ctx *ctx);
const char *gdr_last_error(const gdr_ctx *ctx);
const char *gdr_status_string(gdr_status s);

/* --------------------------------------------------------------- operators
 * A is n x n.  The operator keeps its own device copies (and complex64 /
 * bfloat16 copies for the MIXED path), so the caller's arrays may be freed
 * after creation returns (the stream is synchronised). */

/* CSR (Examples 1-6, Sec. 3-4): int32 rowptr[n+1], int32 col[nnz], c128 vals[nnz]. */
gdr_status gdr_op_csr(gdr_ctx *ctx, long n, long nnz, const int *rowptr, const int *col,
                      const double *vals, gdr_op **out);

/* Wilson-Dirac-style matrix (Example 7, Sec. 4): A = diag_a I - H with
 * (H psi)(x) = sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu)],
 * periodic, chiral gamma basis (gamma_k = [[0,-i s_k],[i s_k,0]], gamma_t = [[0,I],[I,0]]).
 * dims = {Lx, Ly, Lz, Lt} (each >= 2); links: c128 [4][V][3][3], U_mu(x)_{ab}
 * row-major, mu = x,y,z,t.  `store` picks the link storage of the complex64 matvec. */
gdr_status gdr_op_wilson(gdr_ctx *ctx, const int dims[4], double diag_a, const double *links,
                         gdr_link_fmt store, gdr_op **out);
/* A batch of independent CSR matrices (the uneven-size problems solved together by
 * gdr_solve_batch).  Problem p has n[p] rows and nnz[p] entries; rowptr, col and vals
 * are the problems' CSR arrays concatenated (device): problem p's n[p]+1 row pointers
 * (local, starting at 0), then its column indices (local) and c128 values.  n, nnz: host. */
gdr_status gdr_op_csr_batch(gdr_ctx *ctx, int nprob, const long *n, const long *nnz, const int *rowptr,
                            const int *col, const double *vals, gdr_op **out);
void gdr_op_destroy(gdr_op *op);
long gdr_op_n(const gdr_op *op);

/* Matvec (step a1 / a2): Y[:,c] = (A - sigma_c I) X[:,c], c < ncol, in the
 * precision `prec` (FP64: X, Y are c128; MIXED: X, Y are complex64, interleaved
 * floats).  sigma: host c128[ncol].  Leading dimension n.  Asynchronous. */
gdr_status gdr_op_apply(gdr_ctx *ctx, const gdr_op *A, gdr_prec prec, int ncol, const double *sigma,
                        const void *X, void *Y);

/* ------------------------------------------------------------- autotuning
 * The paper fixes the algorithm, not a kernel layout; these calls choose, by
 * timing on the device, how the same arithmetic is launched (the result changes
 * at most in the summation order of a CSR row or of the four hop directions).
 * A matvec shape belongs to an operator and one (vector precision, column
 * count); a matvec of another count uses the shape of the nearest tuned count
 * within a factor 2, else the defaults.  Shapes are not shared between
 * operators and are lost with gdr_op_destroy. */
typedef struct {
  int form;       /* Wilson: 0 one thread per site, 1 direction-split (a warp per direction,
                     32 sites per block), 2 one thread per site and column pair with packed
                     FP32x2 arithmetic (complex64 only; an odd last column is paired with itself).
                     CSR: threads per row, 1, 2, 4 or 8 */
  int threads;    /* threads per block: 64, 128 or 256 (direction-split: 128; pairs: 64 or 128) */
  int col_inner;  /* 1: consecutive blocks take one site/row tile for consecutive columns
                     (links / rows read from HBM once for all columns); g >= 2 (at most
                     65535): that order within groups of g columns (column pairs in form 2),
                     the groups one after another (links read once per group, the group's
                     vectors still in L2 when a neighbour plane reuses them); 0: column-major
                     grid.  GDR_EINVAL for a negative value */
} gdr_shape;

typedef struct {
  gdr_shape best;          /* the matvec shape kept (now in effect for this precision and count) */
  double mv_ms;            /* its time per launch, all columns */
  double mv_ms_default;    /* the default shape's time per launch */
  int candidates;          /* matvec shapes timed */
  int sweep;               /* Arnoldi form kept: 1 persistent sweep, 0 per-phase launches,
                              -1 not tuned (m = 0, or the sweep does not apply to this shape) */
  double cycle_ms_sweep;   /* one Arnoldi pass of m steps on ncol columns, each form, replayed */
  double cycle_ms_launch;  /*   from CUDA graphs (0 when not timed) */
} gdr_tune_result;

/* Time every candidate matvec shape for `ncol` columns of `prec` vectors on A
 * (library scratch vectors with counter-based random entries, about 20 ms of
 * launches per candidate) and keep the fastest on A.  With m > 0, also time one
 * Arnoldi pass of m steps on ncol columns (random start vectors) as the
 * persistent sweep and as one launch per phase, where the sweep applies (short
 * vectors whose bases fit in half of L2), and keep the faster for solves whose
 * stage has these (prec, ncol, m).  For a CSR batch, ncol must be a positive
 * multiple of the problem count (column c belongs to problem c / (ncol/nprob)).
 * out may be NULL.  Synchronises the context stream. */
gdr_status gdr_autotune(gdr_ctx *ctx, gdr_op *A, gdr_prec prec, int ncol, int m, gdr_tune_result *out);

/* Set the matvec shape of A for (prec, ncol) (shape != NULL; validated: a form
 * and thread count listed above), or forget it (shape == NULL; ncol <= 0
 * forgets every shape and Arnoldi choice of A). */
gdr_status gdr_op_set_shape(gdr_op *A, gdr_prec prec, int ncol, const gdr_shape *shape);

/* The shape a matvec of ncol `prec` columns on A launches with now. */
gdr_status gdr_op_get_shape(const gdr_op *A, gdr_prec prec, int ncol, gdr_shape *out);

/* ------------------------------------------------------------------ solves */

/* All shifts of all right-hand sides (Sec. 3 and Sec. 4, Example 5 order):
 * RHS 1 by GMRES-DR(m,k)-Sh, then (nrhs > 1) the extra right-hand side v_{k+1}
 * and RHS 2..nrhs by GMRES(m_p)-Proj(k)-Sh (column-batched unless
 * GDR_FLAG_SEQUENTIAL), then the correction x_i^j += (v_{k+1}^H r_i^j) s_i.
 * MIXED adds FP64 true residuals and refinement / FP64 cleanup per pair.
 * sigma: host c128[ns], sigma[0] the base shift.  B: c128 n x nrhs.
 * X: c128 n x ns x nrhs (X[:, i, j] solves shift i, rhs j), written.
 * defl_out (optional): receives the kept pair A V_k = V_{k+1} Hbar_k (eq. recur1).
 * report (optional, host).  Returns GDR_ENOCONV when a pair missed tol. */
gdr_status gdr_solve_multishift(gdr_ctx *ctx, const gdr_op *A, int ns, const double *sigma, int nrhs,
                                const double *B, double *X, const gdr_params *params,
                                gdr_defl **defl_out, gdr_report *report);

/* Many independent shifted problems (eq. (1) with nrhs = 1 each) solved together:
 * every problem runs GMRES-DR(m,k)-Sh as one column of a batched cycle (one kernel
 * sequence / CUDA graph per cycle for the whole batch), then FP64 true residuals and
 * per-pair refinement / cleanup as in gdr_solve_multishift.  A from gdr_op_csr_batch.
 * sigma: host c128 [nprob x ns], problem p's shifts at sigma[p*ns], sigma[p*ns] its
 * base shift.  B: c128, problem p's right-hand side at offset sum_{q<p} n[q].
 * X: c128, problem p's n[p] x ns solutions (column-major) at offset ns * sum_{q<p} n[q].
 * status (optional, host int[nprob]): GDR_OK or GDR_ENOCONV per problem. */
gdr_status gdr_solve_batch(gdr_ctx *ctx, const gdr_op *A, int ns, const double *sigma, const double *B, double *X,
                           const gdr_params *params, gdr_report *report, int *status);

/* GMRES(m_p)-Proj(k)-Sh with a kept deflation space (Sec. 4), without the
 * correction phase: X[:, i, j] with residuals beta_i r + g_i v_{k+1}.  With
 * GDR_FLAG_EIG_SELECT: over the first k_select approximate eigenvectors of the
 * kept pair (Theorem 1) instead; the report's eig_resid_max is then set.
 * Same argument conventions as gdr_solve_multishift. */
gdr_status gdr_solve_proj(gdr_ctx *ctx, const gdr_op *A, const gdr_defl *defl, int ns, const double *sigma,
                          int nrhs, const double *B, double *X, const gdr_params *params, gdr_report *report);

/* Copy the kept pair out: V (device c128 n x (k+1)) and Hbar (HOST c128
 * (k+1) x k, column-major).  Either may be NULL.  *k_out receives k. */
gdr_status gdr_defl_export(gdr_ctx *ctx, const gdr_defl *defl, double *V, double *Hbar, int *k_out);
void gdr_defl_destroy(gdr_defl *defl);

/* Per-kernel timing.  gdr_profile(ctx, 1) clears the counters and makes every
 * later launch of the context bracketed by CUDA events on its stream (CUDA graphs
 * are not used while it is on); gdr_profile(ctx, 0) switches it off.
 * gdr_profile_report writes a JSON object {kernel: {"launches", "ms", "bytes"}} into
 * buf (len bytes, NUL-terminated), "bytes" being the algorithmic bytes the launches
 * move (0 for the dense FP64 kernels); it synchronises the stream. */
gdr_status gdr_profile(gdr_ctx *ctx, int enable);

/* Failure-detection self-test of the grid barrier used by the persistent
 * Arnoldi sweep (no counterpart in the paper).  Launches `rounds` (>= 1) grid
 * barriers over a cooperative grid.  phantom = 0: every barrier completes,
 * GDR_OK.  phantom = 1: each barrier waits for one block more than the grid
 * has, so the first one ends only by its spin bound (about one second); the
 * kernel then returns normally and the call reports GDR_ETIMEOUT, leaving the
 * context usable.  Synchronises the context stream. */
gdr_status gdr_barrier_selftest(gdr_ctx *ctx, int rounds, int phantom);
gdr_status gdr_profile_report(gdr_ctx *ctx, char *buf, long len);

/* --------------------------------------------------------- step-level calls
 * Single steps of the cycle, exposed for parity checks and benchmarks.  All
 * asynchronous on the context stream; FP64 unless `prec` says otherwise. */

/* Arnoldi step with classical Gram-Schmidt twice (eq. recurAr): with V holding
 * v_0..v_j (n x (j+2) buffer, leading dimension n, vectors in `prec`), compute
 * w = A v_j, h = V_{j+1}^H w twice, v_{j+1} = w / ||w|| into V[:, j+1] and the
 * FP64 column h (c128[j+2]: h_0..h_j, h_{j+1,j}) into `hcol`. */
gdr_status gdr_arnoldi_step(gdr_ctx *ctx, const gdr_op *A, gdr_prec prec, void *V, int j, double *hcol);

/* Arnoldi steps j0..m-1 of A V_m = V_{m+1} Hbar_m (eq. recurAr), continuing, when
 * j0 > 0, from a kept pair A V_{j0} = V_{j0+1} Hbar_{j0} as after a GMRES-DR restart
 * (eq. recur1), in the form the solves use: FP64 by classical Gram-Schmidt twice per
 * step; MIXED in complex64 by Gram-Schmidt with delayed reorthogonalisation (the
 * second pass of step j merged into the projection of step j+1, then a finalising
 * pass for v_m), or twice per step with GDR_FLAG_CGS2 in `flags`.
 * V: n x (m+1), `prec` vectors, leading dimension n; columns 0..j0 given (orthonormal),
 * columns j0+1..m written.  Hbar: c128 (m+1) x m, column-major, device; columns
 * 0..j0-1 given (rows 0..j0), columns j0..m-1 written with zeros below row j+1.
 * m_eff (host, may be NULL): m, or j+1 after a lucky breakdown at step j
 * (h_{j+1,j} <= 1e-12 ||A v_j||; the later columns of V are then zero and those of
 * Hbar unspecified).  GDR_ENAN on a
 * non-finite value.  Synchronises the context stream. */
gdr_status gdr_arnoldi_cycle(gdr_ctx *ctx, const gdr_op *A, gdr_prec prec, void *V, int j0, int m, double *Hbar,
                             unsigned flags, int *m_eff);

/* GMRES-Sh reduced solve (Sec. 2.1, eqs. gsh1-gsh3; GMRES-DR-Sh steps 3-5), FP64:
 * Hbar: c128 (m+1) x m, c: c128[m+1], sigma: host c128[ns], beta: c128[ns] in.
 * Out: D c128 m x ns, s c128[m+1], beta_new c128[ns], norms double[ns]
 * (norms[0] = ||s||, norms[i] = |beta_new_i| ||s||). */
gdr_status gdr_dense_gmres_sh(gdr_ctx *ctx, int m, int ns, const double *Hbar, const double *c,
                              const double *sigma, const double *beta, double *D, double *s,
                              double *beta_new, double *norms);

/* Allocation-free form of gdr_dense_gmres_sh, with the same arguments and
 * results.  The paper has no counterpart of this call: it exists for callers
 * that cannot let the library allocate device memory (code running under an
 * allocator it does not control, such as a host framework's memory pool or a
 * fixed device-memory budget, or a latency-critical loop where cudaMalloc and
 * cudaFree would synchronise the device).  Its workspace is one fixed array
 * in the library's device image (about 180 KB, present on every device that
 * loads the library until the process exits), so it never calls cudaMalloc,
 * cudaFree or an allocating library routine.  Limits: m <= GDR_NOALLOC_MAX_M,
 * ns <= GDR_NOALLOC_MAX_NS; larger sizes return GDR_EINVAL.  The first call on
 * a device looks up the array's device address, so make it before any stream
 * capture; with CUDA's lazy module loading (the default) that first call is also
 * when the array's memory is committed, so a caller with a fixed memory budget
 * should make one call while setting up.  All calls share the one array, which keeps the last call's
 * contents: calls that overlap on the GPU race and must be serialised by the
 * caller.  Synchronises the context stream before returning. */
#define GDR_NOALLOC_MAX_M 96
#define GDR_NOALLOC_MAX_NS 16
gdr_status gdr_dense_gmres_sh_noalloc(gdr_ctx *ctx, int m, int ns, const double *Hbar, const double *c,
                                      const double *sigma, const double *beta, double *D, double *s,
                                      double *beta_new, double *norms);

/* Base least squares of a GMRES cycle (Sec. 2.1: the base system of eqs. gsh1-gsh2,
 * GMRES-DR-Sh step 3): y = argmin || c - (Hbar - sigma1 Ibar) y || for an upper
 * Hessenberg Hbar (c128 (m+1) x m, column-major, zero below the subdiagonal),
 * c: c128[m+1], sigma1: host c128.  Out (device): y c128[m], s = c - (Hbar - sigma1 Ibar) y
 * c128[m+1], formed in FP64.  FP64: Givens QR in FP64.  MIXED: the form of the complex64
 * GMRES(m_p) cycles -- FP32 Givens QR, back substitution and one refinement step with
 * the FP64 residual (y then accurate to about the correction's size, ||s|| within ~1e-9
 * of the minimum); when the correction exceeds 1e-4 ||y|| or a pivot is zero, the FP64
 * form instead.  GDR_EBREAKDOWN on a singular system.
 * Synchronises the context stream. */
gdr_status gdr_dense_ls(gdr_ctx *ctx, gdr_prec prec, int m, const double *sigma1, const double *Hbar,
                        const double *c, double *y, double *s);

/* GMRES-DR restart (Sec. 2.2): harmonic Ritz pairs of Hhat = Hbar - sigma1 Ibar,
 * k of smallest |theta| (ties: larger Im, then larger Re), P_{k+1} = [orth([G;0]), p],
 * p from s; Hk = P^H Hbar P_k ((k+1) x k), ck = P^H s (k+1).
 * prec GDR_PREC_FP64: the eigensolve in FP64.  GDR_PREC_MIXED: the form the
 * solver uses with a complex64 basis -- f refined to FP64 accuracy, the
 * Hessenberg reduction, QR iteration, eigenvectors and the orthonormalisation of
 * P_k in FP32 (P_k orthonormal to ~1e-7, theta to FP32 accuracy), falling back
 * to FP64 where FP32 does not suffice; p, Hk and ck in FP64.
 * In: Hbar c128 (m+1) x m, s c128[m+1], sigma1 host c128.  Out: theta c128[m]
 * (all harmonic Ritz values, unordered), P c128 (m+1) x (k+1), Hk, ck. */
gdr_status gdr_dense_restart(gdr_ctx *ctx, gdr_prec prec, int m, int k, const double *sigma1,
                             const double *Hbar, const double *s, double *theta, double *P, double *Hk,
                             double *ck);

/* Basis update (restart, eq. recur1, fused with the multi-shift update):
 * V (n x nv, `prec`) times coefficients C (c128 nv x (nout + nx)):
 * V[:, 0:nout] <- V C[:, 0:nout]  (in place, nout <= nv) and
 * X[:, i] += V C[:, nout + i] for i < nx (X c128 n x nx). */
gdr_status gdr_basis_update(gdr_ctx *ctx, gdr_prec prec, long n, int nv, void *V, const double *C, int nout,
                            int nx, double *X);

/* Projection dot (Sec. 2.3, GMRES-Proj-Sh step 4: c = V_{k+1}^H r for every
 * column): C[c*nv + i] = v_i^H r_c for the nv vectors of one basis V and ncol
 * columns R.  V: n x nv (`prec`: complex64 for GDR_PREC_MIXED, complex128 for
 * GDR_PREC_FP64), column-major with stride n; R: n x ncol of the same type,
 * column stride ldr >= n; C: c128 nv x ncol (all device).  nv <= GDR_MAX_M + 1.
 * The complex64 form with ncol >= 8 runs on the tensor cores (TF32 inputs,
 * FP32 accumulation: each dot to about 1e-3 of ||v_i|| ||r_c||) when R and V
 * start on 16-byte boundaries, n and ldr are even and nv <= 128, unless flags has
 * GDR_FLAG_NO_TENSOR_CORES; otherwise the CUDA cores form it (FP32 products,
 * FP64 sums).  GDR_ETIMEOUT if a tensor-core wait gave up (C unspecified). */
gdr_status gdr_basis_dot(gdr_ctx *ctx, gdr_prec prec, long n, int nv, const void *V, int ncol, const void *R,
                         long ldr, double *C, unsigned flags);

/* Residual update of the projection (Sec. 2.3, GMRES-Proj-Sh step 4:
 * r_c <- r_c - V_{k+1} (Hbar_k - sigma_1 Ibar) d_c for every column c, with
 * T[:, c] = -(Hbar_k - sigma_1 Ibar) d_c formed by the caller):
 * R[:, c] += V T[:, c] for the nv vectors of one basis V and ncol columns.
 * V: n x nv (`prec`: complex64 for GDR_PREC_MIXED, complex128 for
 * GDR_PREC_FP64), column-major with stride n; T: c128 nv x ncol, column c at
 * T + c*nv; R: n x ncol of V's type, column stride ldr >= n (all device).
 * nv <= GDR_MAX_M + 1.  The complex64 form with ncol >= 8 and nv <= 48 runs
 * on the tensor cores with V and T split into two TF32 parts each (three
 * products, FP32 accumulation: the accuracy of FP32 arithmetic), unless flags
 * has GDR_FLAG_NO_TENSOR_CORES; otherwise the CUDA cores form it in FP32
 * (complex64) or FP64.  GDR_ETIMEOUT if a tensor-core wait gave up (R then
 * unspecified). */
gdr_status gdr_basis_residual_update(gdr_ctx *ctx, gdr_prec prec, long n, int nv, const void *V, int ncol,
                                     const double *T, void *R, long ldr, unsigned flags);

#ifdef __cplusplus
}
#endif
#endif /* GDR_H */
