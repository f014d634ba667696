// Solver driver interfaces (host side).
#pragma once
#include <vector>

#include "kernels.cuh"

// One GMRES-DR(m,k)-Sh run on a batch of columns (independent Krylov spaces in lockstep).
template <typename R>
struct DrJob {
  int ncol = 1, ns = 1, m = 0, k = 0;
  const cx<R>* rhs = nullptr;  // column c at rhs + c*ldrhs
  long ldrhs = 0;
  std::vector<c128> sigma;     // ncol x ns, sigma[c*ns] the base shift of column c
  std::vector<double> tol;     // relative tolerance per column
  const int* nvec = nullptr;   // per-column vector length (device), nullptr: all A->n
  int cpp = 1;                 // operator problem of column c is c / cpp
  c128* X = nullptr;           // X + c*xcs + i*ldx accumulates shift i of column c (FP64)
  long ldx = 0, xcs = 0;
  long max_mvps = 100000;
  int max_cycles = 0;
  bool sweep = true;           // persistent Arnoldi sweep where it fits (sweep_fits)
  bool eig32 = true;           // complex64 basis: harmonic-Ritz eigensolve in FP32
  bool fom = false;            // FOM-Sh / FOM-DR-Sh instead of GMRES-Sh / GMRES-DR-Sh (Sec. 3)
  bool dcgs2 = true;           // complex64 launches: delayed reorthogonalisation (else CGS2)
};

struct DrResult {
  gdr_status status = GDR_OK;
  long mvps = 0;
  long cycles = 0;
  int k_eff = 0;
  bool broke = false;
  bool valid_defl = false;
  void* V = nullptr;       // basis buffer (vector precision); V[:, 0:k+1] is the kept V_{k+1}
  long ldv = 0;
  long vcs = 0;            // stride between the columns' bases
  bool any_broke = false;  // some column had a lucky breakdown (no kept pair for it)
  c128* Hk = nullptr;      // kept Hbar_k ((k+1) x k) on the device
  std::vector<double> norms;
  std::vector<long> col_mvps;  // per column
  std::vector<int> col_conv;
};

// A batch of columns for GMRES(m_p)-Proj(k)-Sh.
template <typename R>
struct ProjJob {
  int ncol = 0, ns = 1, m_p = 0, k = 0;
  bool project = true;
  const cx<R>* Vd = nullptr;   // kept V_{k+1} (n x (k+1), ld ldvd), shared by all columns
  long ldvd = 0;
  const c128* Hk = nullptr;    // kept Hbar_k ((k+1) x k)
  long vdcs = 0, hkcs = 0;     // strides between per-problem kept pairs (0: one pair shared by all)
  int dpp = 1;                 // column c uses kept pair c / dpp
  const cx<R>* rhs = nullptr;  // right-hand sides, column c at rhs + c*ldrhs
  long ldrhs = 0;
  std::vector<c128> sigma;     // ncol x ns, sigma[c*ns] the base shift of column c
  std::vector<double> tol;     // relative tolerance per column
  std::vector<int> mask;       // columns to solve (empty: all)
  const int* nvec = nullptr;   // per-column vector length (device), nullptr: all A->n
  int cpp = 1;                 // operator problem of column c is c / cpp
  c128* X = nullptr;           // X + c*xcs + i*ldx accumulates shift i of column c (FP64)
  long ldx = 0, xcs = 0;
  long max_mvps = 100000;
  bool sweep = true;           // persistent Arnoldi sweep where it fits (sweep_fits)
  const EigSel* eigsel = nullptr;  // project over selected approximate eigenvectors instead (Theorem 1)
  bool dcgs2 = true;           // complex64 launches: delayed reorthogonalisation (else CGS2)
  bool ls32 = true;            // complex64 basis: FP32 least squares + FP64-residual refinement step
};

struct ProjResult {
  gdr_status status = GDR_OK;
  long cycles = 0;
  std::vector<long> mvps;
  std::vector<int> converged;
  std::vector<c128> gamma;     // accumulated gamma_i per column (eq. keyder2), diagnostic
};

// Time one Arnoldi pass of m steps on ncol columns of A (random start vectors) as the
// persistent sweep and as per-phase launches, each replayed from a CUDA graph.
// choice: 1 sweep faster, 0 launches faster, -1 the sweep does not fit (not timed).
template <typename R>
void tune_arnoldi(gdr_ctx* ctx, const gdr_op* A, int ncol, int m, double& t_sweep, double& t_launch, int& choice);

template <typename R>
DrResult dr_sh(gdr_ctx* ctx, const gdr_op* A, const DrJob<R>& job, bool use_graph);

// Independent problems of a CSR batch, one right-hand side each (all with ns shifts).
template <typename R>
gdr_status solve_batch_pipeline(gdr_ctx* ctx, const gdr_op* A, int ns, const std::vector<c128>& sigma,
                                const c128* B, c128* X, const gdr_params& p, gdr_report& rep, int* prob_status);

template <typename R>
ProjResult proj_batch(gdr_ctx* ctx, const gdr_op* A, const ProjJob<R>& job, bool use_graph);

void true_residuals(gdr_ctx* ctx, const gdr_op* A, int ns, const c128* sigma_dev, int nrhs, const c128* B, long ldb,
                    const c128* X, long ldx, c128* R, long ldr, std::vector<double>& relres,
                    const std::vector<double>& bnorm, const std::vector<int>* only = nullptr);

template <typename R>
gdr_status solve_pipeline(gdr_ctx* ctx, const gdr_op* A, const std::vector<c128>& sigma, int nrhs, const c128* B,
                          long ldb, c128* X, long ldx, const gdr_params& p, gdr_defl** defl_out, gdr_report& rep);

