// Autotuner of the operator launch shapes and of the Arnoldi form.
//
// The paper fixes the algorithm, not a kernel design.  What is tuned here is only
// how the same arithmetic is laid onto the GPU:
//  * the matvec (Wilson stencil or CSR): one thread per site or the
//    direction-split form, threads per block, threads per CSR row (the vector
//    width of the row loop), and whether consecutive blocks walk the columns of
//    one tile (links and rows shared through L2) or the tiles of one column;
//  * the Arnoldi pass of short vectors: the persistent sweep kernel or one
//    launch per phase (both replayed as CUDA graphs, as the solver runs them).
// Every candidate computes the same result (up to the summation order of a CSR
// row or of the four hop directions); the fastest measured one is kept on the
// operator for its (vector precision, column count).
#include <cmath>
#include <type_traits>

#include "kernels.cuh"
#include "solver.cuh"

namespace {

// counter-based timing inputs: splitmix64 of (seed, element) -> uniform [-1, 1)
HD unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename R>
__global__ void fill_kernel(long n, long ld, cx<R>* x, unsigned long long seed) {
  const int c = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const unsigned long long h = splitmix64(seed ^ ((unsigned long long)c << 40) ^ (unsigned long long)i);
    const R a = (R)((double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    const R b = (R)((double)(splitmix64(h) >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    x[c * ld + i] = {a, b};
  }
}

// average time of one call of `launch` over `reps` calls after one warm-up call
template <typename F>
double time_calls(gdr_ctx* ctx, F&& launch, int reps) {
  cudaEvent_t a, b;
  GDR_CUDA(cudaEventCreate(&a));
  GDR_CUDA(cudaEventCreate(&b));
  launch();
  GDR_CUDA(cudaEventRecord(a, ctx->stream));
  for (int r = 0; r < reps; ++r) launch();
  GDR_CUDA(cudaEventRecord(b, ctx->stream));
  GDR_CUDA(cudaEventSynchronize(b));
  float ms = 0;
  GDR_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (double)ms / reps;
}

// enough calls for ~`budget_ms` of timing, at least 3
template <typename F>
double time_adaptive(gdr_ctx* ctx, F&& launch, double budget_ms) {
  const double t1 = time_calls(ctx, launch, 1);
  const int reps = (int)std::max(3.0, std::min(200.0, budget_ms / std::max(t1, 1e-3)));
  return time_calls(ctx, launch, reps);
}

std::vector<MvShape> candidates(const gdr_op* A, int ncol, bool f64) {
  std::vector<MvShape> out;
  const int orders = ncol > 1 ? 2 : 1;
  for (int ci = 0; ci < orders; ++ci) {
    if (A->kind == OP_WILSON) {
      for (int t : {64, 128, 256}) out.push_back(MvShape{0, t, ci});
      out.push_back(MvShape{1, 128, ci});
      if (!f64 && ncol > 1) {  // column pairs with packed FP32x2 arithmetic
        for (int t : {64, 128}) out.push_back(MvShape{2, t, ci});
        // many columns: pairs in groups (the order of all pairs at once keeps too
        // many vectors between a site and its t-neighbour for L2)
        const int npair = (ncol + 1) / 2;
        if (ci == 1)
          for (int grp : {2, 4})
            if (npair > grp)
              for (int t : {64, 128}) out.push_back(MvShape{2, t, grp});
      }
    } else {
      for (int tpr : {1, 2, 4, 8})
        for (int t : {128, 256}) out.push_back(MvShape{tpr, t, ci});
    }
  }
  return out;
}

}  // namespace

template <typename R>
void fill_uniform(gdr_ctx* ctx, long n, int cols, long ld, cx<R>* x, unsigned long long seed) {
  dim3 grid((unsigned)std::min<long>((n + 255) / 256, 8L * ctx->num_sms), (unsigned)cols);
  fill_kernel<R><<<grid, 256, 0, ctx->stream>>>(n, ld, x, seed);
  GDR_LAUNCHED(ctx);
}
template void fill_uniform<float>(gdr_ctx*, long, int, long, c64*, unsigned long long);
template void fill_uniform<double>(gdr_ctx*, long, int, long, c128*, unsigned long long);

template <typename R>
static void tune_matvec(gdr_ctx* ctx, gdr_op* A, int ncol, gdr_tune_result& out) {
  constexpr bool F64 = std::is_same<R, double>::value;
  const std::pair<int, int> key{F64 ? 1 : 0, ncol};
  const int cpp = A->kind == OP_CSR_BATCH ? ncol / A->nprob : 1;
  const long ld = pad_ld(A->n);
  cx<R>* X = ctx->get<cx<R>>("tune.X", (size_t)ld * ncol);
  cx<R>* Y = ctx->get<cx<R>>("tune.Y", (size_t)ld * ncol);
  fill_uniform<R>(ctx, ld, ncol, ld, X, 0x5eedull);
  auto run = [&] { op_apply<R>(ctx, A, ncol, nullptr, X, ld, Y, ld, nullptr, 0, cpp); };

  A->mv_tuned.erase(key);
  const MvShape def = mv_default(ctx, A, ncol);
  MvShape best = def;
  double tbest = 1e30, tdef = -1;
  int count = 0;
  for (const MvShape& s : candidates(A, ncol, F64)) {
    A->mv_tuned[key] = s;
    const double t = time_adaptive(ctx, run, 20.0);
    ++count;
    if (s.form == def.form && s.threads == def.threads && s.col_inner == def.col_inner) tdef = t;
    if (t < tbest) {
      tbest = t;
      best = s;
    }
  }
  A->mv_tuned[key] = best;
  out.best = gdr_shape{best.form, best.threads, best.col_inner};
  out.mv_ms = tbest;
  out.mv_ms_default = tdef >= 0 ? tdef : tbest;
  out.candidates = count;
}

gdr_status tune_op(gdr_ctx* ctx, gdr_op* A, gdr_prec prec, int ncol, int m, gdr_tune_result& out) {
  out = gdr_tune_result{};
  out.sweep = -1;
  const bool f64 = prec == GDR_PREC_FP64;
  if (f64) tune_matvec<double>(ctx, A, ncol, out);
  else tune_matvec<float>(ctx, A, ncol, out);
  if (m > 0) {
    int choice = -1;
    if (f64) tune_arnoldi<double>(ctx, A, ncol, m, out.cycle_ms_sweep, out.cycle_ms_launch, choice);
    else tune_arnoldi<float>(ctx, A, ncol, m, out.cycle_ms_sweep, out.cycle_ms_launch, choice);
    out.sweep = choice;
    if (choice >= 0) A->sweep_tuned[{f64 ? 1 : 0, {ncol, m}}] = choice;
  }
  ctx->release("tune.");  // synchronises the stream
  GDR_CUDA(cudaStreamSynchronize(ctx->stream));
  return GDR_OK;
}

int sweep_choice(const gdr_op* A, bool f64, int ncol, int m) {
  auto it = A->sweep_tuned.find({f64 ? 1 : 0, {ncol, m}});
  return it == A->sweep_tuned.end() ? -1 : it->second;
}
