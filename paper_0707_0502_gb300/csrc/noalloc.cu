// Allocation-free form of the GMRES-Sh reduced solve (gdr_dense_gmres_sh).
//
// Some callers cannot let a library allocate device memory: code that runs
// under an allocator it does not control (an embedding framework's memory
// pool, a fixed device-memory budget) or inside a latency-critical loop where
// cudaMalloc / cudaFree would synchronise the device.  This entry point does
// the same work as gdr_dense_gmres_sh but keeps all of its workspace in one
// file-scope __device__ array of fixed size, so it calls no cudaMalloc,
// cudaFree or allocating library routine.  The caller still passes its own
// input and output buffers.
//
// The array exists on every device that loads the library, for the lifetime
// of the process.  It belongs to the library's device code, so under CUDA's lazy
// module loading (the default) its memory is committed when that code is first
// loaded, at the first call on a device: a caller working to a fixed memory
// budget should make one call while setting up.  Its device address is looked up once per device with
// cudaGetSymbolAddress (host code cannot use the symbol itself: on the host it
// names a stand-in, not device memory).  That lookup happens on the first call
// made on a device, so make the first call before any stream capture.  Every
// call shares the one array: calls whose work overlaps on the GPU (two
// streams, two host threads) race and must be serialised by the caller.
#include <mutex>

#include "kernels.cuh"

namespace {

constexpr int NA_MAX_M = GDR_NOALLOC_MAX_M;
constexpr int NA_MAX_NS = GDR_NOALLOC_MAX_NS;

// workspace layout, in complex128 slots
constexpr size_t NA_H = (size_t)(NA_MAX_M + 1) * NA_MAX_M;       // Hbar copy
constexpr size_t NA_C = NA_MAX_M + 1;                             // c copy
constexpr size_t NA_SIG = NA_MAX_NS;                              // shifts
constexpr size_t NA_CF = (size_t)(NA_MAX_M + 1) * (NA_MAX_NS + 1);  // d_i columns (+ s)
constexpr size_t NA_ST = 8;                                       // ColState (80 bytes) + padding
constexpr size_t NA_SACT = (NA_MAX_NS * sizeof(int) + sizeof(c128) - 1) / sizeof(c128);
constexpr size_t NA_SLOTS = NA_H + NA_C + NA_SIG + NA_CF + NA_ST + NA_SACT;
constexpr size_t NA_BYTES = NA_SLOTS * sizeof(c128);
static_assert(sizeof(ColState) <= NA_ST * sizeof(c128), "state slot too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_mu;
void* g_addr[64] = {};  // device address of g_noalloc_scratch, per device

void* scratch_address(int device) {
  GDR_REQUIRE(device >= 0 && device < 64, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    GDR_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_addr[device] = p;
  }
  return g_addr[device];
}

struct InitArgs {
  int m, ns;
  c128 sigma[NA_MAX_NS];
};

// The array keeps the previous call's contents: clear the coefficient
// columns and the state, then set the shifts and the active flags.
__global__ void noalloc_init_kernel(InitArgs a, c128* sig, c128* Cf, long cf_len, ColState* st, int* sact) {
  for (long i = threadIdx.x; i < cf_len; i += blockDim.x) Cf[i] = {0, 0};
  if (threadIdx.x < a.ns) {
    sig[threadIdx.x] = a.sigma[threadIdx.x];
    sact[threadIdx.x] = 1;
  }
  if (threadIdx.x == 0) {
    ColState s = {};
    s.active = 1;
    s.m_eff = a.m;
    *st = s;
  }
}

}  // namespace

extern "C" gdr_status gdr_dense_gmres_sh_noalloc(gdr_ctx* ctx, int m, int ns, const double* Hbar, const double* c,
                                                 const double* sigma, const double* beta, double* D, double* s,
                                                 double* beta_new, double* norms) {
  if (!ctx) return GDR_EINVAL;
  try {
    GDR_REQUIRE(m >= 1 && m <= NA_MAX_M, "gdr_dense_gmres_sh_noalloc: m must be in [1, GDR_NOALLOC_MAX_M]");
    GDR_REQUIRE(ns >= 1 && ns <= NA_MAX_NS, "gdr_dense_gmres_sh_noalloc: ns must be in [1, GDR_NOALLOC_MAX_NS]");
    GDR_REQUIRE(Hbar && c && sigma && beta && D && s && beta_new && norms, "null argument");
    GDR_CUDA(cudaSetDevice(ctx->device));
    c128* base = static_cast<c128*>(scratch_address(ctx->device));
    c128* H = base;
    c128* cv = H + NA_H;
    c128* sg = cv + NA_C;
    c128* Cf = sg + NA_SIG;
    ColState* st = reinterpret_cast<ColState*>(Cf + NA_CF);
    int* sact = reinterpret_cast<int*>(Cf + NA_CF + NA_ST);
    InitArgs ia{};
    ia.m = m;
    ia.ns = ns;
    for (int i = 0; i < ns; ++i) ia.sigma[i] = {sigma[2 * i], sigma[2 * i + 1]};
    const long cf_len = (long)(m + 1) * (ns + 1);
    noalloc_init_kernel<<<1, 128, 0, ctx->stream>>>(ia, sg, Cf, cf_len, st, sact);
    GDR_LAUNCHED(ctx);
    GDR_CUDA(cudaMemcpyAsync(H, Hbar, sizeof(c128) * (m + 1) * m, cudaMemcpyDeviceToDevice, ctx->stream));
    GDR_CUDA(cudaMemcpyAsync(cv, c, sizeof(c128) * (m + 1), cudaMemcpyDeviceToDevice, ctx->stream));
    GDR_CUDA(cudaMemcpyAsync(beta_new, beta, sizeof(c128) * ns, cudaMemcpyDeviceToDevice, ctx->stream));
    DenseCycle d{};
    d.ncol = 1; d.m = m; d.k = 0; d.ns = ns; d.kfull = m + 1;  // general Hbar
    d.H = H; d.cvec = cv; d.sigma = sg;
    d.beta = reinterpret_cast<c128*>(beta_new);
    d.norms = norms;
    d.sact = sact;
    d.Cf = Cf; d.ldc = m + 1; d.ccs = cf_len;
    d.s = reinterpret_cast<c128*>(s);
    d.st = st;
    dense_cycle(ctx, d);
    GDR_CUDA(cudaMemcpy2DAsync(D, m * sizeof(c128), Cf, (m + 1) * sizeof(c128), m * sizeof(c128), ns,
                               cudaMemcpyDeviceToDevice, ctx->stream));
    ColState out;
    GDR_CUDA(cudaMemcpyAsync(&out, st, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
    GDR_CUDA(cudaStreamSynchronize(ctx->stream));
    if (out.err) throw gdr_error((gdr_status)out.err, "singular reduced system");
    return GDR_OK;
  } catch (const gdr_error& e) {
    ctx->err = e.what();
    return e.st;
  } catch (const std::exception& e) {
    ctx->err = e.what();
    return GDR_ECUDA;
  }
}
