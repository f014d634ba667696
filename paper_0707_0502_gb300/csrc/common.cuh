// Shared definitions of the gdr CUDA library: complex types, the context and
// operator handles, device workspace, error handling and launch bookkeeping.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "gdr.h"

#define HD __host__ __device__ __forceinline__
#define DEV __device__ __forceinline__

// ------------------------------------------------------------------ complex

template <typename R>
struct alignas(2 * sizeof(R)) cx {
  R x, y;
};
using c64 = cx<float>;
using c128 = cx<double>;

template <typename R> HD cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R> HD cx<R> operator+(cx<R> a, cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R> HD cx<R> operator-(cx<R> a, cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R> HD cx<R> operator-(cx<R> a) { return {-a.x, -a.y}; }
template <typename R> HD cx<R> operator*(cx<R> a, cx<R> b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename R> HD cx<R> operator*(R s, cx<R> a) { return {s * a.x, s * a.y}; }
template <typename R> HD cx<R>& operator+=(cx<R>& a, cx<R> b) { a.x += b.x; a.y += b.y; return a; }
template <typename R> HD cx<R>& operator-=(cx<R>& a, cx<R> b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename R> HD cx<R> conj(cx<R> a) { return {a.x, -a.y}; }
template <typename R> HD R norm2(cx<R> a) { return a.x * a.x + a.y * a.y; }
// conj(a) * b
template <typename R> HD cx<R> cmulc(cx<R> a, cx<R> b) { return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }
// i * a
template <typename R> HD cx<R> mul_i(cx<R> a) { return {-a.y, a.x}; }
HD c128 to128(c64 a) { return {(double)a.x, (double)a.y}; }
HD c64 to64(c128 a) { return {(float)a.x, (float)a.y}; }
template <typename R> HD cx<R> cvt(c128 a);
template <> HD c128 cvt<double>(c128 a) { return a; }
template <> HD c64 cvt<float>(c128 a) { return to64(a); }
template <typename R> HD c128 up(cx<R> a) { return {(double)a.x, (double)a.y}; }

// ----------------------------------------------------------------- errors

struct gdr_error : std::runtime_error {
  gdr_status st;
  gdr_error(gdr_status s, const std::string& m) : std::runtime_error(m), st(s) {}
};

#define GDR_CUDA(call)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      throw gdr_error(e_ == cudaErrorMemoryAllocation ? GDR_ENOMEM : GDR_ECUDA,                     \
                      std::string(#call) + ": " + cudaGetErrorString(e_) + " (" __FILE__ ":" +      \
                          std::to_string(__LINE__) + ")");                                          \
  } while (0)

#define GDR_REQUIRE(cond, msg)                                                   \
  do {                                                                           \
    if (!(cond)) throw gdr_error(GDR_EINVAL, std::string(msg));                  \
  } while (0)

// after every kernel launch
#define GDR_LAUNCHED(ctx)                                                         \
  do {                                                                            \
    GDR_CUDA(cudaGetLastError());                                                 \
    (ctx)->launches++;                                                            \
  } while (0)

// ------------------------------------------------------------------ handles

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct gdr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  size_t max_smem_optin = 0;
  size_t l2_bytes = 0;
  size_t dense_smem_limit = 0;    // dynamic shared memory available to the dense kernels
  size_t combine_smem_limit = 0;  // ... and to the basis-combination kernel
  bool tc_ok = false;              // tensor-core projection dot usable (tensor-map encoder, shared memory)
  bool tc_update_ok = false;     // the residual-update kernel fits this device
  bool tc_proj = true;             // use it in this solve (GDR_FLAG_NO_TENSOR_CORES clears it)
  int* tc_err = nullptr;           // set by the tensor-core kernel when a wait timed out
  int sweep_blocks[3] = {0, 0, 0};  // co-resident blocks per SM of the sweep kernel (c64, bf16 links, c128)
  std::string err;
  std::map<std::string, DevBuf> ws;  // named device workspace
  void* pinned = nullptr;            // small pinned host buffer for status words
  size_t pinned_bytes = 0;
  long launches = 0;                 // kernels launched (graph replays add their node count)
  long syncs = 0;                    // host waits on the stream by the solver

  // per-kernel timing (gdr_profile): CUDA events around every launch, graphs off
  struct ProfRec {
    const char* name;
    double bytes;
    cudaEvent_t a, b;
  };
  struct ProfAgg {
    long launches = 0;
    double ms = 0, bytes = 0;
  };
  bool profile = false;
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  std::map<std::string, ProfAgg> prof;
  cudaEvent_t take_event() {
    if (ev_pool.empty()) {
      cudaEvent_t e;
      GDR_CUDA(cudaEventCreate(&e));
      return e;
    }
    cudaEvent_t e = ev_pool.back();
    ev_pool.pop_back();
    return e;
  }

  // device workspace `name` of at least `bytes`; contents undefined after growth
  void* get(const std::string& name, size_t bytes) {
    DevBuf& b = ws[name];
    if (b.bytes < bytes) {
      if (b.p) {
        GDR_CUDA(cudaStreamSynchronize(stream));
        GDR_CUDA(cudaFree(b.p));
        b.p = nullptr;
        b.bytes = 0;
      }
      size_t sz = (bytes + 255) & ~size_t(255);
      GDR_CUDA(cudaMalloc(&b.p, sz));
      b.bytes = sz;
    }
    return b.p;
  }
  // free every workspace buffer whose name starts with `prefix`
  void release(const std::string& prefix) {
    bool any = false;
    for (auto it = ws.begin(); it != ws.end();) {
      if (it->first.compare(0, prefix.size(), prefix) == 0) {
        if (!any) GDR_CUDA(cudaStreamSynchronize(stream));
        any = true;
        if (it->second.p) GDR_CUDA(cudaFree(it->second.p));
        it = ws.erase(it);
      } else {
        ++it;
      }
    }
  }
  template <typename T> T* get(const std::string& name, size_t count) {
    return static_cast<T*>(get(name, count * sizeof(T)));
  }
  void* host_status(size_t bytes) {
    if (pinned_bytes < bytes) {
      if (pinned) cudaFreeHost(pinned);
      pinned = nullptr;
      GDR_CUDA(cudaMallocHost(&pinned, bytes));
      pinned_bytes = bytes;
    }
    return pinned;
  }
};

enum OpKind { OP_CSR = 0, OP_WILSON = 1, OP_CSR_BATCH = 2 };

// Launch shape of the operator kernels: set by the autotuner (gdr_autotune) or the
// caller (gdr_op_set_shape) per vector precision and column count, else defaults.
struct MvShape {
  int form = 0;       // Wilson: 0 one thread per site, 1 direction-split; CSR: threads per row (1, 2, 4, 8)
  int threads = 128;  // threads per block
  int col_inner = 0;  // 1: consecutive blocks take one site / row tile for consecutive columns;
                      // g >= 2: the same within groups of g columns (pairs for the pair form)
};

struct gdr_op {
  gdr_ctx* ctx = nullptr;
  OpKind kind = OP_CSR;
  long n = 0;
  // CSR
  long nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  c128* vals128 = nullptr;
  c64* vals64 = nullptr;
  // CSR batch: problem p has nrow[p] rows; its rowptr starts at rowptr + rp_off[p] and
  // its local column indices / values at col + nz_off[p], vals + nz_off[p]
  int nprob = 0;
  long* rp_off = nullptr;
  long* nz_off = nullptr;
  int* nrow = nullptr;
  std::vector<long> nrow_host;
  // Wilson: links stored structure-of-arrays [mu][e][V], e = a*3 + b
  int dims[4] = {0, 0, 0, 0};
  long V = 0;
  double diag_a = 0.0;
  gdr_link_fmt store = GDR_LINK_C64;
  c128* links128 = nullptr;
  c64* links64 = nullptr;
  __nv_bfloat162* links16 = nullptr;
  // launch shapes chosen per (FP64 vectors, column count), and the Arnoldi form chosen
  // per (FP64 vectors, column count, m): 1 persistent sweep, 0 per-phase launches
  std::map<std::pair<int, int>, MvShape> mv_tuned;
  std::map<std::pair<int, std::pair<int, int>>, int> sweep_tuned;
};

struct gdr_defl {
  gdr_ctx* ctx = nullptr;
  long n = 0;
  long ldv = 0;
  int k = 0;
  gdr_prec prec = GDR_PREC_FP64;
  void* V = nullptr;     // n x (k+1) in the solve's vector precision (ld = ldv)
  c128* V128 = nullptr;  // FP64 copy (always present), ld = ldv
  c128* Hk = nullptr;    // device (k+1) x k
  std::vector<c128> Hk_host;
  long wilson_V = 0;     // sites of the Wilson operator it came from (vectors in pair-major order), else 0
};

// leading dimension for basis vectors: multiple of 64 elements
inline long pad_ld(long n) { return (n + 63) / 64 * 64; }

// Allow a kernel the largest dynamic shared memory the device permits next to
// its static shared memory; returns that dynamic limit.
template <typename F>
size_t set_max_dyn_smem(gdr_ctx* ctx, F* f) {
  cudaFuncAttributes a;
  GDR_CUDA(cudaFuncGetAttributes(&a, f));
  const size_t dyn = ctx->max_smem_optin - a.sharedSizeBytes;
  GDR_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  return dyn;
}

// Brackets one kernel launch with CUDA events when profiling is on.
struct KProf {
  gdr_ctx* ctx;
  int idx = -1;
  KProf(gdr_ctx* c, const char* name, double bytes) : ctx(c) {
    if (c->profile) {
      gdr_ctx::ProfRec r{name, bytes, c->take_event(), c->take_event()};
      GDR_CUDA(cudaEventRecord(r.a, c->stream));
      c->prof_pending.push_back(r);
      idx = (int)c->prof_pending.size() - 1;
    }
  }
  ~KProf() {
    if (idx >= 0) cudaEventRecord(ctx->prof_pending[idx].b, ctx->stream);
  }
};

// ---------------------------------------------------- launchers (per file)

// ops.cu: Y[:,c] = (A - sigma_c) X[:,c]   (B != nullptr:  Y = B - (A - sigma_c) X)
// sigma: device c128[ncol] (per column); X/Y/B leading dimensions ldx/ldy/ldb
// For a CSR batch, column c of X/Y/B belongs to problem c / cpp (cpp columns per problem);
// for every operator B's column is B + (c / cpp) * ldb.
template <typename R>
void op_apply(gdr_ctx* ctx, const gdr_op* A, int ncol, const c128* sigma_dev, const cx<R>* X, long ldx,
              cx<R>* Y, long ldy, const cx<R>* B, long ldb, int cpp = 1);
