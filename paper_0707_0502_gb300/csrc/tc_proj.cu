// Projection dot C = V^H R over a kept basis V (n x nv, complex64) shared by many
// columns R (n x ncol, complex64) -- the Minres projection c = V_{k+1}^H r of every
// column of a Proj or refinement batch (Sec. 2.3, GMRES-Proj-Sh step 4) -- on the
// tensor cores (tcgen05, TF32 inputs, FP32 accumulation in tensor memory).
//
// A complex vector of length n is read as 2n interleaved floats (re, im), so with
// K = 2n:  Re(v^H r) = sum_k v[k] r[k]  and  Im(v^H r) = sum_k v'[k] r[k], where v' is
// v with every (re, im) pair replaced by (-im, re).  One CTA takes a K range and up to
// 128 columns: per K stage (32 floats) TMA brings the V tile (128 rows, rows >= nv zero)
// and the R tile (N rows) into shared memory with the 128-byte swizzle the MMA
// descriptors expect, rounding to TF32 on the way; four warps write the primed V tile
// (the pair swap keeps every 16-byte chunk in place, so the swizzle is unaffected); one
// thread issues the MMAs: D_re += V R^T and D_im += V' R^T, D_re / D_im 128 x N FP32 in
// tensor memory.  At the end the four warps read the accumulators back (tcgen05.ld) and
// write FP64 partials per (K range, column, basis vector), which gs_dot_shared_sum adds
// in a fixed order.
//
// TF32 keeps 10 bits of the significand: a coefficient is accurate to ~1e-3 relative.
// That is enough for the projection: the Proj cycle updates the solutions and the
// residuals with the same coefficients, so an error in c only makes one projection
// slightly less than optimal; residuals and solutions stay consistent.
//
// The residual update R += V T over the same basis (the projection's r -= V_{k+1}(Hbar_k -
// sigma_1 Ibar) d_1 of every column, T = -(Hbar_k - sigma_1 Ibar) d_1) is the transposed
// problem: with the real form of V (row 2i: [Re v_j, -Im v_j], row 2i+1: [Im v_j, Re v_j]
// over j) and the coefficients interleaved, R's real rows += A B^T with K = 2 nv.  A tile
// of 64 complex rows is one 128-row MMA; four warps load V (plain coalesced loads) and
// write A in the 128-byte-swizzled K-major layout, the coefficients sit in shared memory
// for the whole launch, and eight warps add the accumulators to R (plain loads and
// stores, one 128-byte line per warp and column).  The residual must stay consistent
// with the solution update (applied in FP64 on the CUDA cores), so the product is split:
// A = A_hi + A_lo and B = B_hi + B_lo with TF32 parts, D = A_hi B_hi + A_lo B_hi + A_hi B_lo,
// which leaves an error of ~2^-21 relative per product, the level of FP32.
//
// Every wait on an mbarrier gives up after about a second, marks the call failed
// (err, checked by the host) and the CTA winds down, freeing its tensor memory.
#include <cuda.h>

#include "kernels.cuh"

namespace {

constexpr int TC_M = 128;      // MMA rows: basis vectors, zero-filled above nv
constexpr int TC_KF = 32;      // floats per K stage: one 128-byte swizzle row
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 256;  // warp 0 TMA, warp 1 MMA, warp 2 tensor-memory owner, warps 4-7 prime + epilogue
constexpr unsigned TC_A_BYTES = TC_M * TC_KF * 4;  // 16 KB

struct TcArgs {
  int ncol, nv, nt;      // columns, basis vectors, MMA N (multiple of 16, <= 128)
  long ksteps;           // K stages of the whole vector (2n / 32 rounded up)
  long ksplit;           // K stages per CTA
  c128* part;            // [K range][ncol][nv] FP64 partials
  int* err;              // set when a wait timed out
};

DEV uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

DEV unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

DEV void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(bar)), "r"(count) : "memory");
}
DEV void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(bar)), "r"(bytes) : "memory");
}
DEV void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(bar)) : "memory");
}
// wait for the phase of parity `par` to complete; false after ~1 s (or once another
// thread of the CTA gave up), with the CTA's abort flag set
DEV bool mbar_wait(uint64_t* bar, unsigned par, volatile int* abort) {
  const uint32_t a = s_addr(bar);
  const unsigned long long t0 = now_ns();
  for (unsigned it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(par)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255) {
      if (*abort) return false;
      if (now_ns() - t0 > 1000000000ull) {
        *abort = 1;
        return false;
      }
    }
  }
}

DEV void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          s_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(s_addr(bar))
      : "memory");
}

// shared-memory operand descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
DEV uint64_t sm_desc(const void* p) {
  uint64_t d = (uint64_t)((s_addr(p) >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused with a swizzled K-major layout)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset: the next group of 8 rows
  d |= (uint64_t)1 << 46;              // descriptor version of this architecture family
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = nt
DEV uint32_t instr_desc(int nt) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

DEV void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
DEV void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(bar))
               : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes, one lane (row) per thread
DEV void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// accumulator layout in tensor memory: D_re in columns [0, nt), D_im from column im_off
HD int tc_im_off(int nt) { return (nt + 31) / 32 * 32; }
HD uint32_t tc_cols(int nt) {
  const int need = 2 * tc_im_off(nt);
  return need <= 32 ? 32u : need <= 64 ? 64u : need <= 128 ? 128u : 256u;
}

__global__ void __launch_bounds__(TC_THREADS, 1) tc_proj_dot_kernel(const __grid_constant__ CUtensorMap mapV,
                                                                   const __grid_constant__ CUtensorMap mapR,
                                                                   TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const unsigned b_bytes = (unsigned)a.nt * TC_KF * 4;
  const unsigned stage_bytes = 2 * TC_A_BYTES + b_bytes;  // V, V', R
  __shared__ __align__(8) uint64_t full[TC_STAGES], primed[TC_STAGES], empty[TC_STAGES], accb;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_s;
  __shared__ long issued_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long k0 = (long)blockIdx.x * a.ksplit;
  const long nk = min(a.ksteps, k0 + a.ksplit) - k0;
  const int col0 = blockIdx.y * a.nt;
  const int im_off = tc_im_off(a.nt);
  const uint32_t tcols = tc_cols(a.nt);
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&primed[s], 128);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accb, 1);
    abort_s = 0;
    issued_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_base)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tm = tmem_base;
  volatile int* abort = &abort_s;

  if (warp == 0 && lane == 0) {  // ---- TMA producer
    long issued = 0;
    for (long it = 0; it < nk && !*abort; ++it) {
      const int s = (int)(it % TC_STAGES);
      const unsigned ph = (unsigned)((it / TC_STAGES) & 1);
      if (it >= TC_STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort)) break;
      unsigned char* st = base + (size_t)s * stage_bytes;
      mbar_arrive_tx(&full[s], TC_A_BYTES + b_bytes);
      const int x = (int)((k0 + it) * TC_KF);  // a multiple of 32 floats: 128-byte aligned
      tma_load_2d(st, &mapV, x, 0, &full[s]);
      tma_load_2d(st + 2 * TC_A_BYTES, &mapR, x, col0, &full[s]);
      issued = it + 1;
    }
    issued_s = issued;
  } else if (warp == 1 && lane == 0) {  // ---- MMA issuer
    const uint32_t idesc = instr_desc(a.nt);
    for (long it = 0; it < nk; ++it) {
      const int s = (int)(it % TC_STAGES);
      const unsigned ph = (unsigned)((it / TC_STAGES) & 1);
      if (!mbar_wait(&full[s], ph, abort) || !mbar_wait(&primed[s], ph, abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* st = base + (size_t)s * stage_bytes;
      const uint64_t dv = sm_desc(st), dp = sm_desc(st + TC_A_BYTES), dr = sm_desc(st + 2 * TC_A_BYTES);
#pragma unroll
      for (int kk = 0; kk < TC_KF / 8; ++kk) {  // 8 TF32 (32 bytes) per MMA
        const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
        mma_tf32(tm, dv + 2 * kk, dr + 2 * kk, idesc, acc);
        mma_tf32(tm + (uint32_t)im_off, dp + 2 * kk, dr + 2 * kk, idesc, acc);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(&accb);  // arrives once every MMA issued above has completed
  } else if (warp >= 4) {  // ---- V' = V with (re, im) -> (-im, re), then the epilogue
    const int t = threadIdx.x - 128;
    for (long it = 0; it < nk; ++it) {
      const int s = (int)(it % TC_STAGES);
      const unsigned ph = (unsigned)((it / TC_STAGES) & 1);
      if (!mbar_wait(&full[s], ph, abort)) break;
      unsigned char* st = base + (size_t)s * stage_bytes;
      const float4* src = reinterpret_cast<const float4*>(st);
      float4* dst = reinterpret_cast<float4*>(st + TC_A_BYTES);
      for (unsigned q = t; q < TC_A_BYTES / 16; q += 128) {
        const float4 v = src[q];
        dst[q] = make_float4(-v.y, v.x, -v.w, v.z);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&primed[s]);
    }
    // the MMAs finish (or time out) before the accumulators are read or freed; this
    // wait does not follow the CTA's abort flag
    int own = 0;
    const bool got = mbar_wait(&accb, 0, &own);
    if (!got) *abort = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncwarp();
    if (__all_sync(0xffffffffu, got && !*abort)) {
      // accumulators: tensor-memory lane = basis vector, column = matrix column
      const int q4 = warp & 3;
      const int row = q4 * 32 + lane;
      const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
      for (int cb = 0; cb < a.nt; cb += 32) {
        float re[32], im[32];
        tmem_ld32(tm + lane_base + (uint32_t)cb, re);
        tmem_ld32(tm + lane_base + (uint32_t)(im_off + cb), im);
        if (row < a.nv) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int c = col0 + cb + j;
            if (cb + j < a.nt && c < a.ncol)
              a.part[((long)blockIdx.x * a.ncol + c) * a.nv + row] = c128{(double)re[j], (double)im[j]};
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort) {
    // wait (bounded) for the last load issued into each stage, then report the failure
    if (warp == 0 && lane == 0) {
      const long issued = issued_s;
      for (long it = issued > TC_STAGES ? issued - TC_STAGES : 0; it < issued; ++it) {
        int own = 0;
        mbar_wait(&full[(int)(it % TC_STAGES)], (unsigned)((it / TC_STAGES) & 1), &own);
      }
      atomicExch(a.err, 1);
    }
    __syncthreads();
  }
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(tcols) : "memory");
  }
}

// ---------------------------------------------------------------- residual update

constexpr int TU_ROWS = 64;         // complex rows per tile: 128 real MMA rows
constexpr int TU_THREADS = 512;     // warp 1 MMA, warp 2 tensor memory, warps 4-7 A tiles, warps 8-15 epilogue
constexpr int TU_MAXNV = 48;        // K = 2 nv <= 96: three 32-float swizzle atoms
constexpr unsigned TU_ATOM_A = 128u * 128u;  // one K atom of A: 128 rows x 128 bytes

struct TuArgs {
  long n, ntiles;
  int nv, ncol, nt, ka, kp;  // basis vectors, columns, columns per tile (<= 128, multiple of 32), K atoms, K padded to 8
  int rmode;                 // 1: R = V T, 2: R += V T
  const c64* V;
  long ldv;
  const c128* C;             // coefficients of column c at C + c * ccs (nv values)
  long ccs;
  float* R;                  // R as floats, column c at R + 2 * c * ldr
  long ldr;
  const ColState* st;
  int* err;
};

DEV uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x = hi + lo, both TF32
DEV void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(tf32_rna(x));
  lo = __uint_as_float(tf32_rna(x - hi));
}
// byte offset of element (row, k) in a K-major, 128-byte-swizzled operand of `rows` rows
DEV unsigned swz_off(int row, int k, int rows) {
  const int a = k >> 5, kin = k & 31;
  return (unsigned)a * (unsigned)rows * 128u + (unsigned)row * 128u + ((unsigned)((kin >> 2) ^ (row & 7)) << 4) +
         (unsigned)(kin & 3) * 4u;
}

__global__ void __launch_bounds__(TU_THREADS, 1) tc_proj_update_kernel(TuArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* Ahi = base;
  unsigned char* Alo = Ahi + (size_t)a.ka * TU_ATOM_A;
  unsigned char* Bhi = Alo + (size_t)a.ka * TU_ATOM_A;
  unsigned char* Blo = Bhi + (size_t)a.ka * a.nt * 128;
  __shared__ __align__(8) uint64_t aready, afree, dfull[2], dempty[2], fin;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_s;
  __shared__ int cmap[128];  // the active columns of this column tile, compacted
  __shared__ int wcnt[4], nact_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col0 = blockIdx.y * a.nt;
  const long my_tiles = blockIdx.x < a.ntiles ? (a.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  // active columns: the MMA width and the epilogue follow their number, and a tile
  // whose columns have all converged has nothing to do
  bool f = false;
  unsigned bal = 0;
  if (warp < 4) {
    const int c = threadIdx.x;
    f = c < a.nt && col0 + c < a.ncol && (!a.st || a.st[col0 + c].active);
    bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcnt[warp] = __popc(bal);
  }
  __syncthreads();
  if (warp < 4) {
    int off = 0;
    for (int w = 0; w < warp; ++w) off += wcnt[w];
    if (f) cmap[off + __popc(bal & ((1u << lane) - 1u))] = threadIdx.x;
    if (threadIdx.x == 0) nact_s = wcnt[0] + wcnt[1] + wcnt[2] + wcnt[3];
  }
  __syncthreads();
  const int nact = nact_s;
  if (nact == 0 || my_tiles == 0) return;  // uniform over the CTA, before any barrier or tensor memory
  const int ne = (nact + 31) / 32 * 32;   // MMA N: compacted columns, zero rows above nact

  if (threadIdx.x == 0) {
    mbar_init(&aready, 128);
    mbar_init(&afree, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&dfull[b], 1);
      mbar_init(&dempty[b], 256);
    }
    mbar_init(&fin, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_base)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // A's padding (k >= 2 nv) stays zero; B = the active columns' coefficients split into
  // TF32 parts, K-major, row k = column cmap[k]
  {
    uint4* z = reinterpret_cast<uint4*>(Ahi);
    const unsigned nz = 2u * a.ka * TU_ATOM_A / 16u;
    for (unsigned q = threadIdx.x; q < nz; q += TU_THREADS) z[q] = make_uint4(0, 0, 0, 0);
    const int kw = a.ka * 32;
    for (int t = threadIdx.x; t < ne * kw; t += TU_THREADS) {
      const int r = t / kw, k = t % kw, j = k >> 1;
      float hi = 0.f, lo = 0.f;
      if (r < nact && j < a.nv) {
        const c128 v = a.C[(long)(col0 + cmap[r]) * a.ccs + j];
        const double x = (k & 1) ? v.y : v.x;
        hi = __uint_as_float(tf32_rna((float)x));
        lo = __uint_as_float(tf32_rna((float)(x - (double)hi)));
      }
      const unsigned off = swz_off(r, k, ne);
      *reinterpret_cast<float*>(Bhi + off) = hi;
      *reinterpret_cast<float*>(Blo + off) = lo;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tm = tmem_base;
  volatile int* abort = &abort_s;

  if (warp == 1) {  // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = instr_desc(ne);
      const uint64_t dah = sm_desc(Ahi), dal = sm_desc(Alo), dbh = sm_desc(Bhi), dbl = sm_desc(Blo);
      const uint32_t astep = TU_ATOM_A >> 4, bstep = (uint32_t)(ne * 128) >> 4;  // one K atom, in 16-byte units
      for (long it = 0; it < my_tiles; ++it) {
        const int b = (int)(it & 1);
        if (!mbar_wait(&aready, (unsigned)(it & 1), abort)) break;
        if (it >= 2 && !mbar_wait(&dempty[b], (unsigned)(((it >> 1) & 1) ^ 1), abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tm + (uint32_t)(b * 128);
        for (int pass = 0; pass < 3; ++pass) {  // hi*hi, lo*hi, hi*lo
          const uint64_t da = pass == 1 ? dal : dah, db = pass == 2 ? dbl : dbh;
          for (int kk = 0; kk < a.kp / 8; ++kk) {
            const uint32_t ka = (uint32_t)(kk >> 2), kin = (uint32_t)(kk & 3) * 2;
            mma_tf32(d, da + ka * astep + kin, db + ka * bstep + kin, idesc, (pass > 0 || kk > 0) ? 1u : 0u);
          }
        }
        mma_commit(&dfull[b]);
        mma_commit(&afree);
      }
      mma_commit(&fin);  // arrives once every MMA issued above has completed
      int own = 0;
      if (!mbar_wait(&fin, 0, &own)) *abort = 1;
    }
  } else if (warp >= 4 && warp < 8) {  // ---- A tiles from V
    // lane = (row, basis vector) as 8 x 4: a load instruction reads 4 runs of 64 bytes of V,
    // and a store writes 8 rows x 32 bytes of A, which the swizzle spreads over all banks
    const int w4 = warp - 4, il = lane >> 2, jl = lane & 3;
    float2 v[2][TU_MAXNV / 4];
    auto load = [&](long it) {
      const long rb = (blockIdx.x + it * (long)gridDim.x) * TU_ROWS + w4 * 16 + il;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long row = rb + 8 * h;
#pragma unroll
        for (int q = 0; q < TU_MAXNV / 4; ++q) {
          const int j = jl + 4 * q;
          v[h][q] = make_float2(0.f, 0.f);
          if (j < a.nv && row < a.n) {
            const c64 x = a.V[(long)j * a.ldv + row];
            v[h][q] = make_float2(x.x, x.y);
          }
        }
      }
    };
    if (my_tiles > 0) load(0);
    for (long it = 0; it < my_tiles; ++it) {
      if (it >= 1 && !mbar_wait(&afree, (unsigned)((it - 1) & 1), abort)) break;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = w4 * 16 + il + 8 * h;  // complex row of the tile: real rows 2i, 2i + 1
#pragma unroll
        for (int q = 0; q < TU_MAXNV / 4; ++q) {
          const int j = jl + 4 * q;
          if (j < a.nv) {
            float rh, rl, ih, il2;
            split_tf32(v[h][q].x, rh, rl);
            split_tf32(v[h][q].y, ih, il2);
            const unsigned o0 = swz_off(2 * i, 2 * j, 128), o1 = swz_off(2 * i + 1, 2 * j, 128);
            *reinterpret_cast<float2*>(Ahi + o0) = make_float2(rh, -ih);
            *reinterpret_cast<float2*>(Ahi + o1) = make_float2(ih, rh);
            *reinterpret_cast<float2*>(Alo + o0) = make_float2(rl, -il2);
            *reinterpret_cast<float2*>(Alo + o1) = make_float2(il2, rl);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&aready);
      if (it + 1 < my_tiles) load(it + 1);
    }
  } else if (warp >= 8) {  // ---- R += D
    const int q4 = warp & 3, half = (warp - 8) >> 2;
    const int m = q4 * 32 + lane;  // real row of the tile = tensor-memory lane
    const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
    const int nch = ne / 32;      // this warp takes chunks half and half + 2 (nch <= 4)
    for (long it = 0; it < my_tiles; ++it) {
      const int b = (int)(it & 1);
      const long r0 = (blockIdx.x + it * (long)gridDim.x) * TU_ROWS;
      const long g = 2 * r0 + m;  // float index within a column
      const bool rowok = g < 2 * a.n;
      // R's current values for both chunks, requested before the accumulators are ready
      float old[2][32];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int cc = half + 2 * u;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int k = cc * 32 + j;
          old[u][j] = (a.rmode == 2 && cc < nch && rowok && k < nact)
                          ? a.R[2 * (long)(col0 + cmap[k]) * a.ldr + g] : 0.f;
        }
      }
      int own = 0;
      const bool got = mbar_wait(&dfull[b], (unsigned)((it >> 1) & 1), &own);
      if (!got) *abort = 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      __syncwarp();
      if (__any_sync(0xffffffffu, !got || *abort)) break;  // warp-uniform: tcgen05.ld is .sync.aligned
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int cc = half + 2 * u;
        if (cc >= nch) break;
        float d[32];
        tmem_ld32(tm + lane_base + (uint32_t)(b * 128 + cc * 32), d);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int k = cc * 32 + j;
          if (rowok && k < nact) a.R[2 * (long)(col0 + cmap[k]) * a.ldr + g] = old[u][j] + d[j];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&dempty[b]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort && threadIdx.x == 0) atomicExch(a.err, 1);
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(256) : "memory");
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// 2-D map of `rows` vectors of 2n floats each (stride ld complex elements), box 32 floats x box_rows,
// TF32 rounding on load, 128-byte swizzle, zero fill outside
bool make_map(CUtensorMap& m, const void* ptr, long n, long ld, int rows, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)(2 * n), (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 8)};
  cuuint32_t box[2] = {(cuuint32_t)TC_KF, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(&m, CU_TENSOR_MAP_DATA_TYPE_TFLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t tc_proj_smem(int nt) { return 1024 + (size_t)TC_STAGES * (2 * TC_A_BYTES + (size_t)nt * TC_KF * 4); }

int tc_proj_splits(gdr_ctx* ctx, long n, int ncol) {
  const int ctiles = (ncol + 127) / 128;
  const long ksteps = (2 * n + TC_KF - 1) / TC_KF;
  const int want = std::max(1, ctx->num_sms / ctiles);
  const long ksplit = (ksteps + want - 1) / want;
  return (int)((ksteps + ksplit - 1) / ksplit);
}

bool tc_proj_dot(gdr_ctx* ctx, long n, const c64* V, long ldv, int nv, const c64* R, long ldr, int ncol, c128* part,
                 int* err, int& nsplit, double prof_bytes) {
  if (nv < 1 || nv > TC_M || ncol < 1 || !ctx->tc_ok) return false;
  const int ctiles = (ncol + 127) / 128;
  const int per = (ncol + ctiles - 1) / ctiles;
  const int nt = std::max(16, (per + 15) / 16 * 16);
  CUtensorMap mv, mr;
  if (!make_map(mv, V, n, ldv, nv, TC_M) || !make_map(mr, R, n, ldr, ncol, nt)) return false;
  TcArgs a;
  a.ncol = ncol;
  a.nv = nv;
  a.nt = nt;
  a.ksteps = (2 * n + TC_KF - 1) / TC_KF;
  nsplit = tc_proj_splits(ctx, n, ncol);
  a.ksplit = (a.ksteps + nsplit - 1) / nsplit;
  a.part = part;
  a.err = err;
  const size_t smem = tc_proj_smem(nt);
  dim3 grid((unsigned)nsplit, (unsigned)ctiles);
  KProf kp(ctx, "tc_proj_dot_c64", prof_bytes);
  tc_proj_dot_kernel<<<grid, TC_THREADS, smem, ctx->stream>>>(mv, mr, a);
  GDR_LAUNCHED(ctx);
  return true;
}

size_t tc_update_smem(int ka, int nt) { return 1024 + 2 * (size_t)ka * TU_ATOM_A + 2 * (size_t)ka * nt * 128; }

bool tc_proj_update(gdr_ctx* ctx, long n, const c64* V, long ldv, int nv, const c128* C, long ccs, int rmode, c64* R,
                    long ldr, int ncol, const ColState* st, int* err, double prof_bytes) {
  if (nv < 1 || nv > TU_MAXNV || ncol < 1 || (rmode != 1 && rmode != 2) || !ctx->tc_ok || !ctx->tc_update_ok)
    return false;
  const int ctiles = (ncol + 127) / 128;
  const int per = (ncol + ctiles - 1) / ctiles;
  TuArgs a;
  a.n = n;
  a.ntiles = (n + TU_ROWS - 1) / TU_ROWS;
  a.nv = nv;
  a.ncol = ncol;
  a.nt = (per + 31) / 32 * 32;
  a.kp = (2 * nv + 7) / 8 * 8;
  a.ka = (a.kp + 31) / 32;
  a.rmode = rmode;
  a.V = V;
  a.ldv = ldv;
  a.C = C;
  a.ccs = ccs;
  a.R = reinterpret_cast<float*>(R);
  a.ldr = ldr;
  a.st = st;
  a.err = err;
  const size_t smem = tc_update_smem(a.ka, a.nt);
  const long want = std::max(1, ctx->num_sms / ctiles);
  dim3 grid((unsigned)std::min<long>(want, a.ntiles), (unsigned)ctiles);
  KProf kp(ctx, "tc_proj_update_c64", prof_bytes);
  tc_proj_update_kernel<<<grid, TU_THREADS, smem, ctx->stream>>>(a);
  GDR_LAUNCHED(ctx);
  return true;
}

void tc_proj_init(gdr_ctx* ctx) {
  ctx->tc_ok = false;
  if (!encoder()) return;
  cudaFuncAttributes at;
  if (cudaFuncGetAttributes(&at, tc_proj_dot_kernel) != cudaSuccess) return;
  const size_t need = tc_proj_smem(128);
  if (need + at.sharedSizeBytes > ctx->max_smem_optin) return;
  if (cudaFuncSetAttribute(tc_proj_dot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need) != cudaSuccess)
    return;
  ctx->tc_ok = true;
  ctx->tc_update_ok = false;
  if (cudaFuncGetAttributes(&at, tc_proj_update_kernel) != cudaSuccess) return;
  const size_t need_u = tc_update_smem(3, 128);
  if (need_u + at.sharedSizeBytes > ctx->max_smem_optin) return;
  if (cudaFuncSetAttribute(tc_proj_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need_u) !=
      cudaSuccess)
    return;
  ctx->tc_update_ok = true;
}
