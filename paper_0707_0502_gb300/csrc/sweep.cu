// Persistent Arnoldi sweep: the steps j = jstart .. jend-1 of one GMRES cycle
// (CGS2 Arnoldi, A V_m = V_{m+1} Hbar_m, eq. recurAr) on every column of a
// batch in ONE cooperative launch, the phases of a step separated by grid
// barriers instead of kernel boundaries.  Meant for short vectors (an
// L2-resident basis), where each of the four launches of arnoldi_step costs
// 10-17 us of mostly fixed latency: here a phase costs its work plus a barrier.
//
// Per step j (nv = j + 1 basis vectors):
//   M   w = s A x          x = v_j (first step) or W2 with s = 1 / h_{j,j-1}
//   D1  h1 = V^H w, ||w||^2; the first dot of a lazy step also stores v_j = s W2
//   UD  w' = w - V h1 (into W2), h2 = V^H w'
//   U   w'' = w' - V h2 (in place), ||w''||^2 partials
//   F   Hbar column j = h1 + h2, h_{j+1,j} = ||w''||, breakdown test, 1/h_{j+1,j}
// with a grid barrier after each phase.  Reductions are deterministic: FP64
// partials per (tile slot, vector) are summed in slot order by every block
// that needs them (identical results in all blocks).  Everything written inside
// the launch by other blocks is read through L2 (ld.global.cg).
//
// The barrier spins with a bounded count (about a second); if it gives up the
// kernel marks every column GDR_ETIMEOUT and returns.  The launch is
// cooperative, so all blocks are co-resident and the bound is only a guard.
#include "kernels.cuh"
#include "vecunits.cuh"
#include "wilson.cuh"

// Phase marks for timing studies; empty in the library build.
#ifndef GDR_SWEEP_MARK
#define GDR_SWEEP_MARK(j, i)
#endif

namespace {

constexpr int ST = 256;                    // threads per block
constexpr int SDU = 8;                     // 16-byte units per lane of a dot tile (tile = ST units)
constexpr long BAR_SPINS = 1L << 20;       // barrier give-up count: ~1 s (a poll is an L2 round trip + 20 ns)

struct SweepBar {
  unsigned count;
  unsigned gen;
  int err;
  int pad;
};

template <typename R>
struct SweepArgs {
  Batch<R> b;
  int kind;                                   // OpKind
  long n;                                     // CSR rows (largest problem of a batch)
  const int* rowptr;
  const int* col;
  const cx<R>* vals;
  const long* rp_off;
  const long* nz_off;
  const int* nrow;
  int Lx, Ly, Lz, Lt;
  long V;
  double diag_a;
  const void* links;
  int jstart, jend;
  int S;                                      // tile slots per column
  int NU;                                     // update blocks per column
  long pstride;                               // partial buffer per column (slots x hs)
  int hs;                                     // m + 2
  c128* partA;
  c128* partB;
  SweepBar* bar;
};

DEV c128 ldcg_c128(const c128* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}
DEV int ldcg_int(const int* p) { return __ldcg(p); }
DEV double ldcg_dbl(const double* p) { return __ldcg(p); }

// 16-byte unit loads through L2
template <typename R> DEV void ldu_cg(const cx<R>* p, long u, long n, cx<R> (&o)[U<R>::K]) {
  if constexpr (sizeof(R) == 4) {
    if (2 * u + 1 < n) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(p) + u);
      o[0] = {v.x, v.y};
      o[1] = {v.z, v.w};
    } else {
      const float2 v = __ldcg(reinterpret_cast<const float2*>(p) + 2 * u);
      o[0] = {v.x, v.y};
      o[1] = {0.f, 0.f};
    }
  } else {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p) + u);
    o[0] = {v.x, v.y};
  }
}

DEV unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
DEV void red_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier on a counter that only grows within a launch: barrier number e
// is passed when the counter reaches e * gridDim.x.  Thread 0 of each block
// arrives with a release-add (ordering the block's writes, made CTA-visible by
// __syncthreads, before the arrival) and polls with acquire loads.  False if it
// gave up (another block's failure or the spin bound).
DEV bool grid_sync(SweepBar* gb, unsigned& epoch, unsigned arrivals = 0) {
  __shared__ int fail;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    fail = 0;
    red_release_gpu(&gb->count, 1u);
    const unsigned target = epoch * (arrivals ? arrivals : gridDim.x);
    long it = 0;
    while (ld_acquire_gpu(&gb->count) < target) {
      if ((++it & 1023) == 0 && (*(volatile int*)&gb->err || it > BAR_SPINS)) {
        atomicExch(&gb->err, 1);
        fail = 1;
        break;
      }
      __nanosleep(20);
    }
  }
  __syncthreads();
  return fail == 0;
}

// out[i] = sum_{s < cnt} p[s * hs + i], i < nval, summed in a fixed order (the same
// in every block); scratch holds ST values
DEV void reduce_slots(const c128* p, int hs, int cnt, int nval, c128* out, c128* scratch) {
  const int ppv = max(1, ST / max(nval, 1));
  const int t = threadIdx.x, i = t / ppv, r = t % ppv;
  c128 s = {0, 0};
  if (i < nval)
    for (int q = r; q < cnt; q += ppv) s += ldcg_c128(p + (long)q * hs + i);
  scratch[t] = s;
  __syncthreads();
  if (t < nval) {
    c128 acc = {0, 0};
    for (int rr = 0; rr < ppv; ++rr) acc += scratch[t * ppv + rr];
    out[t] = acc;
  }
  __syncthreads();
}

DEV void named_sync(int id, int nthreads) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory"); }

// ---------------------------------------------------------------- phase M
template <typename R, typename LT>
DEV void phase_matvec(const SweepArgs<R>& a, int j, bool lazy, unsigned char* sm) {
  const Batch<R>& b = a.b;
  if (a.kind == OP_WILSON) {
    // direction-split Wilson: each half block (128 threads) takes 32 sites, warp mu of
    // the half the two hops in direction mu; partial spinors summed in shared memory
    auto part = reinterpret_cast<cx<R>(*)[32][13]>(sm);  // [8][32][13]
    const LT* links = static_cast<const LT*>(a.links);
    const long V = a.V;
    const long ngroups = (V + 31) / 32, npairs = (ngroups + 1) / 2;
    const int half = threadIdx.x >> 7, mu = (threadIdx.x >> 5) & 3, lane = threadIdx.x & 31;
    const int ht = threadIdx.x & 127;
    for (long it = blockIdx.x; it < (long)b.ncol * npairs; it += gridDim.x) {
      const int c = (int)(it / npairs);
      const long grp = (it % npairs) * 2 + half;
      const bool live = ldcg_int(&b.st[c].run) && grp < ngroups;
      const cx<R>* x = lazy ? b.W2 + c * b.wcs : b.V + c * b.vcs + (long)j * b.ldv;
      const R sc = lazy ? (R)ldcg_dbl(&b.st[c].inv_norm) : R(1);
      const long site0 = grp * 32, site = site0 + lane;
      named_sync(1 + half, 128);  // readers of the previous item are done
      if (live) {
        Spinor<R> acc;
#pragma unroll
        for (int i = 0; i < 12; ++i) acc.s[i] = {0, 0};
        if (site < V) {
          int ix, iy, iz, itt;
          site_coords(site, a.Lx, a.Ly, a.Lz, ix, iy, iz, itt);
          switch (mu) {
            case 0: hop_mu<0, R, LT, true>(links, x, V, site, ix, a.Lx, 1, acc); break;
            case 1: hop_mu<1, R, LT, true>(links, x, V, site, iy, a.Ly, (long)a.Lx, acc); break;
            case 2: hop_mu<2, R, LT, true>(links, x, V, site, iz, a.Lz, (long)a.Lx * a.Ly, acc); break;
            default: hop_mu<3, R, LT, true>(links, x, V, site, itt, a.Lt, (long)a.Lx * a.Ly * a.Lz, acc); break;
          }
        }
#pragma unroll
        for (int i = 0; i < 12; ++i) part[4 * half + mu][lane][i] = acc.s[i];
      }
      named_sync(1 + half, 128);
      if (live) {
        const cx<R> dg = {(R)a.diag_a, R(0)};
        cx<R>* y = b.W + c * b.wcs;
        // output element q: pair q / 64, site q % 64 / 2, half q % 2 (pair-major vector order)
        for (int q = ht; q < 6 * 64; q += 128) {
          const int pr = q >> 6, sl = (q & 63) >> 1, comp = 2 * pr + (q & 1);
          if (site0 + sl >= V) continue;
          const cx<R> h = part[4 * half][sl][comp] + part[4 * half + 1][sl][comp] + part[4 * half + 2][sl][comp] +
                          part[4 * half + 3][sl][comp];
          const long e = 2 * ((long)pr * V + site0) + (q & 63);
          cx<R> xv;
          if constexpr (sizeof(R) == 4) {
            const float2 t = __ldcg(reinterpret_cast<const float2*>(x) + e);
            xv = {t.x, t.y};
          } else {
            const double2 t = __ldcg(reinterpret_cast<const double2*>(x) + e);
            xv = {t.x, t.y};
          }
          y[e] = sc * (dg * xv - h);
        }
      }
    }
  } else {
    const bool batch = a.kind == OP_CSR_BATCH;
    const long nrb = (a.n + ST - 1) / ST;
    for (long it = blockIdx.x; it < (long)b.ncol * nrb; it += gridDim.x) {
      const int c = (int)(it / nrb);
      const long r = (it % nrb) * ST + threadIdx.x;
      if (!ldcg_int(&b.st[c].run)) continue;
      const int p = batch ? c / b.cpp : 0;
      const long rows = batch ? (long)a.nrow[p] : a.n;
      if (r >= rows) continue;
      const int* rp = a.rowptr + (batch ? a.rp_off[p] : 0);
      const int* cl = a.col + (batch ? a.nz_off[p] : 0);
      const cx<R>* vl = a.vals + (batch ? a.nz_off[p] : 0);
      const cx<R>* x = lazy ? b.W2 + c * b.wcs : b.V + c * b.vcs + (long)j * b.ldv;
      const R sc = lazy ? (R)ldcg_dbl(&b.st[c].inv_norm) : R(1);
      cx<R> acc = {0, 0};
      const int p0 = rp[r], p1 = rp[r + 1];
      for (int q = p0; q < p1; ++q) {
        cx<R> xv;
        if constexpr (sizeof(R) == 4) {
          const float2 t = __ldcg(reinterpret_cast<const float2*>(x) + cl[q]);
          xv = {t.x, t.y};
        } else {
          const double2 t = __ldcg(reinterpret_cast<const double2*>(x) + cl[q]);
          xv = {t.x, t.y};
        }
        acc += vl[q] * xv;
      }
      b.W[c * b.wcs + r] = sc * acc;
    }
  }
}

// vector groups of a dot phase: enough blocks for the grid, at least 8 vectors per group
DEV int dot_groups(int S, int ncol, int nvec) {
  const int g = max(1, ((int)gridDim.x + S * ncol - 1) / (S * ncol));
  return max(1, min(g, (nvec + 7) / 8));
}

// ---------------------------------------------------------------- phase D1
template <typename R>
DEV void phase_dot1(const SweepArgs<R>& a, int nv, bool lazy, unsigned char* sm) {
  const Batch<R>& b = a.b;
  constexpr int K = U<R>::K, DU = SDU, TU = DU * 32;
  cx<R>* wt = reinterpret_cast<cx<R>*>(sm);                              // TU*K
  c128* accs = reinterpret_cast<c128*>(sm + sizeof(cx<R>) * TU * K);     // GDR_MAX_M + 2
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = a.S, nvec_tot = nv + 1;
  const int G = dot_groups(S, b.ncol, nvec_tot);
  const int vpg = (nvec_tot + G - 1) / G;
  for (long it = blockIdx.x; it < (long)b.ncol * S * G; it += gridDim.x) {
    const int c = (int)(it / ((long)S * G));
    const int rem = (int)(it % ((long)S * G)), slot = rem % S, grp = rem / S;
    if (!ldcg_int(&b.st[c].run)) continue;  // uniform in the block
    const int i0 = grp * vpg, i1 = min(nvec_tot, i0 + vpg);
    if (i0 >= i1) continue;
    const long n = b.nvec ? (long)b.nvec[c] : b.n, nu = nunits<R>(n);
    const long ntiles = (nu + TU - 1) / TU;
    const cx<R>* V = b.V + c * b.vcs;
    const cx<R>* w = b.W + c * b.wcs;
    const cx<R>* wp = b.W2 + c * b.wcs;
    const R sc = lazy ? (R)ldcg_dbl(&b.st[c].inv_norm) : R(1);
    __syncthreads();
    for (int i = i0 + threadIdx.x; i < i1; i += ST) accs[i] = {0, 0};
    for (long t = slot; t < ntiles; t += S) {
      const long u0 = t * TU;
      __syncthreads();
      for (int q = threadIdx.x; q < TU; q += ST) {
        cx<R> tmp[K];
        if (u0 + q < nu) {
          ldu_cg<R>(w, u0 + q, n, tmp);
        } else {
#pragma unroll
          for (int kk = 0; kk < K; ++kk) tmp[kk] = {0, 0};
        }
#pragma unroll
        for (int kk = 0; kk < K; ++kk) wt[q * K + kk] = tmp[kk];
      }
      __syncthreads();
      for (int i = i0 + warp; i < i1; i += ST / 32) {
        cx<R> s = {0, 0};
        if (i < nv) {
          const bool lz = lazy && i == nv - 1;
          const cx<R>* vi = lz ? wp : V + (long)i * b.ldv;
#pragma unroll
          for (int h0 = 0; h0 < DU; h0 += DU) {
            cx<R> vv[DU][K];
#pragma unroll
            for (int tt = 0; tt < DU; ++tt) {
              const long u = u0 + lane + 32 * (h0 + tt);
              if (u < nu) {
                ldu_cg<R>(vi, u, n, vv[tt]);
              } else {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) vv[tt][kk] = {0, 0};
              }
            }
            if (lz) {
              cx<R>* vo = b.V + c * b.vcs + (long)i * b.ldv;
#pragma unroll
              for (int tt = 0; tt < DU; ++tt) {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) vv[tt][kk] = sc * vv[tt][kk];
                const long u = u0 + lane + 32 * (h0 + tt);
                if (u < nu) stu<R>(vo, u, n, vv[tt]);
              }
            }
#pragma unroll
            for (int tt = 0; tt < DU; ++tt)
#pragma unroll
              for (int kk = 0; kk < K; ++kk) s += cmulc(vv[tt][kk], wt[(lane + 32 * (h0 + tt)) * K + kk]);
          }
        } else {
#pragma unroll
          for (int tt = 0; tt < DU; ++tt)
#pragma unroll
            for (int kk = 0; kk < K; ++kk) s.x += norm2(wt[(lane + 32 * tt) * K + kk]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          s.x += __shfl_xor_sync(FULL, s.x, off);
          s.y += __shfl_xor_sync(FULL, s.y, off);
        }
        if (lane == 0) accs[i] += up(s);
      }
    }
    __syncthreads();
    c128* part = a.partA + c * a.pstride;
    for (int i = i0 + threadIdx.x; i < i1; i += ST) part[(long)slot * a.hs + i] = accs[i];
  }
}

// ---------------------------------------------------------------- phase UD
template <typename R>
DEV void phase_update_dot(const SweepArgs<R>& a, int nv, unsigned char* sm) {
  const Batch<R>& b = a.b;
  constexpr int K = U<R>::K, DU = SDU, TU = DU * 32, JB = 8;
  cx<R>* wt = reinterpret_cast<cx<R>*>(sm);
  c128* accs = reinterpret_cast<c128*>(sm + sizeof(cx<R>) * TU * K);
  c128* h64 = accs + (GDR_MAX_M + 2);
  c128* scratch = h64 + (GDR_MAX_M + 2);
  cx<R>* hs = reinterpret_cast<cx<R>*>(scratch + ST);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = a.S;
  const int G = dot_groups(S, b.ncol, nv);
  const int vpg = (nv + G - 1) / G;
  for (long it = blockIdx.x; it < (long)b.ncol * S * G; it += gridDim.x) {
    const int c = (int)(it / ((long)S * G));
    const int rem = (int)(it % ((long)S * G)), slot = rem % S, grp = rem / S;
    if (!ldcg_int(&b.st[c].run)) continue;
    const int i0 = grp * vpg, i1 = min(nv, i0 + vpg);
    const long n = b.nvec ? (long)b.nvec[c] : b.n, nu = nunits<R>(n);
    const long ntiles = (nu + TU - 1) / TU;
    const cx<R>* V = b.V + c * b.vcs;
    const cx<R>* w = b.W + c * b.wcs;
    cx<R>* wo = b.W2 + c * b.wcs;
    __syncthreads();
    // h1 (and ||w||^2 in slot nv) from the D1 partials
    reduce_slots(a.partA + c * a.pstride, a.hs, S, nv + 1, h64, scratch);
    for (int i = threadIdx.x; i < nv; i += ST) hs[i] = cvt<R>(h64[i]);
    if (slot == 0 && grp == 0)
      for (int i = threadIdx.x; i <= nv; i += ST) b.h1[(long)c * (b.m + 2) + i] = h64[i];
    for (int i = i0 + threadIdx.x; i < i1; i += ST) accs[i] = {0, 0};
    for (long t = slot; t < ntiles; t += S) {
      const long u0 = t * TU;
      __syncthreads();
      for (int q = threadIdx.x; q < TU; q += ST) {
        const long u = u0 + q;
        cx<R> acc[K];
        if (u < nu) {
          ldu_cg<R>(w, u, n, acc);
          for (int g0 = 0; g0 < nv; g0 += JB) {
            cx<R> vv[JB][K];
#pragma unroll
            for (int qq = 0; qq < JB; ++qq)
              if (g0 + qq < nv) ldu_cg<R>(V + (long)(g0 + qq) * b.ldv, u, n, vv[qq]);
#pragma unroll
            for (int qq = 0; qq < JB; ++qq) {
              if (g0 + qq < nv) {
                const cx<R> hi = hs[g0 + qq];
#pragma unroll
                for (int kk = 0; kk < K; ++kk) acc[kk] -= vv[qq][kk] * hi;
              }
            }
          }
          if (grp == 0) stu<R>(wo, u, n, acc);
        } else {
#pragma unroll
          for (int kk = 0; kk < K; ++kk) acc[kk] = {0, 0};
        }
#pragma unroll
        for (int kk = 0; kk < K; ++kk) wt[q * K + kk] = acc[kk];
      }
      __syncthreads();
      for (int i = i0 + warp; i < i1; i += ST / 32) {
        const cx<R>* vi = V + (long)i * b.ldv;
        cx<R> s = {0, 0};
#pragma unroll
        for (int h0 = 0; h0 < DU; h0 += DU) {
          cx<R> vv[DU][K];
#pragma unroll
          for (int tt = 0; tt < DU; ++tt) {
            const long u = u0 + lane + 32 * (h0 + tt);
            if (u < nu) {
              ldu_cg<R>(vi, u, n, vv[tt]);
            } else {
#pragma unroll
              for (int kk = 0; kk < K; ++kk) vv[tt][kk] = {0, 0};
            }
          }
#pragma unroll
          for (int tt = 0; tt < DU; ++tt)
#pragma unroll
            for (int kk = 0; kk < K; ++kk) s += cmulc(vv[tt][kk], wt[(lane + 32 * (h0 + tt)) * K + kk]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          s.x += __shfl_xor_sync(FULL, s.x, off);
          s.y += __shfl_xor_sync(FULL, s.y, off);
        }
        if (lane == 0) accs[i] += up(s);
      }
    }
    __syncthreads();
    c128* part = a.partB + c * a.pstride;
    for (int i = i0 + threadIdx.x; i < i1; i += ST) part[(long)slot * a.hs + i] = accs[i];
  }
}

// ---------------------------------------------------------------- phase U
template <typename R>
DEV void phase_update(const SweepArgs<R>& a, int nv, unsigned char* sm) {
  const Batch<R>& b = a.b;
  constexpr int K = U<R>::K, JB = 8;
  c128* h64 = reinterpret_cast<c128*>(sm);
  c128* scratch = h64 + (GDR_MAX_M + 2);
  cx<R>* hs = reinterpret_cast<cx<R>*>(scratch + ST);
  double* red = reinterpret_cast<double*>(hs + (GDR_MAX_M + 2));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long it = blockIdx.x; it < (long)b.ncol * a.NU; it += gridDim.x) {
    const int c = (int)(it / a.NU), ub = (int)(it % a.NU);
    if (!ldcg_int(&b.st[c].run)) continue;
    const long n = b.nvec ? (long)b.nvec[c] : b.n, nu = nunits<R>(n);
    const cx<R>* V = b.V + c * b.vcs;
    cx<R>* w = b.W2 + c * b.wcs;
    __syncthreads();
    reduce_slots(a.partB + c * a.pstride, a.hs, a.S, nv, h64, scratch);
    for (int i = threadIdx.x; i < nv; i += ST) hs[i] = cvt<R>(h64[i]);
    if (ub == 0)
      for (int i = threadIdx.x; i < nv; i += ST) b.h2[(long)c * (b.m + 2) + i] = h64[i];
    __syncthreads();
    double nrm = 0.0;
    for (long u = (long)ub * ST + threadIdx.x; u < nu; u += (long)a.NU * ST) {
      cx<R> acc[K];
      ldu_cg<R>(w, u, n, acc);
      for (int g0 = 0; g0 < nv; g0 += JB) {
        cx<R> vv[JB][K];
#pragma unroll
        for (int qq = 0; qq < JB; ++qq)
          if (g0 + qq < nv) ldu_cg<R>(V + (long)(g0 + qq) * b.ldv, u, n, vv[qq]);
#pragma unroll
        for (int qq = 0; qq < JB; ++qq) {
          if (g0 + qq < nv) {
            const cx<R> hi = hs[g0 + qq];
#pragma unroll
            for (int kk = 0; kk < K; ++kk) acc[kk] -= vv[qq][kk] * hi;
          }
        }
      }
      stu<R>(w, u, n, acc);
      R q = 0;
#pragma unroll
      for (int kk = 0; kk < K; ++kk) q += norm2(acc[kk]);
      nrm += (double)q;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(FULL, nrm, off);
    if (lane == 0) red[warp] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int q = 0; q < ST / 32; ++q) s += red[q];
      a.partA[c * a.pstride + (long)ub * a.hs] = {s, 0.0};
    }
  }
}

// ---------------------------------------------------------------- phase F
template <typename R>
DEV void phase_finish(const SweepArgs<R>& a, int j) {
  const Batch<R>& b = a.b;
  const int nv = j + 1, m = b.m, hsz = m + 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // one warp per column
  for (long it = (long)blockIdx.x * (ST / 32) + warp; it < b.ncol; it += (long)gridDim.x * (ST / 32)) {
    const int c = (int)it;
    ColState& st = b.st[c];
    if (!ldcg_int(&st.run)) continue;
    c128 s = {0, 0};
    for (int q = lane; q < a.NU; q += 32) s += ldcg_c128(a.partA + c * a.pstride + (long)q * a.hs);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s.x += __shfl_xor_sync(FULL, s.x, off);
    const double wn = sqrt(s.x);
    c128* Hc = b.H + (long)c * (m + 1) * m + (long)j * (m + 1);
    for (int i = lane; i < nv; i += 32)
      Hc[i] = ldcg_c128(b.h1 + (long)c * hsz + i) + ldcg_c128(b.h2 + (long)c * hsz + i);
    if (lane == 0) {
      Hc[nv] = {wn, 0.0};
      const double w0 = sqrt(ldcg_c128(b.h1 + (long)c * hsz + nv).x);
      st.j = j;
      st.wnorm0 = w0;
      if (!isfinite(wn) || !isfinite(w0)) {
        st.nan = 1;
        st.broke = 1;
        st.run = 0;
        st.m_eff = j + 1;
      } else if (wn <= 1e-12 * w0) {
        st.broke = 1;
        st.run = 0;
        st.m_eff = j + 1;
      } else {
        st.inv_norm = 1.0 / wn;
      }
    }
  }
}

template <typename R, typename LT>
__global__ void __launch_bounds__(ST, 2) arnoldi_sweep_kernel(SweepArgs<R> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  bool ok = true;
  unsigned epoch = 0;
  for (int j = a.jstart; j < a.jend && ok; ++j) {
    const bool lazy = j > a.jstart;
    GDR_SWEEP_MARK(j, 0);
    phase_matvec<R, LT>(a, j, lazy, sm);
    ok = grid_sync(a.bar, epoch);
    if (!ok) break;
    GDR_SWEEP_MARK(j, 1);
    phase_dot1<R>(a, j + 1, lazy, sm);
    ok = grid_sync(a.bar, epoch);
    if (!ok) break;
    GDR_SWEEP_MARK(j, 2);
    phase_update_dot<R>(a, j + 1, sm);
    ok = grid_sync(a.bar, epoch);
    if (!ok) break;
    GDR_SWEEP_MARK(j, 3);
    phase_update<R>(a, j + 1, sm);
    ok = grid_sync(a.bar, epoch);
    if (!ok) break;
    GDR_SWEEP_MARK(j, 4);
    phase_finish<R>(a, j);
    ok = grid_sync(a.bar, epoch);
    GDR_SWEEP_MARK(j, 5);
  }
  if (!ok && threadIdx.x == 0)
    for (int c = 0; c < a.b.ncol; ++c) atomicCAS(&a.b.st[c].err, 0, (int)GDR_ETIMEOUT);
}

// Barrier self-test: `rounds` grid barriers; with `phantom` one more arrival is
// expected than there are blocks, so the first barrier can only end by its
// spin bound.  Block 0 writes the outcome.
__global__ void barrier_probe_kernel(SweepBar* gb, int rounds, int phantom, int* out) {
  unsigned epoch = 0;
  bool ok = true;
  for (int r = 0; r < rounds && ok; ++r) ok = grid_sync(gb, epoch, gridDim.x + (phantom ? 1u : 0u));
  if (blockIdx.x == 0 && threadIdx.x == 0) *out = ok ? (int)GDR_OK : (int)GDR_ETIMEOUT;
}

template <typename R>
size_t sweep_smem(int kind) {
  constexpr int K = U<R>::K, TU = SDU * 32;
  const size_t dots = sizeof(cx<R>) * TU * K + sizeof(c128) * (2 * (GDR_MAX_M + 2) + ST) +
                      sizeof(cx<R>) * (GDR_MAX_M + 2) + 64;
  const size_t upd = sizeof(c128) * ((GDR_MAX_M + 2) + ST) + sizeof(cx<R>) * (GDR_MAX_M + 2) + 8 * 32 + 64;
  const size_t wil = (kind == OP_WILSON) ? sizeof(cx<R>) * 8 * 32 * 13 : 0;
  return std::max(dots, std::max(upd, wil));
}

template <typename R, typename LT>
int sweep_occupancy(size_t smem) {
  auto kern = arnoldi_sweep_kernel<R, LT>;
  GDR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int nb = 0;
  GDR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, ST, smem));
  return nb;
}

template <typename R, typename LT>
void launch_sweep(gdr_ctx* ctx, const SweepArgs<R>& a, int grid, size_t smem) {
  void* args[] = {const_cast<SweepArgs<R>*>(&a)};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(ST);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  GDR_CUDA(cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(arnoldi_sweep_kernel<R, LT>), args));
}

}  // namespace

void sweep_init(gdr_ctx* ctx) {
  // the Wilson layout needs the most shared memory; every launch of an instance uses it
  ctx->sweep_blocks[0] = sweep_occupancy<float, c64>(sweep_smem<float>(OP_WILSON));
  ctx->sweep_blocks[1] = sweep_occupancy<float, __nv_bfloat162>(sweep_smem<float>(OP_WILSON));
  ctx->sweep_blocks[2] = sweep_occupancy<double, c128>(sweep_smem<double>(OP_WILSON));
}

template <typename R>
bool sweep_fits(gdr_ctx* ctx, const gdr_op* A, const Batch<R>& b) {
  const int inst = sizeof(R) == 8 ? 2 : (A->kind == OP_WILSON && A->store == GDR_LINK_BF16 ? 1 : 0);
  if (ctx->sweep_blocks[inst] < 1) return false;
  if (b.m + 2 > GDR_MAX_M + 2) return false;
  // the direction-split Wilson form only, i.e. lattices too small for a thread per site
  if (A->kind == OP_WILSON && (A->V + 127) / 128 * b.ncol >= 2L * ctx->num_sms) return false;
  // short vectors (at most 2^17 elements per column) and the whole batch of bases
  // within half of L2: there launch and barrier latency, not bandwidth, sets the pace
  if (b.n > (1L << 17)) return false;
  return (double)b.ncol * b.n * (b.m + 1) * sizeof(cx<R>) <= 0.5 * (double)ctx->l2_bytes;
}

template <typename R>
void sweep_reserve(gdr_ctx* ctx, const Batch<R>& b) {
  const size_t np = (size_t)b.nblk * (b.m + 2) * b.ncol + 64;
  ctx->get<c128>("sweep.partA", np);
  ctx->get<c128>("sweep.partB", np);
  ctx->get<int>("sweep.bar", 16);
}

template <typename R>
void arnoldi_sweep(gdr_ctx* ctx, const gdr_op* A, const Batch<R>& b, int jstart, int jend) {
  if (jend <= jstart) return;
  SweepArgs<R> a{};
  a.b = b;
  a.kind = A->kind;
  a.n = A->n;
  a.rowptr = A->rowptr;
  a.col = A->col;
  if constexpr (sizeof(R) == 4)
    a.vals = A->vals64;
  else
    a.vals = A->vals128;
  a.rp_off = A->rp_off;
  a.nz_off = A->nz_off;
  a.nrow = A->nrow;
  a.Lx = A->dims[0]; a.Ly = A->dims[1]; a.Lz = A->dims[2]; a.Lt = A->dims[3];
  a.V = A->V;
  a.diag_a = A->diag_a;
  a.jstart = jstart;
  a.jend = jend;
  constexpr long TU = SDU * 32;
  const long nu = nunits<R>(b.n);
  a.S = (int)std::max<long>(1, std::min<long>((nu + TU - 1) / TU, b.nblk));
  a.NU = (int)std::max<long>(1, std::min<long>((nu + ST - 1) / ST, b.nblk));
  a.hs = b.m + 2;
  a.pstride = (long)std::max(a.S, a.NU) * a.hs;
  // reserved by sweep_reserve (no allocation here: this may run under stream capture)
  const size_t np = (size_t)b.nblk * (b.m + 2) * b.ncol + 64;
  a.partA = ctx->get<c128>("sweep.partA", np);
  a.partB = ctx->get<c128>("sweep.partB", np);
  a.bar = reinterpret_cast<SweepBar*>(ctx->get<int>("sweep.bar", 16));
  GDR_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(SweepBar), ctx->stream));
  const bool bf16 = A->kind == OP_WILSON && sizeof(R) == 4 && A->store == GDR_LINK_BF16;
  const int inst = sizeof(R) == 8 ? 2 : (bf16 ? 1 : 0);
  if (A->kind == OP_WILSON) {
    if (bf16)
      a.links = A->links16;
    else if constexpr (sizeof(R) == 4)
      a.links = A->links64;
    else
      a.links = A->links128;
  }
  const size_t smem = sweep_smem<R>(OP_WILSON);
  const int nb = ctx->sweep_blocks[inst];
  GDR_REQUIRE(nb >= 1, "arnoldi_sweep: kernel does not fit on an SM");
  // work items of the widest phase, at most the co-resident blocks
  const long mv_items = A->kind == OP_WILSON ? ((A->V + 31) / 32 + 1) / 2 : (A->n + ST - 1) / ST;
  const long items = (long)b.ncol * std::max<long>(mv_items, std::max<long>((long)a.S * ((jend + 8) / 8), a.NU));
  const int grid = (int)std::max<long>(1, std::min<long>((long)nb * ctx->num_sms, items));
  // algorithmic bytes: per step the matvec, dot (+ v_j store), update+dot and update passes
  double bytes = 0.0;
  {
    const double sv = sizeof(cx<R>), nn = col_len(b);
    double mv;
    if (A->kind == OP_WILSON) {
      const double sl = sizeof(R) == 8 ? 8 : (bf16 ? 2 : 4);
      mv = (double)A->V * (4 * 18 * sl + (double)b.ncol * 12 * sv * 2);
    } else {
      mv = (double)A->n * 4 + (double)A->nnz * (4 + sv) + nn * sv * 2;
    }
    for (int j = jstart; j < jend; ++j) {
      const double nv = j + 1;
      bytes += mv + nn * sv * ((nv + 1 + (j > jstart ? 2 : 0)) + (nv + 2) + (nv + 2));
    }
  }
  KProf kp(ctx, sizeof(R) == 4 ? "arnoldi_sweep_c64" : "arnoldi_sweep_c128", bytes * run_share(ctx, b));
  if constexpr (sizeof(R) == 4) {
    if (bf16)
      launch_sweep<R, __nv_bfloat162>(ctx, a, grid, smem);
    else
      launch_sweep<R, cx<R>>(ctx, a, grid, smem);
  } else {
    launch_sweep<R, cx<R>>(ctx, a, grid, smem);
  }
  GDR_LAUNCHED(ctx);
}

gdr_status barrier_selftest(gdr_ctx* ctx, int rounds, int phantom) {
  SweepBar* gb = reinterpret_cast<SweepBar*>(ctx->get<int>("probe.bar", 16));
  int* out = ctx->get<int>("probe.out", 4);
  GDR_CUDA(cudaMemsetAsync(gb, 0, sizeof(SweepBar), ctx->stream));
  GDR_CUDA(cudaMemsetAsync(out, 0xff, sizeof(int), ctx->stream));
  int nb = 0;
  GDR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, barrier_probe_kernel, ST, 0));
  GDR_REQUIRE(nb >= 1, "barrier_selftest: kernel does not fit");
  void* args[] = {&gb, &rounds, &phantom, &out};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ctx->num_sms * std::min(nb, 2)));
  cfg.blockDim = dim3(ST);
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  GDR_CUDA(cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(barrier_probe_kernel), args));
  GDR_LAUNCHED(ctx);
  int h = -1;
  GDR_CUDA(cudaMemcpyAsync(&h, out, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GDR_CUDA(cudaStreamSynchronize(ctx->stream));
  return (gdr_status)h;
}

template bool sweep_fits<float>(gdr_ctx*, const gdr_op*, const Batch<float>&);
template bool sweep_fits<double>(gdr_ctx*, const gdr_op*, const Batch<double>&);
template void sweep_reserve<float>(gdr_ctx*, const Batch<float>&);
template void sweep_reserve<double>(gdr_ctx*, const Batch<double>&);
template void arnoldi_sweep<float>(gdr_ctx*, const gdr_op*, const Batch<float>&, int, int);
template void arnoldi_sweep<double>(gdr_ctx*, const gdr_op*, const Batch<double>&, int, int);
