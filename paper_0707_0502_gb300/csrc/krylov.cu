// Krylov-basis kernels: classical Gram-Schmidt twice (CGS2) for the Arnoldi
// recurrence A V_m = V_{m+1} Hbar_m (eq. recurAr / recur0), the fused basis
// combination used by the GMRES-DR restart (eq. recur1) and the multi-shift
// solution updates x_i += V_m d_i (GMRES-DR-Sh step 5), and small vector ops.
//
// Every kernel works on a batch of independent columns (grid.y = column); a
// column whose state says `run == 0` is skipped.  Reductions are
// deterministic: each block writes FP64 partials, the last block to finish
// (atomic ticket) sums them in block order.
#include <type_traits>

#include "kernels.cuh"
#include "vecunits.cuh"

namespace {

constexpr int NT = 256;  // threads of the reduction kernels
constexpr int JB = 8;    // basis vectors per register chunk (update)



DEV c128 ldcg128(const c128* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

// Reduce NV complex values over the block; threads < nvalid write out[t].
template <typename R, int NV>
DEV void block_reduce(cx<R> (&acc)[NV], c128* out, int nvalid) {
  __shared__ c128 sred[NT / 32][NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc[i].x += __shfl_down_sync(FULL, acc[i].x, off);
      acc[i].y += __shfl_down_sync(FULL, acc[i].y, off);
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) sred[warp][i] = up(acc[i]);
  }
  __syncthreads();
  if (threadIdx.x < nvalid) {
    c128 s = {0, 0};
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += sred[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// sum of the partials p[bk * stride], bk < count (default: one per block), by
// one warp (fixed order: lanes stride the partials, then a shuffle tree),
// result valid in every lane
DEV c128 warp_sum_partials(const c128* p, long stride, int lane, int count = -1) {
  if (count < 0) count = (int)gridDim.x;
  c128 s = {0, 0};
  for (int bk = lane; bk < count; bk += 32) s += ldcg128(p + (long)bk * stride);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s.x += __shfl_xor_sync(FULL, s.x, off);
    s.y += __shfl_xor_sync(FULL, s.y, off);
  }
  return s;
}

// true in exactly one block per column: the last one to finish
DEV bool last_block(unsigned* cnt) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(cnt, 1u) == gridDim.x - 1);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Two-level deterministic sum of the per-slot partials part[s * hs + i] (s < S,
// i < nval) into out[i].  Slots come in groups of RG; the last block to finish
// writing a group's slots (`nblk_group` blocks write into it) sums them, one
// thread per value, into gpart[g * hs + i]; the last group sums the group results.
// FP64 adds are costly on this GPU, so no single block sums all S partials.
// Returns true in the one block that wrote `out` (its threads see `out` after a
// __syncthreads()).
constexpr int RG = 16;
DEV bool reduce2(const c128* part, c128* gpart, int hs, int S, int nval, unsigned* gcnt, unsigned* tcnt, int group,
                 unsigned nblk_group, c128* out) {
  __shared__ bool last_g, last_t;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_g = (atomicAdd(&gcnt[group], 1u) == nblk_group - 1);
  __syncthreads();
  if (!last_g) return false;
  __threadfence();
  const int s0 = group * RG, s1 = min(S, s0 + RG);
  for (int i = threadIdx.x; i < nval; i += NT) {
    c128 acc = {0, 0};
    for (int q = s0; q < s1; ++q) acc += ldcg128(part + (long)q * hs + i);
    gpart[(long)group * hs + i] = acc;
  }
  __threadfence();
  __syncthreads();
  const int ng = (S + RG - 1) / RG;
  if (threadIdx.x == 0) {
    gcnt[group] = 0;
    last_t = (atomicAdd(tcnt, 1u) == (unsigned)ng - 1);
  }
  __syncthreads();
  if (!last_t) return false;
  __threadfence();
  for (int i = threadIdx.x; i < nval; i += NT) {
    c128 acc = {0, 0};
    for (int g = 0; g < ng; ++g) acc += ldcg128(gpart + (long)g * hs + i);
    out[i] = acc;
  }
  if (threadIdx.x == 0) *tcnt = 0;
  return true;
}

// ------------------------------------------------------------ Gram-Schmidt

// h = V^H w (+ ||w||^2): a block stages a tile of w in shared memory, each warp
// takes whole basis vectors and its lanes stream DU units of that vector
// (coalesced, DU loads in flight per lane); one warp reduction per (vector,
// tile), accumulated in FP64.  The grid is S tile slots x G vector groups: the
// block (slot, group) takes the tiles t = slot (mod S) for the vectors of its
// group, and writes one partial per (slot, vector).  Long vectors use G = 1
// (w and V each read once); short ones, with fewer tiles than blocks, split the
// vectors of a tile over G blocks (w re-read G times from L2).

template <typename R>
__global__ void __launch_bounds__(NT, 3) gs_dot_kernel(Batch<R> b, int nv, const cx<R>* __restrict__ W, long wcs,
                                                    c128* __restrict__ hout, int hstride, int wnorm, int S, int G,
                                                    const cx<R>* __restrict__ Wprev) {
  const int c = blockIdx.y;
  if (!b.st[c].run) return;
  constexpr int K = U<R>::K;
  constexpr int DU = DotTile<R>::DU;
  constexpr int TU = DU * 32;  // units per tile
  __shared__ cx<R> wt[TU * K];
  __shared__ c128 accs[GDR_MAX_M + 2];
  const cx<R>* __restrict__ V = b.V + (c / b.vpp) * b.vcs;
  const cx<R>* __restrict__ w = W + c * wcs;
  const long n = b.nvec ? (long)b.nvec[c] : b.n, nu = nunits<R>(n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nvec_tot = nv + (wnorm ? 1 : 0);
  const int slot = blockIdx.x % S, grp = blockIdx.x / S;
  const int vpg = (nvec_tot + G - 1) / G;
  const int i0 = grp * vpg, i1 = min(nvec_tot, i0 + vpg);
  for (int i = i0 + threadIdx.x; i < i1; i += NT) accs[i] = {0, 0};
  const long ntiles = (nu + TU - 1) / TU;
  for (long t = slot; t < ntiles && i0 < i1; t += S) {
    const long u0 = t * TU;
    __syncthreads();  // readers of the previous tile are done
    for (int q = threadIdx.x; q < TU; q += NT) {
      cx<R> tmp[K];
      if (u0 + q < nu) {
        ldu<R>(w, u0 + q, n, tmp);
      } else {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) tmp[kk] = {0, 0};
      }
#pragma unroll
      for (int kk = 0; kk < K; ++kk) wt[q * K + kk] = tmp[kk];
    }
    __syncthreads();
    for (int i = i0 + warp; i < i1; i += NT / 32) {
      cx<R> a = {0, 0};
      if (i < nv) {
        // lazy step: v_{nv-1} is the previous step's unnormalised vector; scale it
        // and store it into V while it is read
        const bool lazy = Wprev && i == nv - 1;
        const cx<R>* vi = lazy ? Wprev + c * wcs : V + (long)i * b.ldv;
        cx<R> vv[DU][K];
#pragma unroll
        for (int tt = 0; tt < DU; ++tt) {
          const long u = u0 + lane + 32 * tt;
          if (u < nu) {
            ldu<R>(vi, u, n, vv[tt]);
          } else {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) vv[tt][kk] = {0, 0};
          }
        }
        if (lazy) {
          const R sc = (R)b.st[c].inv_norm;
          cx<R>* vo = b.V + c * b.vcs + (long)i * b.ldv;
#pragma unroll
          for (int tt = 0; tt < DU; ++tt) {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) vv[tt][kk] = sc * vv[tt][kk];
            const long u = u0 + lane + 32 * tt;
            if (u < nu) stu<R>(vo, u, n, vv[tt]);
          }
        }
#pragma unroll
        for (int tt = 0; tt < DU; ++tt)
#pragma unroll
          for (int kk = 0; kk < K; ++kk) a += cmulc(vv[tt][kk], wt[(lane + 32 * tt) * K + kk]);
      } else {  // ||w||^2
#pragma unroll
        for (int tt = 0; tt < DU; ++tt)
#pragma unroll
          for (int kk = 0; kk < K; ++kk) a.x += norm2(wt[(lane + 32 * tt) * K + kk]);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        a.x += __shfl_xor_sync(FULL, a.x, off);
        a.y += __shfl_xor_sync(FULL, a.y, off);
      }
      if (lane == 0) accs[i] += up(a);
    }
  }
  __syncthreads();
  c128* part = b.part + c * b.pstride;
  for (int i = i0 + threadIdx.x; i < i1; i += NT) part[(long)slot * hstride + i] = accs[i];
  const int rg = slot / RG;
  const unsigned nbg = (unsigned)(min(S, (rg + 1) * RG) - rg * RG) * (unsigned)G;
  reduce2(part, part + (long)b.nblk * hstride, hstride, S, nvec_tot, b.gcnt + 64 * c, b.cnt + 4 * c + 1, rg, nbg,
          hout + (long)c * hstride);
}

// First CGS2 update fused with the second projection: per tile, w' = w - V h
// (all nv vectors; written to Wout by the group-0 block of the tile and staged
// in shared memory), then hout = V^H w' for the block's group of vectors, with
// the tile slot / vector group grid and the partials of gs_dot_kernel.  V is
// read once from HBM for both (the dot re-reads the tile from L1/L2).
template <typename R>
__global__ void __launch_bounds__(NT, 2) gs_update_dot_kernel(Batch<R> b, int nv, const cx<R>* __restrict__ W,
                                                           cx<R>* __restrict__ Wout, long wcs,
                                                           const c128* __restrict__ h, c128* __restrict__ hout,
                                                           int hstride, int S, int G) {
  const int c = blockIdx.y;
  if (!b.st[c].run) return;
  constexpr int K = U<R>::K;
  constexpr int DU = DotTile<R>::DU;
  constexpr int TU = DU * 32;
  __shared__ cx<R> wt[TU * K];
  __shared__ cx<R> hs[GDR_MAX_M + 2];
  __shared__ c128 accs[GDR_MAX_M + 2];
  const cx<R>* __restrict__ V = b.V + c * b.vcs;
  const cx<R>* __restrict__ w = W + c * wcs;
  cx<R>* __restrict__ wo = Wout + c * wcs;
  const long n = b.nvec ? (long)b.nvec[c] : b.n, nu = nunits<R>(n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = blockIdx.x % S, grp = blockIdx.x / S;
  const int vpg = (nv + G - 1) / G;
  const int i0 = grp * vpg, i1 = min(nv, i0 + vpg);
  for (int i = threadIdx.x; i < nv; i += NT) hs[i] = cvt<R>(h[(long)c * hstride + i]);
  for (int i = i0 + threadIdx.x; i < i1; i += NT) accs[i] = {0, 0};
  const long ntiles = (nu + TU - 1) / TU;
  for (long t = slot; t < ntiles; t += S) {
    const long u0 = t * TU;
    __syncthreads();  // hs ready; readers of the previous tile are done
    for (int q = threadIdx.x; q < TU; q += NT) {
      const long u = u0 + q;
      cx<R> acc[K];
      if (u < nu) {
        ldu<R>(w, u, n, acc);
        for (int g0 = 0; g0 < nv; g0 += JB) {
          cx<R> vv[JB][K];
#pragma unroll
          for (int qq = 0; qq < JB; ++qq)
            if (g0 + qq < nv) ldu<R>(V + (long)(g0 + qq) * b.ldv, u, n, vv[qq]);
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
    for (int i = i0 + warp; i < i1; i += NT / 32) {
      const cx<R>* vi = V + (long)i * b.ldv;
      cx<R> a = {0, 0};
      // the tile in two halves (DU/2 loads in flight per lane; the tile is in L1/L2)
#pragma unroll
      for (int t0 = 0; t0 < DU; t0 += DU / 2) {
        cx<R> vv[DU / 2][K];
#pragma unroll
        for (int tt = 0; tt < DU / 2; ++tt) {
          const long u = u0 + lane + 32 * (t0 + tt);
          if (u < nu) {
            ldu<R>(vi, u, n, vv[tt]);
          } else {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) vv[tt][kk] = {0, 0};
          }
        }
#pragma unroll
        for (int tt = 0; tt < DU / 2; ++tt)
#pragma unroll
          for (int kk = 0; kk < K; ++kk) a += cmulc(vv[tt][kk], wt[(lane + 32 * (t0 + tt)) * K + kk]);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        a.x += __shfl_xor_sync(FULL, a.x, off);
        a.y += __shfl_xor_sync(FULL, a.y, off);
      }
      if (lane == 0) accs[i] += up(a);
    }
  }
  __syncthreads();
  c128* part = b.part + c * b.pstride;
  for (int i = i0 + threadIdx.x; i < i1; i += NT) part[(long)slot * hstride + i] = accs[i];
  const int rg = slot / RG;
  const unsigned nbg = (unsigned)(min(S, (rg + 1) * RG) - rg * RG) * (unsigned)G;
  reduce2(part, part + (long)b.nblk * hstride, hstride, S, nv, b.gcnt + 64 * c, b.cnt + 4 * c + 1, rg, nbg,
          hout + (long)c * hstride);
}

template <typename R>
__global__ void __launch_bounds__(NT) gs_update_kernel(Batch<R> b, int nv, cx<R>* __restrict__ W, long wcs,
                                                       const c128* __restrict__ h, int hstride, int final_step) {
  const int c = blockIdx.y;
  if (!b.st[c].run) return;
  constexpr int K = U<R>::K;
  __shared__ cx<R> hs[GDR_MAX_M + 2];
  for (int i = threadIdx.x; i < nv; i += NT) hs[i] = cvt<R>(h[(long)c * hstride + i]);
  __syncthreads();
  const cx<R>* __restrict__ V = b.V + c * b.vcs;
  cx<R>* __restrict__ w = W + c * wcs;
  const long n = b.nvec ? (long)b.nvec[c] : b.n, nu = nunits<R>(n);
  const long gt = blockIdx.x * (long)NT + threadIdx.x, gs = (long)gridDim.x * NT;
  cx<R> nrm[1] = {{0, 0}};
  for (long u = gt; u < nu; u += gs) {
    cx<R> acc[K];
    ldu<R>(w, u, n, acc);
    // basis vectors in groups of JB: all loads of a group are in flight together
    for (int i0 = 0; i0 < nv; i0 += JB) {
      cx<R> vv[JB][K];
#pragma unroll
      for (int q = 0; q < JB; ++q) {
        if (i0 + q < nv) ldu<R>(V + (long)(i0 + q) * b.ldv, u, n, vv[q]);
      }
#pragma unroll
      for (int q = 0; q < JB; ++q) {
        if (i0 + q < nv) {
          const cx<R> hi = hs[i0 + q];
#pragma unroll
          for (int kk = 0; kk < K; ++kk) acc[kk] -= vv[q][kk] * hi;
        }
      }
    }
    stu<R>(w, u, n, acc);
#pragma unroll
    for (int kk = 0; kk < K; ++kk) nrm[0].x += norm2(acc[kk]);
  }
  if (!final_step) return;
  c128* part = b.part + c * b.pstride;
  block_reduce<R, 1>(nrm, part + (long)blockIdx.x * hstride, 1);
  if (!last_block(b.cnt + 4 * c)) return;
  __shared__ double wn_s;
  if (threadIdx.x < 32) {
    const c128 s = warp_sum_partials(part, hstride, threadIdx.x);
    if (threadIdx.x == 0) wn_s = sqrt(s.x);
  }
  __syncthreads();
  const double wn = wn_s;
  const int j = nv - 1;
  const int m = b.m;
  c128* Hc = b.H + (long)c * (m + 1) * m + (long)j * (m + 1);
  for (int i = threadIdx.x; i < nv; i += NT) Hc[i] = b.h1[(long)c * hstride + i] + b.h2[(long)c * hstride + i];
  if (threadIdx.x == 0) {
    Hc[nv] = {wn, 0.0};
    ColState& st = b.st[c];
    const double w0 = sqrt(b.h1[(long)c * hstride + nv].x);
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
    b.cnt[4 * c] = 0;
  }
}

// ------------------------------------------- delayed reorthogonalisation (DCGS2)
//
// Arnoldi with classical Gram-Schmidt whose second (re)orthogonalisation pass is
// delayed by one step and merged into the next step's projection, so a step reads
// the basis twice (one dot pass, one update pass) instead of four times.  At step j
// the basis v_0..v_{j-1} is final and u (the provisional v_j) is orthogonalised once
// and unnormalised, with A v_{j-1} = V_j Hbar[0:j, j-1] + u.  With w = A u, one pass
// gives s = V_j^H u, z = V_j^H w, omega = u^H u, zeta = u^H w; then
//   nu = sqrt(omega - |s|^2),  v_j = (u - V_j s) / nu,
//   Hbar[0:j, j-1] += s,  Hbar[j, j-1] = nu                (the delayed pass for step j-1)
//   t = (zeta - s^H z) / nu,  Hbar[0:j+1, j] = ([z ; t] - Hbar[0:j+1, 0:j] s) / nu
//   u' = (w - V_j z - t v_j) / nu = (w - V_j (z - (t/nu) s) - (t/nu) u) / nu,
// u' being the next step's provisional vector (A v_j = V_{j+1} Hbar[0:j+1, j] + u').
// The first step of a cycle starts from a final v_j (s = 0, nu = 1); after the last
// step a finalising pass (dot + update without w) makes v_m from u.  Lucky breakdown
// of step j-1 (nu <= 1e-12 ||A v_{j-1}||) is detected at step j: m_eff = j.
//
// Dot pass values per column at hd + c * (2m + 8): [s_i, z_i] interleaved (i < j),
// then omega, zeta, w^H w.  Coefficients of the update pass at dc + c * (2m + 8):
// a = s (m+1 slots), b = z - (t/nu) s (m+1 slots), t/nu, 1/nu.

constexpr int DC_FIRST = 1, DC_FINAL = 2;

template <typename R>
__global__ void __launch_bounds__(NT, 3) dcgs2_dot_kernel(Batch<R> b, int j, const cx<R>* __restrict__ Uv, long ucs,
                                                       const cx<R>* __restrict__ W, long wcs, int S, int G,
                                                       int mode) {
  const int c = blockIdx.y;
  if (!b.st[c].run) return;
  constexpr int K = U<R>::K;
  // two staged vectors: half the complex64 tile of gs_dot_kernel keeps 3 blocks per SM
  constexpr int DU = sizeof(R) == 4 ? DotTile<R>::DU / 2 : DotTile<R>::DU;
  constexpr int TU = DU * 32;
  __shared__ cx<R> ut[TU * K];
  __shared__ cx<R> wt[TU * K];
  __shared__ c128 accs[2 * GDR_MAX_M + 8];
  const bool hasw = mode != DC_FINAL;
  const cx<R>* __restrict__ V = b.V + c * b.vcs;
  const cx<R>* __restrict__ u = Uv + c * ucs;
  const cx<R>* __restrict__ w = W + c * wcs;
  const long n = b.nvec ? (long)b.nvec[c] : b.n, nu = nunits<R>(n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nvec_tot = j + 1;  // j basis vectors and the self terms
  const int slot = blockIdx.x % S, grp = blockIdx.x / S;
  const int vpg = (nvec_tot + G - 1) / G;
  const int i0 = grp * vpg, i1 = min(nvec_tot, i0 + vpg);
  const int hs = 2 * b.m + 8;
  const int v0 = 2 * i0, v1 = 2 * i1 + (i1 == nvec_tot ? 1 : 0);  // value range of this block
  for (int i = v0 + threadIdx.x; i < v1; i += NT) accs[i] = {0, 0};
  const long ntiles = (nu + TU - 1) / TU;
  for (long t = slot; t < ntiles && i0 < i1; t += S) {
    const long u0 = t * TU;
    __syncthreads();  // readers of the previous tile are done
    for (int q = threadIdx.x; q < TU; q += NT) {
      cx<R> tu[K], tw[K];
      if (u0 + q < nu) {
        ldu<R>(u, u0 + q, n, tu);
        if (hasw) ldu<R>(w, u0 + q, n, tw);
      }
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        if (u0 + q >= nu) tu[kk] = {0, 0};
        if (u0 + q >= nu || !hasw) tw[kk] = {0, 0};
        ut[q * K + kk] = tu[kk];
        wt[q * K + kk] = tw[kk];
      }
    }
    __syncthreads();
    for (int i = i0 + warp; i < i1; i += NT / 32) {
      cx<R> au = {0, 0}, aw = {0, 0}, ww = {0, 0};
      if (i < j) {
        const cx<R>* vi = V + (long)i * b.ldv;
        cx<R> vv[DU][K];
#pragma unroll
        for (int tt = 0; tt < DU; ++tt) {
          const long uu = u0 + lane + 32 * tt;
          if (uu < nu) {
            ldu<R>(vi, uu, n, vv[tt]);
          } else {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) vv[tt][kk] = {0, 0};
          }
        }
#pragma unroll
        for (int tt = 0; tt < DU; ++tt)
#pragma unroll
          for (int kk = 0; kk < K; ++kk) {
            au += cmulc(vv[tt][kk], ut[(lane + 32 * tt) * K + kk]);
            aw += cmulc(vv[tt][kk], wt[(lane + 32 * tt) * K + kk]);
          }
      } else {  // omega = u^H u (au.x), zeta = u^H w (aw), w^H w (ww.x)
#pragma unroll
        for (int tt = 0; tt < DU; ++tt)
#pragma unroll
          for (int kk = 0; kk < K; ++kk) {
            const cx<R> a = ut[(lane + 32 * tt) * K + kk], bw = wt[(lane + 32 * tt) * K + kk];
            au.x += norm2(a);
            aw += cmulc(a, bw);
            ww.x += norm2(bw);
          }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        au.x += __shfl_xor_sync(FULL, au.x, off);
        au.y += __shfl_xor_sync(FULL, au.y, off);
        aw.x += __shfl_xor_sync(FULL, aw.x, off);
        aw.y += __shfl_xor_sync(FULL, aw.y, off);
        ww.x += __shfl_xor_sync(FULL, ww.x, off);
      }
      if (lane == 0) {
        accs[2 * i] += up(au);
        accs[2 * i + 1] += up(aw);
        if (i == j) accs[2 * i + 2] += up(ww);
      }
    }
  }
  __syncthreads();
  c128* part = b.part + c * b.pstride;
  for (int i = v0 + threadIdx.x; i < v1; i += NT) part[(long)slot * hs + i] = accs[i];
  const int rg = slot / RG;
  const unsigned nbg = (unsigned)(min(S, (rg + 1) * RG) - rg * RG) * (unsigned)G;
  c128* hv = b.hd + (long)c * hs;
  if (!reduce2(part, part + (long)b.nblk * hs, hs, S, 2 * j + 3, b.gcnt + 64 * c, b.cnt + 4 * c + 1, rg, nbg, hv))
    return;
  __syncthreads();

  // ---- coefficients (the block that holds the sums; FP64 except the small H s correction)
  __shared__ c128 ssh[GDR_MAX_M + 2];
  __shared__ double red_d[NT / 32];
  __shared__ c128 red_c[NT / 32];
  __shared__ double nu_s;
  __shared__ int brk_s;
  const int m = b.m;
  const bool first = mode == DC_FIRST;
  c128 szp = {0, 0};
  double ssp = 0;
  for (int i = threadIdx.x; i < j; i += NT) {
    const c128 si = first ? c128{0, 0} : hv[2 * i];
    ssh[i] = si;
    ssp += norm2(si);
    szp += cmulc(si, hv[2 * i + 1]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ssp += __shfl_xor_sync(FULL, ssp, off);
    szp.x += __shfl_xor_sync(FULL, szp.x, off);
    szp.y += __shfl_xor_sync(FULL, szp.y, off);
  }
  if (lane == 0) {
    red_d[warp] = ssp;
    red_c[warp] = szp;
  }
  __syncthreads();
  ColState& st = b.st[c];
  c128* H = b.H + (long)c * (m + 1) * m;
  c128* dc = b.dc + (long)c * hs;
  if (threadIdx.x == 0) {
    double ss = 0;
    c128 sz = {0, 0};
    for (int q = 0; q < NT / 32; ++q) {
      ss += red_d[q];
      sz += red_c[q];
    }
    const double omega = hv[2 * j].x;
    double nuv = first ? 1.0 : sqrt(fmax(omega - ss, 0.0));
    int brk = 0;
    if (!first) {
      if (!isfinite(nuv) || !isfinite(omega)) {
        st.nan = 1;
        brk = 1;
      } else if (nuv <= 1e-12 * st.wnorm0) {
        brk = 1;
      }
      H[(long)(j - 1) * (m + 1) + j] = {nuv, 0.0};
      if (brk) {
        st.broke = 1;
        st.run = 0;
        st.m_eff = j;
      }
    }
    if (!brk) {
      st.inv_norm = 1.0 / nuv;
      st.j = j;
      if (mode != DC_FINAL) {
        const c128 zeta = hv[2 * j + 1];
        const c128 t = (1.0 / nuv) * (zeta - sz);
        dc[2 * (m + 1)] = (1.0 / nuv) * t;  // t / nu
        ssh[GDR_MAX_M + 1] = t;
        const double ww = hv[2 * j + 2].x;
        st.wnorm0 = sqrt(ww) / nuv;
        if (!isfinite(ww)) {
          st.nan = 1;
          st.broke = 1;
          st.run = 0;
          st.m_eff = j + 1;
          brk = 1;
        }
      }
      dc[2 * (m + 1) + 1] = {1.0 / nuv, 0.0};
    }
    nu_s = nuv;
    brk_s = brk;
  }
  __syncthreads();
  if (brk_s) return;
  const double nuv = nu_s;
  // the delayed pass completes column j-1
  if (!first)
    for (int i = threadIdx.x; i < j; i += NT) H[(long)(j - 1) * (m + 1) + i] += ssh[i];
  for (int i = threadIdx.x; i < j; i += NT) dc[i] = ssh[i];
  if (mode == DC_FINAL) return;
  __syncthreads();
  const c128 t = ssh[GDR_MAX_M + 1];
  const c128 tn = (1.0 / nuv) * t;
  for (int i = threadIdx.x; i < j; i += NT) dc[(m + 1) + i] = hv[2 * i + 1] - tn * ssh[i];
  // column j: ([z ; t] - Hbar[0:j+1, 0:j] s) / nu; s is O(rounding), so H s in FP32
  for (int i = threadIdx.x; i <= j; i += NT) {
    c64 hsum = {0.f, 0.f};
    if (!first)
      for (int l = 0; l < j; ++l) hsum += to64(H[(long)l * (m + 1) + i]) * to64(ssh[l]);
    const c128 zi = (i < j) ? hv[2 * i + 1] : t;
    H[(long)j * (m + 1) + i] = (1.0 / nuv) * (zi - to128(hsum));
  }
}

// DCGS2 update pass of step j (every unit of every running column):
//   v_j = (u - V_j a) / nu      into V[:, j]   (not on the first step: v_j is final)
//   u'  = (w - V_j b - (t/nu) u) / nu  into Unew (may alias u; not on the finalising pass)
template <typename R>
__global__ void __launch_bounds__(NT) dcgs2_update_kernel(Batch<R> b, int j, const cx<R>* Uv, long ucs,
                                                          const cx<R>* __restrict__ W, cx<R>* Unew, int mode) {
  const int c = blockIdx.y;
  if (!b.st[c].run) return;
  constexpr int K = U<R>::K;
  const int m = b.m, hs = 2 * m + 8;
  __shared__ cx<R> sa[GDR_MAX_M + 1], sb[GDR_MAX_M + 1];
  __shared__ cx<R> tnu_s;
  __shared__ R inu_s;
  const c128* dc = b.dc + (long)c * hs;
  const bool first = mode == DC_FIRST, fin = mode == DC_FINAL;
  for (int i = threadIdx.x; i < j; i += NT) {
    sa[i] = cvt<R>(dc[i]);
    sb[i] = cvt<R>(dc[(m + 1) + i]);
  }
  if (threadIdx.x == 0) {
    tnu_s = fin ? cx<R>{0, 0} : cvt<R>(dc[2 * (m + 1)]);
    inu_s = (R)dc[2 * (m + 1) + 1].x;
  }
  __syncthreads();
  const cx<R> tnu = tnu_s;
  const R inu = inu_s;
  const cx<R>* __restrict__ V = b.V + c * b.vcs;
  const cx<R>* u = Uv + c * ucs;
  const cx<R>* __restrict__ w = W + c * b.wcs;
  cx<R>* un = Unew + c * b.wcs;
  cx<R>* vj = b.V + c * b.vcs + (long)j * b.ldv;
  const long n = b.nvec ? (long)b.nvec[c] : b.n, nu = nunits<R>(n);
  const long gt = blockIdx.x * (long)NT + threadIdx.x, gs = (long)gridDim.x * NT;
  for (long q = gt; q < nu; q += gs) {
    cx<R> uu[K], acc_a[K], acc_b[K];
    ldu<R>(u, q, n, uu);
    if (!fin) {
      ldu<R>(w, q, n, acc_b);
    } else {
#pragma unroll
      for (int kk = 0; kk < K; ++kk) acc_b[kk] = {0, 0};
    }
#pragma unroll
    for (int kk = 0; kk < K; ++kk) acc_a[kk] = uu[kk];
    for (int g0 = 0; g0 < j; g0 += JB) {
      cx<R> vv[JB][K];
#pragma unroll
      for (int qq = 0; qq < JB; ++qq)
        if (g0 + qq < j) ldu<R>(V + (long)(g0 + qq) * b.ldv, q, n, vv[qq]);
#pragma unroll
      for (int qq = 0; qq < JB; ++qq) {
        if (g0 + qq < j) {
          const cx<R> ai = sa[g0 + qq], bi = sb[g0 + qq];
#pragma unroll
          for (int kk = 0; kk < K; ++kk) {
            if (!first) acc_a[kk] -= vv[qq][kk] * ai;
            if (!fin) acc_b[kk] -= vv[qq][kk] * bi;
          }
        }
      }
    }
    if (!first) {
#pragma unroll
      for (int kk = 0; kk < K; ++kk) acc_a[kk] = inu * acc_a[kk];
      stu<R>(vj, q, n, acc_a);
    }
    if (!fin) {
#pragma unroll
      for (int kk = 0; kk < K; ++kk) acc_b[kk] = inu * (acc_b[kk] - tnu * uu[kk]);
      stu<R>(un, q, n, acc_b);
    }
  }
}

template <typename R>
__global__ void scale_kernel(Batch<R> b, int j, const cx<R>* __restrict__ W, long wcs) {
  const int c = blockIdx.y;
  if (!b.st[c].run) return;
  constexpr int K = U<R>::K;
  const long n = b.nvec ? (long)b.nvec[c] : b.n, nu = nunits<R>(n);
  const R s = (R)b.st[c].inv_norm;
  const cx<R>* w = W + c * wcs;
  cx<R>* v = b.V + c * b.vcs + (long)j * b.ldv;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < nu; u += (long)gridDim.x * blockDim.x) {
    cx<R> a[K];
    ldu<R>(w, u, n, a);
#pragma unroll
    for (int kk = 0; kk < K; ++kk) a[kk] = s * a[kk];
    stu<R>(v, u, n, a);
  }
}

// ||x_c||^2 with FP64 block partials; result written by the last block
template <typename T> struct Real;
template <> struct Real<c64> { using R = float; };
template <> struct Real<c128> { using R = double; };

template <typename T>
__global__ void __launch_bounds__(NT) norms2_kernel(long n, const T* __restrict__ x, long xcs, double* out,
                                                    c128* part, unsigned* cnt, const int* nvec) {
  using R = typename Real<T>::R;
  const int c = blockIdx.y;
  if (nvec) n = nvec[c];
  const T* xc = x + c * xcs;
  cx<R> a[1] = {{0, 0}};
  // FP64 per-thread accumulation for accuracy of ||b||
  double s = 0;
  for (long i = blockIdx.x * (long)NT + threadIdx.x; i < n; i += (long)gridDim.x * NT) {
    const T v = xc[i];
    s += (double)v.x * v.x + (double)v.y * v.y;
  }
  c128 d[1] = {{s, 0}};
  block_reduce<double, 1>(d, part + (long)c * gridDim.x + blockIdx.x, 1);
  (void)a;
  if (!last_block(cnt + 4 * c)) return;
  if (threadIdx.x < 32) {
    const c128 t = warp_sum_partials(part + (long)c * gridDim.x, 1, threadIdx.x);
    if (threadIdx.x == 0) {
      out[c] = t.x;
      cnt[4 * c] = 0;
    }
  }
}

__global__ void __launch_bounds__(NT) dots128_kernel(long n, const c128* __restrict__ u, long ucs,
                                                     const c128* __restrict__ x, long xcs, c128* out, c128* part,
                                                     unsigned* cnt) {
  const int c = blockIdx.y;
  const c128* uc = u + c * ucs;
  const c128* xc = x + c * xcs;
  c128 a[1] = {{0, 0}};
  for (long i = blockIdx.x * (long)NT + threadIdx.x; i < n; i += (long)gridDim.x * NT) a[0] += cmulc(uc[i], xc[i]);
  block_reduce<double, 1>(a, part + (long)c * gridDim.x + blockIdx.x, 1);
  if (!last_block(cnt + 4 * c)) return;
  if (threadIdx.x < 32) {
    const c128 t = warp_sum_partials(part + (long)c * gridDim.x, 1, threadIdx.x);
    if (threadIdx.x == 0) {
      out[c] = t;
      cnt[4 * c] = 0;
    }
  }
}

// start of a cycle: V[:,0] = r / ||r||  (||r||^2 in rn2[c])
template <typename R>
__global__ void start_scale_kernel(Batch<R> b, const cx<R>* __restrict__ r, long rcs, const double* rn2) {
  const int c = blockIdx.y;
  if (!b.st[c].active) return;
  const double rn = sqrt(rn2[c]);
  if (!(rn > 0)) return;
  const R s = (R)(1.0 / rn);
  const cx<R>* rc = r + c * rcs;
  cx<R>* v = b.V + c * b.vcs;
  const long n = b.nvec ? (long)b.nvec[c] : b.n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    v[i] = s * rc[i];
}

template <typename R>
__global__ void start_state_kernel(Batch<R> b, const double* rn2) {
  const int c = blockIdx.x;
  const int m = b.m;
  c128* H = b.H + (long)c * (m + 1) * m;
  for (long i = threadIdx.x; i < (long)(m + 1) * m; i += blockDim.x) H[i] = {0, 0};
  c128* cv = b.cvec + (long)c * (m + 1);
  const double rn = sqrt(rn2[c]);
  for (int i = threadIdx.x; i <= m; i += blockDim.x) cv[i] = {i == 0 ? rn : 0.0, 0.0};
  if (threadIdx.x == 0) {
    ColState& st = b.st[c];
    st.broke = 0;
    st.m_eff = m;
    st.rnorm = rn;
    if (!isfinite(rn)) st.nan = 1;
    // a zero residual needs no cycle
    st.run = (st.active && rn > 0 && isfinite(rn)) ? 1 : 0;
  }
}

// ------------------------------------------------------ basis combination

constexpr int CT = 256;  // threads
constexpr int CR = 64;   // rows per tile

template <typename R>
__global__ void __launch_bounds__(CT) combine_kernel(long n, cx<R>* V, long ldv, long vcs, int nv,
                                                     const c128* __restrict__ C, int ldc, long ccs, int nout, int nx,
                                                     int rmode, c128* X, long ldx, long xcs, cx<R>* Rv, long rcs,
                                                     const ColState* st, const int* nvec, int vpp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = blockIdx.y;
  if (st && !st[c].active) return;
  if (nvec) n = nvec[c];
  if ((long)blockIdx.x * CR >= n) return;
  const int ntot = nout + nx + (rmode ? 1 : 0);
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);             // CR x nv  (row-fast)
  cx<R>* cf = tile + (long)CR * nv;                              // nv x ntot
  cx<R>* Vc = V + (c / vpp) * vcs;                               // basis of column c (nout == 0 when shared)
  const c128* Cc = C + c * ccs;
  const long r0 = blockIdx.x * (long)CR;
  const int rows = (int)min((long)CR, n - r0);
  for (int t = threadIdx.x; t < nv * ntot; t += CT) {
    const int i = t % nv, o = t / nv;
    cf[t] = cvt<R>(Cc[(long)o * ldc + i]);
  }
  for (int t = threadIdx.x; t < CR * nv; t += CT) {
    const int rr = t % CR, i = t / CR;
    tile[t] = (rr < rows) ? Vc[(long)i * ldv + r0 + rr] : cx<R>{0, 0};
  }
  __syncthreads();
  const int rr = threadIdx.x % CR;
  if (rr >= rows) return;
  const long row = r0 + rr;
  for (int o = threadIdx.x / CR; o < ntot; o += CT / CR) {
    cx<R> acc = {0, 0};
    const cx<R>* co = cf + (long)o * nv;
    for (int i = 0; i < nv; ++i) acc += tile[(long)i * CR + rr] * co[i];
    if (o < nout) {
      Vc[(long)o * ldv + row] = acc;
    } else if (o < nout + nx) {
      c128* xp = X + c * xcs + (long)(o - nout) * ldx + row;
      *xp = *xp + up(acc);
    } else {
      cx<R>* rp = Rv + c * rcs + row;
      if (rmode == 1) *rp = acc;
      else *rp = *rp + acc;
    }
  }
}

// -------------------------------------------------------- small vector ops

__global__ void cvt_128_64_kernel(long n, const c128* in, long ics, c64* out, long ocs) {
  const int c = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[c * ocs + i] = to64(in[c * ics + i]);
}
__global__ void cvt_64_128_kernel(long n, const c64* in, long ics, c128* out, long ocs) {
  const int c = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[c * ocs + i] = to128(in[c * ics + i]);
}
__global__ void copy128_kernel(long n, const c128* in, long ics, c128* out, long ocs) {
  const int c = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[c * ocs + i] = in[c * ics + i];
}
__global__ void axpy_cols_kernel(long n, const c128* a, const c128* S, long ssc, c128* X, long xcs) {
  const int c = blockIdx.y;
  const c128 ac = a[c];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    X[c * xcs + i] += ac * S[c * ssc + i];
}
__global__ void scal_cols_kernel(long n, const c128* a, c128* X, long xcs) {
  const int c = blockIdx.y;
  const c128 ac = a[c];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    X[c * xcs + i] = ac * X[c * xcs + i];
}

unsigned grid_for(gdr_ctx* ctx, long work, int threads) {
  long g = (work + threads - 1) / threads;
  long cap = (long)ctx->num_sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

// ------------------------------------------------------------- launchers

double run_share(gdr_ctx* ctx, int ncol, const int* run, int run_stride, const int* nvec) {
  if (!ctx->profile || ncol <= 0 || run == nullptr) return 1.0;
  std::vector<int> rf((size_t)ncol * run_stride), nv(nvec ? ncol : 0);
  GDR_CUDA(cudaMemcpyAsync(rf.data(), run, sizeof(int) * ((size_t)(ncol - 1) * run_stride + 1),
                           cudaMemcpyDeviceToHost, ctx->stream));
  if (nvec) GDR_CUDA(cudaMemcpyAsync(nv.data(), nvec, sizeof(int) * ncol, cudaMemcpyDeviceToHost, ctx->stream));
  GDR_CUDA(cudaStreamSynchronize(ctx->stream));
  double all = 0, on = 0;
  for (int c = 0; c < ncol; ++c) {
    const double len = nvec ? (double)nv[c] : 1.0;
    all += len;
    if (rf[(size_t)c * run_stride]) on += len;
  }
  return all > 0 ? on / all : 1.0;
}

// tile slots S x vector groups G of the dot kernels; S <= nblk bounds the partials
template <typename R>
static void dot_grid(gdr_ctx* ctx, const Batch<R>& b, int nvec, int& S, int& G) {
  constexpr long TU = DotTile<R>::DU * 32;
  const long ntiles = (nunits<R>(b.n) + TU - 1) / TU;
  // as many slots as blocks allow, each slot with the same number of tiles (+-1)
  const long rounds = std::max<long>(1, (ntiles + b.nblk - 1) / b.nblk);
  S = (int)std::max<long>(1, std::min<long>((ntiles + rounds - 1) / rounds, b.nblk));
  const long target = 3L * ctx->num_sms;
  G = 1;
  if (S < target) G = (int)std::min<long>((target + S - 1) / S, (nvec + NT / 32 - 1) / (NT / 32));
  G = std::max(G, 1);
}

template <typename R>
void gs_dot(gdr_ctx* ctx, const Batch<R>& b, int nv, const cx<R>* w, long wcs, c128* h_out, bool wnorm,
            const cx<R>* wprev) {
  int S, G;
  dot_grid(ctx, b, nv + (wnorm ? 1 : 0), S, G);
  dim3 grid((unsigned)(S * G), (unsigned)b.ncol);
  KProf kp(ctx, sizeof(R) == 4 ? "gs_dot_c64" : "gs_dot_c128",
           ((double)nv * basis_len(b) + (wprev ? 2.0 : 1.0) * col_len(b)) * sizeof(cx<R>) * run_share(ctx, b));
  gs_dot_kernel<R><<<grid, NT, 0, ctx->stream>>>(b, nv, w, wcs, h_out, b.m + 2, wnorm ? 1 : 0, S, G, wprev);
  GDR_LAUNCHED(ctx);
}
template <typename R>
void gs_update_dot(gdr_ctx* ctx, const Batch<R>& b, int nv, const cx<R>* w, cx<R>* wout, long wcs, const c128* h,
                   c128* h_out) {
  int S, G;
  dot_grid(ctx, b, nv, S, G);
  dim3 grid((unsigned)(S * G), (unsigned)b.ncol);
  KProf kp(ctx, sizeof(R) == 4 ? "gs_update_dot_c64" : "gs_update_dot_c128",
           (double)(nv + 2) * col_len(b) * sizeof(cx<R>) * run_share(ctx, b));
  gs_update_dot_kernel<R><<<grid, NT, 0, ctx->stream>>>(b, nv, w, wout, wcs, h, h_out, b.m + 2, S, G);
  GDR_LAUNCHED(ctx);
}
template <typename R>
void gs_update(gdr_ctx* ctx, const Batch<R>& b, int nv, cx<R>* w, long wcs, const c128* h, bool final_step) {
  dim3 grid((unsigned)b.nblk, (unsigned)b.ncol);
  KProf kp(ctx, sizeof(R) == 4 ? "gs_update_c64" : "gs_update_c128",
           (double)(nv + 2) * col_len(b) * sizeof(cx<R>) * run_share(ctx, b));
  gs_update_kernel<R><<<grid, NT, 0, ctx->stream>>>(b, nv, w, wcs, h, b.m + 2, final_step ? 1 : 0);
  GDR_LAUNCHED(ctx);
}
template <typename R>
void scale_into(gdr_ctx* ctx, const Batch<R>& b, int j, const cx<R>* w, long wcs) {
  dim3 grid(grid_for(ctx, nunits<R>(b.n), 256), (unsigned)b.ncol);
  KProf kp(ctx, "scale", 2.0 * col_len(b) * sizeof(cx<R>) * run_share(ctx, b));
  scale_kernel<R><<<grid, 256, 0, ctx->stream>>>(b, j, w, wcs);
  GDR_LAUNCHED(ctx);
}

template <typename R>
void arnoldi_step(gdr_ctx* ctx, const gdr_op* A, const Batch<R>& b, int j, int jstart, int jlast, cx<R>*& wlast) {
  const int is = (int)(sizeof(ColState) / sizeof(int)), ds = (int)(sizeof(ColState) / sizeof(double));
  const bool lazy = j > jstart;  // v_j = wlast / h_{j,j-1}, not yet in V
  cx<R>* P = lazy ? wlast : nullptr;
  cx<R>* Wa = (P == b.W) ? b.W2 : b.W;  // receives A v_j
  cx<R>* Wb = (Wa == b.W) ? b.W2 : b.W;  // the other buffer (P itself on a lazy step, free after the first dot)
  if (lazy)
    op_apply_skip(ctx, A, b.ncol, nullptr, P, b.wcs, Wa, b.wcs, nullptr, 0, &b.st[0].run, is, b.cpp,
                  &b.st[0].inv_norm, ds);
  else
    op_apply_skip(ctx, A, b.ncol, nullptr, b.V + (long)j * b.ldv, b.vcs, Wa, b.wcs, nullptr, 0, &b.st[0].run, is,
                  b.cpp);
  gs_dot<R>(ctx, b, j + 1, Wa, b.wcs, b.h1, true, P);
  // fused update + second projection while the basis stays in L2 (its tiles are read
  // twice); separate passes otherwise (each reads V once from HBM)
  const bool fuse = (double)(j + 1) * b.n * sizeof(cx<R>) * b.ncol <= 0.5 * (double)ctx->l2_bytes;
  if (fuse) {
    gs_update_dot<R>(ctx, b, j + 1, Wa, Wb, b.wcs, b.h1, b.h2);
    gs_update<R>(ctx, b, j + 1, Wb, b.wcs, b.h2, true);
    wlast = Wb;
  } else {
    gs_update<R>(ctx, b, j + 1, Wa, b.wcs, b.h1, false);
    gs_dot<R>(ctx, b, j + 1, Wa, b.wcs, b.h2, false);
    gs_update<R>(ctx, b, j + 1, Wa, b.wcs, b.h2, true);
    wlast = Wa;
  }
  if (j == jlast) scale_into<R>(ctx, b, j + 1, wlast, b.wcs);
}

template <typename R>
void arnoldi_dcgs2(gdr_ctx* ctx, const gdr_op* A, const Batch<R>& b, int jstart, int jend) {
  GDR_REQUIRE(b.hd && b.dc, "arnoldi_dcgs2: batch without DCGS2 buffers");
  const int is = (int)(sizeof(ColState) / sizeof(int));
  const double sv = sizeof(cx<R>);
  for (int j = jstart; j <= jend; ++j) {
    const int mode = (j == jend) ? DC_FINAL : (j == jstart ? DC_FIRST : 0);
    // u: the final v_j on the first step, else the provisional vector in W2
    const cx<R>* Uv = (mode == DC_FIRST) ? b.V + (long)j * b.ldv : b.W2;
    const long ucs = (mode == DC_FIRST) ? b.vcs : b.wcs;
    if (mode != DC_FINAL)
      op_apply_skip(ctx, A, b.ncol, nullptr, Uv, ucs, b.W, b.wcs, nullptr, 0, &b.st[0].run, is, b.cpp);
    int S, G;
    dot_grid(ctx, b, j + 1, S, G);
    const double act = run_share(ctx, b);
    {
      KProf kp(ctx, sizeof(R) == 4 ? "dcgs2_dot_c64" : "dcgs2_dot_c128",
               ((double)j + (mode == DC_FINAL ? 1.0 : 2.0)) * col_len(b) * sv * act);
      dcgs2_dot_kernel<R><<<dim3((unsigned)(S * G), (unsigned)b.ncol), NT, 0, ctx->stream>>>(b, j, Uv, ucs, b.W,
                                                                                           b.wcs, S, G, mode);
      GDR_LAUNCHED(ctx);
    }
    {
      const double reads = (double)j + (mode == DC_FINAL ? 1.0 : 2.0);
      const double writes = (mode == 0) ? 2.0 : 1.0;
      KProf kp(ctx, sizeof(R) == 4 ? "dcgs2_update_c64" : "dcgs2_update_c128",
               (reads + writes) * col_len(b) * sv * run_share(ctx, b));
      dcgs2_update_kernel<R><<<dim3((unsigned)b.nblk, (unsigned)b.ncol), NT, 0, ctx->stream>>>(b, j, Uv, ucs, b.W,
                                                                                             b.W2, mode);
      GDR_LAUNCHED(ctx);
    }
  }
}

template <typename R>
void start_cycle(gdr_ctx* ctx, const Batch<R>& b, const cx<R>* r, long rcs) {
  double* rn2 = ctx->get<double>("start_rn2", b.ncol);
  norms2<cx<R>>(ctx, b.n, b.ncol, r, rcs, rn2, b.part, b.nblk, b.cnt, b.nvec);
  dim3 grid(grid_for(ctx, b.n, 256), (unsigned)b.ncol);
  start_scale_kernel<R><<<grid, 256, 0, ctx->stream>>>(b, r, rcs, rn2);
  GDR_LAUNCHED(ctx);
  start_state_kernel<R><<<b.ncol, 256, 0, ctx->stream>>>(b, rn2);
  GDR_LAUNCHED(ctx);
}

template <typename T>
void norms2(gdr_ctx* ctx, long n, int cols, const T* x, long xcs, double* out, c128* part, int nblk, unsigned* cnt,
            const int* nvec) {
  dim3 grid((unsigned)nblk, (unsigned)cols);
  KProf kp(ctx, "norms", (double)n * sizeof(T) * cols);
  norms2_kernel<T><<<grid, NT, 0, ctx->stream>>>(n, x, xcs, out, part, cnt, nvec);
  GDR_LAUNCHED(ctx);
}
void dots128(gdr_ctx* ctx, long n, int cols, const c128* u, long ucs, const c128* x, long xcs, c128* out, c128* part,
             int nblk, unsigned* cnt) {
  dim3 grid((unsigned)nblk, (unsigned)cols);
  dots128_kernel<<<grid, NT, 0, ctx->stream>>>(n, u, ucs, x, xcs, out, part, cnt);
  GDR_LAUNCHED(ctx);
}

template <typename R>
void combine(gdr_ctx* ctx, long n, int ncol, cx<R>* V, long ldv, long vcs, int nv, const c128* C, int ldc, long ccs,
             int nout, int nx, int rmode, c128* X, long ldx, long xcs, cx<R>* Rv, long rcs, const ColState* st,
             const int* nvec, int vpp, double lenh, double vlenh) {
  const int ntot = nout + nx + (rmode ? 1 : 0);
  if (ntot == 0 || ncol == 0) return;
  const size_t smem = sizeof(cx<R>) * ((size_t)CR * nv + (size_t)nv * ntot);
  GDR_REQUIRE(smem <= ctx->combine_smem_limit, "combine: too many basis vectors / outputs for shared memory");
  dim3 grid((unsigned)((n + CR - 1) / CR), (unsigned)ncol);
  // V read once per distinct basis, the rest per column
  const double cl = lenh > 0 ? lenh : (double)n * ncol;
  const double vl = vlenh > 0 ? vlenh : (vcs == 0 ? (double)n : (vpp > 1 ? (double)n * ((ncol + vpp - 1) / vpp) : cl));
  const double act = st ? run_share(ctx, ncol, &st[0].run, (int)(sizeof(ColState) / sizeof(int)), nvec) : 1.0;
  KProf kp(ctx, sizeof(R) == 4 ? "combine_c64" : "combine_c128",
           act * (vl * nv * sizeof(cx<R>) + cl * (nout * sizeof(cx<R>) + 2.0 * nx * sizeof(c128) +
                                                 (rmode == 2 ? 2.0 : (rmode == 1 ? 1.0 : 0.0)) * sizeof(cx<R>))));
  combine_kernel<R><<<grid, CT, smem, ctx->stream>>>(n, V, ldv, vcs, nv, C, ldc, ccs, nout, nx, rmode, X, ldx, xcs,
                                                     Rv, rcs, st, nvec, vpp);
  GDR_LAUNCHED(ctx);
}

void krylov_init(gdr_ctx* ctx) {
  ctx->combine_smem_limit =
      std::min(set_max_dyn_smem(ctx, combine_kernel<float>), set_max_dyn_smem(ctx, combine_kernel<double>));
}

void cvt_128_to_64(gdr_ctx* ctx, long n, int cols, const c128* in, long ics, c64* out, long ocs) {
  dim3 grid(grid_for(ctx, n, 256), (unsigned)cols);
  cvt_128_64_kernel<<<grid, 256, 0, ctx->stream>>>(n, in, ics, out, ocs);
  GDR_LAUNCHED(ctx);
}
void cvt_64_to_128(gdr_ctx* ctx, long n, int cols, const c64* in, long ics, c128* out, long ocs) {
  dim3 grid(grid_for(ctx, n, 256), (unsigned)cols);
  cvt_64_128_kernel<<<grid, 256, 0, ctx->stream>>>(n, in, ics, out, ocs);
  GDR_LAUNCHED(ctx);
}
void copy128(gdr_ctx* ctx, long n, int cols, const c128* in, long ics, c128* out, long ocs) {
  dim3 grid(grid_for(ctx, n, 256), (unsigned)cols);
  copy128_kernel<<<grid, 256, 0, ctx->stream>>>(n, in, ics, out, ocs);
  GDR_LAUNCHED(ctx);
}
void axpy_cols(gdr_ctx* ctx, long n, int cols, const c128* a, const c128* S, long ssc, c128* X, long xcs) {
  dim3 grid(grid_for(ctx, n, 256), (unsigned)cols);
  axpy_cols_kernel<<<grid, 256, 0, ctx->stream>>>(n, a, S, ssc, X, xcs);
  GDR_LAUNCHED(ctx);
}
void scal_cols(gdr_ctx* ctx, long n, int cols, const c128* a, c128* X, long xcs) {
  dim3 grid(grid_for(ctx, n, 256), (unsigned)cols);
  scal_cols_kernel<<<grid, 256, 0, ctx->stream>>>(n, a, X, xcs);
  GDR_LAUNCHED(ctx);
}

template void gs_dot<float>(gdr_ctx*, const Batch<float>&, int, const c64*, long, c128*, bool, const c64*);
template void gs_dot<double>(gdr_ctx*, const Batch<double>&, int, const c128*, long, c128*, bool, const c128*);
template void gs_update<float>(gdr_ctx*, const Batch<float>&, int, c64*, long, const c128*, bool);
template void gs_update<double>(gdr_ctx*, const Batch<double>&, int, c128*, long, const c128*, bool);
template void scale_into<float>(gdr_ctx*, const Batch<float>&, int, const c64*, long);
template void scale_into<double>(gdr_ctx*, const Batch<double>&, int, const c128*, long);
template void arnoldi_step<float>(gdr_ctx*, const gdr_op*, const Batch<float>&, int, int, int, c64*&);
template void arnoldi_step<double>(gdr_ctx*, const gdr_op*, const Batch<double>&, int, int, int, c128*&);
template void arnoldi_dcgs2<float>(gdr_ctx*, const gdr_op*, const Batch<float>&, int, int);
template void arnoldi_dcgs2<double>(gdr_ctx*, const gdr_op*, const Batch<double>&, int, int);
template void start_cycle<float>(gdr_ctx*, const Batch<float>&, const c64*, long);
template void start_cycle<double>(gdr_ctx*, const Batch<double>&, const c128*, long);
template void norms2<c64>(gdr_ctx*, long, int, const c64*, long, double*, c128*, int, unsigned*, const int*);
template void norms2<c128>(gdr_ctx*, long, int, const c128*, long, double*, c128*, int, unsigned*, const int*);
template void combine<float>(gdr_ctx*, long, int, c64*, long, long, int, const c128*, int, long, int, int, int, c128*,
                             long, long, c64*, long, const ColState*, const int*, int, double, double);
template void combine<double>(gdr_ctx*, long, int, c128*, long, long, int, const c128*, int, long, int, int, int,
                              c128*, long, long, c128*, long, const ColState*, const int*, int, double, double);
