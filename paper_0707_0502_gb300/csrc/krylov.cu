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
__global__ void __launch_bounds__(NT, 2) dcgs2_dot_kernel(Batch<R> b, int j, const cx<R>* __restrict__ Uv, long ucs,
                                                       const cx<R>* __restrict__ W, long wcs, int S, int G,
                                                       int mode) {
  const int c = blockIdx.y;
  if (!b.st[c].run) return;
  constexpr int K = U<R>::K;
  constexpr int DU = 8;        // units per lane of a warp's slab
  constexpr int SU = 32 * DU;  // units per slab
  constexpr int NW = NT / 32;
  // Each warp keeps its slab of u and w in registers and streams every basis vector of
  // its group through it (DU loads in flight per lane and vector), reduces the two dots
  // over the warp and adds them to its own FP32 sums in shared memory; no block
  // barrier until the end, so warps never wait for each other.
  __shared__ cx<R> accw[NW][2 * GDR_MAX_M + 8];
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
  for (int v = v0 + lane; v < v1; v += 32) accw[warp][v] = {0, 0};
  __syncwarp();
  const long nslabs = (nu + SU - 1) / SU;
  for (long sl = (long)slot * NW + warp; sl < nslabs && i0 < i1; sl += (long)S * NW) {
    const long ub = sl * SU;
    cx<R> uu[DU][K], ww[DU][K];
#pragma unroll
    for (int t = 0; t < DU; ++t) {
      const long q = ub + lane + 32 * t;
      if (q < nu) {
        ldu<R>(u, q, n, uu[t]);
        if (hasw) {
          ldu<R>(w, q, n, ww[t]);
        } else {
#pragma unroll
          for (int kk = 0; kk < K; ++kk) ww[t][kk] = {0, 0};
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) uu[t][kk] = ww[t][kk] = {0, 0};
      }
    }
    for (int i = i0; i < i1; ++i) {
      cx<R> au = {0, 0}, aw = {0, 0}, wn = {0, 0};
      if (i < j) {
        const cx<R>* vi = V + (long)i * b.ldv;
        cx<R> vv[DU][K];
#pragma unroll
        for (int t = 0; t < DU; ++t) {
          const long q = ub + lane + 32 * t;
          if (q < nu) {
            ldu<R>(vi, q, n, vv[t]);
          } else {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) vv[t][kk] = {0, 0};
          }
        }
#pragma unroll
        for (int t = 0; t < DU; ++t)
#pragma unroll
          for (int kk = 0; kk < K; ++kk) {
            au += cmulc(vv[t][kk], uu[t][kk]);
            aw += cmulc(vv[t][kk], ww[t][kk]);
          }
      } else {  // omega = u^H u (au.x), zeta = u^H w (aw), w^H w (wn.x)
#pragma unroll
        for (int t = 0; t < DU; ++t)
#pragma unroll
          for (int kk = 0; kk < K; ++kk) {
            au.x += norm2(uu[t][kk]);
            aw += cmulc(uu[t][kk], ww[t][kk]);
            wn.x += norm2(ww[t][kk]);
          }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        au.x += __shfl_xor_sync(FULL, au.x, off);
        au.y += __shfl_xor_sync(FULL, au.y, off);
        aw.x += __shfl_xor_sync(FULL, aw.x, off);
        aw.y += __shfl_xor_sync(FULL, aw.y, off);
      }
      if (i == j) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) wn.x += __shfl_xor_sync(FULL, wn.x, off);
      }
      if (lane == (i & 31)) {  // each lane owns the sums of every 32nd vector
        accw[warp][2 * i] += au;
        accw[warp][2 * i + 1] += aw;
        if (i == j) accw[warp][2 * i + 2] += wn;
      }
    }
  }
  __syncthreads();
  c128* part = b.part + c * b.pstride;
  for (int v = v0 + threadIdx.x; v < v1; v += NT) {  // the block's sums, warps in a fixed order, FP64
    c128 sacc = {0, 0};
#pragma unroll
    for (int q = 0; q < NW; ++q) sacc += up(accw[q][v]);
    part[(long)slot * hs + v] = sacc;
  }
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
  // H's FP32 copy (for the H s term below): rebuilt from H on the first step of a cycle
  // (the restart may have rewritten the kept columns), then kept with the two columns
  // each step changes
  c64* Hf = b.Hf ? b.Hf + (long)c * (m + 1) * m : nullptr;
  if (first && Hf)
    for (int q = threadIdx.x; q < j * (m + 1); q += NT) Hf[q] = to64(H[q]);
  // the delayed pass completes column j-1
  if (!first)
    for (int i = threadIdx.x; i <= j; i += NT) {
      c128& hij = H[(long)(j - 1) * (m + 1) + i];
      if (i < j) hij += ssh[i];
      if (Hf) Hf[(long)(j - 1) * (m + 1) + i] = to64(hij);
    }
  for (int i = threadIdx.x; i < j; i += NT) dc[i] = ssh[i];
  if (mode == DC_FINAL) return;
  __shared__ c64 s32[GDR_MAX_M + 1];
  for (int i = threadIdx.x; i < j; i += NT) s32[i] = to64(ssh[i]);
  __syncthreads();
  const c128 t = ssh[GDR_MAX_M + 1];
  const c128 tn = (1.0 / nuv) * t;
  for (int i = threadIdx.x; i < j; i += NT) dc[(m + 1) + i] = hv[2 * i + 1] - tn * ssh[i];
  // column j: ([z ; t] - Hbar[0:j+1, 0:j] s) / nu; s is O(rounding), so H s in FP32 (from the
  // FP32 copy: no conversions on the FP64 pipe, loads issued eight ahead)
  if (Hf)  // the copy's rows below the subdiagonal are zero, as H's are
    for (int i = j + 1 + threadIdx.x; i <= m; i += NT) Hf[(long)j * (m + 1) + i] = {0.f, 0.f};
  for (int i = threadIdx.x; i <= j; i += NT) {
    c64 hsum = {0.f, 0.f};
    if (!first) {
      if (Hf) {
#pragma unroll 8
        for (int l = 0; l < j; ++l) hsum += Hf[(long)l * (m + 1) + i] * s32[l];
      } else {
        for (int l = 0; l < j; ++l) hsum += to64(H[(long)l * (m + 1) + i]) * s32[l];
      }
    }
    const c128 zi = (i < j) ? hv[2 * i + 1] : t;
    const c128 hnew = (1.0 / nuv) * (zi - to128(hsum));
    H[(long)j * (m + 1) + i] = hnew;
    if (Hf) Hf[(long)j * (m + 1) + i] = to64(hnew);
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
  // FP64 per-thread accumulation.  Complex64 vectors carry 2^-24 relative precision, so
  // their squares are summed in FP32 over groups of four elements (relative error
  // <= 8 * 2^-24 per group) and only the group sums in FP64: the FP64 pipe, slow on this
  // part, would otherwise bound the kernel.  FP64 vectors are summed in FP64 throughout.
  double s = 0;
  long i = blockIdx.x * (long)NT + threadIdx.x;
  const long stride = (long)gridDim.x * NT;
  if (sizeof(R) == 4) {
    for (; i + 3 * stride < n; i += 4 * stride) {
      T v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = xc[i + q * stride];
      float f = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) f = fmaf((float)v[q].x, (float)v[q].x, fmaf((float)v[q].y, (float)v[q].y, f));
      s += (double)f;
    }
  }
  for (; i < n; i += stride) {
    const T v = xc[i];
    s += (double)v.x * v.x + (double)v.y * v.y;
  }
  c128 d[1] = {{s, 0}};
  block_reduce<double, 1>(d, part + (long)c * gridDim.x + blockIdx.x, 1);
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
                                                     const ColState* st, const int* nvec, int vpp, cx<R>* Xf) {
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
      if (Xf) {
        cx<R>* fp = Xf + c * xcs + (long)(o - nout) * ldx + row;
        *fp = *fp + acc;
      } else {
        c128* xp = X + c * xcs + (long)(o - nout) * ldx + row;
        *xp = *xp + up(acc);
      }
    } else {
      cx<R>* rp = Rv + c * rcs + row;
      if (rmode == 1) *rp = acc;
      else *rp = *rp + acc;
    }
  }
}

// Basis combination without in-place outputs (the solution update x_i += V_m d_i of a
// cycle and the residual r = V_{m+1} s, per column with its own basis): rows are
// independent, so each thread takes rows in a grid-stride loop and reads its row of V
// directly (coalesced across the warp); the block stages the column's coefficients once.
// Same summation order as combine_kernel.
constexpr int CW_MAXO = 12, CW_MAXCF = 1280;
template <typename R, int NO>  // NO >= ntot outputs, so no unrolled work is predicated off for nothing
__global__ void __launch_bounds__(256) combine_rows_kernel(long n, const cx<R>* __restrict__ V, long ldv, long vcs,
                                                           int nv, const c128* __restrict__ C, int ldc, long ccs,
                                                           int nx, int rmode, c128* X, long ldx, long xcs, cx<R>* Rv,
                                                           long rcs, const ColState* st, const int* nvec, int vpp,
                                                           cx<R>* Xf) {
  __shared__ cx<R> cf[CW_MAXCF];  // ntot x nv
  const int c = blockIdx.y;
  if (st && !st[c].active) return;
  if (nvec) n = nvec[c];
  const int ntot = nx + (rmode ? 1 : 0);
  const c128* Cc = C + c * ccs;
  for (int t = threadIdx.x; t < nv * ntot; t += 256) {
    const int i = t % nv, o = t / nv;
    cf[t] = cvt<R>(Cc[(long)o * ldc + i]);
  }
  __syncthreads();
  const cx<R>* Vc = V + (c / vpp) * vcs;
  for (long row = blockIdx.x * 256L + threadIdx.x; row < n; row += (long)gridDim.x * 256) {
    cx<R> acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = {0, 0};
#pragma unroll 4
    for (int i = 0; i < nv; ++i) {
      const cx<R> v = Vc[(long)i * ldv + row];
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < ntot) acc[o] += v * cf[o * nv + i];
    }
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      if (o >= ntot) break;
      if (o < nx) {
        if (Xf) {  // correction accumulated in the vectors' precision
          cx<R>* fp = Xf + c * xcs + (long)o * ldx + row;
          *fp = *fp + acc[o];
        } else {
          c128* xp = X + c * xcs + (long)o * ldx + row;
          *xp = *xp + up(acc[o]);
        }
      } else {
        cx<R>* rp = Rv + c * rcs + row;
        if (rmode == 1) *rp = acc[o];
        else *rp = *rp + acc[o];
      }
    }
  }
}

// Basis combination for many columns sharing one basis (vcs = 0, no in-place outputs),
// as in the projection over the kept V_{k+1} of the Proj and refinement stages: a
// persistent block stages every column's coefficients once (complex64 or FP64 as the
// vectors, nv x ntot per column) and, for each of its row tiles, the tile of V once,
// then forms every column's outputs from it -- the basis is read from HBM once instead
// of once per column.
template <typename R>
__global__ void __launch_bounds__(CT) combine_shared_kernel(long n, const cx<R>* __restrict__ V, long ldv, int nv,
                                                            const c128* __restrict__ C, int ldc, long ccs, int nx,
                                                            int rmode, c128* X, long ldx, long xcs, cx<R>* Rv,
                                                            long rcs, const ColState* st, int ncol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ntot = nx + (rmode ? 1 : 0);
  cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);  // CR x nv (row-fast)
  cx<R>* cf = tile + (long)CR * nv;                   // ncol x (nv x ntot)
  const long per = (long)nv * ntot;
  for (long t = threadIdx.x; t < per * ncol; t += CT) {
    const int c = (int)(t / per);
    const int q = (int)(t % per), i = q % nv, o = q / nv;
    cf[t] = cvt<R>(C[c * ccs + (long)o * ldc + i]);
  }
  const long ntiles = (n + CR - 1) / CR;
  const int rr = threadIdx.x % CR;
  for (long tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const long r0 = tl * CR;
    const int rows = (int)min((long)CR, n - r0);
    __syncthreads();  // the previous tile's readers are done (and the coefficients staged)
    for (int t = threadIdx.x; t < CR * nv; t += CT) {
      const int r = t % CR, i = t / CR;
      tile[t] = (r < rows) ? V[(long)i * ldv + r0 + r] : cx<R>{0, 0};
    }
    __syncthreads();
    if (rr >= rows) continue;
    const long row = r0 + rr;
    // the (column, output) pairs, four independent accumulations per thread at a time;
    // the CT / CR = 4 thread groups of a row take interleaved pairs
    const long P = (long)ncol * ntot;
    for (long p0 = threadIdx.x / CR; p0 < P; p0 += 4 * (CT / CR)) {
      cx<R> acc[4];
      const cx<R>* co[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long pq = min(p0 + (long)q * (CT / CR), P - 1);
        co[q] = cf + (pq / ntot) * per + (pq % ntot) * nv;
        acc[q] = {0, 0};
      }
      for (int i = 0; i < nv; ++i) {
        const cx<R> t = tile[(long)i * CR + rr];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += t * co[q][i];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long pq = p0 + (long)q * (CT / CR);
        if (pq >= P) break;
        const int c = (int)(pq / ntot), o = (int)(pq % ntot);
        if (st && !st[c].active) continue;
        if (o < nx) {
          c128* xp = X + c * xcs + (long)o * ldx + row;
          *xp = *xp + up(acc[q]);
        } else {
          cx<R>* rp = Rv + c * rcs + row;
          if (rmode == 1) *rp = acc[q];
          else *rp = *rp + acc[q];
        }
      }
    }
  }
}

// h_c = V^H r_c (nv <= NVM basis vectors) for ncol columns sharing one basis V, as in
// the projection c = V_{k+1}^H r of the Proj and refinement stages.  Block (g, slot)
// stages row tiles of V (32 EPL rows x nv, complex64 or FP64 as the vectors) in shared
// memory; its warp w takes column c = 8 g + w, each lane holding its rows of r_c and
// partial sums for every basis vector in registers, flushed to FP64 in shared memory
// every FL tiles.  The column groups of one tile slot are consecutive blocks, so they
// read the same tiles of V close together (L2 reuse): V comes from HBM about once.
// part[(slot * ncol + c) * nv + i] receives each block's FP64 sums; gs_dot_shared_sum
// adds them over the slots in a fixed order.
constexpr int DS_W = 8, DS_EPL = 4, DS_TR = 32 * DS_EPL, DS_FL = 16;

template <typename R, int NVM>
__global__ void __launch_bounds__(DS_W * 32) gs_dot_shared_kernel(long n, const cx<R>* __restrict__ V, long ldv,
                                                                   int nv, const cx<R>* __restrict__ Rv, long rcs,
                                                                   int ncol, const ColState* st, c128* part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* vt = reinterpret_cast<cx<R>*>(smem_raw);                       // nv x DS_TR
  c128* accd = reinterpret_cast<c128*>(vt + (long)NVM * DS_TR);          // DS_W x NVM
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = blockIdx.x, slot = blockIdx.y;
  const int c = grp * DS_W + warp;
  const bool live = c < ncol && (!st || st[c].run);
  for (int i = lane; i < NVM; i += 32) accd[warp * NVM + i] = {0, 0};
  cx<R> acc[NVM];
#pragma unroll
  for (int i = 0; i < NVM; ++i) acc[i] = {0, 0};
  const cx<R>* r = Rv + (long)(live ? c : 0) * rcs;
  const long ntiles = (n + DS_TR - 1) / DS_TR;
  int cnt = 0;
  auto flush = [&]() {
#pragma unroll
    for (int i = 0; i < NVM; ++i) {
      if (i >= nv) break;
      cx<R> a = acc[i];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        a.x += __shfl_xor_sync(FULL, a.x, off);
        a.y += __shfl_xor_sync(FULL, a.y, off);
      }
      if (lane == (i & 31)) accd[warp * NVM + i] += up(a);
      acc[i] = {0, 0};
    }
  };
  for (long tl = slot; tl < ntiles; tl += gridDim.y) {
    const long r0 = tl * DS_TR;
    const int rows = (int)min((long)DS_TR, n - r0);
    __syncthreads();  // the previous tile's readers are done
    for (int t = threadIdx.x; t < nv * DS_TR; t += DS_W * 32) {
      const int i = t / DS_TR, e = t % DS_TR;
      vt[t] = (e < rows) ? V[(long)i * ldv + r0 + e] : cx<R>{0, 0};
    }
    __syncthreads();
    if (!live) continue;
    cx<R> rv[DS_EPL];
#pragma unroll
    for (int q = 0; q < DS_EPL; ++q) {
      const int e = lane + 32 * q;
      rv[q] = (e < rows) ? r[r0 + e] : cx<R>{0, 0};
    }
#pragma unroll
    for (int i = 0; i < NVM; ++i) {
      if (i >= nv) break;
#pragma unroll
      for (int q = 0; q < DS_EPL; ++q) acc[i] += cmulc(vt[i * DS_TR + lane + 32 * q], rv[q]);
    }
    if (++cnt == DS_FL) {
      flush();
      cnt = 0;
    }
  }
  if (!live) return;
  flush();
  __syncwarp();
  for (int i = lane; i < nv; i += 32) part[((long)slot * ncol + c) * nv + i] = accd[warp * NVM + i];
}

// hout[c * hs + i] = sum over the S slots of part[(slot * ncol + c) * nv + i] (fixed order)
__global__ void gs_dot_shared_sum_kernel(int S, int ncol, int nv, const c128* __restrict__ part, c128* hout, int hs,
                                         const ColState* st) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncol * nv) return;
  const int c = t / nv, i = t % nv;
  if (st && !st[c].run) return;
  c128 acc = {0, 0};
  for (int q = 0; q < S; ++q) acc += part[((long)q * ncol + c) * nv + i];
  hout[(long)c * hs + i] = acc;
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

// tile slots of the shared-basis dot: about two blocks per SM in all
static int dot_shared_slots(gdr_ctx* ctx, long n, int ncol) {
  const int groups = (ncol + DS_W - 1) / DS_W;
  const long ntiles = (n + DS_TR - 1) / DS_TR;
  return (int)std::max<long>(1, std::min<long>(ntiles, std::max(1, 2 * ctx->num_sms / groups)));
}

template <typename R>
static bool dot_shared_applies(const Batch<R>& b, int nv, bool wnorm, const cx<R>* wprev) {
  return b.vcs == 0 && b.ncol > 1 && b.nvec == nullptr && nv <= 48 && !wnorm && !wprev;
}

void gs_dot_shared_reserve(gdr_ctx* ctx, long n, int ncol, int nv) {
  const int S = std::max(dot_shared_slots(ctx, n, ncol), tc_proj_splits(ctx, n, ncol));
  ctx->get<c128>("dsh.part", (size_t)S * ncol * nv + 64);
  if (!ctx->tc_err) {
    ctx->tc_err = ctx->get<int>("tc.err", 4);
    GDR_CUDA(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int) * 4, ctx->stream));
  }
}

// the tensor-core forms for complex64 columns: from this many columns on (with fewer the
// CUDA-core kernels are memory-bound anyway)
constexpr int TC_MIN_COLS = 8;

template <typename R, int NVM>
static void gs_dot_shared_launch(gdr_ctx* ctx, const Batch<R>& b, int nv, const cx<R>* w, long wcs, c128* h_out) {
  const int S = dot_shared_slots(ctx, b.n, b.ncol);
  c128* part = ctx->get<c128>("dsh.part", (size_t)S * b.ncol * nv + 64);
  const size_t smem = sizeof(cx<R>) * NVM * DS_TR + sizeof(c128) * DS_W * NVM;
  dim3 grid((unsigned)((b.ncol + DS_W - 1) / DS_W), (unsigned)S);
  {
    KProf kp(ctx, sizeof(R) == 4 ? "gs_dot_shared_c64" : "gs_dot_shared_c128",
             ((double)nv * b.n + col_len(b)) * sizeof(cx<R>) * run_share(ctx, b));
    gs_dot_shared_kernel<R, NVM><<<grid, DS_W * 32, smem, ctx->stream>>>(b.n, b.V, b.ldv, nv, w, wcs, b.ncol, b.st,
                                                                          part);
    GDR_LAUNCHED(ctx);
  }
  const int tot = b.ncol * nv;
  gs_dot_shared_sum_kernel<<<(tot + 255) / 256, 256, 0, ctx->stream>>>(S, b.ncol, nv, part, h_out, b.m + 2, b.st);
  GDR_LAUNCHED(ctx);
}

template <typename R>
void gs_dot(gdr_ctx* ctx, const Batch<R>& b, int nv, const cx<R>* w, long wcs, c128* h_out, bool wnorm,
            const cx<R>* wprev) {
  if (std::is_same<R, float>::value && b.vcs == 0 && b.ncol >= TC_MIN_COLS && b.nvec == nullptr && !wnorm &&
      !wprev && ctx->tc_ok && ctx->tc_proj && ctx->tc_err) {  // tensor cores
    const int S0 = tc_proj_splits(ctx, b.n, b.ncol);
    c128* part = ctx->get<c128>("dsh.part", (size_t)S0 * b.ncol * nv + 64);
    int S = 0;
    const double bytes = ctx->profile ? ((double)nv * b.n + col_len(b)) * sizeof(cx<R>) * run_share(ctx, b) : 0.0;
    if (tc_proj_dot(ctx, b.n, reinterpret_cast<const c64*>(b.V), b.ldv, nv, reinterpret_cast<const c64*>(w), wcs,
                    b.ncol, part, ctx->tc_err, S, bytes)) {
      const int tot = b.ncol * nv;
      gs_dot_shared_sum_kernel<<<(tot + 255) / 256, 256, 0, ctx->stream>>>(S, b.ncol, nv, part, h_out, b.m + 2,
                                                                           b.st);
      GDR_LAUNCHED(ctx);
      return;
    }
  }
  if (dot_shared_applies(b, nv, wnorm, wprev)) {  // one basis for many columns: read it once
    if (nv <= 24) gs_dot_shared_launch<R, 24>(ctx, b, nv, w, wcs, h_out);
    else gs_dot_shared_launch<R, 48>(ctx, b, nv, w, wcs, h_out);
    return;
  }
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

// tile slots S x vector groups G of the DCGS2 dot pass: a block takes NT/32 slabs of 256
// units per round; about two blocks per SM per column, vectors split over G blocks when
// slabs are scarce (short vectors); S <= nblk bounds the partials
template <typename R>
static void dcgs2_grid(gdr_ctx* ctx, const Batch<R>& b, int nvec, int& S, int& G) {
  const long slabs = (nunits<R>(b.n) + 255) / 256;
  const long tiles = (slabs + NT / 32 - 1) / (NT / 32);
  const long target = 2L * ctx->num_sms;
  S = (int)std::max<long>(1, std::min<long>(tiles, std::min<long>(target, b.nblk)));
  G = 1;
  if (S < target) G = (int)std::min<long>((target + S - 1) / S, (nvec + NT / 32 - 1) / (NT / 32));
  G = std::max(G, 1);
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
    dcgs2_grid(ctx, b, j + 1, S, G);
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
  KProf kp(ctx, sizeof(T) == 8 ? "norms_c64" : "norms_c128", (double)n * sizeof(T) * cols);
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
             const int* nvec, int vpp, double lenh, double vlenh, cx<R>* Xf) {
  const int ntot = nout + nx + (rmode ? 1 : 0);
  if (ntot == 0 || ncol == 0) return;
  const size_t smem = sizeof(cx<R>) * ((size_t)CR * nv + (size_t)nv * ntot);
  GDR_REQUIRE(smem <= ctx->combine_smem_limit, "combine: too many basis vectors / outputs for shared memory");
  dim3 grid((unsigned)((n + CR - 1) / CR), (unsigned)ncol);
  // V read once per distinct basis, the rest per column
  const double cl = lenh > 0 ? lenh : (double)n * ncol;
  const double vl = vlenh > 0 ? vlenh : (vcs == 0 ? (double)n : (vpp > 1 ? (double)n * ((ncol + vpp - 1) / vpp) : cl));
  const double act = st ? run_share(ctx, ncol, &st[0].run, (int)(sizeof(ColState) / sizeof(int)), nvec) : 1.0;
  // one basis shared by several columns: stream it once for all of them when their
  // coefficients fit in shared memory beside a row tile
  const size_t smem_sh = sizeof(cx<R>) * ((size_t)CR * nv + (size_t)nv * ntot * ncol);
  if (!Xf && std::is_same<R, float>::value && vcs == 0 && nout == 0 && nx == 0 && (rmode == 1 || rmode == 2) &&
      ncol >= TC_MIN_COLS && nvec == nullptr && vpp == 1 && ctx->tc_ok && ctx->tc_proj && ctx->tc_err) {
    const double bytes = ctx->profile ? act * ((double)n * nv + cl * (rmode == 2 ? 2.0 : 1.0)) * sizeof(cx<R>) : 0.0;
    if (tc_proj_update(ctx, n, reinterpret_cast<const c64*>(V), ldv, nv, C, ccs, rmode, reinterpret_cast<c64*>(Rv),
                       rcs, ncol, st, ctx->tc_err, bytes))
      return;
  }
  if (!Xf && vcs == 0 && nout == 0 && ncol > 1 && nvec == nullptr && smem_sh <= ctx->combine_smem_limit) {
    KProf kp(ctx, sizeof(R) == 4 ? "combine_shared_c64" : "combine_shared_c128",
             act * ((double)n * nv * sizeof(cx<R>) +
                    cl * (2.0 * nx * sizeof(c128) + (rmode == 2 ? 2.0 : (rmode == 1 ? 1.0 : 0.0)) * sizeof(cx<R>))));
    const long ntiles = (n + CR - 1) / CR;
    const unsigned g = (unsigned)std::max<long>(1, std::min<long>(ntiles, 2L * ctx->num_sms));
    combine_shared_kernel<R><<<g, CT, smem_sh, ctx->stream>>>(n, V, ldv, nv, C, ldc, ccs, nx, rmode, X, ldx, xcs, Rv,
                                                              rcs, st, ncol);
    GDR_LAUNCHED(ctx);
    return;
  }
  // profiler names by use: basis restart (in-place outputs), solution update, residual only
  const char* pname = nout > 0 ? (sizeof(R) == 4 ? "combine_restart_c64" : "combine_restart_c128")
                      : nx > 0 ? (sizeof(R) == 4 ? "combine_update_c64" : "combine_update_c128")
                               : (sizeof(R) == 4 ? "combine_resid_c64" : "combine_resid_c128");
  if (nout == 0 && ntot <= CW_MAXO && (long)nv * ntot <= CW_MAXCF) {
    KProf kp(ctx, pname,
             act * (vl * nv * sizeof(cx<R>) + cl * (2.0 * nx * (Xf ? sizeof(cx<R>) : sizeof(c128)) +
                                                   (rmode == 2 ? 2.0 : (rmode == 1 ? 1.0 : 0.0)) * sizeof(cx<R>))));
    // enough blocks per column to fill the GPU on its own: late in a batch few columns
    // are still active, and the blocks of the others return at once
    const long rblk = (n + 255) / 256;
    dim3 g((unsigned)std::max<long>(1, std::min(rblk, 8L * ctx->num_sms)), (unsigned)ncol);
#define GDR_ROWS(NO)                                                                                           \
  combine_rows_kernel<R, NO><<<g, 256, 0, ctx->stream>>>(n, V, ldv, vcs, nv, C, ldc, ccs, nx, rmode, X, ldx, xcs, Rv, \
                                                         rcs, st, nvec, vpp, Xf)
    if (ntot <= 1) GDR_ROWS(1);
    else if (ntot <= 2) GDR_ROWS(2);
    else if (ntot <= 4) GDR_ROWS(4);
    else if (ntot <= 8) GDR_ROWS(8);
    else GDR_ROWS(CW_MAXO);
#undef GDR_ROWS
    GDR_LAUNCHED(ctx);
    return;
  }
  KProf kp(ctx, pname,
           act * (vl * nv * sizeof(cx<R>) + cl * (nout * sizeof(cx<R>) + 2.0 * nx * sizeof(c128) +
                                                 (rmode == 2 ? 2.0 : (rmode == 1 ? 1.0 : 0.0)) * sizeof(cx<R>))));
  combine_kernel<R><<<grid, CT, smem, ctx->stream>>>(n, V, ldv, vcs, nv, C, ldc, ccs, nout, nx, rmode, X, ldx, xcs,
                                                     Rv, rcs, st, nvec, vpp, Xf);
  GDR_LAUNCHED(ctx);
}

void krylov_init(gdr_ctx* ctx) {
  ctx->combine_smem_limit =
      std::min(set_max_dyn_smem(ctx, combine_kernel<float>), set_max_dyn_smem(ctx, combine_kernel<double>));
  ctx->combine_smem_limit = std::min(ctx->combine_smem_limit, set_max_dyn_smem(ctx, combine_shared_kernel<float>));
  ctx->combine_smem_limit = std::min(ctx->combine_smem_limit, set_max_dyn_smem(ctx, combine_shared_kernel<double>));
  set_max_dyn_smem(ctx, gs_dot_shared_kernel<float, 24>);
  set_max_dyn_smem(ctx, gs_dot_shared_kernel<float, 48>);
  set_max_dyn_smem(ctx, gs_dot_shared_kernel<double, 24>);
  set_max_dyn_smem(ctx, gs_dot_shared_kernel<double, 48>);
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
                             long, long, c64*, long, const ColState*, const int*, int, double, double, c64*);
template void combine<double>(gdr_ctx*, long, int, c128*, long, long, int, const c128*, int, long, int, int, int,
                              c128*, long, long, c128*, long, const ColState*, const int*, int, double, double, c128*);
