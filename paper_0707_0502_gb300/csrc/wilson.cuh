// Device functions of the Wilson-Dirac-style hop (spin projection of the chiral
// basis, Example 7 of the paper):
//   (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu),
// with gamma_mu = [[0, B_mu], [B_mu^H, 0]], B_mu unitary 2x2, so that
//   (1 -+ gamma_mu) psi = [h ; -+ B_mu^H h],  h = u -+ B_mu d,  psi = [u ; d].
// Vectors are site-major (site*12 + spin*3 + colour); links are stored
// structure-of-arrays [mu][a*3+b][site].
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace {

template <typename R, typename LT> struct LinkLd;
template <> struct LinkLd<double, c128> {
  static DEV c128 ld(const c128* L, long i) {
    double2 v = __ldg(reinterpret_cast<const double2*>(L) + i);
    return {v.x, v.y};
  }
};
template <> struct LinkLd<float, c64> {
  static DEV c64 ld(const c64* L, long i) {
    float2 v = __ldg(reinterpret_cast<const float2*>(L) + i);
    return {v.x, v.y};
  }
};
template <> struct LinkLd<float, __nv_bfloat162> {
  static DEV c64 ld(const __nv_bfloat162* L, long i) {
    float2 v = __bfloat1622float2(L[i]);
    return {v.x, v.y};
  }
};

// B_mu d (chiral basis; B_x = -i s1, B_y = -i s2, B_z = -i s3, B_t = I)
template <int MU, typename R>
DEV void b_mul(cx<R> d0, cx<R> d1, cx<R>& o0, cx<R>& o1) {
  if (MU == 0) { o0 = -mul_i(d1); o1 = -mul_i(d0); }
  if (MU == 1) { o0 = -d1; o1 = d0; }
  if (MU == 2) { o0 = -mul_i(d0); o1 = mul_i(d1); }
  if (MU == 3) { o0 = d0; o1 = d1; }
}
// B_mu^H g
template <int MU, typename R>
DEV void bh_mul(cx<R> g0, cx<R> g1, cx<R>& o0, cx<R>& o1) {
  if (MU == 0) { o0 = mul_i(g1); o1 = mul_i(g0); }
  if (MU == 1) { o0 = g1; o1 = -g0; }
  if (MU == 2) { o0 = mul_i(g0); o1 = -mul_i(g1); }
  if (MU == 3) { o0 = g0; o1 = g1; }
}

template <typename R> struct Spinor { cx<R> s[12]; };

// CG = true loads through L2 only (ld.global.cg): for vectors written by other
// blocks of the same launch (the persistent sweep); otherwise the read-only path.
template <bool CG> DEV float4 ld4(const float4* p) { return CG ? __ldcg(p) : __ldg(p); }
template <bool CG> DEV double2 ld2(const double2* p) { return CG ? __ldcg(p) : __ldg(p); }

template <typename R, bool CG = false> DEV void load_spinor(const cx<R>* x, long site, Spinor<R>& p) {
  if constexpr (sizeof(R) == 4) {
    const float4* q = reinterpret_cast<const float4*>(x + site * 12);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float4 v = ld4<CG>(q + i);
      p.s[2 * i] = {v.x, v.y};
      p.s[2 * i + 1] = {v.z, v.w};
    }
  } else {
    const double2* q = reinterpret_cast<const double2*>(x + site * 12);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const double2 v = ld2<CG>(q + i);
      p.s[i] = {v.x, v.y};
    }
  }
}

// one hop in direction MU; FWD: (1 - gamma) U(x) psi(x+mu), else (1 + gamma) U(x-mu)^H psi(x-mu)
template <int MU, bool FWD, typename R, typename LT>
DEV void hop(const LT* __restrict__ links, long V, long lsite, const Spinor<R>& p, Spinor<R>& acc) {
  // half spinor h_s = u_s -+ (B d)_s, s = 0, 1, per colour
  cx<R> h[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<R> b0, b1;
    b_mul<MU, R>(p.s[6 + a], p.s[9 + a], b0, b1);
    if (FWD) { h[0][a] = p.s[a] - b0; h[1][a] = p.s[3 + a] - b1; }
    else     { h[0][a] = p.s[a] + b0; h[1][a] = p.s[3 + a] + b1; }
  }
  // g = U h  (forward)  or  U^H h  (backward)
  cx<R> g[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) { g[0][a] = {0, 0}; g[1][a] = {0, 0}; }
  const LT* L = links + (long)MU * 9 * V + lsite;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cx<R> u = LinkLd<R, LT>::ld(L, (long)(a * 3 + b) * V);
      if (FWD) {  // g_a += U_ab h_b
        g[0][a] += u * h[0][b];
        g[1][a] += u * h[1][b];
      } else {    // g_b += conj(U_ab) h_a
        g[0][b] += cmulc(u, h[0][a]);
        g[1][b] += cmulc(u, h[1][a]);
      }
    }
  }
  // reconstruct: upper += g, lower += -+ B^H g
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<R> l0, l1;
    bh_mul<MU, R>(g[0][a], g[1][a], l0, l1);
    acc.s[a] += g[0][a];
    acc.s[3 + a] += g[1][a];
    if (FWD) { acc.s[6 + a] -= l0; acc.s[9 + a] -= l1; }
    else     { acc.s[6 + a] += l0; acc.s[9 + a] += l1; }
  }
}

template <int MU, typename R, typename LT, bool CG = false>
DEV void hop_mu(const LT* __restrict__ links, const cx<R>* x, long V, long site, int coord, int L, long stride,
                Spinor<R>& acc) {
  const long fwd = (coord == L - 1) ? site - (long)(L - 1) * stride : site + stride;
  const long bwd = (coord == 0) ? site + (long)(L - 1) * stride : site - stride;
  Spinor<R> pf, pb;  // both neighbour spinors in flight before either hop's arithmetic
  load_spinor<R, CG>(x, fwd, pf);
  load_spinor<R, CG>(x, bwd, pb);
  hop<MU, true, R, LT>(links, V, site, pf, acc);
  hop<MU, false, R, LT>(links, V, bwd, pb, acc);
}

}  // namespace
