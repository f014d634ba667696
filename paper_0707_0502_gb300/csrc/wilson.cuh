// Device functions of the Wilson-Dirac-style hop (spin projection of the chiral
// basis, Example 7 of the paper):
//   (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu),
// with gamma_mu = [[0, B_mu], [B_mu^H, 0]], B_mu unitary 2x2, so that
//   (1 -+ gamma_mu) psi = [h ; -+ B_mu^H h],  h = u -+ B_mu d,  psi = [u ; d].
// Inside the library a Wilson vector is stored in pair-major order: component
// q = spin*3 + colour of site s is complex element 2 ((q/2) V + s) + q%2, so the
// pair (2p, 2p+1) of consecutive sites is contiguous (one float4 per site for
// complex64, two double2 for complex128) and a warp's loads of one pair are
// coalesced.  The C interface uses site-major order (s*12 + q); wilson_order
// converts at the boundary.  Links are stored structure-of-arrays [mu][a*3+b][site].
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

// element index of component q of site s (pair-major order)
HD long wil_index(long V, long site, int q) { return 2 * ((long)(q >> 1) * V + site) + (q & 1); }

template <typename R, bool CG = false> DEV void load_spinor(const cx<R>* x, long V, long site, Spinor<R>& p) {
  if constexpr (sizeof(R) == 4) {
    const float4* q = reinterpret_cast<const float4*>(x) + site;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float4 v = ld4<CG>(q + i * V);
      p.s[2 * i] = {v.x, v.y};
      p.s[2 * i + 1] = {v.z, v.w};
    }
  } else {
    const double2* q = reinterpret_cast<const double2*>(x) + 2 * site;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const double2 a = ld2<CG>(q + 2 * i * V), b = ld2<CG>(q + 2 * i * V + 1);
      p.s[2 * i] = {a.x, a.y};
      p.s[2 * i + 1] = {b.x, b.y};
    }
  }
}

// components (2p, 2p+1) of site s
template <typename R> DEV void load_pair(const cx<R>* x, long V, long site, int p, cx<R>& a, cx<R>& b) {
  if constexpr (sizeof(R) == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(x) + p * V + site);
    a = {v.x, v.y};
    b = {v.z, v.w};
  } else {
    const double2* q = reinterpret_cast<const double2*>(x) + 2 * (p * V + site);
    const double2 u = __ldg(q), w = __ldg(q + 1);
    a = {u.x, u.y};
    b = {w.x, w.y};
  }
}
template <typename R> DEV void store_pair(cx<R>* y, long V, long site, int p, cx<R> a, cx<R> b) {
  if constexpr (sizeof(R) == 4) {
    reinterpret_cast<float4*>(y)[p * V + site] = make_float4(a.x, a.y, b.x, b.y);
  } else {
    double2* q = reinterpret_cast<double2*>(y) + 2 * (p * V + site);
    q[0] = make_double2(a.x, a.y);
    q[1] = make_double2(b.x, b.y);
  }
}

// lattice coordinates of a site (32-bit division: V < 2^31)
DEV void site_coords(long site, int Lx, int Ly, int Lz, int& ix, int& iy, int& iz, int& it) {
  unsigned q = (unsigned)site;
  ix = (int)(q % (unsigned)Lx); q /= (unsigned)Lx;
  iy = (int)(q % (unsigned)Ly); q /= (unsigned)Ly;
  iz = (int)(q % (unsigned)Lz);
  it = (int)(q / (unsigned)Lz);
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
  load_spinor<R, CG>(x, V, fwd, pf);
  load_spinor<R, CG>(x, V, bwd, pb);
  hop<MU, true, R, LT>(links, V, site, pf, acc);
  hop<MU, false, R, LT>(links, V, bwd, pb, acc);
}

}  // namespace
