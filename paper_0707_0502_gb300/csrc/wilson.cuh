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
  // each complex multiply-add as four FMAs into the accumulator (a product followed by
  // an add would take six floating-point operations: the FP64 residual matvec is bound
  // by them, the complex64 one by instruction issue)
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const cx<R> u = LinkLd<R, LT>::ld(L, (long)(a * 3 + b) * V);
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        if (FWD) {  // g_a += U_ab h_b
          cx<R>& t = g[sp][a];
          const cx<R> hb = h[sp][b];
          t.x = fma(-u.y, hb.y, fma(u.x, hb.x, t.x));
          t.y = fma(u.y, hb.x, fma(u.x, hb.y, t.y));
        } else {    // g_b += conj(U_ab) h_a
          cx<R>& t = g[sp][b];
          const cx<R> ha = h[sp][a];
          t.x = fma(u.y, ha.y, fma(u.x, ha.x, t.x));
          t.y = fma(-u.y, ha.x, fma(u.x, ha.y, t.y));
        }
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

// ---- two columns per thread, packed FP32x2 arithmetic (sm_100 and later)
// A pair value holds one real component of two columns: column 2p in the low lane,
// 2p + 1 in the high lane.  One packed FMA does the work of two scalar ones, and the
// link (the same for both columns) is loaded and converted once for both.
typedef unsigned long long f2;
DEV f2 f2_pack(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
DEV void f2_unpack(f2 v, float& lo, float& hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
DEV f2 f2_add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
DEV f2 f2_sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
DEV f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
DEV f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
struct cx2 {
  f2 re, im;
};
struct Spinor2 {
  cx2 s[12];
};

// u + ph z with ph = 1, i, -1, -i for PH = 0..3
template <int PH>
DEV cx2 addph(cx2 u, cx2 z) {
  if (PH == 0) return {f2_add(u.re, z.re), f2_add(u.im, z.im)};
  if (PH == 1) return {f2_sub(u.re, z.im), f2_add(u.im, z.re)};
  if (PH == 2) return {f2_sub(u.re, z.re), f2_sub(u.im, z.im)};
  return {f2_add(u.re, z.im), f2_sub(u.im, z.re)};
}

// the spinors of site `site` in columns x0 and x1 (pair-major order)
DEV void load_spinor2(const c64* x0, const c64* x1, long V, long site, Spinor2& p) {
  const float4* q0 = reinterpret_cast<const float4*>(x0) + site;
  const float4* q1 = reinterpret_cast<const float4*>(x1) + site;
  float4 a[6], b[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    a[i] = __ldg(q0 + i * V);
    b[i] = __ldg(q1 + i * V);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    p.s[2 * i] = {f2_pack(a[i].x, b[i].x), f2_pack(a[i].y, b[i].y)};
    p.s[2 * i + 1] = {f2_pack(a[i].z, b[i].z), f2_pack(a[i].w, b[i].w)};
  }
}

// The phases of one hop, read off b_mul / bh_mul: with backward-hop signs, the half
// spinor is h_0 = u_0 + ph z_0, h_1 = u_1 + ph' z_1 (z from the lower components d_0,
// d_1) and the lower components gain ph g (from g_0 or g_1); the forward hop negates
// every term (PH + 2).
template <int MU> struct HopTab;
template <> struct HopTab<0> { static constexpr int h0z = 1, h0p = 3, h1z = 0, h1p = 3, r6g = 1, r6p = 1, r9g = 0, r9p = 1; };
template <> struct HopTab<1> { static constexpr int h0z = 1, h0p = 2, h1z = 0, h1p = 0, r6g = 1, r6p = 0, r9g = 0, r9p = 2; };
template <> struct HopTab<2> { static constexpr int h0z = 0, h0p = 3, h1z = 1, h1p = 1, r6g = 0, r6p = 1, r9g = 1, r9p = 3; };
template <> struct HopTab<3> { static constexpr int h0z = 0, h0p = 0, h1z = 1, h1p = 0, r6g = 0, r6p = 0, r9g = 1, r9p = 0; };

// one hop for two columns (see hop): FWD (1 - gamma) U(x) psi(x+mu), else (1 + gamma) U(x-mu)^H psi(x-mu);
// ldu(e) gives link element e = a*3 + b of the hop's link
template <int MU, bool FWD, typename LoadU>
DEV void hop2_core(const Spinor2& p, LoadU ldu, Spinor2& acc) {
  using T = HopTab<MU>;
  constexpr int S = FWD ? 2 : 0;
  cx2 h[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cx2 d[2] = {p.s[6 + a], p.s[9 + a]};
    h[0][a] = addph<(T::h0p + S) & 3>(p.s[a], d[T::h0z]);
    h[1][a] = addph<(T::h1p + S) & 3>(p.s[3 + a], d[T::h1z]);
  }
  cx2 g[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) g[0][a] = g[1][a] = {0ull, 0ull};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const c64 u = ldu(a * 3 + b);
      const f2 ur = f2_pack(u.x, u.x), ui = f2_pack(u.y, u.y), nui = f2_pack(-u.y, -u.y);
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        if (FWD) {  // g_a += U_ab h_b
          cx2& t = g[sp][a];
          const cx2 hb = h[sp][b];
          t.re = f2_fma(nui, hb.im, f2_fma(ur, hb.re, t.re));
          t.im = f2_fma(ui, hb.re, f2_fma(ur, hb.im, t.im));
        } else {    // g_b += conj(U_ab) h_a
          cx2& t = g[sp][b];
          const cx2 ha = h[sp][a];
          t.re = f2_fma(ui, ha.im, f2_fma(ur, ha.re, t.re));
          t.im = f2_fma(nui, ha.re, f2_fma(ur, ha.im, t.im));
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc.s[a] = addph<0>(acc.s[a], g[0][a]);
    acc.s[3 + a] = addph<0>(acc.s[3 + a], g[1][a]);
    acc.s[6 + a] = addph<(T::r6p + S) & 3>(acc.s[6 + a], g[T::r6g][a]);
    acc.s[9 + a] = addph<(T::r9p + S) & 3>(acc.s[9 + a], g[T::r9g][a]);
  }
}

template <int MU, bool FWD, typename LT>
DEV void hop2(const LT* __restrict__ links, long V, long lsite, const Spinor2& p, Spinor2& acc) {
  const LT* L = links + (long)MU * 9 * V + lsite;
  hop2_core<MU, FWD>(p, [&](int e) { return LinkLd<float, LT>::ld(L, (long)e * V); }, acc);
}

template <int MU, typename LT>
DEV void hop_mu2(const LT* __restrict__ links, const c64* x0, const c64* x1, long V, long site, int coord, int L,
                 long stride, Spinor2& acc) {
  const long fwd = (coord == L - 1) ? site - (long)(L - 1) * stride : site + stride;
  const long bwd = (coord == 0) ? site + (long)(L - 1) * stride : site - stride;
  Spinor2 p;
  load_spinor2(x0, x1, V, fwd, p);
  hop2<MU, true, LT>(links, V, site, p, acc);
  load_spinor2(x0, x1, V, bwd, p);
  hop2<MU, false, LT>(links, V, bwd, p, acc);
}

}  // namespace
