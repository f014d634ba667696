// 16-byte vector units shared by the Krylov kernels: two complex64 or one
// complex128 per unit, loaded and stored as one float4 / double2 (a trailing odd
// complex64 element is handled alone).
#pragma once

#include "common.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

// 16-byte units: 2 complex64 or 1 complex128
template <typename R> struct U { static constexpr int K = 16 / (2 * sizeof(R)); };

template <typename R> DEV void ldu(const cx<R>* p, long u, long n, cx<R> (&o)[U<R>::K]);
template <> DEV void ldu<float>(const c64* p, long u, long n, c64 (&o)[2]) {
  if (2 * u + 1 < n) {
    float4 v = *(reinterpret_cast<const float4*>(p) + u);
    o[0] = {v.x, v.y};
    o[1] = {v.z, v.w};
  } else {
    o[0] = p[2 * u];
    o[1] = {0.f, 0.f};
  }
}
template <> DEV void ldu<double>(const c128* p, long u, long, c128 (&o)[1]) {
  double2 v = *(reinterpret_cast<const double2*>(p) + u);
  o[0] = {v.x, v.y};
}
template <typename R> DEV void stu(cx<R>* p, long u, long n, const cx<R> (&o)[U<R>::K]);
template <> DEV void stu<float>(c64* p, long u, long n, const c64 (&o)[2]) {
  if (2 * u + 1 < n) {
    *(reinterpret_cast<float4*>(p) + u) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
  } else {
    p[2 * u] = o[0];
  }
}
template <> DEV void stu<double>(c128* p, long u, long, const c128 (&o)[1]) {
  *(reinterpret_cast<double2*>(p) + u) = make_double2(o[0].x, o[0].y);
}
template <typename R> HD long nunits(long n) { return (n + U<R>::K - 1) / U<R>::K; }

// units per lane of a dot tile (a tile of w is DU * 32 units)
template <typename R> struct DotTile { static constexpr int DU = (U<R>::K == 2) ? 16 : 8; };

}  // namespace
