// sm_103a kernels of the bucket-elimination hot path.
//
// §Tensor network contraction: a bucket multiplies every tensor that holds
// the eliminated variable and sums over it.  With indices ordered by
// elimination position (qt_device.h) one output row y of a bucket is
//     out[y] = sum_{x in {0,1}} prod_i in_i[(pext(y, mask_i) << 1) | x]
// which these kernels evaluate as a stream: for every input a gather of the
// row pair (x = 0, 1), complex products in registers, one add for the sum
// over x, one store.  The work is HBM-bound (about 1 flop per byte), so the
// kernels are organised around coalesced, vectorised loads:
//   * angle sets are the innermost axis: a warp reads 32 x 16 contiguous bytes
//     of every input row (B >= 2, complex64 packs two angle sets per 16 B);
//   * with one angle set (B = 1) the pair x = 0, 1 of an input is adjacent and
//     complex64 loads it as one 16-byte vector.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "qt_device.h"

namespace qt {
namespace dev {

template <class Real> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <class Real>
__device__ __forceinline__ typename Cx<Real>::T cmul(typename Cx<Real>::T a, typename Cx<Real>::T b) {
  typename Cx<Real>::T r;
  r.x = fma(a.x, b.x, -a.y * b.y);
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}

template <class Real>
__device__ __forceinline__ typename Cx<Real>::T cadd(typename Cx<Real>::T a, typename Cx<Real>::T b) {
  typename Cx<Real>::T r;
  r.x = a.x + b.x;
  r.y = a.y + b.y;
  return r;
}

// VB consecutive complex numbers.
template <class Real, int VB> struct Pack { typename Cx<Real>::T c[VB]; };

template <class Real, int VB, bool CG>
__device__ __forceinline__ Pack<Real, VB> ldv(const Real* data, int64_t elem);

template <> __device__ __forceinline__ Pack<float, 2> ldv<float, 2, true>(const float* d, int64_t e) {
  float4 v = __ldcg(reinterpret_cast<const float4*>(d + 2 * e));
  return Pack<float, 2>{{make_float2(v.x, v.y), make_float2(v.z, v.w)}};
}
template <> __device__ __forceinline__ Pack<float, 2> ldv<float, 2, false>(const float* d, int64_t e) {
  float4 v = *reinterpret_cast<const float4*>(d + 2 * e);
  return Pack<float, 2>{{make_float2(v.x, v.y), make_float2(v.z, v.w)}};
}
template <> __device__ __forceinline__ Pack<float, 1> ldv<float, 1, true>(const float* d, int64_t e) {
  return Pack<float, 1>{{__ldcg(reinterpret_cast<const float2*>(d + 2 * e))}};
}
template <> __device__ __forceinline__ Pack<float, 1> ldv<float, 1, false>(const float* d, int64_t e) {
  return Pack<float, 1>{{*reinterpret_cast<const float2*>(d + 2 * e)}};
}
template <> __device__ __forceinline__ Pack<double, 1> ldv<double, 1, true>(const double* d, int64_t e) {
  return Pack<double, 1>{{__ldcg(reinterpret_cast<const double2*>(d + 2 * e))}};
}
template <> __device__ __forceinline__ Pack<double, 1> ldv<double, 1, false>(const double* d, int64_t e) {
  return Pack<double, 1>{{*reinterpret_cast<const double2*>(d + 2 * e)}};
}

// Two adjacent complex numbers (element e even, 16-byte aligned for complex64).
template <class Real, bool CG>
__device__ __forceinline__ Pack<Real, 2> ldpair(const Real* data, int64_t e);
template <> __device__ __forceinline__ Pack<float, 2> ldpair<float, true>(const float* d, int64_t e) {
  return ldv<float, 2, true>(d, e);
}
template <> __device__ __forceinline__ Pack<float, 2> ldpair<float, false>(const float* d, int64_t e) {
  return ldv<float, 2, false>(d, e);
}
template <> __device__ __forceinline__ Pack<double, 2> ldpair<double, true>(const double* d, int64_t e) {
  return Pack<double, 2>{{__ldcg(reinterpret_cast<const double2*>(d + 2 * e)),
                          __ldcg(reinterpret_cast<const double2*>(d + 2 * e + 2))}};
}
template <> __device__ __forceinline__ Pack<double, 2> ldpair<double, false>(const double* d, int64_t e) {
  return Pack<double, 2>{{*reinterpret_cast<const double2*>(d + 2 * e),
                          *reinterpret_cast<const double2*>(d + 2 * e + 2)}};
}

template <class Real, int VB>
__device__ __forceinline__ void stv(Real* d, int64_t e, const Pack<Real, VB>& p);
template <> __device__ __forceinline__ void stv<float, 2>(float* d, int64_t e, const Pack<float, 2>& p) {
  *reinterpret_cast<float4*>(d + 2 * e) = make_float4(p.c[0].x, p.c[0].y, p.c[1].x, p.c[1].y);
}
template <> __device__ __forceinline__ void stv<float, 1>(float* d, int64_t e, const Pack<float, 1>& p) {
  *reinterpret_cast<float2*>(d + 2 * e) = p.c[0];
}
template <> __device__ __forceinline__ void stv<double, 1>(double* d, int64_t e, const Pack<double, 1>& p) {
  *reinterpret_cast<double2*>(d + 2 * e) = p.c[0];
}

// Input row index bits: pext(y, mask) from the precomputed runs.
__device__ __forceinline__ uint32_t pext_in(uint32_t y, const DevInput& in) {
  uint32_t k = 0;
  if (in.nruns >= 0) {
    for (int r = 0; r < in.nruns; ++r) {
      const uint32_t w = in.run[r];
      const uint32_t src = w & 31u, len = (w >> 8) & 63u, dst = (w >> 16) & 31u;
      k |= ((y >> src) & ((1u << len) - 1u)) << dst;
    }
  } else {
    uint32_t m = in.mask;
    int j = 0;
    while (m) {
      const uint32_t low = m & (0u - m);
      if (y & low) k |= 1u << j;
      ++j;
      m ^= low;
    }
  }
  return k;
}

// Rows/vectors of one bucket in [e0, e1), work items split over `nthr` threads.
// PAIR (B == 1): item = output row y.  Otherwise item = (y, v) with v the
// vector of VB angle sets, items per row = B / VB = 1 << bshift when
// bshift >= 0, else B / VB by division.
template <class Real, int VB, bool PAIR, bool CG>
__device__ __forceinline__ void bucket_range(const DevBucket& d, Real* __restrict__ data, int32_t B,
                                             int32_t bshift, int64_t e0, int64_t e1, int64_t tid,
                                             int64_t nthr) {
  using C = typename Cx<Real>::T;
  const int32_t bv_per_row = B / VB;
  const int n_in = d.n_in;
  for (int64_t e = e0 + tid; e < e1; e += nthr) {
    int64_t y, bv;
    if (PAIR) {
      y = e;
      bv = 0;
    } else if (bshift >= 0) {
      y = e >> bshift;
      bv = e - (y << bshift);
    } else {
      y = e / bv_per_row;
      bv = e - y * bv_per_row;
    }
    if (PAIR) {
      C p0, p1;
      for (int i = 0; i < n_in; ++i) {
        const DevInput& in = d.in[i];
        const int64_t r0 = in.off + 2 * (int64_t)pext_in((uint32_t)y, in);
        const Pack<Real, 2> q = ldpair<Real, CG>(data, r0);  // rows x = 0 and x = 1
        const C a0 = q.c[0], a1 = q.c[1];
        if (i == 0) {
          p0 = a0;
          p1 = a1;
        } else {
          p0 = cmul<Real>(p0, a0);
          p1 = cmul<Real>(p1, a1);
        }
      }
      Pack<Real, 1> o{{cadd<Real>(p0, p1)}};
      stv<Real, 1>(data, d.out_off + y, o);
    } else {
      Pack<Real, VB> p0, p1;
      for (int i = 0; i < n_in; ++i) {
        const DevInput& in = d.in[i];
        const int64_t r0 = 2 * (int64_t)pext_in((uint32_t)y, in);
        const int64_t base = in.off + r0 * B + bv * VB;
        Pack<Real, VB> a0 = ldv<Real, VB, CG>(data, base);
        Pack<Real, VB> a1 = ldv<Real, VB, CG>(data, base + B);
        if (i == 0) {
          p0 = a0;
          p1 = a1;
        } else {
#pragma unroll
          for (int v = 0; v < VB; ++v) {
            p0.c[v] = cmul<Real>(p0.c[v], a0.c[v]);
            p1.c[v] = cmul<Real>(p1.c[v], a1.c[v]);
          }
        }
      }
      Pack<Real, VB> o;
#pragma unroll
      for (int v = 0; v < VB; ++v) o.c[v] = cadd<Real>(p0.c[v], p1.c[v]);
      stv<Real, VB>(data, d.out_off + y * B + bv * VB, o);
    }
  }
}

}  // namespace dev
}  // namespace qt
