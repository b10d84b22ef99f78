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
#include <type_traits>

#include "qt_device.h"
#include "qtensor.h"

namespace qt {
namespace dev {

// A real number as an unevaluated sum of two floats, hi + lo with |lo| at
// most half an ulp of hi: about 48 significant bits, all arithmetic on the
// FP32 pipes (this GPU's FP64 rate is a small fraction of its FP32 rate).
// Products use the FMA-exact product error (Dekker's two-product through a
// fused multiply-add), sums Knuth's two-sum; each result is renormalised.
// The relative error of a product or sum is a few units of 2^-46.
struct ff {
  float hi, lo;
  ff() = default;
  __device__ __forceinline__ ff(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ ff(int v) : hi((float)v), lo(0.f) {}
  __device__ __forceinline__ ff(double v) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ ff ff_renorm(float s, float e) {
  const float h = s + e;
  return ff(h, e - (h - s));
}
__device__ __forceinline__ ff operator+(ff a, ff b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
  return ff_renorm(s, e);
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p) + fmaf(a.hi, b.lo, a.lo * b.hi);
  return ff_renorm(p, e);
}

// a * b + c, fused where the type has a fused multiply-add
__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ ff fmad(ff a, ff b, ff c) { return a * b + c; }

struct ff2 {
  ff x, y;
};

template <class Real> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<ff> { using T = ff2; };

template <class Real>
__device__ __forceinline__ typename Cx<Real>::T cmul(typename Cx<Real>::T a, typename Cx<Real>::T b) {
  typename Cx<Real>::T r;
  r.x = fmad(a.x, b.x, -a.y * b.y);
  r.y = fmad(a.x, b.y, a.y * b.x);
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

// Float pairs: one complex number is 16 bytes (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ ff2 ff2_of(float4 v) { return ff2{ff(v.x, v.y), ff(v.z, v.w)}; }
template <> __device__ __forceinline__ Pack<ff, 1> ldv<ff, 1, true>(const ff* d, int64_t e) {
  return Pack<ff, 1>{{ff2_of(__ldcg(reinterpret_cast<const float4*>(d + 2 * e)))}};
}
template <> __device__ __forceinline__ Pack<ff, 1> ldv<ff, 1, false>(const ff* d, int64_t e) {
  return Pack<ff, 1>{{ff2_of(*reinterpret_cast<const float4*>(d + 2 * e))}};
}
template <> __device__ __forceinline__ Pack<ff, 2> ldpair<ff, true>(const ff* d, int64_t e) {
  return Pack<ff, 2>{{ff2_of(__ldcg(reinterpret_cast<const float4*>(d + 2 * e))),
                      ff2_of(__ldcg(reinterpret_cast<const float4*>(d + 2 * e + 2)))}};
}
template <> __device__ __forceinline__ Pack<ff, 2> ldpair<ff, false>(const ff* d, int64_t e) {
  return Pack<ff, 2>{{ff2_of(*reinterpret_cast<const float4*>(d + 2 * e)),
                      ff2_of(*reinterpret_cast<const float4*>(d + 2 * e + 2))}};
}
template <> __device__ __forceinline__ void stv<ff, 1>(ff* d, int64_t e, const Pack<ff, 1>& p) {
  *reinterpret_cast<float4*>(d + 2 * e) = make_float4(p.c[0].x.hi, p.c[0].x.lo, p.c[0].y.hi, p.c[0].y.lo);
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

// Deposit the low bits of x into the set bits of the record's mask (the
// inverse of pext_in), from the same runs with source and destination swapped.
__device__ __forceinline__ uint32_t pdep_in(uint32_t x, const DevInput& in) {
  uint32_t y = 0;
  if (in.nruns >= 0) {
    for (int r = 0; r < in.nruns; ++r) {
      const uint32_t w = in.run[r];
      const uint32_t ybit = w & 31u, len = (w >> 8) & 63u, xbit = (w >> 16) & 31u;
      y |= ((x >> xbit) & ((1u << len) - 1u)) << ybit;
    }
  } else {
    uint32_t m = in.mask;
    int j = 0;
    while (m) {
      const uint32_t low = m & (0u - m);
      if ((x >> j) & 1u) y |= low;
      ++j;
      m ^= low;
    }
  }
  return y;
}

#ifdef QT_DEVICE_CHECKS
// Debug build: an element range outside the data region is recorded in the
// control word (first failure wins) and the access is skipped.
__device__ __forceinline__ bool qt_in_range(DevCtrl* ctrl, int64_t lo, int64_t span, int64_t n, int kind,
                                            int bucket, int input) {
  if (lo >= 0 && lo + span <= n) return true;
  if (ctrl && atomicCAS(&ctrl->bad_kind, 0, kind) == 0) {
    ctrl->bad_bucket = bucket;
    ctrl->bad_input = input;
    ctrl->bad_index = lo;
    atomicCAS(&ctrl->status, 0, (int32_t)QT_EINVAL);
  }
  return false;
}
#define QT_RANGE_OK(lo, span, kind, input) qt_in_range(ctrl, (lo), (span), g.data_elems, (kind), dbg_bucket, (input))
#else
#define QT_RANGE_OK(lo, span, kind, input) true
#endif

// Per-warp shared state of one tile: the bucket record and the pass table
// tab[i][p] = pext(r0 + p * RP, mask_i).

struct WarpTile {
  DevBucket d;
  uint32_t tab[kDevMaxIn][kLaneItems];
  uint32_t lpart[kDevMaxIn][32];  // pext(i_lane, mask) per input and lane
  union {  // an adjoint reduction step's partial sums or a chained forward step's held rows
    struct {
      float f[32][4];             // per-lane partial sums of a reduction step (complex64)
      double d[32][2];            // the same for complex128
    } red;
    float4 chainh[kMaxChain - 1][32];  // per chain level below the last and lane: its held even row
  } x;
  unsigned long long trace_t[2];        // queue trace: claim and ready clock of the current task
};

// Copy a bucket record into the warp's shared slot with typed member
// assignments (lane i < kDevMaxIn copies input slot i, lane 31 the header),
// so every later read of the slot sees the stores through its own type.  Call
// with all 32 lanes; the caller synchronises the warp before reading the
// slot.  Every input slot is copied (the host zero-fills unused ones), so the
// records a step reads past its factors (target, completion and chain
// records) never come from an earlier step.
__device__ __forceinline__ void load_bucket(DevBucket* dst, const DevBucket* src, int lane) {
  if (lane < kDevMaxIn) dst->in[lane] = src->in[lane];
  if (lane == 31) {
    dst->out_off = src->out_off;
    dst->n_rows = src->n_rows;
    dst->out_rank = src->out_rank;
    dst->n_in = src->n_in;
    dst->dep = src->dep;
    dst->ntask = src->ntask;
    dst->kind = src->kind;
    dst->aflags = src->aflags;
    dst->tgt_bits = src->tgt_bits;
    dst->comp_bits = src->comp_bits;
    dst->span = src->span;
    dst->n_dep = src->n_dep;
    dst->chain = src->chain;
    dst->chain_noleaf = src->chain_noleaf;
  }
}

// The same copy for every record slot: lanes 0 .. kDevMaxIn - 1 copy input
// slot `lane` whatever the step's fan-in (the host zero-fills unused slots,
// so the shared copy holds no stale entries), lane 31 the header.  It needs
// no field of the record first, so its loads go out at once.
__device__ __forceinline__ void copy_bucket(DevBucket* dst, const DevBucket* src, int lane) {
  if (lane < kDevMaxIn) dst->in[lane] = src->in[lane];
  if (lane == 31) {
    dst->out_off = src->out_off;
    dst->n_rows = src->n_rows;
    dst->out_rank = src->out_rank;
    dst->n_in = src->n_in;
    dst->dep = src->dep;
    dst->ntask = src->ntask;
    dst->kind = src->kind;
    dst->aflags = src->aflags;
    dst->tgt_bits = src->tgt_bits;
    dst->comp_bits = src->comp_bits;
    dst->span = src->span;
    dst->n_dep = src->n_dep;
    dst->chain = src->chain;
    dst->chain_noleaf = src->chain_noleaf;
  }
}

template <class Real, bool CG>
__device__ __forceinline__ Pack<Real, 2> ldpair_in(const Real* data, int64_t e, bool leaf) {
  return leaf ? ldpair<Real, false>(data, e) : ldpair<Real, CG>(data, e);
}
template <class Real, int VB, bool CG>
__device__ __forceinline__ Pack<Real, VB> ldv_in(const Real* data, int64_t e, bool leaf) {
  return leaf ? ldv<Real, VB, false>(data, e) : ldv<Real, VB, CG>(data, e);
}

// One row of a factor flagged kInNoPair (one value for x = 0 and x = 1) on
// the one-angle-set layout.  Float-pair plans keep every adjoint tensor in
// FP64 (flag kInF64: FP64 has native atomic adds, a float pair only a
// compare-and-swap loop, and FP64 carries at least a float pair's precision);
// such a factor is read as FP64 and split into a float pair here.
template <class Real>
__device__ __forceinline__ Pack<Real, 1> ld_nopair(const Real* data, int64_t e, int32_t fl) {
  if constexpr (std::is_same<Real, ff>::value) {
    if (fl & kInF64) {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(data) + e);
      Pack<ff, 1> r;
      r.c[0].x = ff(v.x);
      r.c[0].y = ff(v.y);
      return r;
    }
  }
  return ldv_in<Real, 1, true>(data, e, fl & kInLeaf);
}

// Lane -> (row within a pass, vector) of the tile geometry.
__device__ __forceinline__ void lane_slot(const TileGeom& g, int lane, int* rip, int* v0, bool* on) {
  if (g.Bv <= 32) {
    *rip = lane / g.Bv;
    *v0 = lane - *rip * g.Bv;
    *on = *rip < g.RP;
  } else {
    *rip = 0;
    *v0 = lane;
    *on = true;
  }
}

// Per-lane part pext(i_lane, mask) of every input of the bucket in w->d,
// into w->lpart.  Call with all 32 lanes after the record is in place; the
// caller synchronises the warp before the parts are read.
__device__ __forceinline__ void lane_parts(WarpTile* w, const TileGeom& g, int lane) {
  int rip, v0;
  bool on;
  lane_slot(g, lane, &rip, &v0, &on);
  const bool red_low = w->d.kind == kStepAdjRed && (w->d.aflags & kAdjRedLow);
  if (w->d.kind == kStepAdjRed && !red_low) {  // lanes index completions: part of y = pdep(i_lane, complement)
    const uint32_t ylane = pdep_in((uint32_t)rip, w->d.in[w->d.n_in + 1]);
    for (int i = 0; i < w->d.n_in; ++i) w->lpart[i][lane] = pext_in(ylane, w->d.in[i]);
    return;
  }
  const int n_rec = w->d.kind == kStepAdj || red_low ? w->d.n_in + 1 : w->d.n_in + w->d.chain;
  for (int i = 0; i < n_rec; ++i) w->lpart[i][lane] = pext_in((uint32_t)rip, w->d.in[i]);
}

// U items of one lane: output row, vector of angle sets, pass, valid flag.
template <int U> struct ItemSet {
  int pp[U];
  uint32_t y[U];  // output rows < 2^31
  int32_t vv[U];
  bool ok[U];
};

template <int U>
__device__ __forceinline__ ItemSet<U> make_items(const TileGeom& g, int q0, int Q, int64_t r0, int64_t r1, int rip,
                                                 int v0, bool lane_on) {
  ItemSet<U> it;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int q = q0 + u;
    const int p = q / g.VC;
    const int vc = q - p * g.VC;
    it.pp[u] = q < Q ? p : 0;
    it.y[u] = (uint32_t)r0 + (uint32_t)(it.pp[u] * g.RP + rip);
    it.vv[u] = vc * 32 + v0;
    it.ok[u] = lane_on && q < Q && (int64_t)it.y[u] < r1 && (g.Bv <= 32 || it.vv[u] < g.Bv);
    if (!it.ok[u]) {  // idle items read a valid element and do not store
      it.y[u] = (uint32_t)r0;
      it.vv[u] = 0;
    }
  }
  return it;
}

// Loads of input i for U items: a0 = rows x = 0, a1 = rows x = 1 (for PAIR,
// VB = 1 and both come from one adjacent pair).
template <class Real, int VB, bool PAIR, bool CG, int U>
__device__ __forceinline__ void load_input(const WarpTile* w, int i, uint32_t lp_i, const ItemSet<U>& it,
                                           Real* __restrict__ data, const TileGeom& g, Pack<Real, VB>* a0,
                                           Pack<Real, VB>* a1, DevCtrl* ctrl, int dbg_bucket) {
  (void)ctrl;
  (void)dbg_bucket;
  const int64_t off = w->d.in[i].off;
  const bool leaf = w->d.in[i].flags & kInLeaf;
  const bool nopair = w->d.in[i].flags & kInNoPair;
  const int B = g.B;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const uint32_t k = it.ok[u] ? w->tab[i][it.pp[u]] + lp_i : 0u;
    if (nopair) {  // one row k, the same factor for x = 0 and x = 1
      const int64_t base = PAIR ? off + (int64_t)k : off + (int64_t)k * B + (int64_t)(it.vv[u] * VB);
      if (QT_RANGE_OK(base, VB, 1, i)) {
        a0[u] = ldv_in<Real, VB, CG>(data, base, leaf);
        a1[u] = a0[u];
      } else {
        a0[u] = Pack<Real, VB>{};
        a1[u] = Pack<Real, VB>{};
      }
    } else if (PAIR) {
      if (QT_RANGE_OK(off + 2 * (int64_t)k, 2, 1, i)) {
        const Pack<Real, 2> q = ldpair_in<Real, CG>(data, off + 2 * (int64_t)k, leaf);
        a0[u].c[0] = q.c[0];
        a1[u].c[0] = q.c[1];
      } else {
        a0[u] = Pack<Real, VB>{};
        a1[u] = Pack<Real, VB>{};
      }
    } else {
      const int64_t base = off + (int64_t)(2 * k) * B + (int64_t)(it.vv[u] * VB);
      if (QT_RANGE_OK(base, B + VB, 1, i)) {
        a0[u] = ldv_in<Real, VB, CG>(data, base, leaf);
        a1[u] = ldv_in<Real, VB, CG>(data, base + B, leaf);
      } else {
        a0[u] = Pack<Real, VB>{};
        a1[u] = Pack<Real, VB>{};
      }
    }
  }
}

template <class Real, int VB>
__device__ __forceinline__ void pmul(Pack<Real, VB>& p, const Pack<Real, VB>& a) {
#pragma unroll
  for (int v = 0; v < VB; ++v) p.c[v] = cmul<Real>(p.c[v], a.c[v]);
}

// Items of one tile: for each input in turn, the loads of U items, then
// their products.  (NIN > 0 would fix the fan-in at compile time and issue
// the loads of all inputs first; that variant is not instantiated: builds
// that used it faulted on the GPU although their index arithmetic checks out
// on the CPU.)
template <class Real, int VB, bool PAIR, bool CG, int U, int NIN>
__device__ __forceinline__ void tile_items(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                           int64_t r1, int lane, int rip, int v0, bool lane_on, DevCtrl* ctrl,
                                           int dbg_bucket) {
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  const int Q = g.P * g.VC;
  const int B = g.B;
  for (int q0 = 0; q0 < Q; q0 += U) {
    const ItemSet<U> it = make_items<U>(g, q0, Q, r0, r1, rip, v0, lane_on);
    Pack<Real, VB> p0[U], p1[U];
    if (NIN > 0) {
      Pack<Real, VB> a0[NIN > 0 ? NIN : 1][U], a1[NIN > 0 ? NIN : 1][U];
#pragma unroll
      for (int i = 0; i < NIN; ++i)
        load_input<Real, VB, PAIR, CG, U>(w, i, w->lpart[i][lane], it, data, g, a0[i], a1[i], ctrl, dbg_bucket);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        p0[u] = a0[0][u];
        p1[u] = a1[0][u];
#pragma unroll
        for (int i = 1; i < NIN; ++i) {
          pmul<Real, VB>(p0[u], a0[i][u]);
          pmul<Real, VB>(p1[u], a1[i][u]);
        }
      }
    } else {
      for (int i = 0; i < n_in; ++i) {
        Pack<Real, VB> a0[U], a1[U];
        load_input<Real, VB, PAIR, CG, U>(w, i, w->lpart[i][lane], it, data, g, a0, a1, ctrl, dbg_bucket);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (i == 0) {
            p0[u] = a0[u];
            p1[u] = a1[u];
          } else {
            pmul<Real, VB>(p0[u], a0[u]);
            pmul<Real, VB>(p1[u], a1[u]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!it.ok[u]) continue;
      Pack<Real, VB> o;
#pragma unroll
      for (int v = 0; v < VB; ++v) o.c[v] = cadd<Real>(p0[u].c[v], p1[u].c[v]);
      const int64_t so = PAIR ? d.out_off + (int64_t)it.y[u]
                              : d.out_off + (int64_t)it.y[u] * B + (int64_t)(it.vv[u] * VB);
      if (QT_RANGE_OK(so, VB, 2, -1)) stv<Real, VB>(data, so, o);
    }
  }
}

// Row-wide forward tile on the register path (RP = 1, VC = 1: every lane of
// the warp works on the same output row, lane l on vector l).  The same loads
// and products as tile_items, two rows per iteration, with the row's operand
// rows read straight from the pass table (the lane part is 0) and no
// per-item bookkeeping; bit-identical to tile_items.  Measured on the bench
// step: two rows per iteration 19.4 ms, one row 24.1 ms, four rows 30.6 ms.
//
// Steps of fan-in 2 and 3 take tile_rows_fixed: the same loads, products and
// order, with the fan-in and the leaf factor's slot (the last input, when
// there is one) fixed at compile time, so each input's base offset stays in a
// register for the tile and no per-row record read, leaf test or loop
// control is left.  It reads exactly inputs 0 .. n_in - 1 of the record.
// Measured on the bench step (kernel time, 64 angle sets): the rolled tile 17.56 ms, this tile with
// two rows per iteration 17.10 ms, with one 17.45 ms (bit-identical results); fan-in 4 spills.
constexpr int kFixedRows = 2;      // output rows per iteration of tile_rows_fixed
constexpr int kFixedMaxFanIn = 3;  // fan-in up to which steps take tile_rows_fixed
static_assert(kFixedRows == 2, "chained steps combine the rows w = 0, 1 of one iteration");

// Chained steps (chain = m > 0, STAGE 4 kernels), row-wide layout: one row y
// of b per iteration.  Its value G_b[y] (the product-sum, never stored) times
// c_1's leaf row L_1[pext(y, chain mask 1)] (the mask's bit 0 is bit 0 of y,
// c_1's eliminated variable) is c_1's term for w_1 = bit 0 of y: an even row
// keeps it (acc), an odd row adds it to the kept one, which completes c_1's
// row y >> 1.  That row times c_2's leaf row at pext(y, chain mask 2) (bit 0
// = bit 1 of y) is c_2's term, kept or added the same way (held per lane in
// the warp's shared slot), and so on up to c_m, whose completed row is the
// output.  Every term and sum takes the consumer's own operands in its own
// order (the intermediate row, then the leaf; the term of w = 0 first), so a
// chained step is bit-identical to the separate steps.  One row per
// iteration and one kept term keep the tile within the 64-register budget
// (two rows per iteration and their leaf rows spilled, and the spills slowed
// every tile of the kernel).
template <class T>
__device__ __forceinline__ float4 as_float4(const T& x) {
  static_assert(sizeof(T) <= sizeof(float4), "a held chain term is at most 16 bytes per lane");
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  memcpy(&r, &x, sizeof(T));
  return r;
}
template <class T>
__device__ __forceinline__ T from_float4(const float4& x) {
  static_assert(sizeof(T) <= sizeof(float4), "a held chain term is at most 16 bytes per lane");
  T r;
  memcpy(&r, &x, sizeof(T));
  return r;
}

template <class Real, int VB, int NIN, bool LEAF>
__device__ __forceinline__ void tile_rows_chain(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                                int64_t r1, int lane) {
  using PK = Pack<Real, VB>;
  const DevBucket& d = w->d;
  const int n_in = NIN > 0 ? NIN : d.n_in;
  const int nrows = (int)(r1 - r0);
  const bool on = lane < g.Bv;
  const int64_t B = g.B;
  const int64_t lo = (int64_t)(on ? lane : 0) * VB;  // idle lanes read vector 0 and store nothing
  const bool leaf1 = !(d.chain_noleaf & 1);
  const int64_t lbase = d.in[n_in].off + lo;  // c_1's leaf factor (row 0 of the data if it has none)
  PK acc;
  for (int q = 0; q < nrows; ++q) {
    const uint32_t y = (uint32_t)(r0 + q);
    const PK L1 = ldv<Real, VB, false>(data, lbase + (int64_t)w->tab[n_in][q] * B);  // with the inputs
    PK p0, p1;
    if (NIN > 0) {
      PK a0[NIN > 0 ? NIN : 1], a1[NIN > 0 ? NIN : 1];
#pragma unroll
      for (int i = 0; i < NIN; ++i) {
        const int64_t e = d.in[i].off + lo + (int64_t)(2 * w->tab[i][q]) * B;
        const bool cached = LEAF && i == NIN - 1;  // the leaf factor, written before the launch
        a0[i] = cached ? ldv<Real, VB, false>(data, e) : ldv<Real, VB, true>(data, e);
        a1[i] = cached ? ldv<Real, VB, false>(data, e + B) : ldv<Real, VB, true>(data, e + B);
      }
      p0 = a0[0];
      p1 = a1[0];
#pragma unroll
      for (int i = 1; i < (NIN > 0 ? NIN : 1); ++i) {
        pmul<Real, VB>(p0, a0[i]);
        pmul<Real, VB>(p1, a1[i]);
      }
    } else {
#pragma unroll 1
      for (int i = 0; i < n_in; ++i) {
        const bool leaf = d.in[i].flags & kInLeaf;
        const int64_t e = d.in[i].off + lo + (int64_t)(2 * w->tab[i][q]) * B;
        const PK a0 = ldv_in<Real, VB, true>(data, e, leaf);
        const PK a1 = ldv_in<Real, VB, true>(data, e + B, leaf);
        if (i == 0) {
          p0 = a0;
          p1 = a1;
        } else {
          pmul<Real, VB>(p0, a0);
          pmul<Real, VB>(p1, a1);
        }
      }
    }
    PK t;
#pragma unroll
    for (int v = 0; v < VB; ++v) t.c[v] = cadd<Real>(p0.c[v], p1.c[v]);  // G_b[y]
    if (leaf1) pmul<Real, VB>(t, L1);
    if ((y & 1u) == 0) {  // c_1's term of w_1 = 0: keep it
      acc = t;
      continue;
    }
#pragma unroll
    for (int v = 0; v < VB; ++v) t.c[v] = cadd<Real>(acc.c[v], t.c[v]);  // c_1's row y >> 1
    int j = 1;
    for (; j < d.chain; ++j) {  // c_(j+1): its term of w = bit j of y
      if (!((d.chain_noleaf >> j) & 1))
        pmul<Real, VB>(t, ldv<Real, VB, false>(data, d.in[n_in + j].off + lo + (int64_t)w->tab[n_in + j][q] * B));
      if (((y >> j) & 1u) == 0) {
        w->x.chainh[j - 1][lane] = as_float4(t);
        break;
      }
      const PK h = from_float4<PK>(w->x.chainh[j - 1][lane]);
#pragma unroll
      for (int v = 0; v < VB; ++v) t.c[v] = cadd<Real>(h.c[v], t.c[v]);
    }
    if (j == d.chain && on) stv<Real, VB>(data, d.out_off + (int64_t)(y >> d.chain) * B + lo, t);
  }
}

template <class Real, int VB, int NIN, bool LEAF>
__device__ __forceinline__ void tile_rows_fixed(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                                int64_t r1, int lane) {
  using PK = Pack<Real, VB>;
  constexpr int U = kFixedRows;
  const DevBucket& d = w->d;
  const int nrows = (int)(r1 - r0);
  const bool on = lane < g.Bv;
  const int64_t B = g.B;
  const int64_t lo = (int64_t)(on ? lane : 0) * VB;  // idle lanes read vector 0 and store nothing
  int64_t base[NIN];
#pragma unroll
  for (int i = 0; i < NIN; ++i) base[i] = d.in[i].off + lo;
  const int64_t out = d.out_off + r0 * B + lo;
  for (int q = 0; q < nrows; q += U) {
    int qq[U];
#pragma unroll
    for (int u = 0; u < U; ++u) qq[u] = q + u < nrows ? q + u : q;
    PK p0[U], p1[U];
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t e = base[i] + (int64_t)(2 * w->tab[i][qq[u]]) * B;
        PK a0, a1;
        if (LEAF && i == NIN - 1) {  // the leaf factor, written before the launch: cached loads
          a0 = ldv<Real, VB, false>(data, e);
          a1 = ldv<Real, VB, false>(data, e + B);
        } else {
          a0 = ldv<Real, VB, true>(data, e);
          a1 = ldv<Real, VB, true>(data, e + B);
        }
        if (i == 0) {
          p0[u] = a0;
          p1[u] = a1;
        } else {
          pmul<Real, VB>(p0[u], a0);
          pmul<Real, VB>(p1[u], a1);
        }
      }
    }
    if (on) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u > 0 && qq[u] == q) break;
        PK o;
#pragma unroll
        for (int v = 0; v < VB; ++v) o.c[v] = cadd<Real>(p0[u].c[v], p1[u].c[v]);
        stv<Real, VB>(data, out + (int64_t)(q + u) * B, o);
      }
    }
  }
}

template <class Real, int VB>
__device__ __forceinline__ void tile_rows_rolled(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                                 int64_t r1, int lane) {
  using PK = Pack<Real, VB>;
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  const int nrows = (int)(r1 - r0);
  const bool on = lane < g.Bv;
  const int64_t B = g.B;
  const int64_t lo = (int64_t)(on ? lane : 0) * VB;  // idle lanes read vector 0 and store nothing
  for (int q = 0; q < nrows; q += 2) {
    const int qb = q + 1 < nrows ? q + 1 : q;
    PK p0[2], p1[2];
#pragma unroll 1  // rolled: no register spills at the 64-register budget, same speed
    for (int i = 0; i < n_in; ++i) {
      const bool leaf = d.in[i].flags & kInLeaf;
      const int64_t base = d.in[i].off + lo;
      const int64_t e0 = base + (int64_t)(2 * w->tab[i][q]) * B;
      const int64_t e1 = base + (int64_t)(2 * w->tab[i][qb]) * B;
      const PK a00 = ldv_in<Real, VB, true>(data, e0, leaf);
      const PK a01 = ldv_in<Real, VB, true>(data, e0 + B, leaf);
      const PK a10 = ldv_in<Real, VB, true>(data, e1, leaf);
      const PK a11 = ldv_in<Real, VB, true>(data, e1 + B, leaf);
      if (i == 0) {
        p0[0] = a00;
        p1[0] = a01;
        p0[1] = a10;
        p1[1] = a11;
      } else {
        pmul<Real, VB>(p0[0], a00);
        pmul<Real, VB>(p1[0], a01);
        pmul<Real, VB>(p0[1], a10);
        pmul<Real, VB>(p1[1], a11);
      }
    }
    if (on) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (u == 1 && qb == q) break;
        PK o;
#pragma unroll
        for (int v = 0; v < VB; ++v) o.c[v] = cadd<Real>(p0[u].c[v], p1[u].c[v]);
        stv<Real, VB>(data, d.out_off + (r0 + q + u) * B + lo, o);
      }
    }
  }
}

// Chained steps (STAGE 4 kernels only): complex64 buckets of fan-in 2 and 3,
// the planner's rule on the row-wide layout.  (A rolled variant for other
// fan-ins and for complex128 and float pairs raised the kernel's spills and
// cost every tile of the bench step 2.7 %, 14.21 -> 13.83 ms without it.)
template <class Real, int VB>
__device__ __forceinline__ void tile_rows_chained(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                                  int64_t r1, int lane, DevCtrl* ctrl) {
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  if (VB == 2 && n_in >= 2 && n_in <= kFixedMaxFanIn) {
    const bool leaf = d.in[n_in - 1].flags & kInLeaf;
    switch (n_in * 2 + (leaf ? 1 : 0)) {
      case 4: return tile_rows_chain<Real, VB, 2, false>(w, data, g, r0, r1, lane);
      case 5: return tile_rows_chain<Real, VB, 2, true>(w, data, g, r0, r1, lane);
      case 6: return tile_rows_chain<Real, VB, 3, false>(w, data, g, r0, r1, lane);
      case 7: return tile_rows_chain<Real, VB, 3, true>(w, data, g, r0, r1, lane);
      default: break;
    }
  }
  if (lane == 0 && ctrl != nullptr) atomicCAS(&ctrl->status, 0, (int32_t)QT_EINVAL);  // never planned
}

template <class Real, int VB>
__device__ __forceinline__ void tile_rows_regs(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                               int64_t r1, int lane) {
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  // (complex64 vectors only: with 16-byte complex numbers, complex128 and float pairs, the
  // unrolled tile spills at the 64-register budget)
  if (VB == 2 && n_in >= 2 && n_in <= kFixedMaxFanIn) {
    const bool leaf = d.in[n_in - 1].flags & kInLeaf;
    switch (n_in * 2 + (leaf ? 1 : 0)) {
      case 4: return tile_rows_fixed<Real, VB, 2, false>(w, data, g, r0, r1, lane);
      case 5: return tile_rows_fixed<Real, VB, 2, true>(w, data, g, r0, r1, lane);
      case 6: return tile_rows_fixed<Real, VB, 3, false>(w, data, g, r0, r1, lane);
      case 7: return tile_rows_fixed<Real, VB, 3, true>(w, data, g, r0, r1, lane);
      default: break;
    }
  }
  tile_rows_rolled<Real, VB>(w, data, g, r0, r1, lane);
}

// Row-wide forward tile with two vector chunks per row (RP = 1, VC = 2: 33 to
// 64 vectors of angle sets, lane l on vectors l and l + 32 of the same output
// row), one row per iteration: the same loads and products as tile_items,
// bit-identical to it, with the operand rows read straight from the pass
// table.  Used for float pairs at 33-64 angle sets (STAGE 3): 67.0 -> 57.9 ms
// on the 100-vertex p = 4 graph at 64 angle sets.  Complex128 keeps the generic
// tile there (this one made it slower, 129 -> 207 ms: its FP64 arithmetic sets
// the pace, and one row per iteration exposes it), and so does complex64.
template <class Real, int VB>
__device__ __forceinline__ void tile_rows_vc2(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                              int64_t r1, int lane) {
  using PK = Pack<Real, VB>;
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  const int nrows = (int)(r1 - r0);
  const bool on1 = lane + 32 < g.Bv;  // (lane < Bv always: Bv > 32)
  const int64_t B = g.B;
  const int64_t lo0 = (int64_t)lane * VB;
  const int64_t lo1 = (int64_t)(on1 ? lane + 32 : lane) * VB;  // idle chunk lanes reread chunk 0, store nothing
  for (int q = 0; q < nrows; ++q) {
    PK p0[2], p1[2];
#pragma unroll 1
    for (int i = 0; i < n_in; ++i) {
      const bool leaf = d.in[i].flags & kInLeaf;
      const int64_t e = d.in[i].off + (int64_t)(2 * w->tab[i][q]) * B;
      const PK a00 = ldv_in<Real, VB, true>(data, e + lo0, leaf);
      const PK a01 = ldv_in<Real, VB, true>(data, e + B + lo0, leaf);
      const PK a10 = ldv_in<Real, VB, true>(data, e + lo1, leaf);
      const PK a11 = ldv_in<Real, VB, true>(data, e + B + lo1, leaf);
      if (i == 0) {
        p0[0] = a00;
        p1[0] = a01;
        p0[1] = a10;
        p1[1] = a11;
      } else {
        pmul<Real, VB>(p0[0], a00);
        pmul<Real, VB>(p1[0], a01);
        pmul<Real, VB>(p0[1], a10);
        pmul<Real, VB>(p1[1], a11);
      }
    }
    const int64_t row = d.out_off + (r0 + q) * B;
    PK o;
#pragma unroll
    for (int v = 0; v < VB; ++v) o.c[v] = cadd<Real>(p0[0].c[v], p1[0].c[v]);
    stv<Real, VB>(data, row + lo0, o);
    if (on1) {
#pragma unroll
      for (int v = 0; v < VB; ++v) o.c[v] = cadd<Real>(p0[1].c[v], p1[1].c[v]);
      stv<Real, VB>(data, row + lo1, o);
    }
  }
}

// Forward tile of the one-angle-set layout on the register path (PAIR: B = 1,
// rows x = 0, 1 of an input adjacent; RP = 32 rows per pass, lane l on row
// r0 + pass * 32 + l).  The same loads and products as tile_items,
// PairPasses passes per iteration (each lane keeps that many rows' loads of an
// input in flight: 4 in complex64, 2 in complex128, where 4 would spill at
// the 64-register budget), without its per-item bookkeeping; bit-identical to
// it.  Rows past
// the step's end or the tile's passes read row 0 of each input (always inside
// the input) and store nothing.
template <class Real> struct PairPasses { static constexpr int value = sizeof(Real) == 4 ? 4 : 2; };
template <class Real> struct AdjPairPasses { static constexpr int value = 2; };

// Lane exchange of one complex number (all 32 lanes).
__device__ __forceinline__ float2 shfl_xor_cx(float2 v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}
__device__ __forceinline__ double2 shfl_xor_cx(double2 v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}
__device__ __forceinline__ ff2 shfl_xor_cx(ff2 v, int m) {
  v.x.hi = __shfl_xor_sync(0xffffffffu, v.x.hi, m);
  v.x.lo = __shfl_xor_sync(0xffffffffu, v.x.lo, m);
  v.y.hi = __shfl_xor_sync(0xffffffffu, v.y.hi, m);
  v.y.lo = __shfl_xor_sync(0xffffffffu, v.y.lo, m);
  return v;
}
__device__ __forceinline__ float2 shfl_down_cx(float2 v, int d) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, d);
  v.y = __shfl_down_sync(0xffffffffu, v.y, d);
  return v;
}
__device__ __forceinline__ double2 shfl_down_cx(double2 v, int d) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, d);
  v.y = __shfl_down_sync(0xffffffffu, v.y, d);
  return v;
}
__device__ __forceinline__ ff2 shfl_down_cx(ff2 v, int d) {
  v.x.hi = __shfl_down_sync(0xffffffffu, v.x.hi, d);
  v.x.lo = __shfl_down_sync(0xffffffffu, v.x.lo, d);
  v.y.hi = __shfl_down_sync(0xffffffffu, v.y.hi, d);
  v.y.lo = __shfl_down_sync(0xffffffffu, v.y.lo, d);
  return v;
}

// Chained step on the one-angle-set layout: lane l holds b's row y = r0 +
// pass * 32 + l, so chain level j pairs lanes l and l ^ 2^(j-1) (bit j - 1 of
// y is c_j's eliminated variable): each lane multiplies its row by its leaf
// element L_j[pext(y, chain mask)] (loaded at the start of the iteration, with
// the inputs), and the lane with that bit 0 adds its partner's product to its
// own (w = 0 first, the consumer's order).  After m levels the lanes whose
// low m bits are 0 hold c_m's rows y >> m.  A group of 2^m rows is either
// inside the step or wholly past its end (n_rows is a power of two >= 2^m),
// so idle lanes only meet idle lanes.
template <class Real, int CM>
__device__ __forceinline__ void chain_pair_leaves(const WarpTile* w, const Real* __restrict__ data, int pp, int lane,
                                                  typename Cx<Real>::T (&L)[CM]) {
  const DevBucket& d = w->d;
#pragma unroll
  for (int j = 0; j < CM; ++j)
    if (!((d.chain_noleaf >> j) & 1)) {
      const uint32_t t = w->tab[d.n_in + j][pp] + w->lpart[d.n_in + j][lane];
      L[j] = ldv<Real, 1, false>(data, d.in[d.n_in + j].off + (int64_t)t).c[0];
    }
}

template <class Real, int CM>
__device__ __forceinline__ void chain_pair_rows(const WarpTile* w, Real* __restrict__ data, int64_t y, bool ok,
                                                int lane, typename Cx<Real>::T o, const typename Cx<Real>::T (&L)[CM]) {
  const DevBucket& d = w->d;
#pragma unroll
  for (int j = 0; j < CM; ++j) {
    if (!((d.chain_noleaf >> j) & 1)) o = cmul<Real>(o, L[j]);
    o = cadd<Real>(o, shfl_xor_cx(o, 1 << j));
  }
  if (ok && (lane & ((1 << CM) - 1)) == 0) {
    Pack<Real, 1> v;
    v.c[0] = o;
    stv<Real, 1>(data, d.out_off + (y >> CM), v);
  }
}

template <class Real, int CM>
__device__ __forceinline__ void tile_pairs_loop(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                                int64_t r1, int lane) {
  using P1 = Pack<Real, 1>;
  constexpr int U = PairPasses<Real>::value;
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  for (int pp = 0; pp < g.P && r0 + (int64_t)pp * 32 < r1; pp += U) {
    int64_t y[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      y[u] = r0 + (int64_t)(pp + u) * 32 + lane;
      ok[u] = pp + u < g.P && y[u] < r1;
    }
    typename Cx<Real>::T L[CM > 0 ? U : 1][CM > 0 ? CM : 1];
    if constexpr (CM > 0) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (pp + u < g.P) chain_pair_leaves<Real, CM>(w, data, pp + u, lane, L[u]);
    }
    P1 p0[U], p1[U];
#pragma unroll 1
    for (int i = 0; i < n_in; ++i) {
      const bool leaf = d.in[i].flags & kInLeaf;
      const uint32_t lp = w->lpart[i][lane];
      Pack<Real, 2> q[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t k = ok[u] ? w->tab[i][pp + u] + lp : 0u;  // idle items read row 0 and store nothing
        q[u] = ldpair_in<Real, true>(data, d.in[i].off + 2 * (int64_t)k, leaf);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        P1 a0, a1;
        a0.c[0] = q[u].c[0];
        a1.c[0] = q[u].c[1];
        if (i == 0) {
          p0[u] = a0;
          p1[u] = a1;
        } else {
          pmul<Real, 1>(p0[u], a0);
          pmul<Real, 1>(p1[u], a1);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if constexpr (CM > 0) {
        if (pp + u >= g.P || r0 + (int64_t)(pp + u) * 32 >= r1) break;  // warp-uniform: past the tile
        chain_pair_rows<Real, CM>(w, data, y[u], ok[u], lane, cadd<Real>(p0[u].c[0], p1[u].c[0]), L[u]);
        continue;
      }
      if (!ok[u]) continue;
      P1 o;
      o.c[0] = cadd<Real>(p0[u].c[0], p1[u].c[0]);
      stv<Real, 1>(data, d.out_off + y[u], o);
    }
  }
}

template <class Real>
__device__ __forceinline__ void tile_pairs_regs(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                                int64_t r1, int lane) {
  tile_pairs_loop<Real, 0>(w, data, g, r0, r1, lane);
}

template <class Real>
__device__ __forceinline__ void atomic_add_cx(Real* data, int64_t e, typename Cx<Real>::T v) {
  atomicAdd(data + 2 * e, v.x);
  atomicAdd(data + 2 * e + 1, v.y);
}

// Float pairs have no hardware atomic add: a compare-and-swap loop on the
// pair's 8 bytes (hi in the low word) adds with the float-pair sum.  The first
// swap expects 0 (targets are cleared before their first add, so a first add
// needs one atomic); every failed swap returns the current value and means
// another lane's add went in, so the loop ends after at most as many retries
// as there are adds to the element in flight.  The retry limit only guards
// that argument: past it the element is set to NaN, so that an add left out
// cannot pass unseen.  Float-pair gradient plans keep their adjoint tensors
// in FP64 (kInF64, below: under contention this loop serialises), so the
// tiles they run never take this path; it completes the float-pair
// instantiation of the generic tiles.
constexpr int kFfCasLimit = 1 << 20;
__device__ __forceinline__ void atomic_add_ff(ff* a, ff v) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(a);
  unsigned long long old = 0ull;
  for (int it = 0; it < kFfCasLimit; ++it) {
    ff cur;
    cur.hi = __uint_as_float((unsigned)old);
    cur.lo = __uint_as_float((unsigned)(old >> 32));
    const ff nv = cur + v;
    const unsigned long long nb =
        (unsigned long long)__float_as_uint(nv.hi) | ((unsigned long long)__float_as_uint(nv.lo) << 32);
    const unsigned long long seen = atomicCAS(p, old, nb);
    if (seen == old) return;
    old = seen;
  }
  atomicExch(p, 0x7fc000007fc00000ull);
}
template <>
__device__ __forceinline__ void atomic_add_cx<ff>(ff* data, int64_t e, ff2 v) {
  atomic_add_ff(data + 2 * e, v.x);
  atomic_add_ff(data + 2 * e + 1, v.y);
}

// Adjoint targets of float-pair plans (target record flag kInF64): every
// adjoint tensor is kept in FP64.  Many tiles add into the same target
// elements (all of a leaf factor's few elements, or a reduction target's
// completions), and a float pair can only be added by the compare-and-swap
// loop above, which serialises under that contention, while FP64 has a
// native atomic add and at least the float pair's precision.  The element
// slots are 16 bytes either way.
template <class Real>
__device__ __forceinline__ bool f64_target(const DevBucket& d) {
  if constexpr (std::is_same<Real, ff>::value) return (d.in[d.n_in].flags & kInF64) != 0;
  else return false;
}
template <class Real>
__device__ __forceinline__ void put_f64_pair(Real* data, int64_t e0, typename Cx<Real>::T c0,
                                             typename Cx<Real>::T c1, bool full) {
  if constexpr (std::is_same<Real, ff>::value) {
    double* q = reinterpret_cast<double*>(data) + 2 * e0;
    const double v0 = (double)c0.x, v1 = (double)c0.y, v2 = (double)c1.x, v3 = (double)c1.y;
    if (full) {
      q[0] = v0;
      q[1] = v1;
      q[2] = v2;
      q[3] = v3;
    } else {
      atomicAdd(q, v0);
      atomicAdd(q + 1, v1);
      atomicAdd(q + 2, v2);
      atomicAdd(q + 3, v3);
    }
  }
}

template <class Real>
__device__ __forceinline__ void put_f64_cx(Real* data, int64_t e, typename Cx<Real>::T c, bool full) {
  if constexpr (std::is_same<Real, ff>::value) {
    double* q = reinterpret_cast<double*>(data) + 2 * e;
    const double v0 = (double)c.x, v1 = (double)c.y;
    if (full) {
      q[0] = v0;
      q[1] = v1;
    } else {
      atomicAdd(q, v0);
      atomicAdd(q + 1, v1);
    }
  }
}

// Atomic add of two adjacent complex numbers (elements e0, e0 + 1).  In
// complex64 at an even e0 (the pair's 16 bytes aligned: every tensor starts
// 256-byte aligned and a pair row at an even element) this is one 16-byte
// vector atomic instead of four scalar ones.
template <class Real>
__device__ __forceinline__ void atomic_add_pair(Real* data, int64_t e0, typename Cx<Real>::T c0,
                                                typename Cx<Real>::T c1) {
  atomic_add_cx<Real>(data, e0, c0);
  atomic_add_cx<Real>(data, e0 + 1, c1);
}
template <>
__device__ __forceinline__ void atomic_add_pair<float>(float* data, int64_t e0, float2 c0, float2 c1) {
  if ((e0 & 1) == 0) {
    atomicAdd(reinterpret_cast<float4*>(data + 2 * e0), make_float4(c0.x, c0.y, c1.x, c1.y));
  } else {
    atomic_add_cx<float>(data, e0, c0);
    atomic_add_cx<float>(data, e0 + 1, c1);
  }
}

// Adjoint step (kStepAdj) on the lean paths: the same factors, products,
// target rows and stores or atomic adds as tile_adjoint, several rows per
// iteration, addressed straight from the pass table.  Factors flagged
// kInNoPair (the output adjoint) give one value for x = 0 and x = 1.
// One angle set (PAIR, 32 rows per pass, lane l on row r0 + pass * 32 + l,
// AdjPairPasses passes per iteration):
template <class Real>
__device__ __forceinline__ void tile_adjoint_pairs(WarpTile* w, Real* __restrict__ data, const TileGeom& g,
                                                   int64_t r0, int64_t r1, int lane) {
  using P1 = Pack<Real, 1>;
  constexpr int U = AdjPairPasses<Real>::value;
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  const bool full = d.aflags & kAdjFull;
  const uint32_t lp_t = w->lpart[n_in][lane];
  for (int pp = 0; pp < g.P && r0 + (int64_t)pp * 32 < r1; pp += U) {
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ok[u] = pp + u < g.P && r0 + (int64_t)(pp + u) * 32 + lane < r1;
    P1 p0[U], p1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      p0[u].c[0].x = 1;
      p0[u].c[0].y = 0;
      p1[u] = p0[u];
    }
#pragma unroll 1
    for (int i = 0; i < n_in; ++i) {
      const int32_t fl = d.in[i].flags;
      const bool leaf = fl & kInLeaf;
      const uint32_t lp = w->lpart[i][lane];
      P1 a0[U], a1[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t k = ok[u] ? w->tab[i][pp + u] + lp : 0u;  // idle items read row 0
        if (fl & kInNoPair) {
          a0[u] = ld_nopair<Real>(data, d.in[i].off + (int64_t)k, fl);
          a1[u] = a0[u];
        } else {
          const Pack<Real, 2> q = ldpair_in<Real, true>(data, d.in[i].off + 2 * (int64_t)k, leaf);
          a0[u].c[0] = q.c[0];
          a1[u].c[0] = q.c[1];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        pmul<Real, 1>(p0[u], a0[u]);
        pmul<Real, 1>(p1[u], a1[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      const int64_t e0 = d.out_off + 2 * (int64_t)(w->tab[n_in][pp + u] + lp_t);
      if (f64_target<Real>(d)) {
        put_f64_pair<Real>(data, e0, p0[u].c[0], p1[u].c[0], full);
      } else if (full) {
        stv<Real, 1>(data, e0, p0[u]);
        stv<Real, 1>(data, e0 + 1, p1[u]);
      } else {
        atomic_add_pair<Real>(data, e0, p0[u].c[0], p1[u].c[0]);
      }
    }
  }
}

// Row-wide tiles (RP = 1, VC = 1: every lane on the same output row):
template <class Real, int VB>
__device__ __forceinline__ void tile_adjoint_rows(WarpTile* w, Real* __restrict__ data, const TileGeom& g,
                                                  int64_t r0, int64_t r1, int lane) {
  using PK = Pack<Real, VB>;
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  const int nrows = (int)(r1 - r0);
  const bool full = d.aflags & kAdjFull;
  const bool on = lane < g.Bv;
  const int64_t B = g.B;
  const int64_t lo = (int64_t)(on ? lane : 0) * VB;
  for (int q = 0; q < nrows; q += 2) {
    const int qq[2] = {q, q + 1 < nrows ? q + 1 : q};
    PK p0[2], p1[2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < VB; ++v) {
        p0[u].c[v].x = 1;
        p0[u].c[v].y = 0;
        p1[u].c[v] = p0[u].c[v];
      }
#pragma unroll 1
    for (int i = 0; i < n_in; ++i) {
      const int32_t fl = d.in[i].flags;
      const bool leaf = fl & kInLeaf;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const uint32_t k = w->tab[i][qq[u]];
        PK a0, a1;
        if (fl & kInNoPair) {
          a0 = ldv_in<Real, VB, true>(data, d.in[i].off + (int64_t)k * B + lo, leaf);
          a1 = a0;
        } else {
          const int64_t e = d.in[i].off + (int64_t)(2 * k) * B + lo;
          a0 = ldv_in<Real, VB, true>(data, e, leaf);
          a1 = ldv_in<Real, VB, true>(data, e + B, leaf);
        }
        pmul<Real, VB>(p0[u], a0);
        pmul<Real, VB>(p1[u], a1);
      }
    }
    if (!on) continue;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && qq[1] == q) break;
      const int64_t e0 = d.out_off + (int64_t)(2 * w->tab[n_in][qq[u]]) * B + lo;
      if (full) {
        stv<Real, VB>(data, e0, p0[u]);
        stv<Real, VB>(data, e0 + B, p1[u]);
      } else if (VB == 2) {  // a lane's two angle sets are adjacent elements
        atomic_add_pair<Real>(data, e0, p0[u].c[0], p0[u].c[VB - 1]);
        atomic_add_pair<Real>(data, e0 + B, p1[u].c[0], p1[u].c[VB - 1]);
      } else {
#pragma unroll
        for (int v = 0; v < VB; ++v) {
          atomic_add_cx<Real>(data, e0 + v, p0[u].c[v]);
          atomic_add_cx<Real>(data, e0 + B + v, p1[u].c[v]);
        }
      }
    }
  }
}

// Adjoint step (kStepAdj): for each item (row y, vector), the product of the
// factors at x = 0 and x = 1 goes to the target rows (k_t << 1) | x,
// k_t = pext(y, mask_t).
template <class Real, int VB, bool PAIR, bool CG, int U>
__device__ __forceinline__ void tile_adjoint(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                             int64_t r1, int lane, int rip, int v0, bool lane_on, DevCtrl* ctrl,
                                             int dbg_bucket) {
  using C = typename Cx<Real>::T;
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  const int Q = g.P * g.VC;
  const int B = g.B;
  const bool full = d.aflags & kAdjFull;
  const uint32_t lp_t = w->lpart[n_in][lane];
  for (int q0 = 0; q0 < Q; q0 += U) {
    const ItemSet<U> it = make_items<U>(g, q0, Q, r0, r1, rip, v0, lane_on);
    Pack<Real, VB> p0[U], p1[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < VB; ++v) {
        p0[u].c[v].x = 1;
        p0[u].c[v].y = 0;
        p1[u].c[v] = p0[u].c[v];
      }
    for (int i = 0; i < n_in; ++i) {
      Pack<Real, VB> a0[U], a1[U];
      load_input<Real, VB, PAIR, CG, U>(w, i, w->lpart[i][lane], it, data, g, a0, a1, ctrl, dbg_bucket);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        pmul<Real, VB>(p0[u], a0[u]);
        pmul<Real, VB>(p1[u], a1[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!it.ok[u]) continue;
      const uint32_t kt = w->tab[n_in][it.pp[u]] + lp_t;
      const int64_t e0 = PAIR ? d.out_off + 2 * (int64_t)kt
                              : d.out_off + (int64_t)(2 * kt) * B + (int64_t)(it.vv[u] * VB);
      const int64_t e1 = PAIR ? e0 + 1 : e0 + B;
      if (!QT_RANGE_OK(e0, 1, 2, -1) || !QT_RANGE_OK(e1, VB, 2, -1)) continue;
      if (full) {
        stv<Real, VB>(data, e0, p0[u]);
        stv<Real, VB>(data, e1, p1[u]);
      } else {
#pragma unroll
        for (int v = 0; v < VB; ++v) {
          atomic_add_cx<Real>(data, e0 + v, p0[u].c[v]);
          atomic_add_cx<Real>(data, e1 + v, p1[u].c[v]);
        }
      }
    }
  }
}

// Zero step (kStepZero): clear rows [r0, r1) x B of the region at out_off.
template <class Real, int VB, bool PAIR, int U>
__device__ __forceinline__ void tile_zero(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                          int64_t r1, int rip, int v0, bool lane_on) {
  const DevBucket& d = w->d;
  const int Q = g.P * g.VC;
  Pack<Real, VB> z{};
  for (int q0 = 0; q0 < Q; q0 += U) {
    const ItemSet<U> it = make_items<U>(g, q0, Q, r0, r1, rip, v0, lane_on);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!it.ok[u]) continue;
      const int64_t e = PAIR ? d.out_off + (int64_t)it.y[u] : d.out_off + (int64_t)it.y[u] * g.B + (int64_t)(it.vv[u] * VB);
      stv<Real, VB>(data, e, z);
    }
  }
}

template <class Real> struct RedBuf;
template <> struct RedBuf<float> {
  static __device__ __forceinline__ float* get(WarpTile* w) { return &w->x.red.f[0][0]; }
};
template <> struct RedBuf<double> {
  static __device__ __forceinline__ double* get(WarpTile* w) { return &w->x.red.d[0][0]; }
};
template <> struct RedBuf<ff> {  // (8-byte elements, the complex128 slots)
  static __device__ __forceinline__ ff* get(WarpTile* w) { return reinterpret_cast<ff*>(&w->x.red.d[0][0]); }
};

// Reduction adjoint step (kStepAdjRed).  The tile's rows q = kt * 2^comp_bits
// + c run over target rows kt and their completions c; since 2^comp_bits >=
// 32 >= RP, all lanes of a pass share kt, which changes every
// 2^comp_bits / RP passes.  Lanes sum Gbar[y] * prod_{factors} at x = 0, 1
// while kt stays fixed; at each change the lanes of each vector of angle sets
// are added (shuffle butterfly when Bv is a power of two, else through shared
// memory) and one atomic add per target element goes to rows (kt << 1) | x.
template <class Real, int VB, bool PAIR>
__device__ __forceinline__ void flush_target(WarpTile* w, Real* __restrict__ data, const TileGeom& g, uint32_t kt,
                                             Pack<Real, VB>& s0, Pack<Real, VB>& s1, int lane, int rip, int v0,
                                             bool lane_on, DevCtrl* ctrl, int dbg_bucket) {
  (void)ctrl;
  (void)dbg_bucket;
  const DevBucket& d = w->d;
  const int B = g.B;
  if ((g.Bv & (g.Bv - 1)) == 0) {  // RP * Bv = 32: butterfly over the lane bits >= Bv
#pragma unroll
    for (int v = 0; v < VB; ++v) {
      for (int off = 16; off >= g.Bv; off >>= 1) {
        s0.c[v] = cadd<Real>(s0.c[v], shfl_xor_cx(s0.c[v], off));
        s1.c[v] = cadd<Real>(s1.c[v], shfl_xor_cx(s1.c[v], off));
      }
    }
  } else {
    Real* red = RedBuf<Real>::get(w);
    const int per = 4 / (int)(sizeof(Real) / 4);
#pragma unroll
    for (int v = 0; v < VB; ++v) {
      for (int x = 0; x < 2; ++x) {
        typename Cx<Real>::T& sv = x == 0 ? s0.c[v] : s1.c[v];
        __syncwarp();
        red[lane * per + 0] = sv.x;
        red[lane * per + 1] = sv.y;
        __syncwarp();
        if (lane_on && rip == 0) {
          typename Cx<Real>::T t;
          t.x = 0;
          t.y = 0;
          for (int r = 0; r < g.RP; ++r) {
            t.x = t.x + red[(r * g.Bv + v0) * per + 0];
            t.y = t.y + red[(r * g.Bv + v0) * per + 1];
          }
          sv = t;
        }
      }
    }
    __syncwarp();
  }
  if (lane_on && rip == 0) {
#pragma unroll
    for (int v = 0; v < VB; ++v) {
      const int64_t e0 = PAIR ? d.out_off + 2 * (int64_t)kt
                              : d.out_off + (int64_t)(2 * kt) * B + (int64_t)(v0 * VB + v);
      const int64_t e1 = PAIR ? e0 + 1 : e0 + B;
      if (QT_RANGE_OK(e0, 1, 2, -1)) atomic_add_cx<Real>(data, e0, s0.c[v]);
      if (QT_RANGE_OK(e1, 1, 2, -1)) atomic_add_cx<Real>(data, e1, s1.c[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < VB; ++v) {
    s0.c[v].x = 0;
    s0.c[v].y = 0;
    s1.c[v] = s0.c[v];
  }
}

template <class Real, int VB, bool PAIR, bool CG, int U>
__device__ __forceinline__ void tile_adjred(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                            int64_t r1, int lane, int rip, int v0, bool lane_on, DevCtrl* ctrl,
                                            int dbg_bucket) {
  const DevBucket& d = w->d;
  if (d.aflags & kAdjRedLow) {  // the one-angle-set lane form: the pair tiles evaluate it, never this one
    if (lane == 0 && ctrl != nullptr) atomicCAS(&ctrl->status, 0, (int32_t)QT_EINVAL);
    return;
  }
  const int n_in = d.n_in;
  const int Q = g.P * g.VC;  // VC == 1 here (Bv <= 32)
  const int seg = (1 << d.comp_bits) / g.RP < Q ? (1 << d.comp_bits) / g.RP : Q;  // passes per target row
  Pack<Real, VB> s0, s1;
#pragma unroll
  for (int v = 0; v < VB; ++v) {
    s0.c[v].x = 0;
    s0.c[v].y = 0;
    s1.c[v] = s0.c[v];
  }
  for (int q0 = 0; q0 < Q; q0 += U) {
    const ItemSet<U> it = make_items<U>(g, q0, Q, r0, r1, rip, v0, lane_on);
    Pack<Real, VB> p0[U], p1[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < VB; ++v) {
        p0[u].c[v].x = 1;
        p0[u].c[v].y = 0;
        p1[u].c[v] = p0[u].c[v];
      }
    for (int i = 0; i < n_in; ++i) {
      Pack<Real, VB> a0[U], a1[U];
      load_input<Real, VB, PAIR, CG, U>(w, i, w->lpart[i][lane], it, data, g, a0, a1, ctrl, dbg_bucket);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        pmul<Real, VB>(p0[u], a0[u]);
        pmul<Real, VB>(p1[u], a1[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + u;
      if (q < Q) {
        if (it.ok[u]) {
#pragma unroll
          for (int v = 0; v < VB; ++v) {
            s0.c[v] = cadd<Real>(s0.c[v], p0[u].c[v]);
            s1.c[v] = cadd<Real>(s1.c[v], p1[u].c[v]);
          }
        }
        if ((q + 1) % seg == 0 || q + 1 == Q) {  // end of a target row's passes (warp-uniform)
          const uint32_t kt = (uint32_t)((r0 + (int64_t)q * g.RP) >> d.comp_bits);
          flush_target<Real, VB, PAIR>(w, data, g, kt, s0, s1, lane, rip, v0, lane_on, ctrl, dbg_bucket);
        }
      }
    }
  }
}

// End of a target group of a one-angle-set reduction step (pass q of the tile
// at r0 is its last): the lanes' sums s0, s1 (x = 0, 1) are summed over the
// lanes that share a target and added to the target's adjoint, and reset.
// Lanes on completions (the default form): one target per group, lane 0 adds.
// kAdjRedLow: lanes on the bucket's five lowest variables; a butterfly over
// the lane bits that are completion bits, then every lane whose completion
// bits are 0 adds its own target element (target row from the pass table).
template <class Real>
__device__ __forceinline__ void adjred_pairs_flush(const WarpTile* w, Real* __restrict__ data, int64_t r0, int q,
                                                   int lane, Pack<Real, 1>& s0, Pack<Real, 1>& s1) {
  const DevBucket& d = w->d;
  if (d.aflags & kAdjRedLow) {
    const uint32_t cl = ~d.in[d.n_in].mask & 31u;  // completion bits among the lane bits (warp-uniform)
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      if (!((cl >> b) & 1u)) continue;
      s0.c[0] = cadd<Real>(s0.c[0], shfl_xor_cx(s0.c[0], 1 << b));
      s1.c[0] = cadd<Real>(s1.c[0], shfl_xor_cx(s1.c[0], 1 << b));
    }
    if (((uint32_t)lane & cl) == 0u) {
      const int64_t e0 = d.out_off + 2 * (int64_t)(w->tab[d.n_in][q] + w->lpart[d.n_in][lane]);
      if (f64_target<Real>(d))
        put_f64_pair<Real>(data, e0, s0.c[0], s1.c[0], false);
      else
        atomic_add_pair<Real>(data, e0, s0.c[0], s1.c[0]);
    }
  } else {
    const uint32_t kt = (uint32_t)((r0 + (int64_t)q * 32) >> d.comp_bits);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      s0.c[0] = cadd<Real>(s0.c[0], shfl_xor_cx(s0.c[0], off));
      s1.c[0] = cadd<Real>(s1.c[0], shfl_xor_cx(s1.c[0], off));
    }
    if (lane == 0) {
      if (f64_target<Real>(d))
        put_f64_pair<Real>(data, d.out_off + 2 * (int64_t)kt, s0.c[0], s1.c[0], false);
      else
        atomic_add_pair<Real>(data, d.out_off + 2 * (int64_t)kt, s0.c[0], s1.c[0]);
    }
  }
  s0.c[0].x = 0;
  s0.c[0].y = 0;
  s1 = s0;
}

// Reduction adjoint step (kStepAdjRed) of the one-angle-set layout (PAIR,
// RP = 32: lane l on completion c = l of pass pp, all lanes of a pass on the
// same target row kt, which changes every 2^comp_bits / 32 passes).  The same
// loads, products, sums and atomic adds as tile_adjred, AdjRedPasses passes
// per iteration (that many rows' loads of every factor in flight per lane),
// without the generic tile's per-item bookkeeping.  The pass table and lane
// parts are those warp_tile builds for the reduction order.
template <class Real> struct AdjRedPasses { static constexpr int value = sizeof(Real) == 4 ? 4 : 2; };

template <class Real>
__device__ __forceinline__ void tile_adjred_pairs(WarpTile* w, Real* __restrict__ data, const TileGeom& g,
                                                  int64_t r0, int64_t r1, int lane) {
  using P1 = Pack<Real, 1>;
  constexpr int U = AdjRedPasses<Real>::value;
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  const int seg = (d.aflags & kAdjRedLow) ? 1 << d.comp_bits : (1 << d.comp_bits) / 32;  // passes per target group
  P1 s0, s1;
  s0.c[0].x = 0;
  s0.c[0].y = 0;
  s1 = s0;
  for (int pp = 0; pp < g.P && r0 + (int64_t)pp * 32 < r1; pp += U) {
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ok[u] = pp + u < g.P && r0 + (int64_t)(pp + u) * 32 + lane < r1;
    P1 p0[U], p1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      p0[u].c[0].x = 1;
      p0[u].c[0].y = 0;
      p1[u] = p0[u];
    }
#pragma unroll 1
    for (int i = 0; i < n_in; ++i) {
      const int32_t fl = d.in[i].flags;
      const bool leaf = fl & kInLeaf;
      const uint32_t lp = w->lpart[i][lane];
      P1 a0[U], a1[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t k = ok[u] ? w->tab[i][pp + u] + lp : 0u;  // idle items read row 0
        if (fl & kInNoPair) {
          a0[u] = ld_nopair<Real>(data, d.in[i].off + (int64_t)k, fl);
          a1[u] = a0[u];
        } else {
          const Pack<Real, 2> q = ldpair_in<Real, true>(data, d.in[i].off + 2 * (int64_t)k, leaf);
          a0[u].c[0] = q.c[0];
          a1[u].c[0] = q.c[1];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        pmul<Real, 1>(p0[u], a0[u]);
        pmul<Real, 1>(p1[u], a1[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = pp + u;
      if (q >= g.P || r0 + (int64_t)q * 32 >= r1) break;  // warp-uniform: the tile's last pass is done
      if (ok[u]) {
        s0.c[0] = cadd<Real>(s0.c[0], p0[u].c[0]);
        s1.c[0] = cadd<Real>(s1.c[0], p1[u].c[0]);
      }
      if ((q + 1) % seg == 0 || q + 1 == g.P || r0 + (int64_t)(q + 1) * 32 >= r1)  // end of a target group's passes
        adjred_pairs_flush<Real>(w, data, r0, q, lane, s0, s1);
    }
  }
}

// Adjoint steps of the one-angle-set layout with the factor count NF fixed at
// compile time (2 to 4 factors: the output adjoint, then the bucket's other
// inputs, each a pair of rows x = 0, 1).  The same loads, products and stores or atomic adds as
// tile_adjoint_pairs and tile_adjred_pairs, but every factor's loads of U
// passes are issued before the first product: U * NF loads in flight per lane
// and one memory round trip per U passes, where the rolled factor loop makes
// NF round trips.  AdjNfPasses keeps the loaded values within the 64-register
// budget.
template <class Real, int NF> struct AdjNfPasses {
  static constexpr int value = sizeof(Real) == 4 ? 2 : (NF <= 2 ? 2 : 1);
};

template <class Real, int NF, int U>
__device__ __forceinline__ void load_factors_nf(const WarpTile* w, const Real* __restrict__ data, int pp,
                                                const bool (&ok)[U], const uint32_t (&lp)[NF],
                                                Pack<Real, 1> (&p0)[U], Pack<Real, 1> (&p1)[U]) {
  const DevBucket& d = w->d;
  Pack<Real, 1> g0[U];  // factor 0, the output adjoint: one value for x = 0 and x = 1
  Pack<Real, 2> q[NF - 1][U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const uint32_t k = ok[u] ? w->tab[0][pp + u] + lp[0] : 0u;  // idle items read row 0
    g0[u] = ld_nopair<Real>(data, d.in[0].off + (int64_t)k, d.in[0].flags);
  }
#pragma unroll
  for (int i = 1; i < NF; ++i) {
    const bool leaf = d.in[i].flags & kInLeaf;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t k = ok[u] ? w->tab[i][pp + u] + lp[i] : 0u;
      q[i - 1][u] = ldpair_in<Real, true>(data, d.in[i].off + 2 * (int64_t)k, leaf);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    p0[u] = g0[u];
    p1[u] = g0[u];
#pragma unroll
    for (int i = 1; i < NF; ++i) {
      Pack<Real, 1> a0, a1;
      a0.c[0] = q[i - 1][u].c[0];
      a1.c[0] = q[i - 1][u].c[1];
      pmul<Real, 1>(p0[u], a0);
      pmul<Real, 1>(p1[u], a1);
    }
  }
}

// Whether the adjoint step in w->d has the factor form of the NF tiles: the
// output adjoint first (one value per output row), every other factor a pair.
__device__ __forceinline__ bool adj_nf_form(const DevBucket& d) {
  if (d.n_in < 2 || d.n_in > 4 || !(d.in[0].flags & kInNoPair)) return false;
  for (int i = 1; i < d.n_in; ++i)
    if (d.in[i].flags & kInNoPair) return false;
  return true;
}

template <class Real, int NF>
__device__ __forceinline__ void tile_adjoint_pairs_nf(WarpTile* w, Real* __restrict__ data, const TileGeom& g,
                                                      int64_t r0, int64_t r1, int lane) {
  using P1 = Pack<Real, 1>;
  constexpr int U = AdjNfPasses<Real, NF>::value;
  const DevBucket& d = w->d;
  const bool full = d.aflags & kAdjFull;
  const uint32_t lp_t = w->lpart[NF][lane];
  uint32_t lp[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) lp[i] = w->lpart[i][lane];
  for (int pp = 0; pp < g.P && r0 + (int64_t)pp * 32 < r1; pp += U) {
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ok[u] = pp + u < g.P && r0 + (int64_t)(pp + u) * 32 + lane < r1;
    P1 p0[U], p1[U];
    load_factors_nf<Real, NF, U>(w, data, pp, ok, lp, p0, p1);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      const int64_t e0 = d.out_off + 2 * (int64_t)(w->tab[NF][pp + u] + lp_t);
      if (f64_target<Real>(d)) {
        put_f64_pair<Real>(data, e0, p0[u].c[0], p1[u].c[0], full);
      } else if (full) {
        stv<Real, 1>(data, e0, p0[u]);
        stv<Real, 1>(data, e0 + 1, p1[u]);
      } else {
        atomic_add_pair<Real>(data, e0, p0[u].c[0], p1[u].c[0]);
      }
    }
  }
}

template <class Real, int NF>
__device__ __forceinline__ void tile_adjred_pairs_nf(WarpTile* w, Real* __restrict__ data, const TileGeom& g,
                                                     int64_t r0, int64_t r1, int lane) {
  using P1 = Pack<Real, 1>;
  constexpr int U = AdjNfPasses<Real, NF>::value;
  const DevBucket& d = w->d;
  const int seg = (d.aflags & kAdjRedLow) ? 1 << d.comp_bits : (1 << d.comp_bits) / 32;  // passes per target group
  uint32_t lp[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) lp[i] = w->lpart[i][lane];
  P1 s0, s1;
  s0.c[0].x = 0;
  s0.c[0].y = 0;
  s1 = s0;
  for (int pp = 0; pp < g.P && r0 + (int64_t)pp * 32 < r1; pp += U) {
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ok[u] = pp + u < g.P && r0 + (int64_t)(pp + u) * 32 + lane < r1;
    P1 p0[U], p1[U];
    load_factors_nf<Real, NF, U>(w, data, pp, ok, lp, p0, p1);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = pp + u;
      if (q >= g.P || r0 + (int64_t)q * 32 >= r1) break;  // warp-uniform: the tile's last pass is done
      if (ok[u]) {
        s0.c[0] = cadd<Real>(s0.c[0], p0[u].c[0]);
        s1.c[0] = cadd<Real>(s1.c[0], p1[u].c[0]);
      }
      if ((q + 1) % seg == 0 || q + 1 == g.P || r0 + (int64_t)(q + 1) * 32 >= r1)  // end of a target group's passes
        adjred_pairs_flush<Real>(w, data, r0, q, lane, s0, s1);
    }
  }
}

// Multi-row lean tiles (STAGE 5: 2 to 32 rows per warp pass, one vector chunk
// per row; complex64 with 2 to 32 angle sets, complex128 and float pairs with
// 2 to 16).  Lane l works on row rip = l / Bv of each pass and vector v0 =
// l % Bv; lanes with rip >= RP are idle (they read row 0 and store nothing).
// The same loads, products and stores or atomic adds as the generic tiles
// (tile_items, tile_adjoint, tile_adjred), addressed straight from the pass
// table and the lane parts, MrowPasses passes per iteration, without the
// generic tiles' per-item bookkeeping: forward steps bit-identical to them.
// Measured against the generic tile: 100-vertex p = 4 energy at 4 / 16 / 32
// angle sets 3.22 / 7.65 / 12.35 -> 1.98 / 5.53 / 10.19 ms; 60-vertex p = 4
// energy + gradient at 16 angle sets 114.9 -> 89.8 ms.
template <class Real> struct MrowPasses { static constexpr int value = 2; };

template <class Real, int VB>
__device__ __forceinline__ void tile_mrows(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                           int64_t r1, int lane) {
  using PK = Pack<Real, VB>;
  constexpr int U = MrowPasses<Real>::value;
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  int rip, v0;
  bool on;
  lane_slot(g, lane, &rip, &v0, &on);
  const int64_t B = g.B;
  const int64_t lo = (int64_t)(on ? v0 : 0) * VB;
  for (int pp = 0; pp < g.P && r0 + (int64_t)pp * g.RP < r1; pp += U) {
    int64_t y[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      y[u] = r0 + (int64_t)(pp + u) * g.RP + rip;
      ok[u] = on && pp + u < g.P && y[u] < r1;
    }
    PK p0[U], p1[U];
#pragma unroll 1
    for (int i = 0; i < n_in; ++i) {
      const bool leaf = d.in[i].flags & kInLeaf;
      const uint32_t lp = w->lpart[i][lane];
      PK a0[U], a1[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t k = ok[u] ? w->tab[i][pp + u] + lp : 0u;  // idle items read row 0 and store nothing
        const int64_t e = d.in[i].off + (int64_t)(2 * k) * B + (ok[u] ? lo : 0);
        a0[u] = ldv_in<Real, VB, true>(data, e, leaf);
        a1[u] = ldv_in<Real, VB, true>(data, e + B, leaf);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (i == 0) {
          p0[u] = a0[u];
          p1[u] = a1[u];
        } else {
          pmul<Real, VB>(p0[u], a0[u]);
          pmul<Real, VB>(p1[u], a1[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      PK o;
#pragma unroll
      for (int v = 0; v < VB; ++v) o.c[v] = cadd<Real>(p0[u].c[v], p1[u].c[v]);
      stv<Real, VB>(data, d.out_off + y[u] * B + lo, o);
    }
  }
}

// Factor rows of one item of an adjoint step on the multi-row layout: a
// factor flagged kInNoPair (the output adjoint) gives one row for x = 0 and 1.
template <class Real, int VB, int U>
__device__ __forceinline__ void mrows_factors(const WarpTile* w, const Real* __restrict__ data, const TileGeom& g,
                                              int pp, int lane, const bool (&ok)[U], int64_t lo, Pack<Real, VB> (&p0)[U],
                                              Pack<Real, VB> (&p1)[U]) {
  const DevBucket& d = w->d;
  const int64_t B = g.B;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < VB; ++v) {
      p0[u].c[v].x = 1;
      p0[u].c[v].y = 0;
      p1[u].c[v] = p0[u].c[v];
    }
#pragma unroll 1
  for (int i = 0; i < d.n_in; ++i) {
    const int32_t fl = d.in[i].flags;
    const bool leaf = fl & kInLeaf;
    const uint32_t lp = w->lpart[i][lane];
    Pack<Real, VB> a0[U], a1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t k = ok[u] ? w->tab[i][pp + u] + lp : 0u;
      const int64_t l = ok[u] ? lo : 0;
      if (fl & kInNoPair) {
        if constexpr (VB == 1)
          a0[u] = ld_nopair<Real>(data, d.in[i].off + (int64_t)k * B + l, fl);
        else
          a0[u] = ldv_in<Real, VB, true>(data, d.in[i].off + (int64_t)k * B + l, leaf);
        a1[u] = a0[u];
      } else {
        const int64_t e = d.in[i].off + (int64_t)(2 * k) * B + l;
        a0[u] = ldv_in<Real, VB, true>(data, e, leaf);
        a1[u] = ldv_in<Real, VB, true>(data, e + B, leaf);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      pmul<Real, VB>(p0[u], a0[u]);
      pmul<Real, VB>(p1[u], a1[u]);
    }
  }
}

template <class Real, int VB>
__device__ __forceinline__ void tile_adjoint_mrows(WarpTile* w, Real* __restrict__ data, const TileGeom& g,
                                                   int64_t r0, int64_t r1, int lane) {
  using PK = Pack<Real, VB>;
  constexpr int U = MrowPasses<Real>::value;
  const DevBucket& d = w->d;
  const int n_in = d.n_in;
  const bool full = d.aflags & kAdjFull;
  int rip, v0;
  bool on;
  lane_slot(g, lane, &rip, &v0, &on);
  const int64_t B = g.B;
  const int64_t lo = (int64_t)(on ? v0 : 0) * VB;
  const uint32_t lp_t = w->lpart[n_in][lane];
  for (int pp = 0; pp < g.P && r0 + (int64_t)pp * g.RP < r1; pp += U) {
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ok[u] = on && pp + u < g.P && r0 + (int64_t)(pp + u) * g.RP + rip < r1;
    PK p0[U], p1[U];
    mrows_factors<Real, VB, U>(w, data, g, pp, lane, ok, lo, p0, p1);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      const uint32_t kt = w->tab[n_in][pp + u] + lp_t;
      const int64_t e0 = d.out_off + (int64_t)(2 * kt) * B + lo;
      if (f64_target<Real>(d)) {
#pragma unroll
        for (int v = 0; v < VB; ++v) {
          put_f64_cx<Real>(data, e0 + v, p0[u].c[v], full);
          put_f64_cx<Real>(data, e0 + B + v, p1[u].c[v], full);
        }
      } else if (full) {
        stv<Real, VB>(data, e0, p0[u]);
        stv<Real, VB>(data, e0 + B, p1[u]);
      } else if (VB == 2) {  // a lane's two angle sets are adjacent elements
        atomic_add_pair<Real>(data, e0, p0[u].c[0], p0[u].c[VB - 1]);
        atomic_add_pair<Real>(data, e0 + B, p1[u].c[0], p1[u].c[VB - 1]);
      } else {
#pragma unroll
        for (int v = 0; v < VB; ++v) {
          atomic_add_cx<Real>(data, e0 + v, p0[u].c[v]);
          atomic_add_cx<Real>(data, e0 + B + v, p1[u].c[v]);
        }
      }
    }
  }
}

// Reduction adjoint step (kStepAdjRed) on the multi-row layout: rows q =
// kt * 2^comp_bits + c with the lanes' rip on the low completion bits (their
// lane parts from the complement record), so one pass holds RP completions of
// one target row.  A lane sums its passes while the target row stays the
// same (2^comp_bits / RP passes), then the RP lanes of each vector are summed
// in a shuffle tree and lane rip = 0 adds the target element.
template <class Real, int VB>
__device__ __forceinline__ void tile_adjred_mrows(WarpTile* w, Real* __restrict__ data, const TileGeom& g,
                                                  int64_t r0, int64_t r1, int lane) {
  using PK = Pack<Real, VB>;
  constexpr int U = MrowPasses<Real>::value;
  const DevBucket& d = w->d;
  int rip, v0;
  bool on;
  lane_slot(g, lane, &rip, &v0, &on);
  const int64_t B = g.B;
  const int64_t lo = (int64_t)(on ? v0 : 0) * VB;
  const int seg = (1 << d.comp_bits) / g.RP;  // passes per target row (>= 1: comp_bits >= 5, RP <= 32)
  PK s0, s1;
#pragma unroll
  for (int v = 0; v < VB; ++v) {
    s0.c[v].x = 0;
    s0.c[v].y = 0;
    s1.c[v] = s0.c[v];
  }
  for (int pp = 0; pp < g.P && r0 + (int64_t)pp * g.RP < r1; pp += U) {
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ok[u] = on && pp + u < g.P && r0 + (int64_t)(pp + u) * g.RP + rip < r1;
    PK p0[U], p1[U];
    mrows_factors<Real, VB, U>(w, data, g, pp, lane, ok, lo, p0, p1);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = pp + u;
      if (q >= g.P || r0 + (int64_t)q * g.RP >= r1) break;  // warp-uniform: the tile's last pass is done
      if (ok[u]) {
#pragma unroll
        for (int v = 0; v < VB; ++v) {
          s0.c[v] = cadd<Real>(s0.c[v], p0[u].c[v]);
          s1.c[v] = cadd<Real>(s1.c[v], p1[u].c[v]);
        }
      }
      if ((q + 1) % seg == 0 || q + 1 == g.P || r0 + (int64_t)(q + 1) * g.RP >= r1) {  // end of a target row
        const uint32_t kt = (uint32_t)((r0 + (int64_t)q * g.RP) >> d.comp_bits);
        for (int off = g.RP / 2; off >= 1; off >>= 1)  // (warp-uniform; lanes rip < off take rip + off's sums)
#pragma unroll
          for (int v = 0; v < VB; ++v) {
            s0.c[v] = cadd<Real>(s0.c[v], shfl_down_cx(s0.c[v], off * g.Bv));
            s1.c[v] = cadd<Real>(s1.c[v], shfl_down_cx(s1.c[v], off * g.Bv));
          }
        if (on && rip == 0) {
          const int64_t e0 = d.out_off + (int64_t)(2 * kt) * B + lo;
          if (f64_target<Real>(d)) {
#pragma unroll
            for (int v = 0; v < VB; ++v) {
              put_f64_cx<Real>(data, e0 + v, s0.c[v], false);
              put_f64_cx<Real>(data, e0 + B + v, s1.c[v], false);
            }
          } else if (VB == 2) {
            atomic_add_pair<Real>(data, e0, s0.c[0], s0.c[VB - 1]);
            atomic_add_pair<Real>(data, e0 + B, s1.c[0], s1.c[VB - 1]);
          } else {
#pragma unroll
            for (int v = 0; v < VB; ++v) {
              atomic_add_cx<Real>(data, e0 + v, s0.c[v]);
              atomic_add_cx<Real>(data, e0 + B + v, s1.c[v]);
            }
          }
        }
#pragma unroll
        for (int v = 0; v < VB; ++v) {
          s0.c[v].x = 0;
          s0.c[v].y = 0;
          s1.c[v] = s0.c[v];
        }
      }
    }
  }
}

// One warp evaluates output rows [r0, r1) of the bucket in w->d (all B angle
// sets).  r0 is a multiple of g.R.  The pass table tab[i][p] =
// pext(r0 + p * RP, mask_i) is built here; the lane parts must already be in
// w->lpart.  Per item an input row is one table read plus one add.
template <class Real, int VB, bool PAIR, bool CG, bool GRAD = false, int STAGE = 0>
__device__ __forceinline__ void warp_tile(WarpTile* w, Real* __restrict__ data, const TileGeom& g, int64_t r0,
                                          int64_t r1, int lane, DevCtrl* ctrl = nullptr, int dbg_bucket = -1) {
  const DevBucket& d = w->d;
  const int n_rec = d.kind == kStepAdj ? d.n_in + 1 : d.n_in + (STAGE == 4 && d.kind == kStepFwd ? d.chain : 0);
  int rip, v0;
  bool lane_on;
  lane_slot(g, lane, &rip, &v0, &lane_on);
  const int P = g.P;
  if (GRAD && d.kind == kStepAdjRed && (d.aflags & kAdjRedLow)) {  // row q = (h << 5) | lane, RP = 32
    const uint32_t hmask = (1u << d.comp_bits) - 1u;
    for (int pp = lane; pp < P; pp += 32) {
      const uint32_t h = (uint32_t)((r0 + (int64_t)pp * g.RP) >> 5);
      const uint32_t yp = pdep_in(h & hmask, d.in[d.n_in + 1]) | pdep_in(h >> d.comp_bits, d.in[d.n_in + 2]);
      for (int i = 0; i <= d.n_in; ++i) w->tab[i][pp] = pext_in(yp, d.in[i]);
    }
  } else if (GRAD && d.kind == kStepAdjRed) {  // row q = kt * 2^comp_bits + c: y = pdep(kt, mask_t) | pdep(c, ~mask_t)
    const uint32_t cmask = (1u << d.comp_bits) - 1u;
    for (int pp = lane; pp < P; pp += 32) {
      const uint32_t q = (uint32_t)(r0 + (int64_t)pp * g.RP);
      const uint32_t yp = pdep_in(q >> d.comp_bits, d.in[d.n_in]) | pdep_in(q & cmask, d.in[d.n_in + 1]);
      for (int i = 0; i < d.n_in; ++i) w->tab[i][pp] = pext_in(yp, d.in[i]);
    }
  } else {
    for (int pp = lane; pp < P; pp += 32) {
      const uint32_t yp = (uint32_t)(r0 + (int64_t)pp * g.RP);
      for (int i = 0; i < n_rec; ++i) w->tab[i][pp] = pext_in(yp, d.in[i]);
    }
  }
  __syncwarp();
  if (!GRAD || d.kind == kStepFwd) {  // (adjoint tiles below are compiled only into GRAD kernels)
    // STAGE 2: every forward tile of a row-wide or one-angle-set plan on the
    // lean row / pair path (the launcher picks STAGE 2 only for those
    // shapes; any other shape is reported, not computed); STAGE 4: the same
    // plus chained steps (a kernel of its own for plans that have them: the
    // chained tiles compiled into the STAGE 2 kernel made its other tiles 20 %
    // slower); STAGE 0: the generic register path
    bool done = false;
    if (STAGE == 4 && d.chain > 0) {  // chained steps: the STAGE 4 lean tiles only (the launcher picks STAGE 4
                                      // for every plan that has them)
      if constexpr (STAGE == 4 && !GRAD) {
        if (!PAIR && g.RP == 1 && g.VC == 1)
          tile_rows_chained<Real, VB>(w, data, g, r0, r1, lane, ctrl);
        else if (PAIR && g.RP == 32 && g.VC == 1 && d.chain == 1)  // (one consumer: the planner's cap)
          tile_pairs_loop<Real, 1>(w, data, g, r0, r1, lane);
        else if (lane == 0 && ctrl != nullptr)
          atomicCAS(&ctrl->status, 0, (int32_t)QT_EINVAL);
      } else {
        if (lane == 0 && ctrl != nullptr) atomicCAS(&ctrl->status, 0, (int32_t)QT_EINVAL);
      }
      done = true;
    } else if (STAGE == 5) {  // multi-row lean tiles (a kernel of its own)
      if (!PAIR && g.RP > 1 && g.VC == 1)
        tile_mrows<Real, VB>(w, data, g, r0, r1, lane);
      else if (lane == 0 && ctrl != nullptr)
        atomicCAS(&ctrl->status, 0, (int32_t)QT_EINVAL);
      done = true;
    } else if (STAGE == 2 || STAGE == 4) {
      if (PAIR && g.RP == 32 && g.VC == 1)
        tile_pairs_regs<Real>(w, data, g, r0, r1, lane);
      else if (!PAIR && g.RP == 1 && g.VC == 1)
        tile_rows_regs<Real, VB>(w, data, g, r0, r1, lane);
      else if (lane == 0 && ctrl != nullptr)
        atomicCAS(&ctrl->status, 0, (int32_t)QT_EINVAL);
      done = true;
    }
    if (STAGE == 3 && !done) {  // float pairs with two vector chunks per row (a kernel of its own: compiled
                       // into the STAGE 2 kernel, this tile raised that kernel's spills)
      if (!PAIR && g.RP == 1 && g.VC == 2)
        tile_rows_vc2<Real, VB>(w, data, g, r0, r1, lane);
      else if (lane == 0 && ctrl != nullptr)
        atomicCAS(&ctrl->status, 0, (int32_t)QT_EINVAL);
      done = true;
    }
    if (!done) tile_items<Real, VB, PAIR, CG, 2, 0>(w, data, g, r0, r1, lane, rip, v0, lane_on, ctrl, dbg_bucket);
  } else {
    if constexpr (GRAD) {
      if (std::is_same<Real, ff>::value &&
          !(STAGE == 2 ? PAIR && g.RP == 32 && g.VC == 1
                       : STAGE == 5 && !PAIR && g.RP > 1 && g.VC == 1 &&
                             (d.kind == kStepZero || !(d.aflags & kAdjRedLow)))) {
        // float-pair gradients run on the pair and multi-row tiles only (those take the FP64 adjoint tensors)
        if (lane == 0 && ctrl != nullptr) atomicCAS(&ctrl->status, 0, (int32_t)QT_EINVAL);
        return;
      }
      if (d.kind == kStepAdj) {
        if (STAGE == 2 && PAIR && g.RP == 32 && g.VC == 1) {
          const bool nf = adj_nf_form(d);
          if (nf && d.n_in == 2)
            tile_adjoint_pairs_nf<Real, 2>(w, data, g, r0, r1, lane);
          else if (nf && d.n_in == 3)
            tile_adjoint_pairs_nf<Real, 3>(w, data, g, r0, r1, lane);
          else if (nf && d.n_in == 4)
            tile_adjoint_pairs_nf<Real, 4>(w, data, g, r0, r1, lane);
          else
            tile_adjoint_pairs<Real>(w, data, g, r0, r1, lane);
        }
        else if (STAGE == 2 && !PAIR && g.RP == 1 && g.VC == 1)
          tile_adjoint_rows<Real, VB>(w, data, g, r0, r1, lane);
        else if (STAGE == 5 && !PAIR && g.RP > 1 && g.VC == 1)
          tile_adjoint_mrows<Real, VB>(w, data, g, r0, r1, lane);
        else
          tile_adjoint<Real, VB, PAIR, CG, 2>(w, data, g, r0, r1, lane, rip, v0, lane_on, ctrl, dbg_bucket);
      } else if (d.kind == kStepAdjRed) {
        if (STAGE == 2 && PAIR && g.RP == 32 && g.VC == 1) {
          const bool nf = adj_nf_form(d);
          if (nf && d.n_in == 2)
            tile_adjred_pairs_nf<Real, 2>(w, data, g, r0, r1, lane);
          else if (nf && d.n_in == 3)
            tile_adjred_pairs_nf<Real, 3>(w, data, g, r0, r1, lane);
          else if (nf && d.n_in == 4)
            tile_adjred_pairs_nf<Real, 4>(w, data, g, r0, r1, lane);
          else
            tile_adjred_pairs<Real>(w, data, g, r0, r1, lane);
        }
        else if (STAGE == 5 && !PAIR && g.RP > 1 && g.VC == 1 && !(d.aflags & kAdjRedLow))
          tile_adjred_mrows<Real, VB>(w, data, g, r0, r1, lane);
        else
          tile_adjred<Real, VB, PAIR, CG, 2>(w, data, g, r0, r1, lane, rip, v0, lane_on, ctrl, dbg_bucket);
      } else {
        tile_zero<Real, VB, PAIR, 2>(w, data, g, r0, r1, rip, v0, lane_on);
      }
    }
  }
}

}  // namespace dev
}  // namespace qt
