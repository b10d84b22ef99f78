// Global kernels of the forward (energy) path.  See kernels.cuh for the
// bucket product-sum device function and the data layout.
#include "kernels.cuh"
#include "kernels_api.h"

namespace qt {
namespace dev {

// Angle table (qt_device.h, kTrigStride doubles per angle set and layer):
// the cos and sin values the ZZ and mixer leaves take, and log r of each.
//
// complex128: the FP64 cos and sin, log r = 0.
// complex64: every leaf is stored as a float pair (c, s), and any such pair
// is exactly r (cos t', sin t') with r = |(c, s)| and t' = atan2(s, c): a
// stored gate (ZZ phase or mixer) is r times the exact gate at the angle t'.
// The pair is chosen to put t' as close to t as the float grid allows: the
// larger of |cos t|, |sin t| is stepped over the floats within kUnitSearch
// ulps of its rounded value, the other component is the float nearest to
// the same ratio, and the candidate with the smallest angle |t' - t| (from
// its cross product with (cos t, sin t), in FP64) wins.  Nearest
// rounding of both leaves up to about 4e-8 rad of angle error and a norm
// error of the same size; the search brings the angle error under about
// 1.5e-8 rad at every angle (less where the two components' grids do not
// step together), and the norm error is divided out per network in FP64
// (energy_kernel and leafgrad_kernel, with the network's leaf counts).
// The search runs a warp per angle: FP64 arithmetic is scarce on this GPU
// and a thread per angle took 0.22 ms of the bench step.
constexpr int kUnitSearch = 48;

__device__ __forceinline__ float step_ulps(float x, int k) { return __int_as_float(__float_as_int(x) + k); }

// One warp searches the float pair of one angle t: lane l tries the
// candidates j = l, l + 32, l + 64 (< 2 kUnitSearch + 1; candidate j steps the
// larger component by k = 0, 1, -1, 2, -2, ... ulps), scoring |cross product|
// with (cos t, sin t) (the angle error times the pair's length, which is 1 to
// within 2e-6 on all candidates) plus 1e-12 |k|, so near-ties go to the nearest
// float; a warp argmin (smallest score, then smallest j) picks the pair.
__device__ void unit_pair_f32_warp(double t, int lane, double* c_out, double* s_out, double* log_r) {
  double st, ct;
  sincos(t, &st, &ct);
  const bool cbig = fabs(ct) >= fabs(st);
  const double big = cbig ? ct : st, small = cbig ? st : ct;
  const double ratio = small / big;
  const float b0 = (float)big;  // |big| >= 1/sqrt(2): stepping its bits never crosses zero
  double best = 1e300;
  int best_j = 1 << 30;
  for (int j = lane; j <= 2 * kUnitSearch; j += 32) {
    const int k = (j & 1) ? (j + 1) / 2 : -(j / 2);
    const float bk = step_ulps(b0, k);
    const float sk = (float)((double)bk * ratio);
    const double err = fabs(fma((double)sk, big, -(double)bk * small)) + 1e-12 * (double)abs(k);
    if (err < best) {
      best = err;
      best_j = j;
    }
  }
  for (int off = 16; off >= 1; off >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oj = __shfl_xor_sync(0xffffffffu, best_j, off);
    if (ob < best || (ob == best && oj < best_j)) {
      best = ob;
      best_j = oj;
    }
  }
  const int k = (best_j & 1) ? (best_j + 1) / 2 : -(best_j / 2);
  const float bb = step_ulps(b0, k);
  const float sb = (float)((double)bb * ratio);
  const double c = cbig ? (double)bb : (double)sb, s = cbig ? (double)sb : (double)bb;
  *c_out = c;
  *s_out = s;
  *log_r = 0.5 * log(c * c + s * s);
}

// complex128 (and float pairs): one thread per (angle set, layer)
__global__ void trig_kernel_f64(const double* __restrict__ gamma, const double* __restrict__ beta, int32_t p,
                                int32_t B, double* __restrict__ trig) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * p) return;
  double* t = trig + (int64_t)kTrigStride * i;
  double sg, cg, sb, cb;
  sincos(gamma[i], &sg, &cg);
  sincos(beta[i], &sb, &cb);
  t[0] = cg;
  t[1] = sg;
  t[2] = cb;
  t[3] = sb;
  t[4] = 0.0;
  t[5] = 0.0;
}

// complex64: one warp per (angle set, layer, gamma or beta)
__global__ void trig_kernel_f32(const double* __restrict__ gamma, const double* __restrict__ beta, int32_t p,
                                int32_t B, double* __restrict__ trig) {
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wg >= 2 * (int64_t)B * p) return;  // whole warps leave together
  const int32_t i = (int32_t)(wg >> 1);
  const bool is_beta = wg & 1;
  double c, s, lr;
  unit_pair_f32_warp(is_beta ? beta[i] : gamma[i], lane, &c, &s, &lr);
  if (lane == 0) {
    double* t = trig + (int64_t)kTrigStride * i;
    t[is_beta ? 2 : 0] = c;
    t[is_beta ? 3 : 1] = s;
    t[is_beta ? 5 : 4] = lr;
  }
}

// |+> amplitude 1/sqrt(2) as the leaves store it, and log of its ratio to
// the exact value (the |+> part of a network's norm correction).
template <class Real> __device__ __forceinline__ double plus_amp() { return (double)(Real)0.70710678118654752440; }
template <class Real> __device__ __forceinline__ double log_r_plus() {
  return sizeof(Real) == sizeof(double) ? 0.0 : log(plus_amp<Real>() * 1.41421356237309504880);
}

// log of the stored-gate norm product of network k at angle set b (0 for
// complex128): sum over its leaves of log r.
__device__ __forceinline__ double network_log_r(const int32_t* __restrict__ counts, int32_t k, int32_t b, int32_t p,
                                                const double* __restrict__ trig, double lr_plus) {
  const int32_t* c = counts + (int64_t)k * (2 * p + 1);
  double acc = (double)c[2 * p] * lr_plus;
  for (int32_t q = 0; q < p; ++q) {
    const double* t = trig + ((int64_t)b * p + q) * kTrigStride;
    acc += (double)c[q] * t[4] + (double)c[p + q] * t[5];
  }
  return acc;
}

// Value of one leaf at its index bits (§Diagonal gate simplification and
// eq. (zz_gates_circ) in this library's convention):
//   |+>  : 1/sqrt(2)
//   ZZ_q : exp(-i gamma_q z_a z_b) = cos g - i s sin g, s = +1 if bits equal else -1
//   MIX_q: cos b if new == old else -i sin b
//   OBS  : +1 for bit 0, -1 for bit 1
// conj = 1 takes the complex conjugate (bra half of the network).
// Fields of a packed leaf (qt_device.h): layer, and the bit of slot 0 / 1 at
// leaf-factor index z (a fixed slot gives its fixed value).
__device__ __forceinline__ int32_t leaf_layer(uint32_t w) { return (int32_t)((w >> 19) & 127u); }
__device__ __forceinline__ uint32_t leaf_bit0(uint32_t w, uint32_t z) {
  return (w >> 15) & 1u ? (w >> 16) & 1u : (z >> ((w >> 5) & 31u)) & 1u;
}
__device__ __forceinline__ uint32_t leaf_bit1(uint32_t w, uint32_t z) {
  return (w >> 17) & 1u ? (w >> 18) & 1u : (z >> ((w >> 10) & 31u)) & 1u;
}

// The leaf's value as it is stored for precision Real (the ZZ and mixer
// values come from the angle table, already Real-exact; the |+> amplitude
// is rounded to Real), returned in FP64 so that products of leaves are
// taken in FP64 and rounded to Real once.
template <class Real>
__device__ __forceinline__ double2 leaf_value_bits(uint32_t w, uint32_t b0, uint32_t b1, const double* tr) {
  const uint32_t kind = w & 3u, conj = (w >> 2) & 1u;
  double2 v;
  if (kind == 0u) {
    v.x = plus_amp<Real>();
    v.y = 0.0;
  } else if (kind == 1u) {
    const double s = (b0 == b1) ? 1.0 : -1.0;
    v.x = tr[0];
    v.y = -s * tr[1];
  } else if (kind == 2u) {
    if (b0 == b1) {
      v.x = tr[2];
      v.y = 0.0;
    } else {
      v.x = 0.0;
      v.y = -tr[3];
    }
  } else {
    v.x = b0 ? -1.0 : 1.0;
    v.y = 0.0;
  }
  if (conj) v.y = -v.y;
  return v;
}

template <class Real>
__device__ __forceinline__ double2 leaf_value(uint32_t w, uint32_t z, const double* tr) {
  return leaf_value_bits<Real>(w, leaf_bit0(w, z), leaf_bit1(w, z), tr);
}

// Product of Real-exact leaf values, accumulated without rounding error worth
// speaking of and rounded to Real once.  complex128: FP64 products.
// complex64: FP64 arithmetic is scarce on this GPU (a small fraction of the
// FP32 rate), so the running product is kept as an unevaluated sum of two
// floats per component (hi + lo, about 48 significant bits) and each leaf,
// an exact float, is multiplied in with error-free transformations on the
// FP32 pipes (the product's rounding error from an FMA, the sum's from the
// two-sum identity).
template <class Real> struct LeafAcc;
template <> struct LeafAcc<double> {
  double2 v = make_double2(1.0, 0.0);
  __device__ __forceinline__ void mul(double2 l) { v = cmul<double>(v, l); }
  __device__ __forceinline__ double2 rounded() const { return v; }
};
__device__ __forceinline__ void two_prod(float a, float b, float* p, float* e) {
  *p = a * b;
  *e = fmaf(a, b, -*p);
}
__device__ __forceinline__ void two_sum(float a, float b, float* s, float* e) {
  *s = a + b;
  const float bb = *s - a;
  *e = (a - (*s - bb)) + (b - bb);
}
template <> struct LeafAcc<float> {
  float rh = 1.f, rl = 0.f, ih = 0.f, il = 0.f;  // re = rh + rl, im = ih + il
  __device__ __forceinline__ void mul(double2 l) {
    const float lr = (float)l.x, li = (float)l.y;  // exact: leaves are stored as floats
    float p1, e1, p2, e2, p3, e3, p4, e4;
    two_prod(rh, lr, &p1, &e1);
    two_prod(ih, li, &p2, &e2);
    two_prod(rh, li, &p3, &e3);
    two_prod(ih, lr, &p4, &e4);
    float s, t;
    two_sum(p1, -p2, &s, &t);  // re = rh lr - ih li + (lo parts)
    t += (e1 - e2) + (rl * lr - il * li);
    const float nrh = s + t, nrl = t - (nrh - s);
    two_sum(p3, p4, &s, &t);   // im = rh li + ih lr + (lo parts)
    t += (e3 + e4) + (rl * li + il * lr);
    const float nih = s + t, nil = t - (nih - s);
    rh = nrh;
    rl = nrl;
    ih = nih;
    il = nil;
  }
  // hi is the float nearest to hi + lo (each update renormalises the pair)
  __device__ __forceinline__ float2 rounded() const { return make_float2(rh, ih); }
};
// Float pairs: the product of the leaves (each an FP64 value split into a
// pair) in float-pair arithmetic.
template <> struct LeafAcc<ff> {
  ff2 v = ff2{ff(1.0f, 0.0f), ff(0.0f, 0.0f)};
  __device__ __forceinline__ void mul(double2 l) { v = cmul<ff>(v, ff2{ff(l.x), ff(l.y)}); }
  __device__ __forceinline__ ff2 rounded() const { return v; }
};

// Leaf factors for up to LeafTabB<Real> angle sets: one block per factor.
// Each leaf takes at most 4 values (its two slot bits) per angle set; the
// block tabulates them in 32 KB of shared memory once (the stored values are
// Real-exact, so the table holds them in Real), then every element of the
// factor is the product, in leaf order, of one table entry per leaf
// (LeafAcc: rounded to Real once) -- the same values multiplied in the same
// order as leaf_factor_kernel.
template <class Real> struct LeafTabB { static constexpr int value = 32768 / (kDevMaxLeaves * 4 * 2 * (int)sizeof(Real)); };

template <class Real>
__device__ __forceinline__ typename Cx<Real>::T to_real(double2 v) {
  typename Cx<Real>::T r;
  r.x = (Real)v.x;
  r.y = (Real)v.y;
  return r;
}

template <class Real>
__global__ void leaf_factor_tab_kernel(const DevLeafFactor* __restrict__ lf, int32_t n_lf,
                                       const double* __restrict__ trig, int32_t p, int32_t B,
                                       Real* __restrict__ data) {
  using C = typename Cx<Real>::T;
  __shared__ C tab[kDevMaxLeaves][4][LeafTabB<Real>::value];
  __shared__ uint32_t words[kDevMaxLeaves];
  for (int32_t f = blockIdx.x; f < n_lf; f += gridDim.x) {
    const DevLeafFactor& F = lf[f];
    const int32_t nl = F.n_leaves;
    __syncthreads();  // the previous factor's readers are done with the table
    for (int32_t i = threadIdx.x; i < nl * 4 * B; i += blockDim.x) {
      const int32_t l = i / (4 * B), c = (i / B) & 3, b = i % B;
      const uint32_t w = F.leaf[l];
      const int32_t layer = leaf_layer(w);
      // a fixed slot reads its fixed value whatever the combination says
      const uint32_t b0 = (w >> 15) & 1u ? (w >> 16) & 1u : (uint32_t)(c & 1);
      const uint32_t b1 = (w >> 17) & 1u ? (w >> 18) & 1u : (uint32_t)(c >> 1);
      tab[l][c][b] = to_real<Real>(
          leaf_value_bits<Real>(w, b0, b1, trig + ((int64_t)b * p + (layer > 0 ? layer - 1 : 0)) * kTrigStride));
    }
    if (threadIdx.x < nl) words[threadIdx.x] = F.leaf[threadIdx.x];
    __syncthreads();
    const int32_t n = (1 << F.rank) * B;
    for (int32_t idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const uint32_t z = idx / B;
      const int32_t b = idx - (int32_t)z * B;
      LeafAcc<Real> acc;
      for (int32_t l = 0; l < nl; ++l) {
        const uint32_t w = words[l];
        const uint32_t c = ((z >> ((w >> 5) & 31u)) & 1u) | (((z >> ((w >> 10) & 31u)) & 1u) << 1);
        const C t = tab[l][c][b];
        acc.mul(make_double2((double)t.x, (double)t.y));
      }
      reinterpret_cast<C*>(data)[F.off + idx] = acc.rounded();
    }
  }
}

template <class Real>
__global__ void leaf_factor_kernel(const DevLeafFactor* __restrict__ lf, int32_t n_lf,
                                   const double* __restrict__ trig, int32_t p, int32_t B,
                                   Real* __restrict__ data) {
  using C = typename Cx<Real>::T;
  for (int32_t f = blockIdx.x; f < n_lf; f += gridDim.x) {
    const DevLeafFactor F = lf[f];
    const int32_t n = (1 << F.rank) * B;
    for (int32_t idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const uint32_t z = idx / B;
      const int32_t b = idx - (int32_t)z * B;
      LeafAcc<Real> acc;
      for (int32_t l = 0; l < F.n_leaves; ++l) {
        const uint32_t w = F.leaf[l];
        const int32_t layer = leaf_layer(w);
        const double* tr = trig + ((int64_t)b * p + (layer > 0 ? layer - 1 : 0)) * kTrigStride;
        acc.mul(leaf_value<Real>(w, z, tr));
      }
      reinterpret_cast<C*>(data)[F.off + idx] = acc.rounded();
    }
  }
}

// One launch per bucket (the plain per-bucket path): warp w of the grid
// takes tiles w, w + n_warps, ... of the bucket.
template <class Real, int VB, bool PAIR>
__global__ void __launch_bounds__(256, 4) bucket_kernel(const DevBucket d, Real* __restrict__ data, const TileGeom g,
                                                     int64_t n_tiles) {
  __shared__ WarpTile tiles[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpTile* w = &tiles[wid];
  load_bucket(&w->d, &d, lane);
  __syncwarp();
  lane_parts(w, g, lane);
  __syncwarp();
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; t < n_tiles; t += n_warps) {
    const int64_t r0 = t * g.R;
    const int64_t r1 = r0 + g.R < d.n_rows ? r0 + g.R : d.n_rows;
    warp_tile<Real, VB, PAIR, false>(w, data, g, r0, r1, lane);
    __syncwarp();
  }
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}
__device__ __forceinline__ uint32_t smid() {
  uint32_t v;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
  return v;
}

__device__ __forceinline__ int32_t ld_acquire(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Persistent queue, one task = one chunk of a bucket's warp tiles (one tile,
// or `span` consecutive tiles for the widest buckets of a very long queue) or
// one group of single-tile buckets.  Each warp takes tasks in queue order (lane 0: atomicAdd on the
// queue head, issued one task ahead so its latency overlaps a tile), waits
// until every step on its step's dependency list has all its tiles done
// (lane q polls the entries q, q + 32, ...), evaluates the tile(s) and counts
// the bucket's tile done.  Every
// awaited tile comes earlier in the queue and is held by a running warp that
// only waits on still earlier tiles, so every wait ends.  Waits are bounded:
// after `spin_limit` polls (or as soon as another warp has failed) the warp
// records QT_ETIMEOUT in the control word and no warp takes a task after that.
// Consecutive tiles of one bucket on a warp reuse its record and skip the
// wait (done counters only grow).
//
// STAGE: 0 generic register path; 2 row-wide and one-angle-set plans on the
// lean register tiles: every forward tile takes tile_rows_regs or
// tile_pairs_regs and the generic forward tile is not compiled in.
template <class Real, int VB, bool PAIR, bool GRAD, int STAGE>
__global__ void __launch_bounds__(256, (STAGE == 4 && PAIR) ? 3 : 4) persistent_kernel(const DevBucket* __restrict__ buckets,
                                                            const DevTask* __restrict__ tasks, int32_t n_tasks,
                                                            DevCtrl* ctrl, int32_t* done, Real* __restrict__ data,
                                                            const TileGeom g, int32_t spin_limit,
                                                            const DevDep* __restrict__ deps,
                                                            unsigned long long* __restrict__ trace) {
  __shared__ WarpTile tiles[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpTile* w = &tiles[wid];
  // Lane 0 claims tasks (the warp acts on broadcasts); the lanes poll a
  // step's dependency list side by side.
  int32_t t = 0, cached = -1;  // cached: bucket whose record and lane parts are in *w
  if (lane == 0) t = atomicAdd(&ctrl->head, 1);
  t = __shfl_sync(0xffffffffu, t, 0);
  while (t < n_tasks) {
    int32_t t_next = n_tasks, failed = 0;
    const DevTask task = tasks[t];
    if (trace != nullptr && lane == 0) w->trace_t[0] = globaltimer();
    if (lane == 0 && *((volatile int32_t*)&ctrl->status) == 0) t_next = atomicAdd(&ctrl->head, 1);
    if (task.bucket != cached) {  // uniform; a warp that ran a chunk of this step already saw its inputs
      // The task carries its step's dependency list; lane q waits for the
      // entries q, q + 32, ... (each poll bounded).  The first entry's load
      // and the copy of the step's record (static, written before the
      // launch) are issued together, so the record arrives during the wait.
      const int32_t nd = task.n_dep, d0 = task.dep;
      DevDep dd{0, 0};
      if (lane < nd) dd = deps[d0 + lane];
      copy_bucket(&w->d, buckets + task.bucket, lane);
      for (int32_t q = lane; q < nd && !failed; q += 32) {
        if (q != lane) dd = deps[d0 + q];
        int32_t polls = 0;
        while (ld_acquire(done + dd.step) < dd.need) {
          ++polls;
          if (polls > spin_limit || ((polls & 63) == 0 && *((volatile int32_t*)&ctrl->status) != 0)) {
            if (atomicCAS(&ctrl->status, 0, (int32_t)QT_ETIMEOUT) == 0) ctrl->spins = dd.step;
            failed = 1;
            break;
          }
          __nanosleep(100);
        }
      }
      __syncwarp();  // every lane's acquire (and record store) before any lane reads
      lane_parts(w, g, lane);
      __syncwarp();
      cached = task.bucket;
    }
    failed = __any_sync(0xffffffffu, failed);
    t_next = __shfl_sync(0xffffffffu, t_next, 0);
    if (failed) break;
    if (trace != nullptr && lane == 0) w->trace_t[1] = globaltimer();
    const int32_t n_group = task.chunk < 0 ? -task.chunk : 1;
    for (int32_t k = 0; k < n_group; ++k) {
      const int32_t b = task.bucket + k;
      if (b != cached) {  // uniform: every lane holds the same b and cached
        load_bucket(&w->d, buckets + b, lane);
        __syncwarp();
        lane_parts(w, g, lane);
        __syncwarp();
        cached = b;
      }
#ifdef QT_DEVICE_CHECKS
      if (w->d.n_in < 1 || w->d.n_in > kDevMaxIn || w->d.n_rows < 1) {
        if (lane == 0 && atomicCAS(&ctrl->bad_kind, 0, 4) == 0) {
          ctrl->bad_bucket = b;
          ctrl->bad_index = w->d.n_in;
          atomicCAS(&ctrl->status, 0, (int32_t)QT_EINVAL);
        }
        break;
      }
#endif
      // a group runs the single tile of each of its steps; a chunk runs
      // `span` consecutive tiles of one step
      const int64_t n_rows = w->d.n_rows;
      const int64_t span = task.chunk < 0 ? 1 : (int64_t)w->d.span;
      const int64_t t0 = task.chunk < 0 ? 0 : (int64_t)task.chunk * span;
      for (int64_t tt = t0; tt < t0 + span; ++tt) {
        const int64_t r0 = tt * g.R;
        if (r0 >= n_rows) break;
        const int64_t r1 = r0 + g.R < n_rows ? r0 + g.R : n_rows;
        warp_tile<Real, VB, PAIR, true, GRAD, STAGE>(w, data, g, r0, r1, lane, ctrl, b);
        __syncwarp();  // the next tile or step reuses the warp's tables and reads what this one wrote
      }
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(done + task.bucket + n_group - 1, 1);
    if (trace != nullptr && lane == 0) {
      unsigned long long* r = trace + 4 * (int64_t)t;
      r[0] = w->trace_t[0];
      r[1] = w->trace_t[1];
      r[2] = globaltimer();
      r[3] = ((unsigned long long)smid() << 16) | (unsigned long long)wid;
    }
    t = t_next;
  }
}

// Final step (§QAOA algorithm, E = sum_k E_k): per angle set, the value of
// each edge network is the product of its scalar bucket results, taken in
// FP64 and divided by the network's stored-gate norm product (complex64:
// exp(network_log_r); 1 for complex128), and E = sum_e (1 - Re <Z_j Z_k>_e)
// / 2 in a fixed order.  One warp per angle set: lane l sums the edges l,
// l + 32, ... in order, then a fixed butterfly adds the 32 partial sums.
template <class Real>
__global__ void energy_kernel(const Real* __restrict__ data, const int64_t* __restrict__ scal_off,
                              const int32_t* __restrict__ scal_begin, const int32_t* __restrict__ net_first,
                              const int32_t* __restrict__ counts, const double* __restrict__ trig, int32_t p,
                              int32_t n_edges, int32_t B, double* __restrict__ energy, double* __restrict__ edge_zz) {
  const int32_t b = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;  // whole warps leave together
  const double lr_plus = log_r_plus<Real>();
  double E = 0.0;
  for (int32_t e = lane; e < n_edges; e += 32) {
    // <Z_j Z_k> = sum over the edge's networks (2^s slices) of the product of
    // each network's scalar results
    double zr = 0.0, zi = 0.0;
    for (int32_t k = net_first[e]; k < net_first[e + 1]; ++k) {
      double nr = 1.0, ni = 0.0;
      for (int32_t s = scal_begin[k]; s < scal_begin[k + 1]; ++s) {
        const int64_t o = scal_off[s] + b;
        const double vr = (double)data[2 * o], vi = (double)data[2 * o + 1];
        const double tr = nr * vr - ni * vi;
        ni = nr * vi + ni * vr;
        nr = tr;
      }
      if (sizeof(Real) != sizeof(double)) {
        const double corr = exp(-network_log_r(counts, k, b, p, trig, lr_plus));
        nr *= corr;
        ni *= corr;
      }
      zr += nr;
      zi += ni;
    }
    if (edge_zz) {
      edge_zz[((int64_t)e * B + b) * 2 + 0] = zr;
      edge_zz[((int64_t)e * B + b) * 2 + 1] = zi;
    }
    E += 0.5 * (1.0 - zr);
  }
  for (int off = 16; off > 0; off >>= 1) E += __shfl_xor_sync(0xffffffffu, E, off);
  if (energy && lane == 0) energy[b] = E;
}

// Derivative of one leaf value with respect to its own angle (the ZZ angle
// gamma_q for kind 1, the mixer angle beta_q for kind 2), at index bits z:
//   ZZ : d/dg exp(-i s g) = -i s exp(-i s g); the bra copy is the conjugate
//   MIX: d/db cos b = -sin b;  d/db (-i sin b) = -i cos b; conjugate for the bra
__device__ __forceinline__ double2 leaf_deriv(uint32_t w, uint32_t z, const double* tr) {
  const uint32_t kind = w & 3u, conj = (w >> 2) & 1u;
  const uint32_t b0 = leaf_bit0(w, z);
  const uint32_t b1 = leaf_bit1(w, z);
  double2 v = make_double2(0.0, 0.0);
  if (kind == 1u) {
    const double s = (b0 == b1) ? 1.0 : -1.0;
    const double2 val = make_double2(tr[0], -s * tr[1]);  // ket value
    v = make_double2(s * val.y, -s * val.x);              // -i s val
  } else if (kind == 2u) {
    v = (b0 == b1) ? make_double2(-tr[3], 0.0) : make_double2(0.0, -tr[2]);
  }
  if (conj) v.y = -v.y;
  return v;
}

// Per leaf factor F and angle set b: for every leaf l of F that carries an
// angle, sum_z Lbar_F[z] * dl(z) * prod_{l' != l} l'(z) (FP64), written to
// part[(f * B + b) * kDevMaxLeaves + l] (zero for leaves without an angle).
// One warp per (F, b); lanes split the 2^rank index values z.  For each z the
// products over the other leaves come from a prefix pass (Lbar times the
// leaves before l) and a suffix pass (the leaves after l), so a z costs
// O(n_leaves) instead of O(n_leaves^2); each leaf's sum is reduced over the
// warp with shuffles.
//
// The parts are divided by the factor's network's stored-gate norm product
// (complex64, see trig_kernel_f32): to first order that is the derivative of the
// exact network at the stored angles.
template <class Real>
__global__ void leafgrad_kernel(const DevLeafFactor* __restrict__ lf, int32_t n_lf, int64_t lbar_shift,
                                const double* __restrict__ trig, const int32_t* __restrict__ counts, int32_t p,
                                int32_t B, const Real* __restrict__ data, double2* __restrict__ part) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (int64_t)n_lf * B) return;
  const int32_t f = (int32_t)(warp / B), b = (int32_t)(warp % B);
  const DevLeafFactor F = lf[f];
  const int32_t n = F.n_leaves;
  double2 acc[kDevMaxLeaves], pre[kDevMaxLeaves], val[kDevMaxLeaves];
  for (int32_t l = 0; l < kDevMaxLeaves; ++l) acc[l] = make_double2(0.0, 0.0);
  for (uint32_t z = (uint32_t)lane; z < (1u << F.rank); z += 32u) {
    const int64_t o = F.off + lbar_shift + (int64_t)z * B + b;
    double2 run;  // Lbar_F[z] (float-pair plans keep adjoints in FP64)
    if constexpr (std::is_same<Real, ff>::value)
      run = reinterpret_cast<const double2*>(data)[o];
    else
      run = make_double2((double)data[2 * o], (double)data[2 * o + 1]);
    for (int32_t l = 0; l < n; ++l) {  // prefix: Lbar times the leaves before l
      const uint32_t w = F.leaf[l];
      const int32_t layer = leaf_layer(w);
      val[l] = leaf_value<Real>(w, z, trig + ((int64_t)b * p + (layer > 0 ? layer - 1 : 0)) * kTrigStride);
      pre[l] = run;
      run = cmul<double>(run, val[l]);
    }
    double2 suf = make_double2(1.0, 0.0);  // the leaves after l
    for (int32_t l = n - 1; l >= 0; --l) {
      const uint32_t w = F.leaf[l];
      const uint32_t kind = w & 3u;
      if (kind == 1u || kind == 2u) {
        const double2 d = leaf_deriv(w, z, trig + ((int64_t)b * p + leaf_layer(w) - 1) * kTrigStride);
        const double2 t = cmul<double>(cmul<double>(pre[l], d), suf);
        acc[l].x += t.x;
        acc[l].y += t.y;
      }
      suf = cmul<double>(suf, val[l]);
    }
  }
  for (int32_t l = 0; l < n; ++l)
    for (int off = 16; off > 0; off >>= 1) {
      acc[l].x += __shfl_xor_sync(0xffffffffu, acc[l].x, off);
      acc[l].y += __shfl_xor_sync(0xffffffffu, acc[l].y, off);
    }
  const double corr = sizeof(Real) == sizeof(double) ? 1.0
                                                     : exp(-network_log_r(counts, F.net, b, p, trig, log_r_plus<Real>()));
  if (lane == 0)
    for (int32_t l = 0; l < kDevMaxLeaves; ++l)
      part[warp * kDevMaxLeaves + l] = l < n ? make_double2(acc[l].x * corr, acc[l].y * corr) : make_double2(0.0, 0.0);
}

// dZ_e/dtheta for every edge e, angle set b and angle theta (0..p-1: gamma,
// p..2p-1: beta): the per-leaf parts of the edge's factors whose leaf carries
// theta.  One warp per (edge, angle set, group of kEdgeGradAngles angles):
// lane l takes the edge's factors l, l + 32, ... and sums, per angle of the
// group, the parts of their leaves that carry it; a fixed butterfly adds the
// lanes (a thread per (edge, angle set, angle) walking all the edge's factors
// alone took 0.3 ms of the 60-vertex p = 4 gradient).
constexpr int kEdgeGradAngles = 8;

__global__ void edgegrad_kernel(const DevLeafFactor* __restrict__ lf, const int32_t* __restrict__ leaf_first,
                                int32_t n_edges, int32_t p, int32_t B, const double2* __restrict__ part,
                                double* __restrict__ dz) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int32_t ng = (2 * p + kEdgeGradAngles - 1) / kEdgeGradAngles;
  if (warp >= (int64_t)n_edges * B * ng) return;  // whole warps leave together
  const int32_t gi = (int32_t)(warp % ng);
  const int32_t b = (int32_t)((warp / ng) % B);
  const int32_t e = (int32_t)(warp / ((int64_t)ng * B));
  const int32_t th0 = gi * kEdgeGradAngles;
  double ar[kEdgeGradAngles], ai[kEdgeGradAngles];
#pragma unroll
  for (int k = 0; k < kEdgeGradAngles; ++k) ar[k] = ai[k] = 0.0;
  for (int32_t f = leaf_first[e] + lane; f < leaf_first[e + 1]; f += 32) {
    const int32_t nl = lf[f].n_leaves;
    for (int32_t l = 0; l < nl; ++l) {
      const uint32_t w = lf[f].leaf[l];
      const uint32_t kind = w & 3u;
      if (kind != 1u && kind != 2u) continue;
      const int32_t slot = (kind == 1u ? leaf_layer(w) - 1 : p + leaf_layer(w) - 1) - th0;
      if (slot < 0 || slot >= kEdgeGradAngles) continue;
      const double2 v = part[((int64_t)f * B + b) * kDevMaxLeaves + l];
#pragma unroll
      for (int k = 0; k < kEdgeGradAngles; ++k)
        if (slot == k) {
          ar[k] += v.x;
          ai[k] += v.y;
        }
    }
  }
#pragma unroll
  for (int k = 0; k < kEdgeGradAngles; ++k)
    for (int off = 16; off > 0; off >>= 1) {
      ar[k] += __shfl_xor_sync(0xffffffffu, ar[k], off);
      ai[k] += __shfl_xor_sync(0xffffffffu, ai[k], off);
    }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kEdgeGradAngles; ++k) {
      const int32_t th = th0 + k;
      if (th >= 2 * p) break;
      const int64_t idx = ((int64_t)e * B + b) * 2 * p + th;
      dz[2 * idx] = ar[k];
      dz[2 * idx + 1] = ai[k];
    }
}

// dE/dtheta = -1/2 sum_e Re dZ_e/dtheta, edges summed in order (E = sum_e (1 - Z_e) / 2).
__global__ void gradreduce_kernel(const double* __restrict__ dz, int32_t n_edges, int32_t p, int32_t B,
                                  double* __restrict__ grad) {
  const int32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * 2 * p) return;
  double acc = 0.0;
  for (int32_t e = 0; e < n_edges; ++e) acc += dz[2 * ((int64_t)e * B * 2 * p + idx)];
  grad[idx] = -0.5 * acc;
}

}  // namespace dev

// ------------------------------------------------------------- launchers ---

cudaError_t launch_trig(int dtype, const double* gamma, const double* beta, int32_t p, int32_t B, double* trig,
                        cudaStream_t s) {
  const int32_t n = B * p;
  if (dtype == QT_C64) {
    const int64_t threads = (int64_t)n * 2 * 32;  // a warp per (angle set, layer, gamma or beta)
    dev::trig_kernel_f32<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(gamma, beta, p, B, trig);
  } else {
    dev::trig_kernel_f64<<<(n + 127) / 128, 128, 0, s>>>(gamma, beta, p, B, trig);
  }
  return cudaGetLastError();
}

cudaError_t launch_leaf_factors(int dtype, const DevLeafFactor* lf, int32_t n_lf, const double* trig,
                                int32_t p, int32_t B, void* data, cudaStream_t s) {
  if (n_lf == 0) return cudaSuccess;
  const int32_t tab_b = dtype == QT_C64 ? dev::LeafTabB<float>::value : dev::LeafTabB<double>::value;
  if (B <= tab_b) {
    const int32_t grid = n_lf < 65535 ? n_lf : 65535;
    if (dtype == QT_C64)
      dev::leaf_factor_tab_kernel<float><<<grid, 256, 0, s>>>(lf, n_lf, trig, p, B, (float*)data);
    else if (dtype == QT_C64X2)
      dev::leaf_factor_tab_kernel<dev::ff><<<grid, 256, 0, s>>>(lf, n_lf, trig, p, B, (dev::ff*)data);
    else
      dev::leaf_factor_tab_kernel<double><<<grid, 256, 0, s>>>(lf, n_lf, trig, p, B, (double*)data);
    return cudaGetLastError();
  }
  const int32_t grid = n_lf < 152 * 16 ? n_lf : 152 * 16;
  if (dtype == QT_C64)
    dev::leaf_factor_kernel<float><<<grid, 128, 0, s>>>(lf, n_lf, trig, p, B, (float*)data);
  else if (dtype == QT_C64X2)
    dev::leaf_factor_kernel<dev::ff><<<grid, 128, 0, s>>>(lf, n_lf, trig, p, B, (dev::ff*)data);
  else
    dev::leaf_factor_kernel<double><<<grid, 128, 0, s>>>(lf, n_lf, trig, p, B, (double*)data);
  return cudaGetLastError();
}

int vector_width(int dtype, int32_t B) { return (dtype == QT_C64 && B > 1 && B % 2 == 0) ? 2 : 1; }

TileGeom tile_geom(int dtype, int32_t B, int32_t lane_items) {
  TileGeom g;
  const int vb = vector_width(dtype, B);
  g.B = B;
  g.Bv = B == 1 ? 1 : B / vb;
  if (g.Bv <= 32) {
    int rp = 1;
    while (rp * 2 * g.Bv <= 32) rp *= 2;
    g.RP = rp;
    g.VC = 1;
  } else {
    g.RP = 1;
    g.VC = (g.Bv + 31) / 32;
  }
  const int32_t cap = lane_items > 0 && lane_items <= kLaneItems ? lane_items : kLaneItems;
  int P = 1;
  while (P * 2 * g.VC <= cap) P *= 2;
  g.P = P;
  g.R = P * g.RP;
  g.wait_limit = 1 << 22;
  g.data_elems = 0;
  return g;
}

cudaError_t launch_bucket(int dtype, const DevBucket& d, int32_t B, int32_t lane_items, void* data,
                          int32_t max_blocks, cudaStream_t s) {
  const int vb = vector_width(dtype, B);
  const bool pair = (B == 1);
  const TileGeom g = tile_geom(dtype, B, lane_items);
  const int64_t n_tiles = (d.n_rows + g.R - 1) / g.R;
  int64_t blocks = (n_tiles + 7) / 8;
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  if (dtype == QT_C64) {
    if (pair)
      dev::bucket_kernel<float, 1, true><<<(int)blocks, 256, 0, s>>>(d, (float*)data, g, n_tiles);
    else if (vb == 2)
      dev::bucket_kernel<float, 2, false><<<(int)blocks, 256, 0, s>>>(d, (float*)data, g, n_tiles);
    else
      dev::bucket_kernel<float, 1, false><<<(int)blocks, 256, 0, s>>>(d, (float*)data, g, n_tiles);
  } else if (dtype == QT_C64X2) {
    if (pair)
      dev::bucket_kernel<dev::ff, 1, true><<<(int)blocks, 256, 0, s>>>(d, (dev::ff*)data, g, n_tiles);
    else
      dev::bucket_kernel<dev::ff, 1, false><<<(int)blocks, 256, 0, s>>>(d, (dev::ff*)data, g, n_tiles);
  } else {
    if (pair)
      dev::bucket_kernel<double, 1, true><<<(int)blocks, 256, 0, s>>>(d, (double*)data, g, n_tiles);
    else
      dev::bucket_kernel<double, 1, false><<<(int)blocks, 256, 0, s>>>(d, (double*)data, g, n_tiles);
  }
  return cudaGetLastError();
}

// Row-wide tile shapes (one output row per pass: complex64 with even B in
// [34, 64], complex128 with B in [17, 32], float pairs with B in [17, 64], one
// or two vector chunks per row) take the lean row tiles; one angle set takes
// the lean pair tile; other batches the generic register tile.
bool row_wide(int dtype, int32_t B) {
  if (B <= 1 || !(dtype == QT_C128 || dtype == QT_C64X2 || vector_width(dtype, B) == 2)) return false;
  const TileGeom g = tile_geom(dtype, B, 0);
  return g.RP == 1 && (g.VC == 1 || (g.VC == 2 && dtype == QT_C64X2));
}

bool chain_fusion_ok(int dtype, int32_t B) {
  return B == 1 || (row_wide(dtype, B) && tile_geom(dtype, B, 0).VC == 1);  // the pair tiles or the row tiles
}

template <class Real, int VB, bool PAIR, bool GRAD, int ST>
static const void* pk_fn() {
  return (const void*)dev::persistent_kernel<Real, VB, PAIR, GRAD, ST>;
}

// Shapes with 2 to 16 rows per warp pass and one vector chunk per row
// (complex64 with an even number of angle sets up to 32, complex128 and float
// pairs up to 16): the multi-row lean tiles (STAGE 5).
static bool multi_row(int dtype, int32_t B) {
  if (B <= 1 || row_wide(dtype, B) || (dtype == QT_C64 && vector_width(dtype, B) != 2)) return false;
  const TileGeom g = tile_geom(dtype, B, 0);
  return g.RP > 1 && g.VC == 1;
}

// Kernel variant of a launch: the lean pair tile (one angle set), the lean
// row tile (row-wide shapes), the multi-row lean tiles, else the generic
// register tile.
template <bool GRAD>
static const void* persistent_fn_g(int dtype, int32_t B) {
  const bool pair = (B == 1);
  const bool lean = pair || row_wide(dtype, B);
  if (multi_row(dtype, B)) {
    if (dtype == QT_C64) return pk_fn<float, 2, false, GRAD, 5>();
    if (dtype == QT_C64X2) return pk_fn<dev::ff, 1, false, GRAD, 5>();
    // complex128 gradients keep the generic tile: the multi-row adjoint tiles spill there
    // (60-vertex p = 4, 4 angle sets: 145.8 -> 160.5 ms)
    if constexpr (!GRAD) return pk_fn<double, 1, false, false, 5>();
  }
  if (dtype == QT_C64) {
    if (pair) return pk_fn<float, 1, true, GRAD, 2>();
    if (vector_width(dtype, B) == 2) return lean ? pk_fn<float, 2, false, GRAD, 2>() : pk_fn<float, 2, false, GRAD, 0>();
    return pk_fn<float, 1, false, GRAD, 0>();
  }
  if (dtype == QT_C64X2) {  // float pairs: gradients for 1 to 16 angle sets (the pair and multi-row tiles)
    if constexpr (GRAD) {
      return pair ? pk_fn<dev::ff, 1, true, true, 2>() : nullptr;
    } else {
      if (pair) return pk_fn<dev::ff, 1, true, false, 2>();
      if (!lean) return pk_fn<dev::ff, 1, false, false, 0>();
      return tile_geom(dtype, B, 0).VC == 2 ? pk_fn<dev::ff, 1, false, false, 3>() : pk_fn<dev::ff, 1, false, false, 2>();
    }
  }
  if (pair) return pk_fn<double, 1, true, GRAD, 2>();
  return lean ? pk_fn<double, 1, false, GRAD, 2>() : pk_fn<double, 1, false, GRAD, 0>();
}

// Forward plans with chained steps take the STAGE 4 variant of their lean
// tile (chain_fusion_ok's shapes: one angle set, or row-wide with one
// vector chunk per row).
static const void* persistent_fn_chains(int dtype, int32_t B) {
  if (!chain_fusion_ok(dtype, B)) return nullptr;
  const bool pair = (B == 1);
  if (dtype == QT_C64) return pair ? pk_fn<float, 1, true, false, 4>() : pk_fn<float, 2, false, false, 4>();
  if (dtype == QT_C64X2) return pair ? pk_fn<dev::ff, 1, true, false, 4>() : pk_fn<dev::ff, 1, false, false, 4>();
  return pair ? pk_fn<double, 1, true, false, 4>() : pk_fn<double, 1, false, false, 4>();
}

static const void* persistent_fn(int dtype, bool grad, int32_t B, bool chains) {
  if (chains) return grad ? nullptr : persistent_fn_chains(dtype, B);
  return grad ? persistent_fn_g<true>(dtype, B) : persistent_fn_g<false>(dtype, B);
}

cudaError_t launch_persistent(int dtype, bool grad, bool chains, const DevBucket* buckets, const DevTask* tasks,
                              int32_t n_tasks, DevCtrl* ctrl, int32_t* done, int32_t B, int32_t lane_items, void* data,
                              int64_t data_elems, int32_t grid, int32_t spin_limit, const DevDep* deps,
                              unsigned long long* trace, cudaStream_t s) {
  TileGeom g = tile_geom(dtype, B, lane_items);
  g.data_elems = data_elems;
  g.wait_limit = 1 << 22;
  const void* fn = persistent_fn(dtype, grad, B, chains);
  if (!fn) return cudaErrorInvalidValue;  // no such variant (float-pair gradients take at most 16 angle sets)
  void* args[] = {(void*)&buckets, (void*)&tasks, (void*)&n_tasks, (void*)&ctrl, (void*)&done, (void*)&data,
                  (void*)&g, (void*)&spin_limit, (void*)&deps, (void*)&trace};
  return cudaLaunchKernel(fn, dim3(grid), dim3(256), args, 0, s);
}

cudaError_t persistent_occupancy(int dtype, bool grad, bool chains, int32_t B, int* blocks_per_sm) {
  const void* fn = persistent_fn(dtype, grad, B, chains);
  if (!fn) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, 256, 0);
}

cudaError_t launch_energy(int dtype, const void* data, const int64_t* scal_off, const int32_t* scal_begin,
                          const int32_t* net_first, const int32_t* counts, const double* trig, int32_t p,
                          int32_t n_edges, int32_t B, double* energy, double* edge_zz, cudaStream_t s) {
  const int32_t grid = (B + 3) / 4;  // 4 warps (angle sets) per block
  if (dtype == QT_C64)
    dev::energy_kernel<float><<<grid, 128, 0, s>>>((const float*)data, scal_off, scal_begin, net_first, counts, trig,
                                                   p, n_edges, B, energy, edge_zz);
  else if (dtype == QT_C64X2)
    dev::energy_kernel<dev::ff><<<grid, 128, 0, s>>>((const dev::ff*)data, scal_off, scal_begin, net_first, counts,
                                                     trig, p, n_edges, B, energy, edge_zz);
  else
    dev::energy_kernel<double><<<grid, 128, 0, s>>>((const double*)data, scal_off, scal_begin, net_first, counts,
                                                    trig, p, n_edges, B, energy, edge_zz);
  return cudaGetLastError();
}

cudaError_t launch_gradient(int dtype, const DevLeafFactor* lf, int32_t n_lf, const int32_t* leaf_first,
                            int32_t n_edges, int64_t lbar_shift, const double* trig, const int32_t* counts, int32_t p,
                            int32_t B, const void* data, double* part, double* dz, double* grad, cudaStream_t s) {
  const int64_t n1 = (int64_t)n_lf * B;
  if (n1 > 0) {
    if (dtype == QT_C64)
      dev::leafgrad_kernel<float><<<(int)((n1 * 32 + 127) / 128), 128, 0, s>>>(
          lf, n_lf, lbar_shift, trig, counts, p, B, (const float*)data, (double2*)part);
    else if (dtype == QT_C64X2)
      dev::leafgrad_kernel<dev::ff><<<(int)((n1 * 32 + 127) / 128), 128, 0, s>>>(
          lf, n_lf, lbar_shift, trig, counts, p, B, (const dev::ff*)data, (double2*)part);
    else
      dev::leafgrad_kernel<double><<<(int)((n1 * 32 + 127) / 128), 128, 0, s>>>(
          lf, n_lf, lbar_shift, trig, counts, p, B, (const double*)data, (double2*)part);
  }
  const int64_t n2 = (int64_t)n_edges * B * ((2 * p + dev::kEdgeGradAngles - 1) / dev::kEdgeGradAngles) * 32;
  dev::edgegrad_kernel<<<(int)((n2 + 127) / 128), 128, 0, s>>>(lf, leaf_first, n_edges, p, B, (const double2*)part, dz);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dev::gradreduce_kernel<<<(B * 2 * p + 127) / 128, 128, 0, s>>>(dz, n_edges, p, B, grad);
  return cudaGetLastError();
}

}  // namespace qt
