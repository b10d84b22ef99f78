// Global kernels of the forward (energy) path.  See kernels.cuh for the
// bucket product-sum device function and the data layout.
#include "kernels.cuh"
#include "kernels_api.h"

namespace qt {
namespace dev {

// Angle table: trig[(b * p + q) * 4 + {0,1,2,3}] = cos g, sin g, cos b, sin b.
__global__ void trig_kernel(const double* __restrict__ gamma, const double* __restrict__ beta, int32_t p,
                            int32_t B, double* __restrict__ trig) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * p) return;
  double sg, cg, sb, cb;
  sincos(gamma[i], &sg, &cg);
  sincos(beta[i], &sb, &cb);
  trig[4 * i + 0] = cg;
  trig[4 * i + 1] = sg;
  trig[4 * i + 2] = cb;
  trig[4 * i + 3] = sb;
}

// Value of one leaf at its index bits (§Diagonal gate simplification and
// eq. (zz_gates_circ) in this library's convention):
//   |+>  : 1/sqrt(2)
//   ZZ_q : exp(-i gamma_q z_a z_b) = cos g - i s sin g, s = +1 if bits equal else -1
//   MIX_q: cos b if new == old else -i sin b
//   OBS  : +1 for bit 0, -1 for bit 1
// conj = 1 takes the complex conjugate (bra half of the network).
template <class Real>
__device__ __forceinline__ typename Cx<Real>::T leaf_value(uint32_t w, uint32_t z, const double* tr) {
  const uint32_t kind = w & 3u, conj = (w >> 2) & 1u;
  const uint32_t b0 = (z >> ((w >> 5) & 31u)) & 1u;
  const uint32_t b1 = (z >> ((w >> 10) & 31u)) & 1u;
  typename Cx<Real>::T v;
  if (kind == 0u) {
    v.x = (Real)0.70710678118654752440;
    v.y = 0;
  } else if (kind == 1u) {
    const Real s = (b0 == b1) ? (Real)1 : (Real)-1;
    v.x = (Real)tr[0];
    v.y = -s * (Real)tr[1];
  } else if (kind == 2u) {
    if (b0 == b1) {
      v.x = (Real)tr[2];
      v.y = 0;
    } else {
      v.x = 0;
      v.y = -(Real)tr[3];
    }
  } else {
    v.x = b0 ? (Real)-1 : (Real)1;
    v.y = 0;
  }
  if (conj) v.y = -v.y;
  return v;
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
      C acc;
      acc.x = 1;
      acc.y = 0;
      for (int32_t l = 0; l < F.n_leaves; ++l) {
        const uint32_t w = F.leaf[l];
        const int32_t layer = (int32_t)(w >> 16);
        const double* tr = trig + ((int64_t)b * p + (layer > 0 ? layer - 1 : 0)) * 4;
        acc = cmul<Real>(acc, leaf_value<Real>(w, z, tr));
      }
      reinterpret_cast<C*>(data)[F.off + idx] = acc;
    }
  }
}

// One launch per bucket (the plain per-bucket path).
template <class Real, int VB, bool PAIR>
__global__ void __launch_bounds__(256) bucket_kernel(const DevBucket d, Real* __restrict__ data,
                                                     int32_t B, int32_t bshift, int64_t n_items) {
  bucket_range<Real, VB, PAIR, false>(d, data, B, bshift, 0, n_items,
                                      (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                      (int64_t)gridDim.x * blockDim.x);
}

__device__ __forceinline__ int32_t ld_acquire(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Persistent queue: CTAs take tasks (bucket tile) in queue order.  A task
// first waits until its bucket's predecessor (the previous bucket of the
// same edge chain) has all its tiles done.  Every predecessor comes earlier
// in the queue, so it was taken by a CTA that is running, and the wait ends.
// The wait is bounded: after `spin_limit` polls it records QT_ETIMEOUT and
// every CTA stops taking tasks.
template <class Real, int VB, bool PAIR>
__global__ void __launch_bounds__(256) persistent_kernel(const DevBucket* __restrict__ buckets,
                                                         const DevTask* __restrict__ tasks, int32_t n_tasks,
                                                         DevCtrl* ctrl, int32_t* done, Real* __restrict__ data,
                                                         int32_t B, int32_t bshift, int64_t tile_items,
                                                         int32_t spin_limit) {
  __shared__ DevBucket sd;
  __shared__ int32_t s_task;
  for (;;) {
    if (threadIdx.x == 0) {
      int32_t t = n_tasks;
      if (*((volatile int32_t*)&ctrl->status) == 0) t = atomicAdd(&ctrl->head, 1);
      if (t < n_tasks) {
        const int32_t dep = buckets[tasks[t].bucket].dep;
        if (dep >= 0) {
          const int32_t need = buckets[dep].ntask;
          int32_t polls = 0;
          while (ld_acquire(done + dep) < need) {
            if (++polls > spin_limit) {
              atomicCAS(&ctrl->status, 0, (int32_t)QT_ETIMEOUT);
              ctrl->spins = dep;
              t = n_tasks;
              break;
            }
            __nanosleep(64);
          }
        }
      }
      s_task = t;
    }
    __syncthreads();
    const int32_t t = s_task;
    if (t >= n_tasks) break;
    const DevTask task = tasks[t];
    {
      const int32_t* src = reinterpret_cast<const int32_t*>(buckets + task.bucket);
      int32_t* dst = reinterpret_cast<int32_t*>(&sd);
      for (int32_t i = threadIdx.x; i < (int32_t)(sizeof(DevBucket) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int64_t n_items = PAIR ? sd.n_rows : sd.n_rows * (B / VB);
    const int64_t e0 = (int64_t)task.tile * tile_items;
    const int64_t e1 = e0 + tile_items < n_items ? e0 + tile_items : n_items;
    bucket_range<Real, VB, PAIR, true>(sd, data, B, bshift, e0, e1, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + task.bucket, 1);
    }
  }
}

// Final step (§QAOA algorithm, E = sum_k E_k): per angle set, the value of
// each edge network is the product of its scalar bucket results, taken in
// FP64, and E = sum_e (1 - Re <Z_j Z_k>_e) / 2 in a fixed order.
template <class Real>
__global__ void energy_kernel(const Real* __restrict__ data, const int64_t* __restrict__ scal_off,
                              const int32_t* __restrict__ scal_begin, int32_t n_edges, int32_t B,
                              double* __restrict__ energy, double* __restrict__ edge_zz) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double E = 0.0;
  for (int32_t e = 0; e < n_edges; ++e) {
    double zr = 1.0, zi = 0.0;
    for (int32_t s = scal_begin[e]; s < scal_begin[e + 1]; ++s) {
      const int64_t o = scal_off[s] + b;
      const double vr = (double)data[2 * o], vi = (double)data[2 * o + 1];
      const double nr = zr * vr - zi * vi;
      zi = zr * vi + zi * vr;
      zr = nr;
    }
    if (edge_zz) {
      edge_zz[((int64_t)e * B + b) * 2 + 0] = zr;
      edge_zz[((int64_t)e * B + b) * 2 + 1] = zi;
    }
    E += 0.5 * (1.0 - zr);
  }
  if (energy) energy[b] = E;
}

}  // namespace dev

// ------------------------------------------------------------- launchers ---

static int items_shift(int32_t B, int vb) {
  const int32_t per = B / vb;
  if (per <= 0 || (per & (per - 1))) return -1;
  return __builtin_ctz((unsigned)per);
}

cudaError_t launch_trig(const double* gamma, const double* beta, int32_t p, int32_t B, double* trig,
                        cudaStream_t s) {
  const int32_t n = B * p;
  dev::trig_kernel<<<(n + 127) / 128, 128, 0, s>>>(gamma, beta, p, B, trig);
  return cudaGetLastError();
}

cudaError_t launch_leaf_factors(int dtype, const DevLeafFactor* lf, int32_t n_lf, const double* trig,
                                int32_t p, int32_t B, void* data, cudaStream_t s) {
  if (n_lf == 0) return cudaSuccess;
  const int32_t grid = n_lf < 152 * 16 ? n_lf : 152 * 16;
  if (dtype == QT_C64)
    dev::leaf_factor_kernel<float><<<grid, 128, 0, s>>>(lf, n_lf, trig, p, B, (float*)data);
  else
    dev::leaf_factor_kernel<double><<<grid, 128, 0, s>>>(lf, n_lf, trig, p, B, (double*)data);
  return cudaGetLastError();
}

int vector_width(int dtype, int32_t B) { return (dtype == QT_C64 && B > 1 && B % 2 == 0) ? 2 : 1; }

cudaError_t launch_bucket(int dtype, const DevBucket& d, int32_t B, void* data, int32_t max_blocks,
                          cudaStream_t s) {
  const int vb = vector_width(dtype, B);
  const bool pair = (B == 1);
  const int64_t n_items = pair ? d.n_rows : d.n_rows * (B / vb);
  const int bshift = items_shift(B, vb);
  int64_t blocks = (n_items + 255) / 256;
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  if (dtype == QT_C64) {
    if (pair)
      dev::bucket_kernel<float, 1, true><<<(int)blocks, 256, 0, s>>>(d, (float*)data, B, bshift, n_items);
    else if (vb == 2)
      dev::bucket_kernel<float, 2, false><<<(int)blocks, 256, 0, s>>>(d, (float*)data, B, bshift, n_items);
    else
      dev::bucket_kernel<float, 1, false><<<(int)blocks, 256, 0, s>>>(d, (float*)data, B, bshift, n_items);
  } else {
    if (pair)
      dev::bucket_kernel<double, 1, true><<<(int)blocks, 256, 0, s>>>(d, (double*)data, B, bshift, n_items);
    else
      dev::bucket_kernel<double, 1, false><<<(int)blocks, 256, 0, s>>>(d, (double*)data, B, bshift, n_items);
  }
  return cudaGetLastError();
}

cudaError_t launch_persistent(int dtype, const DevBucket* buckets, const DevTask* tasks, int32_t n_tasks,
                              DevCtrl* ctrl, int32_t* done, int32_t B, void* data, int64_t tile_items,
                              int32_t grid, int32_t spin_limit, cudaStream_t s) {
  const int vb = vector_width(dtype, B);
  const bool pair = (B == 1);
  const int bshift = items_shift(B, vb);
  if (dtype == QT_C64) {
    if (pair)
      dev::persistent_kernel<float, 1, true><<<grid, 256, 0, s>>>(buckets, tasks, n_tasks, ctrl, done,
                                                                  (float*)data, B, bshift, tile_items, spin_limit);
    else if (vb == 2)
      dev::persistent_kernel<float, 2, false><<<grid, 256, 0, s>>>(buckets, tasks, n_tasks, ctrl, done,
                                                                   (float*)data, B, bshift, tile_items, spin_limit);
    else
      dev::persistent_kernel<float, 1, false><<<grid, 256, 0, s>>>(buckets, tasks, n_tasks, ctrl, done,
                                                                   (float*)data, B, bshift, tile_items, spin_limit);
  } else {
    if (pair)
      dev::persistent_kernel<double, 1, true><<<grid, 256, 0, s>>>(buckets, tasks, n_tasks, ctrl, done,
                                                                   (double*)data, B, bshift, tile_items, spin_limit);
    else
      dev::persistent_kernel<double, 1, false><<<grid, 256, 0, s>>>(buckets, tasks, n_tasks, ctrl, done,
                                                                    (double*)data, B, bshift, tile_items, spin_limit);
  }
  return cudaGetLastError();
}

cudaError_t persistent_occupancy(int dtype, int32_t B, int* blocks_per_sm) {
  const int vb = vector_width(dtype, B);
  const bool pair = (B == 1);
  const void* fn;
  if (dtype == QT_C64)
    fn = pair ? (const void*)dev::persistent_kernel<float, 1, true>
              : (vb == 2 ? (const void*)dev::persistent_kernel<float, 2, false>
                         : (const void*)dev::persistent_kernel<float, 1, false>);
  else
    fn = pair ? (const void*)dev::persistent_kernel<double, 1, true>
              : (const void*)dev::persistent_kernel<double, 1, false>;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, 256, 0);
}

cudaError_t launch_energy(int dtype, const void* data, const int64_t* scal_off, const int32_t* scal_begin,
                          int32_t n_edges, int32_t B, double* energy, double* edge_zz, cudaStream_t s) {
  const int32_t grid = (B + 127) / 128;
  if (dtype == QT_C64)
    dev::energy_kernel<float><<<grid, 128, 0, s>>>((const float*)data, scal_off, scal_begin, n_edges, B,
                                                   energy, edge_zz);
  else
    dev::energy_kernel<double><<<grid, 128, 0, s>>>((const double*)data, scal_off, scal_begin, n_edges, B,
                                                    energy, edge_zz);
  return cudaGetLastError();
}

}  // namespace qt
