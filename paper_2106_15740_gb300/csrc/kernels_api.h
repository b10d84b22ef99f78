// Host-callable launchers of the kernels in kernels.cu (no kernel code here).
#pragma once

#include <cuda_runtime.h>

#include "qt_device.h"
#include "qtensor.h"

namespace qt {

int vector_width(int dtype, int32_t B);
TileGeom tile_geom(int dtype, int32_t B, int32_t lane_items);
cudaError_t launch_trig(int dtype, const double* gamma, const double* beta, int32_t p, int32_t B, double* trig,
                        cudaStream_t s);
cudaError_t launch_leaf_factors(int dtype, const DevLeafFactor* lf, int32_t n_lf, const double* trig,
                                int32_t p, int32_t B, void* data, cudaStream_t s);
cudaError_t launch_bucket(int dtype, const DevBucket& d, int32_t B, int32_t lane_items, void* data,
                          int32_t max_blocks, cudaStream_t s);
bool row_wide(int dtype, int32_t B);
// Whether the forward persistent kernel of (dtype, B) evaluates chained steps
// (chain > 0): the one-angle-set pair tiles, and the row-wide lean tiles with
// one vector chunk per row.
bool chain_fusion_ok(int dtype, int32_t B);
// chains: the plan has chained steps (a forward plan; its kernel is the STAGE 4 variant)
cudaError_t launch_persistent(int dtype, bool grad, bool chains, const DevBucket* buckets, const DevTask* tasks,
                              int32_t n_tasks, DevCtrl* ctrl, int32_t* done, int32_t B, int32_t lane_items, void* data,
                              int64_t data_elems, int32_t grid, int32_t spin_limit, const DevDep* deps,
                              unsigned long long* trace, cudaStream_t s);
cudaError_t persistent_occupancy(int dtype, bool grad, bool chains, int32_t B, int* blocks_per_sm);
cudaError_t launch_energy(int dtype, const void* data, const int64_t* scal_off, const int32_t* scal_begin,
                          const int32_t* net_first, const int32_t* counts, const double* trig, int32_t p,
                          int32_t n_edges, int32_t B, double* energy, double* edge_zz, cudaStream_t s);

cudaError_t launch_gradient(int dtype, const DevLeafFactor* lf, int32_t n_lf, const int32_t* leaf_first,
                            int32_t n_edges, int64_t lbar_shift, const double* trig, const int32_t* counts, int32_t p,
                            int32_t B, const void* data, double* part, double* dz, double* grad, cudaStream_t s);

}  // namespace qt
