// Energy plans: all edge networks of a graph compiled into device records.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <utility>
#include <vector>

#include "qt_device.h"
#include "qt_internal.h"

struct qt_network {
  qt::Network net;
};

namespace qt {

struct WsLayout {
  size_t ctrl = 0, done = 0, buckets = 0, tasks = 0, deps = 0, leaf = 0, leaf_first = 0, scal_off = 0, scal_begin = 0,
         net_first = 0, counts = 0;
  size_t angles = 0, results = 0, trig = 0, dz = 0, gpart = 0, data = 0, total = 0;
};

// Process-wide serial number of plans (never reused, unlike their addresses).
inline uint64_t next_plan_uid() {
  static std::atomic<uint64_t> counter{0};
  return ++counter;
}

struct Plan {
  uint64_t uid = next_plan_uid();
  Graph G;
  int32_t p = 0;
  qt_plan_options opt{};
  int32_t elem_bytes = 16;
  std::vector<EdgePlan> edges;             // networks: one per edge, or 2^s per sliced edge
  std::vector<int32_t> widths;             // per planned graph edge
  std::vector<int32_t> slices;             // per planned graph edge: sliced variables s
  int32_t n_orig = 0;                      // planned graph edges
  std::vector<int32_t> net_first;          // first network of each planned edge (n_orig + 1)

  // device images (uploaded into the workspace)
  std::vector<DevBucket> buckets;          // steps of all edges (forward, then adjoint), concatenated
  std::vector<int32_t> edge_first;         // first step of each edge (n_edges + 1)
  bool has_chains = false;                 // some forward step is chained (the launch takes the STAGE 4 kernel)
  std::vector<DevLeafFactor> leaf;
  std::vector<int32_t> leaf_first;         // first leaf factor of each edge (n_edges + 1)
  int64_t lbar_shift = 0;                  // leaf-adjoint element = leaf element + lbar_shift
  int64_t lbar_elems = 0;
  std::vector<DevTask> tasks;
  std::vector<int32_t> deps;               // dependency lists of the queued steps (DevBucket dep, n_dep)
  std::vector<DevDep> dev_deps;            // the same lists as the device reads them (step, done count)
  // data elements each step touches: ranges acc_first[s] .. acc_first[s + 1] of
  // [acc_lo, acc_hi), acc_w = 1 for a write (or an accumulation)
  std::vector<int32_t> acc_first;
  std::vector<int64_t> acc_lo, acc_hi;
  std::vector<uint8_t> acc_w;
  std::vector<int64_t> scal_off;           // element offsets of scalar results
  std::vector<int32_t> scal_begin;         // CSR over edges
  std::vector<int32_t> net_counts;         // per network: ZZ and mixer leaves per layer, |+> leaves (2p + 1)
  int64_t tile_items = 0;                  // output rows per warp tile
  int32_t spin_limit = 1 << 22;            // polls of a bounded dependency wait
  int32_t n_slots = 0;
  int64_t data_elems = 0;
  WsLayout ws;

  // statistics
  double alg_bytes = 0.0, flops = 0.0;
  std::vector<double> edge_bytes;          // per planned graph edge: algorithmic bytes of its networks

  // the plan's units are bitstrings of single amplitudes, not edges
  bool amplitude = false;

  // queue trace buffer (device, 4 x uint64 per task) or null
  unsigned long long* trace = nullptr;

  // failure-detection hook: step whose uploaded tile count is made unreachable
  int32_t stall_step = -1;

  // state
  const void* bound_ws = nullptr;
  int device = -1;

  // profiling: event pairs around the contraction, one per call
  bool profile = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  size_t events_used = 0;
  ~Plan();
};

// Compile edge plans into device records and a workspace layout.
qt_status compile_plan(Plan* P);
// Evaluate with device pointers on a stream.
qt_status run_plan(Plan* P, const double* gamma, const double* beta, double* energy, double* edge_zz,
                   double* grad, void* ws, size_t ws_bytes, void* stream);
qt_status check_plan(Plan* P, void* stream);
qt_status plan_kernel_times(Plan* P, float* ms, int32_t cap, int32_t* n);

}  // namespace qt

struct qt_plan {
  qt::Plan P;
};
