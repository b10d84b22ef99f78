// Allocation-free evaluation of an energy plan.
//
// Some callers cannot hand this library a device workspace: a host program
// that runs under a fixed device-memory budget reserved at start-up, or a
// plug-in whose host application owns every device allocation and offers no
// allocator to call, may not call cudaMalloc (or any allocating library,
// PyTorch's caching allocator included) while it serves requests.  For them
// qt_plan_energy_static evaluates a plan with its scratch space -- bucket
// descriptors, task queue, dependency counters, leaf factors and the
// intermediate-tensor arenas -- in a file-scope device array of fixed size
// instead of a caller workspace.  The caller still passes its inputs (angles)
// and outputs (energies, optional per-edge values) as device pointers.
//
// The array lives in the library's device image: every GPU that loads the
// library holds kStaticScratchBytes of it until the process exits.  Host code
// cannot use the array's name as a device address (on the host it names a
// stand-in object), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device.  That first call should therefore come before any stream
// capture on that device.
//
// All calls share the one array and it keeps the previous call's contents,
// so each call re-uploads its plan's descriptors and clears the control words
// and dependency counters that must start at zero; everything else is written
// before it is read.  Calls whose work overlaps on the GPU (different streams,
// or different host threads) race on the array and give wrong results.
#include <cuda_runtime.h>

#include <mutex>

#include "engine.h"

namespace qt {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mutex;
static void* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
static qt_status static_scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(QT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(QT_EINVAL, "device index above the static-scratch table");
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(QT_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_static_ptr[dev] = ptr;
  }
  *out = g_static_ptr[dev];
  return QT_OK;
}

}  // namespace qt

extern "C" qt_status qt_plan_energy_static(qt_plan* plan, const double* gamma, const double* beta,
                                           double* energy, double* edge_zz, void* stream) {
  using namespace qt;
  if (!plan) return fail(QT_EINVAL, "plan is NULL");
  Plan& P = plan->P;
  if (P.amplitude) return fail(QT_ESTATE, "amplitude plan: use qt_plan_amplitudes");
  if (P.ws.total > kStaticScratchBytes)
    return fail(QT_ENOMEM, "plan needs " + std::to_string(P.ws.total) + " bytes of scratch; the static scratch holds " +
                               std::to_string(kStaticScratchBytes) + " bytes (use qt_plan_energy with a workspace)");
  void* ws = nullptr;
  qt_status st = static_scratch_address(&ws);
  if (st != QT_OK) return st;
  P.bound_ws = nullptr;  // another plan may have used the array since: upload again
  return run_plan(&P, gamma, beta, energy, edge_zz, nullptr, ws, kStaticScratchBytes, stream);
}

extern "C" size_t qt_static_scratch_bytes(void) { return qt::kStaticScratchBytes; }
