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
// stand-in object), so the device address is looked up with
// cudaGetSymbolAddress, with the device current, on the first call made in a
// CUDA context (the device's primary context, or a new one after the context
// was reset).  That first call should therefore come before any stream
// capture on that device.
//
// All calls share the one array and it keeps the previous call's contents.
// The library records, per device and context, which plan's descriptors the
// array holds: a call with another plan uploads its own descriptors (and
// waits for its stream, since the host copies must be complete before it
// returns), a call with the same plan does not.  Every call clears the
// control words and dependency counters that must start at zero on its
// stream; everything else is written before it is read.  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// the array and give wrong results.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "engine.h"

namespace qt {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Per device: the context the address was looked up in (0: none or unknown),
// the array's device address there and the plan whose descriptors it holds.
struct StaticSlot {
  unsigned long long ctx_id = 0;
  void* ptr = nullptr;
  uint64_t plan_uid = 0;
};
static std::mutex g_static_mutex;
static StaticSlot g_static_slot[kMaxDevices];

// Id of the current CUDA context (unique for the process lifetime), from the
// driver's cuCtxGetCurrent / cuCtxGetId through the runtime's entry-point
// lookup (the library links no driver library).  0 when no context is
// current yet or the lookup is not available.
static unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)f;
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context, and whether
// the array already holds plan `uid`'s descriptors there.  Caller holds the
// mutex.
static qt_status static_scratch_slot(StaticSlot** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(QT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(QT_EINVAL, "device index above the static-scratch table");
  StaticSlot& slot = g_static_slot[dev];
  const unsigned long long ctx = current_context_id();
  if (ctx == 0 || ctx != slot.ctx_id || !slot.ptr) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(QT_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    slot.ptr = ptr;
    slot.ctx_id = current_context_id();  // the lookup made the context current if it was not
    slot.plan_uid = 0;                   // a new context: the array holds no plan yet
  }
  *out = &slot;
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
  std::lock_guard<std::mutex> lock(g_static_mutex);
  StaticSlot* slot = nullptr;
  qt_status st = static_scratch_slot(&slot);
  if (st != QT_OK) return st;
  // Another plan (or none) in the array, or a context whose identity is not
  // known: upload this plan's descriptors again.
  if (slot->ctx_id == 0 || slot->plan_uid != P.uid) P.bound_ws = nullptr;
  slot->plan_uid = 0;  // unknown until the call has gone through
  st = run_plan(&P, gamma, beta, energy, edge_zz, nullptr, slot->ptr, kStaticScratchBytes, stream);
  if (st == QT_OK) slot->plan_uid = P.uid;
  return st;
}

extern "C" size_t qt_static_scratch_bytes(void) { return qt::kStaticScratchBytes; }
