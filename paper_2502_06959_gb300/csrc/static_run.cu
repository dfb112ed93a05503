// hsf_run_static: the amplitude run for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where
// they need amplitudes: for example code that runs while another runtime owns every
// device allocation, or a latency-critical loop where an allocation could block or
// fail.  hsf_run needs a caller-provided workspace; this entry point instead uses a
// fixed scratch array compiled into the library, so the call itself allocates
// nothing.  It hands that array to hsf_run as the workspace, so results are the same.
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes.  Every GPU that
// loads the library keeps it until the process exits.  All calls share it, and it
// keeps the last call's contents; hsf_run zeroes the accumulators it needs at the start
// of each run.  Calls that overlap on the GPU (on different streams, or from different
// host threads without ordering) race on this array: order them.
//
// Host code cannot use the array's name as a device address, so the address is looked
// up once per device with cudaGetSymbolAddress, with that device current, on the first
// call made on that device.  Make that first call before any stream capture.  The cached
// address does not survive a device reset (cudaDeviceReset, or the primary context being
// destroyed and created again): the module is then loaded anew and the array may move, so
// do not call this entry point again in the same process after such a reset.
#include <mutex>

#include "plan.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_addr[256] = {nullptr};

}  // namespace

extern "C" hsf_status hsf_run_static(hsf_plan *plan, const uint64_t *bitstrings, size_t num,
                                     uint64_t window, uint64_t path_begin, uint64_t path_end,
                                     void *out, void *stream) {
  if (!plan) return hsf::set_error(HSF_EINVAL, "hsf_run_static: NULL plan");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hsf::set_error(HSF_ECUDA, "hsf_run_static: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 256) return hsf::set_error(HSF_EINVAL, "hsf_run_static: device %d out of range", dev);
  void *ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
      void *ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess)
        return hsf::set_error(HSF_ECUDA, "hsf_run_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_static_addr[dev] = ptr;
    }
    ws = g_static_addr[dev];
  }
  size_t need = 0;
  const hsf_status ws_st = hsf_workspace_size(plan, num, window, kStaticScratchBytes, &need);
  if (ws_st != HSF_OK && ws_st != HSF_ENOMEM) return ws_st;   // a bad request, not a size limit
  if (ws_st == HSF_ENOMEM)
    return hsf::set_error(HSF_ENOMEM,
                          "hsf_run_static: this request needs more than the %zu-byte static scratch "
                          "even with the smallest path chunk; use hsf_run with a caller workspace",
                          kStaticScratchBytes);
  return hsf_run(plan, bitstrings, num, window, path_begin, path_end, out, ws, kStaticScratchBytes, stream);
}
