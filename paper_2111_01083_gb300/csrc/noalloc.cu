// pfmm_execute_static: the periodic operator without a caller workspace.
//
// Who needs it: callers that cannot allocate device memory.  A plain C host
// program that only receives device pointers from another component (and has
// no device allocator of its own), or a caller that must not issue
// cudaMalloc/cudaFree between launches on a busy stream, because those calls
// synchronise the device and would stall other work.  Such callers pass
// inputs and outputs only; the scratch memory the operator needs comes from
// a fixed array compiled into this library.
//
// How: the scratch is a file-scope __device__ array of kStaticScratchBytes
// (32 MiB).  Every GPU on which the library's module is loaded holds that
// array until the process exits.  Host code cannot use the array's name as a
// device address, so the first call on each device looks the address up
// with cudaGetSymbolAddress (with that device current) and caches it; make
// that first call before any stream capture.  The call then runs the same
// kernels as pfmm_execute, using the array as the workspace; the regions that
// must start at zero are cleared on every call, so the contents left by an
// earlier call do not matter.  All calls on a device share the one array:
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller.  Conditions the
// kernels detect (non-finite input, non-zero net charge or force, points
// outside a singly periodic strip) go to the status word inside the array, as
// they go to a workspace's status word for pfmm_execute; the caller reads and
// clears it with pfmm_get_status(plan, NULL, stream), which synchronises the
// stream.  The next call clears the word as it starts, so read it before.
#include <mutex>

#include "pfmm_impl.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

}  // namespace

namespace pfmm {

// Device address of the static scratch array on the current device (looked
// up on the first use per device and cached; see the file comment).  The
// cache assumes the device's context lives as long as the process: the
// library must not be used across cudaDeviceReset.
pfmm_status static_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(PFMM_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return set_error(PFMM_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_static_ptr[dev] = ptr;
  }
  *out = g_static_ptr[dev];
  return PFMM_OK;
}

}  // namespace pfmm

extern "C" pfmm_status pfmm_execute_static(pfmm_plan* plan, int64_t ns, const double* src, const double* q, int64_t nt,
                                           const double* trg, double* pot, double* grad, void* stream) {
  if (!plan) return pfmm::set_error(PFMM_ERR_INVALID_ARG, "NULL plan");
  size_t need = 0;
  pfmm_status s = pfmm_workspace_size(plan, &need);
  if (s != PFMM_OK) return s;
  if (need > kStaticScratchBytes)
    return pfmm::set_error(PFMM_ERR_WORKSPACE,
                           "pfmm_execute_static: this plan needs %zu bytes of scratch, the static array holds %zu "
                           "(use pfmm_execute with a caller workspace, or smaller ns_max/nt_max/nrhs)",
                           need, kStaticScratchBytes);
  void* ptr = nullptr;
  s = pfmm::static_scratch(&ptr);
  if (s != PFMM_OK) return s;
  return pfmm_execute(plan, ptr, kStaticScratchBytes, ns, src, q, nt, trg, pot, grad, stream);
}
