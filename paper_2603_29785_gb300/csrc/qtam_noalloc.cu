// qtam_forward_noalloc: the forward transform with its scratch memory in a
// fixed, library-owned device array instead of a caller-supplied workspace.
//
// Who needs it: callers that cannot allocate device memory when they run
// the transform -- code inside a real-time loop or a host callback where a
// cudaMalloc would stall, plug-ins whose host application owns every device
// allocation, or a pipeline that has handed its whole memory budget to a pool
// it does not control.  They pass the input and output buffers only; the
// long-FFT scratch lives in g_qtam_noalloc_scratch below.
//
// Limits and sharing:
//  - the array holds QTAM_NOALLOC_SCRATCH_BYTES (32 MiB); every GPU that
//    loads the library keeps it reserved until the process exits;
//  - a call whose batch needs more scratch than that (qtam_workspace_size)
//    is rejected with QTAM_ERR_WORKSPACE before anything is launched;
//  - all calls on a device share the one array, and the array keeps the last
//    call's contents.  Nothing in it needs to start at zero: every scratch
//    element is written by the forward path before it is read.  Two calls
//    whose kernels overlap on the GPU (different streams, no ordering between
//    them) race on the array and give wrong results; order them on one stream
//    or with events.
//  - the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture begins.
#include <mutex>
#include <string>

#include "../../include/qtam.h"
#include "qtam_internal.h"

#define QTAM_NOALLOC_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_qtam_noalloc_scratch[QTAM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (looked up once per device).
qtam_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) {
    qtam::set_last_error("qtam_forward_noalloc: device index out of range");
    return QTAM_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaError_t e = cudaSetDevice(device);
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_qtam_noalloc_scratch);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess || !p) {
      qtam::set_last_error(std::string("qtam_forward_noalloc: cudaGetSymbolAddress failed: ") +
                           cudaGetErrorString(e));
      return QTAM_ERR_CUDA;
    }
    g_noalloc_addr[device] = p;
  }
  *out = g_noalloc_addr[device];
  return QTAM_OK;
}

}  // namespace

extern "C" qtam_status qtam_forward_noalloc(qtam_plan_t plan, const void* x, int64_t batch, void* y, void* stream) {
  if (!plan) {
    qtam::set_last_error("qtam_forward_noalloc: plan is NULL");
    return QTAM_ERR_INVALID_ARG;
  }
  size_t need = 0;
  qtam_status s = qtam_workspace_size(plan, batch, &need);
  if (s != QTAM_OK) return s;
  if (need > QTAM_NOALLOC_SCRATCH_BYTES) {
    qtam::set_last_error("qtam_forward_noalloc: batch needs " + std::to_string(need) +
                         " bytes of scratch, more than the fixed " +
                         std::to_string((size_t)QTAM_NOALLOC_SCRATCH_BYTES) +
                         "; use a smaller batch or qtam_forward with a workspace");
    return QTAM_ERR_WORKSPACE;
  }
  const int device = qtam::plan_device(plan);
  if (device < 0) {
    qtam::set_last_error("qtam_forward_noalloc: host-only plan (device = -1) cannot run transforms");
    return QTAM_ERR_NO_DEVICE;
  }
  if (batch == 0) return QTAM_OK;
  void* scratch = nullptr;
  if ((s = noalloc_scratch(device, &scratch)) != QTAM_OK) return s;
  return qtam_forward(plan, x, batch, y, scratch, QTAM_NOALLOC_SCRATCH_BYTES, stream);
}
