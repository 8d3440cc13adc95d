// stiffness_apply_noalloc: the FP64 stiffness apply with its cell-local
// scratch in a fixed device array of this library instead of memory owned by
// the context, for callers that must not allocate device memory at the time
// of the call.
#include <mutex>
#include <string>

#include "internal.h"
#include "kernels.h"

namespace fdm {
namespace {

// One cell-local FP64 result per (cell, node): ncell * (p+1)^3 doubles at
// most.  16 MiB, reserved on every GPU that loads the library until exit.
constexpr int64_t kNoAllocScratchElems = int64_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on device dev, looked up once per
// device with that device current (the host-side symbol is only a stand-in,
// never a device pointer).  The caller's current device is restored.
cudaError_t scratch_on_device(int dev, double **out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return e;
    if (cur != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != dev) {
      const cudaError_t e2 = cudaSetDevice(cur);
      if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace fdm

extern "C" int stiffness_apply_noalloc(fdm_ctx *c, const double *u, double *y, void *stream) {
  using namespace fdm;
  if (!c || !u || !y) return FDM_EINVAL;
  try {
    const OpArgs a = ctx_op_args64(c);
    const int64_t need = (int64_t)a.g.ncell * a.g.n * a.g.n * a.g.n;
    if (need > kNoAllocScratchElems)
      fail(FDM_EINVAL, "stiffness_apply_noalloc: ncell*(p+1)^3 = " + std::to_string(need) +
                           " exceeds the fixed scratch of " + std::to_string(kNoAllocScratchElems) + " doubles");
    const int dev = ctx_device(c);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != dev)
      fail(FDM_EINVAL, "stiffness_apply_noalloc: the context's device (" + std::to_string(dev) +
                           ") must be the current device");
    double *scratch = nullptr;
    cudaError_t e = scratch_on_device(dev, &scratch);
    if (e != cudaSuccess)
      fail(FDM_ECUDA, std::string("stiffness_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    // both stiffness paths of launch_operator (box cells, curved cells) are
    // one cell kernel that writes the whole scratch, then one node gather
    launch_operator<double, double, double>(a, false, u, y, scratch, (cudaStream_t)stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) fail(FDM_ECUDA, std::string("stiffness_apply_noalloc: ") + cudaGetErrorString(e));
    ctx_count_launches(c, 2);
  } catch (const Error &err) {
    return ctx_fail(c, err.code, err.msg);
  }
  return FDM_OK;
}
