// Allocation-free plenoptic forward projection.
//
// The regular plenoptic forward keeps its array-plane intermediate in a
// buffer the plan allocated with cudaMalloc.  Some callers cannot allocate
// device memory at the point where they project: code running inside a
// memory-pool-managed framework that forbids raw cudaMalloc, real-time loops
// where an allocation (and the implicit device synchronisation it can cause)
// is not allowed, or callers holding a plan built elsewhere whose memory
// budget is fixed.  For them, lt_forward_camera_noalloc stages the
// intermediate in a fixed static device array instead and allocates nothing
// (the per-lenslet sub-image buffer it also uses was allocated with the plan).
//
// Limits and sharing rules (also in include/lt.h):
//   * the array holds kNoAllocScratchFloats floats (16 MiB); every GPU that
//     loads this library reserves it (once the module is loaded) until exit;
//   * all calls share it and it keeps the last call's contents.  Stage one
//     overwrites every element it later reads, so nothing needs clearing, but
//     two calls that overlap in time on the GPU (different streams, or
//     different plans on one device) race on it;
//   * the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before any stream capture.  Under CUDA's lazy module loading (the
//     default since CUDA 12.2) that lookup is also what loads this file's
//     module on the device, so the 16 MiB are reserved, and the call may
//     synchronise, at that first call rather than when the library loads;
//     later calls reserve nothing.
#include <mutex>

#include "lt.h"
#include "lt_host.h"

namespace {

constexpr long long kNoAllocScratchFloats = 4LL * 1024 * 1024;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of the static array on the current device (set up once per
// device).  In host code the symbol itself is only a host-side stand-in.
lt_status scratch_on_current_device(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lt::cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return lt::set_error(LT_EUNSUPPORTED, "device ordinal %d above the supported %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return lt::cuda_error(e, "cudaGetSymbolAddress(static scratch)");
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LT_OK;
}

}  // namespace

extern "C" lt_status lt_forward_camera_noalloc(lt_plan* plan, int32_t cam, const float* x, float* y_cam,
                                               void* stream) {
  lt::clear_error();
  if (!plan) return lt::set_error(LT_EINVAL, "plan is NULL");
  if (cam < 0 || cam >= (int)plan->cams.size()) return lt::set_error(LT_EINVAL, "camera index %d out of range", cam);
  if (!x || !y_cam) return lt::set_error(LT_EINVAL, "NULL argument");
  lt::CameraPlan& c = plan->cams[cam];
  if (c.desc.kind != LT_CAM_PLENOPTIC)
    return lt::set_error(LT_EINVAL, "camera %d is not plenoptic (the allocation-free path stages the array plane)", cam);
  const long long need = (long long)plan->frames * c.K * c.Na;
  if (need > kNoAllocScratchFloats)
    return lt::set_error(LT_EINVAL,
                         "array plane of %lld floats (frames x cells x array pixels) exceeds the static "
                         "scratch of %lld floats; use lt_forward_camera",
                         need, kNoAllocScratchFloats);
  float* fa = nullptr;
  lt_status s = scratch_on_current_device(&fa);
  if (s != LT_OK) return s;
  const long long fa_fs = (long long)c.K * c.Na;
  cudaStream_t st = (cudaStream_t)stream;
  // the same stage-one call as lt_forward_camera (rotated cameras through the
  // plan's own rotation scratch), with the static array as its output
  s = lt::stage1_forward(plan, c, x, fa, fa_fs, st);
  if (s != LT_OK) return s;
  cudaError_t e = lt::launch_stage2_forward(fa, y_cam, c.s2, plan->frames, fa_fs, c.M, c.d_zbuf, st);
  return e == cudaSuccess ? LT_OK : lt::cuda_error(e, "allocation-free stage 2");
}
