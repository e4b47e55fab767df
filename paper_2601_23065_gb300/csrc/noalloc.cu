// Allocation-free variant of the path-traced render.
//
// Some callers cannot allocate device memory themselves: a plugin hosted by
// an application whose memory manager owns the whole device heap, or a
// latency-critical loop that must not pay for cudaMalloc and the device-wide
// synchronisation it can imply.  For them this entry point takes its render
// workspace from one fixed scratch array compiled into the library instead of
// a caller buffer.  The array is a file-scope __device__ object: every GPU
// that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace eagpt {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB per device

// The scratch.  Host code must not pass this name to a kernel (on the host it
// is only a stand-in for the device object); its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_render_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_scratch_mu;
void* g_scratch_ptr[64] = {nullptr};
}  // namespace

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.  The address belongs to the
// device's context as it was at that first call; a device reset invalidates
// it (documented in the header).
static cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_render_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace eagpt

using namespace eagpt;

extern "C" {

size_t eagpt_render_path_traced_noalloc_max_bytes(void) { return kNoAllocScratchBytes; }

eagpt_status eagpt_render_path_traced_noalloc(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                              const eagpt_camera* cam, const eagpt_params* params, int32_t spp,
                                              int32_t max_bounces, int32_t rr_start_bounce, uint64_t seed,
                                              float* out_rgb, eagpt_stream_t stream) {
  if (!cam || cam->width <= 0 || cam->height <= 0 || spp <= 0)
    return set_error(EAGPT_ERR_INVALID_ARGUMENT, "camera size and spp must be positive");
  // smallest workspace the render accepts: one sample per pass (emitter
  // sampling needs two more ray queues)
  const int kind = params && (params->flags & EAGPT_FLAG_EMITTER_SAMPLING) ? 2 : 1;
  const size_t need = eagpt_render_workspace_min_bytes(cam, spp, kind);
  if (need > kNoAllocScratchBytes) {
    char buf[256];
    std::snprintf(buf, sizeof(buf),
                  "render needs at least %zu bytes of scratch for %d x %d pixels; the allocation-free entry point "
                  "has %zu (use eagpt_render_path_traced with a caller workspace)",
                  need, cam->width, cam->height, kNoAllocScratchBytes);
    return set_error(EAGPT_ERR_INVALID_ARGUMENT, buf);
  }
  void* ws = nullptr;
  const cudaError_t e = scratch_address(&ws);
  if (e != cudaSuccess) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "scratch lookup (cudaGetSymbolAddress): %s", cudaGetErrorString(e));
    return set_error(EAGPT_ERR_CUDA, buf);
  }
  // The render zeroes its own queue counters at every pass and starts its
  // per-pixel sums from the first pass, so nothing left in the scratch by an
  // earlier call is read.
  return render_entry(scene, bvh, cam, params, 1, spp, max_bounces, rr_start_bounce, seed, out_rgb, nullptr, nullptr,
                      nullptr, ws, kNoAllocScratchBytes, stream);
}

}  // extern "C"
