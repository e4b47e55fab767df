// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace eagpt {

// bvh.cu
cudaError_t launch_build(const eagpt_scene& sc, const Consts& C, char* base, const BvhLayout& L, cudaStream_t st,
                         int* launches);
int launch_refit(char* base, const BvhLayout& L, cudaStream_t st);
void launch_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* hist, int64_t n,
                       cudaStream_t st);
// bvh_tree.cu
cudaError_t launch_tree(const uint32_t* sorted_keys, char* base, const BvhLayout& L, cudaStream_t st);
cudaError_t launch_records_update(const eagpt_scene& sc, const Consts& C, char* base, const BvhLayout& L,
                                  cudaStream_t st);
// the emitter table (emitter sampling) from the scene's current radiance and emission
cudaError_t launch_emitter_table(const eagpt_scene& sc, const Consts& C, char* base, const BvhLayout& L,
                                 cudaStream_t st);

// render.cu
struct RenderArgs {
  BvhView bvh;
  Consts C;
  eagpt_camera cam;
  int kind;         // 0 single bounce, 1 path tracing, 2 single bounce with incident radiance (out_li)
  int spp, max_bounces, rr_start;
  int s_first;      // samples s_first .. s_first + spp - 1 of each pixel are rendered
  uint64_t seed;
  float* out_rgb;
  float* out_aux;
  float* out_samples;
  float* out_li;
  int64_t* out_stats;
  void* ws;
  size_t ws_bytes;
  float4* sb_cache;  // single bounce: per-sample secondary (R, T), sample-major, or NULL
  // level of detail (path tracing without emitter sampling): bounce segments
  // k >= lod_from trace bvh_lod; lod_from = 0 (the default) turns it off
  BvhView bvh_lod;
  int lod_from;
};

struct RenderLayout {
  size_t summary, prim, acc, slots, q0, q1, counters, e0, e1, total;
  int64_t npix, batch_paths;
  int batch_spp;
};

// mis: path tracing with emitter sampling (side queues of RayExt)
RenderLayout render_layout(int64_t npix, int spp, int batch_spp, bool mis = false);
int choose_batch_spp(int64_t npix, int spp, size_t ws_bytes, bool mis = false);
cudaError_t launch_render(const RenderArgs& a, cudaStream_t st, int* launches);
cudaError_t render_summary(const void* ws, int64_t* out, cudaStream_t st);
cudaError_t launch_trace_rays(const BvhView& bvh, const Consts& C, int mode, const float* rays, int64_t n_rays,
                              float* out_rec, int32_t* out_hits, int max_hits, int32_t* out_nhits, cudaStream_t st);

cudaError_t launch_primary_records(const BvhView& bvh, const Consts& C, const eagpt_camera& cam, int mode,
                                   int64_t npix, void* prim, cudaStream_t st);

cudaError_t launch_radiance(const BvhView& bvh, const Consts& C, const eagpt_camera& cam, float* out_rgb, float* aux,
                            cudaStream_t st);

// backward.cu
cudaError_t launch_radiance_backward(const BvhView& bvh, const Consts& C, const eagpt_camera& cam,
                                     const eagpt_scene& sc, const eagpt_scene_grad& gr, const float* dL,
                                     cudaStream_t st);
size_t backward_workspace_bytes(int64_t npix, int spp, int batch);
int backward_choose_batch(int64_t npix, int spp, size_t ws_bytes);
cudaError_t launch_backward(const BvhView& bvh, const Consts& C, const eagpt_camera& cam, const eagpt_scene& sc,
                            const eagpt_scene_grad& gr, int spp, uint64_t seed, const float* dL, void* ws,
                            size_t ws_bytes, cudaStream_t st, const float4* sb_cache = nullptr);

// optim.cu
int64_t pq_partials(int64_t n);
cudaError_t launch_pq_l1(const float* pred, const float* target, int64_t n, float peak, float lambda_c, float* grad,
                         double* out_loss, double* partials, cudaStream_t st);
cudaError_t launch_shade_adjoint(const BvhView& bvh, const Consts& C, const eagpt_camera& cam, const float* dL,
                                 const float* li, float* grad, cudaStream_t st);
cudaError_t launch_adam(float* p, float* g, float* m, float* v, int64_t n, const eagpt_adam& cfg, int64_t step,
                        int zero_grad, float* mirror, const uint32_t* inv_idx, int field, cudaStream_t st);

// device error words of each translation unit (read and cleared)
uint32_t take_errors_bvh();
uint32_t take_errors_render();
uint32_t take_errors_backward();
uint32_t take_errors_tree();
uint32_t take_errors_edit();
uint32_t take_errors_serve();
uint32_t take_errors_optim();

// lod.cu: merged surfels of the level of detail (group keys, sort, merge);
// reads the group count back to *out_count (synchronises the stream)
size_t lod_workspace_bytes(int64_t n);
cudaError_t launch_lod(const eagpt_scene& sc, const float origin[3], float inv_h, float tau_E,
                       const eagpt_scene_mut& out, uint64_t* out_keys, void* ws, int64_t* out_count,
                       cudaStream_t st);

// edit.cu
cudaError_t launch_select(const eagpt_scene& sc, int shape, const float* v, int32_t* out, int64_t capacity,
                          int64_t* out_count, uint32_t* scratch_blocks, cudaStream_t st);
size_t select_scratch_bytes(int64_t n);
cudaError_t launch_edit(const eagpt_scene_mut& sc, const eagpt_edit& e, cudaStream_t st);
size_t delete_scratch_bytes(int64_t n);
cudaError_t launch_delete(const eagpt_scene_mut& sc, const int32_t* idx, int64_t count, void* scratch,
                          int64_t* out_n, cudaStream_t st);

// capi.cu: argument checks + render launch shared by the render entry points;
// set_error records the thread-local message of eagpt_last_error()
eagpt_status render_entry(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                          const eagpt_params* params, int kind, int32_t spp, int32_t max_bounces, int32_t rr_start,
                          uint64_t seed, float* out_rgb, float* out_aux, float* out_samples, int64_t* out_stats,
                          void* ws, size_t ws_bytes, eagpt_stream_t stream);
eagpt_status set_error(eagpt_status s, const char* msg);
BvhView bvh_view(const eagpt_bvh& b);
eagpt_status apply_edit_core(eagpt_scene_mut* scene, eagpt_bvh* bvh, const eagpt_params* params,
                             const eagpt_edit* edit, float rebuild_ratio, int32_t* out_rebuilt, cudaStream_t st);

// number of SMs of the current device (cached per device)
int device_sms();
// blocks of a persistent launch of a kBlock-thread kernel on the current
// device (resident blocks per SM x SMs; cached per kernel and device)
int persistent_grid(const void* kernel);

// profiler.cu: every kernel launch goes through a LaunchScope (counts the
// launch; with profiling on, records CUDA events around it on its stream)
class LaunchScope {
 public:
  LaunchScope(cudaStream_t st, const char* name);
  ~LaunchScope();
  LaunchScope(const LaunchScope&) = delete;
  LaunchScope& operator=(const LaunchScope&) = delete;

 private:
  cudaStream_t st_;
  const char* name_;
  cudaEvent_t a_;
};
int64_t launch_count();
void profile_begin();
int profile_end(eagpt_kernel_time* out, int capacity);

#define EAGPT_LAUNCH(st, name, ...)           \
  do {                                        \
    ::eagpt::LaunchScope _scope((st), name); \
    __VA_ARGS__;                              \
  } while (0)

}  // namespace eagpt
