// extern "C" entry points: argument checks on the host, then kernel launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "common.cuh"
#include "internal.h"

using namespace eagpt;

namespace {

thread_local std::string g_msg;

eagpt_status fail(eagpt_status s, const char* fmt, const char* a = nullptr, long long b = 0) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), fmt, a ? a : "", b);
  g_msg = buf;
  return s;
}

eagpt_status cuda_fail(cudaError_t e, const char* where) {
  g_msg = std::string(where) + ": " + cudaGetErrorString(e);
  return EAGPT_ERR_CUDA;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

eagpt_status check_params(const eagpt_params* p) {
  if (!p) return fail(EAGPT_ERR_INVALID_ARGUMENT, "params is NULL%s");
  if (!(p->T_min > 0.f && p->T_min < 1.f)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "T_min must be in (0, 1)%s");
  if (!(p->alpha_max > 0.f && p->alpha_max < 1.f))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "alpha_max must be in (0, 1)%s");
  if (!(p->alpha_min >= 0.f && p->alpha_min <= p->alpha_max))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "alpha_min must be in [0, alpha_max]%s");
  if (!(p->support_sigma > 0.f && std::isfinite(p->support_sigma)))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "support_sigma must be positive%s");
  if (!(p->bounce_offset >= 0.f && std::isfinite(p->bounce_offset)))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "bounce_offset must be >= 0%s");
  if (!std::isfinite(p->tau_E)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "tau_E must be finite%s");
  if (p->flags & ~(int32_t)EAGPT_FLAG_EMITTER_SAMPLING)
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "params.flags has unknown bits%s");
  return EAGPT_OK;
}

eagpt_status check_scene(const eagpt_scene* s) {
  if (!s) return fail(EAGPT_ERR_INVALID_ARGUMENT, "scene is NULL%s");
  if (s->n < 0 || s->n > kMaxSurfels) return fail(EAGPT_ERR_INVALID_ARGUMENT, "scene.n out of range: %s%lld", "", s->n);
  if (s->n > 0) {
    const void* ptrs[7] = {s->pos, s->quat, s->scale, s->opacity, s->albedo, s->radiance, s->emissive};
    const char* names[7] = {"pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive"};
    for (int i = 0; i < 7; ++i) {
      if (!ptrs[i]) return fail(EAGPT_ERR_INVALID_ARGUMENT, "scene.%s is NULL", names[i]);
      if (!aligned(ptrs[i], 4)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "scene.%s is not 4-byte aligned", names[i]);
    }
  }
  return EAGPT_OK;
}

eagpt_status check_camera(const eagpt_camera* c) {
  if (!c) return fail(EAGPT_ERR_INVALID_ARGUMENT, "camera is NULL%s");
  if (c->width <= 0 || c->height <= 0) return fail(EAGPT_ERR_INVALID_ARGUMENT, "camera size must be positive%s");
  if ((int64_t)c->width * c->height > (int64_t)1 << 30)
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "camera has too many pixels%s");
  if (!(c->fx != 0.f && c->fy != 0.f && std::isfinite(c->fx) && std::isfinite(c->fy)))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "camera focal lengths must be finite and non-zero%s");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(c->c2w[i])) return fail(EAGPT_ERR_INVALID_ARGUMENT, "camera c2w must be finite%s");
  return EAGPT_OK;
}

eagpt_status check_bvh(const eagpt_bvh* b, const eagpt_scene* s, const eagpt_params* p) {
  if (!b) return fail(EAGPT_ERR_INVALID_ARGUMENT, "bvh is NULL%s");
  if (b->n != s->n) return fail(EAGPT_ERR_INVALID_ARGUMENT, "bvh was built for another surfel count%s");
  if (b->scene_version != s->version)
    return fail(EAGPT_ERR_STALE_BVH, "bvh was built for scene version %s%lld", "", (long long)b->scene_version);
  if (b->support_sigma != p->support_sigma)
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "bvh was built with another support_sigma%s");
  if (s->n > 0) {
    if (!b->storage || !aligned(b->storage, 256))
      return fail(EAGPT_ERR_INVALID_ARGUMENT, "bvh storage must be non-NULL and 256-byte aligned%s");
    if (b->bytes < bvh_layout(s->n).total) return fail(EAGPT_ERR_OUT_OF_MEMORY, "bvh storage too small%s");
  }
  return EAGPT_OK;
}

BvhView make_view(const eagpt_bvh& b) {
  BvhView v{};
  v.n = b.n;
  if (b.n > 0) {
    const BvhLayout L = bvh_layout(b.n);
    char* base = (char*)b.storage;
    v.trace = (const TraceRec*)(base + L.trace);
    v.shade = (const ShadeRec*)(base + L.shade);
    v.nodes = (const Node4*)(base + L.nodes);
    v.root = 0;  // node 0: Karras root, or the single node of a small scene
    v.bounds_bits = (const uint32_t*)(base + L.header);
    v.hdr = (const BvhHeader*)(base + L.header);
    v.em_idx = (const uint32_t*)(base + L.em_idx);
    v.em_cdf = (const double*)(base + L.em_cdf);
  }
  return v;
}

}  // namespace

extern "C" {

void eagpt_default_params(eagpt_params* p) {
  if (!p) return;
  p->tau_E = 0.1f;
  p->T_min = 1e-3f;
  p->alpha_min = 1.0f / 255.0f;
  p->alpha_max = 0.99f;
  p->support_sigma = 3.0f;
  p->bounce_offset = 1e-3f;
  p->flags = 0;
}

const char* eagpt_last_error(void) { return g_msg.c_str(); }

const char* eagpt_version(void) { return "eagpt 0.1 (sm_103a)"; }

size_t eagpt_bvh_bytes(int64_t n) {
  if (n < 0 || n > kMaxSurfels) return 0;
  return bvh_layout(n).total;
}

eagpt_status eagpt_build_bvh(const eagpt_scene* scene, const eagpt_params* params, void* storage, size_t bytes,
                             eagpt_bvh* out, eagpt_stream_t stream) {
  eagpt_status s;
  if ((s = check_scene(scene)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if (!out) return fail(EAGPT_ERR_INVALID_ARGUMENT, "out is NULL%s");
  const BvhLayout L = bvh_layout(scene->n);
  if (scene->n > 0) {
    if (!storage || !aligned(storage, 256))
      return fail(EAGPT_ERR_INVALID_ARGUMENT, "storage must be non-NULL and 256-byte aligned%s");
    if (bytes < L.total) return fail(EAGPT_ERR_OUT_OF_MEMORY, "storage too small: need %s%lld bytes", "", (long long)L.total);
  }
  cudaStream_t st = (cudaStream_t)stream;
  float area = 0.f;
  if (scene->n > 0) {
    cudaError_t e = launch_build(*scene, make_consts(*params), (char*)storage, L, st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "build_bvh launch");
    double a = 0.0;
    e = cudaMemcpyAsync(&a, (char*)storage + L.header + offsetof(BvhHeader, area_sum), sizeof(double),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "build_bvh");
    area = (float)a;
  }
  out->storage = storage;
  out->bytes = bytes;
  out->n = scene->n;
  out->scene_version = scene->version;
  out->support_sigma = params->support_sigma;
  out->build_area = area;
  return EAGPT_OK;
}

size_t eagpt_render_workspace_bytes(const eagpt_camera* cam, int32_t spp, int32_t kind) {
  if (!cam || cam->width <= 0 || cam->height <= 0 || spp <= 0 || kind < 0 || kind > 2) return 0;
  const int64_t npix = (int64_t)cam->width * cam->height;
  // one pass over all samples, capped at 2^27 paths per pass (~8.6 GB)
  int64_t batch = spp;
  const int64_t cap = (int64_t)1 << 27;
  if (npix * batch > cap) batch = cap / npix > 0 ? cap / npix : 1;
  return render_layout(npix, spp, (int)batch, kind == 2).total;
}

size_t eagpt_render_workspace_min_bytes(const eagpt_camera* cam, int32_t spp, int32_t kind) {
  if (!cam || cam->width <= 0 || cam->height <= 0 || spp <= 0 || kind < 0 || kind > 2) return 0;
  return render_layout((int64_t)cam->width * cam->height, spp, 1, kind == 2).total;
}

}  // extern "C"

namespace eagpt {
eagpt_status set_error(eagpt_status s, const char* msg) {
  g_msg = msg;
  return s;
}
}  // namespace eagpt

extern "C" {

static eagpt_status render_common(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                                  const eagpt_params* params, int kind, int32_t spp, int32_t max_bounces,
                                  int32_t rr_start, uint64_t seed, float* out_rgb, float* out_aux, float* out_samples,
                                  int64_t* out_stats, void* ws, size_t ws_bytes, eagpt_stream_t stream,
                                  float* out_li = nullptr, float4* sb_cache = nullptr, int32_t first_sample = 0,
                                  const eagpt_bvh* lod_bvh = nullptr, int32_t lod_from = 0) {
  eagpt_status s;
  if ((s = check_scene(scene)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if ((s = check_camera(cam)) != EAGPT_OK) return s;
  if ((s = check_bvh(bvh, scene, params)) != EAGPT_OK) return s;
  if (spp <= 0 || spp > (1 << 24)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "spp must be in [1, 2^24]%s");
  if (first_sample < 0 || (int64_t)first_sample + spp > (int64_t)1 << 24)
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "first_sample must be >= 0 with first_sample + spp <= 2^24%s");
  if (kind == 1 && (max_bounces < 0 || max_bounces > 60))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "max_bounces must be in [0, 60]%s");
  if (!out_rgb) return fail(EAGPT_ERR_INVALID_ARGUMENT, "out_rgb is NULL%s");
  if (!ws || !aligned(ws, 256)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "workspace must be non-NULL and 256-byte aligned%s");
  const int64_t npix = (int64_t)cam->width * cam->height;
  const bool mis = kind == 1 && (params->flags & EAGPT_FLAG_EMITTER_SAMPLING);
  if (choose_batch_spp(npix, spp, ws_bytes, mis) < 1)
    return fail(EAGPT_ERR_OUT_OF_MEMORY, "workspace too small: need at least %s%lld bytes", "",
                (long long)render_layout(npix, spp, 1, mis).total);
  RenderArgs a{};
  a.bvh = make_view(*bvh);
  a.C = make_consts(*params);
  a.cam = *cam;
  a.kind = kind == 0 && out_li ? 2 : kind;
  a.out_li = out_li;
  a.spp = spp;
  a.s_first = first_sample;
  a.max_bounces = kind == 0 ? 1 : max_bounces;
  a.rr_start = kind == 0 ? (1 << 30) : rr_start;
  a.seed = seed;
  a.out_rgb = out_rgb;
  a.out_aux = out_aux;
  a.out_samples = out_samples;
  a.out_stats = out_stats;
  a.ws = ws;
  a.ws_bytes = ws_bytes;
  a.sb_cache = sb_cache;
  if (lod_bvh) {
    a.bvh_lod = make_view(*lod_bvh);
    a.lod_from = lod_from;
  }
  cudaError_t e = launch_render(a, (cudaStream_t)stream, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "render launch");
  return EAGPT_OK;
}

}  // extern "C"

namespace eagpt {
eagpt_status render_entry(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                          const eagpt_params* params, int kind, int32_t spp, int32_t max_bounces, int32_t rr_start,
                          uint64_t seed, float* out_rgb, float* out_aux, float* out_samples, int64_t* out_stats,
                          void* ws, size_t ws_bytes, eagpt_stream_t stream) {
  return render_common(scene, bvh, cam, params, kind, spp, max_bounces, rr_start, seed, out_rgb, out_aux,
                       out_samples, out_stats, ws, ws_bytes, stream);
}
}  // namespace eagpt

extern "C" {

eagpt_status eagpt_render_single_bounce(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                                        const eagpt_params* params, int32_t spp, uint64_t seed, float* out_rgb,
                                        float* out_aux, float* out_samples, void* workspace, size_t workspace_bytes,
                                        eagpt_stream_t stream) {
  return render_common(scene, bvh, cam, params, 0, spp, 1, 1 << 30, seed, out_rgb, out_aux, out_samples, nullptr,
                       workspace, workspace_bytes, stream);
}

eagpt_status eagpt_render_single_bounce_incident(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                                 const eagpt_camera* cam, const eagpt_params* params, int32_t spp,
                                                 uint64_t seed, float* out_rgb, float* out_li, void* workspace,
                                                 size_t workspace_bytes, eagpt_stream_t stream) {
  if (!out_li) return fail(EAGPT_ERR_INVALID_ARGUMENT, "out_li is NULL%s");
  return render_common(scene, bvh, cam, params, 0, spp, 1, 1 << 30, seed, out_rgb, nullptr, nullptr, nullptr,
                       workspace, workspace_bytes, stream, out_li);
}

eagpt_status eagpt_render_path_traced(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                                      const eagpt_params* params, int32_t spp, int32_t max_bounces,
                                      int32_t rr_start_bounce, uint64_t seed, float* out_rgb, float* out_aux,
                                      float* out_samples, int64_t* out_stats, void* workspace,
                                      size_t workspace_bytes, eagpt_stream_t stream) {
  return render_common(scene, bvh, cam, params, 1, spp, max_bounces, rr_start_bounce, seed, out_rgb, out_aux,
                       out_samples, out_stats, workspace, workspace_bytes, stream);
}

eagpt_status eagpt_render_segments(const void* workspace, int64_t* out_segments, eagpt_stream_t stream) {
  if (!workspace || !aligned(workspace, 256) || !out_segments)
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "workspace (256-byte aligned) and out_segments are required%s");
  const cudaError_t e = render_summary(workspace, out_segments, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "segment summary read");
  return EAGPT_OK;
}

eagpt_status eagpt_render_path_traced_range(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                            const eagpt_camera* cam, const eagpt_params* params,
                                            int32_t first_sample, int32_t spp, int32_t max_bounces,
                                            int32_t rr_start_bounce, uint64_t seed, float* out_rgb, float* out_aux,
                                            float* out_samples, int64_t* out_stats, void* workspace,
                                            size_t workspace_bytes, eagpt_stream_t stream) {
  return render_common(scene, bvh, cam, params, 1, spp, max_bounces, rr_start_bounce, seed, out_rgb, out_aux,
                       out_samples, out_stats, workspace, workspace_bytes, stream, nullptr, nullptr, first_sample);
}

eagpt_status eagpt_render_path_traced_lod(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                          const eagpt_scene* lod_scene, const eagpt_bvh* lod_bvh,
                                          int32_t lod_from_bounce, const eagpt_camera* cam,
                                          const eagpt_params* params, int32_t first_sample, int32_t spp,
                                          int32_t max_bounces, int32_t rr_start_bounce, uint64_t seed,
                                          float* out_rgb, float* out_aux, float* out_samples, int64_t* out_stats,
                                          void* workspace, size_t workspace_bytes, eagpt_stream_t stream) {
  eagpt_status s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if (params->flags & EAGPT_FLAG_EMITTER_SAMPLING)
    return fail(EAGPT_ERR_NOT_SUPPORTED, "the level-of-detail render has no emitter sampling%s");
  if (lod_from_bounce < 1) return fail(EAGPT_ERR_INVALID_ARGUMENT, "lod_from_bounce must be >= 1%s");
  if ((s = check_scene(lod_scene)) != EAGPT_OK) return s;
  if ((s = check_bvh(lod_bvh, lod_scene, params)) != EAGPT_OK) return s;
  return render_common(scene, bvh, cam, params, 1, spp, max_bounces, rr_start_bounce, seed, out_rgb, out_aux,
                       out_samples, out_stats, workspace, workspace_bytes, stream, nullptr, nullptr, first_sample,
                       lod_bvh, lod_from_bounce);
}

size_t eagpt_lod_workspace_bytes(int64_t n) { return n < 0 ? 0 : lod_workspace_bytes(n); }

eagpt_status eagpt_build_lod(const eagpt_scene* scene, const eagpt_params* params, const float origin[3],
                             float cell_size, eagpt_scene_mut* out, uint64_t* out_keys, int64_t* out_count,
                             void* workspace, size_t workspace_bytes, eagpt_stream_t stream) {
  eagpt_status s;
  if ((s = check_scene(scene)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if (!origin || !out_count || !out) return fail(EAGPT_ERR_INVALID_ARGUMENT, "origin, out and out_count are required%s");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(origin[k])) return fail(EAGPT_ERR_INVALID_ARGUMENT, "origin must be finite%s");
  const float inv_h = 1.0f / cell_size;
  if (!(cell_size > 0.f) || !std::isfinite(cell_size) || !std::isfinite(inv_h))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "cell_size must be positive and finite with a finite inverse%s");
  if (out->n < scene->n)
    return fail(EAGPT_ERR_OUT_OF_MEMORY, "out holds fewer surfels than the scene (capacity %s%lld)", "",
                (long long)out->n);
  if (scene->n > 0) {
    float* optrs[7] = {out->pos, out->quat, out->scale, out->opacity, out->albedo, out->radiance, out->emissive};
    for (int i = 0; i < 7; ++i)
      if (!optrs[i] || !aligned(optrs[i], 4))
        return fail(EAGPT_ERR_INVALID_ARGUMENT, "out arrays must be non-NULL and 4-byte aligned%s");
    if (out_keys && !aligned(out_keys, 8)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "out_keys must be 8-byte aligned%s");
    if (!workspace || !aligned(workspace, 256))
      return fail(EAGPT_ERR_INVALID_ARGUMENT, "workspace must be non-NULL and 256-byte aligned%s");
    if (workspace_bytes < lod_workspace_bytes(scene->n))
      return fail(EAGPT_ERR_OUT_OF_MEMORY, "workspace too small: need %s%lld bytes", "",
                  (long long)lod_workspace_bytes(scene->n));
  }
  const cudaError_t e =
      launch_lod(*scene, origin, inv_h, params->tau_E, *out, out_keys, workspace, out_count, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "level-of-detail merge");
  return EAGPT_OK;
}

size_t eagpt_render_backward_workspace_bytes(const eagpt_camera* cam, int32_t spp) {
  if (!cam || cam->width <= 0 || cam->height <= 0 || spp <= 0) return 0;
  const int64_t npix = (int64_t)cam->width * cam->height;
  int64_t batch = spp;
  const int64_t cap = (int64_t)1 << 26;
  if (npix * batch > cap) batch = cap / npix > 0 ? cap / npix : 1;
  return backward_workspace_bytes(npix, spp, (int)batch);
}

size_t eagpt_render_backward_workspace_min_bytes(const eagpt_camera* cam, int32_t spp) {
  if (!cam || cam->width <= 0 || cam->height <= 0 || spp <= 0) return 0;
  return backward_workspace_bytes((int64_t)cam->width * cam->height, spp, 1);
}

static eagpt_status backward_common(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                                    const eagpt_params* params, int32_t spp, uint64_t seed, const float* dL_drgb,
                                    const eagpt_scene_grad* grads, void* ws, size_t ws_bytes, eagpt_stream_t stream,
                                    const float4* sb_cache) {
  eagpt_status s;
  if ((s = check_scene(scene)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if ((s = check_camera(cam)) != EAGPT_OK) return s;
  if ((s = check_bvh(bvh, scene, params)) != EAGPT_OK) return s;
  if (spp <= 0 || spp > (1 << 24)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "spp must be in [1, 2^24]%s");
  if (!dL_drgb) return fail(EAGPT_ERR_INVALID_ARGUMENT, "dL_drgb is NULL%s");
  if (!grads || grads->n != scene->n) return fail(EAGPT_ERR_INVALID_ARGUMENT, "grads must match the scene%s");
  if (scene->n > 0 && (!grads->pos || !grads->quat || !grads->scale || !grads->opacity || !grads->albedo ||
                       !grads->radiance))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "every gradient array is required%s");
  if (!ws || !aligned(ws, 256)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "workspace must be non-NULL and 256-byte aligned%s");
  const int64_t npix = (int64_t)cam->width * cam->height;
  if (backward_choose_batch(npix, spp, ws_bytes) < 1)
    return fail(EAGPT_ERR_OUT_OF_MEMORY, "workspace too small: need at least %s%lld bytes", "",
                (long long)backward_workspace_bytes(npix, spp, 1));
  if (scene->n == 0) return EAGPT_OK;
  cudaError_t e = launch_backward(make_view(*bvh), make_consts(*params), *cam, *scene, *grads, spp, seed, dL_drgb, ws,
                                  ws_bytes, (cudaStream_t)stream, sb_cache);
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  return EAGPT_OK;
}

eagpt_status eagpt_render_single_bounce_backward(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                                 const eagpt_camera* cam, const eagpt_params* params, int32_t spp,
                                                 uint64_t seed, const float* dL_drgb, const eagpt_scene_grad* grads,
                                                 void* ws, size_t ws_bytes, eagpt_stream_t stream) {
  return backward_common(scene, bvh, cam, params, spp, seed, dL_drgb, grads, ws, ws_bytes, stream, nullptr);
}

size_t eagpt_single_bounce_cache_bytes(const eagpt_camera* cam, int32_t spp) {
  if (!cam || cam->width <= 0 || cam->height <= 0 || spp <= 0) return 0;
  return (size_t)cam->width * cam->height * (size_t)spp * sizeof(float4);
}

eagpt_status eagpt_render_single_bounce_cached(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                               const eagpt_camera* cam, const eagpt_params* params, int32_t spp,
                                               uint64_t seed, float* out_rgb, float* sample_cache, void* ws,
                                               size_t ws_bytes, eagpt_stream_t stream) {
  if (!sample_cache || !aligned(sample_cache, 16))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "sample_cache must be non-NULL and 16-byte aligned%s");
  return render_common(scene, bvh, cam, params, 0, spp, 1, 0, seed, out_rgb, nullptr, nullptr, nullptr, ws, ws_bytes,
                       stream, nullptr, (float4*)sample_cache);
}

eagpt_status eagpt_render_single_bounce_backward_cached(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                                        const eagpt_camera* cam, const eagpt_params* params,
                                                        int32_t spp, uint64_t seed, const float* dL_drgb,
                                                        const float* sample_cache, const eagpt_scene_grad* grads,
                                                        void* ws, size_t ws_bytes, eagpt_stream_t stream) {
  if (!sample_cache || !aligned(sample_cache, 16))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "sample_cache must be non-NULL and 16-byte aligned%s");
  return backward_common(scene, bvh, cam, params, spp, seed, dL_drgb, grads, ws, ws_bytes, stream,
                         (const float4*)sample_cache);
}

eagpt_status eagpt_render_radiance(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                                   const eagpt_params* params, float* out_rgb, float* out_aux,
                                   eagpt_stream_t stream) {
  eagpt_status s;
  if ((s = check_scene(scene)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if ((s = check_camera(cam)) != EAGPT_OK) return s;
  if ((s = check_bvh(bvh, scene, params)) != EAGPT_OK) return s;
  if (!out_rgb) return fail(EAGPT_ERR_INVALID_ARGUMENT, "out_rgb is NULL%s");
  cudaError_t e = launch_radiance(make_view(*bvh), make_consts(*params), *cam, out_rgb, out_aux, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "radiance launch");
  return EAGPT_OK;
}

eagpt_status eagpt_render_radiance_backward(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                                            const eagpt_params* params, const float* dL_drgb,
                                            const eagpt_scene_grad* grads, eagpt_stream_t stream) {
  eagpt_status s;
  if ((s = check_scene(scene)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if ((s = check_camera(cam)) != EAGPT_OK) return s;
  if ((s = check_bvh(bvh, scene, params)) != EAGPT_OK) return s;
  if (!dL_drgb) return fail(EAGPT_ERR_INVALID_ARGUMENT, "dL_drgb is NULL%s");
  if (!grads || grads->n != scene->n) return fail(EAGPT_ERR_INVALID_ARGUMENT, "grads must match the scene%s");
  if (scene->n > 0 && (!grads->pos || !grads->quat || !grads->scale || !grads->opacity || !grads->albedo ||
                       !grads->radiance))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "every gradient array is required%s");
  if (scene->n == 0) return EAGPT_OK;
  cudaError_t e = launch_radiance_backward(make_view(*bvh), make_consts(*params), *cam, *scene, *grads, dL_drgb,
                                           (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "radiance backward launch");
  return EAGPT_OK;
}

size_t eagpt_select_scratch_bytes(int64_t n) { return n < 0 ? 0 : select_scratch_bytes(n); }

eagpt_status eagpt_select(const eagpt_scene* scene, int32_t shape, const float* params, int32_t* out_idx,
                          int64_t capacity, int64_t* out_count, void* scratch, size_t scratch_bytes,
                          eagpt_stream_t stream) {
  eagpt_status s;
  if ((s = check_scene(scene)) != EAGPT_OK) return s;
  if (shape != 0 && shape != 1) return fail(EAGPT_ERR_INVALID_ARGUMENT, "shape must be 0 (box) or 1 (sphere)%s");
  if (!params || !out_count) return fail(EAGPT_ERR_INVALID_ARGUMENT, "params and out_count are required%s");
  if (capacity < 0 || (capacity > 0 && !out_idx)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "bad out_idx/capacity%s");
  if (scene->n > 0 && (!scratch || scratch_bytes < select_scratch_bytes(scene->n)))
    return fail(EAGPT_ERR_OUT_OF_MEMORY, "select scratch too small%s");
  cudaError_t e = launch_select(*scene, shape, params, out_idx, capacity, out_count, (uint32_t*)scratch,
                                (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "select launch");
  return EAGPT_OK;
}

eagpt_status eagpt_apply_edit(eagpt_scene_mut* scene, eagpt_bvh* bvh, const eagpt_params* params,
                              const eagpt_edit* edit, float rebuild_ratio, int32_t* out_rebuilt,
                              eagpt_stream_t stream) {
  if (!scene || !edit) return fail(EAGPT_ERR_INVALID_ARGUMENT, "scene and edit are required%s");
  eagpt_scene cs;
  std::memcpy(&cs, scene, sizeof(cs));  // same layout, const view
  eagpt_status s;
  if ((s = check_scene(&cs)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if ((s = check_bvh(bvh, &cs, params)) != EAGPT_OK) return s;
  if (edit->op < EAGPT_EDIT_SET_EMISSION || edit->op > EAGPT_EDIT_RIGID)
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "unknown edit op%s");
  if (edit->reserved != 0) return fail(EAGPT_ERR_INVALID_ARGUMENT, "edit.reserved must be 0%s");
  if (edit->count < 0 || edit->count > scene->n || (edit->count > 0 && !edit->idx))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "edit count/idx invalid%s");
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(edit->value[k])) return fail(EAGPT_ERR_INVALID_ARGUMENT, "edit values must be finite%s");
  return apply_edit_core(scene, bvh, params, edit, rebuild_ratio, out_rebuilt, (cudaStream_t)stream);
}

}  // extern "C"

namespace eagpt {

BvhView bvh_view(const eagpt_bvh& b) { return make_view(b); }

// The edit after its arguments were checked: edit, records, refit or
// rebuild, version bump.
eagpt_status apply_edit_core(eagpt_scene_mut* scene, eagpt_bvh* bvh, const eagpt_params* params,
                             const eagpt_edit* edit, float rebuild_ratio, int32_t* out_rebuilt, cudaStream_t st) {
  eagpt_scene cs;
  std::memcpy(&cs, scene, sizeof(cs));
  if (out_rebuilt) *out_rebuilt = 0;
  cudaError_t e = launch_edit(*scene, *edit, st);
  if (e != cudaSuccess) return cuda_fail(e, "edit launch");
  if (scene->n > 0) {
    const BvhLayout L = bvh_layout(scene->n);
    char* base = (char*)bvh->storage;
    const Consts C = make_consts(*params);
    e = launch_records_update(cs, C, base, L, st);
    if (e != cudaSuccess) return cuda_fail(e, "edit records");
    if (edit->op == EAGPT_EDIT_TRANSLATE || edit->op == EAGPT_EDIT_RIGID) {
      launch_refit(base, L, st);
      double a = 0.0;
      e = cudaMemcpyAsync(&a, base + L.header + offsetof(BvhHeader, area_sum), sizeof(double),
                          cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "refit");
      if (rebuild_ratio > 0.f && a > (double)rebuild_ratio * (double)bvh->build_area) {
        e = launch_build(cs, C, base, L, st, nullptr);
        double b = 0.0;
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(&b, base + L.header + offsetof(BvhHeader, area_sum), sizeof(double),
                              cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "rebuild");
        bvh->build_area = (float)b;
        if (out_rebuilt) *out_rebuilt = 1;
      }
    }
  }
  scene->version += 1;
  bvh->scene_version = scene->version;
  return EAGPT_OK;
}

}  // namespace eagpt

extern "C" {

eagpt_status eagpt_trace_rays(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_params* params,
                              int32_t mode, const float* rays, int64_t n_rays, float* out_rec, int32_t* out_hits,
                              int32_t max_hits, int32_t* out_nhits, eagpt_stream_t stream) {
  eagpt_status s;
  if ((s = check_scene(scene)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if ((s = check_bvh(bvh, scene, params)) != EAGPT_OK) return s;
  if (mode != 0 && mode != 1) return fail(EAGPT_ERR_INVALID_ARGUMENT, "mode must be 0 or 1%s");
  if (n_rays < 0) return fail(EAGPT_ERR_INVALID_ARGUMENT, "n_rays must be >= 0%s");
  if (n_rays > 0 && (!rays || !out_rec)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "rays and out_rec are required%s");
  if (out_hits && max_hits <= 0) return fail(EAGPT_ERR_INVALID_ARGUMENT, "max_hits must be positive%s");
  cudaError_t e = launch_trace_rays(make_view(*bvh), make_consts(*params), mode, rays, n_rays, out_rec, out_hits,
                                    max_hits, out_nhits, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "trace_rays launch");
  return EAGPT_OK;
}

int64_t eagpt_launch_count(void) { return launch_count(); }

eagpt_status eagpt_profile_begin(void) {
  profile_begin();
  return EAGPT_OK;
}

eagpt_status eagpt_profile_end(eagpt_kernel_time* out, int32_t capacity, int32_t* n_out) {
  if (capacity < 0) return fail(EAGPT_ERR_INVALID_ARGUMENT, "capacity must be >= 0%s");
  const int n = profile_end(out, capacity);
  if (n_out) *n_out = n;
  return EAGPT_OK;
}

eagpt_status eagpt_sync_status(eagpt_stream_t stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  const uint32_t word =
      take_errors_bvh() | take_errors_render() | take_errors_backward() | take_errors_tree() | take_errors_edit() |
      take_errors_serve() | take_errors_optim();
  if (word) {
    char buf[128];
    std::snprintf(buf, sizeof(buf), "device check failed (error bits 0x%x)", word);
    g_msg = buf;
    return EAGPT_ERR_DEVICE_CHECK;
  }
  return EAGPT_OK;
}

}  // extern "C"

// --------------------------------------------------------------------------
// optimisation of the shading parameters (Eq. 7, Eq. 10)
// --------------------------------------------------------------------------
namespace {

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct FitLayout {
  size_t pred, li, dL, grad, partials, render, total;
};

FitLayout fit_layout(int field, int64_t npix_max, int64_t n, size_t render_bytes) {
  FitLayout L{};
  size_t o = 0;
  const size_t img = up256((size_t)npix_max * 3 * sizeof(float));
  L.pred = o;
  o += img;
  L.li = o;
  if (field == 0) o += img;
  L.dL = o;
  o += img;
  L.grad = o;
  o += up256((size_t)(n > 0 ? n : 1) * 3 * sizeof(float));
  L.partials = o;
  o += up256((size_t)pq_partials(3 * npix_max) * sizeof(double) + sizeof(double));
  L.render = o;
  o += render_bytes;
  L.total = o;
  return L;
}

eagpt_status check_adam(const eagpt_adam* a) {
  if (!a) return fail(EAGPT_ERR_INVALID_ARGUMENT, "adam config is NULL%s");
  if (!(a->lr > 0.f && std::isfinite(a->lr))) return fail(EAGPT_ERR_INVALID_ARGUMENT, "adam.lr must be > 0%s");
  if (!(a->beta1 >= 0.f && a->beta1 < 1.f && a->beta2 >= 0.f && a->beta2 < 1.f))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "adam betas must be in [0, 1)%s");
  if (!(a->eps > 0.f && std::isfinite(a->eps))) return fail(EAGPT_ERR_INVALID_ARGUMENT, "adam.eps must be > 0%s");
  if (!(a->lo <= a->hi)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "adam.lo must be <= adam.hi%s");
  return EAGPT_OK;
}

eagpt_status check_fit(const eagpt_fit_config* c) {
  if (!c) return fail(EAGPT_ERR_INVALID_ARGUMENT, "fit config is NULL%s");
  if (c->field != 0 && c->field != 1) return fail(EAGPT_ERR_INVALID_ARGUMENT, "field must be 0 or 1%s");
  if (c->field == 0 && (c->spp <= 0 || c->spp > (1 << 24)))
    return fail(EAGPT_ERR_INVALID_ARGUMENT, "spp must be in [1, 2^24]%s");
  if (!(c->peak > 0.f && std::isfinite(c->peak))) return fail(EAGPT_ERR_INVALID_ARGUMENT, "peak must be > 0%s");
  if (!std::isfinite(c->lambda_c)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "lambda_c must be finite%s");
  return check_adam(&c->adam);
}

size_t fit_render_bytes(const eagpt_fit_config* cfg, int64_t npix_max, bool full) {
  if (cfg->field != 0) return 0;
  int64_t batch = cfg->spp;
  const int64_t cap = (int64_t)1 << 27;
  if (!full) batch = 1;
  else if (npix_max * batch > cap) batch = cap / npix_max > 0 ? cap / npix_max : 1;
  return render_layout(npix_max, cfg->spp, (int)batch).total;
}

}  // namespace

extern "C" {

eagpt_status eagpt_render_shading_backward(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                                           const eagpt_params* params, int32_t field, const float* dL_drgb,
                                           const float* li, float* grad, eagpt_stream_t stream) {
  eagpt_status s;
  if ((s = check_scene(scene)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if ((s = check_camera(cam)) != EAGPT_OK) return s;
  if ((s = check_bvh(bvh, scene, params)) != EAGPT_OK) return s;
  if (field != 0 && field != 1) return fail(EAGPT_ERR_INVALID_ARGUMENT, "field must be 0 (albedo) or 1 (radiance)%s");
  if (field == 0 && !li) return fail(EAGPT_ERR_INVALID_ARGUMENT, "the albedo gradient needs li%s");
  if (field == 1 && li) return fail(EAGPT_ERR_INVALID_ARGUMENT, "li must be NULL for the radiance gradient%s");
  if (!dL_drgb) return fail(EAGPT_ERR_INVALID_ARGUMENT, "dL_drgb is NULL%s");
  if (scene->n > 0 && !grad) return fail(EAGPT_ERR_INVALID_ARGUMENT, "grad is NULL%s");
  if (scene->n == 0) return EAGPT_OK;
  cudaError_t e = launch_shade_adjoint(make_view(*bvh), make_consts(*params), *cam, dL_drgb, li, grad,
                                       (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "shading backward launch");
  return EAGPT_OK;
}

size_t eagpt_pq_l1_scratch_bytes(int64_t n) {
  if (n < 0) return 0;
  return (size_t)(pq_partials(n) + 1) * sizeof(double);
}

eagpt_status eagpt_pq_l1_loss(const float* pred, const float* target, int64_t n, float peak, float lambda_c,
                              float* out_grad, double* out_loss, void* scratch, size_t scratch_bytes,
                              eagpt_stream_t stream) {
  if (n < 0) return fail(EAGPT_ERR_INVALID_ARGUMENT, "n must be >= 0%s");
  if (n > 0 && (!pred || !target)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "pred and target are required%s");
  if (!(peak > 0.f && std::isfinite(peak))) return fail(EAGPT_ERR_INVALID_ARGUMENT, "peak must be > 0%s");
  if (!std::isfinite(lambda_c)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "lambda_c must be finite%s");
  if (n > 0 && (!scratch || !aligned(scratch, 8) || scratch_bytes < eagpt_pq_l1_scratch_bytes(n)))
    return fail(EAGPT_ERR_OUT_OF_MEMORY, "scratch too small or misaligned%s");
  cudaError_t e = launch_pq_l1(pred, target, n, peak, lambda_c, out_grad, out_loss, (double*)scratch,
                               (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pq_l1 launch");
  return EAGPT_OK;
}

eagpt_status eagpt_adam_step(float* param, float* grad, float* m, float* v, int64_t n, const eagpt_adam* cfg,
                             int64_t step, int32_t zero_grad, eagpt_stream_t stream) {
  eagpt_status s;
  if ((s = check_adam(cfg)) != EAGPT_OK) return s;
  if (n < 0 || step < 1) return fail(EAGPT_ERR_INVALID_ARGUMENT, "n must be >= 0 and step >= 1%s");
  if (n > 0 && (!param || !grad || !m || !v)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "every array is required%s");
  cudaError_t e = launch_adam(param, grad, m, v, n, *cfg, step, zero_grad != 0, nullptr, nullptr, 0,
                              (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "adam launch");
  return EAGPT_OK;
}

size_t eagpt_fit_workspace_bytes(const eagpt_fit_config* cfg, const eagpt_camera* cams, int32_t n_views, int64_t n) {
  if (!cfg || !cams || n_views <= 0 || n < 0 || (cfg->field != 0 && cfg->field != 1)) return 0;
  if (cfg->field == 0 && cfg->spp <= 0) return 0;
  int64_t npix = 0;
  for (int v = 0; v < n_views; ++v) {
    if (cams[v].width <= 0 || cams[v].height <= 0) return 0;
    const int64_t p = (int64_t)cams[v].width * cams[v].height;
    npix = p > npix ? p : npix;
  }
  return fit_layout(cfg->field, npix, n, fit_render_bytes(cfg, npix, true)).total;
}

eagpt_status eagpt_fit(const eagpt_fit_config* cfg, eagpt_scene_mut* scene, eagpt_bvh* bvh, const eagpt_params* params,
                       const eagpt_camera* cams, const float* const* targets, int32_t n_views,
                       const int32_t* view_order, int64_t first_step, int32_t iters, float* m, float* v,
                       double* out_loss, void* ws, size_t ws_bytes, eagpt_stream_t stream) {
  eagpt_status s;
  if ((s = check_fit(cfg)) != EAGPT_OK) return s;
  if (!scene) return fail(EAGPT_ERR_INVALID_ARGUMENT, "scene is NULL%s");
  eagpt_scene cs;
  std::memcpy(&cs, scene, sizeof(cs));
  if ((s = check_scene(&cs)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if ((s = check_bvh(bvh, &cs, params)) != EAGPT_OK) return s;
  if (n_views <= 0 || !cams || !targets) return fail(EAGPT_ERR_INVALID_ARGUMENT, "need n_views >= 1 cameras and targets%s");
  if (iters < 0 || first_step < 0) return fail(EAGPT_ERR_INVALID_ARGUMENT, "iters and first_step must be >= 0%s");
  int64_t npix_max = 0;
  for (int k = 0; k < n_views; ++k) {
    if ((s = check_camera(&cams[k])) != EAGPT_OK) return s;
    if (!targets[k]) return fail(EAGPT_ERR_INVALID_ARGUMENT, "targets[%s%lld] is NULL", "", k);
    const int64_t p = (int64_t)cams[k].width * cams[k].height;
    npix_max = p > npix_max ? p : npix_max;
  }
  if (view_order)
    for (int k = 0; k < iters; ++k)
      if (view_order[k] < 0 || view_order[k] >= n_views)
        return fail(EAGPT_ERR_INVALID_ARGUMENT, "view_order[%s%lld] out of range", "", k);
  if (cs.n > 0 && (!m || !v)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "adam moments m and v are required%s");
  if (!ws || !aligned(ws, 256)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "workspace must be non-NULL and 256-byte aligned%s");
  const size_t need_min = fit_layout(cfg->field, npix_max, cs.n, fit_render_bytes(cfg, npix_max, false)).total;
  if (ws_bytes < need_min)
    return fail(EAGPT_ERR_OUT_OF_MEMORY, "workspace too small: need at least %s%lld bytes", "", (long long)need_min);
  if (iters == 0 || cs.n == 0) return EAGPT_OK;

  cudaStream_t st = (cudaStream_t)stream;
  const FitLayout L = fit_layout(cfg->field, npix_max, cs.n, 0);
  char* base = (char*)ws;
  float* pred = (float*)(base + L.pred);
  float* li = cfg->field == 0 ? (float*)(base + L.li) : nullptr;
  float* dL = (float*)(base + L.dL);
  float* grad = (float*)(base + L.grad);
  double* partials = (double*)(base + L.partials);
  void* rws = base + L.render;
  const size_t rws_bytes = ws_bytes - L.render;
  const BvhView view = make_view(*bvh);
  const Consts C = make_consts(*params);
  const BvhLayout BL = bvh_layout(cs.n);
  float* mirror = (float*)((char*)bvh->storage + BL.shade);
  const uint32_t* inv_idx = (const uint32_t*)((char*)bvh->storage + BL.inv_idx);
  float* field_ptr = cfg->field == 0 ? scene->albedo : scene->radiance;
  const int mirror_field = cfg->field == 0 ? 0 : 4;
  const int64_t np = cs.n * 3;

  cudaError_t e = cudaMemsetAsync(grad, 0, (size_t)np * sizeof(float), st);
  for (int k = 0; k < iters && e == cudaSuccess; ++k) {
    const int64_t t = first_step + k + 1;
    const int vi = view_order ? view_order[k] : (int)((first_step + k) % n_views);
    const eagpt_camera& cam = cams[vi];
    const int64_t npix = (int64_t)cam.width * cam.height;
    if (cfg->field == 0) {
      if (choose_batch_spp(npix, cfg->spp, rws_bytes) < 1) return fail(EAGPT_ERR_OUT_OF_MEMORY, "render workspace%s");
      RenderArgs a{};
      a.bvh = view;
      a.C = C;
      a.cam = cam;
      a.kind = 2;
      a.spp = cfg->spp;
      a.max_bounces = 1;
      a.rr_start = 1 << 30;
      a.seed = cfg->seed + (uint64_t)t;
      a.out_rgb = pred;
      a.out_li = li;
      a.ws = rws;
      a.ws_bytes = rws_bytes;
      e = launch_render(a, st, nullptr);
    } else {
      e = launch_radiance(view, C, cam, pred, nullptr, st);
    }
    if (e == cudaSuccess)
      e = launch_pq_l1(pred, targets[vi], 3 * npix, cfg->peak, cfg->lambda_c, dL, out_loss ? out_loss + k : nullptr,
                       partials, st);
    if (e == cudaSuccess) e = launch_shade_adjoint(view, C, cam, dL, li, grad, st);
    if (e == cudaSuccess)
      e = launch_adam(field_ptr, grad, m, v, np, cfg->adam, t, 1, mirror, inv_idx, mirror_field, st);
  }
  // new radiance changes the emitters' sampling weights
  if (e == cudaSuccess && cfg->field == 1) {
    std::memcpy(&cs, scene, sizeof(cs));
    e = launch_emitter_table(cs, C, (char*)bvh->storage, BL, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "fit launch");
  scene->version += 1;
  bvh->scene_version = scene->version;
  return EAGPT_OK;
}

}  // extern "C"

// --------------------------------------------------------------------------
// insert / delete surfels (the scene's surfel count changes: full rebuild)
// --------------------------------------------------------------------------
extern "C" {

size_t eagpt_delete_scratch_bytes(int64_t n) { return n < 0 ? 0 : delete_scratch_bytes(n); }

eagpt_status eagpt_delete_surfels(eagpt_scene_mut* scene, eagpt_bvh* bvh, const eagpt_params* params,
                                  const int32_t* idx, int64_t count, void* scratch, size_t scratch_bytes,
                                  eagpt_stream_t stream) {
  eagpt_status s;
  if (!scene) return fail(EAGPT_ERR_INVALID_ARGUMENT, "scene is NULL%s");
  eagpt_scene cs;
  std::memcpy(&cs, scene, sizeof(cs));
  if ((s = check_scene(&cs)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if ((s = check_bvh(bvh, &cs, params)) != EAGPT_OK) return s;
  if (count < 0 || (count > 0 && !idx)) return fail(EAGPT_ERR_INVALID_ARGUMENT, "bad idx/count%s");
  if (!scratch || !aligned(scratch, 256) || scratch_bytes < delete_scratch_bytes(cs.n))
    return fail(EAGPT_ERR_OUT_OF_MEMORY, "delete scratch too small or misaligned%s");
  int64_t m = 0;
  cudaError_t e = launch_delete(*scene, idx, count, scratch, &m, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "delete launch");
  scene->n = m;
  scene->version += 1;
  std::memcpy(&cs, scene, sizeof(cs));
  return eagpt_build_bvh(&cs, params, bvh->storage, bvh->bytes, bvh, stream);
}

eagpt_status eagpt_insert_surfels(eagpt_scene_mut* scene, int64_t capacity, const eagpt_scene* src, eagpt_bvh* bvh,
                                  const eagpt_params* params, eagpt_stream_t stream) {
  eagpt_status s;
  if (!scene) return fail(EAGPT_ERR_INVALID_ARGUMENT, "scene is NULL%s");
  eagpt_scene cs;
  std::memcpy(&cs, scene, sizeof(cs));
  if ((s = check_scene(&cs)) != EAGPT_OK) return s;
  if ((s = check_scene(src)) != EAGPT_OK) return s;
  if ((s = check_params(params)) != EAGPT_OK) return s;
  if ((s = check_bvh(bvh, &cs, params)) != EAGPT_OK) return s;
  const int64_t m = src->n, n = cs.n;
  if (n + m > capacity) return fail(EAGPT_ERR_OUT_OF_MEMORY, "the scene arrays hold %s%lld surfels", "", capacity);
  if (n + m > kMaxSurfels) return fail(EAGPT_ERR_INVALID_ARGUMENT, "too many surfels%s");
  if (n + m > 0 && bvh_layout(n + m).total > bvh->bytes)
    return fail(EAGPT_ERR_OUT_OF_MEMORY, "bvh storage too small: need %s%lld bytes", "",
                (long long)bvh_layout(n + m).total);
  cudaStream_t st = (cudaStream_t)stream;
  float* dst[7] = {scene->pos, scene->quat, scene->scale, scene->opacity, scene->albedo, scene->radiance,
                   scene->emissive};
  const float* from[7] = {src->pos, src->quat, src->scale, src->opacity, src->albedo, src->radiance, src->emissive};
  const int comps[7] = {3, 4, 2, 1, 3, 3, 1};
  for (int f = 0; f < 7 && m > 0; ++f) {
    if (!dst[f]) return fail(EAGPT_ERR_INVALID_ARGUMENT, "scene arrays are required%s");
    cudaError_t e = cudaMemcpyAsync(dst[f] + n * comps[f], from[f], (size_t)m * comps[f] * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "insert copy");
  }
  scene->n = n + m;
  scene->version += 1;
  std::memcpy(&cs, scene, sizeof(cs));
  return eagpt_build_bvh(&cs, params, bvh->storage, bvh->bytes, bvh, stream);
}

}  // extern "C"
