/*
 * eagpt.h -- C ABI of the GB300 surfel path tracer (emission-aware 2D Gaussian
 * path tracing, arXiv 2601.23065).
 *
 * Conventions (all entry points):
 *  - Every buffer is owned by the caller.  Pointers documented "device" must
 *    point to memory of the current CUDA device; "host" pointers are read or
 *    written before the call returns.  The library never allocates device
 *    memory on these paths; the *_bytes() queries give the sizes to allocate.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and is asynchronous unless stated otherwise.
 *  - Argument errors are detected on the host and returned immediately;
 *    nothing is enqueued then.  Errors found on the device (a traversal stack
 *    overflow, a bad index) are recorded in a device-side error word and
 *    reported by eagpt_sync_status().  No C++ exception crosses this ABI.
 *  - eagpt_last_error() returns a thread-local message for the last failure.
 *  - Floating-point data is FP32, structure-of-arrays, C-contiguous.
 */
#ifndef EAGPT_H
#define EAGPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* eagpt_stream_t; /* == cudaStream_t */

typedef enum {
  EAGPT_OK = 0,
  EAGPT_ERR_INVALID_ARGUMENT = 1,
  EAGPT_ERR_OUT_OF_MEMORY = 2,   /* a caller buffer is smaller than required */
  EAGPT_ERR_CUDA = 3,            /* a CUDA runtime call failed               */
  EAGPT_ERR_STALE_BVH = 4,       /* BVH built for another scene version      */
  EAGPT_ERR_TIMEOUT = 5,         /* a bounded wait ran out                   */
  EAGPT_ERR_NOT_SUPPORTED = 6,
  EAGPT_ERR_DEVICE_CHECK = 7     /* a device-side check failed               */
} eagpt_status;

/* ------------------------------------------------------------------------
 * Scene: n emission-aware 2D Gaussian surfels (Sec. 3.1, Eq. 1 and Eq. 3).
 *   pos      n x 3  centre p
 *   quat     n x 4  rotation q = (w, x, y, z); need not be unit length, it is
 *                   normalised before use; the tangent axes t_u, t_v are the
 *                   first two columns of its rotation, the normal n = t_u x t_v
 *   scale    n x 2  in-plane scales (s_u, s_v) > 0
 *   opacity  n      sigma in [0, 1]
 *   albedo   n x 3  diffuse albedo rho (BRDF rho/pi, Sec. 3.3 after Eq. 6)
 *   radiance n x 3  linear radiance r (emitters: emission; others: the
 *                   radiance cache of Sec. 3.3)
 *   emissive n      emissive term e in [0, 1] (Eq. 3-4)
 * All device pointers.  `version` is a caller-maintained counter of scene
 * edits; eagpt_apply_edit() increments it.
 * ------------------------------------------------------------------------ */
typedef struct {
  int64_t n;
  const float *pos, *quat, *scale, *opacity, *albedo, *radiance, *emissive;
  uint64_t version;
} eagpt_scene;

typedef struct {
  int64_t n;
  float *pos, *quat, *scale, *opacity, *albedo, *radiance, *emissive;
  uint64_t version;
} eagpt_scene_mut;

/* Gradients, same layout as the scene (device pointers, accumulated +=).
 * There is no emissive gradient: e enters only through threshold tests. */
typedef struct {
  int64_t n;
  float *pos, *quat, *scale, *opacity, *albedo, *radiance;
} eagpt_scene_grad;

/* OpenCV pinhole camera: +x right, +y down, +z forward in camera space;
 * c2w is the row-major 3 x 4 camera-to-world matrix [R | centre].  The ray of
 * pixel (x, y) goes through the pixel centre (x + 0.5, y + 0.5) and is shared
 * by all samples of the pixel (the viewing direction is fixed per pixel in
 * Eq. 6 and Eq. 8).  Pixel linear index = y * width + x. */
typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy;
  float c2w[12];
} eagpt_camera;

/* Method constants.  tau_E is printed in the paper (Sec. 3.3, Eq. 4); the
 * rest are readings of values the paper leaves unstated. */
typedef struct {
  float tau_E;          /* emitter threshold on E, Eq. 4 (0.1)                */
  float T_min;          /* stop blending once transmittance < T_min (1e-3),   */
                        /* Eq. 2 "preset threshold"                            */
  float alpha_min;      /* hits with alpha < alpha_min are skipped (1/255)    */
  float alpha_max;      /* alpha = min(sigma * g, alpha_max) (0.99)           */
  float support_sigma;  /* Gaussian support u^2 + v^2 <= support^2 (3)        */
  float bounce_offset;  /* new origin X + offset * N~ (1e-3 scene units)      */
  int32_t flags;        /* EAGPT_FLAG_* bits; others must be 0 (default 0)    */
} eagpt_params;

/* flags of eagpt_params */
enum {
  /* Path tracing (Eq. 8) with emitter sampling and multiple importance
   * sampling (the variance reduction the paper names as future work).  At
   * every reflection vertex one emitter surfel i (e_i > tau_E) is chosen with
   * probability q_i proportional to mean(r_i) sigma_i s_u,i s_v,i (FP64
   * cumulative sums in surfel-index order), a point of its support disc is
   * drawn from the truncated Gaussian (radius by inverse CDF, uniform angle)
   * and the segment towards it is traced.  The blended radiance is a sum of
   * per-surfel terms w_i r_i (Eq. 2); each emitter term is estimated by both
   * the cosine-sampled continuation (pdf p_B = cos / pi) and the emitter
   * sample (pdf p_L = q_i g_i(u, v) t^2 / |w . n_i|), combined with the power
   * heuristic.  The expectation is that of Eq. 8.  Draws: the emitter sample
   * of reflection k uses Philox counter (pixel, sample, k, 1): u0 selects the
   * emitter, u1 the radius, u2 the angle.  Single-bounce renders and the
   * serving loop ignore / reject it. */
  EAGPT_FLAG_EMITTER_SAMPLING = 1
};

void eagpt_default_params(eagpt_params* out);

/* ------------------------------------------------------------------------
 * Acceleration structure: a software LBVH over the support bounds of the
 * surfels, whose subtrees of at most 256 surfels are rebuilt with the surface
 * area heuristic, collapsed to a 4-wide BVH (the paper uses a hardware BVH,
 * Sec. 4.2; any BVH that returns every hit gives the same image).  Storage is one caller-owned device
 * buffer of eagpt_bvh_bytes(n) bytes, 256-byte aligned.  The handle is a
 * plain host struct filled by eagpt_build_bvh().
 * ------------------------------------------------------------------------ */
typedef struct {
  void* storage;          /* device, caller-owned                          */
  size_t bytes;
  int64_t n;              /* surfels                                       */
  uint64_t scene_version; /* version of the scene it was built/refit for   */
  float support_sigma;    /* support radius the bounds were built with     */
  float build_area;       /* surface-area sum at build (refit heuristic)   */
} eagpt_bvh;

size_t eagpt_bvh_bytes(int64_t n);

/* Builds the BVH of `scene` into `storage` (device) and fills *out (host).
 * Reads the scene's device arrays; the surface-area sum is read back to the
 * host, so this call synchronises `stream` once. */
eagpt_status eagpt_build_bvh(const eagpt_scene* scene, const eagpt_params* params, void* storage,
                             size_t bytes, eagpt_bvh* out, eagpt_stream_t stream);

/* ------------------------------------------------------------------------
 * Rendering.  kind: 0 = single-bounce radiance-cache estimator (Eq. 6),
 * 1 = multi-bounce path tracing (Eq. 8).
 * Workspace: eagpt_render_workspace_bytes() gives a size that renders all
 * samples of the camera in as few passes as the size cap allows; any size of
 * at least eagpt_render_workspace_min_bytes() works (samples are then done
 * in several passes, with identical results).  256-byte aligned, device.
 * ------------------------------------------------------------------------ */
/* kind for the workspace queries: 0 single bounce, 1 path tracing, 2 path
 * tracing with EAGPT_FLAG_EMITTER_SAMPLING (32 more bytes per queued ray). */
size_t eagpt_render_workspace_bytes(const eagpt_camera* cam, int32_t spp, int32_t kind);
size_t eagpt_render_workspace_min_bytes(const eagpt_camera* cam, int32_t spp, int32_t kind);

/* Single-bounce render (Eq. 6): a pixel whose primary blend has E > tau_E
 * shows its blended radiance R (Eq. 4); any other hit pixel shows
 * P (.) mean_s R(w_s), where w_s is a cosine-weighted direction about the
 * blended normal from X + offset N~ and R(w_s) is the secondary segment's
 * blended radiance (the radiance cache, with no emitter test).
 *   out_rgb     device, H x W x 3
 *   out_aux     device or NULL, H x W x 12 primary record per pixel:
 *               N~ (3), D~, R (3), E, P (3), A   (Eq. 3)
 *   out_samples device or NULL, H x W x spp x 3 per-sample contributions
 * Random numbers: Philox4x32-10 with counter (pixel, sample, bounce, 0) and
 * key (seed low, seed high); draws u_j = (x_j >> 8) * 2^-24; u0, u1 pick the
 * cosine direction (radius sqrt(u0), angle 2 pi u1), u2 the roulette test. */
eagpt_status eagpt_render_single_bounce(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                        const eagpt_camera* cam, const eagpt_params* params,
                                        int32_t spp, uint64_t seed, float* out_rgb, float* out_aux,
                                        float* out_samples, void* workspace, size_t workspace_bytes,
                                        eagpt_stream_t stream);

/* Path-traced render (Eq. 8): paths leave the pixel's primary vertex and
 * bounce (cosine-weighted, throughput *= P per vertex) until a vertex with
 * E > tau_E, whose blended radiance (non-emitter radiance dropped, Sec. 3.4)
 * is the sample's value; a path that exceeds max_bounces reflections or
 * misses the scene contributes 0.  From bounce rr_start_bounce on, Russian
 * roulette keeps a path with probability q = min(1, max(throughput)) and
 * divides the throughput by q (not in the paper; rr_start > max_bounces
 * disables it).  max_bounces = 0 renders emitters only.
 * Buffers as in eagpt_render_single_bounce.  out_stats (device or NULL,
 * int64[16], accumulated +=; a counting variant of the kernels runs):
 *   [0] primary segments  [1] secondary segments  [2] paths started
 *   [3..6]  secondary segments: blended hits, BVH nodes visited, surfel
 *           tests, traversal rounds
 *   [7]     deepest traversal stack of a secondary segment (maximum)
 *   [8..11] the same as [3..6] for the primary segments
 *   [12..15] unused (0). */
eagpt_status eagpt_render_path_traced(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                      const eagpt_camera* cam, const eagpt_params* params, int32_t spp,
                                      int32_t max_bounces, int32_t rr_start_bounce, uint64_t seed,
                                      float* out_rgb, float* out_aux, float* out_samples,
                                      int64_t* out_stats, void* workspace, size_t workspace_bytes,
                                      eagpt_stream_t stream);

/* Segments traced by the last render into `workspace` (any of the render
 * entry points above), kept without the counting variant:
 *   out_segments[0] primary segments (one per pixel)
 *   out_segments[1] secondary segments the bounce kernels traced (with
 *                   emitter sampling: the continuations; emitter-sample
 *                   segments are counted only by out_stats)
 * host array of 2.  Synchronises `stream` (a 16-byte device-to-host copy).
 * Not part of the method; it lets a caller report segments per second. */
eagpt_status eagpt_render_segments(const void* workspace, int64_t* out_segments, eagpt_stream_t stream);

/* Samples first_sample .. first_sample + spp - 1 of every pixel of the path-
 * traced render (Eq. 8): the same paths, with the same Philox counters
 * (pixel, sample, bounce), as those samples of eagpt_render_path_traced()
 * with a larger spp, so a frame of S samples can be rendered as consecutive
 * slices (progressive rendering) whose images, each the mean of its own
 * samples, average to the frame's estimate.  out_rgb receives the slice's
 * mean; out_samples (H x W x spp x 3) its samples in order.  Other arguments,
 * buffers and errors as in eagpt_render_path_traced();
 * EAGPT_ERR_INVALID_ARGUMENT if first_sample < 0 or first_sample + spp >
 * 2^24. */
eagpt_status eagpt_render_path_traced_range(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                            const eagpt_camera* cam, const eagpt_params* params,
                                            int32_t first_sample, int32_t spp, int32_t max_bounces,
                                            int32_t rr_start_bounce, uint64_t seed, float* out_rgb, float* out_aux,
                                            float* out_samples, int64_t* out_stats, void* workspace,
                                            size_t workspace_bytes, eagpt_stream_t stream);

/* ------------------------------------------------------------------------
 * Level of detail.  The paper names a level-of-detail hierarchy over the
 * reconstruction as the way to fewer ray-Gaussian intersections per ray
 * (Sec. 5, conclusion, and Appendix D, path tracing: fewer Gaussians, fewer
 * hits per ray, a faster render) and gives no algorithm.  This library's
 * reading:
 *
 * eagpt_build_lod(): merges the surfels of `scene` group by group.  A
 *   surfel's group is (the cell of a uniform grid with corner `origin` (host,
 *   3 floats) and edge `cell_size` holding its centre p, the coordinate axis
 *   its normal is closest to, e > tau_E).  Cell coordinates
 *   floor((p - origin) * (1 / cell_size)) are taken in FP32 (each operation
 *   rounded to nearest) and clamped to [0, 2^20 - 1]; the axis is the largest
 *   |component| (lowest axis on a tie) of (2(xz + wy), 2(yz - wx),
 *   (ww + zz) - (xx + yy)) from the raw quaternion (w, x, y, z), products
 *   and sums rounded to FP32 in that order.  Each group becomes one surfel by
 *   moment matching, with weights w_i = sigma_i s_u,i s_v,i (all-zero
 *   weights: unit weights and sigma 0) and W = sum w_i:
 *     p = weighted mean centre; n = normalised weighted sum of the normals
 *     turned to the group axis' positive side; the union's second moment
 *     sum w_i (d_i d_i^T + s_u,i^2 t_u,i t_u,i^T + s_v,i^2 t_v,i t_v,i^T) / W
 *     about p, projected on the plane of n, gives t_u (principal axis),
 *     t_v = n x t_u and s_u^2, s_v^2 (its variances along them);
 *     sigma = W / (s_u s_v), the group's footprint (may exceed 1: alpha is
 *     still clamped at alpha_max); rho, r, e = weighted means.
 *   Merged surfels are written in ascending group key (cell x << 43 |
 *   cell y << 23 | cell z << 3 | axis << 1 | emitter) to out's device arrays
 *   (capacity out->n >= scene->n surfels, else EAGPT_ERR_OUT_OF_MEMORY);
 *   out_keys (device, nullable, 8-byte aligned) receives the keys.  The
 *   group count is written to *out_count (host): the call synchronises
 *   `stream` once to read it.  out->n and out->version are not modified.
 *   out's arrays must not overlap the scene's (the merge reads every
 *   surfel of a group after earlier groups are written).  The result is
 *   deterministic: each group's sums run over its surfels in ascending
 *   index order (no floating-point atomics).  Of `params` (validated as
 *   for every call) only tau_E is used.  Every buffer is caller-owned.
 *   workspace: device, eagpt_lod_workspace_bytes(scene->n) bytes, 256-byte
 *   aligned.  Positions must be finite and scales positive.
 *   EAGPT_ERR_INVALID_ARGUMENT for a non-finite origin or a cell_size that
 *   is not positive and finite (with a finite inverse).
 *
 * eagpt_render_path_traced_lod(): eagpt_render_path_traced_range() (Eq. 8)
 *   in which the bounce segments k >= lod_from_bounce (k = 1 is the segment
 *   after the first reflection) trace lod_scene through lod_bvh (built by
 *   eagpt_build_bvh() over the first *out_count merged surfels); the primary
 *   segment and the bounce segments k < lod_from_bounce trace scene.  With
 *   lod_from_bounce > max_bounces the image is the plain render's, bit for
 *   bit.  EAGPT_ERR_NOT_SUPPORTED with EAGPT_FLAG_EMITTER_SAMPLING;
 *   EAGPT_ERR_INVALID_ARGUMENT if lod_from_bounce < 1; lod_bvh is checked
 *   against lod_scene as bvh against scene.  Other arguments, buffers and
 *   errors as in eagpt_render_path_traced_range().
 * ------------------------------------------------------------------------ */
size_t eagpt_lod_workspace_bytes(int64_t n);
eagpt_status eagpt_build_lod(const eagpt_scene* scene, const eagpt_params* params, const float origin[3],
                             float cell_size, eagpt_scene_mut* out, uint64_t* out_keys, int64_t* out_count,
                             void* workspace, size_t workspace_bytes, eagpt_stream_t stream);
eagpt_status eagpt_render_path_traced_lod(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                          const eagpt_scene* lod_scene, const eagpt_bvh* lod_bvh,
                                          int32_t lod_from_bounce, const eagpt_camera* cam,
                                          const eagpt_params* params, int32_t first_sample, int32_t spp,
                                          int32_t max_bounces, int32_t rr_start_bounce, uint64_t seed,
                                          float* out_rgb, float* out_aux, float* out_samples, int64_t* out_stats,
                                          void* workspace, size_t workspace_bytes, eagpt_stream_t stream);


/* ------------------------------------------------------------------------
 * Scene editing (the paper's edits: relight / toggle emitters, recolour,
 * move selected Gaussians; teaser and Sec. 4.3; selection by boxes,
 * Appendix D).
 *
 * eagpt_select(): indices of the surfels whose centre p lies in a shape, in
 *   increasing index order.  shape 0: box, params = (lo3, hi3); shape 1:
 *   sphere, params = (centre3, radius, -, -).  params is a host array of 6.
 *   out_idx: device int32[capacity]; *out_count (device int64) receives the
 *   full count even when it exceeds capacity (then only capacity are
 *   written).  scratch: device, eagpt_select_scratch_bytes(n) bytes.
 *
 * eagpt_apply_edit(): modifies the listed surfels in place, updates the BVH
 *   records and refits; then increments scene->version and sets
 *   bvh->scene_version to it (both host structs).  Ops (idx: device int32,
 *   distinct indices; per_index: device or NULL):
 *   SET_EMISSION     e, r <- per_index (4 per surfel: e, r, g, b) or value[0..3]
 *   TOGGLE_EMISSION  e <- 1 - e; a surfel that becomes an emitter takes the
 *                    radiance per_index (3 per surfel) when given
 *   SCALE_ALBEDO     rho <- clamp(rho * value[0..2], 0, 1)
 *   TRANSLATE        p <- p + value[0..2]
 *   RIGID            value = (q_R (w,x,y,z), centre c (3), translation t (3)):
 *                    p <- R(q_R)(p - c) + c + t,  q <- q_R q
 *   Geometry ops refit the BVH (surfels keep their BVH positions); when the
 *   refit's node surface-area sum exceeds rebuild_ratio times the area at
 *   build (rebuild_ratio > 0), the BVH is rebuilt instead and *out_rebuilt
 *   (host, nullable) is set to 1.  Geometry ops read the area back, so they
 *   synchronise `stream` once; appearance ops do not.
 * ------------------------------------------------------------------------ */
typedef enum {
  EAGPT_EDIT_SET_EMISSION = 0,
  EAGPT_EDIT_TOGGLE_EMISSION = 1,
  EAGPT_EDIT_SCALE_ALBEDO = 2,
  EAGPT_EDIT_TRANSLATE = 3,
  EAGPT_EDIT_RIGID = 4
} eagpt_edit_op;

typedef struct {
  int32_t op;             /* eagpt_edit_op */
  int32_t reserved;       /* must be 0 */
  int64_t count;          /* listed surfels */
  const int32_t* idx;     /* device, count indices */
  const float* per_index; /* device or NULL */
  float value[16];
} eagpt_edit;

size_t eagpt_select_scratch_bytes(int64_t n);
eagpt_status eagpt_select(const eagpt_scene* scene, int32_t shape, const float* params, int32_t* out_idx,
                          int64_t capacity, int64_t* out_count, void* scratch, size_t scratch_bytes,
                          eagpt_stream_t stream);
eagpt_status eagpt_apply_edit(eagpt_scene_mut* scene, eagpt_bvh* bvh, const eagpt_params* params,
                              const eagpt_edit* edit, float rebuild_ratio, int32_t* out_rebuilt,
                              eagpt_stream_t stream);

/* ------------------------------------------------------------------------
 * Inserting and deleting surfels (the teaser's insert / import and delete
 * edits).  The surfel count changes, so the BVH is rebuilt in place into its
 * storage (this synchronises `stream`); scene->version and
 * bvh->scene_version are incremented.  No paper passage fixes an algorithm:
 * the result is defined as the edited list of surfels.
 *
 * eagpt_delete_surfels(): removes the surfels listed in idx (device int32,
 *   count entries; duplicates allowed) and keeps the others in their order
 *   at the front of the arrays; scene->n becomes the number kept.  Indices
 *   outside [0, n) are skipped and reported by eagpt_sync_status().
 *   scratch: device, eagpt_delete_scratch_bytes(n) bytes, 256-byte aligned.
 * eagpt_insert_surfels(): appends the src->n surfels of src (device arrays)
 *   after the scene's n; the scene arrays must hold `capacity` >= n + src->n
 *   surfels and bvh->bytes >= eagpt_bvh_bytes(n + src->n), else
 *   EAGPT_ERR_OUT_OF_MEMORY and nothing changes.
 * ------------------------------------------------------------------------ */
size_t eagpt_delete_scratch_bytes(int64_t n);
eagpt_status eagpt_delete_surfels(eagpt_scene_mut* scene, eagpt_bvh* bvh, const eagpt_params* params,
                                  const int32_t* idx, int64_t count, void* scratch, size_t scratch_bytes,
                                  eagpt_stream_t stream);
eagpt_status eagpt_insert_surfels(eagpt_scene_mut* scene, int64_t capacity, const eagpt_scene* src, eagpt_bvh* bvh,
                                  const eagpt_params* params, eagpt_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving: a persistent request loop over one resident scene (the paper's
 * edit-then-path-trace use, Sec. 3.4, served to many clients).
 *
 * A host thread runs waves: each wave takes the next samples of the admitted
 * renders, puts all their paths into one shared wavefront queue of
 * queue_paths paths (rays carry a request id) and runs the path-tracing
 * kernels once over it (continuous batching).  Requests still rendering the
 * previous scene version (admitted before an edit) are planned first, so a
 * wave holds two versions only when the older one's remaining work does not
 * fill it.  Within a version the queue is filled shortest remaining work first
 * (pixels x samples left x bounces): one sample per request while it fits,
 * the longest-admitted request always included, then the rest of the queue in
 * shortest-remaining-work order, so small requests do not wait on large ones
 * and no request starves.  Two waves are in
 * flight, each on its own stream with its own queues: the next wave is
 * planned and enqueued while the current one runs, and its first bounces
 * overlap the current wave's last ones.  A request completes when the wave
 * holding its last samples has finished.  Submitted renders are admitted before
 * the next wave, in submission order, when one of max_active request slots
 * and arena memory for the request's primary records and sums (64 bytes per
 * pixel) are free.  A request's image equals, bit for bit, what
 * eagpt_render_path_traced() renders with the same arguments: it does not
 * depend on the other requests in the mix.
 * Edits apply in submission order: renders submitted earlier finish on the
 * scene before the edit, later ones see the edit.  Two scene+BVH versions
 * are kept (the caller's and one in the arena): an edit copies the current
 * version into the other slot once no running render uses it, edits and
 * refits the copy on a stream of its own (the waves in flight keep running;
 * later waves wait for the edit) and makes it current.  The caller's scene arrays and BVH
 * storage belong to the server until eagpt_server_destroy() returns; the
 * final scene is in the slot eagpt_server_scene() reports.
 * Memory: all device memory comes from the caller's arena (device, 256-byte
 * aligned, eagpt_server_arena_bytes() for a start: the second scene version,
 * per in-flight wave 112 bytes per queue path, plus 64 bytes per admitted
 * pixel); nothing is allocated on the device.  At creation the server makes
 * two CUDA streams and a few events of its own and allocates two small
 * pinned host buffers (request tables and queue counters of the two waves).
 * An edit is done once the device has applied it.
 * Failure handling: a request past its timeout (timeout_s > 0) ends as
 * TIMED_OUT; eagpt_server_wait() takes its own timeout and returns
 * EAGPT_ERR_TIMEOUT; a CUDA error fails the running requests.
 * ------------------------------------------------------------------------ */
typedef struct eagpt_server_t* eagpt_server;

typedef struct {
  void* arena;            /* device, caller-owned */
  size_t arena_bytes;
  int64_t queue_paths;    /* paths of one wave (all requests), >= the largest image's pixels */
  int32_t max_active;     /* request slots, 1..64 */
  float rebuild_ratio;    /* refit-vs-rebuild threshold for geometry edits (e.g. 1.5) */
} eagpt_server_config;

typedef struct {
  eagpt_camera cam;
  int32_t spp, max_bounces, rr_start_bounce;
  uint64_t seed;
  float* out_rgb;         /* device, H x W x 3; written when the request is done */
  double timeout_s;       /* 0: none */
} eagpt_render_request;

typedef enum {
  EAGPT_REQ_QUEUED = 0,
  EAGPT_REQ_RUNNING = 1,
  EAGPT_REQ_DONE = 2,
  EAGPT_REQ_FAILED = 3,
  EAGPT_REQ_CANCELLED = 4,
  EAGPT_REQ_TIMED_OUT = 5
} eagpt_request_state;

typedef struct {
  int32_t state;          /* eagpt_request_state */
  int32_t rebuilt;        /* edits: the BVH was rebuilt */
  double t_submit, t_admit, t_done;  /* seconds, steady clock */
  uint64_t scene_version; /* version the request rendered (or produced) */
} eagpt_request_info;

typedef struct {
  int64_t submitted, admitted, completed, failed, edits, rebuilds, waves;
  int64_t segments, paths;  /* traced in all waves (primary segments included) */
  double busy_s;            /* wall time spent in waves */
  int64_t arena_free_bytes;
} eagpt_server_stats;

size_t eagpt_server_arena_bytes(int64_t n, int64_t queue_paths);
eagpt_status eagpt_server_create(const eagpt_scene_mut* scene, const eagpt_bvh* bvh, const eagpt_params* params,
                                 const eagpt_server_config* cfg, eagpt_server* out);
eagpt_status eagpt_server_submit_render(eagpt_server server, const eagpt_render_request* req, uint64_t* out_id);
/* idx and per_index of the edit must stay valid until the edit is done */
eagpt_status eagpt_server_submit_edit(eagpt_server server, const eagpt_edit* edit, uint64_t* out_id);
eagpt_status eagpt_server_poll(eagpt_server server, uint64_t id, eagpt_request_info* out);
eagpt_status eagpt_server_wait(eagpt_server server, uint64_t id, double timeout_s, eagpt_request_info* out);
eagpt_status eagpt_server_cancel(eagpt_server server, uint64_t id);
eagpt_status eagpt_server_get_stats(eagpt_server server, eagpt_server_stats* out);
eagpt_status eagpt_server_scene(eagpt_server server, eagpt_scene_mut* scene, eagpt_bvh* bvh);
eagpt_status eagpt_server_destroy(eagpt_server server);

/* ------------------------------------------------------------------------
 * Allocation-free path-traced render.  The paper has no counterpart: this is
 * a deployment variant of eagpt_render_path_traced() for callers that cannot
 * allocate device memory themselves -- a plugin inside a host application
 * whose memory manager owns the device heap, or a latency-critical loop that
 * must not pay for cudaMalloc.  It renders exactly what
 * eagpt_render_path_traced() renders (same kernels, same arguments, no aux,
 * sample or stats output) but takes its workspace from a fixed scratch array
 * of eagpt_render_path_traced_noalloc_max_bytes() bytes (32 MiB) compiled
 * into the library; every GPU that loads the library holds that array until
 * the process exits.  The call itself allocates nothing.
 *  - Size limit: a render whose smallest workspace (one sample per pass,
 *    eagpt_render_workspace_min_bytes(), of kind 2 with emitter sampling)
 *    exceeds the scratch is rejected with EAGPT_ERR_INVALID_ARGUMENT and a
 *    message naming both sizes.  Larger
 *    renders fit in fewer samples per pass; results do not depend on it.
 *  - Set-up: the first call on each device looks up the scratch's device
 *    address (cudaGetSymbolAddress, with that device current) and caches it;
 *    make that first call before any stream capture begins.  The cached
 *    address is that of the device's context at the first call: a process
 *    that resets the device (cudaDeviceReset) must not call this entry point
 *    on that device afterwards.
 *  - Sharing: all calls on a device share the one scratch array, which keeps
 *    the last call's contents (the render zeroes what it needs zeroed).  Calls
 *    whose work overlaps on the GPU (different streams, or different host
 *    threads) race on it: serialise them, e.g. on one stream.
 *  - out_rgb: device, H x W x 3. */
size_t eagpt_render_path_traced_noalloc_max_bytes(void);
eagpt_status eagpt_render_path_traced_noalloc(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                              const eagpt_camera* cam, const eagpt_params* params, int32_t spp,
                                              int32_t max_bounces, int32_t rr_start_bounce, uint64_t seed,
                                              float* out_rgb, eagpt_stream_t stream);

/* ------------------------------------------------------------------------
 * Adjoint of the single-bounce render (Eq. 6; differentiable 2D Gaussian ray
 * tracing, Sec. 3.2-3.3, with the gradient of Eq. 7 extended from the albedo
 * to every surfel parameter).  For L = sum_p sum_c dL_drgb[p][c] * I[p][c]
 * with I the image eagpt_render_single_bounce() renders with the same
 * arguments, adds dL/dtheta to `grads` (device arrays, accumulated +=):
 * through both segments, through the bounce origin X(D~) + offset N~ and the
 * cosine direction w'(N~); discrete decisions (support, alpha limits, the
 * transmittance stop, tau_E) are held fixed.  Hit lists are recomputed (every
 * segment is re-traced), so the workspace is O(pixels x samples per pass).
 *   dL_drgb   device, H x W x 3
 *   workspace eagpt_render_backward_workspace_bytes() (full speed) or at
 *             least eagpt_render_backward_workspace_min_bytes(); 256-byte
 *             aligned
 * FP32 atomics: the summation order of the gradients is not deterministic. */
size_t eagpt_render_backward_workspace_bytes(const eagpt_camera* cam, int32_t spp);
size_t eagpt_render_backward_workspace_min_bytes(const eagpt_camera* cam, int32_t spp);

/* Forward-to-adjoint sample cache (Eq. 6 and its adjoint).  The adjoint of
 * the single-bounce render needs, for every sample, the blended radiance R
 * and transmittance T of its secondary segment (the suffix sums of the
 * front-to-back adjoint of Eq. 2 are R - R_<=i); without a cache it re-traces
 * each secondary segment once for them before the adjoint pass.  The cached
 * forward stores them, and the cached adjoint reads them instead of tracing:
 * one traversal per secondary segment fewer, for 16 bytes per sample of
 * device memory.
 *   sample_cache device, eagpt_single_bounce_cache_bytes() bytes, 16-byte
 *                aligned: float4 (R, T) per (sample, pixel), sample-major
 *                (index sample * W * H + pixel); entries of pixels whose
 *                primary segment misses or is emissive are not written.
 * eagpt_render_single_bounce_cached() renders exactly the image
 * eagpt_render_single_bounce() renders (same kernels and arithmetic; no aux
 * or sample output) and fills the cache.  Its R and T are the bits the
 * adjoint's own trace would produce, so
 * eagpt_render_single_bounce_backward_cached(), given the cache of a
 * forward with the same scene, BVH, camera, params, spp and seed, adds the
 * same gradients as eagpt_render_single_bounce_backward() (up to the
 * nondeterministic order of the FP32 atomics).  A cache from other
 * arguments, or a scene edited in between, gives wrong gradients; nothing
 * checks it.  Workspaces as for the uncached calls.  The forward returns
 * EAGPT_ERR_NOT_SUPPORTED when the library was built without the per-lane
 * refill bounce kernel. */
size_t eagpt_single_bounce_cache_bytes(const eagpt_camera* cam, int32_t spp);
eagpt_status eagpt_render_single_bounce_cached(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                               const eagpt_camera* cam, const eagpt_params* params, int32_t spp,
                                               uint64_t seed, float* out_rgb, float* sample_cache, void* workspace,
                                               size_t workspace_bytes, eagpt_stream_t stream);
eagpt_status eagpt_render_single_bounce_backward_cached(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                                        const eagpt_camera* cam, const eagpt_params* params,
                                                        int32_t spp, uint64_t seed, const float* dL_drgb,
                                                        const float* sample_cache, const eagpt_scene_grad* grads,
                                                        void* workspace, size_t workspace_bytes,
                                                        eagpt_stream_t stream);
eagpt_status eagpt_render_single_bounce_backward(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                                 const eagpt_camera* cam, const eagpt_params* params,
                                                 int32_t spp, uint64_t seed, const float* dL_drgb,
                                                 const eagpt_scene_grad* grads, void* workspace,
                                                 size_t workspace_bytes, eagpt_stream_t stream);

/* ------------------------------------------------------------------------
 * Radiant-scene (0-bounce) render and its adjoint.  Each pixel shows the
 * blended radiance R of its pixel-centre primary segment (Eq. 1-2 applied to
 * the per-surfel radiance r), the image a radiant scene (Sec. 3.2) and a
 * light-baked scene (Eq. 10) are viewed as.  No sampling; deterministic.
 *   out_rgb  device, H x W x 3 (written; 0 where the ray misses)
 *   out_aux  device or NULL, H x W x 12: the primary record per pixel in
 *            the layout eagpt_render_single_bounce() writes
 * The backward adds, for L = sum dL_drgb[p][c] * R[p][c], dL/dtheta into
 * `grads` (device arrays, +=) through the positions, rotations, scales,
 * opacities and radiances of every blended surfel; support, alpha limits and
 * the transmittance stop are held fixed.  FP32 atomics: the summation order is
 * not deterministic.  No workspace; no allocation. */
eagpt_status eagpt_render_radiance(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                                   const eagpt_params* params, float* out_rgb, float* out_aux,
                                   eagpt_stream_t stream);
eagpt_status eagpt_render_radiance_backward(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                                            const eagpt_params* params, const float* dL_drgb,
                                            const eagpt_scene_grad* grads, eagpt_stream_t stream);

/* ------------------------------------------------------------------------
 * Optimisation of the shading parameters (Stage 1, Eq. 7: albedo rho through
 * the single-bounce render with r fixed; light baking, Eq. 10: radiance r
 * through the 0-bounce render).  Geometry is not changed, so the BVH stays
 * valid; the updates are written to the scene and to the BVH's own copy.
 * ------------------------------------------------------------------------ */

/* Single-bounce render (Eq. 6) that also writes, per pixel, the incident
 * radiance estimate L_i = mean_s R(w_s) that multiplies P in Eq. 6 (0 for
 * emitter and missed pixels), the factor the albedo gradient needs.  out_rgb
 * equals eagpt_render_single_bounce()'s up to FP32 rounding (P is applied to
 * the sample mean instead of to each sample).  out_li: device, H x W x 3.
 * Workspace as for eagpt_render_single_bounce(). */
eagpt_status eagpt_render_single_bounce_incident(const eagpt_scene* scene, const eagpt_bvh* bvh,
                                                 const eagpt_camera* cam, const eagpt_params* params, int32_t spp,
                                                 uint64_t seed, float* out_rgb, float* out_li, void* workspace,
                                                 size_t workspace_bytes, eagpt_stream_t stream);

/* Gradient of L = sum dL_drgb[p][c] * I[p][c] with respect to one shading
 * field, through the primary segment's blend (Eq. 2) with its decisions held
 * fixed: each blended surfel i of pixel p gets w_i g_p added (w_i =
 * T_{i-1} alpha_i).
 *   field 0: albedo rho of the single-bounce image (Eq. 6-7), g_p =
 *            dL_drgb[p] (.) li[p], li from eagpt_render_single_bounce_incident
 *            with the same scene, camera, spp and seed
 *   field 1: radiance r of the 0-bounce image (Eq. 10), g_p = dL_drgb[p];
 *            li must be NULL
 *   grad     device, n x 3, accumulated (+=); FP32 atomics (the summation
 *            order is not deterministic). */
eagpt_status eagpt_render_shading_backward(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_camera* cam,
                                           const eagpt_params* params, int32_t field, const float* dL_drgb,
                                           const float* li, float* grad, eagpt_stream_t stream);

/* The colour loss of Eq. 7 and Eq. 10 on n linear values (e.g. H x W x 3):
 *   L = lambda_c / n * sum_k | PQ(pred_k / peak) - PQ(target_k / peak) |
 * with PQ the SMPTE ST 2084 inverse EOTF (Sec. 3.2) and the normalised value
 * clamped to [1e-10, 1] (derivative 0 where the clamp is active); peak = the
 * linear value mapped to PQ 1 (10000 cd/m^2).  out_grad (device, n, written,
 * or NULL) = dL/dpred, sign(0) = 0; out_loss (device, one double, or NULL).
 * The loss is summed in FP64 in a fixed order (deterministic).  scratch:
 * device, eagpt_pq_l1_scratch_bytes(n) bytes, 8-byte aligned. */
size_t eagpt_pq_l1_scratch_bytes(int64_t n);
eagpt_status eagpt_pq_l1_loss(const float* pred, const float* target, int64_t n, float peak, float lambda_c,
                              float* out_grad, double* out_loss, void* scratch, size_t scratch_bytes,
                              eagpt_stream_t stream);

/* Adam (Kingma and Ba 2015, Algorithm 1) with bias correction, followed by a
 * projection of the parameter onto [lo, hi]. */
typedef struct {
  float lr, beta1, beta2, eps;
  float lo, hi;
} eagpt_adam;

/* One Adam step t = step (>= 1) on n parameters (device arrays, updated in
 * place; m and v start at 0 for step 1).  zero_grad != 0 clears grad after
 * reading it. */
eagpt_status eagpt_adam_step(float* param, float* grad, float* m, float* v, int64_t n, const eagpt_adam* cfg,
                             int64_t step, int32_t zero_grad, eagpt_stream_t stream);

/* The optimisation loop, one call for `iters` steps with no host
 * synchronisation: per step, view v = view_order[k] (host, iters entries) or,
 * when view_order is NULL, (first_step + k) mod n_views; render (field 0:
 * eagpt_render_single_bounce_incident with spp and seed + step; field 1:
 * eagpt_render_radiance), the PQ-L1 loss against targets[v], the shading
 * gradient, an Adam step t = first_step + k + 1 on the field (lo/hi
 * projection), written to the scene and the BVH.  Afterwards scene->version
 * and bvh->scene_version are both incremented once.
 *   cams         host, n_views cameras
 *   targets      host array of n_views device pointers (H_v x W_v x 3)
 *   m, v         device, n x 3 each: the Adam moments (caller-owned; zero
 *                before the first step)
 *   out_loss     device, iters doubles (the loss of each step before its
 *                update), or NULL
 *   workspace    eagpt_fit_workspace_bytes(); 256-byte aligned */
typedef struct {
  int32_t field;      /* 0 albedo (Eq. 7), 1 radiance (Eq. 10) */
  int32_t spp;        /* single-bounce samples per pixel (field 0) */
  uint64_t seed;      /* step t renders with seed + t */
  float peak;         /* PQ normalisation (see eagpt_pq_l1_loss) */
  float lambda_c;
  eagpt_adam adam;
} eagpt_fit_config;

size_t eagpt_fit_workspace_bytes(const eagpt_fit_config* cfg, const eagpt_camera* cams, int32_t n_views, int64_t n);
eagpt_status eagpt_fit(const eagpt_fit_config* cfg, eagpt_scene_mut* scene, eagpt_bvh* bvh, const eagpt_params* params,
                       const eagpt_camera* cams, const float* const* targets, int32_t n_views,
                       const int32_t* view_order, int64_t first_step, int32_t iters, float* m, float* v,
                       double* out_loss, void* workspace, size_t workspace_bytes, eagpt_stream_t stream);

/* ------------------------------------------------------------------------
 * Tracing of caller rays (the per-segment operation of Eq. 1-3).
 *   rays     device, n_rays x 6: origin (3), unit direction (3); hits need
 *            t > 0
 *   mode     0: radiance as stored; 1: radiance of non-emitters dropped
 *   out_rec  device, n_rays x 12: N~ (3), D~, R (3), E, P (3), A
 *   out_hits device or NULL, n_rays x max_hits blended surfel indices in
 *            blending order (-1 padded); out_nhits device or NULL, n_rays
 * ------------------------------------------------------------------------ */
eagpt_status eagpt_trace_rays(const eagpt_scene* scene, const eagpt_bvh* bvh, const eagpt_params* params,
                              int32_t mode, const float* rays, int64_t n_rays, float* out_rec,
                              int32_t* out_hits, int32_t max_hits, int32_t* out_nhits,
                              eagpt_stream_t stream);

/* ------------------------------------------------------------------------
 * Launch accounting (host side, no device memory).
 * eagpt_launch_count(): kernels this library has launched in this process.
 * eagpt_profile_begin(): from now on, CUDA events are recorded on the
 *   launching stream around every kernel launch of this library.
 * eagpt_profile_end(): waits for those events, writes up to `capacity`
 *   per-kernel aggregates (host array) and stops recording; *n_out gets the
 *   number of distinct kernels.  Not a paper operation: measurement only.
 * ------------------------------------------------------------------------ */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
} eagpt_kernel_time;

int64_t eagpt_launch_count(void);
eagpt_status eagpt_profile_begin(void);
eagpt_status eagpt_profile_end(eagpt_kernel_time* out, int32_t capacity, int32_t* n_out);

/* ------------------------------------------------------------------------
 * Device status: synchronises `stream`, returns and clears the device-side
 * error word (EAGPT_ERR_DEVICE_CHECK when any kernel recorded an error).
 * ------------------------------------------------------------------------ */
eagpt_status eagpt_sync_status(eagpt_stream_t stream);
const char* eagpt_last_error(void);
const char* eagpt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EAGPT_H */
