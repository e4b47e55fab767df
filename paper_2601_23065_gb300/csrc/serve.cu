// Continuous-batching serving loop for path-traced renders and scene edits.
//
// One host thread owns a CUDA stream and runs waves.  A wave takes the next
// slice of samples of every admitted render, generates their first bounces
// into one shared ray queue (each ray carries its request id), runs the
// bounce kernels over the shared queue, and accumulates every request's
// samples into its own pixels in sample order.  Requests submitted while a
// wave runs are admitted before the next wave when a request slot and arena
// memory are free, so their paths share the device with the running ones.
// Two waves are in flight, each on its own stream with its own ray queues,
// per-sample values and request table: the host plans and enqueues wave
// n + 1 while wave n runs, so wave n + 1's first bounces fill the GPU while
// wave n's last, short bounces drain, and the host learns of a wave's end
// from a CUDA event.  Only the accumulation is ordered across the streams (a
// request's running sums take its waves in order), and a request's primary
// records are made visible to both streams when it is admitted.  A request is
// done when the wave that holds its last samples has finished.
// A path's arithmetic and its random numbers depend only on its request
// (seed, pixel, sample, bounce), and every pixel adds its samples in order,
// so a request's image is bitwise the same alone and in any mix.
//
// Edits are applied in submission order: renders submitted before an edit see
// the old scene, later ones the new.  The server keeps two scene+BVH
// versions: an edit copies the current version into the other slot (once no
// running request uses it), edits and refits the copy on a stream of its own
// beside the waves in flight, and makes it current, while requests admitted
// earlier finish on the old version.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "trace.cuh"
#include "wave.cuh"

namespace eagpt {

EAGPT_DEFINE_ERROR_READER(take_errors_serve)

constexpr int kSrvMaxActive = 64;
constexpr int kSrvMaxBounces = 60;
constexpr int kSrvCounterWords = 2 * (kSrvMaxBounces + 2) + 8;
constexpr int kSrvK = 12;  // k-buffer of the traversal rounds

struct __align__(16) ReqDev {
  eagpt_camera cam;
  uint64_t seed;
  int64_t npix;
  int64_t path_off;  // first flattened path of this request in the wave
  int64_t pix_off;   // first flattened pixel of this request in the wave
  PrimRec* prim;
  float4* acc;
  float4* slots;
  float* out_rgb;
  int32_t spp, max_bounces, rr_start, s0, batch, version, first, last;
};

__device__ __forceinline__ int find_req(const int64_t* offs, int nreq, int64_t t) {
  int r = 0;
  for (int k = 1; k < nreq; ++k) r = offs[k] <= t ? k : r;
  return r;
}

__global__ void __launch_bounds__(kBlock) k_srv_generate(const ReqDev* __restrict__ reqs, int nreq, int64_t total,
                                                         Consts C, Ray* q_out, uint32_t* counters) {
  __shared__ int64_t offs[kSrvMaxActive];
  for (int k = threadIdx.x; k < nreq; k += blockDim.x) offs[k] = reqs[k].path_off;
  __syncthreads();
  const int64_t t = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  bool take = false;
  Ray r;
  if (t < total) {
    const int q = find_req(offs, nreq, t);
    const ReqDev& R = reqs[q];
    const int64_t local = t - R.path_off;
    const int64_t pixel = local % R.npix;
    const int sl = (int)(local / R.npix);
    const PrimRec p = R.prim[pixel];
    if (prim_is_path_start(p, C)) {
      take = first_bounce(p, C, R.cam, 1, R.max_bounces, R.rr_start, R.seed, (uint32_t)pixel, (uint32_t)(R.s0 + sl),
                          (uint32_t)q, r);
      if (!take) R.slots[local] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  const uint32_t at = warp_append(take, &counters[2 * 1]);
  if (take) q_out[at] = r;
}

// One bounce of every queued path of every admitted request, with the
// per-lane refill of the single-request bounce kernel: a lane whose segment
// is finished takes the next queued ray at once; traversal runs in chunks of
// kSrvSteps node/leaf steps.  Each ray traces the BVH version of its request;
// kMixed is false when every request of the wave uses version 0's view (the
// common case), which spares the per-ray choice between the two views.
constexpr int kSrvSteps = 64;

template <bool kMixed>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_srv_bounce(BvhView v0, BvhView v1,
                                                                   const ReqDev* __restrict__ reqs, Consts C, int k,
                                                                   const Ray* __restrict__ q_in, Ray* q_out,
                                                                   uint32_t* counters) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  __shared__ float s_blend[11 * kBlock];
  const int lane = threadIdx.x & 31;
  const uint32_t count = counters[2 * k];
  TraceCounters cnt{0, 0, 0, 0, 0};
  RayTrace<kSrvK> rt;
  SmemBlendVisitor vis(v0.shade, C, 1, s_blend + threadIdx.x, kBlock);
  uint32_t qi = 0, rq = 0;
  bool active = false, exhausted = false;
  for (;;) {
    const bool want = !active && !exhausted;
    const uint32_t wmask = __ballot_sync(0xffffffffu, want);
    if (wmask) {
      const int leader = __ffs(wmask) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&counters[2 * k + 1], (uint32_t)__popc(wmask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (want) {
        const uint32_t idx = base + (uint32_t)__popc(wmask & ((1u << lane) - 1u));
        if (idx < count) {
          qi = idx;
          rq = __float_as_uint(q_in[qi].c.w);
          const BvhView& bvh = (kMixed && reqs[rq].version) ? v1 : v0;
          ray_begin(rt, f3(q_in[qi].a), f3(q_in[qi].b), bvh);
          vis.shade = bvh.shade;
          vis.reset();
          active = true;
        } else {
          exhausted = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, active)) break;
    bool take = false;
    Ray nr;
    if (active) {
      const ReqDev& R = reqs[rq];
      const BvhView& bvh = (kMixed && R.version) ? v1 : v0;
      if (round_steps<kSrvK, false>(rt, bvh, C, s_stack + threadIdx.x, kBlock, kSrvSteps, cnt)) {
        if (round_blend<kSrvK, false>(rt, bvh, C, vis, cnt)) {
          const SegRec s = finish(vis.get());
          const Ray r = q_in[qi];
          const uint32_t pixel = __float_as_uint(r.a.w), sample = __float_as_uint(r.b.w);
          float3 contrib;
          take = shade_bounce(1, k, R.max_bounces, R.rr_start, R.seed, C, r, s, contrib, nr);
          if (!take)
            R.slots[(int64_t)(sample - (uint32_t)R.s0) * R.npix + pixel] =
                make_float4(contrib.x, contrib.y, contrib.z, 0.f);
          active = false;
        } else {
          round_next(rt, bvh);
        }
      }
    }
    __syncwarp();
    const uint32_t at = warp_append(take, &counters[2 * (k + 1)]);
    if (take) q_out[at] = nr;
  }
}

__global__ void __launch_bounds__(kBlock) k_srv_accumulate(const ReqDev* __restrict__ reqs, int nreq,
                                                           int64_t total_pix, Consts C) {
  __shared__ int64_t offs[kSrvMaxActive];
  for (int k = threadIdx.x; k < nreq; k += blockDim.x) offs[k] = reqs[k].pix_off;
  __syncthreads();
  const int64_t t = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  if (t >= total_pix) return;
  const ReqDev& R = reqs[find_req(offs, nreq, t)];
  const int64_t i = t - R.pix_off;
  const PrimRec p = R.prim[i];
  const bool hit = p.c.w >= 0.f;
  const bool emit = hit && p.b.w > C.tau_E;
  if (!hit || emit) {
    if (R.last) {
      const float3 v = emit ? f3(p.b) : make_float3(0.f, 0.f, 0.f);
      R.out_rgb[3 * i] = v.x;
      R.out_rgb[3 * i + 1] = v.y;
      R.out_rgb[3 * i + 2] = v.z;
    }
    return;
  }
  float4 a = R.first ? make_float4(0.f, 0.f, 0.f, 0.f) : R.acc[i];
  for (int s = 0; s < R.batch; ++s) {
    const float4 c = R.slots[(int64_t)s * R.npix + i];
    a.x += c.x;
    a.y += c.y;
    a.z += c.z;
  }
  if (R.last) {
    const float inv = 1.f / (float)R.spp;
    R.out_rgb[3 * i] = a.x * inv;
    R.out_rgb[3 * i + 1] = a.y * inv;
    R.out_rgb[3 * i + 2] = a.z * inv;
  } else {
    R.acc[i] = a;
  }
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over a fixed device range (256-byte granules).
class Arena {
 public:
  void init(size_t base, size_t bytes) {
    free_.clear();
    if (bytes) free_[base] = bytes;
  }
  bool alloc(size_t bytes, size_t* out) {
    bytes = align256(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *out = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align256(bytes ? bytes : 1);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_bytes() const {
    size_t s = 0;
    for (auto& kv : free_) s += kv.second;
    return s;
  }

 private:
  std::map<size_t, size_t> free_;
};

struct Req {
  uint64_t id = 0;
  int kind = 0;  // 0 render, 1 edit
  eagpt_render_request rr{};
  eagpt_edit edit{};
  int32_t state = EAGPT_REQ_QUEUED;
  double t_submit = 0, t_admit = 0, t_done = 0, deadline = 0;
  int version = 0;
  uint64_t scene_version = 0;
  int64_t npix = 0;
  int s_next = 0;
  size_t off = 0, bytes = 0;
  int32_t rebuilt = 0;
  int inflight = 0;  // waves in flight that hold samples of this request
};

}  // namespace

struct Server {
  eagpt_params params{};
  eagpt_server_config cfg{};
  eagpt_scene_mut scene[2]{};
  eagpt_bvh bvh[2]{};
  int current = 0;
  int users[2] = {0, 0};  // running renders per version
  char* base = nullptr;
  // per wave slot: stream, two ray queues, per-sample values (queue_cap of
  // them), queue counters
  cudaStream_t streams[2] = {nullptr, nullptr};
  Ray* q[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  float4* slots[2] = {nullptr, nullptr};
  uint32_t* counters[2] = {nullptr, nullptr};
  int64_t queue_cap = 0;
  cudaEvent_t ev_ref = nullptr;   // time origin of the busy-time account
  cudaEvent_t ev_sync = nullptr;  // cross-stream ordering (admission)
  cudaStream_t edit_stream = nullptr;  // edits: their own stream, waited for by both wave streams
  cudaEvent_t ev_edit = nullptr;
  cudaEvent_t ev_acc[2] = {nullptr, nullptr};
  float last_done_ms = 0.f;
  // the two waves in flight: device request tables, their pinned host
  // sources, pinned copies of the wave's queue counters, start and end events
  struct Wave {
    bool busy = false;
    std::vector<uint64_t> ids;   // requests in the wave
    std::vector<char> last;      // the wave holds the request's last samples
    int64_t paths = 0, pixels = 0;
    int max_b = 0;
  };
  ReqDev* table_d[2] = {nullptr, nullptr};
  ReqDev* table_h[2] = {nullptr, nullptr};
  uint32_t* cnt_h[2] = {nullptr, nullptr};
  cudaEvent_t ev_start[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
  // makes the other stream wait for what `from` has enqueued so far
  cudaError_t join_other(int from) {
    cudaError_t e = cudaEventRecord(ev_sync, streams[from]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(streams[from ^ 1], ev_sync, 0);
    return e;
  }
  Wave wv[2];
  int next_slot = 0, oldest = 0, in_flight = 0;
  Arena arena;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending;
  std::map<uint64_t, Req> reqs;
  std::vector<uint64_t> active;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  eagpt_server_stats stats{};
  std::string error;

  void run();
  bool admit_locked(Req& r);
  void finish_locked(Req& r, int32_t state);
  bool apply_edit_locked(Req& r, std::unique_lock<std::mutex>& lk);
  bool plannable_locked() const;
  void release_cancelled_locked(Req& r);
  void enqueue_wave(std::unique_lock<std::mutex>& lk);
  void complete_oldest(std::unique_lock<std::mutex>& lk);
  void fail_all_locked(cudaError_t e);
};

static size_t scene_bytes(int64_t n) { return align256((size_t)(n > 0 ? n : 1) * 19 * sizeof(float)); }

bool Server::admit_locked(Req& r) {
  const int64_t npix = (int64_t)r.rr.cam.width * r.rr.cam.height;
  // the request's own memory: primary records and running sums; its
  // per-sample values of a wave live in the shared wave buffer
  const size_t bytes = align256((size_t)npix * sizeof(PrimRec)) + align256((size_t)npix * sizeof(float4));
  size_t off = 0;
  if (!arena.alloc(bytes, &off)) return false;
  r.npix = npix;
  r.off = off;
  r.bytes = bytes;
  r.version = current;
  r.scene_version = scene[current].version;
  r.s_next = 0;
  r.state = EAGPT_REQ_RUNNING;
  r.t_admit = now_s();
  users[current] += 1;
  active.push_back(r.id);
  // primary records of the request on its scene version
  PrimRec* prim = (PrimRec*)(base + off);
  launch_primary_records(bvh_view(bvh[current]), make_consts(params), r.rr.cam, 1, npix, prim, streams[next_slot]);
  join_other(next_slot);  // the request's later waves may run on the other stream
  stats.admitted += 1;
  return true;
}

void Server::finish_locked(Req& r, int32_t state) {
  if (r.state == EAGPT_REQ_RUNNING) {
    arena.release(r.off, r.bytes);
    users[r.version] -= 1;
    active.erase(std::remove(active.begin(), active.end(), r.id), active.end());
  }
  r.state = state;
  r.t_done = now_s();
  if (state == EAGPT_REQ_DONE) stats.completed += 1;
  else stats.failed += 1;
  cv_done.notify_all();
}

bool Server::apply_edit_locked(Req& r, std::unique_lock<std::mutex>& lk) {
  const int target = 1 - current;
  if (users[target] > 0) return false;  // the other version is still rendering
  const int64_t n = scene[current].n;
  // the edit runs on its own stream, beside the waves in flight (none of
  // them reads the target slot, which has no users); both wave streams wait
  // for it before their next work
  cudaStream_t st = edit_stream;
  // copy the current version into the target slot, then edit the copy
  const float* src[7] = {scene[current].pos, scene[current].quat, scene[current].scale, scene[current].opacity,
                         scene[current].albedo, scene[current].radiance, scene[current].emissive};
  float* dst[7] = {scene[target].pos, scene[target].quat, scene[target].scale, scene[target].opacity,
                   scene[target].albedo, scene[target].radiance, scene[target].emissive};
  const int width[7] = {3, 4, 2, 1, 3, 3, 1};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 7 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(dst[k], src[k], (size_t)n * width[k] * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && n > 0)
    e = cudaMemcpyAsync(bvh[target].storage, bvh[current].storage, bvh_layout(n).total, cudaMemcpyDeviceToDevice,
                        st);
  if (e != cudaSuccess) {
    error = cudaGetErrorString(e);
    finish_locked(r, EAGPT_REQ_FAILED);
    return true;
  }
  scene[target].version = scene[current].version;
  void* storage = bvh[target].storage;
  const size_t sbytes = bvh[target].bytes;
  bvh[target] = bvh[current];
  bvh[target].storage = storage;
  bvh[target].bytes = sbytes;
  const eagpt_status est =
      apply_edit_core(&scene[target], &bvh[target], &params, &r.edit, cfg.rebuild_ratio, &r.rebuilt, st);
  cudaError_t je = est == EAGPT_OK ? cudaEventRecord(ev_edit, st) : cudaErrorUnknown;
  for (int k = 0; k < 2 && je == cudaSuccess; ++k) je = cudaStreamWaitEvent(streams[k], ev_edit, 0);
  if (est != EAGPT_OK || je != cudaSuccess) {
    error = "edit failed";
    finish_locked(r, EAGPT_REQ_FAILED);
    return true;
  }
  // the edit is done when the device has applied it (callers may read the
  // edited scene, e.g. to select surfels for the next edit); the waves in
  // flight keep the GPU busy meanwhile
  lk.unlock();
  const cudaError_t se = cudaStreamSynchronize(st);
  lk.lock();
  if (se != cudaSuccess) {
    error = cudaGetErrorString(se);
    finish_locked(r, EAGPT_REQ_FAILED);
    return true;
  }
  current = target;
  r.scene_version = scene[current].version;
  r.t_admit = now_s();
  r.state = EAGPT_REQ_RUNNING;
  stats.edits += 1;
  if (r.rebuilt) stats.rebuilds += 1;
  r.state = EAGPT_REQ_DONE;
  r.t_done = now_s();
  stats.completed += 1;
  cv_done.notify_all();
  return true;
}

// Samples of each active render in the next wave.  Requests still rendering
// the previous scene version (admitted before an edit) come first, so that a
// wave holds both versions only when the older one's remaining work no longer
// fills it: two BVHs in one wave share the caches, and the plain order of a
// request stream (the renders before an edit, then the edit) renders one
// version at a time.  Within a version the queue is filled shortest
// remaining work first (pixels x samples left x bounces), which keeps small
// requests from waiting on large ones: one sample per request first, in that
// order while it fits but with the longest-admitted request ahead of all, so
// that it always progresses and no request starves; then the rest of the
// queue in shortest-remaining-work order.  The batches only change which wave
// a sample is traced in: every image still sums its samples in sample order.
static void plan_group(const std::vector<const Req*>& act, const std::vector<size_t>& group, int64_t& left,
                       std::vector<int>& batch) {
  const size_t n = group.size();
  if (!n) return;
  std::vector<size_t> order = group;
  auto work = [&](size_t k) {
    const Req& r = *act[k];
    return (double)r.npix * (double)(r.rr.spp - r.s_next) * (double)std::max(1, r.rr.max_bounces);
  };
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work(a) < work(b); });
  std::vector<size_t> first = order;
  size_t oldest = group[0];
  for (size_t k : group)
    if (act[k]->t_admit < act[oldest]->t_admit) oldest = k;
  first.erase(std::find(first.begin(), first.end(), oldest));
  first.insert(first.begin(), oldest);
  for (size_t k : first) {
    const Req& r = *act[k];
    if (r.s_next < r.rr.spp && r.npix <= left) {
      batch[k] = 1;
      left -= r.npix;
    }
  }
  for (size_t k : order) {
    const Req& r = *act[k];
    if (!batch[k]) continue;
    const int64_t more = std::min<int64_t>(r.rr.spp - r.s_next - batch[k], left / std::max<int64_t>(1, r.npix));
    batch[k] += (int)more;
    left -= more * r.npix;
  }
}

static std::vector<int> plan_wave(const std::vector<const Req*>& act, int64_t queue_cap, int current) {
  std::vector<int> batch(act.size(), 0);
  int64_t left = queue_cap;
  for (int older = 1; older >= 0; --older) {
    std::vector<size_t> group;
    for (size_t k = 0; k < act.size(); ++k)
      if ((act[k]->version != current) == (older == 1)) group.push_back(k);
    plan_group(act, group, left, batch);
  }
  return batch;
}

// A running request the caller cancelled keeps its memory until no wave in
// flight holds its samples (a later admission may reuse the memory on the
// other stream).
void Server::release_cancelled_locked(Req& r) {
  if (r.inflight > 0 || std::find(active.begin(), active.end(), r.id) == active.end()) return;
  r.state = EAGPT_REQ_RUNNING;
  finish_locked(r, EAGPT_REQ_CANCELLED);
}

bool Server::plannable_locked() const {
  for (uint64_t id : active) {
    const Req& r = reqs.at(id);
    if (r.state == EAGPT_REQ_RUNNING && r.s_next < r.rr.spp) return true;
  }
  return false;
}

void Server::fail_all_locked(cudaError_t e) {
  error = cudaGetErrorString(e);
  std::vector<uint64_t> ids = active;
  for (uint64_t id : ids) finish_locked(reqs[id], EAGPT_REQ_FAILED);
}

// Plans the next wave from the requests' sample counters, enqueues it on the
// stream and returns without waiting for it (lock held on entry and exit).
void Server::enqueue_wave(std::unique_lock<std::mutex>& lk) {
  const int slot = next_slot;
  if (wv[slot].busy) complete_oldest(lk);  // its table slot is still in use
  if (!plannable_locked()) return;
  Wave& W = wv[slot];
  W.ids.clear();
  W.last.clear();
  std::vector<const Req*> act;
  std::vector<uint64_t> act_ids;
  for (uint64_t id : active) {
    const Req& r = reqs[id];
    if (r.state == EAGPT_REQ_RUNNING && r.s_next < r.rr.spp) {
      act.push_back(&r);
      act_ids.push_back(id);
    }
  }
  const std::vector<int> plan = plan_wave(act, queue_cap, current);
  int64_t paths = 0, pixels = 0;
  int maxB = 0, nreq = 0;
  ReqDev* tab = table_h[slot];
  for (size_t k = 0; k < act.size(); ++k) {
    if (plan[k] == 0) continue;
    Req& r = reqs[act_ids[k]];
    ReqDev d{};
    d.cam = r.rr.cam;
    d.seed = r.rr.seed;
    d.npix = r.npix;
    d.path_off = paths;
    d.pix_off = pixels;
    d.prim = (PrimRec*)(base + r.off);
    d.acc = (float4*)(base + r.off + align256((size_t)r.npix * sizeof(PrimRec)));
    d.slots = slots[slot] + paths;
    d.out_rgb = r.rr.out_rgb;
    d.spp = r.rr.spp;
    d.max_bounces = r.rr.max_bounces;
    d.rr_start = r.rr.rr_start_bounce;
    d.s0 = r.s_next;
    d.batch = plan[k];
    d.version = r.version;
    d.first = r.s_next == 0;
    d.last = r.s_next + d.batch >= r.rr.spp;
    paths += r.npix * d.batch;
    pixels += r.npix;
    maxB = std::max(maxB, r.rr.max_bounces);
    tab[nreq++] = d;
    W.ids.push_back(r.id);
    W.last.push_back((char)d.last);
    r.s_next += d.batch;  // the next plan continues after this wave's samples
    r.inflight += 1;
  }
  if (nreq == 0) return;
  W.paths = paths;
  W.pixels = pixels;
  W.max_b = maxB;
  W.busy = true;
  next_slot ^= 1;
  in_flight += 1;
  const BvhView v0 = bvh_view(bvh[0]), v1 = bvh_view(bvh[1]);
  // one BVH version for the whole wave (the usual case) or a per-ray choice
  bool mixed = false;
  for (int k = 1; k < nreq; ++k) mixed |= tab[k].version != tab[0].version;
  const BvhView only = tab[0].version ? v1 : v0;
  const Consts C = make_consts(params);
  ReqDev* table = table_d[slot];
  cudaStream_t stream = streams[slot];
  uint32_t* cnt = counters[slot];
  Ray* const* qs = q[slot];
  const bool chain = in_flight > 1;  // the previous wave (other stream) may still accumulate
  lk.unlock();
  cudaError_t e = cudaEventRecord(ev_start[slot], stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(table, tab, (size_t)nreq * sizeof(ReqDev), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, kSrvCounterWords * sizeof(uint32_t), stream);
  const int grid = persistent_grid((const void*)k_srv_bounce<false>);
  const int grid_mixed = persistent_grid((const void*)k_srv_bounce<true>);
  if (e == cudaSuccess) {
    EAGPT_LAUNCH(stream, "k_srv_generate",
                 k_srv_generate<<<(unsigned)((paths + kBlock - 1) / kBlock), kBlock, 0, stream>>>(table, nreq, paths, C,
                                                                                                  qs[0], cnt));
    for (int k = 1; k <= maxB; ++k) {
      if (mixed)
        EAGPT_LAUNCH(stream, "k_srv_bounce",
                     k_srv_bounce<true><<<grid_mixed, kBlock, 0, stream>>>(v0, v1, table, C, k, qs[(k - 1) & 1],
                                                                           qs[k & 1], cnt));
      else
        EAGPT_LAUNCH(stream, "k_srv_bounce",
                     k_srv_bounce<false><<<grid, kBlock, 0, stream>>>(only, only, table, C, k, qs[(k - 1) & 1],
                                                                      qs[k & 1], cnt));
    }
    // a request's running sums take its waves in order
    if (chain) e = cudaStreamWaitEvent(stream, ev_acc[slot ^ 1], 0);
    if (e == cudaSuccess)
      EAGPT_LAUNCH(stream, "k_srv_accumulate",
                   k_srv_accumulate<<<(unsigned)((pixels + kBlock - 1) / kBlock), kBlock, 0, stream>>>(table, nreq,
                                                                                                      pixels, C));
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev_acc[slot], stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cnt_h[slot], cnt, kSrvCounterWords * sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev_done[slot], stream);
  lk.lock();
  if (e != cudaSuccess) {
    W.busy = false;
    in_flight -= 1;
    fail_all_locked(e);
  }
}

// Waits (lock released) for the oldest wave in flight, then books it: its
// segments, and the requests whose last samples it held are done.
void Server::complete_oldest(std::unique_lock<std::mutex>& lk) {
  if (in_flight == 0) return;
  const int slot = oldest;
  lk.unlock();
  cudaError_t e = cudaEventSynchronize(ev_done[slot]);
  float t_start = 0.f, t_done = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_start, ev_ref, ev_start[slot]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_done, ev_ref, ev_done[slot]);
  lk.lock();
  Wave& W = wv[slot];
  W.busy = false;
  oldest ^= 1;
  in_flight -= 1;
  stats.waves += 1;
  for (uint64_t id : W.ids) {
    auto it = reqs.find(id);
    if (it != reqs.end()) it->second.inflight -= 1;
  }
  if (e != cudaSuccess) {
    fail_all_locked(e);
    return;
  }
  // GPU time of the waves, overlapping waves counted once
  stats.busy_s += std::max(0.f, t_done - std::max(t_start, last_done_ms)) * 1e-3;
  last_done_ms = std::max(last_done_ms, t_done);
  const uint32_t* cnt = cnt_h[slot];
  int64_t segs = W.pixels;
  for (int k = 1; k <= W.max_b; ++k) segs += cnt[2 * k];
  stats.segments += segs;
  stats.paths += W.paths;
  const double t = now_s();
  for (size_t k = 0; k < W.ids.size(); ++k) {
    auto it = reqs.find(W.ids[k]);
    if (it == reqs.end()) continue;
    Req& r = it->second;
    if (r.state == EAGPT_REQ_CANCELLED) {
      release_cancelled_locked(r);
      continue;
    }
    if (r.state != EAGPT_REQ_RUNNING) continue;
    if (W.last[k]) finish_locked(r, EAGPT_REQ_DONE);
    else if (r.deadline > 0 && t > r.deadline) finish_locked(r, EAGPT_REQ_TIMED_OUT);
  }
}

void Server::run() {
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    // requests cancelled or past their deadline while queued
    const double t = now_s();
    for (auto it = pending.begin(); it != pending.end();) {
      Req& r = reqs[*it];
      if (r.state == EAGPT_REQ_CANCELLED || (r.deadline > 0 && t > r.deadline)) {
        if (r.state != EAGPT_REQ_CANCELLED) finish_locked(r, EAGPT_REQ_TIMED_OUT);
        it = pending.erase(it);
      } else {
        ++it;
      }
    }
    // running requests cancelled by the caller
    std::vector<uint64_t> ids = active;
    for (uint64_t id : ids)
      if (reqs[id].state == EAGPT_REQ_CANCELLED) release_cancelled_locked(reqs[id]);
    // admission in submission order
    while (!pending.empty()) {
      Req& r = reqs[pending.front()];
      bool done;
      if (r.kind == 1) {
        done = apply_edit_locked(r, lk);
      } else {
        done = (int)active.size() < cfg.max_active && admit_locked(r);
      }
      if (!done) break;
      pending.pop_front();
    }
    if (plannable_locked()) {
      enqueue_wave(lk);
      continue;
    }
    if (in_flight > 0) {
      complete_oldest(lk);
      continue;
    }
    if (active.empty()) {
      if (stop && pending.empty()) break;
      if (stop) {
        // nothing can be admitted any more: fail what is left
        for (uint64_t id : pending) finish_locked(reqs[id], EAGPT_REQ_FAILED);
        pending.clear();
        break;
      }
    }
    cv_work.wait_for(lk, std::chrono::milliseconds(5));
  }
}

}  // namespace eagpt

using namespace eagpt;

struct eagpt_server_t {
  Server s;
};

static void release_host(Server& S) {
  for (int k = 0; k < 2; ++k) {
    if (S.table_h[k]) cudaFreeHost(S.table_h[k]);
    if (S.cnt_h[k]) cudaFreeHost(S.cnt_h[k]);
    if (S.ev_start[k]) cudaEventDestroy(S.ev_start[k]);
    if (S.ev_done[k]) cudaEventDestroy(S.ev_done[k]);
    if (S.ev_acc[k]) cudaEventDestroy(S.ev_acc[k]);
    if (S.streams[k]) cudaStreamDestroy(S.streams[k]);
    S.table_h[k] = nullptr;
    S.cnt_h[k] = nullptr;
    S.ev_start[k] = S.ev_done[k] = S.ev_acc[k] = nullptr;
    S.streams[k] = nullptr;
  }
  if (S.ev_ref) cudaEventDestroy(S.ev_ref);
  if (S.ev_sync) cudaEventDestroy(S.ev_sync);
  if (S.ev_edit) cudaEventDestroy(S.ev_edit);
  if (S.edit_stream) cudaStreamDestroy(S.edit_stream);
  S.ev_ref = S.ev_sync = S.ev_edit = nullptr;
  S.edit_stream = nullptr;
}

// Arena bytes the server keeps for itself: the second scene version and its
// BVH, and per wave slot two ray queues, the per-sample values, the counters
// and the request table.
static size_t fixed_bytes(int64_t n, int64_t queue_paths) {
  return scene_bytes(n) + align256(bvh_layout(n).total) +
         2 * (2 * align256((size_t)queue_paths * sizeof(Ray)) + align256((size_t)queue_paths * sizeof(float4)) +
              align256(kSrvCounterWords * 4) + align256(kSrvMaxActive * sizeof(ReqDev)));
}

extern "C" {

size_t eagpt_server_arena_bytes(int64_t n, int64_t queue_paths) {
  if (n < 0 || queue_paths <= 0) return 0;
  // the server's own buffers, and primary records and sums for as many
  // pixels as the queue holds paths
  return fixed_bytes(n, queue_paths) + (size_t)queue_paths * (sizeof(float4) + sizeof(PrimRec));
}

eagpt_status eagpt_server_create(const eagpt_scene_mut* scene, const eagpt_bvh* bvh, const eagpt_params* params,
                                 const eagpt_server_config* cfg, eagpt_server* out) {
  if (!scene || !bvh || !params || !cfg || !out) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "null argument");
  if (params->flags & EAGPT_FLAG_EMITTER_SAMPLING)
    return set_error(EAGPT_ERR_NOT_SUPPORTED, "the serving loop renders without emitter sampling");
  if (cfg->max_active < 1 || cfg->max_active > kSrvMaxActive)
    return set_error(EAGPT_ERR_INVALID_ARGUMENT, "max_active must be in [1, 64]");
  if (cfg->queue_paths < 1) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "queue_paths must be positive");
  if (!cfg->arena || ((uintptr_t)cfg->arena & 255))
    return set_error(EAGPT_ERR_INVALID_ARGUMENT, "arena must be non-NULL and 256-byte aligned");
  if (bvh->scene_version != scene->version || bvh->n != scene->n)
    return set_error(EAGPT_ERR_STALE_BVH, "bvh does not match the scene");
  const int64_t n = scene->n;
  const size_t fixed = fixed_bytes(n, cfg->queue_paths);
  if (cfg->arena_bytes < fixed + 4096)
    return set_error(EAGPT_ERR_OUT_OF_MEMORY, "arena too small for the second scene version and the queues");
  eagpt_server_t* h = new eagpt_server_t();
  Server& S = h->s;
  S.params = *params;
  S.cfg = *cfg;
  S.base = (char*)cfg->arena;
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o += align256(b);
    return at;
  };
  S.scene[0] = *scene;
  S.bvh[0] = *bvh;
  // version slot 1 lives in the arena
  const size_t sc = take(scene_bytes(n));
  float* f = (float*)(S.base + sc);
  S.scene[1] = *scene;
  S.scene[1].pos = f;
  S.scene[1].quat = f + 3 * n;
  S.scene[1].scale = f + 7 * n;
  S.scene[1].opacity = f + 9 * n;
  S.scene[1].albedo = f + 10 * n;
  S.scene[1].radiance = f + 13 * n;
  S.scene[1].emissive = f + 16 * n;
  S.bvh[1] = *bvh;
  S.bvh[1].bytes = bvh_layout(n).total;
  S.bvh[1].storage = S.base + take(S.bvh[1].bytes);
  for (int k = 0; k < 2; ++k) {
    S.q[k][0] = (Ray*)(S.base + take((size_t)cfg->queue_paths * sizeof(Ray)));
    S.q[k][1] = (Ray*)(S.base + take((size_t)cfg->queue_paths * sizeof(Ray)));
    S.slots[k] = (float4*)(S.base + take((size_t)cfg->queue_paths * sizeof(float4)));
    S.counters[k] = (uint32_t*)(S.base + take(kSrvCounterWords * 4));
    S.table_d[k] = (ReqDev*)(S.base + take(kSrvMaxActive * sizeof(ReqDev)));
  }
  S.queue_cap = cfg->queue_paths;
  S.arena.init(o, cfg->arena_bytes - o);
  // set-up (not per wave): the two streams, the pinned host sides of the
  // two request tables and counter copies, the events
  cudaError_t e = cudaEventCreate(&S.ev_ref);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.ev_sync, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.ev_edit, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S.edit_stream, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&S.streams[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&S.table_h[k], kSrvMaxActive * sizeof(ReqDev), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&S.cnt_h[k], kSrvCounterWords * sizeof(uint32_t), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreate(&S.ev_start[k]);
    if (e == cudaSuccess) e = cudaEventCreate(&S.ev_done[k]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.ev_acc[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventRecord(S.ev_ref, S.streams[0]);
  if (e != cudaSuccess) {
    release_host(S);
    delete h;
    return set_error(EAGPT_ERR_CUDA, cudaGetErrorString(e));
  }
  int dev = 0;
  cudaGetDevice(&dev);
  S.worker = std::thread([&S, dev]() {
    cudaSetDevice(dev);
    S.run();
  });
  *out = h;
  return EAGPT_OK;
}

static eagpt_status submit(eagpt_server h, Req&& r, uint64_t* out_id) {
  if (!h) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "server is NULL");
  Server& S = h->s;
  std::lock_guard<std::mutex> g(S.mu);
  if (S.stop) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "server is shutting down");
  r.id = S.next_id++;
  r.t_submit = now_s();
  r.state = EAGPT_REQ_QUEUED;
  if (out_id) *out_id = r.id;
  S.pending.push_back(r.id);
  S.reqs[r.id] = r;
  S.stats.submitted += 1;
  S.cv_work.notify_one();
  return EAGPT_OK;
}

eagpt_status eagpt_server_submit_render(eagpt_server h, const eagpt_render_request* req, uint64_t* out_id) {
  if (!req || !req->out_rgb) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "request and out_rgb are required");
  if (req->cam.width <= 0 || req->cam.height <= 0 || req->spp <= 0 || req->max_bounces < 0 ||
      req->max_bounces > kSrvMaxBounces)
    return set_error(EAGPT_ERR_INVALID_ARGUMENT, "bad camera size, spp or max_bounces");
  if (h && (int64_t)req->cam.width * req->cam.height > h->s.queue_cap)
    return set_error(EAGPT_ERR_OUT_OF_MEMORY, "image has more pixels than the server's queue holds paths");
  Req r;
  r.kind = 0;
  r.rr = *req;
  r.deadline = req->timeout_s > 0 ? now_s() + req->timeout_s : 0.0;
  return submit(h, std::move(r), out_id);
}

eagpt_status eagpt_server_submit_edit(eagpt_server h, const eagpt_edit* edit, uint64_t* out_id) {
  if (!edit || edit->reserved != 0 || edit->op < EAGPT_EDIT_SET_EMISSION || edit->op > EAGPT_EDIT_RIGID ||
      edit->count < 0 || (edit->count > 0 && !edit->idx))
    return set_error(EAGPT_ERR_INVALID_ARGUMENT, "bad edit");
  Req r;
  r.kind = 1;
  r.edit = *edit;
  return submit(h, std::move(r), out_id);
}

static void fill_info(const Req& r, eagpt_request_info* out) {
  out->state = r.state;
  out->rebuilt = r.rebuilt;
  out->t_submit = r.t_submit;
  out->t_admit = r.t_admit;
  out->t_done = r.t_done;
  out->scene_version = r.scene_version;
}

eagpt_status eagpt_server_poll(eagpt_server h, uint64_t id, eagpt_request_info* out) {
  if (!h || !out) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "null argument");
  std::lock_guard<std::mutex> g(h->s.mu);
  auto it = h->s.reqs.find(id);
  if (it == h->s.reqs.end()) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "unknown request id");
  fill_info(it->second, out);
  return EAGPT_OK;
}

eagpt_status eagpt_server_wait(eagpt_server h, uint64_t id, double timeout_s, eagpt_request_info* out) {
  if (!h) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "server is NULL");
  Server& S = h->s;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.reqs.find(id);
  if (it == S.reqs.end()) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "unknown request id");
  auto finished = [&]() { return it->second.state >= EAGPT_REQ_DONE; };
  if (timeout_s > 0) {
    if (!S.cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), finished)) {
      if (out) fill_info(it->second, out);
      return set_error(EAGPT_ERR_TIMEOUT, "request not finished within the timeout");
    }
  } else {
    S.cv_done.wait(lk, finished);
  }
  if (out) fill_info(it->second, out);
  return EAGPT_OK;
}

eagpt_status eagpt_server_cancel(eagpt_server h, uint64_t id) {
  if (!h) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "server is NULL");
  std::lock_guard<std::mutex> g(h->s.mu);
  auto it = h->s.reqs.find(id);
  if (it == h->s.reqs.end()) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "unknown request id");
  Req& r = it->second;
  if (r.state == EAGPT_REQ_QUEUED) {
    r.state = EAGPT_REQ_CANCELLED;
    r.t_done = now_s();
    h->s.stats.failed += 1;
    h->s.cv_done.notify_all();
  } else if (r.state == EAGPT_REQ_RUNNING) {
    r.state = EAGPT_REQ_CANCELLED;  // released by the loop before the next wave
  }
  h->s.cv_work.notify_one();
  return EAGPT_OK;
}

eagpt_status eagpt_server_get_stats(eagpt_server h, eagpt_server_stats* out) {
  if (!h || !out) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "null argument");
  std::lock_guard<std::mutex> g(h->s.mu);
  *out = h->s.stats;
  out->arena_free_bytes = (int64_t)h->s.arena.free_bytes();
  return EAGPT_OK;
}

eagpt_status eagpt_server_scene(eagpt_server h, eagpt_scene_mut* scene, eagpt_bvh* bvh) {
  if (!h) return set_error(EAGPT_ERR_INVALID_ARGUMENT, "server is NULL");
  std::lock_guard<std::mutex> g(h->s.mu);
  if (scene) *scene = h->s.scene[h->s.current];
  if (bvh) *bvh = h->s.bvh[h->s.current];
  return EAGPT_OK;
}

eagpt_status eagpt_server_destroy(eagpt_server h) {
  if (!h) return EAGPT_OK;
  {
    std::lock_guard<std::mutex> g(h->s.mu);
    h->s.stop = true;
    h->s.cv_work.notify_all();
  }
  if (h->s.worker.joinable()) h->s.worker.join();
  cudaStreamSynchronize(h->s.streams[0]);
  cudaStreamSynchronize(h->s.streams[1]);
  release_host(h->s);
  delete h;
  return EAGPT_OK;
}

}  // extern "C"
