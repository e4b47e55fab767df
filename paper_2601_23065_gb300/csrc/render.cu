// Wavefront renderer: single-bounce estimator (Eq. 6) and path tracing (Eq. 8).
//
//   k_primary     one pinhole ray per pixel, traced once and shared by all
//                 samples (the viewing direction is fixed per pixel); writes
//                 the pixel's blended record (N~, D~, R, E, P, A).
//   k_generate    per (sample, pixel) of a sample batch: first bounce of every
//                 path of a non-emitter primary hit -> ray queue 1.
//   k_bounce<k>   persistent, warp-fetched: trace the queued ray, blend, then
//                 either end the path (its contribution goes to its own slot)
//                 or sample the next bounce and append it to queue k+1 with a
//                 warp-ballot compaction (one atomic per warp).
//   k_accumulate  per pixel: the batch's slots in sample order (deterministic,
//                 independent of the batch size), final mean.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "trace.cuh"
#include "wave.cuh"

namespace eagpt {

#ifndef EAGPT_KBUF
#define EAGPT_KBUF 12
#endif
constexpr int kK = EAGPT_KBUF;  // k-buffer size (hits collected per traversal round)

EAGPT_DEFINE_ERROR_READER(take_errors_render)

// Reorder each bounce's ray queue by (direction octant, origin Morton code)
// so that the rays of a warp walk similar parts of the BVH.
#ifndef EAGPT_SORT_RAYS
#define EAGPT_SORT_RAYS 0
#endif
constexpr bool kSortRays = EAGPT_SORT_RAYS != 0;
#ifndef EAGPT_MIS_SPLIT
#define EAGPT_MIS_SPLIT 1
#endif
constexpr bool kMisSplit = EAGPT_MIS_SPLIT != 0;
#ifndef EAGPT_PATH_PERSIST
#define EAGPT_PATH_PERSIST 0
#endif
constexpr bool kPathPersist = EAGPT_PATH_PERSIST != 0;

// Blend sums of the bounce kernel in shared memory instead of registers.
#ifndef EAGPT_SMEM_BLEND
#define EAGPT_SMEM_BLEND 1
#endif

__global__ void k_ray_keys(const Ray* __restrict__ q, const uint32_t* __restrict__ count_ptr, int64_t cap,
                           const uint32_t* __restrict__ bounds_bits, uint32_t* keys, uint32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= cap) return;
  const uint32_t count = *count_ptr;
  uint32_t key = 0xFFFFFFFFu;
  if (i < count) {
    const float4 a = q[i].a, b = q[i].b;
    const float lo0 = ord2f(bounds_bits[0]), lo1 = ord2f(bounds_bits[1]), lo2 = ord2f(bounds_bits[2]);
    const float hi0 = ord2f(bounds_bits[3]), hi1 = ord2f(bounds_bits[4]), hi2 = ord2f(bounds_bits[5]);
    const float ext = fmaxf(fmaxf(hi0 - lo0, hi1 - lo1), fmaxf(hi2 - lo2, 1e-20f));
    const float sc = 511.0f / ext;
    const uint32_t x = (uint32_t)fminf(fmaxf((a.x - lo0) * sc, 0.f), 511.f);
    const uint32_t y = (uint32_t)fminf(fmaxf((a.y - lo1) * sc, 0.f), 511.f);
    const uint32_t z = (uint32_t)fminf(fmaxf((a.z - lo2) * sc, 0.f), 511.f);
    const uint32_t oct = (b.x < 0.f ? 4u : 0u) | (b.y < 0.f ? 2u : 0u) | (b.z < 0.f ? 1u : 0u);
    key = (oct << 27) | (expand_bits10(x) << 2) | (expand_bits10(y) << 1) | expand_bits10(z);
  }
  keys[i] = key;
  vals[i] = (uint32_t)i;
}

// counters block: per bounce k, [2k] = rays queued for bounce k, [2k+1] = fetch
constexpr int kMaxBounces = 60;
// per bounce k: queue length (2k) and fetch index (2k + 1); then the fetch
// indices of the emitter-sample pass (kNeeFetch + k)
constexpr int kNeeFetch = 2 * (kMaxBounces + 2) + 8;
constexpr int kCounterWords = kNeeFetch + kMaxBounces + 2;

RenderLayout render_layout(int64_t npix, int spp, int batch_spp, bool mis) {
  RenderLayout L{};
  L.npix = npix;
  L.batch_spp = batch_spp;
  L.batch_paths = npix * (int64_t)batch_spp;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.prim = take((size_t)npix * sizeof(PrimRec));
  L.acc = take((size_t)npix * sizeof(float4));
  L.slots = take((size_t)L.batch_paths * sizeof(float4));
  L.q0 = take((size_t)L.batch_paths * sizeof(Ray));
  L.q1 = take((size_t)L.batch_paths * sizeof(Ray));
  L.counters = take(kCounterWords * sizeof(uint32_t));
  if (mis) {
    L.e0 = take((size_t)L.batch_paths * sizeof(RayExt));
    L.e1 = take((size_t)L.batch_paths * sizeof(RayExt));
  }
  if (kSortRays) {
    L.sk0 = take((size_t)L.batch_paths * 4);
    L.sk1 = take((size_t)L.batch_paths * 4);
    L.sv0 = take((size_t)L.batch_paths * 4);
    L.sv1 = take((size_t)L.batch_paths * 4);
    L.shist = take((size_t)256 * ((L.batch_paths + kSortTileItems - 1) / kSortTileItems) * 4);
  }
  L.total = o;
  (void)spp;
  return L;
}

int choose_batch_spp(int64_t npix, int spp, size_t ws_bytes, bool mis) {
  int lo = 1, hi = spp;
  if (render_layout(npix, spp, 1, mis).total > ws_bytes) return 0;
  while (lo < hi) {  // largest batch that fits
    const int mid = lo + (hi - lo + 1) / 2;
    if (render_layout(npix, spp, mid, mis).total <= ws_bytes) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// --------------------------------------------------------------------------
__device__ __forceinline__ void write_aux(float* aux, int64_t i, const SegRec& s) {
  float* o = aux + 12 * i;
  o[0] = s.Nn.x;
  o[1] = s.Nn.y;
  o[2] = s.Nn.z;
  o[3] = s.Dn;
  o[4] = s.R.x;
  o[5] = s.R.y;
  o[6] = s.R.z;
  o[7] = s.E;
  o[8] = s.P.x;
  o[9] = s.P.y;
  o[10] = s.P.z;
  o[11] = s.A;
}

__device__ __forceinline__ void add_stats(int64_t* stats, int slot, uint32_t v) {
  // warp-aggregated counter update
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd((unsigned long long*)(stats + slot), (unsigned long long)v);
}

template <bool kCount>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_primary(BvhView bvh, Consts C, eagpt_camera cam, int mode, int64_t npix,
                                                    PrimRec* prim, float* aux, int64_t* stats) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  const int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  TraceCounters cnt{0, 0, 0, 0, 0};
  if (i < npix) {
    float3 O, w;
    camera_ray(cam, (uint32_t)i, O, w);
    BlendVisitor vis(bvh.shade, C, w, mode);
    trace_segment<kK, kCount>(bvh, C, O, w, 0.f, s_stack + threadIdx.x, kBlock, vis, cnt);
    const SegRec s = finish(vis.b);
    PrimRec p;
    p.a = make_float4(s.Nn.x, s.Nn.y, s.Nn.z, s.Dn);
    p.b = make_float4(s.R.x, s.R.y, s.R.z, s.E);
    p.c = make_float4(s.P.x, s.P.y, s.P.z, s.hit ? s.A : -1.f);  // A < 0 marks a miss
    prim[i] = p;
    if (aux) write_aux(aux, i, s);
  }
  if (kCount) {
    add_stats(stats, 0, i < npix ? 1u : 0u);
    add_stats(stats, 8, cnt.blended);
    add_stats(stats, 9, cnt.nodes);
    add_stats(stats, 10, cnt.tests);
    add_stats(stats, 11, cnt.rounds);
  }
}

// First bounce of every path of the batch [s0, s0 + batch) (Sec. 3.1 "Light
// Bouncing"): X = O + D~ w, throughput P (the cosine pdf cancels cos/pi of
// the diffuse BRDF), cosine-weighted direction about N~ from X + offset N~.
template <bool kCount>
__global__ void __launch_bounds__(kBlock) k_generate(const PrimRec* __restrict__ prim, Consts C, eagpt_camera cam,
                                                     int kind, int max_bounces, int rr_start, uint64_t seed, int64_t npix,
                                                     int s0, int batch, Ray* q_out, uint32_t* counters, float4* slots,
                                                     int64_t* stats, RayExt* e_out) {
  const int64_t t = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  const int64_t total = npix * (int64_t)batch;
  bool take = false;
  Ray r;
  int64_t slot = 0;
  bool started = false;
  if (t < total) {
    const int64_t pixel = t % npix;
    const int sl = (int)(t / npix);
    slot = t;
    const PrimRec p = prim[pixel];
    if (prim_is_path_start(p, C)) {
      started = true;
      take = first_bounce(p, C, cam, kind, max_bounces, rr_start, seed, (uint32_t)pixel, (uint32_t)(s0 + sl), 0u, r);
      if (!take) slots[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  const uint32_t at = warp_append(take, &counters[2 * 1]);
  if (take) {
    q_out[at] = r;
    if (e_out) {
      // the first reflection leaves the primary vertex: its normal, the
      // cosine pdf of the direction, nothing gathered yet
      const PrimRec p = prim[t % npix];
      const float3 Nn = make_float3(p.a.x, p.a.y, p.a.z);
      RayExt x;
      x.n = make_float4(Nn.x, Nn.y, Nn.z, dot3(f3(r.b), Nn) * 0.318309886183790672f);
      x.l = make_float4(0.f, 0.f, 0.f, 0.f);
      e_out[at] = x;
    }
  }
  if (kCount) add_stats(stats, 2, started ? 1u : 0u);
}

// One bounce k of every queued path (Eq. 6 for kind 0, Eq. 8 for kind 1).
template <bool kCount>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_bounce(BvhView bvh, Consts C, int kind, int k, int max_bounces,
                                                   int rr_start, uint64_t seed, int64_t npix, int s0,
                                                   const Ray* __restrict__ q_in, Ray* q_out, uint32_t* counters,
                                                   float4* slots, int64_t* stats, const uint32_t* __restrict__ perm) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
#if EAGPT_SMEM_BLEND
  __shared__ float s_blend[11 * kBlock];
#endif
  const int lane = threadIdx.x & 31;
  const uint32_t count = counters[2 * k];
  const int mode = kind == 1 ? 1 : 0;
  TraceCounters cnt{0, 0, 0, 0, 0};
  uint32_t traced = 0;
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&counters[2 * k + 1], 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= count) break;
    const uint32_t idx = base + lane;
    bool take = false;
    Ray nr;
    const uint32_t work0 = cnt.nodes + cnt.tests;
    if (idx < count) {
      ++traced;
      const uint32_t qi = perm ? perm[idx] : idx;
#if EAGPT_SMEM_BLEND
      // origin and direction stay in registers for the traversal; pixel,
      // sample, throughput and tag are read again after it (volatile loads,
      // so the first read is not kept alive across the trace)
      const float4 ra = q_in[qi].a, rb = q_in[qi].b;
      const float3 O = f3(ra), w = f3(rb);
      SmemBlendVisitor vis(bvh.shade, C, mode, s_blend + threadIdx.x, kBlock);
      trace_segment<kK, kCount>(bvh, C, O, w, 0.f, s_stack + threadIdx.x, kBlock, vis, cnt);
      const SegRec s = finish(vis.get());
      Ray r;
      r.a = make_float4(O.x, O.y, O.z, __ldcv(&q_in[qi].a.w));
      r.b = make_float4(w.x, w.y, w.z, __ldcv(&q_in[qi].b.w));
      r.c = __ldcv(&q_in[qi].c);
#else
      const Ray r = q_in[qi];
      const float3 O = f3(r.a), w = f3(r.b);
      BlendVisitor vis(bvh.shade, C, w, mode);
      trace_segment<kK, kCount>(bvh, C, O, w, 0.f, s_stack + threadIdx.x, kBlock, vis, cnt);
      const SegRec s = finish(vis.b);
#endif
      const uint32_t pixel = __float_as_uint(r.a.w), sample = __float_as_uint(r.b.w);
      float3 contrib;
      take = shade_bounce(kind, k, max_bounces, rr_start, seed, C, r, s, contrib, nr);
      if (!take) slots[(int64_t)(sample - (uint32_t)s0) * npix + pixel] = make_float4(contrib.x, contrib.y, contrib.z, 0.f);
    }
    __syncwarp();
    if (kCount) {
      // balance of the batch: the lanes' work against 32 x the slowest lane's
      const uint32_t wr = cnt.nodes + cnt.tests - work0;
      uint32_t mx = wr;
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      add_stats(stats, 12, wr);
      add_stats(stats, 13, lane == 0 ? 32u * mx : 0u);
    }
    const uint32_t at = warp_append(take, &counters[2 * (k + 1)]);
    if (take) q_out[at] = nr;
  }
  if (kCount) {
    add_stats(stats, 1, traced);
    add_stats(stats, 3, cnt.blended);
    add_stats(stats, 4, cnt.nodes);
    add_stats(stats, 5, cnt.tests);
    add_stats(stats, 6, cnt.rounds);
    uint32_t m = cnt.max_stack;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax((unsigned long long*)(stats + 7), (unsigned long long)m);
  }
}

// The bounce kernel with per-lane refill: a lane whose segment is finished
// takes the next queued ray at once (one atomic per warp for all the lanes
// that want one) instead of waiting for the slowest ray of a 32-ray batch.
// Traversal runs in chunks of kRefillSteps node/leaf steps; between chunks
// the lanes whose round is complete blend it, and finished segments are shaded
// and their continuation appended (warp-ballot compaction, as in k_bounce).
#ifndef EAGPT_REFILL
#define EAGPT_REFILL 1
#endif
#ifndef EAGPT_REFILL_STEPS
#define EAGPT_REFILL_STEPS 64
#endif
constexpr int kRefillSteps = EAGPT_REFILL_STEPS;
bool render_has_refill() { return EAGPT_REFILL != 0; }

template <bool kCount, bool kCache = false>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_bounce_r(BvhView bvh, Consts C, int kind, int k, int max_bounces,
                                                     int rr_start, uint64_t seed, int64_t npix, int s0,
                                                     const Ray* __restrict__ q_in, Ray* q_out, uint32_t* counters,
                                                     float4* slots, int64_t* stats, const uint32_t* __restrict__ perm,
                                                     float4* sb_cache) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  __shared__ float s_blend[11 * kBlock];
  const int lane = threadIdx.x & 31;
  const uint32_t count = counters[2 * k];
  const int mode = kind == 1 ? 1 : 0;
  TraceCounters cnt{0, 0, 0, 0, 0};
  uint32_t traced = 0;
  RayTrace<kK> rt;
  SmemBlendVisitor vis(bvh.shade, C, mode, s_blend + threadIdx.x, kBlock);
  uint32_t qi = 0;
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
          qi = perm ? perm[idx] : idx;
          ray_begin(rt, f3(q_in[qi].a), f3(q_in[qi].b));
          round_begin(rt, bvh);
          vis.reset();
          active = true;
          ++traced;
          if (kCount) ++cnt.rounds;
        } else {
          exhausted = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, active)) break;
    bool take = false;
    Ray nr;
    if (active && round_steps<kK, kCount>(rt, bvh, C, s_stack + threadIdx.x, kBlock, kRefillSteps, cnt)) {
      if (round_blend<kK, kCount>(rt, bvh, C, vis, cnt)) {
        const Blend bl = vis.get();
        const SegRec s = finish(bl);
        const float4 rt_cache = make_float4(bl.R.x, bl.R.y, bl.R.z, bl.T);
        Ray r;
        r.a = make_float4(rt.O.x, rt.O.y, rt.O.z, __ldcv(&q_in[qi].a.w));
        r.b = make_float4(rt.w.x, rt.w.y, rt.w.z, __ldcv(&q_in[qi].b.w));
        r.c = __ldcv(&q_in[qi].c);
        const uint32_t pixel = __float_as_uint(r.a.w), sample = __float_as_uint(r.b.w);
        // single bounce: the secondary segment's R and T for the adjoint
        if (kCache) sb_cache[(int64_t)sample * npix + pixel] = rt_cache;
        float3 contrib;
        take = shade_bounce(kind, k, max_bounces, rr_start, seed, C, r, s, contrib, nr);
        if (!take)
          slots[(int64_t)(sample - (uint32_t)s0) * npix + pixel] = make_float4(contrib.x, contrib.y, contrib.z, 0.f);
        active = false;
      } else {
        round_begin(rt, bvh);
        if (kCount) ++cnt.rounds;
      }
    }
    __syncwarp();
    const uint32_t at = warp_append(take, &counters[2 * (k + 1)]);
    if (take) q_out[at] = nr;
  }
  if (kCount) {
    add_stats(stats, 1, traced);
    add_stats(stats, 3, cnt.blended);
    add_stats(stats, 4, cnt.nodes);
    add_stats(stats, 5, cnt.tests);
    add_stats(stats, 6, cnt.rounds);
    uint32_t m = cnt.max_stack;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax((unsigned long long*)(stats + 7), (unsigned long long)m);
  }
}

// Counting variant's totals of one kernel (segments traced, blended hits,
// node steps, tests, rounds, deepest stack).
__device__ __forceinline__ void flush_counts(int64_t* stats, uint32_t traced, const TraceCounters& cnt) {
  add_stats(stats, 1, traced);
  add_stats(stats, 3, cnt.blended);
  add_stats(stats, 4, cnt.nodes);
  add_stats(stats, 5, cnt.tests);
  add_stats(stats, 6, cnt.rounds);
  uint32_t m = cnt.max_stack;
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax((unsigned long long*)(stats + 7), (unsigned long long)m);
}

// Path tracing with every path kept by one lane from its first bounce to its
// end (EAGPT_PATH_PERSIST): a lane takes the next first-bounce ray from the
// generator's queue, traces and shades each of its segments in turn (the
// throughput, pixel and sample in a shared-memory payload, the bounce index in
// a register) and writes the path's slot when it ends, so one launch per pass
// replaces the per-bounce launches and their tails, and no ray goes through a
// queue between bounces.  Per path the arithmetic is k_bounce_r's.
template <bool kCount>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_path_r(BvhView bvh, Consts C, int kind, int max_bounces,
                                                   int rr_start, uint64_t seed, int64_t npix, int s0,
                                                   const Ray* __restrict__ q_in, uint32_t* counters, float4* slots,
                                                   int64_t* stats) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  __shared__ float s_blend[11 * kBlock];
  __shared__ float s_pay[5 * kBlock];  // pixel, sample (bits), throughput
  const int lane = threadIdx.x & 31;
  float* pay = s_pay + threadIdx.x;
  const uint32_t count = counters[2];
  const int mode = kind == 1 ? 1 : 0;
  TraceCounters cnt{0, 0, 0, 0, 0};
  uint32_t traced = 0;
  RayTrace<kK> rt;
  SmemBlendVisitor vis(bvh.shade, C, mode, s_blend + threadIdx.x, kBlock);
  int kb = 1;
  bool active = false, pending = false, exhausted = false;  // pending: rt holds the next segment's ray
  for (;;) {
    const bool want = !active && !pending && !exhausted;
    const uint32_t wmask = __ballot_sync(0xffffffffu, want);
    if (wmask) {
      const int leader = __ffs(wmask) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&counters[3], (uint32_t)__popc(wmask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (want) {
        const uint32_t idx = base + (uint32_t)__popc(wmask & ((1u << lane) - 1u));
        if (idx < count) {
          const Ray r = q_in[idx];
          pay[0] = r.a.w;
          pay[kBlock] = r.b.w;
          pay[2 * kBlock] = r.c.x;
          pay[3 * kBlock] = r.c.y;
          pay[4 * kBlock] = r.c.z;
          kb = 1;
          ray_begin(rt, f3(r.a), f3(r.b));
          pending = true;
        } else {
          exhausted = true;
        }
      }
    }
    if (pending) {
      round_begin(rt, bvh);
      vis.reset();
      active = true;
      pending = false;
      ++traced;
      if (kCount) ++cnt.rounds;
    }
    if (!__any_sync(0xffffffffu, active)) break;
    if (active && round_steps<kK, kCount>(rt, bvh, C, s_stack + threadIdx.x, kBlock, kRefillSteps, cnt)) {
      if (round_blend<kK, kCount>(rt, bvh, C, vis, cnt)) {
        const SegRec s = finish(vis.get());
        Ray r;
        r.a = make_float4(rt.O.x, rt.O.y, rt.O.z, pay[0]);
        r.b = make_float4(rt.w.x, rt.w.y, rt.w.z, pay[kBlock]);
        r.c = make_float4(pay[2 * kBlock], pay[3 * kBlock], pay[4 * kBlock], 0.f);
        float3 contrib;
        Ray nr;
        if (shade_bounce(kind, kb, max_bounces, rr_start, seed, C, r, s, contrib, nr)) {
          pay[2 * kBlock] = nr.c.x;
          pay[3 * kBlock] = nr.c.y;
          pay[4 * kBlock] = nr.c.z;
          ++kb;
          ray_begin(rt, f3(nr.a), f3(nr.b));
          pending = true;
        } else {
          const uint32_t pixel = __float_as_uint(r.a.w), sample = __float_as_uint(r.b.w);
          slots[(int64_t)(sample - (uint32_t)s0) * npix + pixel] = make_float4(contrib.x, contrib.y, contrib.z, 0.f);
        }
        active = false;
      } else {
        round_begin(rt, bvh);
        if (kCount) ++cnt.rounds;
      }
    }
  }
  if (kCount) flush_counts(stats, traced, cnt);
}

// The emitter sample's estimate added to the radiance L gathered at a vertex
// (Sec. 3.4 path tracing with emitter sampling): beta r_i w_i p_B p_L /
// (p_L^2 + p_B^2), p_B = cos / pi, with explicit roundings so that every
// kernel that gathers gives the same bits.
__device__ __forceinline__ float3 nee_gather(float3 L, float4 beta, float4 ri, float wt, float cosx, float pl) {
  const float pb = __fmul_rn(cosx, 0.318309886183790672f);
  const float f = __fdiv_rn(__fmul_rn(__fmul_rn(wt, pb), pl), __fmaf_rn(pl, pl, __fmul_rn(pb, pb)));
  return make_float3(__fmaf_rn(__fmul_rn(beta.x, ri.x), f, L.x), __fmaf_rn(__fmul_rn(beta.y, ri.y), f, L.y),
                     __fmaf_rn(__fmul_rn(beta.z, ri.z), f, L.z));
}

// Path tracing with emitter sampling: every queued ray first traces its
// emitter sample (the segment from its origin towards a point on a sampled
// emitter, Philox (pixel, sample, k, 1)), adds that estimate to the path's
// gathered radiance, then traces its own continuation with power-heuristic
// weights on emitter hits, and shades it (shade_bounce_mis).  Per-lane
// refill and chunked traversal as in k_bounce_r.
template <bool kCount>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_bounce_mis(BvhView bvh, Consts C, int k, int max_bounces,
                                                       int rr_start, uint64_t seed, int64_t npix, int s0,
                                                       const Ray* __restrict__ q_in, Ray* q_out,
                                                       const RayExt* __restrict__ e_in, RayExt* e_out,
                                                       uint32_t* counters, float4* slots, int64_t* stats) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  __shared__ float s_blend[11 * kBlock];
  __shared__ float s_gath[4 * kBlock];  // radiance gathered by the emitter samples, cos at the vertex
  const int lane = threadIdx.x & 31;
  float* gath = s_gath + threadIdx.x;
  const uint32_t count = counters[2 * k];
  TraceCounters cnt{0, 0, 0, 0, 0};
  uint32_t traced = 0;
  RayTrace<kK> rt;
  SmemBlendVisitorT<true> vis(bvh.shade, C, 1, s_blend + threadIdx.x, kBlock);
  // the emitter segment's state shares the blend slot (the phases never overlap)
  NeeVisitorSM nee;
  nee.shade = bvh.shade;
  nee.C = C;
  nee.s = s_blend + threadIdx.x;
  nee.stride = kBlock;
  uint32_t qi = 0;
  int phase = 0;  // 0: emitter-sample segment, 1: continuation
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
          const float4 ra = q_in[qi].a, rb = q_in[qi].b;
          const float4 xn = e_in[qi].n, xl = e_in[qi].l;
          gath[0] = xl.x;
          gath[kBlock] = xl.y;
          gath[2 * kBlock] = xl.z;
          uint32_t jt;
          float3 wl;
          float cosx;
          if (sample_emitter(bvh, C, seed, __float_as_uint(ra.w), __float_as_uint(rb.w), (uint32_t)k, f3(ra), f3(xn),
                             jt, wl, cosx)) {
            gath[3 * kBlock] = cosx;
            phase = 0;
            nee.reset(jt);
            ray_begin(rt, f3(ra), wl);
          } else {
            phase = 1;
            vis.pb2 = xn.w * xn.w;
            vis.reset();
            ray_begin(rt, f3(ra), f3(rb));
          }
          round_begin(rt, bvh);
          active = true;
          ++traced;
          if (kCount) ++cnt.rounds;
        } else {
          exhausted = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, active)) break;
    bool take = false;
    Ray nr;
    RayExt nx;
    if (active && round_steps<kK, kCount>(rt, bvh, C, s_stack + threadIdx.x, kBlock, kRefillSteps, cnt)) {
      if (phase == 0) {
        if (round_blend<kK, kCount>(rt, bvh, C, nee, cnt)) {
          // the emitter sample's estimate: beta r_i w_i p_B p_L / (p_L^2 + p_B^2)
          if (nee.found() && nee.E() > C.tau_E) {
            const float4 beta = __ldcv(&q_in[qi].c);
            const float4 ri = __ldg(&bvh.shade[nee.target()].s1);
            const float3 L = nee_gather(make_float3(gath[0], gath[kBlock], gath[2 * kBlock]), beta, ri, nee.wt(),
                                        gath[3 * kBlock], nee.pl());
            gath[0] = L.x;
            gath[kBlock] = L.y;
            gath[2 * kBlock] = L.z;
          }
          phase = 1;
          const float4 xn = e_in[qi].n;
          vis.pb2 = xn.w * xn.w;
          vis.reset();
          ray_begin(rt, f3(q_in[qi].a), f3(q_in[qi].b));
          round_begin(rt, bvh);
          ++traced;
          if (kCount) ++cnt.rounds;
        } else {
          round_begin(rt, bvh);
          if (kCount) ++cnt.rounds;
        }
      } else if (round_blend<kK, kCount>(rt, bvh, C, vis, cnt)) {
        const SegRec sg = finish(vis.get());
        Ray r;
        r.a = make_float4(rt.O.x, rt.O.y, rt.O.z, __ldcv(&q_in[qi].a.w));
        r.b = make_float4(rt.w.x, rt.w.y, rt.w.z, __ldcv(&q_in[qi].b.w));
        r.c = __ldcv(&q_in[qi].c);
        RayExt x;
        x.n = e_in[qi].n;
        x.l = make_float4(gath[0], gath[kBlock], gath[2 * kBlock], 0.f);
        const uint32_t pixel = __float_as_uint(r.a.w), sample = __float_as_uint(r.b.w);
        float3 contrib;
        take = shade_bounce_mis(k, max_bounces, rr_start, seed, C, r, x, sg, contrib, nr, nx);
        if (!take)
          slots[(int64_t)(sample - (uint32_t)s0) * npix + pixel] = make_float4(contrib.x, contrib.y, contrib.z, 0.f);
        active = false;
      } else {
        round_begin(rt, bvh);
        if (kCount) ++cnt.rounds;
      }
    }
    __syncwarp();
    const uint32_t at = warp_append(take, &counters[2 * (k + 1)]);
    if (take) {
      q_out[at] = nr;
      e_out[at] = nx;
    }
  }
  if (kCount) {
    add_stats(stats, 1, traced);
    add_stats(stats, 3, cnt.blended);
    add_stats(stats, 4, cnt.nodes);
    add_stats(stats, 5, cnt.tests);
    add_stats(stats, 6, cnt.rounds);
    uint32_t m = cnt.max_stack;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax((unsigned long long*)(stats + 7), (unsigned long long)m);
  }
}


// Emitter sampling split in two passes per bounce, each with one visitor's
// state (EAGPT_MIS_SPLIT): k_nee traces every queued ray's emitter sample and
// adds its estimate to the ray's gathered radiance (RayExt l, in place);
// k_cont_mis then traces the continuations with power-heuristic weights and
// shades them.  Per segment the arithmetic is k_bounce_mis's.
template <bool kCount>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_nee(BvhView bvh, Consts C, int k, uint64_t seed,
                                                const Ray* __restrict__ q_in, RayExt* e_io, uint32_t* counters,
                                                int64_t* stats) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  __shared__ float s_nee[6 * kBlock];  // the visitor's state (5 words) and cos at the vertex
  const int lane = threadIdx.x & 31;
  const uint32_t count = counters[2 * k];
  float* cosp = s_nee + 5 * kBlock + threadIdx.x;
  TraceCounters cnt{0, 0, 0, 0, 0};
  uint32_t traced = 0;
  RayTrace<kK> rt;
  NeeVisitorSM nee;
  nee.shade = bvh.shade;
  nee.C = C;
  nee.s = s_nee + threadIdx.x;
  nee.stride = kBlock;
  uint32_t qi = 0;
  bool active = false, exhausted = false;
  for (;;) {
    const bool want = !active && !exhausted;
    const uint32_t wmask = __ballot_sync(0xffffffffu, want);
    if (wmask) {
      const int leader = __ffs(wmask) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&counters[kNeeFetch + k], (uint32_t)__popc(wmask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (want) {
        const uint32_t idx = base + (uint32_t)__popc(wmask & ((1u << lane) - 1u));
        if (idx < count) {
          qi = idx;
          const float4 ra = q_in[qi].a, rb = q_in[qi].b;
          uint32_t jt;
          float3 wl;
          float cosx;
          if (sample_emitter(bvh, C, seed, __float_as_uint(ra.w), __float_as_uint(rb.w), (uint32_t)k, f3(ra),
                             f3(e_io[qi].n), jt, wl, cosx)) {
            *cosp = cosx;
            nee.reset(jt);
            ray_begin(rt, f3(ra), wl);
            round_begin(rt, bvh);
            active = true;
            ++traced;
            if (kCount) ++cnt.rounds;
          }
        } else {
          exhausted = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, active)) break;
    if (active && round_steps<kK, kCount>(rt, bvh, C, s_stack + threadIdx.x, kBlock, kRefillSteps, cnt)) {
      if (round_blend<kK, kCount>(rt, bvh, C, nee, cnt)) {
        if (nee.found() && nee.E() > C.tau_E) {
          const float4 beta = __ldg(&q_in[qi].c);
          const float4 ri = __ldg(&bvh.shade[nee.target()].s1);
          const float4 l = e_io[qi].l;
          const float3 L = nee_gather(f3(l), beta, ri, nee.wt(), *cosp, nee.pl());
          e_io[qi].l = make_float4(L.x, L.y, L.z, l.w);
        }
        active = false;
      } else {
        round_begin(rt, bvh);
        if (kCount) ++cnt.rounds;
      }
    }
  }
  if (kCount) flush_counts(stats, traced, cnt);
}

template <bool kCount>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_cont_mis(BvhView bvh, Consts C, int k, int max_bounces,
                                                     int rr_start, uint64_t seed, int64_t npix, int s0,
                                                     const Ray* __restrict__ q_in, Ray* q_out,
                                                     const RayExt* __restrict__ e_in, RayExt* e_out,
                                                     uint32_t* counters, float4* slots, int64_t* stats) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  __shared__ float s_blend[11 * kBlock];
  const int lane = threadIdx.x & 31;
  const uint32_t count = counters[2 * k];
  TraceCounters cnt{0, 0, 0, 0, 0};
  uint32_t traced = 0;
  RayTrace<kK> rt;
  SmemBlendVisitorT<true> vis(bvh.shade, C, 1, s_blend + threadIdx.x, kBlock);
  uint32_t qi = 0;
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
          const float pbw = e_in[qi].n.w;
          vis.pb2 = pbw * pbw;
          vis.reset();
          ray_begin(rt, f3(q_in[qi].a), f3(q_in[qi].b));
          round_begin(rt, bvh);
          active = true;
          ++traced;
          if (kCount) ++cnt.rounds;
        } else {
          exhausted = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, active)) break;
    bool take = false;
    Ray nr;
    RayExt nx;
    if (active && round_steps<kK, kCount>(rt, bvh, C, s_stack + threadIdx.x, kBlock, kRefillSteps, cnt)) {
      if (round_blend<kK, kCount>(rt, bvh, C, vis, cnt)) {
        const SegRec sg = finish(vis.get());
        Ray r;
        r.a = make_float4(rt.O.x, rt.O.y, rt.O.z, __ldg(&q_in[qi].a.w));
        r.b = make_float4(rt.w.x, rt.w.y, rt.w.z, __ldg(&q_in[qi].b.w));
        r.c = __ldg(&q_in[qi].c);
        RayExt x;
        x.n = e_in[qi].n;
        x.l = e_in[qi].l;
        const uint32_t pixel = __float_as_uint(r.a.w), sample = __float_as_uint(r.b.w);
        float3 contrib;
        take = shade_bounce_mis(k, max_bounces, rr_start, seed, C, r, x, sg, contrib, nr, nx);
        if (!take)
          slots[(int64_t)(sample - (uint32_t)s0) * npix + pixel] = make_float4(contrib.x, contrib.y, contrib.z, 0.f);
        active = false;
      } else {
        round_begin(rt, bvh);
        if (kCount) ++cnt.rounds;
      }
    }
    __syncwarp();
    const uint32_t at = warp_append(take, &counters[2 * (k + 1)]);
    if (take) {
      q_out[at] = nr;
      e_out[at] = nx;
    }
  }
  if (kCount) flush_counts(stats, traced, cnt);
}

// Per pixel: add the batch's samples in order; on the last batch write the
// mean.  Emitter pixels show R (Eq. 4), missed pixels 0.  With out_li (the
// incident-radiance variant of the single-bounce render) the slots hold the
// secondary radiance R(w_s) alone: L_i = mean_s R(w_s) is written to out_li
// and P (.) L_i to out_rgb; emitter and missed pixels get L_i = 0.
__global__ void __launch_bounds__(kBlock) k_accumulate(const PrimRec* __restrict__ prim, Consts C, int64_t npix,
                                                       int s0, int batch, int spp, int first, int last,
                                                       const float4* __restrict__ slots, float4* acc,
                                                       float* out_rgb, float* out_samples, float* out_li) {
  const int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  if (i >= npix) return;
  const PrimRec p = prim[i];
  const bool hit = p.c.w >= 0.f;
  const bool emit = hit && p.b.w > C.tau_E;
  if (!hit || emit) {
    const float3 v = emit ? f3(p.b) : make_float3(0.f, 0.f, 0.f);
    if (out_li && last) {
      out_li[3 * i] = 0.f;
      out_li[3 * i + 1] = 0.f;
      out_li[3 * i + 2] = 0.f;
    }
    if (out_samples)
      for (int s = 0; s < batch; ++s) {
        float* o = out_samples + 3 * (i * spp + s0 + s);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
      }
    if (last) {
      out_rgb[3 * i] = v.x;
      out_rgb[3 * i + 1] = v.y;
      out_rgb[3 * i + 2] = v.z;
    }
    return;
  }
  float4 a = first ? make_float4(0.f, 0.f, 0.f, 0.f) : acc[i];
  const float3 P = out_li ? make_float3(p.c.x, p.c.y, p.c.z) : make_float3(1.f, 1.f, 1.f);
  for (int s = 0; s < batch; ++s) {
    const float4 c = slots[(int64_t)s * npix + i];
    a.x += c.x;
    a.y += c.y;
    a.z += c.z;
    if (out_samples) {
      float* o = out_samples + 3 * (i * spp + s0 + s);
      o[0] = out_li ? P.x * c.x : c.x;
      o[1] = out_li ? P.y * c.y : c.y;
      o[2] = out_li ? P.z * c.z : c.z;
    }
  }
  if (last) {
    const float inv = 1.f / (float)spp;
    if (out_li) {
      const float3 li = make_float3(a.x * inv, a.y * inv, a.z * inv);
      out_li[3 * i] = li.x;
      out_li[3 * i + 1] = li.y;
      out_li[3 * i + 2] = li.z;
      out_rgb[3 * i] = P.x * li.x;
      out_rgb[3 * i + 1] = P.y * li.y;
      out_rgb[3 * i + 2] = P.z * li.z;
    } else {
      out_rgb[3 * i] = a.x * inv;
      out_rgb[3 * i + 1] = a.y * inv;
      out_rgb[3 * i + 2] = a.z * inv;
    }
  } else {
    acc[i] = a;
  }
}

// --------------------------------------------------------------------------
// caller rays
// --------------------------------------------------------------------------
struct RecordVisitor {
  BlendVisitor blend;
  int32_t* hits;
  int max_hits;
  __device__ __forceinline__ RecordVisitor(const ShadeRec* s, const Consts& c, float3 w, int m, int32_t* h, int mh)
      : blend(s, c, w, m), hits(h), max_hits(mh) {}
  __device__ __forceinline__ bool operator()(const TraceRec& R, uint32_t j, const HitGeom& g) {
    if (hits && (int)blend.b.n_hits < max_hits) hits[blend.b.n_hits] = (int32_t)__float_as_uint(R.r1.w);
    return blend(R, j, g);
  }
};

__global__ void __launch_bounds__(kBlock) k_trace_rays(BvhView bvh, Consts C, int mode, const float* __restrict__ rays,
                                                       int64_t n_rays, float* out_rec, int32_t* out_hits, int max_hits,
                                                       int32_t* out_nhits) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  const int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  if (i >= n_rays) return;
  const float3 O = make_float3(rays[6 * i], rays[6 * i + 1], rays[6 * i + 2]);
  const float3 w = make_float3(rays[6 * i + 3], rays[6 * i + 4], rays[6 * i + 5]);
  int32_t* hits = out_hits ? out_hits + i * (int64_t)max_hits : nullptr;
  if (hits)
    for (int k = 0; k < max_hits; ++k) hits[k] = -1;
  RecordVisitor vis(bvh.shade, C, w, mode, hits, max_hits);
  TraceCounters cnt{0, 0, 0, 0, 0};
  trace_segment<kK, false>(bvh, C, O, w, 0.f, s_stack + threadIdx.x, kBlock, vis, cnt);
  const SegRec s = finish(vis.blend.b);
  write_aux(out_rec, i, s);
  if (out_nhits) out_nhits[i] = (int32_t)vis.blend.b.n_hits;
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
int device_sms() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  if (dev < 0 || dev >= 64) return 1;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

template <class F>
static int persistent_blocks(F kernel) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
  if (per_sm < 1) per_sm = 1;
  return per_sm * device_sms();
}

static inline unsigned nblocks(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

template <bool kCount>
static cudaError_t render_impl(const RenderArgs& a, cudaStream_t st, int* launches) {
  const int64_t npix = (int64_t)a.cam.width * a.cam.height;
  const bool mis = a.kind == 1 && (a.C.flags & EAGPT_FLAG_EMITTER_SAMPLING);
  const int batch = choose_batch_spp(npix, a.spp, a.ws_bytes, mis);
  const RenderLayout L = render_layout(npix, a.spp, batch, mis);
  char* ws = (char*)a.ws;
  RayExt* ex[2] = {mis ? (RayExt*)(ws + L.e0) : nullptr, mis ? (RayExt*)(ws + L.e1) : nullptr};
  PrimRec* prim = (PrimRec*)(ws + L.prim);
  float4* acc = (float4*)(ws + L.acc);
  float4* slots = (float4*)(ws + L.slots);
  Ray* q[2] = {(Ray*)(ws + L.q0), (Ray*)(ws + L.q1)};
  uint32_t* counters = (uint32_t*)(ws + L.counters);
  const int mode = a.kind == 1 ? 1 : 0;
  const int B = a.kind == 1 ? a.max_bounces : 1;
  int nl = 0;
  EAGPT_LAUNCH(st, "k_primary", k_primary<kCount><<<nblocks(npix), kBlock, 0, st>>>(a.bvh, a.C, a.cam, mode, npix, prim, a.out_aux, a.out_stats));
  ++nl;
  static int bounce_grid[2] = {0, 0}, mis_grid[2] = {0, 0}, cache_grid[2] = {0, 0};
  if (!bounce_grid[kCount])
    bounce_grid[kCount] = EAGPT_REFILL ? persistent_blocks(k_bounce_r<kCount>) : persistent_blocks(k_bounce<kCount>);
  const bool cache = EAGPT_REFILL && a.kind == 0 && a.sb_cache;
  if (cache && !cache_grid[kCount]) cache_grid[kCount] = persistent_blocks(k_bounce_r<kCount, true>);
  static int nee_grid[2] = {0, 0};
  static int path_grid[2] = {0, 0};
  if (mis && !mis_grid[kCount])
    mis_grid[kCount] = kMisSplit ? persistent_blocks(k_cont_mis<kCount>) : persistent_blocks(k_bounce_mis<kCount>);
  if (mis && kMisSplit && !nee_grid[kCount]) nee_grid[kCount] = persistent_blocks(k_nee<kCount>);
  for (int s0 = 0; s0 < a.spp; s0 += batch) {
    const int nb = a.spp - s0 < batch ? a.spp - s0 : batch;
    cudaMemsetAsync(counters, 0, kCounterWords * sizeof(uint32_t), st);
    EAGPT_LAUNCH(st, "k_generate", k_generate<kCount><<<nblocks(npix * nb), kBlock, 0, st>>>(prim, a.C, a.cam, a.kind, B, a.rr_start, a.seed, npix,
                                                              s0, nb, q[0], counters, slots, a.out_stats, ex[0]));
    ++nl;
    const bool persist = kPathPersist && a.kind == 1 && !mis && !kSortRays && EAGPT_REFILL && B >= 2;
    if (persist) {
      if (!path_grid[kCount]) path_grid[kCount] = persistent_blocks(k_path_r<kCount>);
      EAGPT_LAUNCH(st, "k_bounce", k_path_r<kCount><<<path_grid[kCount], kBlock, 0, st>>>(a.bvh, a.C, a.kind, B, a.rr_start, a.seed,
                                                                                        npix, s0, q[0], counters, slots,
                                                                                        a.out_stats));
      ++nl;
    }
    for (int k = 1; k <= (persist ? 0 : B); ++k) {
      const uint32_t* perm = nullptr;
      if (kSortRays) {
        uint32_t *k0 = (uint32_t*)(ws + L.sk0), *k1 = (uint32_t*)(ws + L.sk1);
        uint32_t *v0 = (uint32_t*)(ws + L.sv0), *v1 = (uint32_t*)(ws + L.sv1);
        const int64_t cap = npix * nb;
        EAGPT_LAUNCH(st, "k_ray_keys", k_ray_keys<<<nblocks(cap), kBlock, 0, st>>>(q[(k - 1) & 1], &counters[2 * k], cap,
                                                                                   a.bvh.bounds_bits, k0, v0));
        launch_sort_pairs(k0, v0, k1, v1, (uint32_t*)(ws + L.shist), cap, st);
        perm = v0;
      }
      if (mis && kMisSplit) {
        EAGPT_LAUNCH(st, "k_bounce", k_nee<kCount><<<nee_grid[kCount], kBlock, 0, st>>>(a.bvh, a.C, k, a.seed, q[(k - 1) & 1],
                                                                                      ex[(k - 1) & 1], counters,
                                                                                      a.out_stats));
        ++nl;
        EAGPT_LAUNCH(st, "k_bounce", k_cont_mis<kCount><<<mis_grid[kCount], kBlock, 0, st>>>(a.bvh, a.C, k, B, a.rr_start, a.seed, npix,
                                                                                           s0, q[(k - 1) & 1], q[k & 1],
                                                                                           ex[(k - 1) & 1], ex[k & 1],
                                                                                           counters, slots, a.out_stats));
      } else if (mis)
        EAGPT_LAUNCH(st, "k_bounce", k_bounce_mis<kCount><<<mis_grid[kCount], kBlock, 0, st>>>(a.bvh, a.C, k, B, a.rr_start, a.seed, npix, s0,
                                                                   q[(k - 1) & 1], q[k & 1], ex[(k - 1) & 1], ex[k & 1],
                                                                   counters, slots, a.out_stats));
      else if (cache)
        EAGPT_LAUNCH(st, "k_bounce", k_bounce_r<kCount, true><<<cache_grid[kCount], kBlock, 0, st>>>(a.bvh, a.C, a.kind, k, B, a.rr_start, a.seed, npix,
                                                                        s0, q[(k - 1) & 1], q[k & 1], counters, slots,
                                                                        a.out_stats, perm, a.sb_cache));
      else if (EAGPT_REFILL)
        EAGPT_LAUNCH(st, "k_bounce", k_bounce_r<kCount><<<bounce_grid[kCount], kBlock, 0, st>>>(a.bvh, a.C, a.kind, k, B, a.rr_start, a.seed, npix,
                                                                  s0, q[(k - 1) & 1], q[k & 1], counters, slots,
                                                                  a.out_stats, perm, nullptr));
      else
        EAGPT_LAUNCH(st, "k_bounce", k_bounce<kCount><<<bounce_grid[kCount], kBlock, 0, st>>>(a.bvh, a.C, a.kind, k, B, a.rr_start, a.seed, npix,
                                                                s0, q[(k - 1) & 1], q[k & 1], counters, slots,
                                                                a.out_stats, perm));
      ++nl;
    }
    EAGPT_LAUNCH(st, "k_accumulate", k_accumulate<<<nblocks(npix), kBlock, 0, st>>>(prim, a.C, npix, s0, nb, a.spp, s0 == 0, s0 + nb >= a.spp, slots,
                                                   acc, a.out_rgb, a.out_samples, a.kind == 2 ? a.out_li : nullptr));
    ++nl;
  }
  if (launches) *launches += nl;
  return cudaGetLastError();
}

cudaError_t launch_render(const RenderArgs& a, cudaStream_t st, int* launches) {
  return a.out_stats ? render_impl<true>(a, st, launches) : render_impl<false>(a, st, launches);
}

cudaError_t launch_trace_rays(const BvhView& bvh, const Consts& C, int mode, const float* rays, int64_t n_rays,
                              float* out_rec, int32_t* out_hits, int max_hits, int32_t* out_nhits, cudaStream_t st) {
  if (n_rays > 0)
    EAGPT_LAUNCH(st, "k_trace_rays", k_trace_rays<<<nblocks(n_rays), kBlock, 0, st>>>(bvh, C, mode, rays, n_rays, out_rec, out_hits, max_hits,
                                                     out_nhits));
  return cudaGetLastError();
}

}  // namespace eagpt

namespace eagpt {

// Primary records only (used by the adjoint, which re-traces them).
cudaError_t launch_primary_records(const BvhView& bvh, const Consts& C, const eagpt_camera& cam, int mode,
                                   int64_t npix, void* prim, cudaStream_t st) {
  EAGPT_LAUNCH(st, "k_primary",
               k_primary<false><<<nblocks(npix), kBlock, 0, st>>>(bvh, C, cam, mode, npix, (PrimRec*)prim, nullptr,
                                                                 nullptr));
  return cudaGetLastError();
}

}  // namespace eagpt

namespace eagpt {

// 0-bounce (radiance) render: every pixel shows the blended radiance R of its
// primary segment (the radiant scene of Sec. 3.2; light-baked scenes are
// viewed this way, Eq. 10).
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_radiance(BvhView bvh, Consts C, eagpt_camera cam, int64_t npix,
                                                                 float* out_rgb, float* aux) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  const int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  if (i >= npix) return;
  float3 O, w;
  camera_ray(cam, (uint32_t)i, O, w);
  BlendVisitor vis(bvh.shade, C, w, 0);
  TraceCounters cnt{0, 0, 0, 0, 0};
  trace_segment<kK, false>(bvh, C, O, w, 0.f, s_stack + threadIdx.x, kBlock, vis, cnt);
  const SegRec s = finish(vis.b);
  out_rgb[3 * i] = s.R.x;
  out_rgb[3 * i + 1] = s.R.y;
  out_rgb[3 * i + 2] = s.R.z;
  if (aux) write_aux(aux, i, s);
}

cudaError_t launch_radiance(const BvhView& bvh, const Consts& C, const eagpt_camera& cam, float* out_rgb, float* aux,
                            cudaStream_t st) {
  const int64_t npix = (int64_t)cam.width * cam.height;
  if (bvh.n <= 0) return cudaMemsetAsync(out_rgb, 0, (size_t)npix * 3 * sizeof(float), st);
  EAGPT_LAUNCH(st, "k_radiance", k_radiance<<<nblocks(npix), kBlock, 0, st>>>(bvh, C, cam, npix, out_rgb, aux));
  return cudaGetLastError();
}

}  // namespace eagpt
