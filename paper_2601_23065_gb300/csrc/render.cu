// Wavefront renderer: single-bounce estimator (Eq. 6) and path tracing (Eq. 8).
//
//   k_primary     one pinhole ray per pixel, traced once and shared by all
//                 samples (the viewing direction is fixed per pixel); writes
//                 the pixel's blended record (N~, D~, R, E, P, A).
//   k_generate    per (sample, pixel) of a sample batch: first bounce of every
//                 path of a non-emitter primary hit -> ray queue 1.
//   k_bounce_r    one launch per bounce k, persistent with per-lane refill:
//                 trace the queued ray, blend, then either end the path (its
//                 contribution goes to its own slot) or sample the next
//                 bounce and append it to queue k+1 with a warp-ballot
//                 compaction (one atomic per warp).
//   k_nee,        path tracing with emitter sampling: per bounce, the emitter
//   k_cont_mis    samples of the queued rays, then their continuations.
//   k_accumulate  per pixel: the batch's slots in sample order (deterministic,
//                 independent of the batch size), final mean.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "internal.h"
#include "trace.cuh"
#include "wave.cuh"

namespace eagpt {

constexpr int kK = 12;  // k-buffer size (hits collected per traversal round)

EAGPT_DEFINE_ERROR_READER(take_errors_render)

// counters block: per bounce k, [2k] = rays queued for bounce k, [2k+1] = fetch
constexpr int kMaxBounces = 60;
// per bounce k: queue length (2k) and fetch index (2k + 1); then the fetch
// indices of the emitter-sample pass (kNeeFetch + k)
constexpr int kNeeFetch = 2 * (kMaxBounces + 2) + 8;
constexpr int kCounterWords = kNeeFetch + kMaxBounces + 2;

// Segment counts of the last render into a workspace (always kept, without the
// counting variant): [0] primary segments, [1] secondary segments traced by
// the bounce kernels (continuations; emitter-sample segments not included).
constexpr int kSummaryWords = 4;

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
  L.summary = take(kSummaryWords * sizeof(int64_t));
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
    trace_segment<kK, kCount>(bvh, C, O, w, s_stack + threadIdx.x, kBlock, vis, cnt);
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

// The bounce kernel with per-lane refill: a lane whose segment is finished
// takes the next queued ray at once (one atomic per warp for all the lanes
// that want one) instead of waiting for the slowest ray of a 32-ray batch.
// Traversal runs in chunks of kRefillSteps node/leaf steps; between chunks
// the lanes whose round is complete blend it, and finished segments are shaded
// and their continuation appended (warp-ballot compaction).
constexpr int kRefillSteps = 64;

template <bool kCount, bool kCache = false>
__global__ void __launch_bounds__(kBlock, kMinBlocks) k_bounce_r(BvhView bvh, Consts C, int kind, int k, int max_bounces,
                                                     int rr_start, uint64_t seed, int64_t npix, int s0,
                                                     const Ray* __restrict__ q_in, Ray* q_out, uint32_t* counters,
                                                     float4* slots, int64_t* stats, float4* sb_cache) {
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
          qi = idx;
          ray_begin(rt, f3(q_in[qi].a), f3(q_in[qi].b), bvh);
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
        round_next(rt, bvh);
        if (kCount) ++cnt.rounds;
      }
    }
    __syncwarp();
    const uint32_t at = warp_append(take, &counters[2 * (k + 1)]);
    if (take) q_out[at] = nr;
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

// Path tracing with emitter sampling, two passes per bounce, each with one
// visitor's state: k_nee traces every queued ray's emitter sample and
// adds its estimate to the ray's gathered radiance (RayExt l, in place);
// k_cont_mis then traces the continuations with power-heuristic weights and
// shades them.  Per-lane refill and chunked traversal as in k_bounce_r.
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
            ray_begin(rt, f3(ra), wl, bvh);
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
        round_next(rt, bvh);
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
          ray_begin(rt, f3(q_in[qi].a), f3(q_in[qi].b), bvh);
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
        round_next(rt, bvh);
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

// Adds one pass's secondary segments (the queue lengths of its bounces) to the
// workspace's summary; the first pass also sets the primary segments.
__global__ void k_pass_summary(const uint32_t* __restrict__ counters, int B, int64_t npix, int first,
                               int64_t* summary) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t sec = 0;
  for (int k = 1; k <= B; ++k) sec += counters[2 * k];
  if (first) {
    summary[0] = npix;
    summary[1] = 0;
  }
  summary[1] += sec;
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
  trace_segment<kK, false>(bvh, C, O, w, s_stack + threadIdx.x, kBlock, vis, cnt);
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

// Blocks of a persistent launch of `kernel` (kBlock threads, no dynamic
// shared memory) on the current device: resident blocks per SM x SMs, cached
// per (kernel, device).
int persistent_grid(const void* kernel) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> g(mu);
    const auto it = cache.find({kernel, dev});
    if (it != cache.end()) return it->second;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
  if (per_sm < 1) per_sm = 1;
  const int grid = per_sm * device_sms();
  std::lock_guard<std::mutex> g(mu);
  cache[{kernel, dev}] = grid;
  return grid;
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
  const bool cache = a.kind == 0 && a.sb_cache;
  const int bounce_grid = persistent_grid(cache ? (const void*)k_bounce_r<kCount, true> : (const void*)k_bounce_r<kCount, false>);
  const int nee_grid = mis ? persistent_grid((const void*)k_nee<kCount>) : 0;
  const int mis_grid = mis ? persistent_grid((const void*)k_cont_mis<kCount>) : 0;
  for (int s0 = 0; s0 < a.spp; s0 += batch) {
    const int nb = a.spp - s0 < batch ? a.spp - s0 : batch;
    // every pass starts from zeroed queue counters (the workspace may hold an
    // earlier render's)
    const cudaError_t me = cudaMemsetAsync(counters, 0, kCounterWords * sizeof(uint32_t), st);
    if (me != cudaSuccess) return me;
    // sample numbers (Philox counters, slot offsets) of this pass
    const int sa = a.s_first + s0;
    EAGPT_LAUNCH(st, "k_generate", k_generate<kCount><<<nblocks(npix * nb), kBlock, 0, st>>>(prim, a.C, a.cam, a.kind, B, a.rr_start, a.seed, npix,
                                                              sa, nb, q[0], counters, slots, a.out_stats, ex[0]));
    ++nl;
    for (int k = 1; k <= B; ++k) {
      if (mis) {
        EAGPT_LAUNCH(st, "k_bounce", k_nee<kCount><<<nee_grid, kBlock, 0, st>>>(a.bvh, a.C, k, a.seed, q[(k - 1) & 1],
                                                                              ex[(k - 1) & 1], counters, a.out_stats));
        ++nl;
        EAGPT_LAUNCH(st, "k_bounce", k_cont_mis<kCount><<<mis_grid, kBlock, 0, st>>>(a.bvh, a.C, k, B, a.rr_start, a.seed, npix,
                                                                                   sa, q[(k - 1) & 1], q[k & 1],
                                                                                   ex[(k - 1) & 1], ex[k & 1],
                                                                                   counters, slots, a.out_stats));
      } else if (cache) {
        EAGPT_LAUNCH(st, "k_bounce", k_bounce_r<kCount, true><<<bounce_grid, kBlock, 0, st>>>(a.bvh, a.C, a.kind, k, B, a.rr_start, a.seed, npix,
                                                                        sa, q[(k - 1) & 1], q[k & 1], counters, slots,
                                                                        a.out_stats, a.sb_cache));
      } else {
        // with a level of detail, bounce segments k >= lod_from trace the
        // merged surfels
        const BvhView& bk = a.lod_from > 0 && k >= a.lod_from ? a.bvh_lod : a.bvh;
        EAGPT_LAUNCH(st, "k_bounce", k_bounce_r<kCount, false><<<bounce_grid, kBlock, 0, st>>>(bk, a.C, a.kind, k, B, a.rr_start, a.seed, npix,
                                                                  sa, q[(k - 1) & 1], q[k & 1], counters, slots,
                                                                  a.out_stats, nullptr));
      }
      ++nl;
    }
    EAGPT_LAUNCH(st, "k_accumulate", k_accumulate<<<nblocks(npix), kBlock, 0, st>>>(prim, a.C, npix, s0, nb, a.spp, s0 == 0, s0 + nb >= a.spp, slots,
                                                   acc, a.out_rgb, a.out_samples, a.kind == 2 ? a.out_li : nullptr));
    ++nl;
    EAGPT_LAUNCH(st, "k_pass_summary", k_pass_summary<<<1, 32, 0, st>>>(counters, B, npix, s0 == 0,
                                                                       (int64_t*)(ws + L.summary)));
    ++nl;
  }
  if (launches) *launches += nl;
  return cudaGetLastError();
}

// Reads the segment summary of the last render into `ws` (synchronous).
cudaError_t render_summary(const void* ws, int64_t* out, cudaStream_t st) {
  const RenderLayout L = render_layout(1, 1, 1, false);  // the summary's offset does not depend on the sizes
  cudaError_t e = cudaMemcpyAsync(out, (const char*)ws + L.summary, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
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
  trace_segment<kK, false>(bvh, C, O, w, s_stack + threadIdx.x, kBlock, vis, cnt);
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
