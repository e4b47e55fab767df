// Per-path steps of the wavefront renderer, shared by the single-request
// render (render.cu) and the batched serving loop (serve.cu), so that a path
// computes bit-identical values in both.
#pragma once

#include "common.cuh"
#include "trace.cuh"

namespace eagpt {

struct __align__(16) Ray {
  float4 a;  // origin, pixel (bits)
  float4 b;  // direction, sample (bits)
  float4 c;  // throughput, request id (bits; 0 outside the serving loop)
};

// Side record of a queued ray when emitter sampling is on (same queue
// index): the normal of the vertex the ray leaves, the cosine-sampling pdf of
// its direction, and the radiance the path's emitter samples gathered so far.
struct __align__(16) RayExt {
  float4 n;  // N~ of the origin vertex, p_B = (w . N~) / pi
  float4 l;  // accumulated radiance, unused
};

struct __align__(16) PrimRec {
  float4 a;  // N~, D~
  float4 b;  // R, E
  float4 c;  // P, A (A < 0 marks a miss)
};

__device__ __forceinline__ bool prim_is_path_start(const PrimRec& p, const Consts& C) {
  return p.c.w >= 0.f && !(p.b.w > C.tau_E);
}

// First bounce of one path (Sec. 3.1 "Light Bouncing"): X = O + D~ w,
// throughput P (the cosine pdf cancels cos/pi of the diffuse BRDF), Russian
// roulette when it starts at bounce 1, cosine-weighted direction about N~
// from X + offset N~.  Returns false when the path ends here (its value 0).
__device__ __forceinline__ bool first_bounce(const PrimRec& p, const Consts& C, const eagpt_camera& cam, int kind,
                                             int max_bounces, int rr_start, uint64_t seed, uint32_t pixel,
                                             uint32_t sample, uint32_t tag, Ray& r) {
  const int B = kind == 1 ? max_bounces : 1;
  // kind 2 (single bounce, incident radiance): unit throughput, P is applied
  // per pixel after the sample mean
  float3 beta = kind == 2 ? make_float3(1.f, 1.f, 1.f) : make_float3(p.c.x, p.c.y, p.c.z);
  if (B < 1) return false;
  const float4 u = draws(seed, pixel, sample, 1u);
  if (kind == 1 && rr_start <= 1) {
    const float q = fminf(1.f, fmaxf(beta.x, fmaxf(beta.y, beta.z)));
    if (!(u.z < q)) return false;
    beta = (1.f / q) * beta;
  }
  float3 O, w;
  camera_ray(cam, pixel, O, w);
  const float3 Nn = make_float3(p.a.x, p.a.y, p.a.z);
  const float3 X = O + p.a.w * w;
  const float3 O2 = X + C.bounce_offset * Nn;
  const float3 w2 = cosine_direction(Nn, u.x, u.y);
  r.a = make_float4(O2.x, O2.y, O2.z, __uint_as_float(pixel));
  r.b = make_float4(w2.x, w2.y, w2.z, __uint_as_float(sample));
  r.c = make_float4(beta.x, beta.y, beta.z, __uint_as_float(tag));
  return true;
}

// Shading after the segment of bounce k (Eq. 6 for kind 0, Eq. 8 for kind
// 1): either the path ends with `contrib` (returns false) or continues with
// the next bounce's ray `nr` (returns true).
__device__ __forceinline__ bool shade_bounce(int kind, int k, int max_bounces, int rr_start, uint64_t seed,
                                             const Consts& C, const Ray& r, const SegRec& s, float3& contrib,
                                             Ray& nr) {
  const float3 O = f3(r.a), w = f3(r.b);
  const uint32_t pixel = __float_as_uint(r.a.w), sample = __float_as_uint(r.b.w);
  float3 beta = f3(r.c);
  contrib = make_float3(0.f, 0.f, 0.f);
  if (kind != 1) {
    contrib = mul3(beta, s.R);  // the secondary's radiance is the cache
    return false;
  }
  if (!s.hit) return false;  // miss: no light
  if (s.E > C.tau_E) {
    contrib = mul3(beta, s.R);  // first emissive vertex
    return false;
  }
  if (k >= max_bounces) return false;  // bounce limit: discarded
  beta = mul3(beta, s.P);
  const float4 u = draws(seed, pixel, sample, (uint32_t)(k + 1));
  if (k + 1 >= rr_start) {
    const float q = fminf(1.f, fmaxf(beta.x, fmaxf(beta.y, beta.z)));
    if (!(u.z < q)) return false;
    beta = (1.f / q) * beta;
  }
  const float3 X = O + s.Dn * w;
  const float3 O2 = X + C.bounce_offset * s.Nn;
  const float3 w2 = cosine_direction(s.Nn, u.x, u.y);
  nr.a = make_float4(O2.x, O2.y, O2.z, r.a.w);
  nr.b = make_float4(w2.x, w2.y, w2.z, r.b.w);
  nr.c = make_float4(beta.x, beta.y, beta.z, r.c.w);
  return true;
}

// Emitter sample of the reflection at origin O2 with normal Nn (draws
// (pixel, sample, k, 1)): an emitter chosen by the FP64 running weight sums, a
// point of its support disc from the truncated Gaussian; returns false when
// there is no emitter or the direction is below the tangent plane.
__device__ __forceinline__ bool sample_emitter(const BvhView& bvh, const Consts& C, uint64_t seed, uint32_t pixel,
                                               uint32_t sample, uint32_t k, float3 O2, float3 Nn, uint32_t& jt,
                                               float3& wl, float& cosx) {
  const uint32_t ne = bvh.hdr->em_count;
  if (ne == 0) return false;
  const float4 u = draws_w(seed, pixel, sample, k, 1u);
  const double x = (double)u.x * bvh.hdr->em_total;  // u.x is exact in FP64
  uint32_t lo = 0, hi = ne - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (bvh.em_cdf[mid] > x) hi = mid;
    else lo = mid + 1;
  }
  jt = bvh.em_idx[lo];
  const TraceRec* R = bvh.trace + jt;
  const float4 r0 = __ldg(&R->r0), r2 = __ldg(&R->r2), r3 = __ldg(&R->r3);
  // r2 = t_u / s_u and r3 = t_v / s_v: s_u t_u = r2 / |r2|^2
  const float ia = 1.f / (r2.x * r2.x + r2.y * r2.y + r2.z * r2.z);
  const float ib = 1.f / (r3.x * r3.x + r3.y * r3.y + r3.z * r3.z);
  // log1p keeps the relative accuracy of log(1 - x) for small x (small u1)
  const float rho = sqrtf(-2.f * log1pf(-u.y * (1.f - expf(-0.5f * C.support2))));
  float sn, cs;
  sincospif(2.f * u.z, &sn, &cs);
  const float a = rho * cs * ia, b = rho * sn * ib;
  const float3 y = make_float3(r0.x + a * r2.x + b * r3.x, r0.y + a * r2.y + b * r3.y, r0.z + a * r2.z + b * r3.z);
  const float3 d = y - O2;
  const float inv = rsqrtf(dot3(d, d));
  wl = inv * d;
  cosx = dot3(wl, Nn);
  return cosx > 0.f;
}

// Shading after the continuation segment of bounce k with emitter sampling:
// as shade_bounce for path tracing, but every way the path ends returns the
// radiance its emitter samples gathered (ext.l) plus, at an emissive vertex,
// the weighted R of the segment; a continuation carries the normal, its
// direction's p_B and that radiance in next.
__device__ __forceinline__ bool shade_bounce_mis(int k, int max_bounces, int rr_start, uint64_t seed,
                                                 const Consts& C, const Ray& r, const RayExt& ext, const SegRec& s,
                                                 float3& contrib, Ray& nr, RayExt& next) {
  const float3 O = f3(r.a), w = f3(r.b);
  const uint32_t pixel = __float_as_uint(r.a.w), sample = __float_as_uint(r.b.w);
  float3 beta = f3(r.c);
  const float3 L = f3(ext.l);
  contrib = L;
  if (!s.hit) return false;
  if (s.E > C.tau_E) {
    contrib = L + mul3(beta, s.R);  // s.R carries the power-heuristic weights
    return false;
  }
  if (k >= max_bounces) return false;
  beta = mul3(beta, s.P);
  const float4 u = draws(seed, pixel, sample, (uint32_t)(k + 1));
  if (k + 1 >= rr_start) {
    const float q = fminf(1.f, fmaxf(beta.x, fmaxf(beta.y, beta.z)));
    if (!(u.z < q)) return false;
    beta = (1.f / q) * beta;
  }
  const float3 X = O + s.Dn * w;
  const float3 O2 = X + C.bounce_offset * s.Nn;
  const float3 w2 = cosine_direction(s.Nn, u.x, u.y);
  nr.a = make_float4(O2.x, O2.y, O2.z, r.a.w);
  nr.b = make_float4(w2.x, w2.y, w2.z, r.b.w);
  nr.c = make_float4(beta.x, beta.y, beta.z, r.c.w);
  next.n = make_float4(s.Nn.x, s.Nn.y, s.Nn.z, dot3(w2, s.Nn) * 0.318309886183790672f);
  next.l = make_float4(L.x, L.y, L.z, 0.f);
  return true;
}

// Warp-aggregated append of the lanes with `take` set; returns each such
// lane's index in the queue.  All 32 lanes must call it.
__device__ __forceinline__ uint32_t warp_append(bool take, uint32_t* counter) {
  const uint32_t mask = __ballot_sync(0xffffffffu, take);
  const int lane = threadIdx.x & 31;
  uint32_t base = 0;
  if (lane == 0 && mask) base = atomicAdd(counter, (uint32_t)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, 0);
  return base + __popc(mask & ((1u << lane) - 1u));
}

}  // namespace eagpt
