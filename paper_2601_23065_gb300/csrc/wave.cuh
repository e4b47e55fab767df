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
