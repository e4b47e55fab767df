// Adjoint of the single-bounce render (Eq. 6) with respect to every surfel
// parameter: centre p, raw quaternion q, scales s, opacity sigma, albedo rho,
// radiance r.  Hit lists are recomputed, not stored: each segment is traced
// twice with the forward traversal (bit-identical hits), once to get its
// blended values and once to run the front-to-back adjoint of Eq. 2, whose
// suffix sums S_i = sum_{j>i} w_j v_j are V - V_{<=i}.
//
//   k_bwd_secondary  per (sample, pixel): rebuild the sample's bounce ray
//                    exactly as the forward did, trace, adjoint with
//                    dL/dR2 = g (.) P1 / S, scatter surfel gradients with
//                    atomics, and store the sample's dL/dN~1, dL/dD~1 (through
//                    the bounce origin X + offset N~ and the cosine direction)
//                    and dL/dP1 = g (.) R2 / S.
//   k_bwd_primary    per pixel: sum the samples in order, take the adjoints
//                    through N~ = N/|N| and D~ = D/A, adjoint of the primary
//                    segment (emitter pixels: dL/dR1 = g).
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "trace.cuh"

namespace eagpt {

EAGPT_DEFINE_ERROR_READER(take_errors_backward)

constexpr int kKb = 12;           // k-buffer of the adjoint's traversals
constexpr int kBwdMinBlocks = 5;  // resident blocks per SM of the secondary adjoint

struct __align__(16) PrimRecB {
  float4 a, b, c;  // same layout as the forward's primary record
};

// Raw blended sums of one segment (first pass).
struct RawVisitor {
  BlendVisitor blend;
  __device__ __forceinline__ RawVisitor(const ShadeRec* s, const Consts& c, float3 w, int m) : blend(s, c, w, m) {}
  __device__ __forceinline__ bool operator()(const TraceRec& R, uint32_t j, const HitGeom& h) {
    return blend(R, j, h);
  }
};

// First pass when only the blended radiance R is differentiated (the
// secondary segment of Eq. 6, the 0-bounce image): R and T with the forward's
// exact arithmetic (same stopping decisions), nothing else.
struct RBlendVisitor {
  const ShadeRec* shade;
  Consts C;
  int mode;
  float3 R;
  float T;
  uint32_t n_hits;
  __device__ __forceinline__ RBlendVisitor(const ShadeRec* s, const Consts& c, int m)
      : shade(s), C(c), mode(m), R(make_float3(0.f, 0.f, 0.f)), T(1.f), n_hits(0) {}
  __device__ __forceinline__ bool operator()(const TraceRec&, uint32_t j, const HitGeom& h) {
    const ShadeRec* sp = shade + j;
    const float4 s1 = __ldg(&sp->s1);
    const float wgt = __fmul_rn(T, h.alpha);
    const float re = (mode == 1 && !(__ldg(&sp->s0.w) > C.tau_E)) ? 0.f : wgt;
    R = make_float3(__fmaf_rn(re, s1.x, R.x), __fmaf_rn(re, s1.y, R.y), __fmaf_rn(re, s1.z, R.z));
    T = __fmul_rn(T, __fsub_rn(1.f, h.alpha));
    ++n_hits;
    return T < C.T_min;
  }
};

// dL/dq_raw from dL/d(t_u, t_v, n) of the normalised-quaternion frame
// (partial derivatives of the rotation columns, then the projection of the
// normalisation q / |q|).
__device__ __forceinline__ float4 quat_adjoint(float4 q, float3 a, float3 b, float3 c) {
  const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  const float gw = 2.f * (a.y * z - a.z * y - b.x * z + b.z * x + c.x * y - c.y * x);
  const float gx = 2.f * (a.y * y + a.z * z + b.x * y - 2.f * b.y * x + b.z * w + c.x * z - c.y * w - 2.f * c.z * x);
  const float gy = 2.f * (-2.f * a.x * y + a.y * x - a.z * w + b.x * x + b.z * z + c.x * w + c.y * z - 2.f * c.z * y);
  const float gz = 2.f * (-2.f * a.x * z + a.y * w + a.z * x - b.x * w - 2.f * b.y * z + b.z * y + c.x * x + c.y * y);
  const float proj = w * gw + x * gx + y * gy + z * gz;
  return make_float4((gw - w * proj) * inv, (gx - x * proj) * inv, (gy - y * proj) * inv, (gz - z * proj) * inv);
}

// Front-to-back adjoint of one segment (second pass).  gN, gD, gR, gP, gA
// are the adjoints of the raw blended sums N, D, R, P and of A = 1 - T_n;
// V holds the raw sums of the first pass.
template <bool kOnlyR>
struct AdjointVisitorT {
  const ShadeRec* shade;
  eagpt_scene sc;
  eagpt_scene_grad gr;
  Consts C;
  float3 O, w;
  int mode;
  float3 gN, gR, gP;
  float gD, gA;
  Blend V;      // totals from the first pass
  Blend run;    // running sums up to and including the current hit
  float3 dO, dw;
  __device__ __forceinline__ bool operator()(const TraceRec& R, uint32_t j, const HitGeom& h) {
    const uint32_t id = __float_as_uint(R.r1.w);
    const ShadeRec* sp = shade + j;
    const float4 s0 = __ldg(&sp->s0), s1 = __ldg(&sp->s1);
    const float a = h.alpha;
    const float Tp = run.T;  // transmittance before this hit
    const float wgt = Tp * a;
    const float sgn = h.d > 0.f ? -1.f : 1.f;
    const float3 n = f3(R.r1);
    const float3 vN = sgn * n;
    const float remit = (mode == 1 && !(s0.w > C.tau_E)) ? 0.f : 1.f;
    const float3 vR = remit * make_float3(s1.x, s1.y, s1.z);
    const float3 vP = make_float3(s0.x, s0.y, s0.z);
    // running sums including this hit
    if (!kOnlyR) {
      run.N = run.N + wgt * vN;
      run.P = run.P + wgt * vP;
      run.D += wgt * h.t;
    }
    run.R = run.R + wgt * vR;
    run.T = Tp * (1.f - a);
    const float inv1a = 1.f / (1.f - a);
    // dL/dalpha: T_{i-1} v_i - S_i / (1 - alpha_i), S_i = V - V_{<=i}
    float da = dot3(gR, Tp * vR - inv1a * (V.R - run.R));
    if (!kOnlyR) {
      da += gA * V.T * inv1a;
      da += dot3(gN, Tp * vN - inv1a * (V.N - run.N));
      da += dot3(gP, Tp * vP - inv1a * (V.P - run.P));
      da += gD * (Tp * h.t - inv1a * (V.D - run.D));
      // albedo
      atomicAdd(&gr.albedo[3 * id + 0], wgt * gP.x);
      atomicAdd(&gr.albedo[3 * id + 1], wgt * gP.y);
      atomicAdd(&gr.albedo[3 * id + 2], wgt * gP.z);
    }
    if (remit != 0.f) {
      atomicAdd(&gr.radiance[3 * id + 0], wgt * gR.x);
      atomicAdd(&gr.radiance[3 * id + 1], wgt * gR.y);
      atomicAdd(&gr.radiance[3 * id + 2], wgt * gR.z);
    }
    // alpha = sigma g unless clamped
    float dG = 0.f;
    const float sigma = R.r0.w;
    const bool clamped = h.sg >= C.alpha_max;
    const float g = sigma > 0.f ? h.sg / sigma : 0.f;
    if (!clamped) {
      atomicAdd(&gr.opacity[id], da * g);
      dG = da * sigma;
    }
    const float du = -dG * g * h.u, dv = -dG * g * h.v;
    const float su = sc.scale[2 * id], sv = sc.scale[2 * id + 1];
    const float3 ta = f3(R.r2), tb = f3(R.r3);       // t_u / s_u, t_v / s_v
    const float3 tu = su * ta, tv = sv * tb;
    const float3 p = f3(R.r0);
    const float3 op = O - p;
    const float3 Dx = op + h.t * w;                   // x - p
    const float3 dDx = du * ta + dv * tb;
    const float3 dtu = (du / su) * Dx, dtv = (dv / sv) * Dx;
    atomicAdd(&gr.scale[2 * id + 0], -du * h.u / su);
    atomicAdd(&gr.scale[2 * id + 1], -dv * h.v / sv);
    float3 dn = kOnlyR ? make_float3(0.f, 0.f, 0.f) : (wgt * sgn) * gN;
    const float dt = kOnlyR ? dot3(dDx, w) : wgt * gD + dot3(dDx, w);
    // Dx = O - p + t w
    dO = dO + dDx;
    dw = dw + h.t * dDx;
    float3 dp = make_float3(-dDx.x, -dDx.y, -dDx.z);
    // t = ((p - O) . n) / (w . n)
    const float invd = 1.f / h.d;
    dp = dp + (dt * invd) * n;
    dO = dO - (dt * invd) * n;
    dn = dn + (dt * invd) * (make_float3(-op.x, -op.y, -op.z) - h.t * w);
    dw = dw - (dt * h.t * invd) * n;
    atomicAdd(&gr.pos[3 * id + 0], dp.x);
    atomicAdd(&gr.pos[3 * id + 1], dp.y);
    atomicAdd(&gr.pos[3 * id + 2], dp.z);
    const float4 q = make_float4(sc.quat[4 * id], sc.quat[4 * id + 1], sc.quat[4 * id + 2], sc.quat[4 * id + 3]);
    const float4 dq = quat_adjoint(q, dtu, dtv, dn);
    atomicAdd(&gr.quat[4 * id + 0], dq.x);
    atomicAdd(&gr.quat[4 * id + 1], dq.y);
    atomicAdd(&gr.quat[4 * id + 2], dq.z);
    atomicAdd(&gr.quat[4 * id + 3], dq.w);
    return run.T < C.T_min;
  }
};

using AdjointVisitor = AdjointVisitorT<false>;

__device__ __forceinline__ void init_blend(Blend& b) {
  b.N = b.R = b.P = make_float3(0.f, 0.f, 0.f);
  b.D = b.E = 0.f;
  b.T = 1.f;
  b.n_hits = 0;
}

// dL/dn of w' = l0 b1(n) + l1 b2(n) + l2 n for the basis of Duff et al.
// (the basis branch is held fixed).
__device__ __forceinline__ float3 cosine_direction_adjoint(float3 n, float u0, float u1, float3 dw) {
  const float sgn = copysignf(1.0f, n.z);
  const float a = -1.0f / (sgn + n.z);
  const float a2 = a * a;
  const float r = sqrtf(u0);
  float s, c;
  sincospif(2.0f * u1, &s, &c);
  const float l0 = r * c, l1 = r * s, l2 = sqrtf(fmaxf(0.0f, 1.0f - u0));
  // rows of the Jacobians of b1 and b2 (columns n_x, n_y, n_z)
  const float3 J1x = make_float3(2.f * sgn * n.x * a, 0.f, sgn * n.x * n.x * a2);
  const float3 J1y = make_float3(sgn * n.y * a, sgn * n.x * a, sgn * n.x * n.y * a2);
  const float3 J1z = make_float3(-sgn, 0.f, 0.f);
  const float3 J2x = make_float3(n.y * a, n.x * a, n.x * n.y * a2);
  const float3 J2y = make_float3(0.f, 2.f * n.y * a, n.y * n.y * a2);
  const float3 J2z = make_float3(0.f, -1.f, 0.f);
  const float3 g1 = dw.x * J1x + dw.y * J1y + dw.z * J1z;
  const float3 g2 = dw.x * J2x + dw.y * J2y + dw.z * J2z;
  return l0 * g1 + l1 * g2 + l2 * dw;
}

// Re-tracing form (no forward sample cache): the secondary segment is traced
// once for its blended R and T, then again for the adjoint.
__global__ void __launch_bounds__(kBlock, kBwdMinBlocks) k_bwd_secondary(BvhView bvh, Consts C, eagpt_camera cam, eagpt_scene sc,
                                                          eagpt_scene_grad gr, const PrimRecB* __restrict__ prim,
                                                          const float* __restrict__ dL, int spp, uint64_t seed,
                                                          int64_t npix, int s0, int batch, float4* per_sample) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  const int64_t t = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  if (t >= npix * (int64_t)batch) return;
  const int64_t pixel = t % npix;
  const int sl = (int)(t / npix);
  const PrimRecB p = prim[pixel];
  float4 outA = make_float4(0.f, 0.f, 0.f, 0.f), outB = make_float4(0.f, 0.f, 0.f, 0.f);
  if (p.c.w >= 0.f && !(p.b.w > C.tau_E)) {
    const uint32_t sample = (uint32_t)(s0 + sl);
    const float4 u = draws(seed, (uint32_t)pixel, sample, 1u);
    float3 O, w;
    camera_ray(cam, (uint32_t)pixel, O, w);
    const float3 Nn = make_float3(p.a.x, p.a.y, p.a.z);
    const float3 X = O + p.a.w * w;
    const float3 O2 = X + C.bounce_offset * Nn;
    const float3 w2 = cosine_direction(Nn, u.x, u.y);
    TraceCounters cnt{0, 0, 0, 0, 0};
    // the secondary segment enters the pixel only through its R (Eq. 6)
    RBlendVisitor v1(bvh.shade, C, 0);
    trace_segment<kKb, false>(bvh, C, O2, w2, s_stack + threadIdx.x, kBlock, v1, cnt);
    const float invS = 1.f / (float)spp;
    const float3 g = make_float3(dL[3 * pixel], dL[3 * pixel + 1], dL[3 * pixel + 2]);
    const float3 P1 = make_float3(p.c.x, p.c.y, p.c.z);
    if (v1.n_hits > 0) {
      AdjointVisitorT<true> av;
      av.shade = bvh.shade;
      av.sc = sc;
      av.gr = gr;
      av.C = C;
      av.O = O2;
      av.w = w2;
      av.mode = 0;
      av.gN = av.gP = make_float3(0.f, 0.f, 0.f);
      av.gR = invS * mul3(g, P1);
      av.gD = av.gA = 0.f;
      init_blend(av.V);
      av.V.R = v1.R;
      av.V.T = v1.T;
      init_blend(av.run);
      av.dO = av.dw = make_float3(0.f, 0.f, 0.f);
      trace_segment<kKb, false>(bvh, C, O2, w2, s_stack + threadIdx.x, kBlock, av, cnt);
      // O2 = O + D~1 w + offset N~1 ; w2 = basis(N~1) l
      const float gDn = dot3(av.dO, w);
      const float3 gNn = C.bounce_offset * av.dO + cosine_direction_adjoint(Nn, u.x, u.y, av.dw);
      const float3 gP1 = invS * mul3(g, v1.R);
      outA = make_float4(gNn.x, gNn.y, gNn.z, gDn);
      outB = make_float4(gP1.x, gP1.y, gP1.z, 0.f);
    }
  }
  per_sample[2 * t] = outA;
  per_sample[2 * t + 1] = outB;
}

// The cached adjoint of the secondary segments: the forward stored each
// sample's secondary R and T (sample-major, written by the single-bounce
// render from the same bit-identical blend), so the values pass is read
// instead of traced (T < 1 exactly when the segment blended a hit, alpha >=
// alpha_min > 0).  Persistent with per-lane refill, as the forward bounce
// kernel: a lane whose sample is done takes the next one, and traversal runs
// in chunks of kBwdSteps node or leaf steps, so lanes of a warp do not idle
// while one traces a long segment.  Per sample it computes what
// k_bwd_secondary computes after its values trace, in the same order of
// blended hits.
constexpr int kBwdSteps = 64;

__global__ void __launch_bounds__(kBlock, kBwdMinBlocks) k_bwd_secondary_r(BvhView bvh, Consts C, eagpt_camera cam, eagpt_scene sc,
                                                            eagpt_scene_grad gr, const PrimRecB* __restrict__ prim,
                                                            const float* __restrict__ dL, int spp, uint64_t seed,
                                                            int64_t npix, int s0, int batch, float4* per_sample,
                                                            const float4* __restrict__ sb_cache, uint32_t* counter) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  const int lane = threadIdx.x & 31;
  const int64_t total = npix * (int64_t)batch;
  const float invS = 1.f / (float)spp;
  TraceCounters cnt{0, 0, 0, 0, 0};
  RayTrace<kKb> rt;
  AdjointVisitorT<true> av;
  av.shade = bvh.shade;
  av.sc = sc;
  av.gr = gr;
  av.C = C;
  av.mode = 0;
  int64_t t = 0;
  bool active = false, exhausted = false;
  for (;;) {
    const bool want = !active && !exhausted;
    const uint32_t wmask = __ballot_sync(0xffffffffu, want);
    if (wmask) {
      const int leader = __ffs(wmask) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(wmask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (want) {
        const int64_t idx = (int64_t)base + __popc(wmask & ((1u << lane) - 1u));
        if (idx < total) {
          t = idx;
          const int64_t pixel = t % npix;
          const int sl = (int)(t / npix);
          const PrimRecB p = prim[pixel];
          if (p.c.w >= 0.f && !(p.b.w > C.tau_E)) {
            const uint32_t sample = (uint32_t)(s0 + sl);
            const float4 c = sb_cache[(int64_t)sample * npix + pixel];
            if (c.w < 1.f) {  // the secondary segment blended a hit
              const float4 u = draws(seed, (uint32_t)pixel, sample, 1u);
              float3 O, w;
              camera_ray(cam, (uint32_t)pixel, O, w);
              const float3 Nn = make_float3(p.a.x, p.a.y, p.a.z);
              const float3 O2 = (O + p.a.w * w) + C.bounce_offset * Nn;
              const float3 w2 = cosine_direction(Nn, u.x, u.y);
              const float3 g = make_float3(dL[3 * pixel], dL[3 * pixel + 1], dL[3 * pixel + 2]);
              av.O = O2;
              av.w = w2;
              av.gN = av.gP = make_float3(0.f, 0.f, 0.f);
              av.gR = invS * mul3(g, make_float3(p.c.x, p.c.y, p.c.z));
              av.gD = av.gA = 0.f;
              init_blend(av.V);
              av.V.R = make_float3(c.x, c.y, c.z);
              av.V.T = c.w;
              init_blend(av.run);
              av.dO = av.dw = make_float3(0.f, 0.f, 0.f);
              ray_begin(rt, O2, w2, bvh);
              active = true;
            }
          }
          if (!active) {
            per_sample[2 * t] = make_float4(0.f, 0.f, 0.f, 0.f);
            per_sample[2 * t + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        } else {
          exhausted = true;
        }
      }
    }
    if (!__any_sync(0xffffffffu, active)) break;
    if (active && round_steps<kKb, false>(rt, bvh, C, s_stack + threadIdx.x, kBlock, kBwdSteps, cnt)) {
      if (round_blend<kKb, false>(rt, bvh, C, av, cnt)) {
        // O2 = O + D~1 w + offset N~1 ; w2 = basis(N~1) l  (the sample's
        // primary data are re-read here rather than kept across the trace)
        const int64_t pixel = t % npix;
        const uint32_t sample = (uint32_t)(s0 + (int)(t / npix));
        const PrimRecB p = prim[pixel];
        const float4 u = draws(seed, (uint32_t)pixel, sample, 1u);
        float3 O, w;
        camera_ray(cam, (uint32_t)pixel, O, w);
        const float3 Nn = make_float3(p.a.x, p.a.y, p.a.z);
        const float4 c = sb_cache[(int64_t)sample * npix + pixel];
        const float3 g = make_float3(dL[3 * pixel], dL[3 * pixel + 1], dL[3 * pixel + 2]);
        const float gDn = dot3(av.dO, w);
        const float3 gNn = C.bounce_offset * av.dO + cosine_direction_adjoint(Nn, u.x, u.y, av.dw);
        const float3 gP1 = invS * mul3(g, make_float3(c.x, c.y, c.z));
        per_sample[2 * t] = make_float4(gNn.x, gNn.y, gNn.z, gDn);
        per_sample[2 * t + 1] = make_float4(gP1.x, gP1.y, gP1.z, 0.f);
        active = false;
      } else {
        round_next(rt, bvh);
      }
    }
  }
}

__global__ void k_bwd_reduce(int64_t npix, int batch, int first, const float4* __restrict__ per_sample, float4* acc) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npix) return;
  float4 a = first ? make_float4(0.f, 0.f, 0.f, 0.f) : acc[2 * i];
  float4 b = first ? make_float4(0.f, 0.f, 0.f, 0.f) : acc[2 * i + 1];
  for (int s = 0; s < batch; ++s) {
    const float4 x = per_sample[2 * ((int64_t)s * npix + i)];
    const float4 y = per_sample[2 * ((int64_t)s * npix + i) + 1];
    a.x += x.x;
    a.y += x.y;
    a.z += x.z;
    a.w += x.w;
    b.x += y.x;
    b.y += y.y;
    b.z += y.z;
  }
  acc[2 * i] = a;
  acc[2 * i + 1] = b;
}

__global__ void __launch_bounds__(kBlock) k_bwd_primary(BvhView bvh, Consts C, eagpt_camera cam, eagpt_scene sc,
                                                        eagpt_scene_grad gr, const PrimRecB* __restrict__ prim,
                                                        const float* __restrict__ dL, int64_t npix,
                                                        const float4* __restrict__ acc) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  const int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  if (i >= npix) return;
  const PrimRecB p = prim[i];
  if (!(p.c.w >= 0.f)) return;  // miss
  float3 O, w;
  camera_ray(cam, (uint32_t)i, O, w);
  TraceCounters cnt{0, 0, 0, 0, 0};
  RawVisitor v1(bvh.shade, C, w, 0);
  trace_segment<kKb, false>(bvh, C, O, w, s_stack + threadIdx.x, kBlock, v1, cnt);
  const Blend& V = v1.blend.b;
  AdjointVisitor av;
  av.shade = bvh.shade;
  av.sc = sc;
  av.gr = gr;
  av.C = C;
  av.O = O;
  av.w = w;
  av.mode = 0;
  av.V = V;
  init_blend(av.run);
  av.dO = av.dw = make_float3(0.f, 0.f, 0.f);
  const float3 g = make_float3(dL[3 * i], dL[3 * i + 1], dL[3 * i + 2]);
  if (p.b.w > C.tau_E) {
    // emitter pixel: I = R1
    av.gN = av.gP = make_float3(0.f, 0.f, 0.f);
    av.gR = g;
    av.gD = av.gA = 0.f;
  } else {
    const float4 a = acc[2 * i], b = acc[2 * i + 1];
    const float3 gNn = f3(a);
    const float gDn = a.w;
    const float A = 1.f - V.T;
    const float nn = sqrtf(dot3(V.N, V.N));
    const float3 Nn = (1.f / nn) * V.N;
    const float proj = dot3(Nn, gNn);
    av.gN = (1.f / nn) * (gNn - proj * Nn);
    av.gD = gDn / A;
    av.gA = -gDn * V.D / (A * A);
    av.gP = f3(b);
    av.gR = make_float3(0.f, 0.f, 0.f);
  }
  trace_segment<kKb, false>(bvh, C, O, w, s_stack + threadIdx.x, kBlock, av, cnt);
}

// --------------------------------------------------------------------------
struct BwdLayout {
  size_t prim, acc, per_sample, counter, total;
  int batch;
};

static BwdLayout bwd_layout(int64_t npix, int batch) {
  BwdLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.prim = take((size_t)npix * sizeof(PrimRecB));
  L.acc = take((size_t)npix * 2 * sizeof(float4));
  L.per_sample = take((size_t)npix * batch * 2 * sizeof(float4));
  L.counter = take(sizeof(uint32_t));  // work counter of the refill kernel
  L.total = o;
  L.batch = batch;
  return L;
}

size_t backward_workspace_bytes(int64_t npix, int spp, int batch) {
  (void)spp;
  return bwd_layout(npix, batch).total;
}

int backward_choose_batch(int64_t npix, int spp, size_t ws_bytes) {
  if (bwd_layout(npix, 1).total > ws_bytes) return 0;
  int lo = 1, hi = spp;
  while (lo < hi) {
    const int mid = lo + (hi - lo + 1) / 2;
    if (bwd_layout(npix, mid).total <= ws_bytes) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

static inline unsigned nb(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

cudaError_t launch_backward(const BvhView& bvh, const Consts& C, const eagpt_camera& cam, const eagpt_scene& sc,
                            const eagpt_scene_grad& gr, int spp, uint64_t seed, const float* dL, void* ws,
                            size_t ws_bytes, cudaStream_t st, const float4* sb_cache) {
  const int64_t npix = (int64_t)cam.width * cam.height;
  const int batch = backward_choose_batch(npix, spp, ws_bytes);
  const BwdLayout L = bwd_layout(npix, batch);
  char* base = (char*)ws;
  PrimRecB* prim = (PrimRecB*)(base + L.prim);
  float4* acc = (float4*)(base + L.acc);
  float4* per = (float4*)(base + L.per_sample);
  cudaError_t e = launch_primary_records(bvh, C, cam, 0, npix, (void*)prim, st);
  if (e != cudaSuccess) return e;
  for (int s0 = 0; s0 < spp; s0 += batch) {
    const int n = spp - s0 < batch ? spp - s0 : batch;
    if (sb_cache) {
      uint32_t* counter = (uint32_t*)(base + L.counter);
      e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), st);
      if (e != cudaSuccess) return e;
      EAGPT_LAUNCH(st, "k_bwd_secondary",
                   k_bwd_secondary_r<<<persistent_grid((const void*)k_bwd_secondary_r), kBlock, 0, st>>>(
                       bvh, C, cam, sc, gr, prim, dL, spp, seed, npix, s0, n, per, sb_cache, counter));
    } else {
      EAGPT_LAUNCH(st, "k_bwd_secondary",
                   k_bwd_secondary<<<nb(npix * n), kBlock, 0, st>>>(bvh, C, cam, sc, gr, prim, dL, spp, seed, npix, s0,
                                                                    n, per));
    }
    EAGPT_LAUNCH(st, "k_bwd_reduce", k_bwd_reduce<<<nb(npix), kBlock, 0, st>>>(npix, n, s0 == 0, per, acc));
  }
  EAGPT_LAUNCH(st, "k_bwd_primary",
               k_bwd_primary<<<nb(npix), kBlock, 0, st>>>(bvh, C, cam, sc, gr, prim, dL, npix, acc));
  return cudaGetLastError();
}

}  // namespace eagpt

namespace eagpt {

// Adjoint of the 0-bounce render: dL/dR of each pixel's primary segment.
__global__ void __launch_bounds__(kBlock) k_radiance_bwd(BvhView bvh, Consts C, eagpt_camera cam, eagpt_scene sc,
                                                         eagpt_scene_grad gr, const float* __restrict__ dL,
                                                         int64_t npix) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  const int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  if (i >= npix) return;
  float3 O, w;
  camera_ray(cam, (uint32_t)i, O, w);
  TraceCounters cnt{0, 0, 0, 0, 0};
  RBlendVisitor v1(bvh.shade, C, 0);
  trace_segment<kKb, false>(bvh, C, O, w, s_stack + threadIdx.x, kBlock, v1, cnt);
  if (v1.n_hits == 0) return;
  AdjointVisitorT<true> av;
  av.shade = bvh.shade;
  av.sc = sc;
  av.gr = gr;
  av.C = C;
  av.O = O;
  av.w = w;
  av.mode = 0;
  init_blend(av.V);
  av.V.R = v1.R;
  av.V.T = v1.T;
  init_blend(av.run);
  av.dO = av.dw = make_float3(0.f, 0.f, 0.f);
  av.gN = av.gP = make_float3(0.f, 0.f, 0.f);
  av.gR = make_float3(dL[3 * i], dL[3 * i + 1], dL[3 * i + 2]);
  av.gD = av.gA = 0.f;
  trace_segment<kKb, false>(bvh, C, O, w, s_stack + threadIdx.x, kBlock, av, cnt);
}

cudaError_t launch_radiance_backward(const BvhView& bvh, const Consts& C, const eagpt_camera& cam,
                                     const eagpt_scene& sc, const eagpt_scene_grad& gr, const float* dL,
                                     cudaStream_t st) {
  const int64_t npix = (int64_t)cam.width * cam.height;
  if (bvh.n <= 0) return cudaSuccess;
  EAGPT_LAUNCH(st, "k_radiance_bwd", k_radiance_bwd<<<nb(npix), kBlock, 0, st>>>(bvh, C, cam, sc, gr, dL, npix));
  return cudaGetLastError();
}

}  // namespace eagpt
