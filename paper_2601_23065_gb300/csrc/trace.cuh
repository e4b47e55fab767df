// Segment tracing through the surfel BVH (Sec. 3.1, Eq. 1-3).
//
// A segment (origin O, unit direction w, hits with t > 0) is traced in
// rounds.  Each round walks the BVH from the root and keeps the K nearest
// not-yet-blended hits, ordered by (t, BVH position), in a register k-buffer;
// child boxes entered beyond the buffer's K-th hit are culled.  The round's
// hits are then handed in order to a visitor (the front-to-back blend of
// Eq. 2, or the adjoint), which may stop the segment (transmittance below
// T_min).  A new round starts after the last handed hit only when the buffer
// was full, so every hit is visited exactly once and in depth order.
// (Resuming a round from the subtrees the previous one culled, instead of
// from the root, saves the re-walk of the tree's top but measured slower on
// GB300: the saved visits hit the L1/L2, the bookkeeping does not.)
//
// The intersection is written with explicit round-to-nearest intrinsics so
// that recomputing it for a buffered hit gives bit-identical t and alpha.
#pragma once

#include "common.cuh"

namespace eagpt {

// 32 bytes in one 256-bit load of read-only data (p 32-byte aligned)
__device__ __forceinline__ void ld_v8(const void* p, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

// A surfel's trace record in two 256-bit loads.
__device__ __forceinline__ TraceRec load_trace(const TraceRec* rp) {
  TraceRec R;
  ld_v8(rp, R.r0, R.r1);
  ld_v8((const char*)rp + 32, R.r2, R.r3);
  return R;
}

// A surfel's shade record in one 256-bit load.
__device__ __forceinline__ void load_shade(const ShadeRec* sp, float4& s0, float4& s1) { ld_v8(sp, s0, s1); }

__device__ __forceinline__ float dot3_rn(float3 a, float3 b) {
  return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}

struct HitGeom {
  float t, alpha, sg, u, v, d;
};

// Ray-surfel hit (Eq. 1): plane distance t, local (u, v), response
// g = exp(-(u^2 + v^2)/2), alpha = min(sigma g, alpha_max).  Returns false if
// the ray is parallel, outside the support or below alpha_min.  The t > 0
// test (against the last blended key) is left to the caller.
__device__ __forceinline__ bool intersect(const TraceRec& R, float3 O, float3 w, const Consts& C, HitGeom& h) {
  const float3 p = f3(R.r0), n = f3(R.r1), a = f3(R.r2), b = f3(R.r3);
  const float d = dot3_rn(w, n);
  if (!(fabsf(d) >= 1e-12f)) return false;
  const float3 op = make_float3(__fsub_rn(O.x, p.x), __fsub_rn(O.y, p.y), __fsub_rn(O.z, p.z));
  const float t = __fdiv_rn(-dot3_rn(op, n), d);
  const float3 x = make_float3(__fmaf_rn(t, w.x, op.x), __fmaf_rn(t, w.y, op.y), __fmaf_rn(t, w.z, op.z));
  const float u = dot3_rn(x, a), v = dot3_rn(x, b);
  const float q = __fmaf_rn(u, u, __fmul_rn(v, v));
  if (!(q <= C.support2)) return false;
  const float sg = __fmul_rn(R.r0.w, expf(-0.5f * q));  // expf: within 2 ulps
  const float alpha = fminf(sg, C.alpha_max);
  if (!(alpha >= C.alpha_min)) return false;
  h.t = t;
  h.alpha = alpha;
  h.sg = sg;
  h.u = u;
  h.v = v;
  h.d = d;
  return true;
}

__device__ __forceinline__ bool key_less(float ta, uint32_t ia, float tb, uint32_t ib) {
  return ta < tb || (ta == tb && ia < ib);
}

// Counters of the work one segment did (enabled by the kCount template flag).
struct TraceCounters {
  uint32_t nodes, tests, blended, rounds, max_stack;
};

// Traversal state of one segment.  `stack` arguments point at this thread's
// column of a shared-memory array (kStackSize entries, `stride` words apart).
template <int K>
struct RayTrace {
  float3 O, w, inv;
  float t_last;
  uint32_t j_last;
  float kt[K];
  uint32_t kj[K];
  int count, sp;
  uint32_t cur;
};

template <int K>
__device__ __forceinline__ uint32_t pop(RayTrace<K>& r, const uint32_t* stack, int stride) {
  return r.sp > 0 ? stack[(--r.sp) * stride] : kEmptyChild;
}

// One single-surfel leaf: a hit with key (t, j) above the last blended key
// enters the sorted register buffer (the farthest drops out when it is full).
template <int K, bool kCount>
__device__ __forceinline__ void leaf_step(RayTrace<K>& r, const BvhView& bvh, const Consts& C, uint32_t leaf,
                                          TraceCounters& cnt) {
  const uint32_t j = leaf & kLeafStartMask;
  const TraceRec R = load_trace(bvh.trace + j);
  if (kCount) ++cnt.tests;
  HitGeom h;
  if (!intersect(R, r.O, r.w, C, h)) return;
  if (!key_less(r.t_last, r.j_last, h.t, j)) return;  // already blended (or behind)
  if (r.count == K && !key_less(h.t, j, r.kt[K - 1], r.kj[K - 1])) return;
  float ct = h.t;
  uint32_t cj = j;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const bool lt = key_less(ct, cj, r.kt[i], r.kj[i]);
    const float tt = r.kt[i];
    const uint32_t tj = r.kj[i];
    r.kt[i] = lt ? ct : tt;
    r.kj[i] = lt ? cj : tj;
    ct = lt ? tt : ct;
    cj = lt ? tj : cj;
  }
  r.count = r.count < K ? r.count + 1 : K;
}

// One BVH4 node: slab-test the four child boxes against [t_last, tmax] (tmax
// = the K-th hit when the buffer is full), push the hit children but the
// nearest (farthest first) and return the nearest, or kEmptyChild.  The node
// is read in four 256-bit loads (rows: lo x, y | lo z, hi x | hi y, z | links,
// pad); per axis the plane the ray enters first is the low one when the
// direction is positive, so the near and far planes are picked in registers
// by the direction's signs and each distance is one FMA, p inv - O inv (the
// rounding of O inv is a few ulps of |O|, well inside the boxes' 1e-5
// relative inflation).  Returns false on stack overflow.
template <int K>
__device__ __forceinline__ bool node_step(RayTrace<K>& r, const BvhView& bvh, uint32_t node, uint32_t* stack,
                                          int stride, uint32_t& next) {
  const float inf = __int_as_float(0x7f800000);
  const float tmax = r.count == K ? r.kt[K - 1] : inf;
  const float* nb = (const float*)(bvh.nodes + node);
  float v[32];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[8 * q]), "=f"(v[8 * q + 1]), "=f"(v[8 * q + 2]), "=f"(v[8 * q + 3]), "=f"(v[8 * q + 4]),
          "=f"(v[8 * q + 5]), "=f"(v[8 * q + 6]), "=f"(v[8 * q + 7])
        : "l"(nb + 8 * q));
  uint32_t c[4] = {__float_as_uint(v[24]), __float_as_uint(v[25]), __float_as_uint(v[26]), __float_as_uint(v[27])};
  float e[4];
  {
    const float3 inv = r.inv;
    const bool px = !(inv.x < 0.f), py = !(inv.y < 0.f), pz = !(inv.z < 0.f);
    const float ox = r.O.x * inv.x, oy = r.O.y * inv.y, oz = r.O.z * inv.z;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float nx = px ? v[k] : v[12 + k], fx = px ? v[12 + k] : v[k];
      const float ny = py ? v[4 + k] : v[16 + k], fy = py ? v[16 + k] : v[4 + k];
      const float nz = pz ? v[8 + k] : v[20 + k], fz = pz ? v[20 + k] : v[8 + k];
      const float t0 = fmaxf(fmaxf(__fmaf_rn(nx, inv.x, -ox), __fmaf_rn(ny, inv.y, -oy)),
                             fmaxf(__fmaf_rn(nz, inv.z, -oz), r.t_last));
      const float t1 = fminf(fminf(__fmaf_rn(fx, inv.x, -ox), __fmaf_rn(fy, inv.y, -oy)),
                             fminf(__fmaf_rn(fz, inv.z, -oz), tmax));
      e[k] = (t0 <= t1 && c[k] != kEmptyChild) ? t0 : inf;
    }
  }
  // front-to-back order: sorting network on (entry, link)
#define EAGPT_CSWAP(i, j)                         \
  if (e[j] < e[i]) {                              \
    const float tf = e[i];                        \
    e[i] = e[j];                                  \
    e[j] = tf;                                    \
    const uint32_t tc = c[i];                     \
    c[i] = c[j];                                  \
    c[j] = tc;                                    \
  }
  EAGPT_CSWAP(0, 1)
  EAGPT_CSWAP(2, 3)
  EAGPT_CSWAP(0, 2)
  EAGPT_CSWAP(1, 3)
  EAGPT_CSWAP(1, 2)
#undef EAGPT_CSWAP
  next = kEmptyChild;
  if (e[0] != inf) {
    const int m = (e[1] != inf) + (e[2] != inf) + (e[3] != inf);
    if (r.sp + m > kStackSize) {
      raise_error(kErrStackOverflow);
      return false;
    }
    if (e[3] != inf) stack[(r.sp++) * stride] = c[3];
    if (e[2] != inf) stack[(r.sp++) * stride] = c[2];
    if (e[1] != inf) stack[(r.sp++) * stride] = c[1];
    next = c[0];
  }
  return true;
}

template <int K>
__device__ __forceinline__ void round_reset(RayTrace<K>& r, const BvhView& bvh) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    r.kt[i] = __int_as_float(0x7f800000);  // +inf
    r.kj[i] = 0xFFFFFFFFu;
  }
  r.count = 0;
  r.sp = 0;
  r.cur = bvh.n > 0 ? bvh.root : kEmptyChild;
}

// A new segment and its first round.
template <int K>
__device__ __forceinline__ void ray_begin(RayTrace<K>& r, float3 O, float3 w, const BvhView& bvh) {
  const float big = 1e30f;
  r.O = O;
  r.w = w;
  r.inv = make_float3(fabsf(w.x) > 1e-30f ? 1.0f / w.x : copysignf(big, w.x),
                      fabsf(w.y) > 1e-30f ? 1.0f / w.y : copysignf(big, w.y),
                      fabsf(w.z) > 1e-30f ? 1.0f / w.z : copysignf(big, w.z));
  r.t_last = 0.f;
  r.j_last = 0xFFFFFFFFu;
  round_reset(r, bvh);
}

// The next round of an unfinished segment (after round_blend returned false):
// a walk from the root for the hits beyond the last blended key.
template <int K>
__device__ __forceinline__ void round_next(RayTrace<K>& r, const BvhView& bvh) {
  round_reset(r, bvh);
}

// At most `steps` node or leaf steps of the current round; true once the
// round's walk is complete.  A stack overflow (recorded as a device error)
// ends the walk.
template <int K, bool kCount>
__device__ __forceinline__ bool round_steps(RayTrace<K>& r, const BvhView& bvh, const Consts& C, uint32_t* stack,
                                            int stride, int steps, TraceCounters& cnt) {
  for (int s = 0; s < steps && r.cur != kEmptyChild; ++s) {
    if (r.cur & kLeafBit) {
      leaf_step<K, kCount>(r, bvh, C, r.cur, cnt);
      r.cur = pop(r, stack, stride);
    } else {
      if (kCount) ++cnt.nodes;
      uint32_t next;
      if (!node_step<K>(r, bvh, r.cur, stack, stride, next)) {
        r.cur = kEmptyChild;
        break;
      }
      if (kCount && (uint32_t)r.sp > cnt.max_stack) cnt.max_stack = (uint32_t)r.sp;
      r.cur = next != kEmptyChild ? next : pop(r, stack, stride);
    }
  }
  return r.cur == kEmptyChild;
}

// Blends the round's hits in order; true when the segment is finished (the
// visitor stopped it, or the buffer was not full), otherwise the next round
// starts after the last key (call round_next).
template <int K, bool kCount, class Visitor>
__device__ __forceinline__ bool round_blend(RayTrace<K>& r, const BvhView& bvh, const Consts& C, Visitor& vis,
                                            TraceCounters& cnt) {
  bool stop = false;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    if (i < r.count && !stop) {
      const uint32_t j = r.kj[i];
      const TraceRec R = load_trace(bvh.trace + j);
      HitGeom h;
      intersect(R, r.O, r.w, C, h);  // bit-identical to the collection pass
      if (kCount) ++cnt.blended;
      stop = vis(R, j, h);
    }
  }
  if (stop || r.count < K) return true;
  r.t_last = r.kt[K - 1];
  r.j_last = r.kj[K - 1];
  return false;
}

// Traces one segment to its end and calls vis(R, j, h) for every blended hit
// in order; vis returns true to stop.
template <int K, bool kCount, class Visitor>
__device__ __forceinline__ void trace_segment(const BvhView& bvh, const Consts& C, float3 O, float3 w,
                                              uint32_t* stack, int stride, Visitor& vis, TraceCounters& cnt) {
  if (bvh.n <= 0) return;
  RayTrace<K> r;
  ray_begin(r, O, w, bvh);
  for (;;) {
    if (kCount) ++cnt.rounds;
    round_steps<K, kCount>(r, bvh, C, stack, stride, 1 << 30, cnt);
    if (round_blend<K, kCount>(r, bvh, C, vis, cnt)) return;
    round_next(r, bvh);
  }
}

// Blend state of one segment (Eq. 2): raw sums N, D, R, E, P and T.
struct Blend {
  float3 N, R, P;
  float D, E, T;
  uint32_t n_hits;
};

// The front-to-back blend of Eq. 2-3.  mode 1 drops the radiance of
// non-emitters (path tracing, Sec. 3.4).
struct BlendVisitor {
  const ShadeRec* shade;
  Consts C;
  float3 w;
  int mode;
  Blend b;
  __device__ __forceinline__ BlendVisitor(const ShadeRec* s, const Consts& c, float3 dir, int m)
      : shade(s), C(c), w(dir), mode(m) {
    b.N = b.R = b.P = make_float3(0.f, 0.f, 0.f);
    b.D = b.E = 0.f;
    b.T = 1.f;
    b.n_hits = 0;
  }
  // explicit roundings (one FMA per sum), shared with SmemBlendVisitor, so
  // that every kernel that blends produces the same bits
  __device__ __forceinline__ bool operator()(const TraceRec& R, uint32_t j, const HitGeom& h) {
    const ShadeRec* sp = shade + j;
    float4 s0, s1;
    load_shade(sp, s0, s1);
    const float wgt = __fmul_rn(b.T, h.alpha);
    const float sgn = h.d > 0.f ? -wgt : wgt;  // normal facing the ray origin
    const float re = (mode == 1 && !(s0.w > C.tau_E)) ? 0.f : wgt;
    b.N = make_float3(__fmaf_rn(sgn, R.r1.x, b.N.x), __fmaf_rn(sgn, R.r1.y, b.N.y), __fmaf_rn(sgn, R.r1.z, b.N.z));
    b.D = __fmaf_rn(wgt, h.t, b.D);
    b.R = make_float3(__fmaf_rn(re, s1.x, b.R.x), __fmaf_rn(re, s1.y, b.R.y), __fmaf_rn(re, s1.z, b.R.z));
    b.E = __fmaf_rn(wgt, s0.w, b.E);
    b.P = make_float3(__fmaf_rn(wgt, s0.x, b.P.x), __fmaf_rn(wgt, s0.y, b.P.y), __fmaf_rn(wgt, s0.z, b.P.z));
    b.T = __fmul_rn(b.T, __fsub_rn(1.f, h.alpha));
    ++b.n_hits;
    return b.T < C.T_min;
  }
};

// The same blend with the running sums (all but T) in this thread's slot of
// a shared-memory array, s[k * stride] for k = 0..10 (N xyz, R xyz, P xyz, D,
// E): during a multi-round traversal they stay out of the register file.
// kMis: the continuation segment of the emitter-sampling path tracer; each
// emitter hit's radiance term is weighted by the power heuristic
// p_B^2 / (p_B^2 + p_L^2), p_L = c g(u, v) t^2 / |w . n| with c the emitter's
// density factor kept in its shade record (s1.w, 0 for non-emitters).
template <bool kMis>
struct SmemBlendVisitorT {
  const ShadeRec* shade;
  Consts C;
  int mode;
  float* s;
  int stride;
  float T;
  uint32_t n_hits;
  float pb2;  // kMis: p_B^2 of the segment's direction
  __device__ __forceinline__ SmemBlendVisitorT(const ShadeRec* sh, const Consts& c, int m, float* slot, int str)
      : shade(sh), C(c), mode(m), s(slot), stride(str), T(1.f), n_hits(0), pb2(0.f) {
    reset();
  }
  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int k = 0; k < 11; ++k) s[k * stride] = 0.f;
    T = 1.f;
    n_hits = 0;
  }
  __device__ __forceinline__ bool operator()(const TraceRec& R, uint32_t j, const HitGeom& h) {
    const ShadeRec* sp = shade + j;
    float4 s0, s1;
    load_shade(sp, s0, s1);
    const float wgt = __fmul_rn(T, h.alpha);
    const float sgn = h.d > 0.f ? -wgt : wgt;
    float re = (mode == 1 && !(s0.w > C.tau_E)) ? 0.f : wgt;
    if (kMis && re != 0.f) {
      const float pl = s1.w * expf(-0.5f * (h.u * h.u + h.v * h.v)) * (h.t * h.t) / fabsf(h.d);
      re = re * (pb2 / (pb2 + pl * pl));
    }
    s[0 * stride] = __fmaf_rn(sgn, R.r1.x, s[0 * stride]);
    s[1 * stride] = __fmaf_rn(sgn, R.r1.y, s[1 * stride]);
    s[2 * stride] = __fmaf_rn(sgn, R.r1.z, s[2 * stride]);
    s[3 * stride] = __fmaf_rn(re, s1.x, s[3 * stride]);
    s[4 * stride] = __fmaf_rn(re, s1.y, s[4 * stride]);
    s[5 * stride] = __fmaf_rn(re, s1.z, s[5 * stride]);
    s[6 * stride] = __fmaf_rn(wgt, s0.x, s[6 * stride]);
    s[7 * stride] = __fmaf_rn(wgt, s0.y, s[7 * stride]);
    s[8 * stride] = __fmaf_rn(wgt, s0.z, s[8 * stride]);
    s[9 * stride] = __fmaf_rn(wgt, h.t, s[9 * stride]);
    s[10 * stride] = __fmaf_rn(wgt, s0.w, s[10 * stride]);
    T = __fmul_rn(T, __fsub_rn(1.f, h.alpha));
    ++n_hits;
    return T < C.T_min;
  }
  __device__ __forceinline__ Blend get() const {
    Blend b;
    b.N = make_float3(s[0], s[stride], s[2 * stride]);
    b.R = make_float3(s[3 * stride], s[4 * stride], s[5 * stride]);
    b.P = make_float3(s[6 * stride], s[7 * stride], s[8 * stride]);
    b.D = s[9 * stride];
    b.E = s[10 * stride];
    b.T = T;
    b.n_hits = n_hits;
    return b;
  }
};
using SmemBlendVisitor = SmemBlendVisitorT<false>;

// NeeVisitor with its state (E, target weight, light pdf, found flag, target
// record) in a per-thread shared-memory slot s[k * stride], k = 0..4, and only
// T in a register.
struct NeeVisitorSM {
  const ShadeRec* shade;
  Consts C;
  float* s;
  int stride;
  float T;
  __device__ __forceinline__ void reset(uint32_t target) {
    T = 1.f;
    s[0] = 0.f;
    s[stride] = 0.f;
    s[2 * stride] = 0.f;
    s[3 * stride] = 0.f;
    s[4 * stride] = __uint_as_float(target);
  }
  __device__ __forceinline__ float E() const { return s[0]; }
  __device__ __forceinline__ float wt() const { return s[stride]; }
  __device__ __forceinline__ float pl() const { return s[2 * stride]; }
  __device__ __forceinline__ bool found() const { return s[3 * stride] != 0.f; }
  __device__ __forceinline__ uint32_t target() const { return __float_as_uint(s[4 * stride]); }
  __device__ __forceinline__ bool operator()(const TraceRec&, uint32_t j, const HitGeom& h) {
    const ShadeRec* sp = shade + j;
    const float wgt = __fmul_rn(T, h.alpha);
    s[0] = __fmaf_rn(wgt, __ldg(&sp->s0.w), s[0]);
    if (j == target()) {
      s[stride] = wgt;
      s[2 * stride] = __ldg(&sp->s1.w) * expf(-0.5f * (h.u * h.u + h.v * h.v)) * (h.t * h.t) / fabsf(h.d);
      s[3 * stride] = 1.f;
    }
    T = __fmul_rn(T, __fsub_rn(1.f, h.alpha));
    return T < C.T_min;
  }
};

// The emitter-sample segment: the blend's E and T (same arithmetic and
// stopping rule as the other visitors) and, when the target emitter record jt
// is blended, its weight w = T_{i-1} alpha and its light pdf.
struct NeeVisitor {
  const ShadeRec* shade;
  Consts C;
  uint32_t jt;
  float T, E, wt, pl;
  bool found;
  __device__ __forceinline__ void reset(uint32_t target) {
    jt = target;
    T = 1.f;
    E = 0.f;
    wt = 0.f;
    pl = 0.f;
    found = false;
  }
  __device__ __forceinline__ bool operator()(const TraceRec&, uint32_t j, const HitGeom& h) {
    const ShadeRec* sp = shade + j;
    const float wgt = __fmul_rn(T, h.alpha);
    E = __fmaf_rn(wgt, __ldg(&sp->s0.w), E);
    if (j == jt) {
      found = true;
      wt = wgt;
      pl = __ldg(&sp->s1.w) * expf(-0.5f * (h.u * h.u + h.v * h.v)) * (h.t * h.t) / fabsf(h.d);
    }
    T = __fmul_rn(T, __fsub_rn(1.f, h.alpha));
    return T < C.T_min;
  }
};

// Normalised record of a blended segment: N~ = N/|N|, D~ = D/A, A = 1 - T.
struct SegRec {
  float3 Nn, R, P;
  float Dn, E, A;
  bool hit;
};

__device__ __forceinline__ SegRec finish(const Blend& b) {
  SegRec s;
  s.A = 1.f - b.T;
  s.R = b.R;
  s.P = b.P;
  s.E = b.E;
  s.hit = b.n_hits > 0;
  if (s.hit) {
    const float inv = rsqrtf(dot3(b.N, b.N));
    s.Nn = inv * b.N;
    s.Dn = b.D / s.A;
  } else {
    s.Nn = make_float3(0.f, 0.f, 0.f);
    s.Dn = 0.f;
  }
  return s;
}

}  // namespace eagpt
