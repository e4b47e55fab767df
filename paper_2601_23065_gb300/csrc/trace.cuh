// Segment tracing through the surfel BVH (Sec. 3.1, Eq. 1-3).
//
// A segment (origin O, unit direction w, hits with t > t_lo) is traced in
// rounds.  Each round walks the BVH once and keeps the K nearest not-yet-
// blended hits, ordered by (t, BVH position), in a register k-buffer; the
// round's hits are then handed in order to a visitor (the front-to-back blend
// of Eq. 2, or the adjoint), which may stop the segment (transmittance below
// T_min).  A new round starts after the last handed hit only when the buffer
// was full, so every hit is visited exactly once and in depth order.
//
// The intersection is written with explicit round-to-nearest intrinsics so
// that recomputing it for a buffered hit gives bit-identical t and alpha.
#pragma once

#include "common.cuh"

#ifndef EAGPT_WHILE_WHILE
#define EAGPT_WHILE_WHILE 0
#endif
#ifndef EAGPT_INLINE_LEAVES
#define EAGPT_INLINE_LEAVES 0
#endif

namespace eagpt {

#ifndef EAGPT_V8REC
#define EAGPT_V8REC 1
#endif

// the 256-bit load's form (cache operator and hint): 0 read-only (.nc),
// 1 plain, 2 .ca, 3 read-only with an L1 evict-last hint
#ifndef EAGPT_V8_KIND
#define EAGPT_V8_KIND 0
#endif
#if EAGPT_V8_KIND == 1
#define EAGPT_LD_V8 "ld.global.v8.f32"
#elif EAGPT_V8_KIND == 2
#define EAGPT_LD_V8 "ld.global.ca.v8.f32"
#elif EAGPT_V8_KIND == 3
#define EAGPT_LD_V8 "ld.global.nc.L1::evict_last.v8.f32"
#else
#define EAGPT_LD_V8 "ld.global.nc.v8.f32"
#endif

// 32 bytes in one 256-bit load of read-only data (p 32-byte aligned)
__device__ __forceinline__ void ld_v8(const void* p, float4& a, float4& b) {
  asm(EAGPT_LD_V8 " {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

// A surfel's trace record (EAGPT_V8REC: two 256-bit loads instead of four).
__device__ __forceinline__ TraceRec load_trace(const TraceRec* rp) {
  TraceRec R;
#if EAGPT_V8REC
  ld_v8(rp, R.r0, R.r1);
  ld_v8((const char*)rp + 32, R.r2, R.r3);
#else
  R.r0 = __ldg(&rp->r0);
  R.r1 = __ldg(&rp->r1);
  R.r2 = __ldg(&rp->r2);
  R.r3 = __ldg(&rp->r3);
#endif
  return R;
}

// A surfel's shade record.
__device__ __forceinline__ void load_shade(const ShadeRec* sp, float4& s0, float4& s1) {
#if EAGPT_V8REC
  ld_v8(sp, s0, s1);
#else
  s0 = __ldg(&sp->s0);
  s1 = __ldg(&sp->s1);
#endif
}

__device__ __forceinline__ float dot3_rn(float3 a, float3 b) {
  return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}

struct HitGeom {
  float t, alpha, sg, u, v, d;
};

// Ray-surfel hit (Eq. 1): plane distance t, local (u, v), response
// g = exp(-(u^2 + v^2)/2), alpha = min(sigma g, alpha_max).  Returns false if
// the ray is parallel, outside the support or below alpha_min.  The t > t_lo
// test is left to the caller.
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

// Slab test of an axis-aligned box against [tmin, tmax]; returns the entry t.
__device__ __forceinline__ bool box_hit(float3 lo, float3 hi, float3 O, float3 inv, float tmin, float tmax,
                                        float& t_enter) {
  const float tx0 = (lo.x - O.x) * inv.x, tx1 = (hi.x - O.x) * inv.x;
  const float ty0 = (lo.y - O.y) * inv.y, ty1 = (hi.y - O.y) * inv.y;
  const float tz0 = (lo.z - O.z) * inv.z, tz1 = (hi.z - O.z) * inv.z;
  const float t0 = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tmin));
  const float t1 = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
  t_enter = t0;
  return t0 <= t1;
}

__device__ __forceinline__ bool key_less(float ta, uint32_t ia, float tb, uint32_t ib) {
  return ta < tb || (ta == tb && ia < ib);
}

#ifndef EAGPT_FAST_SLAB
#define EAGPT_FAST_SLAB 1
#endif

// Counters of the work one segment did (enabled by the kCount template flag).
struct TraceCounters {
  uint32_t nodes, tests, blended, rounds, max_stack;
};

// One leaf: test its surfels and keep the K nearest keys above the last
// blended key in the sorted register buffer.
template <int K, bool kCount>
__device__ __forceinline__ void leaf_step(const BvhView& bvh, const Consts& C, float3 O, float3 w, uint32_t leaf,
                                          float t_last, uint32_t j_last, float (&kt)[K], uint32_t (&kj)[K],
                                          int& count, TraceCounters& cnt) {
  const uint32_t start = leaf & kLeafStartMask;
  const uint32_t cnum = ((leaf >> kLeafCountShift) & 3u) + 1u;
  for (uint32_t j = start; j < start + cnum; ++j) {
    const TraceRec* rp = bvh.trace + j;
    const TraceRec R = load_trace(rp);
    if (kCount) ++cnt.tests;
    HitGeom h;
    if (!intersect(R, O, w, C, h)) continue;
    if (!key_less(t_last, j_last, h.t, j)) continue;  // already blended (or behind)
    if (count == K && !key_less(h.t, j, kt[K - 1], kj[K - 1])) continue;
    float ct = h.t;
    uint32_t cj = j;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const bool lt = key_less(ct, cj, kt[i], kj[i]);
      const float tt = kt[i];
      const uint32_t tj = kj[i];
      kt[i] = lt ? ct : tt;
      kj[i] = lt ? cj : tj;
      ct = lt ? tt : ct;
      cj = lt ? tj : cj;
    }
    count = count < K ? count + 1 : K;
  }
}

// L2 prefetch of the children a node step pushes (EAGPT_PREFETCH): when the
// frame's working set exceeds the L2, a popped child's node or surfel record
// otherwise comes from DRAM on the traversal's dependent chain.
#ifndef EAGPT_PREFETCH
#define EAGPT_PREFETCH 0
#endif
// BVH4 nodes read with 256-bit loads (four per node instead of seven 128-bit;
// 1-2 % faster on the L1-bound bounce kernel)
#ifndef EAGPT_V8NODE
#define EAGPT_V8NODE 1
#endif
__device__ __forceinline__ void prefetch_child(const BvhView& bvh, uint32_t c) {
  const void* p = (c & kLeafBit) ? (const void*)(bvh.trace + (c & kLeafStartMask))
#if EAGPT_QNODE4
                                 : (const void*)(bvh.nodes4q + c);
#else
                                 : (const void*)(bvh.nodes + c);
#endif
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// One BVH4 node: slab-test the four child boxes against [t_last, tmax],
// push the hit children but the nearest (farthest first) and return the
// nearest, or kEmptyChild when none is hit.  Returns false on stack overflow.
__device__ __forceinline__ bool node_step(const BvhView& bvh, uint32_t node, float3 O, float3 inv, float t_last,
                                          float tmax, uint32_t* stack, int stride, int& sp, uint32_t& next) {
  const float inf = __int_as_float(0x7f800000);
  float e[4];
#if EAGPT_QNODE4
  // quantised node: near/far planes by direction sign, decoded exactly as the
  // builder checked them, one FMA per plane
  const Node4q* qp = bvh.nodes4q + node;
  const uint4 u0 = __ldg(&qp->u0), ch = __ldg(&qp->u1), u2 = __ldg(&qp->u2), u3 = __ldg(&qp->u3);
  uint32_t c[4] = {ch.x, ch.y, ch.z, ch.w};
  {
    const float ox = __uint_as_float(u0.x), oy = __uint_as_float(u0.y), oz = __uint_as_float(u0.z);
    const float sx = __uint_as_float((u0.w & 0xFFu) << 23), sy = __uint_as_float(((u0.w >> 8) & 0xFFu) << 23);
    const float sz = __uint_as_float(((u0.w >> 16) & 0xFFu) << 23);
    const bool px = inv.x >= 0.f, py = inv.y >= 0.f, pz = inv.z >= 0.f;
    const uint32_t nqx = px ? u2.x : u3.x, fqx = px ? u3.x : u2.x;
    const uint32_t nqy = py ? u2.y : u3.y, fqy = py ? u3.y : u2.y;
    const uint32_t nqz = pz ? u2.z : u3.z, fqz = pz ? u3.z : u2.z;
    const float oix = O.x * inv.x, oiy = O.y * inv.y, oiz = O.z * inv.z;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int sh = 8 * k;
      const float nx = __fmaf_rn((float)((nqx >> sh) & 0xFFu), sx, ox), fx = __fmaf_rn((float)((fqx >> sh) & 0xFFu), sx, ox);
      const float ny = __fmaf_rn((float)((nqy >> sh) & 0xFFu), sy, oy), fy = __fmaf_rn((float)((fqy >> sh) & 0xFFu), sy, oy);
      const float nz = __fmaf_rn((float)((nqz >> sh) & 0xFFu), sz, oz), fz = __fmaf_rn((float)((fqz >> sh) & 0xFFu), sz, oz);
      const float t0 = fmaxf(fmaxf(__fmaf_rn(nx, inv.x, -oix), __fmaf_rn(ny, inv.y, -oiy)),
                             fmaxf(__fmaf_rn(nz, inv.z, -oiz), t_last));
      const float t1 = fminf(fminf(__fmaf_rn(fx, inv.x, -oix), __fmaf_rn(fy, inv.y, -oiy)),
                             fminf(__fmaf_rn(fz, inv.z, -oiz), tmax));
      e[k] = (t0 <= t1 && c[k] != kEmptyChild) ? t0 : inf;
    }
  }
#elif EAGPT_V8NODE
  // the whole 128-byte node in four 32-byte loads (rows: lo x, y | lo z, hi x
  // | hi y, z | links, pad), near and far planes picked in registers by the
  // direction's signs, then the same one-FMA plane distances as below
  const float* nb = (const float*)(bvh.nodes + node);
  float v[32];
#pragma unroll
  for (int r = 0; r < 4; ++r)
    asm(EAGPT_LD_V8 " {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[8 * r]), "=f"(v[8 * r + 1]), "=f"(v[8 * r + 2]), "=f"(v[8 * r + 3]), "=f"(v[8 * r + 4]),
          "=f"(v[8 * r + 5]), "=f"(v[8 * r + 6]), "=f"(v[8 * r + 7])
        : "l"(nb + 8 * r));
  uint32_t c[4] = {__float_as_uint(v[24]), __float_as_uint(v[25]), __float_as_uint(v[26]), __float_as_uint(v[27])};
  {
    const bool px = !(inv.x < 0.f), py = !(inv.y < 0.f), pz = !(inv.z < 0.f);
    const float ox = O.x * inv.x, oy = O.y * inv.y, oz = O.z * inv.z;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float nx = px ? v[k] : v[12 + k], fx = px ? v[12 + k] : v[k];
      const float ny = py ? v[4 + k] : v[16 + k], fy = py ? v[16 + k] : v[4 + k];
      const float nz = pz ? v[8 + k] : v[20 + k], fz = pz ? v[20 + k] : v[8 + k];
      const float t0 = fmaxf(fmaxf(__fmaf_rn(nx, inv.x, -ox), __fmaf_rn(ny, inv.y, -oy)),
                             fmaxf(__fmaf_rn(nz, inv.z, -oz), t_last));
      const float t1 = fminf(fminf(__fmaf_rn(fx, inv.x, -ox), __fmaf_rn(fy, inv.y, -oy)),
                             fminf(__fmaf_rn(fz, inv.z, -oz), tmax));
      e[k] = (t0 <= t1 && c[k] != kEmptyChild) ? t0 : inf;
    }
  }
#else
  const Node4* np = bvh.nodes + node;
  const uint4 ch = __ldg(&np->child);
  uint32_t c[4] = {ch.x, ch.y, ch.z, ch.w};
#if EAGPT_FAST_SLAB
  // Per axis the plane the ray enters first is the low one when the
  // direction is positive: load the near and far planes directly (the SoA
  // node keeps lo at byte 16 a and hi at 48 + 16 a) and form t = p inv - O inv
  // with one FMA, so no per-child min/max is needed.  The rounding of O inv
  // is a few ulps of |O|, well inside the boxes' 1e-5 relative inflation.
  {
    const char* base = (const char*)np;
    const int sx = inv.x < 0.f ? 48 : 0, sy = inv.y < 0.f ? 48 : 0, sz = inv.z < 0.f ? 48 : 0;
    const float4 nx = __ldg((const float4*)(base + sx)), fx = __ldg((const float4*)(base + 48 - sx));
    const float4 ny = __ldg((const float4*)(base + 16 + sy)), fy = __ldg((const float4*)(base + 64 - sy));
    const float4 nz = __ldg((const float4*)(base + 32 + sz)), fz = __ldg((const float4*)(base + 80 - sz));
    const float ox = O.x * inv.x, oy = O.y * inv.y, oz = O.z * inv.z;
    const float nxa[4] = {nx.x, nx.y, nx.z, nx.w}, nya[4] = {ny.x, ny.y, ny.z, ny.w};
    const float nza[4] = {nz.x, nz.y, nz.z, nz.w}, fxa[4] = {fx.x, fx.y, fx.z, fx.w};
    const float fya[4] = {fy.x, fy.y, fy.z, fy.w}, fza[4] = {fz.x, fz.y, fz.z, fz.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float t0 = fmaxf(fmaxf(__fmaf_rn(nxa[k], inv.x, -ox), __fmaf_rn(nya[k], inv.y, -oy)),
                             fmaxf(__fmaf_rn(nza[k], inv.z, -oz), t_last));
      const float t1 = fminf(fminf(__fmaf_rn(fxa[k], inv.x, -ox), __fmaf_rn(fya[k], inv.y, -oy)),
                             fminf(__fmaf_rn(fza[k], inv.z, -oz), tmax));
      e[k] = (t0 <= t1 && c[k] != kEmptyChild) ? t0 : inf;
    }
  }
#else
  const float4 lx = __ldg(&np->lox), ly = __ldg(&np->loy), lz = __ldg(&np->loz);
  const float4 hx = __ldg(&np->hix), hy = __ldg(&np->hiy), hz = __ldg(&np->hiz);
  {
    const float lxa[4] = {lx.x, lx.y, lx.z, lx.w}, lya[4] = {ly.x, ly.y, ly.z, ly.w};
    const float lza[4] = {lz.x, lz.y, lz.z, lz.w}, hxa[4] = {hx.x, hx.y, hx.z, hx.w};
    const float hya[4] = {hy.x, hy.y, hy.z, hy.w}, hza[4] = {hz.x, hz.y, hz.z, hz.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float te;
      const bool h = box_hit(make_float3(lxa[k], lya[k], lza[k]), make_float3(hxa[k], hya[k], hza[k]), O, inv,
                             t_last, tmax, te);
      e[k] = (h && c[k] != kEmptyChild) ? te : inf;
    }
  }
#endif
#endif  // EAGPT_QNODE4
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
    if (sp + m > kStackSize) {
      raise_error(kErrStackOverflow);
      return false;
    }
    if (e[3] != inf) stack[(sp++) * stride] = c[3];
    if (e[2] != inf) stack[(sp++) * stride] = c[2];
    if (e[1] != inf) stack[(sp++) * stride] = c[1];
    next = c[0];
    if (EAGPT_PREFETCH) {
      if (e[1] != inf) prefetch_child(bvh, c[1]);
      if (e[2] != inf) prefetch_child(bvh, c[2]);
      if (e[3] != inf) prefetch_child(bvh, c[3]);
    }
  }
  return true;
}

// One quantised BVH8 node (see Node8): decode the eight child boxes, slab-
// test them, order the hit children front to back (Batcher's 19-comparator
// network for 8 keys), push all but the nearest.
__device__ __forceinline__ bool node_step8(const BvhView& bvh, uint32_t node, float3 O, float3 inv, float t_last,
                                           float tmax, uint32_t* stack, int stride, int& sp, uint32_t& next) {
  const Node8* np = bvh.nodes8 + node;
  const uint4 u0 = __ldg(&np->u0), u1 = __ldg(&np->u1), u2 = __ldg(&np->u2);
  const uint4 u3 = __ldg(&np->u3), u4 = __ldg(&np->u4), u5 = __ldg(&np->u5);
  const float ox = __uint_as_float(u0.x), oy = __uint_as_float(u0.y), oz = __uint_as_float(u0.z);
  const float sx = __uint_as_float((u0.w & 0xFFu) << 23), sy = __uint_as_float(((u0.w >> 8) & 0xFFu) << 23);
  const float sz = __uint_as_float(((u0.w >> 16) & 0xFFu) << 23);
  const float inf = __int_as_float(0x7f800000);
  float e[8];
  uint32_t c[8] = {u1.x, u1.y, u1.z, u1.w, u2.x, u2.y, u2.z, u2.w};
  const uint32_t qlx[2] = {u3.x, u3.y}, qly[2] = {u3.z, u3.w}, qlz[2] = {u4.x, u4.y};
  const uint32_t qhx[2] = {u4.z, u4.w}, qhy[2] = {u5.x, u5.y}, qhz[2] = {u5.z, u5.w};
#if EAGPT_FAST_SLAB
  // near/far planes by direction sign, decoded exactly as the builder checked
  // them (fma(q, quantum, origin)), then one FMA per plane as in node_step
  const bool px = inv.x >= 0.f, py = inv.y >= 0.f, pz = inv.z >= 0.f;
  const uint32_t nqx[2] = {px ? qlx[0] : qhx[0], px ? qlx[1] : qhx[1]}, fqx[2] = {px ? qhx[0] : qlx[0], px ? qhx[1] : qlx[1]};
  const uint32_t nqy[2] = {py ? qly[0] : qhy[0], py ? qly[1] : qhy[1]}, fqy[2] = {py ? qhy[0] : qly[0], py ? qhy[1] : qly[1]};
  const uint32_t nqz[2] = {pz ? qlz[0] : qhz[0], pz ? qlz[1] : qhz[1]}, fqz[2] = {pz ? qhz[0] : qlz[0], pz ? qhz[1] : qlz[1]};
  const float oix = O.x * inv.x, oiy = O.y * inv.y, oiz = O.z * inv.z;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int w = k >> 2, sh = 8 * (k & 3);
    const float nx = __fmaf_rn((float)((nqx[w] >> sh) & 0xFFu), sx, ox), fx = __fmaf_rn((float)((fqx[w] >> sh) & 0xFFu), sx, ox);
    const float ny = __fmaf_rn((float)((nqy[w] >> sh) & 0xFFu), sy, oy), fy = __fmaf_rn((float)((fqy[w] >> sh) & 0xFFu), sy, oy);
    const float nz = __fmaf_rn((float)((nqz[w] >> sh) & 0xFFu), sz, oz), fz = __fmaf_rn((float)((fqz[w] >> sh) & 0xFFu), sz, oz);
    const float t0 = fmaxf(fmaxf(__fmaf_rn(nx, inv.x, -oix), __fmaf_rn(ny, inv.y, -oiy)),
                           fmaxf(__fmaf_rn(nz, inv.z, -oiz), t_last));
    const float t1 = fminf(fminf(__fmaf_rn(fx, inv.x, -oix), __fmaf_rn(fy, inv.y, -oiy)),
                           fminf(__fmaf_rn(fz, inv.z, -oiz), tmax));
    e[k] = (t0 <= t1 && c[k] != kEmptyChild) ? t0 : inf;
  }
#else
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int w = k >> 2, sh = 8 * (k & 3);
    const float3 lo = make_float3(__fmaf_rn((float)((qlx[w] >> sh) & 0xFFu), sx, ox),
                                  __fmaf_rn((float)((qly[w] >> sh) & 0xFFu), sy, oy),
                                  __fmaf_rn((float)((qlz[w] >> sh) & 0xFFu), sz, oz));
    const float3 hi = make_float3(__fmaf_rn((float)((qhx[w] >> sh) & 0xFFu), sx, ox),
                                  __fmaf_rn((float)((qhy[w] >> sh) & 0xFFu), sy, oy),
                                  __fmaf_rn((float)((qhz[w] >> sh) & 0xFFu), sz, oz));
    float te;
    const bool h = box_hit(lo, hi, O, inv, t_last, tmax, te);
    e[k] = (h && c[k] != kEmptyChild) ? te : inf;
  }
#endif
#define EAGPT_CSWAP(i, j)                         \
  if (e[j] < e[i]) {                              \
    const float tf = e[i];                        \
    e[i] = e[j];                                  \
    e[j] = tf;                                    \
    const uint32_t tc = c[i];                     \
    c[i] = c[j];                                  \
    c[j] = tc;                                    \
  }
  EAGPT_CSWAP(0, 1) EAGPT_CSWAP(2, 3) EAGPT_CSWAP(4, 5) EAGPT_CSWAP(6, 7)
  EAGPT_CSWAP(0, 2) EAGPT_CSWAP(1, 3) EAGPT_CSWAP(4, 6) EAGPT_CSWAP(5, 7)
  EAGPT_CSWAP(1, 2) EAGPT_CSWAP(5, 6)
  EAGPT_CSWAP(0, 4) EAGPT_CSWAP(1, 5) EAGPT_CSWAP(2, 6) EAGPT_CSWAP(3, 7)
  EAGPT_CSWAP(2, 4) EAGPT_CSWAP(3, 5)
  EAGPT_CSWAP(1, 2) EAGPT_CSWAP(3, 4) EAGPT_CSWAP(5, 6)
#undef EAGPT_CSWAP
  next = kEmptyChild;
  if (e[0] != inf) {
    int m = 0;
#pragma unroll
    for (int k = 1; k < 8; ++k) m += e[k] != inf;
    if (sp + m > kStackSize) {
      raise_error(kErrStackOverflow);
      return false;
    }
#pragma unroll
    for (int k = 7; k >= 1; --k)
      if (e[k] != inf) stack[(sp++) * stride] = c[k];
    next = c[0];
  }
  return true;
}

// Like node_step, but the hit leaf children are returned in `leaves` (nl of
// them) instead of being pushed; only inner children are ordered and pushed.
__device__ __forceinline__ bool node_step_split(const BvhView& bvh, uint32_t node, float3 O, float3 inv,
                                                float t_last, float tmax, uint32_t* stack, int stride, int& sp,
                                                uint32_t& next, uint32_t (&leaves)[4], int& nl) {
  const Node4* np = bvh.nodes + node;
  const float4 lx = __ldg(&np->lox), ly = __ldg(&np->loy), lz = __ldg(&np->loz);
  const float4 hx = __ldg(&np->hix), hy = __ldg(&np->hiy), hz = __ldg(&np->hiz);
  const uint4 ch = __ldg(&np->child);
  const float inf = __int_as_float(0x7f800000);
  float e[4];
  uint32_t c[4] = {ch.x, ch.y, ch.z, ch.w};
  {
    const float lxa[4] = {lx.x, lx.y, lx.z, lx.w}, lya[4] = {ly.x, ly.y, ly.z, ly.w};
    const float lza[4] = {lz.x, lz.y, lz.z, lz.w}, hxa[4] = {hx.x, hx.y, hx.z, hx.w};
    const float hya[4] = {hy.x, hy.y, hy.z, hy.w}, hza[4] = {hz.x, hz.y, hz.z, hz.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float te;
      const bool h = box_hit(make_float3(lxa[k], lya[k], lza[k]), make_float3(hxa[k], hya[k], hza[k]), O, inv,
                             t_last, tmax, te);
      const bool ok = h && c[k] != kEmptyChild;
      const bool leaf = ok && (c[k] & kLeafBit);
      leaves[k] = leaf ? c[k] : kEmptyChild;
      nl += leaf;
      e[k] = (ok && !leaf) ? te : inf;
    }
  }
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
    if (sp + m > kStackSize) {
      raise_error(kErrStackOverflow);
      return false;
    }
    if (e[3] != inf) stack[(sp++) * stride] = c[3];
    if (e[2] != inf) stack[(sp++) * stride] = c[2];
    if (e[1] != inf) stack[(sp++) * stride] = c[1];
    next = c[0];
  }
  return true;
}

__device__ __forceinline__ uint32_t pop(const uint32_t* stack, int stride, int& sp) {
  return sp > 0 ? stack[(--sp) * stride] : kEmptyChild;
}

// Walks the BVH for hits with key (t, j) > (t_last, j_last), up to K of
// them, nearest first.  `stack` points at this thread's column of a
// shared-memory stack with `stride` words between entries.
template <int K, bool kCount>
__device__ __forceinline__ int collect_round(const BvhView& bvh, const Consts& C, float3 O, float3 w, float3 inv,
                                             float t_last, uint32_t j_last, float (&kt)[K], uint32_t (&kj)[K],
                                             uint32_t* stack, int stride, TraceCounters& cnt) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    kt[i] = __int_as_float(0x7f800000);  // +inf
    kj[i] = 0xFFFFFFFFu;
  }
  int count = 0;
  int sp = 0;
#if EAGPT_WHILE_WHILE
  // Inner nodes are walked until every lane of the warp holds a leaf (or is
  // done), then the leaves are processed together (Aila and Laine,
  // "Understanding the efficiency of ray traversal on GPUs", HPG 2009).
  uint32_t node = bvh.root, leaf = kEmptyChild;
  for (;;) {
    while (node != kEmptyChild && !(node & kLeafBit)) {
      if (kCount) ++cnt.nodes;
      const float tmax = count == K ? kt[K - 1] : __int_as_float(0x7f800000);
      uint32_t next;
      if (!node_step(bvh, node, O, inv, t_last, tmax, stack, stride, sp, next)) return count;
      node = next != kEmptyChild ? next : pop(stack, stride, sp);
      if (node != kEmptyChild && (node & kLeafBit) && leaf == kEmptyChild) {
        leaf = node;
        node = pop(stack, stride, sp);
      }
      if (!__any_sync(__activemask(), leaf == kEmptyChild)) break;
    }
    while (leaf != kEmptyChild) {
      leaf_step<K, kCount>(bvh, C, O, w, leaf, t_last, j_last, kt, kj, count, cnt);
      leaf = kEmptyChild;
      if (node != kEmptyChild && (node & kLeafBit)) {
        leaf = node;
        node = pop(stack, stride, sp);
      }
    }
    if (node == kEmptyChild) break;
  }
#elif EAGPT_INLINE_LEAVES
  // Leaf children are tested during their parent's visit; only inner nodes
  // go through the stack.
  uint32_t cur = bvh.root;
  while (cur != kEmptyChild) {
    if (kCount) ++cnt.nodes;
    const float tmax = count == K ? kt[K - 1] : __int_as_float(0x7f800000);
    uint32_t next, leaves[4];
    int nl = 0;
    if (!node_step_split(bvh, cur, O, inv, t_last, tmax, stack, stride, sp, next, leaves, nl)) return count;
    if (nl) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (leaves[k] != kEmptyChild) leaf_step<K, kCount>(bvh, C, O, w, leaves[k], t_last, j_last, kt, kj, count, cnt);
    }
    cur = next != kEmptyChild ? next : pop(stack, stride, sp);
  }
#else
  uint32_t cur = bvh.root;
  while (cur != kEmptyChild) {
    if (cur & kLeafBit) {
      leaf_step<K, kCount>(bvh, C, O, w, cur, t_last, j_last, kt, kj, count, cnt);
      cur = pop(stack, stride, sp);
    } else {
      if (kCount) ++cnt.nodes;
      const float tmax = count == K ? kt[K - 1] : __int_as_float(0x7f800000);
      uint32_t next;
      const bool ok = kBvh8 ? node_step8(bvh, cur, O, inv, t_last, tmax, stack, stride, sp, next)
                            : node_step(bvh, cur, O, inv, t_last, tmax, stack, stride, sp, next);
      if (!ok) return count;
      if (kCount && (uint32_t)sp > cnt.max_stack) cnt.max_stack = (uint32_t)sp;
      cur = next != kEmptyChild ? next : pop(stack, stride, sp);
    }
  }
#endif
  return count;
}

// Blend state of one segment (Eq. 2): raw sums N, D, R, E, P and T.
struct Blend {
  float3 N, R, P;
  float D, E, T;
  uint32_t n_hits;
};

// Traces one segment and calls vis(R, j, h) for every blended hit in order;
// vis returns true to stop.  Returns the hit count handed to the visitor.
template <int K, bool kCount, class Visitor>
__device__ __forceinline__ void trace_segment(const BvhView& bvh, const Consts& C, float3 O, float3 w, float t_lo,
                                              uint32_t* stack, int stride, Visitor& vis, TraceCounters& cnt) {
  if (bvh.n <= 0) return;
  const float big = 1e30f;
  const float3 inv = make_float3(fabsf(w.x) > 1e-30f ? 1.0f / w.x : copysignf(big, w.x),
                                 fabsf(w.y) > 1e-30f ? 1.0f / w.y : copysignf(big, w.y),
                                 fabsf(w.z) > 1e-30f ? 1.0f / w.z : copysignf(big, w.z));
  float t_last = t_lo;
  uint32_t j_last = 0xFFFFFFFFu;
  for (;;) {
    float kt[K];
    uint32_t kj[K];
    if (kCount) ++cnt.rounds;
    const int count = collect_round<K, kCount>(bvh, C, O, w, inv, t_last, j_last, kt, kj, stack, stride, cnt);
    bool stop = false;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if (i < count && !stop) {
        const uint32_t j = kj[i];
        const TraceRec* rp = bvh.trace + j;
        const TraceRec R = load_trace(rp);
        HitGeom h;
        intersect(R, O, w, C, h);  // bit-identical to the collection pass
        if (kCount) ++cnt.blended;
        stop = vis(R, j, h);
      }
    }
    if (stop || count < K) return;
    t_last = kt[K - 1];
    j_last = kj[K - 1];
  }
}

// Resumable form of trace_segment for a loop that refills lanes with new
// rays as soon as theirs finish: the same rounds, split into bounded chunks
// of traversal steps.
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
__device__ __forceinline__ void ray_begin(RayTrace<K>& r, float3 O, float3 w) {
  const float big = 1e30f;
  r.O = O;
  r.w = w;
  r.inv = make_float3(fabsf(w.x) > 1e-30f ? 1.0f / w.x : copysignf(big, w.x),
                      fabsf(w.y) > 1e-30f ? 1.0f / w.y : copysignf(big, w.y),
                      fabsf(w.z) > 1e-30f ? 1.0f / w.z : copysignf(big, w.z));
  r.t_last = 0.f;
  r.j_last = 0xFFFFFFFFu;
}

template <int K>
__device__ __forceinline__ void round_begin(RayTrace<K>& r, const BvhView& bvh) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    r.kt[i] = __int_as_float(0x7f800000);
    r.kj[i] = 0xFFFFFFFFu;
  }
  r.count = 0;
  r.sp = 0;
  r.cur = bvh.n > 0 ? bvh.root : kEmptyChild;
}

// At most `steps` node or leaf steps of the current round; true once the
// round's walk is complete.  A stack overflow (recorded as a device error)
// ends the walk.
template <int K, bool kCount>
__device__ __forceinline__ bool round_steps(RayTrace<K>& r, const BvhView& bvh, const Consts& C, uint32_t* stack,
                                            int stride, int steps, TraceCounters& cnt) {
  for (int s = 0; s < steps && r.cur != kEmptyChild; ++s) {
    if (r.cur & kLeafBit) {
      leaf_step<K, kCount>(bvh, C, r.O, r.w, r.cur, r.t_last, r.j_last, r.kt, r.kj, r.count, cnt);
      r.cur = pop(stack, stride, r.sp);
    } else {
      if (kCount) ++cnt.nodes;
      const float tmax = r.count == K ? r.kt[K - 1] : __int_as_float(0x7f800000);
      uint32_t next;
      const bool ok = kBvh8 ? node_step8(bvh, r.cur, r.O, r.inv, r.t_last, tmax, stack, stride, r.sp, next)
                            : node_step(bvh, r.cur, r.O, r.inv, r.t_last, tmax, stack, stride, r.sp, next);
      if (!ok) {
        r.cur = kEmptyChild;
        break;
      }
      if (kCount && (uint32_t)r.sp > cnt.max_stack) cnt.max_stack = (uint32_t)r.sp;
      r.cur = next != kEmptyChild ? next : pop(stack, stride, r.sp);
    }
  }
  return r.cur == kEmptyChild;
}

// Blends the round's hits in order (as trace_segment does); true when the
// segment is finished, otherwise the next round starts after the last key.
template <int K, bool kCount, class Visitor>
__device__ __forceinline__ bool round_blend(RayTrace<K>& r, const BvhView& bvh, const Consts& C, Visitor& vis,
                                            TraceCounters& cnt) {
  bool stop = false;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    if (i < r.count && !stop) {
      const uint32_t j = r.kj[i];
      const TraceRec* rp = bvh.trace + j;
      const TraceRec R = load_trace(rp);
      HitGeom h;
      intersect(R, r.O, r.w, C, h);
      if (kCount) ++cnt.blended;
      stop = vis(R, j, h);
    }
  }
  if (stop || r.count < K) return true;
  r.t_last = r.kt[K - 1];
  r.j_last = r.kj[K - 1];
  return false;
}

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
