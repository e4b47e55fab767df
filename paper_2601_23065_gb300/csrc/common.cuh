// Device-side layouts and helpers shared by the kernels of the surfel path
// tracer.  Everything here is FP32/uint32 and written for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/eagpt.h"

namespace eagpt {

// ---------------------------------------------------------------------------
// Sizes and encodings
// ---------------------------------------------------------------------------
constexpr int kLeafMax = 1;  // surfels per BVH leaf
constexpr int kStackSize = 48;  // traversal stack entries per ray (shared memory)
constexpr int kMinBlocks = 6;  // resident trace blocks per SM the compiler must allow
constexpr int kBlock = 128;          // threads per block of the trace kernels
constexpr uint32_t kLeafBit = 0x80000000u;
constexpr int kLeafCountShift = 29;  // leaf: bit31 | (count-1) << 29 | start
constexpr uint32_t kLeafStartMask = (1u << kLeafCountShift) - 1u;
constexpr uint32_t kEmptyChild = 0xFFFFFFFFu;  // no child (empty box)
constexpr int64_t kMaxSurfels = (int64_t)kLeafStartMask;  // start must fit

// device error word bits
enum : uint32_t {
  kErrStackOverflow = 1u << 0,
  kErrBadIndex = 1u << 1,
  kErrQueueOverflow = 1u << 2,
};

// ---------------------------------------------------------------------------
// Records (all 16-byte aligned so every load is a 128-bit load)
//
// Trace record, 64 B, in BVH (Morton) order:
//   r0 = (p.x, p.y, p.z, sigma)
//   r1 = (n.x, n.y, n.z, original index as bits)
//   r2 = (a.x, a.y, a.z, 0)     a = t_u / s_u
//   r3 = (b.x, b.y, b.z, 0)     b = t_v / s_v
// Shade record, 32 B, same order:
//   s0 = (rho.r, rho.g, rho.b, e)
//   s1 = (r.r, r.g, r.b, 0)
// BVH4 node, 128 B (one cache line): the boxes of its four children in
// structure-of-arrays form and the four child links
//   lox = (lo.x of children 0..3), loy, loz, hix, hiy, hiz likewise
//   child = (link0..link3): node index, encoded leaf, or kEmptyChild
// ---------------------------------------------------------------------------
struct __align__(16) TraceRec {
  float4 r0, r1, r2, r3;
};
struct __align__(16) ShadeRec {
  float4 s0, s1;
};
struct __align__(128) Node4 {
  float4 lox, loy, loz, hix, hiy, hiz;
  uint4 child;
  uint4 pad;
};

constexpr int kMaxCollapseLevels = 96;  // BVH levels built top-down

// Offsets of the arrays inside the caller's BVH storage buffer (a pure
// function of n, so the host never reads the device to find them).
struct BvhLayout {
  size_t header, trace, shade, nodes, prim_lo, prim_hi, ibox_lo, ibox_hi, leaf_parent, inode_parent,
      sorted_idx, inv_idx, keys0, keys1, vals0, vals1, hist, visit, child_bin, irange, src4, front0, front1,
      levels, em_idx, em_cdf, total;
  int64_t n, n_inodes, n_tiles;
};

// Device header at the start of the BVH storage.
struct BvhHeader {
  uint32_t bounds_bits[6];  // scene centroid bounds, ordered-int encoded
  uint32_t root;            // root node index (0) or encoded leaf
  uint32_t pad0;
  double area_sum;          // sum of node surface areas after the last refit
  double em_total;          // emitter table: sum of the selection weights
  uint32_t em_count;        // emitters with a positive weight
  uint32_t pad[5];
};

constexpr int kSortTileItems = 4096;  // keys per radix-sort tile (256 x 16)

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline BvhLayout bvh_layout(int64_t n) {
  BvhLayout L{};
  L.n = n;
  L.n_inodes = n > 1 ? n - 1 : 1;
  L.n_tiles = (n + kSortTileItems - 1) / kSortTileItems;
  if (L.n_tiles < 1) L.n_tiles = 1;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  size_t nn = (size_t)(n > 0 ? n : 1);
  L.header = take(sizeof(BvhHeader));
  L.trace = take(nn * sizeof(TraceRec));
  L.shade = take(nn * sizeof(ShadeRec));
  L.nodes = take((size_t)L.n_inodes * sizeof(Node4));
  L.prim_lo = take(nn * sizeof(float4));
  L.prim_hi = take(nn * sizeof(float4));
  L.ibox_lo = take((size_t)L.n_inodes * sizeof(float4));
  L.ibox_hi = take((size_t)L.n_inodes * sizeof(float4));
  L.leaf_parent = take(nn * 4);
  L.inode_parent = take((size_t)L.n_inodes * 4);
  L.sorted_idx = take(nn * 4);
  L.inv_idx = take(nn * 4);
  L.keys0 = take(nn * 4);
  L.keys1 = take(nn * 4);
  L.vals0 = take(nn * 4);
  L.vals1 = take(nn * 4);
  L.hist = take((size_t)256 * L.n_tiles * 4);
  L.visit = take((size_t)L.n_inodes * 4);
  L.child_bin = take((size_t)L.n_inodes * 8);
  L.irange = take((size_t)L.n_inodes * 8);
  L.src4 = take((size_t)L.n_inodes * 32);  // per node: the binary code of each of up to 8 children
  L.front0 = take((size_t)L.n_inodes * 8);
  L.front1 = take((size_t)L.n_inodes * 8);
  L.levels = take((size_t)(kMaxCollapseLevels + 2) * 4);
  L.em_idx = take(nn * 4);   // record index of the k-th emitter, in surfel-index order
  L.em_cdf = take(nn * 8);   // running sums of the emitter weights (FP64)
  L.total = o;
  return L;
}

// Device view of a built BVH.
struct BvhView {
  const TraceRec* trace;
  const ShadeRec* shade;
  const Node4* nodes;    // BVH4 nodes
  uint32_t root;  // node index, or an encoded leaf when n <= kLeafMax
  int64_t n;
  const uint32_t* bounds_bits;  // scene centroid bounds (BvhHeader), ordered-int encoded
  const BvhHeader* hdr;         // the header (emitter count and total)
  const uint32_t* em_idx;       // emitter table: record index per emitter
  const double* em_cdf;         // emitter table: running weight sums
};

// Method constants as passed to kernels.
struct Consts {
  float tau_E, T_min, alpha_min, alpha_max, support2, bounce_offset;
  int flags;
};

inline Consts make_consts(const eagpt_params& p) {
  Consts c;
  c.tau_E = p.tau_E;
  c.T_min = p.T_min;
  c.alpha_min = p.alpha_min;
  c.alpha_max = p.alpha_max;
  c.support2 = p.support_sigma * p.support_sigma;
  c.bounce_offset = p.bounce_offset;
  c.flags = p.flags;
  return c;
}

// ---------------------------------------------------------------------------
// device error word (sticky until eagpt_sync_status reads it).  Each
// translation unit has its own copy (no relocatable device code); each
// exports a host reader, see EAGPT_DEFINE_ERROR_READER.
// ---------------------------------------------------------------------------
static __device__ uint32_t g_error_word = 0;

#define EAGPT_DEFINE_ERROR_READER(fn)                                      \
  uint32_t fn() {                                                          \
    uint32_t w = 0;                                                        \
    const uint32_t zero = 0;                                               \
    if (cudaMemcpyFromSymbol(&w, g_error_word, sizeof(w)) != cudaSuccess) \
      return 0xFFFFFFFFu;                                                  \
    cudaMemcpyToSymbol(g_error_word, &zero, sizeof(zero));                 \
    return w;                                                              \
  }

__device__ __forceinline__ void raise_error(uint32_t bits) { atomicOr(&g_error_word, bits); }

// float <-> order-preserving uint32 (bounds kept as atomically updatable ints)
__device__ __forceinline__ uint32_t f2ord(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

__device__ __forceinline__ uint32_t expand_bits10(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds with
// multipliers 0xD2511F53, 0xCD9E8D57 and key increments 0x9E3779B9,
// 0xBB67AE85.  Counter (pixel, sample, bounce, 0), key = 64-bit seed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Uniform in [0, 1) from the top 24 bits: exact in FP32.
__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

__device__ __forceinline__ float4 draws(uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t bounce) {
  const uint4 o = philox4x32_10(make_uint4(pixel, sample, bounce, 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  return make_float4(u24(o.x), u24(o.y), u24(o.z), u24(o.w));
}

// The same stream with counter word 3 = word (word 1: the emitter sample of
// reflection `bounce`).
__device__ __forceinline__ float4 draws_w(uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t bounce,
                                          uint32_t word) {
  const uint4 o = philox4x32_10(make_uint4(pixel, sample, bounce, word),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  return make_float4(u24(o.x), u24(o.y), u24(o.z), u24(o.w));
}

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 mul3(float3 a, float3 b) { return make_float3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Orthonormal basis about unit n (Duff, Burgess, Christensen, Hery, Kensler,
// Liani, Villemin, JCGT 2017) and the cosine-weighted direction of the
// uniforms (u0, u1): radius sqrt(u0), angle 2 pi u1 (pdf cos / pi).
__device__ __forceinline__ float3 cosine_direction(float3 n, float u0, float u1) {
  const float sgn = copysignf(1.0f, n.z);
  const float a = -1.0f / (sgn + n.z);
  const float b = n.x * n.y * a;
  const float3 b1 = make_float3(1.0f + sgn * n.x * n.x * a, sgn * b, -sgn * n.x);
  const float3 b2 = make_float3(b, sgn + n.y * n.y * a, -n.y);
  const float r = sqrtf(u0);
  float s, c;
  sincospif(2.0f * u1, &s, &c);
  const float lz = sqrtf(fmaxf(0.0f, 1.0f - u0));
  return (r * c) * b1 + (r * s) * b2 + lz * n;
}

// Pinhole ray through the centre of pixel (x, y).
__device__ __forceinline__ void camera_ray(const eagpt_camera& cam, uint32_t pixel, float3& O, float3& w) {
  const uint32_t x = pixel % (uint32_t)cam.width, y = pixel / (uint32_t)cam.width;
  const float dx = ((float)x + 0.5f - cam.cx) / cam.fx;
  const float dy = ((float)y + 0.5f - cam.cy) / cam.fy;
  O = make_float3(cam.c2w[3], cam.c2w[7], cam.c2w[11]);
  float3 d = make_float3(cam.c2w[0] * dx + cam.c2w[1] * dy + cam.c2w[2], cam.c2w[4] * dx + cam.c2w[5] * dy + cam.c2w[6],
                         cam.c2w[8] * dx + cam.c2w[9] * dy + cam.c2w[10]);
  const float inv = rsqrtf(dot3(d, d));
  w = inv * d;
}

}  // namespace eagpt
