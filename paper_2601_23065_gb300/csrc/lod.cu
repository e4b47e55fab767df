// Level of detail: merged surfels for the deeper bounces.
//
// The paper names a level-of-detail hierarchy over the reconstruction as the
// way to fewer ray-Gaussian intersections per ray (Sec. 5, conclusion, and
// Appendix D, path tracing: fewer Gaussians, fewer hits, a faster render) and
// gives no algorithm.  The library's reading: surfels are grouped by
// (grid cell of the centre, the coordinate axis the normal is closest to,
// emitter class e > tau_E) and every group becomes one surfel by moment
// matching of its Gaussians; path-traced bounce segments from a chosen bounce
// on trace the merged surfels (render.cu, eagpt_render_path_traced_lod).
//
//   k_lod_keys     63-bit group key per surfel.  The three integer decisions
//                  are taken in FP32 with round-to-nearest intrinsics in a
//                  fixed order, so that any FP32 evaluation in that order
//                  agrees bit for bit
//   sort           stable radix sort of (key, surfel): low word, then high
//                  word (ties keep ascending surfel order)
//   k_lod_heads    group starts per block of sorted positions
//   k_lod_scan     one block: exclusive scan of the block counts, the group
//                  count and the end sentinel
//   k_lod_starts   first sorted position of every group
//   k_lod_merge    one thread per group, two passes over its members:
//                  weights w = sigma s_u s_v; centre, aligned normal and
//                  weighted means; then the union's second moment about the
//                  centre projected on the merged plane, whose principal axes
//                  and variances give t_u, t_v, s_u, s_v; sigma = W/(s_u s_v)
//                  keeps the group's footprint (it may exceed 1; alpha is
//                  still clamped at alpha_max when traced)
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace eagpt {

constexpr int kLodBlock = 256;
constexpr uint32_t kLodCellMax = (1u << 20) - 1u;

struct LodLayout {
  size_t hi, lo, ka, va, kb, vb, hist, blocks, starts, count, total;
  int64_t n_tiles, n_blocks;
};

static inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

static LodLayout lod_layout(int64_t n) {
  LodLayout L{};
  const size_t w = up256((size_t)(n > 0 ? n : 1) * 4);
  L.n_tiles = (n + kSortTileItems - 1) / kSortTileItems;
  L.n_blocks = (n + kLodBlock - 1) / kLodBlock;
  size_t o = 0;
  L.hi = o, o += w;
  L.lo = o, o += w;
  L.ka = o, o += w;
  L.va = o, o += w;
  L.kb = o, o += w;
  L.vb = o, o += w;
  L.hist = o, o += up256((size_t)256 * (L.n_tiles > 0 ? L.n_tiles : 1) * 4);
  L.blocks = o, o += up256((size_t)(L.n_blocks + 1) * 4);
  L.starts = o, o += up256((size_t)(n + 1) * 4);
  L.count = o, o += 256;
  L.total = o;
  return L;
}

// ---------------------------------------------------------------------------
// group keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lod_cell(float p, float o, float inv_h) {
  const float x = floorf(__fmul_rn(__fsub_rn(p, o), inv_h));
  return (uint32_t)fminf(fmaxf(x, 0.f), (float)kLodCellMax);
}

__global__ void k_lod_keys(eagpt_scene sc, float3 origin, float inv_h, float tau_E, uint32_t* hi, uint32_t* lo,
                           uint32_t* ka, uint32_t* va) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= sc.n) return;
  const float* p = sc.pos + 3 * i;
  const float* q = sc.quat + 4 * i;
  const uint64_t cx = lod_cell(p[0], origin.x, inv_h), cy = lod_cell(p[1], origin.y, inv_h),
                 cz = lod_cell(p[2], origin.z, inv_h);
  // direction of the normal up to a positive factor (third rotation column
  // times |q|^2), products and sums rounded in this order
  const float w = q[0], x = q[1], y = q[2], z = q[3];
  const float nx = 2.f * __fadd_rn(__fmul_rn(x, z), __fmul_rn(w, y));
  const float ny = 2.f * __fsub_rn(__fmul_rn(y, z), __fmul_rn(w, x));
  const float nz = __fsub_rn(__fadd_rn(__fmul_rn(w, w), __fmul_rn(z, z)), __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)));
  const float ax = fabsf(nx), ay = fabsf(ny), az = fabsf(nz);
  const uint64_t axis = (ax >= ay && ax >= az) ? 0u : (ay >= az ? 1u : 2u);
  const uint64_t em = sc.emissive[i] > tau_E ? 1u : 0u;
  const uint64_t key = (cx << 43) | (cy << 23) | (cz << 3) | (axis << 1) | em;
  hi[i] = (uint32_t)(key >> 32);
  lo[i] = (uint32_t)key;
  ka[i] = (uint32_t)key;
  va[i] = (uint32_t)i;
}

// high key words in the order of the low-word sort
__global__ void k_lod_gather_hi(const uint32_t* __restrict__ hi, const uint32_t* __restrict__ perm, int64_t n,
                                uint32_t* out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) out[j] = hi[perm[j]];
}

// ---------------------------------------------------------------------------
// group starts
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool lod_head(const uint32_t* hi, const uint32_t* lo, const uint32_t* perm, int64_t j) {
  if (j == 0) return true;
  const uint32_t a = perm[j], b = perm[j - 1];
  return hi[a] != hi[b] || lo[a] != lo[b];
}

__global__ void __launch_bounds__(kLodBlock) k_lod_heads(const uint32_t* __restrict__ hi,
                                                          const uint32_t* __restrict__ lo,
                                                          const uint32_t* __restrict__ perm, int64_t n,
                                                          uint32_t* block_counts) {
  __shared__ uint32_t warp_sum[kLodBlock / 32];
  const int64_t j = blockIdx.x * (int64_t)kLodBlock + threadIdx.x;
  const bool h = j < n && lod_head(hi, lo, perm, j);
  const uint32_t b = __ballot_sync(0xffffffffu, h);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int k = 0; k < kLodBlock / 32; ++k) s += warp_sum[k];
    block_counts[blockIdx.x] = s;
  }
}

// Exclusive scan of nb block counts in one block of 1024 threads; writes the
// group count and starts[count] = n.
__global__ void __launch_bounds__(1024) k_lod_scan(uint32_t* block_counts, int64_t nb, int64_t n, uint32_t* starts,
                                                   int64_t* count) {
  __shared__ uint32_t part[1024];
  const int64_t per = (nb + 1023) / 1024;
  const int64_t b = threadIdx.x * per, e = b + per < nb ? b + per : nb;
  uint32_t s = 0;
  for (int64_t i = b; i < e; ++i) s += block_counts[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int64_t i = b; i < e; ++i) {
    const uint32_t v = block_counts[i];
    block_counts[i] = run;
    run += v;
  }
  if (threadIdx.x == 1023) {
    *count = (int64_t)part[1023];
    starts[part[1023]] = (uint32_t)n;
  }
}

__global__ void __launch_bounds__(kLodBlock) k_lod_starts(const uint32_t* __restrict__ hi,
                                                           const uint32_t* __restrict__ lo,
                                                           const uint32_t* __restrict__ perm, int64_t n,
                                                           const uint32_t* __restrict__ block_offsets,
                                                           uint32_t* starts) {
  __shared__ uint32_t warp_off[kLodBlock / 32];
  const int64_t j = blockIdx.x * (int64_t)kLodBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool h = j < n && lod_head(hi, lo, perm, j);
  const uint32_t b = __ballot_sync(0xffffffffu, h);
  if (lane == 0) warp_off[warp] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int k = 0; k < kLodBlock / 32; ++k) {
      const uint32_t c = warp_off[k];
      warp_off[k] = run;
      run += c;
    }
  }
  __syncthreads();
  if (h) starts[block_offsets[blockIdx.x] + warp_off[warp] + __popc(b & ((1u << lane) - 1u))] = (uint32_t)j;
}

// ---------------------------------------------------------------------------
// merge
// ---------------------------------------------------------------------------
struct Frame {
  float3 tu, tv, n;
};

__device__ __forceinline__ Frame lod_frame(const float* q) {
  const float inv = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
  Frame f;
  f.tu = make_float3(1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y));
  f.tv = make_float3(2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x));
  f.n = make_float3(2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y));
  return f;
}

__device__ __forceinline__ float3 f3(const float* p) { return make_float3(p[0], p[1], p[2]); }
__device__ __forceinline__ float dotf(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 crossf(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 axpy(float a, float3 x, float3 y) {
  return make_float3(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z));
}
__device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

// symmetric 3x3 accumulated as (xx, yy, zz, xy, xz, yz)
struct Sym3 {
  float xx, yy, zz, xy, xz, yz;
};
__device__ __forceinline__ void add_outer(Sym3& m, float a, float3 v) {
  m.xx = fmaf(a * v.x, v.x, m.xx);
  m.yy = fmaf(a * v.y, v.y, m.yy);
  m.zz = fmaf(a * v.z, v.z, m.zz);
  m.xy = fmaf(a * v.x, v.y, m.xy);
  m.xz = fmaf(a * v.x, v.z, m.xz);
  m.yz = fmaf(a * v.y, v.z, m.yz);
}
__device__ __forceinline__ float quad(const Sym3& m, float3 a, float3 b) {
  return a.x * (m.xx * b.x + m.xy * b.y + m.xz * b.z) + a.y * (m.xy * b.x + m.yy * b.y + m.yz * b.z) +
         a.z * (m.xz * b.x + m.yz * b.y + m.zz * b.z);
}

struct LodOut {
  float *pos, *quat, *scale, *opacity, *albedo, *radiance, *emissive;
  unsigned long long* keys;
};

__global__ void k_lod_merge(eagpt_scene sc, const uint32_t* __restrict__ hi, const uint32_t* __restrict__ lo,
                            const uint32_t* __restrict__ perm, const uint32_t* __restrict__ starts,
                            const int64_t* __restrict__ count, LodOut out) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= *count) return;
  const uint32_t j0 = starts[g], j1 = starts[g + 1];
  const uint32_t i0 = perm[j0];
  const int axis = (int)((lo[i0] >> 1) & 3u);
  const float3 pref = f3(sc.pos + 3 * (int64_t)i0);
  // pass 1: weights, centre offset, aligned normal, weighted means (unit
  // weights when every weight is zero)
  float W = 0.f;
  float3 s1 = make_float3(0.f, 0.f, 0.f), ns = s1, rho = s1, rad = s1;
  float em = 0.f;
  bool unit = false;
  for (int pass = 0; pass < 2; ++pass) {
    W = 0.f;
    s1 = ns = rho = rad = make_float3(0.f, 0.f, 0.f);
    em = 0.f;
    for (uint32_t j = j0; j < j1; ++j) {
      const int64_t i = perm[j];
      const float wi = unit ? 1.f : sc.opacity[i] * sc.scale[2 * i] * sc.scale[2 * i + 1];
      const Frame f = lod_frame(sc.quat + 4 * i);
      const float3 d = f3(sc.pos + 3 * i);
      const float3 o = make_float3(d.x - pref.x, d.y - pref.y, d.z - pref.z);
      const float sgn = comp(f.n, axis) < 0.f ? -wi : wi;
      W += wi;
      s1 = axpy(wi, o, s1);
      ns = axpy(sgn, f.n, ns);
      rho = axpy(wi, f3(sc.albedo + 3 * i), rho);
      rad = axpy(wi, f3(sc.radiance + 3 * i), rad);
      em = fmaf(wi, sc.emissive[i], em);
    }
    if (W > 0.f) break;
    unit = true;
  }
  const float invW = 1.f / W;
  const float3 mu = make_float3(s1.x * invW, s1.y * invW, s1.z * invW);
  const float nl = rsqrtf(dotf(ns, ns));
  const float3 n = make_float3(ns.x * nl, ns.y * nl, ns.z * nl);
  // pass 2: second moment about the centre
  Sym3 M{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (uint32_t j = j0; j < j1; ++j) {
    const int64_t i = perm[j];
    const float wi = unit ? 1.f : sc.opacity[i] * sc.scale[2 * i] * sc.scale[2 * i + 1];
    const Frame f = lod_frame(sc.quat + 4 * i);
    const float3 p = f3(sc.pos + 3 * i);
    const float3 d = make_float3((p.x - pref.x) - mu.x, (p.y - pref.y) - mu.y, (p.z - pref.z) - mu.z);
    const float su = sc.scale[2 * i], sv = sc.scale[2 * i + 1];
    add_outer(M, wi, d);
    add_outer(M, wi * su * su, f.tu);
    add_outer(M, wi * sv * sv, f.tv);
  }
  M.xx *= invW, M.yy *= invW, M.zz *= invW, M.xy *= invW, M.xz *= invW, M.yz *= invW;
  // in-plane basis (Duff et al. 2017, "Building an Orthonormal Basis,
  // Revisited") and the 2x2 moment in it
  const float sg = copysignf(1.f, n.z);
  const float a = -1.f / (sg + n.z), b = n.x * n.y * a;
  const float3 e1 = make_float3(1.f + sg * n.x * n.x * a, sg * b, -sg * n.x);
  const float3 e2 = make_float3(b, sg + n.y * n.y * a, -n.y);
  const float m11 = quad(M, e1, e1), m22 = quad(M, e2, e2), m12 = quad(M, e1, e2);
  // principal axis: angle 0.5 atan2(2 m12, m11 - m22)
  const float th = 0.5f * atan2f(2.f * m12, m11 - m22);
  float c, s;
  sincosf(th, &s, &c);
  float3 tu = make_float3(c * e1.x + s * e2.x, c * e1.y + s * e2.y, c * e1.z + s * e2.z);
  const float tl = rsqrtf(dotf(tu, tu));
  tu = make_float3(tu.x * tl, tu.y * tl, tu.z * tl);
  const float3 tv = crossf(n, tu);
  const float su = sqrtf(fmaxf(quad(M, tu, tu), 0.f));
  const float sv = sqrtf(fmaxf(quad(M, tv, tv), 0.f));
  // quaternion of the rotation with columns (tu, tv, n), Shepperd's method
  const float r00 = tu.x, r10 = tu.y, r20 = tu.z, r01 = tv.x, r11 = tv.y, r21 = tv.z, r02 = n.x, r12 = n.y, r22 = n.z;
  const float tr = r00 + r11 + r22;
  float qw, qx, qy, qz;
  if (tr >= r00 && tr >= r11 && tr >= r22) {
    const float h = 2.f * sqrtf(1.f + tr), ih = 1.f / h;
    qw = 0.25f * h, qx = (r21 - r12) * ih, qy = (r02 - r20) * ih, qz = (r10 - r01) * ih;
  } else if (r00 >= r11 && r00 >= r22) {
    const float h = 2.f * sqrtf(1.f + r00 - r11 - r22), ih = 1.f / h;
    qw = (r21 - r12) * ih, qx = 0.25f * h, qy = (r01 + r10) * ih, qz = (r02 + r20) * ih;
  } else if (r11 >= r22) {
    const float h = 2.f * sqrtf(1.f + r11 - r00 - r22), ih = 1.f / h;
    qw = (r02 - r20) * ih, qx = (r01 + r10) * ih, qy = 0.25f * h, qz = (r12 + r21) * ih;
  } else {
    const float h = 2.f * sqrtf(1.f + r22 - r00 - r11), ih = 1.f / h;
    qw = (r10 - r01) * ih, qx = (r02 + r20) * ih, qy = (r12 + r21) * ih, qz = 0.25f * h;
  }
  out.pos[3 * g] = pref.x + mu.x;
  out.pos[3 * g + 1] = pref.y + mu.y;
  out.pos[3 * g + 2] = pref.z + mu.z;
  out.quat[4 * g] = qw;
  out.quat[4 * g + 1] = qx;
  out.quat[4 * g + 2] = qy;
  out.quat[4 * g + 3] = qz;
  out.scale[2 * g] = su;
  out.scale[2 * g + 1] = sv;
  out.opacity[g] = unit ? 0.f : W / (su * sv);
  out.albedo[3 * g] = rho.x * invW;
  out.albedo[3 * g + 1] = rho.y * invW;
  out.albedo[3 * g + 2] = rho.z * invW;
  out.radiance[3 * g] = rad.x * invW;
  out.radiance[3 * g + 1] = rad.y * invW;
  out.radiance[3 * g + 2] = rad.z * invW;
  out.emissive[g] = em * invW;
  if (out.keys) out.keys[g] = ((unsigned long long)hi[i0] << 32) | lo[i0];
}

static inline unsigned lod_blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

size_t lod_workspace_bytes(int64_t n) { return lod_layout(n).total; }

cudaError_t launch_lod(const eagpt_scene& sc, const float origin[3], float inv_h, float tau_E,
                       const eagpt_scene_mut& out, uint64_t* out_keys, void* ws, int64_t* out_count,
                       cudaStream_t st) {
  const int64_t n = sc.n;
  const LodLayout L = lod_layout(n);
  char* base = (char*)ws;
  uint32_t* hi = (uint32_t*)(base + L.hi);
  uint32_t* lo = (uint32_t*)(base + L.lo);
  uint32_t* ka = (uint32_t*)(base + L.ka);
  uint32_t* va = (uint32_t*)(base + L.va);
  uint32_t* kb = (uint32_t*)(base + L.kb);
  uint32_t* vb = (uint32_t*)(base + L.vb);
  uint32_t* hist = (uint32_t*)(base + L.hist);
  uint32_t* blocks = (uint32_t*)(base + L.blocks);
  uint32_t* starts = (uint32_t*)(base + L.starts);
  int64_t* count = (int64_t*)(base + L.count);
  cudaError_t e;
  if (n == 0) {
    *out_count = 0;
    return cudaSuccess;
  }
  EAGPT_LAUNCH(st, "k_lod_keys", k_lod_keys<<<lod_blocks(n, kLodBlock), kLodBlock, 0, st>>>(
                                     sc, make_float3(origin[0], origin[1], origin[2]), inv_h, tau_E, hi, lo, ka, va));
  // low words, then (stable) high words: the pairs end sorted by the full key
  launch_sort_pairs(ka, va, kb, vb, hist, n, st);
  EAGPT_LAUNCH(st, "k_lod_gather_hi",
               k_lod_gather_hi<<<lod_blocks(n, kLodBlock), kLodBlock, 0, st>>>(hi, va, n, kb));
  launch_sort_pairs(kb, va, ka, vb, hist, n, st);
  EAGPT_LAUNCH(st, "k_lod_heads",
               k_lod_heads<<<(unsigned)L.n_blocks, kLodBlock, 0, st>>>(hi, lo, va, n, blocks));
  EAGPT_LAUNCH(st, "k_lod_scan", k_lod_scan<<<1, 1024, 0, st>>>(blocks, L.n_blocks, n, starts, count));
  EAGPT_LAUNCH(st, "k_lod_starts",
               k_lod_starts<<<(unsigned)L.n_blocks, kLodBlock, 0, st>>>(hi, lo, va, n, blocks, starts));
  LodOut o{out.pos, out.quat, out.scale, out.opacity, out.albedo, out.radiance, out.emissive,
           (unsigned long long*)out_keys};
  EAGPT_LAUNCH(st, "k_lod_merge",
               k_lod_merge<<<lod_blocks(n, 128), 128, 0, st>>>(sc, hi, lo, va, starts, count, o));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(out_count, count, sizeof(int64_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

}  // namespace eagpt
