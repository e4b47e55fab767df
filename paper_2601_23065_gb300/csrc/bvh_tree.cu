// Tree stage of the BVH build, and refits.
//
//   k_hierarchy   binary radix tree over the sorted Morton codes (Karras,
//                 "Maximizing parallelism in the construction of BVHs,
//                 octrees, and k-d trees", HPG 2012); ties between equal codes
//                 are broken by position, so the tree is always complete.
//                 Records children, parents and the surfel range of every
//                 internal node.
//   k_refit       bottom-up boxes of the binary tree (visit counters: the
//                 second child to arrive computes the parent), and the sum of
//                 node surface areas (the refit-quality measure).
//   k_collapse    top-down, one level per launch: every BVH node takes a
//                 binary node and opens its largest-area internal child until
//                 it has four (or eight) children; subtrees of at most kLeafMax surfels
//                 become leaves.  Records, per BVH4 child, the binary node it
//                 stands for, so a refit only has to copy boxes.
//   k_bvh_boxes   copies refit binary boxes into the BVH child slots
//                 (re-quantising them for the 8-wide quantised nodes).
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace eagpt {

EAGPT_DEFINE_ERROR_READER(take_errors_tree)

__device__ __forceinline__ int delta(const uint32_t* __restrict__ keys, int64_t n, int64_t i, int64_t j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t a = keys[i], b = keys[j];
  if (a != b) return __clz(a ^ b);
  return __clzll((unsigned long long)(i ^ j));  // >= 33 for positions < 2^31: ties sort by position
}

// child code: >= 0 binary internal node, < 0 ~surfel position
__global__ void k_hierarchy(const uint32_t* __restrict__ keys, int64_t n, uint32_t* leaf_parent,
                            uint32_t* inode_parent, int32_t* child_bin, int2* irange) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = delta(keys, n, i, i - d);
  int64_t lmax = 2;
  while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
  int64_t l = 0;
  for (int64_t t = lmax / 2; t >= 1; t /= 2)
    if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  const int64_t j = i + l * d;
  const int dnode = delta(keys, n, i, j);
  int64_t s = 0;
  int64_t t = l;
  do {
    t = (t + 1) / 2;
    if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  const int64_t split = i + s * d + (d < 0 ? -1 : 0);
  const int64_t first = i < j ? i : j, last = i < j ? j : i;
  irange[i] = make_int2((int)first, (int)last);
  if (first == split) {
    leaf_parent[split] = (uint32_t)i;
    child_bin[2 * i] = ~(int32_t)split;
  } else {
    inode_parent[split] = (uint32_t)i;
    child_bin[2 * i] = (int32_t)split;
  }
  if (last == split + 1) {
    leaf_parent[split + 1] = (uint32_t)i;
    child_bin[2 * i + 1] = ~(int32_t)(split + 1);
  } else {
    inode_parent[split + 1] = (uint32_t)i;
    child_bin[2 * i + 1] = (int32_t)(split + 1);
  }
  if (i == 0) inode_parent[0] = 0xFFFFFFFFu;
}

__global__ void k_clear_u32(uint32_t* p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0u;
}

__device__ __forceinline__ float box_area(float4 lo, float4 hi) {
  const float dx = fmaxf(hi.x - lo.x, 0.f), dy = fmaxf(hi.y - lo.y, 0.f), dz = fmaxf(hi.z - lo.z, 0.f);
  return 2.f * (dx * dy + dy * dz + dz * dx);
}

__global__ void k_refit(int64_t n, const float4* __restrict__ plo, const float4* __restrict__ phi, float4* ilo,
                        float4* ihi, const uint32_t* __restrict__ leaf_parent,
                        const uint32_t* __restrict__ inode_parent, const int32_t* __restrict__ child_bin,
                        uint32_t* visit, BvhHeader* hdr) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  uint32_t node = leaf_parent[j];
  float area = 0.f;
  while (node != 0xFFFFFFFFu) {
    __threadfence();
    if (atomicAdd(&visit[node], 1u) == 0u) break;  // first arrival: the sibling finishes
    __threadfence();
    const int32_t c0 = child_bin[2 * node], c1 = child_bin[2 * node + 1];
    const float4 lo0 = c0 < 0 ? plo[~c0] : __ldcg(&ilo[c0]);
    const float4 hi0 = c0 < 0 ? phi[~c0] : __ldcg(&ihi[c0]);
    const float4 lo1 = c1 < 0 ? plo[~c1] : __ldcg(&ilo[c1]);
    const float4 hi1 = c1 < 0 ? phi[~c1] : __ldcg(&ihi[c1]);
    const float4 lo = make_float4(fminf(lo0.x, lo1.x), fminf(lo0.y, lo1.y), fminf(lo0.z, lo1.z), 0.f);
    const float4 hi = make_float4(fmaxf(hi0.x, hi1.x), fmaxf(hi0.y, hi1.y), fmaxf(hi0.z, hi1.z), 0.f);
    __stcg(&ilo[node], lo);
    __stcg(&ihi[node], hi);
    area += box_area(lo, hi);
    node = inode_parent[node];
  }
  if (area > 0.f) atomicAdd(&hdr->area_sum, (double)area);
}

struct TreeArrays {
  const float4 *plo, *phi, *ilo, *ihi;
  const int32_t* child_bin;
  const int2* irange;
};

__device__ __forceinline__ int64_t subtree_count(const TreeArrays& T, int32_t code) {
  if (code < 0) return 1;
  const int2 r = T.irange[code];
  return (int64_t)r.y - r.x + 1;
}

__device__ __forceinline__ void code_box(const TreeArrays& T, int32_t code, float4& lo, float4& hi) {
  if (code < 0) {
    lo = T.plo[~code];
    hi = T.phi[~code];
  } else {
    lo = T.ilo[code];
    hi = T.ihi[code];
  }
}

__device__ __forceinline__ void set_child_box(Node4& nd, int k, float4 lo, float4 hi) {
  float* lx = &nd.lox.x;
  float* ly = &nd.loy.x;
  float* lz = &nd.loz.x;
  float* hx = &nd.hix.x;
  float* hy = &nd.hiy.x;
  float* hz = &nd.hiz.x;
  lx[k] = lo.x;
  ly[k] = lo.y;
  lz[k] = lo.z;
  hx[k] = hi.x;
  hy[k] = hi.y;
  hz[k] = hi.z;
}

// Quantises the child boxes of a BVH8 node (see Node8): origin = union lo,
// quantum 2^e per axis with extent / quantum <= 254, lower bounds rounded
// down and upper bounds up, each checked against the exact decode
// origin + q * quantum the traversal uses.
__device__ __forceinline__ Node8 make_node8(const float4* lo, const float4* hi, const uint32_t* link, int nc) {
  float o[3] = {3e38f, 3e38f, 3e38f}, top[3] = {-3e38f, -3e38f, -3e38f};
  for (int k = 0; k < nc; ++k) {
    const float l[3] = {lo[k].x, lo[k].y, lo[k].z}, h[3] = {hi[k].x, hi[k].y, hi[k].z};
    for (int a = 0; a < 3; ++a) {
      o[a] = fminf(o[a], l[a]);
      top[a] = fmaxf(top[a], h[a]);
    }
  }
  uint32_t eb[3];
  float s[3];
  for (int a = 0; a < 3; ++a) {
    int e = -100;
    const float x = (top[a] - o[a]) / 254.0f;
    if (x > 0.f) {
      frexpf(x, &e);  // x <= 2^e
      e = max(-100, min(100, e));
    }
    eb[a] = (uint32_t)(e + 127);
    s[a] = __int_as_float((int)(eb[a] << 23));
  }
  uint32_t qlo[3][2] = {{0, 0}, {0, 0}, {0, 0}}, qhi[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  for (int k = 0; k < nc; ++k) {
    const float l[3] = {lo[k].x, lo[k].y, lo[k].z}, h[3] = {hi[k].x, hi[k].y, hi[k].z};
    for (int a = 0; a < 3; ++a) {
      int ql = (int)floorf((l[a] - o[a]) / s[a]);
      ql = max(0, min(255, ql));
      while (ql > 0 && __fmaf_rn((float)ql, s[a], o[a]) > l[a]) --ql;
      int qh = (int)ceilf((h[a] - o[a]) / s[a]);
      qh = max(0, min(255, qh));
      while (qh < 255 && __fmaf_rn((float)qh, s[a], o[a]) < h[a]) ++qh;
      qlo[a][k >> 2] |= (uint32_t)ql << (8 * (k & 3));
      qhi[a][k >> 2] |= (uint32_t)qh << (8 * (k & 3));
    }
  }
  Node8 n;
  n.u0 = make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]),
                    eb[0] | (eb[1] << 8) | (eb[2] << 16));
  uint32_t L[8];
  for (int k = 0; k < 8; ++k) L[k] = k < nc ? link[k] : kEmptyChild;
  n.u1 = make_uint4(L[0], L[1], L[2], L[3]);
  n.u2 = make_uint4(L[4], L[5], L[6], L[7]);
  n.u3 = make_uint4(qlo[0][0], qlo[0][1], qlo[1][0], qlo[1][1]);
  n.u4 = make_uint4(qlo[2][0], qlo[2][1], qhi[0][0], qhi[0][1]);
  n.u5 = make_uint4(qhi[1][0], qhi[1][1], qhi[2][0], qhi[2][1]);
  return n;
}

// Quantised BVH4 node (see Node4q): the same quantisation as make_node8 for
// four children (origin = union lo, quantum 2^e per axis with extent /
// quantum <= 254, bounds rounded outward and checked against the exact
// decode fma(q, 2^e, origin) the traversal uses).
__device__ __forceinline__ Node4q make_node4q(const float4* lo, const float4* hi, const uint32_t* link, int nc) {
  float o[3] = {3e38f, 3e38f, 3e38f}, top[3] = {-3e38f, -3e38f, -3e38f};
  for (int k = 0; k < nc; ++k) {
    const float l[3] = {lo[k].x, lo[k].y, lo[k].z}, h[3] = {hi[k].x, hi[k].y, hi[k].z};
    for (int a = 0; a < 3; ++a) {
      o[a] = fminf(o[a], l[a]);
      top[a] = fmaxf(top[a], h[a]);
    }
  }
  uint32_t eb[3];
  float s[3];
  for (int a = 0; a < 3; ++a) {
    int e = -100;
    const float x = (top[a] - o[a]) / 254.0f;
    if (x > 0.f) {
      frexpf(x, &e);  // x <= 2^e
      e = max(-100, min(100, e));
    }
    eb[a] = (uint32_t)(e + 127);
    s[a] = __int_as_float((int)(eb[a] << 23));
  }
  uint32_t qlo[3] = {0, 0, 0}, qhi[3] = {0, 0, 0};
  for (int k = 0; k < nc; ++k) {
    const float l[3] = {lo[k].x, lo[k].y, lo[k].z}, h[3] = {hi[k].x, hi[k].y, hi[k].z};
    for (int a = 0; a < 3; ++a) {
      int ql = (int)floorf((l[a] - o[a]) / s[a]);
      ql = max(0, min(255, ql));
      while (ql > 0 && __fmaf_rn((float)ql, s[a], o[a]) > l[a]) --ql;
      int qh = (int)ceilf((h[a] - o[a]) / s[a]);
      qh = max(0, min(255, qh));
      while (qh < 255 && __fmaf_rn((float)qh, s[a], o[a]) < h[a]) ++qh;
      qlo[a] |= (uint32_t)ql << (8 * k);
      qhi[a] |= (uint32_t)qh << (8 * k);
    }
  }
  Node4q n;
  n.u0 = make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]),
                    eb[0] | (eb[1] << 8) | (eb[2] << 16));
  n.u1 = make_uint4(nc > 0 ? link[0] : kEmptyChild, nc > 1 ? link[1] : kEmptyChild, nc > 2 ? link[2] : kEmptyChild,
                    nc > 3 ? link[3] : kEmptyChild);
  n.u2 = make_uint4(qlo[0], qlo[1], qlo[2], 0u);
  n.u3 = make_uint4(qhi[0], qhi[1], qhi[2], 0u);
  return n;
}

// One level of the top-down collapse.// One level of the top-down collapse.  Frontier entries are (binary node,
// BVH node).  levels[lv] holds this level's frontier size, levels[lv + 1]
// collects the next one; levels[kMaxCollapseLevels + 1] counts BVH nodes.
template <int W>
__global__ void k_collapse(TreeArrays T, void* nodes_out, int32_t* src4, const int2* __restrict__ front_in,
                           int2* front_out, uint32_t* levels, int lv, int64_t cap) {
  const uint32_t count = levels[lv];
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < count; f += (int64_t)gridDim.x * blockDim.x) {
    const int2 e = front_in[f];
    int32_t ch[W];
    int nc = 2;
    ch[0] = T.child_bin[2 * e.x];
    ch[1] = T.child_bin[2 * e.x + 1];
    while (nc < W) {
      int best = -1;
      float best_area = -1.f;
      for (int k = 0; k < nc; ++k) {
        if (ch[k] >= 0 && subtree_count(T, ch[k]) > kLeafMax) {
          float4 lo, hi;
          code_box(T, ch[k], lo, hi);
          const float a = box_area(lo, hi);
          if (a > best_area) {
            best_area = a;
            best = k;
          }
        }
      }
      if (best < 0) break;
      const int32_t b = ch[best];
      ch[best] = T.child_bin[2 * b];
      ch[nc++] = T.child_bin[2 * b + 1];
    }
    uint32_t link[W];
    float4 blo[W], bhi[W];
    for (int k = 0; k < W; ++k) {
      link[k] = kEmptyChild;
      src4[8 * (int64_t)e.y + k] = k < nc ? ch[k] : INT32_MIN;
      if (k >= nc) continue;
      code_box(T, ch[k], blo[k], bhi[k]);
      const int64_t cnt = subtree_count(T, ch[k]);
      if (cnt <= kLeafMax) {
        const int64_t first = ch[k] < 0 ? (int64_t)~ch[k] : (int64_t)T.irange[ch[k]].x;
        link[k] = kLeafBit | ((uint32_t)(cnt - 1) << kLeafCountShift) | (uint32_t)first;
      } else {
        const uint32_t id = atomicAdd(&levels[kMaxCollapseLevels + 1], 1u);
        if ((int64_t)id >= cap) {
          raise_error(kErrBadIndex);
          continue;
        }
        const uint32_t slot = atomicAdd(&levels[lv + 1], 1u);
        front_out[slot] = make_int2(ch[k], (int)id);
        link[k] = id;
      }
    }
    if (W == 8) {
      ((Node8*)nodes_out)[e.y] = make_node8(blo, bhi, link, nc);
    } else if (kQ4) {
      ((Node4q*)nodes_out)[e.y] = make_node4q(blo, bhi, link, nc);
    } else {
      Node4 nd;
      nd.lox = nd.loy = nd.loz = make_float4(1e30f, 1e30f, 1e30f, 1e30f);
      nd.hix = nd.hiy = nd.hiz = make_float4(-1e30f, -1e30f, -1e30f, -1e30f);
      for (int k = 0; k < nc && k < 4; ++k) set_child_box(nd, k, blo[k], bhi[k]);
      nd.child = make_uint4(link[0], link[1 % W], link[2 % W], link[3 % W]);
      nd.pad = make_uint4(0u, 0u, 0u, 0u);
      ((Node4*)nodes_out)[e.y] = nd;
    }
  }
}

__global__ void k_collapse_init(uint32_t* levels, int2* front0) {
  const int i = threadIdx.x;
  for (int k = i; k < kMaxCollapseLevels + 2; k += blockDim.x) levels[k] = 0u;
  __syncthreads();
  if (i == 0) {
    levels[0] = 1u;                        // the root's frontier
    levels[kMaxCollapseLevels + 1] = 1u;   // BVH4 node 0 is the root
    front0[0] = make_int2(0, 0);
  }
}

// A frontier left after the last level means the tree was deeper than the
// collapse budget: recorded as a device error.
__global__ void k_collapse_check(const uint32_t* levels) {
  if (threadIdx.x == 0 && levels[kMaxCollapseLevels] != 0u) raise_error(kErrBadIndex);
}

// Refresh the child boxes of every BVH node from the binary boxes (links
// unchanged).
__global__ void k_bvh_boxes(TreeArrays T, void* nodes_out, const int32_t* __restrict__ src4,
                            const uint32_t* __restrict__ levels) {
  const uint32_t count = levels[kMaxCollapseLevels + 1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    if (kBvh8) {
      Node8* nodes = (Node8*)nodes_out;
      const Node8 old = nodes[i];
      const uint32_t link[8] = {old.u1.x, old.u1.y, old.u1.z, old.u1.w, old.u2.x, old.u2.y, old.u2.z, old.u2.w};
      float4 lo[8], hi[8];
      int nc = 0;
      for (int k = 0; k < 8; ++k) {
        const int32_t c = src4[8 * i + k];
        if (c == INT32_MIN) break;
        code_box(T, c, lo[k], hi[k]);
        nc = k + 1;
      }
      nodes[i] = make_node8(lo, hi, link, nc);
    } else if (kQ4) {
      Node4q* nodes = (Node4q*)nodes_out;
      const Node4q old = nodes[i];
      const uint32_t link[4] = {old.u1.x, old.u1.y, old.u1.z, old.u1.w};
      float4 lo[4], hi[4];
      int nc = 0;
      for (int k = 0; k < 4; ++k) {
        const int32_t c = src4[8 * i + k];
        if (c == INT32_MIN) break;
        code_box(T, c, lo[k], hi[k]);
        nc = k + 1;
      }
      nodes[i] = make_node4q(lo, hi, link, nc);
    } else {
      Node4* nodes = (Node4*)nodes_out;
      Node4 nd = nodes[i];
      for (int k = 0; k < 4; ++k) {
        const int32_t c = src4[8 * i + k];
        if (c == INT32_MIN) continue;
        float4 lo, hi;
        code_box(T, c, lo, hi);
        set_child_box(nd, k, lo, hi);
      }
      nodes[i] = nd;
    }
  }
}

// n <= kLeafMax: a single node whose first child is one leaf.
__global__ void k_small_root(int64_t n, const float4* __restrict__ plo, const float4* __restrict__ phi,
                             void* nodes_out, int32_t* src4, uint32_t* levels, BvhHeader* hdr) {
  float4 lo = make_float4(3e38f, 3e38f, 3e38f, 0.f), hi = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
  for (int64_t j = 0; j < n; ++j) {
    lo = make_float4(fminf(lo.x, plo[j].x), fminf(lo.y, plo[j].y), fminf(lo.z, plo[j].z), 0.f);
    hi = make_float4(fmaxf(hi.x, phi[j].x), fmaxf(hi.y, phi[j].y), fmaxf(hi.z, phi[j].z), 0.f);
  }
  const uint32_t leaf = kLeafBit | ((uint32_t)(n - 1) << kLeafCountShift);
  if (kQ4) {
    ((Node4q*)nodes_out)[0] = make_node4q(&lo, &hi, &leaf, 1);
  } else if (kBvh8) {
    ((Node8*)nodes_out)[0] = make_node8(&lo, &hi, &leaf, 1);
  } else {
    Node4 nd;
    nd.lox = nd.loy = nd.loz = make_float4(1e30f, 1e30f, 1e30f, 1e30f);
    nd.hix = nd.hiy = nd.hiz = make_float4(-1e30f, -1e30f, -1e30f, -1e30f);
    set_child_box(nd, 0, lo, hi);
    nd.child = make_uint4(leaf, kEmptyChild, kEmptyChild, kEmptyChild);
    nd.pad = make_uint4(0u, 0u, 0u, 0u);
    ((Node4*)nodes_out)[0] = nd;
  }
  for (int k = 0; k < 8; ++k) src4[k] = INT32_MIN;
  for (int k = 0; k < kMaxCollapseLevels + 2; ++k) levels[k] = 0u;
  levels[kMaxCollapseLevels + 1] = 1u;
  hdr->area_sum = box_area(lo, hi);
}

// --------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

static TreeArrays tree_arrays(char* base, const BvhLayout& L) {
  TreeArrays T;
  T.plo = (const float4*)(base + L.prim_lo);
  T.phi = (const float4*)(base + L.prim_hi);
  T.ilo = (const float4*)(base + L.ibox_lo);
  T.ihi = (const float4*)(base + L.ibox_hi);
  T.child_bin = (const int32_t*)(base + L.child_bin);
  T.irange = (const int2*)(base + L.irange);
  return T;
}

// --------------------------------------------------------------------------
// PLOC hierarchy (Meister and Bittner, "Parallel Locally-Ordered Clustering
// for Bounding Volume Hierarchy Construction", IEEE TVCG 2018).  Clusters
// start as the surfels in Morton order.  Every round each cluster looks at
// the kPlocRadius clusters on either side and picks the one whose union box
// has the least surface area; mutual nearest neighbours merge into a new
// binary node that takes the lower position, and the list is compacted in
// order.  Pairs are ranked by (area, lower position, higher position), a
// total order, so every nearest-neighbour chain ends in a mutual pair and
// each round merges at least the closest pair of the list.  Internal nodes
// are numbered in reverse creation order, so the last merge (the root) is
// node 0; irange holds (0, leaves - 1) per node, which is all the collapse
// reads when every leaf holds one surfel.
// --------------------------------------------------------------------------
#ifndef EAGPT_PLOC
#define EAGPT_PLOC 0
#endif
#ifndef EAGPT_PLOC_RADIUS
#define EAGPT_PLOC_RADIUS 16
#endif
constexpr bool kUsePloc = EAGPT_PLOC != 0 && kLeafMax == 1;
constexpr int kPlocRadius = EAGPT_PLOC_RADIUS;
constexpr int kPlocBlock = 256;
constexpr int kPlocPer = 4;                          // positions per thread in count / scatter
constexpr int kPlocTile = kPlocBlock * kPlocPer;     // positions per tile
constexpr int kPlocMaxRounds = 1 << 14;

struct PlocState {  // in the collapse's level counters (cleared by k_collapse_init afterwards)
  uint32_t m, base, m_next, created;
};

__device__ __forceinline__ void cluster_box(const TreeArrays& T, int32_t c, float4& lo, float4& hi) {
  code_box(T, c, lo, hi);
}

__device__ __forceinline__ float union_half_area(float4 alo, float4 ahi, float4 blo, float4 bhi) {
  const float dx = fmaxf(ahi.x, bhi.x) - fminf(alo.x, blo.x);
  const float dy = fmaxf(ahi.y, bhi.y) - fminf(alo.y, blo.y);
  const float dz = fmaxf(ahi.z, bhi.z) - fminf(alo.z, blo.z);
  return dx * dy + dy * dz + dz * dx;
}

__global__ void k_ploc_init(int32_t* cl, int64_t n, PlocState* ps, uint32_t* inode_parent) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) cl[i] = ~(int32_t)i;
  if (i == 0) {
    ps->m = (uint32_t)n;
    ps->base = 0u;
    ps->m_next = 0u;
    ps->created = 0u;
    inode_parent[0] = 0xFFFFFFFFu;  // node 0 is the root
  }
}

// Tie-break of equal areas: a hash of the pair (lower, higher position), so
// that runs of identical boxes resolve like a random matching instead of a
// chain that merges one pair per round.
__device__ __forceinline__ uint32_t pair_hash(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return h;
}

// Nearest neighbour of every cluster within +-kPlocRadius positions, by
// (area, pair hash, position); the scan runs in increasing position, which
// for pairs that share i is increasing (lower, higher) order.
__global__ void __launch_bounds__(kPlocBlock) k_ploc_nn(TreeArrays T, const int32_t* __restrict__ cl,
                                                        const PlocState* __restrict__ ps, int32_t* nn) {
  __shared__ float4 s_lo[kPlocBlock + 2 * kPlocRadius], s_hi[kPlocBlock + 2 * kPlocRadius];
  const int64_t m = ps->m;
  const int64_t start = (int64_t)blockIdx.x * kPlocBlock;
  if (start >= m) return;  // uniform for the block
  for (int k = threadIdx.x; k < kPlocBlock + 2 * kPlocRadius; k += kPlocBlock) {
    const int64_t p = start - kPlocRadius + k;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    if (p >= 0 && p < m) cluster_box(T, cl[p], lo, hi);
    s_lo[k] = lo;
    s_hi[k] = hi;
  }
  __syncthreads();
  const int64_t i = start + threadIdx.x;
  if (i >= m) return;
  const float4 lo = s_lo[threadIdx.x + kPlocRadius], hi = s_hi[threadIdx.x + kPlocRadius];
  float best = __int_as_float(0x7f800000);
  uint32_t bh = 0xFFFFFFFFu;
  int64_t bj = -1;
#pragma unroll 4
  for (int d = -kPlocRadius; d <= kPlocRadius; ++d) {
    const int64_t j = i + d;
    if (d == 0 || j < 0 || j >= m) continue;
    const float a = union_half_area(lo, hi, s_lo[threadIdx.x + kPlocRadius + d], s_hi[threadIdx.x + kPlocRadius + d]);
    const uint32_t h = d < 0 ? pair_hash((uint32_t)j, (uint32_t)i) : pair_hash((uint32_t)i, (uint32_t)j);
    if (a < best || (a == best && h < bh) || bj < 0) {
      best = a;
      bh = h;
      bj = j;
    }
  }
  nn[i] = (int32_t)bj;
}

__device__ __forceinline__ void ploc_flags(const int32_t* __restrict__ nn, int64_t i, uint32_t& keep, uint32_t& fresh) {
  const int32_t j = nn[i];
  const bool mutual = j >= 0 && nn[j] == (int32_t)i;
  keep = (mutual && j < i) ? 0u : 1u;      // the higher of a merging pair leaves the list
  fresh = (mutual && i < j) ? 1u : 0u;     // the lower becomes the new node
}

// Per tile: how many clusters stay and how many nodes are made.
__global__ void __launch_bounds__(kPlocBlock) k_ploc_count(const int32_t* __restrict__ nn,
                                                           const PlocState* __restrict__ ps, uint32_t* tile_sums) {
  __shared__ uint32_t s_k[kPlocBlock / 32], s_f[kPlocBlock / 32];
  const int64_t m = ps->m;
  const int64_t t0 = (int64_t)blockIdx.x * kPlocTile;
  if (t0 >= m) return;
  uint32_t k = 0, f = 0;
  for (int r = 0; r < kPlocPer; ++r) {
    const int64_t i = t0 + (int64_t)threadIdx.x * kPlocPer + r;
    if (i < m) {
      uint32_t a, b;
      ploc_flags(nn, i, a, b);
      k += a;
      f += b;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    k += __shfl_xor_sync(0xffffffffu, k, o);
    f += __shfl_xor_sync(0xffffffffu, f, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_k[threadIdx.x >> 5] = k;
    s_f[threadIdx.x >> 5] = f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0, b = 0;
    for (int w = 0; w < kPlocBlock / 32; ++w) {
      a += s_k[w];
      b += s_f[w];
    }
    tile_sums[2 * blockIdx.x] = a;
    tile_sums[2 * blockIdx.x + 1] = b;
  }
}

// Exclusive scan of the tile sums (in place), in one block; totals to ps.
__global__ void __launch_bounds__(1024) k_ploc_scan_tiles(uint32_t* tile_sums, PlocState* ps) {
  __shared__ uint32_t s_k[1024], s_f[1024];
  const int64_t m = ps->m;
  const int64_t tiles = (m + kPlocTile - 1) / kPlocTile;
  uint32_t carry_k = 0, carry_f = 0;
  for (int64_t c0 = 0; c0 < tiles; c0 += 1024) {
    const int64_t t = c0 + threadIdx.x;
    const uint32_t vk = t < tiles ? tile_sums[2 * t] : 0u, vf = t < tiles ? tile_sums[2 * t + 1] : 0u;
    s_k[threadIdx.x] = vk;
    s_f[threadIdx.x] = vf;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
      const uint32_t ak = threadIdx.x >= o ? s_k[threadIdx.x - o] : 0u;
      const uint32_t af = threadIdx.x >= o ? s_f[threadIdx.x - o] : 0u;
      __syncthreads();
      s_k[threadIdx.x] += ak;
      s_f[threadIdx.x] += af;
      __syncthreads();
    }
    if (t < tiles) {
      tile_sums[2 * t] = carry_k + s_k[threadIdx.x] - vk;
      tile_sums[2 * t + 1] = carry_f + s_f[threadIdx.x] - vf;
    }
    carry_k += s_k[1023];
    carry_f += s_f[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ps->m_next = carry_k;
    ps->created = carry_f;
  }
}

// Compaction in order plus the new nodes: position i of the tile goes to
// (tile offset + stays before it in the tile); a merging pair's node gets id
// (n - 2) - (nodes made before it).
__global__ void __launch_bounds__(kPlocBlock) k_ploc_scatter(TreeArrays T, const int32_t* __restrict__ cl_in,
                                                             int32_t* cl_out, const int32_t* __restrict__ nn,
                                                             const PlocState* __restrict__ ps,
                                                             const uint32_t* __restrict__ tile_off, int64_t n,
                                                             int32_t* child_bin, uint32_t* leaf_parent,
                                                             uint32_t* inode_parent, int2* irange, float4* ilo,
                                                             float4* ihi) {
  __shared__ uint32_t s_k[kPlocBlock / 32], s_f[kPlocBlock / 32];
  const int64_t m = ps->m;
  const int64_t t0 = (int64_t)blockIdx.x * kPlocTile;
  if (t0 >= m) return;
  uint32_t kf[kPlocPer], ff[kPlocPer];
  uint32_t k = 0, f = 0;
#pragma unroll
  for (int r = 0; r < kPlocPer; ++r) {
    const int64_t i = t0 + (int64_t)threadIdx.x * kPlocPer + r;
    kf[r] = ff[r] = 0u;
    if (i < m) ploc_flags(nn, i, kf[r], ff[r]);
    k += kf[r];
    f += ff[r];
  }
  // exclusive scan over the block (warp scan, then the warp totals)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t ik = k, iff = f;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, ik, o), b = __shfl_up_sync(0xffffffffu, iff, o);
    if (lane >= o) {
      ik += a;
      iff += b;
    }
  }
  if (lane == 31) {
    s_k[warp] = ik;
    s_f[warp] = iff;
  }
  __syncthreads();
  uint32_t wk = 0, wf = 0;
  for (int w = 0; w < warp; ++w) {
    wk += s_k[w];
    wf += s_f[w];
  }
  uint32_t pk = tile_off[2 * blockIdx.x] + wk + ik - k;
  uint32_t pf = tile_off[2 * blockIdx.x + 1] + wf + iff - f;
  const uint32_t base = ps->base;
#pragma unroll
  for (int r = 0; r < kPlocPer; ++r) {
    const int64_t i = t0 + (int64_t)threadIdx.x * kPlocPer + r;
    if (i >= m || !kf[r]) continue;
    const int32_t c = cl_in[i];
    if (ff[r]) {
      const int32_t c1 = cl_in[nn[i]];
      const int32_t id = (int32_t)((n - 2) - (int64_t)(base + pf));
      ++pf;
      child_bin[2 * id] = c;
      child_bin[2 * id + 1] = c1;
      if (c < 0) leaf_parent[~c] = (uint32_t)id; else inode_parent[c] = (uint32_t)id;
      if (c1 < 0) leaf_parent[~c1] = (uint32_t)id; else inode_parent[c1] = (uint32_t)id;
      float4 lo0, hi0, lo1, hi1;
      code_box(T, c, lo0, hi0);
      code_box(T, c1, lo1, hi1);
      ilo[id] = make_float4(fminf(lo0.x, lo1.x), fminf(lo0.y, lo1.y), fminf(lo0.z, lo1.z), 0.f);
      ihi[id] = make_float4(fmaxf(hi0.x, hi1.x), fmaxf(hi0.y, hi1.y), fmaxf(hi0.z, hi1.z), 0.f);
      const int32_t n0 = c < 0 ? 1 : T.irange[c].y + 1, n1 = c1 < 0 ? 1 : T.irange[c1].y + 1;
      irange[id] = make_int2(0, n0 + n1 - 1);
      cl_out[pk++] = id;
    } else {
      cl_out[pk++] = c;
    }
  }
}

__global__ void k_ploc_advance(PlocState* ps) {
  ps->m = ps->m_next;
  ps->base += ps->created;
}

static void launch_binary_refit(char* base, const BvhLayout& L, cudaStream_t st);

// Builds the binary tree by PLOC; synchronises the stream once per round to
// read the cluster count.  Returns false when the round limit is reached.
static cudaError_t launch_ploc(char* base, const BvhLayout& L, cudaStream_t st) {
  const int64_t n = L.n;
  TreeArrays T = tree_arrays(base, L);
  int32_t* cl[2] = {(int32_t*)(base + L.front0), (int32_t*)(base + L.front1)};
  int32_t* nn = (int32_t*)(base + L.keys1);
  uint32_t* tiles = (uint32_t*)(base + L.hist);
  PlocState* ps = (PlocState*)(base + L.levels);
  int32_t* child_bin = (int32_t*)(base + L.child_bin);
  uint32_t* leaf_parent = (uint32_t*)(base + L.leaf_parent);
  uint32_t* inode_parent = (uint32_t*)(base + L.inode_parent);
  int2* irange = (int2*)(base + L.irange);
  float4* ilo = (float4*)(base + L.ibox_lo);
  float4* ihi = (float4*)(base + L.ibox_hi);
  EAGPT_LAUNCH(st, "k_ploc_init", k_ploc_init<<<blocks_for(n, 256), 256, 0, st>>>(cl[0], n, ps, inode_parent));
  int64_t m = n;
  int cur = 0;
  for (int round = 0; m > 1; ++round) {
    if (round >= kPlocMaxRounds) return cudaErrorUnknown;
    EAGPT_LAUNCH(st, "k_ploc_nn", k_ploc_nn<<<blocks_for(m, kPlocBlock), kPlocBlock, 0, st>>>(T, cl[cur], ps, nn));
    const unsigned nt = blocks_for(m, kPlocTile);
    EAGPT_LAUNCH(st, "k_ploc_count", k_ploc_count<<<nt, kPlocBlock, 0, st>>>(nn, ps, tiles));
    EAGPT_LAUNCH(st, "k_ploc_scan_tiles", k_ploc_scan_tiles<<<1, 1024, 0, st>>>(tiles, ps));
    EAGPT_LAUNCH(st, "k_ploc_scatter",
                 k_ploc_scatter<<<nt, kPlocBlock, 0, st>>>(T, cl[cur], cl[cur ^ 1], nn, ps, tiles, n, child_bin,
                                                           leaf_parent, inode_parent, irange, ilo, ihi));
    EAGPT_LAUNCH(st, "k_ploc_advance", k_ploc_advance<<<1, 1, 0, st>>>(ps));
    uint32_t mh = 0;
    cudaError_t e = cudaMemcpyAsync(&mh, &ps->m, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if ((int64_t)mh >= m) return cudaErrorUnknown;  // no progress: impossible by construction
    m = mh;
    cur ^= 1;
  }
  return cudaGetLastError();
}

static void launch_binary_refit(char* base, const BvhLayout& L, cudaStream_t st) {
  BvhHeader* hdr = (BvhHeader*)(base + L.header);
  cudaMemsetAsync(&hdr->area_sum, 0, sizeof(double), st);
  EAGPT_LAUNCH(st, "k_clear_u32",
               k_clear_u32<<<blocks_for(L.n_inodes, 256), 256, 0, st>>>((uint32_t*)(base + L.visit), L.n_inodes));
  EAGPT_LAUNCH(st, "k_refit",
               k_refit<<<blocks_for(L.n, 256), 256, 0, st>>>(
                   L.n, (const float4*)(base + L.prim_lo), (const float4*)(base + L.prim_hi),
                   (float4*)(base + L.ibox_lo), (float4*)(base + L.ibox_hi), (const uint32_t*)(base + L.leaf_parent),
                   (const uint32_t*)(base + L.inode_parent), (const int32_t*)(base + L.child_bin),
                   (uint32_t*)(base + L.visit), hdr));
}

cudaError_t launch_tree(const uint32_t* sorted_keys, char* base, const BvhLayout& L, cudaStream_t st) {
  const int64_t n = L.n;
  BvhHeader* hdr = (BvhHeader*)(base + L.header);
  void* nodes = (void*)(base + L.nodes);
  int32_t* src4 = (int32_t*)(base + L.src4);
  uint32_t* levels = (uint32_t*)(base + L.levels);
  if (n <= kLeafMax) {
    EAGPT_LAUNCH(st, "k_small_root",
                 k_small_root<<<1, 1, 0, st>>>(n, (const float4*)(base + L.prim_lo), (const float4*)(base + L.prim_hi),
                                               nodes, src4, levels, hdr));
    return cudaGetLastError();
  }
  if (kUsePloc) {
    const cudaError_t e = launch_ploc(base, L, st);
    if (e != cudaSuccess) return e;
  } else {
    EAGPT_LAUNCH(st, "k_hierarchy",
                 k_hierarchy<<<blocks_for(n - 1, 256), 256, 0, st>>>(
                     sorted_keys, n, (uint32_t*)(base + L.leaf_parent), (uint32_t*)(base + L.inode_parent),
                     (int32_t*)(base + L.child_bin), (int2*)(base + L.irange)));
  }
  launch_binary_refit(base, L, st);
  int2* fr[2] = {(int2*)(base + L.front0), (int2*)(base + L.front1)};
  EAGPT_LAUNCH(st, "k_collapse_init", k_collapse_init<<<1, 128, 0, st>>>(levels, fr[0]));
  const TreeArrays T = tree_arrays(base, L);
  // the frontier of a level never exceeds the node count; a grid of a few
  // blocks per SM strides over it
  const unsigned grid = (unsigned)(4 * device_sms());
  // levels are launched in groups of 8; after each group the next frontier's
  // size is read back, and the remaining (empty) levels are skipped
  for (int lv = 0; lv < kMaxCollapseLevels; ++lv) {
    EAGPT_LAUNCH(st, "k_collapse",
                 k_collapse<kBvhWidth><<<grid, 256, 0, st>>>(T, nodes, src4, fr[lv & 1], fr[(lv + 1) & 1], levels, lv,
                                                 L.n_inodes));
    if ((lv & 7) == 7 && lv + 1 < kMaxCollapseLevels) {
      uint32_t next = 1;
      cudaError_t e = cudaMemcpyAsync(&next, levels + lv + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return e;
      if (next == 0) break;
    }
  }
  EAGPT_LAUNCH(st, "k_collapse_check", k_collapse_check<<<1, 32, 0, st>>>(levels));
  return cudaGetLastError();
}

int launch_refit(char* base, const BvhLayout& L, cudaStream_t st) {
  if (L.n <= kLeafMax) {
    EAGPT_LAUNCH(st, "k_small_root",
                 k_small_root<<<1, 1, 0, st>>>(L.n, (const float4*)(base + L.prim_lo),
                                               (const float4*)(base + L.prim_hi), (void*)(base + L.nodes),
                                               (int32_t*)(base + L.src4), (uint32_t*)(base + L.levels),
                                               (BvhHeader*)(base + L.header)));
    return 1;
  }
  launch_binary_refit(base, L, st);
  EAGPT_LAUNCH(st, "k_bvh_boxes",
               k_bvh_boxes<<<(unsigned)(4 * device_sms()), 256, 0, st>>>(
                   tree_arrays(base, L), (void*)(base + L.nodes), (const int32_t*)(base + L.src4),
                   (const uint32_t*)(base + L.levels)));
  return 3;
}

}  // namespace eagpt
