// Tree stage of the BVH build, and refits.
//
//   k_hierarchy   binary radix tree over the sorted Morton codes (Karras,
//                 "Maximizing parallelism in the construction of BVHs,
//                 octrees, and k-d trees", HPG 2012); ties between equal codes
//                 are broken by position, so the tree is always complete.
//                 Records children, parents and the surfel range of every
//                 internal node.
//   k_treelets    rebuilds every maximal subtree of at most 256 surfels with
//                 the surface area heuristic (sweep over sorted centres)
//   k_refit       bottom-up boxes of the binary tree (visit counters: the
//                 second child to arrive computes the parent), and the sum of
//                 node surface areas (the refit-quality measure).
//   k_collapse    top-down, one level per launch: every BVH node takes a
//                 binary node and opens its largest-area internal child until
//                 it has four children; single surfels become leaves.
//                 Records, per BVH4 child, the binary node it stands for, so
//                 a refit only has to copy boxes.
//   k_bvh_boxes   copies refit binary boxes into the BVH child slots.
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

__device__ __forceinline__ float box_area(float4 lo, float4 hi) {
  const float dx = fmaxf(hi.x - lo.x, 0.f), dy = fmaxf(hi.y - lo.y, 0.f), dz = fmaxf(hi.z - lo.z, 0.f);
  return 2.f * (dx * dy + dy * dz + dz * dx);
}

// Treelet restructuring.  The radix tree orders surfels along the Morton
// curve of their centres, which at the bottom of the tree groups thin surfels
// of different sizes and orientations by where their centres fall.  Every
// maximal subtree of at most kTreelet surfels is rebuilt top-down with the
// surface area heuristic (SAH) over their boxes: at each node the centres are
// sorted along each axis and every split point is scored by
// area(left) x |left| + area(right) x |right|; the cheapest one is taken.
// The subtree keeps its root and its internal node slots; only child links,
// parents and subtree sizes change, and the records keep their positions, so
// treelets rebuild independently.  A node's surfel range is then read only
// for its size (one surfel per leaf).
//
// A radix-tree subtree rooted at r covers the positions [f, l], and its
// internal nodes are the slots [f, l] except the end of the range that r is
// not (r is f or l): the slots and surfels of a treelet follow from its range.
constexpr int kTreelet = 256;
constexpr int kTreeletWarps = 4;  // one treelet per warp, four warps per block
static_assert(kLeafMax == 1, "restructured nodes keep only the size of their surfel range");
static_assert(kTreelet <= 256, "a treelet's surfels are indexed by bytes");

// Roots of the treelets: internal nodes of 3..kTreelet surfels whose parent
// holds more (or the root), appended to a list.
__global__ void k_treelet_roots(int64_t n, const int2* __restrict__ irange, const uint32_t* __restrict__ inode_parent,
                                uint32_t* roots, uint32_t* count) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n - 1; r += (int64_t)gridDim.x * blockDim.x) {
    const int2 rr = irange[r];
    const int m = rr.y - rr.x + 1;
    if (m < 3 || m > kTreelet) continue;  // two surfels have one topology
    const uint32_t p = inode_parent[r];
    if (p != 0xFFFFFFFFu) {
      const int2 pr = irange[p];
      if (pr.y - pr.x + 1 <= kTreelet) continue;  // not a maximal subtree
    }
    roots[atomicAdd(count, 1u)] = (uint32_t)r;
  }
}

struct Box6 {
  float lx, ly, lz, hx, hy, hz;
};
__device__ __forceinline__ Box6 box_empty() { return {3e38f, 3e38f, 3e38f, -3e38f, -3e38f, -3e38f}; }
__device__ __forceinline__ void box_grow(Box6& b, const Box6& o) {
  b.lx = fminf(b.lx, o.lx);
  b.ly = fminf(b.ly, o.ly);
  b.lz = fminf(b.lz, o.lz);
  b.hx = fmaxf(b.hx, o.hx);
  b.hy = fmaxf(b.hy, o.hy);
  b.hz = fmaxf(b.hz, o.hz);
}
__device__ __forceinline__ Box6 box_shfl_down(const Box6& b, int o) {
  return {__shfl_down_sync(0xffffffffu, b.lx, o), __shfl_down_sync(0xffffffffu, b.ly, o),
          __shfl_down_sync(0xffffffffu, b.lz, o), __shfl_down_sync(0xffffffffu, b.hx, o),
          __shfl_down_sync(0xffffffffu, b.hy, o), __shfl_down_sync(0xffffffffu, b.hz, o)};
}
__device__ __forceinline__ Box6 box_shfl_up(const Box6& b, int o) {
  return {__shfl_up_sync(0xffffffffu, b.lx, o), __shfl_up_sync(0xffffffffu, b.ly, o),
          __shfl_up_sync(0xffffffffu, b.lz, o), __shfl_up_sync(0xffffffffu, b.hx, o),
          __shfl_up_sync(0xffffffffu, b.hy, o), __shfl_up_sync(0xffffffffu, b.hz, o)};
}
__device__ __forceinline__ float box6_area(const Box6& b) {
  return box_area(make_float4(b.lx, b.ly, b.lz, 0.f), make_float4(b.hx, b.hy, b.hz, 0.f));
}

// One warp's working set: box centres and half extents (the heuristic needs
// the areas only approximately), the three centre orders of the pending
// nodes, and the pending nodes themselves.
struct TreeletWork {
  float c[3][kTreelet];
  float e[3][kTreelet];
  float sfx[kTreelet];
  uint8_t ord[3][kTreelet];
  uint8_t tmp[kTreelet];
  uint8_t left[kTreelet];
  uint16_t t_first[kTreelet], t_count[kTreelet];
  int32_t t_id[kTreelet];
  uint8_t t_axis[kTreelet];  // an order that is valid over the node's range (the parent's split axis)
};

__device__ __forceinline__ Box6 item_box(const TreeletWork& W, int v) {
  return {W.c[0][v] - W.e[0][v], W.c[1][v] - W.e[1][v], W.c[2][v] - W.e[2][v],
          W.c[0][v] + W.e[0][v], W.c[1][v] + W.e[1][v], W.c[2][v] + W.e[2][v]};
}

__global__ void __launch_bounds__(32 * kTreeletWarps) k_treelets(const uint32_t* __restrict__ roots,
                                                                 const uint32_t* __restrict__ count,
                                                                 const float4* __restrict__ plo,
                                                                 const float4* __restrict__ phi, int32_t* child_bin,
                                                                 int2* irange, uint32_t* leaf_parent,
                                                                 uint32_t* inode_parent) {
  __shared__ TreeletWork s_work[kTreeletWarps];
  TreeletWork& W = s_work[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t nroots = *count;
  const uint32_t warps = gridDim.x * kTreeletWarps;
  for (uint32_t q = blockIdx.x * kTreeletWarps + (threadIdx.x >> 5); q < nroots; q += warps) {
    const int32_t r = (int32_t)roots[q];
    const int2 rr = irange[r];
    const int f = rr.x, m = rr.y - rr.x + 1;
    if (m < 3 || m > kTreelet || (r != f && r != rr.y)) {
      raise_error(kErrBadIndex);
      continue;
    }
    const int excl = r == f ? rr.y : f;  // the range's slot that is not this subtree's
    for (int i = lane; i < m; i += 32) {
      const float4 lo = plo[f + i], hi = phi[f + i];
      // a NaN centre sorts last (the orders stay permutations)
      const float cx0 = 0.5f * (lo.x + hi.x), cy0 = 0.5f * (lo.y + hi.y), cz0 = 0.5f * (lo.z + hi.z);
      const float cx = cx0 == cx0 ? cx0 : 3e38f, cy = cy0 == cy0 ? cy0 : 3e38f, cz = cz0 == cz0 ? cz0 : 3e38f;
      W.c[0][i] = cx;
      W.c[1][i] = cy;
      W.c[2][i] = cz;
      W.e[0][i] = fmaxf(cx - lo.x, hi.x - cx);
      W.e[1][i] = fmaxf(cy - lo.y, hi.y - cy);
      W.e[2][i] = fmaxf(cz - lo.z, hi.z - cz);
    }
    __syncwarp();
    // each axis's centre order: rank by comparison, ties by index
    for (int a = 0; a < 3; ++a)
      for (int i = lane; i < m; i += 32) {
        const float ci = W.c[a][i];
        int rank = 0;
        for (int j = 0; j < m; ++j) {
          const float cj = W.c[a][j];
          rank += (cj < ci || (cj == ci && j < i)) ? 1 : 0;
        }
        W.ord[a][rank] = (uint8_t)i;
      }
    if (lane == 0) {
      W.t_first[0] = 0;
      W.t_count[0] = (uint16_t)m;
      W.t_id[0] = r;
      W.t_axis[0] = 0;
    }
    __syncwarp();
    int nt = 1, next = f;
    while (nt > 0) {
      --nt;
      const int s = W.t_first[nt], k = W.t_count[nt];
      const int32_t id = W.t_id[nt];
      const int valid_axis = W.t_axis[nt];
      __syncwarp();
      // every split point of every axis: lane L scores the positions of its
      // chunk [L cs, (L + 1) cs), the boxes of the other chunks by warp scans
      const int cs = (k + 31) >> 5;
      const int b0 = min(k, lane * cs), b1 = min(k, b0 + cs);
      float best = __int_as_float(0x7f800000);
      // two surfels have one split, read from the order valid over the range
      // (a node of three or more surfels has all three orders valid)
      int best_axis = valid_axis, best_split = k >> 1;
      for (int a = 0; a < (k > 2 ? 3 : 0); ++a) {
        Box6 agg = box_empty();
        for (int j = b0; j < b1; ++j) box_grow(agg, item_box(W, W.ord[a][s + j]));
        // boxes of the chunks after and before this lane's
        Box6 suf = agg, pre = agg;
        for (int o = 1; o < 32; o <<= 1) {
          const Box6 d = box_shfl_down(suf, o);
          if (lane + o < 32) box_grow(suf, d);
          const Box6 u = box_shfl_up(pre, o);
          if (lane >= o) box_grow(pre, u);
        }
        Box6 after = box_shfl_down(suf, 1), before = box_shfl_up(pre, 1);
        if (lane == 31) after = box_empty();
        if (lane == 0) before = box_empty();
        Box6 run = after;
        for (int j = b1 - 1; j >= b0; --j) {
          box_grow(run, item_box(W, W.ord[a][s + j]));
          W.sfx[j] = box6_area(run);  // the items [j, k)
        }
        run = before;
        float lbest = __int_as_float(0x7f800000);
        int lsplit = k;
        for (int j = b0; j < b1; ++j) {
          if (j >= 1) {
            const float cost = box6_area(run) * (float)j + W.sfx[j] * (float)(k - j);
            if (cost < lbest) {
              lbest = cost;
              lsplit = j;
            }
          }
          box_grow(run, item_box(W, W.ord[a][s + j]));
        }
        // the warp's cheapest split of this axis (ties: the lower position)
        for (int o = 16; o > 0; o >>= 1) {
          const float oc = __shfl_xor_sync(0xffffffffu, lbest, o);
          const int os = __shfl_xor_sync(0xffffffffu, lsplit, o);
          if (oc < lbest || (oc == lbest && os < lsplit)) {
            lbest = oc;
            lsplit = os;
          }
        }
        if (lbest < best) {
          best = lbest;
          best_axis = a;
          best_split = lsplit;
        }
      }
      __syncwarp();
      // the left child's items: the first best_split of the chosen order; the
      // two other orders are partitioned stably (only a child of three or
      // more surfels is split by order again)
      const bool reorder = best_split > 2 || k - best_split > 2;
      if (reorder)
        for (int j = lane; j < k; j += 32) W.left[W.ord[best_axis][s + j]] = (uint8_t)(j < best_split);
      __syncwarp();
      for (int a = 0; a < (reorder ? 3 : 0); ++a) {
        if (a == best_axis) continue;
        int nl = 0, nr = best_split;
        for (int b = 0; b < k; b += 32) {
          const int j = b + lane;
          const bool valid = j < k;
          const uint8_t v = valid ? W.ord[a][s + j] : 0;
          const bool isl = valid && W.left[v];
          const uint32_t ml = __ballot_sync(0xffffffffu, isl);
          const uint32_t mr = __ballot_sync(0xffffffffu, valid && !isl);
          if (isl) W.tmp[nl + __popc(ml & lt)] = v;
          else if (valid) W.tmp[nr + __popc(mr & lt)] = v;
          nl += __popc(ml);
          nr += __popc(mr);
        }
        __syncwarp();
        for (int j = lane; j < k; j += 32) W.ord[a][s + j] = W.tmp[j];
        __syncwarp();
      }
      for (int side = 0; side < 2; ++side) {
        const int cfirst = side == 0 ? s : s + best_split;
        const int ck = side == 0 ? best_split : k - best_split;
        int32_t code;
        if (ck == 1) {
          const int32_t leaf = f + W.ord[best_axis][cfirst];
          code = ~leaf;
          if (lane == 0) leaf_parent[leaf] = (uint32_t)id;
        } else {
          while (next == r || next == excl) ++next;
          const int32_t cid = next++;
          code = cid;
          if (lane == 0) {
            inode_parent[cid] = (uint32_t)id;
            irange[cid] = make_int2(f, f + ck - 1);  // the size is what is read
            W.t_first[nt] = (uint16_t)cfirst;
            W.t_count[nt] = (uint16_t)ck;
            W.t_id[nt] = cid;
            W.t_axis[nt] = (uint8_t)best_axis;
          }
          ++nt;
        }
        if (lane == 0) child_bin[2 * (int64_t)id + side] = code;
      }
      __syncwarp();
    }
    if (next > rr.y + 1) raise_error(kErrBadIndex);  // more slots than the range holds
  }
}

__global__ void k_clear_u32(uint32_t* p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0u;
}


__global__ void k_refit(int64_t n, const float4* __restrict__ plo, const float4* __restrict__ phi, float4* ilo,
                        float4* ihi, const uint32_t* __restrict__ leaf_parent,
                        const uint32_t* __restrict__ inode_parent, const int32_t* __restrict__ child_bin,
                        uint32_t* visit, BvhHeader* hdr) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  uint32_t node = leaf_parent[j];
  float area = 0.f;
  // a path to the root has fewer than n internal nodes: more means the parent
  // links hold a cycle, recorded as a device error rather than followed
  for (int64_t steps = 0; node != 0xFFFFFFFFu; ++steps) {
    if (steps >= n) {
      raise_error(kErrBadIndex);
      break;
    }
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

// One level of the top-down collapse.  Frontier entries are (binary node,
// BVH node).  levels[lv] holds this level's frontier size, levels[lv + 1]
// collects the next one; levels[kMaxCollapseLevels + 1] counts BVH nodes.
__global__ void k_collapse(TreeArrays T, Node4* nodes_out, int32_t* src4, const int2* __restrict__ front_in,
                           int2* front_out, uint32_t* levels, int lv, int64_t cap) {
  const uint32_t count = levels[lv];
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < count; f += (int64_t)gridDim.x * blockDim.x) {
    const int2 e = front_in[f];
    int32_t ch[4];
    int nc = 2;
    ch[0] = T.child_bin[2 * e.x];
    ch[1] = T.child_bin[2 * e.x + 1];
    while (nc < 4) {
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
    uint32_t link[4];
    float4 blo[4], bhi[4];
    for (int k = 0; k < 4; ++k) {
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
    Node4 nd;
    nd.lox = nd.loy = nd.loz = make_float4(1e30f, 1e30f, 1e30f, 1e30f);
    nd.hix = nd.hiy = nd.hiz = make_float4(-1e30f, -1e30f, -1e30f, -1e30f);
    for (int k = 0; k < nc; ++k) set_child_box(nd, k, blo[k], bhi[k]);
    nd.child = make_uint4(link[0], link[1], link[2], link[3]);
    nd.pad = make_uint4(0u, 0u, 0u, 0u);
    nodes_out[e.y] = nd;
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
__global__ void k_bvh_boxes(TreeArrays T, Node4* nodes, const int32_t* __restrict__ src4,
                            const uint32_t* __restrict__ levels) {
  const uint32_t count = levels[kMaxCollapseLevels + 1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
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

// n <= kLeafMax: a single node whose first child is one leaf.
__global__ void k_small_root(int64_t n, const float4* __restrict__ plo, const float4* __restrict__ phi,
                             Node4* nodes_out, int32_t* src4, uint32_t* levels, BvhHeader* hdr) {
  float4 lo = make_float4(3e38f, 3e38f, 3e38f, 0.f), hi = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
  for (int64_t j = 0; j < n; ++j) {
    lo = make_float4(fminf(lo.x, plo[j].x), fminf(lo.y, plo[j].y), fminf(lo.z, plo[j].z), 0.f);
    hi = make_float4(fmaxf(hi.x, phi[j].x), fmaxf(hi.y, phi[j].y), fmaxf(hi.z, phi[j].z), 0.f);
  }
  const uint32_t leaf = kLeafBit | ((uint32_t)(n - 1) << kLeafCountShift);
  Node4 nd;
  nd.lox = nd.loy = nd.loz = make_float4(1e30f, 1e30f, 1e30f, 1e30f);
  nd.hix = nd.hiy = nd.hiz = make_float4(-1e30f, -1e30f, -1e30f, -1e30f);
  set_child_box(nd, 0, lo, hi);
  nd.child = make_uint4(leaf, kEmptyChild, kEmptyChild, kEmptyChild);
  nd.pad = make_uint4(0u, 0u, 0u, 0u);
  nodes_out[0] = nd;
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
  Node4* nodes = (Node4*)(base + L.nodes);
  int32_t* src4 = (int32_t*)(base + L.src4);
  uint32_t* levels = (uint32_t*)(base + L.levels);
  if (n <= kLeafMax) {
    EAGPT_LAUNCH(st, "k_small_root",
                 k_small_root<<<1, 1, 0, st>>>(n, (const float4*)(base + L.prim_lo), (const float4*)(base + L.prim_hi),
                                               nodes, src4, levels, hdr));
    return cudaGetLastError();
  }
  EAGPT_LAUNCH(st, "k_hierarchy",
               k_hierarchy<<<blocks_for(n - 1, 256), 256, 0, st>>>(
                   sorted_keys, n, (uint32_t*)(base + L.leaf_parent), (uint32_t*)(base + L.inode_parent),
                   (int32_t*)(base + L.child_bin), (int2*)(base + L.irange)));
  // treelet roots go to the refit's visit counters (cleared before the refit),
  // their count to the collapse's level counters (cleared before the collapse)
  uint32_t* roots = (uint32_t*)(base + L.visit);
  cudaError_t me = cudaMemsetAsync(levels, 0, sizeof(uint32_t), st);
  if (me != cudaSuccess) return me;
  EAGPT_LAUNCH(st, "k_treelet_roots",
               k_treelet_roots<<<blocks_for(n - 1, 256), 256, 0, st>>>(
                   n, (const int2*)(base + L.irange), (const uint32_t*)(base + L.inode_parent), roots, levels));
  EAGPT_LAUNCH(st, "k_treelets",
               k_treelets<<<(unsigned)(5 * device_sms()), 32 * kTreeletWarps, 0, st>>>(
                   roots, levels, (const float4*)(base + L.prim_lo), (const float4*)(base + L.prim_hi),
                   (int32_t*)(base + L.child_bin), (int2*)(base + L.irange), (uint32_t*)(base + L.leaf_parent),
                   (uint32_t*)(base + L.inode_parent)));
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
                 k_collapse<<<grid, 256, 0, st>>>(T, nodes, src4, fr[lv & 1], fr[(lv + 1) & 1], levels, lv,
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
                                               (const float4*)(base + L.prim_hi), (Node4*)(base + L.nodes),
                                               (int32_t*)(base + L.src4), (uint32_t*)(base + L.levels),
                                               (BvhHeader*)(base + L.header)));
    return 1;
  }
  launch_binary_refit(base, L, st);
  EAGPT_LAUNCH(st, "k_bvh_boxes",
               k_bvh_boxes<<<(unsigned)(4 * device_sms()), 256, 0, st>>>(
                   tree_arrays(base, L), (Node4*)(base + L.nodes), (const int32_t*)(base + L.src4),
                   (const uint32_t*)(base + L.levels)));
  return 3;
}

}  // namespace eagpt
