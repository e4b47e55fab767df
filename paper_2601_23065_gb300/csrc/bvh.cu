// LBVH over the support bounds of the surfels.
//
//   1. centroid bounds (block reduction + ordered-int atomics)
//   2. 30-bit Morton codes of the centres inside the bounding cube
//   3. stable LSD radix sort of (code, index), 8 bits per pass
//   4. records: per sorted position, the surfel frame from its quaternion,
//      a = t_u/s_u, b = t_v/s_v, the trace and shade records and the bound of
//      its support ellipse
//   5. tree stage (bvh_tree.cu): binary radix tree, bottom-up boxes, collapse
//      into the 4-wide BVH that the renderer traverses
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace eagpt {

EAGPT_DEFINE_ERROR_READER(take_errors_bvh)

__global__ void k_init_header(BvhHeader* hdr) {
  if (threadIdx.x < 3) {
    hdr->bounds_bits[threadIdx.x] = 0xFFFFFFFFu;     // min
    hdr->bounds_bits[3 + threadIdx.x] = 0u;           // max
  }
  if (threadIdx.x == 0) hdr->area_sum = 0.0;
}

__global__ void k_bounds(const float* __restrict__ pos, int64_t n, BvhHeader* hdr) {
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float v = pos[3 * i + k];
      lo[k] = fminf(lo[k], v);
      hi[k] = fmaxf(hi[k], v);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicMin(&hdr->bounds_bits[k], f2ord(lo[k]));
      atomicMax(&hdr->bounds_bits[3 + k], f2ord(hi[k]));
    }
  }
}

__global__ void k_morton(const float* __restrict__ pos, int64_t n, const BvhHeader* hdr, uint32_t* keys,
                         uint32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float lo0 = ord2f(hdr->bounds_bits[0]), lo1 = ord2f(hdr->bounds_bits[1]), lo2 = ord2f(hdr->bounds_bits[2]);
  const float hi0 = ord2f(hdr->bounds_bits[3]), hi1 = ord2f(hdr->bounds_bits[4]), hi2 = ord2f(hdr->bounds_bits[5]);
  const float ext = fmaxf(fmaxf(hi0 - lo0, hi1 - lo1), fmaxf(hi2 - lo2, 1e-20f));
  const float s = 1023.0f / ext;
  const uint32_t x = (uint32_t)fminf(fmaxf((pos[3 * i + 0] - lo0) * s, 0.f), 1023.f);
  const uint32_t y = (uint32_t)fminf(fmaxf((pos[3 * i + 1] - lo1) * s, 0.f), 1023.f);
  const uint32_t z = (uint32_t)fminf(fmaxf((pos[3 * i + 2] - lo2) * s, 0.f), 1023.f);
  keys[i] = (expand_bits10(x) << 2) | (expand_bits10(y) << 1) | expand_bits10(z);
  vals[i] = (uint32_t)i;
}

// --------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits, tiles of kSortTileItems keys
// --------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = kSortTileItems / kSortThreads;  // 16

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                            uint32_t* hist, int64_t n_tiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)kSortTileItems;
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t i = base + k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of the digit-major histogram (256 x n_tiles) in one block.
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* hist, int64_t total) {
  __shared__ uint32_t part[1024];
  const int64_t per = (total + 1023) / 1024;
  const int64_t b = threadIdx.x * per, e = b + per < total ? b + per : total;
  uint32_t s = 0;
  for (int64_t i = b; i < e; ++i) s += hist[i];
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
    const uint32_t v = hist[i];
    hist[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint32_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin, uint32_t* kout,
                                                               uint32_t* vout, int64_t n, int shift,
                                                               const uint32_t* __restrict__ hist, int64_t n_tiles) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t base_d[256];       // global offset of digit d for this tile (running)
  __shared__ uint32_t wcount[W][256];    // per-warp digit counts in this chunk
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  base_d[threadIdx.x] = hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
  const int64_t tile0 = blockIdx.x * (int64_t)kSortTileItems;
  for (int k = 0; k < kSortItems; ++k) {
    for (int w = 0; w < W; ++w) wcount[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = tile0 + k * kSortThreads + threadIdx.x;
    const bool valid = i < n;
    const uint32_t key = valid ? kin[i] : 0u;
    const uint32_t d = valid ? (key >> shift) & 0xFFu : 256u + lane;  // invalid lanes never match
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wcount[warp][d] = __popc(peers);
    __syncthreads();
    // exclusive prefix over warps per digit, in place; thread t owns digit t
    {
      uint32_t run = 0;
      for (int w = 0; w < W; ++w) {
        const uint32_t c = wcount[w][threadIdx.x];
        wcount[w][threadIdx.x] = run;
        run += c;
      }
      __syncthreads();
      if (valid) {
        const uint32_t dst = base_d[d] + wcount[warp][d] + rank;
        kout[dst] = key;
        vout[dst] = vin[i];
      }
      __syncthreads();
      base_d[threadIdx.x] += run;
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// records of the sorted surfels
// --------------------------------------------------------------------------
__global__ void k_records(eagpt_scene sc, Consts C, const uint32_t* __restrict__ order, TraceRec* trace,
                          ShadeRec* shade, float4* plo, float4* phi, uint32_t* inv_idx, int64_t n, int write_inv) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t i = order[j];
  if (write_inv) inv_idx[i] = (uint32_t)j;
  const float* q = sc.quat + 4 * (int64_t)i;
  float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
  const float qi = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  qw *= qi;
  qx *= qi;
  qy *= qi;
  qz *= qi;
  const float3 tu = make_float3(1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy + qw * qz), 2.f * (qx * qz - qw * qy));
  const float3 tv = make_float3(2.f * (qx * qy - qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz + qw * qx));
  const float3 nn = cross3(tu, tv);
  const float su = sc.scale[2 * (int64_t)i], sv = sc.scale[2 * (int64_t)i + 1];
  const float3 p = make_float3(sc.pos[3 * (int64_t)i], sc.pos[3 * (int64_t)i + 1], sc.pos[3 * (int64_t)i + 2]);
  TraceRec R;
  R.r0 = make_float4(p.x, p.y, p.z, sc.opacity[i]);
  R.r1 = make_float4(nn.x, nn.y, nn.z, __uint_as_float(i));
  R.r2 = make_float4(tu.x / su, tu.y / su, tu.z / su, 0.f);
  R.r3 = make_float4(tv.x / sv, tv.y / sv, tv.z / sv, 0.f);
  trace[j] = R;
  ShadeRec S;
  S.s0 = make_float4(sc.albedo[3 * (int64_t)i], sc.albedo[3 * (int64_t)i + 1], sc.albedo[3 * (int64_t)i + 2],
                     sc.emissive[i]);
  S.s1 = make_float4(sc.radiance[3 * (int64_t)i], sc.radiance[3 * (int64_t)i + 1], sc.radiance[3 * (int64_t)i + 2], 0.f);
  shade[j] = S;
  // support ellipse {p + s_u x t_u + s_v y t_v : x^2 + y^2 <= S^2}: half extent
  // along axis k is S sqrt((s_u t_u,k)^2 + (s_v t_v,k)^2); inflated so that
  // FP32 slab tests stay conservative.
  const float S2 = sqrtf(C.support2);
  float h[3];
  const float tuv[2][3] = {{tu.x, tu.y, tu.z}, {tv.x, tv.y, tv.z}};
  const float pc[3] = {p.x, p.y, p.z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float a = su * tuv[0][k], b = sv * tuv[1][k];
    h[k] = S2 * sqrtf(a * a + b * b) * (1.f + 1e-5f) + 1e-5f * fabsf(pc[k]) + 1e-6f;
  }
  plo[j] = make_float4(p.x - h[0], p.y - h[1], p.z - h[2], 0.f);
  phi[j] = make_float4(p.x + h[0], p.y + h[1], p.z + h[2], 0.f);
}

// --------------------------------------------------------------------------
// host driver
// --------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// --------------------------------------------------------------------------
// Emitter table of the emitter-sampling path tracer: the emitters (e > tau_E
// and a positive weight) in surfel-index order with their record indices,
// FP64 running sums of the weights mean(r) sigma s_u s_v (summed by one
// thread in that order, so the sums are exactly those of a sequential FP64
// loop), and in each emitter's shade record (s1.w) the density factor
// q_i / (2 pi (1 - exp(-S^2 / 2)) s_u s_v) of its emitter samples.
// --------------------------------------------------------------------------
constexpr int kEmBlock = 256;

__device__ __forceinline__ double emitter_weight(const eagpt_scene& sc, const Consts& C, int64_t i) {
  if (!(sc.emissive[i] > C.tau_E)) return 0.0;
  double m = __dadd_rn(__dadd_rn((double)sc.radiance[3 * i], (double)sc.radiance[3 * i + 1]),
                       (double)sc.radiance[3 * i + 2]);
  m = __ddiv_rn(m, 3.0);
  return __dmul_rn(__dmul_rn(__dmul_rn(m, (double)sc.opacity[i]), (double)sc.scale[2 * i]),
                   (double)sc.scale[2 * i + 1]);
}

__global__ void __launch_bounds__(kEmBlock) k_em_count(eagpt_scene sc, Consts C, uint32_t* block_counts) {
  __shared__ uint32_t warp_tot[kEmBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kEmBlock + threadIdx.x;
  const uint32_t b = __ballot_sync(0xffffffffu, i < sc.n && emitter_weight(sc, C, i) > 0.0);
  if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kEmBlock / 32; ++w) t += warp_tot[w];
    block_counts[blockIdx.x] = t;
  }
}

// exclusive scan of the block counts in one block of 1024 threads
__global__ void __launch_bounds__(1024) k_em_scan(uint32_t* block_counts, int64_t nb) {
  __shared__ uint32_t part[1024];
  const int64_t per = (nb + 1023) / 1024;
  const int64_t b = threadIdx.x * per, e = b + per < nb ? b + per : nb;
  uint32_t s = 0;
  for (int64_t k = b; k < e; ++k) s += block_counts[k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int64_t k = b; k < e; ++k) {
    const uint32_t v = block_counts[k];
    block_counts[k] = run;
    run += v;
  }
  if (threadIdx.x == 1023) block_counts[nb] = part[1023];  // total
}

__global__ void __launch_bounds__(kEmBlock) k_em_write(eagpt_scene sc, Consts C, const uint32_t* __restrict__ offs,
                                                       const uint32_t* __restrict__ inv_idx, uint32_t* em_idx,
                                                       double* em_w) {
  __shared__ uint32_t warp_off[kEmBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kEmBlock + threadIdx.x;
  const double w = i < sc.n ? emitter_weight(sc, C, i) : 0.0;
  const bool in = w > 0.0;
  const uint32_t b = __ballot_sync(0xffffffffu, in);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_off[warp] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int k = 0; k < kEmBlock / 32; ++k) {
      const uint32_t c = warp_off[k];
      warp_off[k] = run;
      run += c;
    }
  }
  __syncthreads();
  if (in) {
    const uint32_t at = offs[blockIdx.x] + warp_off[warp] + __popc(b & ((1u << lane) - 1u));
    em_idx[at] = inv_idx[i];
    em_w[at] = w;
  }
}

// The running sums (in place) and each emitter's density factor, in one block:
// the weights are staged in shared memory chunk by chunk (coalesced loads) and
// one thread adds them in emitter order, so the sums are exactly those of a
// sequential FP64 loop; the density factors are then written in parallel.
constexpr int kEmChunk = 4096;

__global__ void __launch_bounds__(1024) k_em_finalize(const uint32_t* __restrict__ total_count,
                                                      const uint32_t* __restrict__ em_idx, double* em_cdf,
                                                      const uint32_t* __restrict__ sorted_idx,
                                                      const float* __restrict__ scale, ShadeRec* shade, BvhHeader* hdr,
                                                      double norm) {
  __shared__ double s_w[kEmChunk];
  __shared__ double s_total;
  const uint32_t ne = *total_count;
  if (threadIdx.x == 0) s_total = 0.0;
  // pass 1: the total, in emitter order
  for (uint32_t c0 = 0; c0 < ne; c0 += kEmChunk) {
    const uint32_t m = ne - c0 < (uint32_t)kEmChunk ? ne - c0 : (uint32_t)kEmChunk;
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) s_w[k] = em_cdf[c0 + k];
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = s_total;
      for (uint32_t k = 0; k < m; ++k) t = __dadd_rn(t, s_w[k]);
      s_total = t;
    }
  }
  __syncthreads();
  const double total = s_total;
  // pass 2: running sums (one thread) and density factors (all threads)
  double run = 0.0;
  for (uint32_t c0 = 0; c0 < ne; c0 += kEmChunk) {
    const uint32_t m = ne - c0 < (uint32_t)kEmChunk ? ne - c0 : (uint32_t)kEmChunk;
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) {
      const double w = em_cdf[c0 + k];
      s_w[k] = w;
      const uint32_t j = em_idx[c0 + k];
      const uint32_t i = sorted_idx[j];
      const double c = __ddiv_rn(__ddiv_rn(w, total), __dmul_rn(__dmul_rn(norm, (double)scale[2 * (int64_t)i]),
                                                                 (double)scale[2 * (int64_t)i + 1]));
      shade[j].s1.w = (float)c;
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (uint32_t k = 0; k < m; ++k) {
        run = __dadd_rn(run, s_w[k]);
        s_w[k] = run;
      }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) em_cdf[c0 + k] = s_w[k];
  }
  if (threadIdx.x == 0) {
    hdr->em_total = total;
    hdr->em_count = ne;
  }
}

static cudaError_t launch_emitters(const eagpt_scene& sc, const Consts& C, char* base, const BvhLayout& L,
                                   cudaStream_t st) {
  const int64_t n = sc.n;
  const int64_t nb = (n + kEmBlock - 1) / kEmBlock;
  uint32_t* counts = (uint32_t*)(base + L.hist);  // free after the sort
  EAGPT_LAUNCH(st, "k_em_count", k_em_count<<<(unsigned)nb, kEmBlock, 0, st>>>(sc, C, counts));
  EAGPT_LAUNCH(st, "k_em_scan", k_em_scan<<<1, 1024, 0, st>>>(counts, nb));
  EAGPT_LAUNCH(st, "k_em_write", k_em_write<<<(unsigned)nb, kEmBlock, 0, st>>>(sc, C, counts,
                                                (const uint32_t*)(base + L.inv_idx), (uint32_t*)(base + L.em_idx),
                                                (double*)(base + L.em_cdf)));
  const double S2 = (double)C.support2;
  const double norm = 2.0 * 3.14159265358979323846 * (1.0 - std::exp(-0.5 * S2));
  EAGPT_LAUNCH(st, "k_em_finalize", k_em_finalize<<<1, 1024, 0, st>>>(counts + nb, (const uint32_t*)(base + L.em_idx),
                                                    (double*)(base + L.em_cdf), (const uint32_t*)(base + L.sorted_idx),
                                                    sc.scale, (ShadeRec*)(base + L.shade),
                                                    (BvhHeader*)(base + L.header), norm));
  return cudaGetLastError();
}

cudaError_t launch_build(const eagpt_scene& sc, const Consts& C, char* base, const BvhLayout& L, cudaStream_t st,
                         int* launches) {
  const int64_t n = sc.n;
  BvhHeader* hdr = (BvhHeader*)(base + L.header);
  int nl = 0;
  EAGPT_LAUNCH(st, "k_init_header", k_init_header<<<1, 32, 0, st>>>(hdr));
  ++nl;
  EAGPT_LAUNCH(st, "k_bounds", k_bounds<<<blocks_for(n, 256) < 1024 ? blocks_for(n, 256) : 1024, 256, 0, st>>>(sc.pos, n, hdr));
  ++nl;
  uint32_t *k0 = (uint32_t*)(base + L.keys0), *k1 = (uint32_t*)(base + L.keys1);
  uint32_t *v0 = (uint32_t*)(base + L.vals0), *v1 = (uint32_t*)(base + L.vals1);
  uint32_t* hist = (uint32_t*)(base + L.hist);
  EAGPT_LAUNCH(st, "k_morton", k_morton<<<blocks_for(n, 256), 256, 0, st>>>(sc.pos, n, hdr, k0, v0));
  ++nl;
  for (int shift = 0; shift < 30; shift += 8) {
    EAGPT_LAUNCH(st, "k_sort_hist", k_sort_hist<<<(unsigned)L.n_tiles, kSortThreads, 0, st>>>(k0, n, shift, hist, L.n_tiles));
    EAGPT_LAUNCH(st, "k_sort_scan", k_sort_scan<<<1, 1024, 0, st>>>(hist, 256 * L.n_tiles));
    EAGPT_LAUNCH(st, "k_sort_scatter", k_sort_scatter<<<(unsigned)L.n_tiles, kSortThreads, 0, st>>>(k0, v0, k1, v1, n, shift, hist, L.n_tiles));
    nl += 3;
    uint32_t* t = k0;
    k0 = k1;
    k1 = t;
    t = v0;
    v0 = v1;
    v1 = t;
  }
  // after 4 passes the sorted keys/values are back in keys0/vals0
  uint32_t* sorted_idx = (uint32_t*)(base + L.sorted_idx);
  cudaMemcpyAsync(sorted_idx, v0, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
  TraceRec* trace = (TraceRec*)(base + L.trace);
  ShadeRec* shade = (ShadeRec*)(base + L.shade);
  float4* plo = (float4*)(base + L.prim_lo);
  float4* phi = (float4*)(base + L.prim_hi);
  EAGPT_LAUNCH(st, "k_records", k_records<<<blocks_for(n, 256), 256, 0, st>>>(sc, C, sorted_idx, trace, shade, plo, phi,
                                                (uint32_t*)(base + L.inv_idx), n, 1));
  ++nl;
  cudaError_t e = launch_tree(k0, base, L, st);
  if (e != cudaSuccess) return e;
  e = launch_emitters(sc, C, base, L, st);
  if (e != cudaSuccess) return e;
  if (launches) *launches += nl + 4;
  return cudaGetLastError();
}

cudaError_t launch_records_update(const eagpt_scene& sc, const Consts& C, char* base, const BvhLayout& L,
                                  cudaStream_t st) {
  // recompute every record (O(n), cheap next to a render) in the existing order
  EAGPT_LAUNCH(st, "k_records", k_records<<<blocks_for(L.n, 256), 256, 0, st>>>(sc, C, (const uint32_t*)(base + L.sorted_idx),
                                                  (TraceRec*)(base + L.trace), (ShadeRec*)(base + L.shade),
                                                  (float4*)(base + L.prim_lo), (float4*)(base + L.prim_hi),
                                                  (uint32_t*)(base + L.inv_idx), L.n, 0));
  return launch_emitters(sc, C, base, L, st);
}

cudaError_t launch_emitter_table(const eagpt_scene& sc, const Consts& C, char* base, const BvhLayout& L,
                                 cudaStream_t st) {
  return sc.n > 0 ? launch_emitters(sc, C, base, L, st) : cudaSuccess;
}

}  // namespace eagpt

namespace eagpt {

// Stable LSD radix sort of (key, value) pairs, 8 bits per pass, 4 passes
// (32-bit keys); the sorted pairs end in k0 / v0.  hist holds 256 words per
// tile of kSortTileItems keys.
void launch_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* hist, int64_t n,
                       cudaStream_t st) {
  const int64_t tiles = (n + kSortTileItems - 1) / kSortTileItems;
  if (n <= 0) return;
  for (int shift = 0; shift < 32; shift += 8) {
    EAGPT_LAUNCH(st, "k_sort_hist", k_sort_hist<<<(unsigned)tiles, kSortThreads, 0, st>>>(k0, n, shift, hist, tiles));
    EAGPT_LAUNCH(st, "k_sort_scan", k_sort_scan<<<1, 1024, 0, st>>>(hist, 256 * tiles));
    EAGPT_LAUNCH(st, "k_sort_scatter",
                 k_sort_scatter<<<(unsigned)tiles, kSortThreads, 0, st>>>(k0, v0, k1, v1, n, shift, hist, tiles));
    uint32_t* t = k0;
    k0 = k1;
    k1 = t;
    t = v0;
    v0 = v1;
    v1 = t;
  }
}

}  // namespace eagpt
