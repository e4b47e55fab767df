// Scene edits (teaser and Sec. 4.3 of the paper: relighting, recolouring,
// moving selected Gaussians; box selection, Appendix D) applied in place on
// the device,
// followed by an update of the affected BVH records and a refit.
//
//   k_select       surfels whose centre lies in a box or a sphere -> ordered
//                  index list (per-block counts, one-block scan, ordered write)
//   k_edit         the edit on each listed surfel
//   k_edit_records trace/shade records and support bounds of the listed
//                  surfels, at their BVH positions
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace eagpt {

EAGPT_DEFINE_ERROR_READER(take_errors_edit)

constexpr int kSelBlock = 256;

__device__ __forceinline__ bool selected(const float* pos, int64_t i, int shape, const float* v) {
  const float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  if (shape == 0) return x >= v[0] && y >= v[1] && z >= v[2] && x <= v[3] && y <= v[4] && z <= v[5];
  const float dx = x - v[0], dy = y - v[1], dz = z - v[2];
  return dx * dx + dy * dy + dz * dz <= v[3] * v[3];
}

struct SelShape {
  int shape;  // 0 box (lo3, hi3), 1 sphere (centre3, radius)
  float v[6];
};

__global__ void __launch_bounds__(kSelBlock) k_select_count(const float* __restrict__ pos, int64_t n, SelShape s,
                                                            uint32_t* block_counts) {
  __shared__ uint32_t warp_tot[kSelBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kSelBlock + threadIdx.x;
  const bool in = i < n && selected(pos, i, s.shape, s.v);
  const uint32_t b = __ballot_sync(0xffffffffu, in);
  if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kSelBlock / 32; ++w) t += warp_tot[w];
    block_counts[blockIdx.x] = t;
  }
}

// exclusive scan of the block counts (one block); total -> *count
__global__ void __launch_bounds__(1024) k_select_scan(uint32_t* block_counts, int64_t nb, int64_t* count) {
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
  if (threadIdx.x == 1023) *count = (int64_t)part[1023];
}

__global__ void __launch_bounds__(kSelBlock) k_select_write(const float* __restrict__ pos, int64_t n, SelShape s,
                                                            const uint32_t* __restrict__ block_offsets,
                                                            int32_t* out, int64_t capacity) {
  __shared__ uint32_t warp_off[kSelBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kSelBlock + threadIdx.x;
  const bool in = i < n && selected(pos, i, s.shape, s.v);
  const uint32_t b = __ballot_sync(0xffffffffu, in);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_off[warp] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < kSelBlock / 32; ++w) {
      const uint32_t c = warp_off[w];
      warp_off[w] = run;
      run += c;
    }
  }
  __syncthreads();
  if (in) {
    const int64_t at = (int64_t)block_offsets[blockIdx.x] + warp_off[warp] + __popc(b & ((1u << lane) - 1u));
    if (at < capacity) out[at] = (int32_t)i;
  }
}

// --------------------------------------------------------------------------
struct EditArgs {
  int op;
  int64_t count;
  const int32_t* idx;
  const float* per_index;
  float v[16];
};

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.f), 1.f); }

__global__ void k_edit(eagpt_scene_mut sc, EditArgs a) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= a.count) return;
  const int32_t i = a.idx[k];
  if (i < 0 || i >= sc.n) {
    raise_error(kErrBadIndex);
    return;
  }
  switch (a.op) {
    case EAGPT_EDIT_SET_EMISSION: {
      // per_index: (e, r, g, b) per listed surfel, or the constants v[0..3]
      const float* src = a.per_index ? a.per_index + 4 * k : a.v;
      sc.emissive[i] = src[0];
      sc.radiance[3 * (int64_t)i] = src[1];
      sc.radiance[3 * (int64_t)i + 1] = src[2];
      sc.radiance[3 * (int64_t)i + 2] = src[3];
      break;
    }
    case EAGPT_EDIT_TOGGLE_EMISSION: {
      // e <- 1 - e; a surfel that becomes an emitter takes the radiance given
      // per index (3 values), one that stops being one keeps its radiance as
      // a cache (ignored by path tracing)
      const float e = 1.f - sc.emissive[i];
      sc.emissive[i] = e;
      if (e > 0.5f && a.per_index) {
        sc.radiance[3 * (int64_t)i] = a.per_index[3 * k];
        sc.radiance[3 * (int64_t)i + 1] = a.per_index[3 * k + 1];
        sc.radiance[3 * (int64_t)i + 2] = a.per_index[3 * k + 2];
      }
      break;
    }
    case EAGPT_EDIT_SCALE_ALBEDO: {
      for (int c = 0; c < 3; ++c) {
        float* r = sc.albedo + 3 * (int64_t)i + c;
        *r = clamp01(*r * a.v[c]);
      }
      break;
    }
    case EAGPT_EDIT_TRANSLATE: {
      for (int c = 0; c < 3; ++c) sc.pos[3 * (int64_t)i + c] += a.v[c];
      break;
    }
    case EAGPT_EDIT_RIGID: {
      // v = (qw, qx, qy, qz, cx, cy, cz, tx, ty, tz): p <- R (p - c) + c + t,
      // q <- q_R q (Hamilton product), with q_R normalised
      float qw = a.v[0], qx = a.v[1], qy = a.v[2], qz = a.v[3];
      const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
      qw *= inv;
      qx *= inv;
      qy *= inv;
      qz *= inv;
      float* p = sc.pos + 3 * (int64_t)i;
      const float dx = p[0] - a.v[4], dy = p[1] - a.v[5], dz = p[2] - a.v[6];
      const float r00 = 1.f - 2.f * (qy * qy + qz * qz), r01 = 2.f * (qx * qy - qw * qz), r02 = 2.f * (qx * qz + qw * qy);
      const float r10 = 2.f * (qx * qy + qw * qz), r11 = 1.f - 2.f * (qx * qx + qz * qz), r12 = 2.f * (qy * qz - qw * qx);
      const float r20 = 2.f * (qx * qz - qw * qy), r21 = 2.f * (qy * qz + qw * qx), r22 = 1.f - 2.f * (qx * qx + qy * qy);
      p[0] = r00 * dx + r01 * dy + r02 * dz + a.v[4] + a.v[7];
      p[1] = r10 * dx + r11 * dy + r12 * dz + a.v[5] + a.v[8];
      p[2] = r20 * dx + r21 * dy + r22 * dz + a.v[6] + a.v[9];
      float* q = sc.quat + 4 * (int64_t)i;
      const float bw = q[0], bx = q[1], by = q[2], bz = q[3];
      q[0] = qw * bw - qx * bx - qy * by - qz * bz;
      q[1] = qw * bx + qx * bw + qy * bz - qz * by;
      q[2] = qw * by - qx * bz + qy * bw + qz * bx;
      q[3] = qw * bz + qx * by - qy * bx + qz * bw;
      break;
    }
    default:
      raise_error(kErrBadIndex);
  }
}

// --------------------------------------------------------------------------
static inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_select(const eagpt_scene& sc, int shape, const float* v, int32_t* out, int64_t capacity,
                          int64_t* out_count, uint32_t* scratch_blocks, cudaStream_t st) {
  SelShape s;
  s.shape = shape;
  for (int k = 0; k < 6; ++k) s.v[k] = v[k];
  const int64_t blocks = (sc.n + kSelBlock - 1) / kSelBlock;
  if (blocks == 0) {
    return cudaMemsetAsync(out_count, 0, sizeof(int64_t), st);
  }
  EAGPT_LAUNCH(st, "k_select_count",
               k_select_count<<<(unsigned)blocks, kSelBlock, 0, st>>>(sc.pos, sc.n, s, scratch_blocks));
  EAGPT_LAUNCH(st, "k_select_scan", k_select_scan<<<1, 1024, 0, st>>>(scratch_blocks, blocks, out_count));
  EAGPT_LAUNCH(st, "k_select_write", k_select_write<<<(unsigned)blocks, kSelBlock, 0, st>>>(
                                         sc.pos, sc.n, s, scratch_blocks, out, capacity));
  return cudaGetLastError();
}

size_t select_scratch_bytes(int64_t n) { return (size_t)((n + kSelBlock - 1) / kSelBlock + 1) * 4; }

cudaError_t launch_edit(const eagpt_scene_mut& sc, const eagpt_edit& e, cudaStream_t st) {
  EditArgs a;
  a.op = e.op;
  a.count = e.count;
  a.idx = e.idx;
  a.per_index = e.per_index;
  for (int k = 0; k < 16; ++k) a.v[k] = e.value[k];
  if (e.count > 0) EAGPT_LAUNCH(st, "k_edit", k_edit<<<nb(e.count, 256), 256, 0, st>>>(sc, a));
  return cudaGetLastError();
}

}  // namespace eagpt

namespace eagpt {

// --------------------------------------------------------------------------
// Deletion: the listed surfels leave the scene and the others keep their
// order.  keep[i] = 0 for listed i; the kept positions are counted per
// block, scanned, and written as an ordered gather map; every field is then
// gathered into a scratch array and copied back over the front of its array.
// --------------------------------------------------------------------------
__global__ void k_del_init(uint32_t* keep, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) keep[i] = 1u;
}

__global__ void k_del_mark(uint32_t* keep, int64_t n, const int32_t* __restrict__ idx, int64_t count) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int32_t i = idx[k];
  if (i < 0 || i >= n) {
    raise_error(kErrBadIndex);  // skipped and reported
    return;
  }
  keep[i] = 0u;
}

__global__ void __launch_bounds__(kSelBlock) k_del_count(const uint32_t* __restrict__ keep, int64_t n,
                                                         uint32_t* block_counts) {
  __shared__ uint32_t warp_tot[kSelBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kSelBlock + threadIdx.x;
  const uint32_t b = __ballot_sync(0xffffffffu, i < n && keep[i]);
  if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kSelBlock / 32; ++w) t += warp_tot[w];
    block_counts[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kSelBlock) k_del_map(const uint32_t* __restrict__ keep, int64_t n,
                                                       const uint32_t* __restrict__ block_offsets, int32_t* map) {
  __shared__ uint32_t warp_off[kSelBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kSelBlock + threadIdx.x;
  const bool in = i < n && keep[i];
  const uint32_t b = __ballot_sync(0xffffffffu, in);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_off[warp] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < kSelBlock / 32; ++w) {
      const uint32_t c = warp_off[w];
      warp_off[w] = run;
      run += c;
    }
  }
  __syncthreads();
  if (in) map[(int64_t)block_offsets[blockIdx.x] + warp_off[warp] + __popc(b & ((1u << lane) - 1u))] = (int32_t)i;
}

__global__ void k_del_gather(const float* __restrict__ src, float* dst, const int32_t* __restrict__ map,
                             int64_t m, int comps) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m * comps) return;
  const int64_t d = t / comps;
  const int c = (int)(t - d * comps);
  dst[t] = src[(int64_t)map[d] * comps + c];
}

size_t delete_scratch_bytes(int64_t n) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const size_t blocks = (nn + kSelBlock - 1) / kSelBlock + 1;
  return align256(nn * 4) + align256(blocks * 4) + align256(nn * 4) + align256(nn * 16) + 256;
}

// Deletes the listed surfels (in place); returns the new count in *out_n
// (synchronises the stream to read it).
cudaError_t launch_delete(const eagpt_scene_mut& sc, const int32_t* idx, int64_t count, void* scratch,
                          int64_t* out_n, cudaStream_t st) {
  const int64_t n = sc.n;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const int64_t blocks = (n + kSelBlock - 1) / kSelBlock;
  char* s = (char*)scratch;
  uint32_t* keep = (uint32_t*)s;
  s += align256(nn * 4);
  uint32_t* bc = (uint32_t*)s;
  s += align256(((nn + kSelBlock - 1) / kSelBlock + 1) * 4);
  int32_t* map = (int32_t*)s;
  s += align256(nn * 4);
  float* tmp = (float*)s;
  s += align256(nn * 16);
  int64_t* dcount = (int64_t*)s;
  if (n == 0) {
    *out_n = 0;
    return cudaSuccess;
  }
  EAGPT_LAUNCH(st, "k_del_init", k_del_init<<<nb(n, 256), 256, 0, st>>>(keep, n));
  if (count > 0) EAGPT_LAUNCH(st, "k_del_mark", k_del_mark<<<nb(count, 256), 256, 0, st>>>(keep, n, idx, count));
  EAGPT_LAUNCH(st, "k_del_count", k_del_count<<<(unsigned)blocks, kSelBlock, 0, st>>>(keep, n, bc));
  EAGPT_LAUNCH(st, "k_select_scan", k_select_scan<<<1, 1024, 0, st>>>(bc, blocks, dcount));
  EAGPT_LAUNCH(st, "k_del_map", k_del_map<<<(unsigned)blocks, kSelBlock, 0, st>>>(keep, n, bc, map));
  int64_t m = 0;
  cudaError_t e = cudaMemcpyAsync(&m, dcount, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  float* fields[7] = {sc.pos, sc.quat, sc.scale, sc.opacity, sc.albedo, sc.radiance, sc.emissive};
  const int comps[7] = {3, 4, 2, 1, 3, 3, 1};
  for (int f = 0; f < 7 && m > 0; ++f) {
    EAGPT_LAUNCH(st, "k_del_gather",
                 k_del_gather<<<nb(m * comps[f], 256), 256, 0, st>>>(fields[f], tmp, map, m, comps[f]));
    e = cudaMemcpyAsync(fields[f], tmp, (size_t)m * comps[f] * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  *out_n = m;
  return cudaGetLastError();
}

}  // namespace eagpt
