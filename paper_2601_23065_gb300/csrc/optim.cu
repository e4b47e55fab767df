// Optimisation of the shading parameters against target images: the Stage-1
// albedo recovery of Eq. 7 (single-bounce render, rho only, r fixed) and the
// light baking of Eq. 10 (0-bounce render, r only).  Both losses are
// lambda_c L_c((pred)_PQ, (target)_PQ) with the SMPTE ST 2084 curve (Sec. 3.2).
//
//   k_pq_l1         per element: PQ of both images, |difference| into a
//                   per-block FP64 partial sum, dL/dpred (HBM-bound, 1 pass)
//   k_sum_partials  one block: the partials in a fixed order (deterministic)
//   k_shade_adjoint per pixel: re-trace the primary segment with the forward's
//                   decisions and add w_i g to the gradient of each blended
//                   surfel (w_i = T_{i-1} alpha_i, the blend weight of Eq. 2)
//   k_adam          per parameter: Adam (Kingma and Ba 2015, Algorithm 1),
//                   projection onto [lo, hi], gradient zeroed, and the new
//                   value written to the scene array and to the BVH's copy
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "trace.cuh"

namespace eagpt {

EAGPT_DEFINE_ERROR_READER(take_errors_optim)

namespace {

constexpr int kPqThreads = 256;
constexpr int kPqPerThread = 8;
constexpr int64_t kPqChunk = (int64_t)kPqThreads * kPqPerThread;  // elements per partial sum

// SMPTE ST 2084 inverse EOTF constants (exact binary fractions of the standard)
constexpr float kM1 = 2610.f / 16384.f;
constexpr float kM2 = 2523.f / 4096.f * 128.f;
constexpr float kC1 = 3424.f / 4096.f;
constexpr float kC2 = 2413.f / 4096.f * 32.f;
constexpr float kC3 = 2392.f / 4096.f * 32.f;
constexpr float kYLo = 1e-10f;  // floor of the point the slope is taken at

// PQ of clamp(x / peak, 0, 1) and its slope in x: taken at max(Y, kYLo) below
// the peak (the curve's slope is unbounded at 0), 0 at or above it.
__device__ __forceinline__ float pq(float x, float inv_peak, float& dpq) {
  const float Yr = x * inv_peak;
  const float Y = fminf(fmaxf(Yr, kYLo), 1.f);
  const float y = powf(Y, kM1);
  const float den = 1.f + kC3 * y;
  const float f = (kC1 + kC2 * y) / den;
  const float v = powf(f, kM2);
  // d/dY f^m2 = m2 f^(m2-1) (c2 - c1 c3) / (1 + c3 y)^2 * m1 y / Y
  dpq = Yr < 1.f ? kM2 * (v / f) * (kC2 - kC1 * kC3) / (den * den) * kM1 * (y / Y) * inv_peak : 0.f;
  return Yr > 0.f ? (Yr < kYLo ? powf((kC1 + kC2 * powf(Yr, kM1)) / (1.f + kC3 * powf(Yr, kM1)), kM2) : v)
                  : powf(kC1, kM2);
}

__global__ void __launch_bounds__(kPqThreads) k_pq_l1(const float* __restrict__ pred, const float* __restrict__ target,
                                                      int64_t n, float inv_peak, float scale, float* grad,
                                                      double* partials) {
  __shared__ double s_sum[kPqThreads / 32];
  const int64_t base = blockIdx.x * kPqChunk;
  double acc = 0.0;
#pragma unroll
  for (int r = 0; r < kPqPerThread; ++r) {
    const int64_t k = base + (int64_t)r * kPqThreads + threadIdx.x;  // coalesced
    if (k < n) {
      float dp, dt;
      const float a = pq(pred[k], inv_peak, dp);
      const float b = pq(target[k], inv_peak, dt);
      const float d = a - b;
      acc += (double)fabsf(d);
      if (grad) grad[k] = d > 0.f ? scale * dp : (d < 0.f ? -scale * dp : 0.f);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kPqThreads / 32; ++w) t += s_sum[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) k_sum_partials(const double* __restrict__ partials, int64_t m, double scale,
                                                      double* out) {
  __shared__ double s[256];
  double t = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += 256) t += partials[i];
  s[threadIdx.x] = t;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0] * scale;
}

// Blend weights of the primary segment in the forward's order and with its
// stopping rule; each blended surfel gets w_i g added to its gradient.
struct ShadeAdjointVisitor {
  Consts C;
  float3 g;
  float* grad;
  float T;
  __device__ __forceinline__ bool operator()(const TraceRec& R, uint32_t, const HitGeom& h) {
    const uint32_t id = __float_as_uint(R.r1.w);
    const float wgt = T * h.alpha;
    atomicAdd(&grad[3 * id + 0], wgt * g.x);
    atomicAdd(&grad[3 * id + 1], wgt * g.y);
    atomicAdd(&grad[3 * id + 2], wgt * g.z);
    T *= (1.f - h.alpha);
    return T < C.T_min;
  }
};

__global__ void __launch_bounds__(kBlock, kMinBlocks) k_shade_adjoint(BvhView bvh, Consts C, eagpt_camera cam,
                                                                      const float* __restrict__ dL,
                                                                      const float* __restrict__ li, float* grad,
                                                                      int64_t npix) {
  __shared__ uint32_t s_stack[kStackSize * kBlock];
  const int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x;
  if (i >= npix) return;
  float3 g = make_float3(dL[3 * i], dL[3 * i + 1], dL[3 * i + 2]);
  if (li) g = make_float3(g.x * li[3 * i], g.y * li[3 * i + 1], g.z * li[3 * i + 2]);
  if (g.x == 0.f && g.y == 0.f && g.z == 0.f) return;
  float3 O, w;
  camera_ray(cam, (uint32_t)i, O, w);
  ShadeAdjointVisitor v{C, g, grad, 1.f};
  TraceCounters cnt{0, 0, 0, 0, 0};
  trace_segment<16, false>(bvh, C, O, w, s_stack + threadIdx.x, kBlock, v, cnt);
}

struct AdamArgs {
  float lr, beta1, beta2, eps, lo, hi;
  float inv_bc1, inv_sqrt_bc2;  // 1 / (1 - beta1^t), 1 / sqrt(1 - beta2^t)
};

__global__ void __launch_bounds__(256) k_adam(float* p, float* g, float* m, float* v, int64_t n, AdamArgs a,
                                              int zero_grad, float* mirror, const uint32_t* __restrict__ inv_idx,
                                              int field) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = a.beta1 * m[k] + (1.f - a.beta1) * gk;
  const float vk = a.beta2 * v[k] + (1.f - a.beta2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  float x = p[k] - a.lr * (mk * a.inv_bc1) / (sqrtf(vk) * a.inv_sqrt_bc2 + a.eps);
  x = fminf(fmaxf(x, a.lo), a.hi);
  p[k] = x;
  if (zero_grad) g[k] = 0.f;
  if (mirror) {
    // the BVH's shade record of surfel k / 3: s0.xyz = albedo, s1.xyz = radiance
    const int64_t i = k / 3;
    mirror[8 * (int64_t)inv_idx[i] + field + (int)(k - 3 * i)] = x;
  }
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int64_t pq_partials(int64_t n) { return (n + kPqChunk - 1) / kPqChunk; }

cudaError_t launch_pq_l1(const float* pred, const float* target, int64_t n, float peak, float lambda_c, float* grad,
                         double* out_loss, double* partials, cudaStream_t st) {
  if (n <= 0) {
    if (out_loss) return cudaMemsetAsync(out_loss, 0, sizeof(double), st);
    return cudaSuccess;
  }
  const int64_t m = pq_partials(n);
  const float scale = (float)((double)lambda_c / (double)n);
  EAGPT_LAUNCH(st, "k_pq_l1",
               k_pq_l1<<<(unsigned)m, kPqThreads, 0, st>>>(pred, target, n, 1.f / peak, scale, grad, partials));
  if (out_loss)
    EAGPT_LAUNCH(st, "k_sum_partials",
                 k_sum_partials<<<1, 256, 0, st>>>(partials, m, (double)lambda_c / (double)n, out_loss));
  return cudaGetLastError();
}

cudaError_t launch_shade_adjoint(const BvhView& bvh, const Consts& C, const eagpt_camera& cam, const float* dL,
                                 const float* li, float* grad, cudaStream_t st) {
  const int64_t npix = (int64_t)cam.width * cam.height;
  if (bvh.n <= 0) return cudaSuccess;
  EAGPT_LAUNCH(st, "k_shade_adjoint",
               k_shade_adjoint<<<blocks(npix, kBlock), kBlock, 0, st>>>(bvh, C, cam, dL, li, grad, npix));
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* g, float* m, float* v, int64_t n, const eagpt_adam& cfg, int64_t step,
                        int zero_grad, float* mirror, const uint32_t* inv_idx, int field, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  AdamArgs a;
  a.lr = cfg.lr;
  a.beta1 = cfg.beta1;
  a.beta2 = cfg.beta2;
  a.eps = cfg.eps;
  a.lo = cfg.lo;
  a.hi = cfg.hi;
  a.inv_bc1 = (float)(1.0 / (1.0 - std::pow((double)cfg.beta1, (double)step)));
  a.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(1.0 - std::pow((double)cfg.beta2, (double)step)));
  EAGPT_LAUNCH(st, "k_adam",
               k_adam<<<blocks(n, 256), 256, 0, st>>>(p, g, m, v, n, a, zero_grad, mirror, inv_idx, field));
  return cudaGetLastError();
}

}  // namespace eagpt
