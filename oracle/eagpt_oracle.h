/* FP64 brute-force oracle for emission-aware 2D Gaussian surfel path tracing.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA path.
 *
 * Every floating-point computation is done in double precision from the FP32
 * scene and camera parameters.  There is no acceleration structure: every
 * segment tests every surfel.  Random numbers come from the oracle's own
 * Philox4x32-10 (Salmon et al., SC'11), keyed by (pixel, sample, bounce).
 */
#ifndef EAGPT_ORACLE_H
#define EAGPT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Scene parameters in double precision (the Python wrapper widens the FP32
 * scene exactly; finite-difference tests perturb these doubles). */
typedef struct {
  int64_t n;
  const double *pos, *quat, *scale, *opacity, *albedo, *radiance, *emissive;
} ora_scene;

typedef struct {
  int32_t width, height;
  double fx, fy, cx, cy;
  double c2w[12]; /* row-major 3x4: [R | centre], OpenCV camera axes */
} ora_camera;

typedef struct {
  double tau_E;          /* emitter threshold, Eq. 4: 0.1                  */
  double T_min;          /* transmittance stop threshold (Eq. 2 "preset")  */
  double alpha_min;      /* smallest blended alpha                          */
  double alpha_max;      /* alpha clamp                                     */
  double support_sigma;  /* Gaussian support radius in sigmas               */
  double bounce_offset;  /* origin offset along the shading normal          */
  int32_t emitters_reflect; /* 1: general rendering equation (test-only)    */
  double fp32_eps;       /* unit roundoff used by the near-boundary flags;
                            0 disables flagging                              */
  double cond_tol;       /* flag a sample (a traced segment) whose estimated
                            FP32 relative error in any channel (any blended
                            value) exceeds cond_tol (ORA_FLAG_COND); 0
                            disables                                         */
  int32_t mis;           /* 1: path tracing with emitter sampling and
                            multiple importance sampling (see ora_render)   */
} ora_params;

/* near-boundary flag bits (a decision the FP32 path may take differently) */
enum {
  ORA_FLAG_SUPPORT = 1u << 0,  /* u^2+v^2 near the support radius          */
  ORA_FLAG_TLO = 1u << 1,      /* t near the segment start                  */
  ORA_FLAG_AMIN = 1u << 2,     /* alpha near alpha_min                      */
  ORA_FLAG_AMAX = 1u << 3,     /* sigma*g near alpha_max                    */
  ORA_FLAG_ORDER = 1u << 4,    /* two blended hits nearly tied in t         */
  ORA_FLAG_TSTOP = 1u << 5,    /* transmittance near T_min at the stop      */
  ORA_FLAG_EMIT = 1u << 6,     /* E near tau_E                              */
  ORA_FLAG_RR = 1u << 7,       /* Russian-roulette draw near the threshold  */
  ORA_FLAG_ONB = 1u << 8,      /* normal z near 0 (basis branch)            */
  ORA_FLAG_GRAZE = 1u << 9,    /* ray nearly parallel to a surfel plane     */
  ORA_FLAG_COND = 1u << 10,    /* sample ill-conditioned in FP32            */
  ORA_FLAG_HEMI = 1u << 11,    /* emitter-sample direction near the tangent
                                  plane of its vertex                       */
};

/* Result of one traced segment (Eq. 2-3). */
typedef struct {
  double N[3], D, R[3], E, P[3], A; /* raw composites; A = 1 - T_n        */
  double Nn[3], Dn;                 /* normalised N/|N| and D/A           */
  int32_t n_hits;                   /* blended hits                       */
  uint32_t flags;
  /* first-order FP32 error estimates (0 when fp32_eps = 0): relative error
   * of R and P, absolute error of E, angle error of N~, length error of D~ */
  double eR, eP, eE, eN, eD;
} ora_segment;

/* Philox4x32-10 of one 128-bit counter under a 64-bit key. */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Orthonormal basis around unit n (Duff et al. 2017) and the cosine-weighted
 * direction for uniforms (u0, u1); writes the world-space direction. */
void ora_cosine_direction(const double n[3], double u0, double u1, double out[3]);

/* Trace one segment from O along unit w, blending hits with t > t_lo.
 * mode 0: radiance cache (r as stored); mode 1: path tracing (r * [e > tau_E]).
 * hit_idx (nullable) receives up to max_hits blended surfel indices in order. */
int ora_trace_segment(const ora_scene* sc, const ora_params* prm, const double O[3],
                      const double w[3], double t_lo, int32_t mode, ora_segment* out,
                      int32_t* hit_idx, int32_t max_hits);

/* Batch of rays (origin 3, direction 3 per ray; direction unit length)
 * traced with t_lo = 0.
 * out_rec: 12 doubles per ray (Nn3, Dn, R3, E, P3, A); out_nhits; out_flags;
 * hit_idx: max_hits int32 per ray (-1 padded).
 * out_dev (nullable): 12 doubles per ray, per record column the largest
 *         change over the two conditioning re-traces (ray perturbed at FP32
 *         rounding scale, every sigma g by +-4 ulps; 0 when prm->fp32_eps or
 *         prm->cond_tol is 0 or the ray hits nothing); +inf on every column
 *         when a re-trace changes the blended surfel list. */
int ora_trace_rays(const ora_scene* sc, const ora_params* prm, const double* rays, int64_t n_rays,
                   int32_t mode, double* out_rec, int32_t* out_nhits, uint32_t* out_flags,
                   int32_t* hit_idx, int32_t max_hits, double* out_dev, int32_t n_threads);

/* Emitter sampling (path tracing with mis = 1): the solid-angle density at
 * origin O of sampling direction w by the emitter-sampling strategy, summed
 * over every emitter surfel whose plane the ray O + t w (t > 0) crosses
 * inside its support, with no occlusion: sum_i q_i g_i(u, v) t^2 / |w . n_i|.
 * Returns the number of emitter surfels crossed (-1 on error). */
int ora_light_pdf(const ora_scene* sc, const ora_params* prm, const double O[3], const double w[3],
                  double* out_pdf);

/* Primary record of listed pixels: 12 doubles per pixel as in ora_trace_rays.
 * mode as in ora_trace_segment. */
int ora_primary(const ora_scene* sc, const ora_camera* cam, const ora_params* prm, int32_t mode,
                const int32_t* pixels, int64_t n_pix, double* out_rec, uint32_t* out_flags,
                int32_t n_threads);

/* Render listed pixels (linear index y*W+x).
 * kind 0: single-bounce radiance-cache estimator (Eq. 6), bounce limit ignored;
 * kind 1: multi-bounce path tracing (Eq. 8) with max_bounces and Russian
 *         roulette from bounce rr_start on.
 * out_rgb: 3 doubles per pixel (mean over spp).
 * out_samples (nullable): spp*3 doubles per pixel, per-sample contributions.
 * out_sample_flags (nullable): spp flags per pixel (OR over the sample's
 *         segments, including the primary segment).
 * out_segments (nullable): segments traced per pixel (primary counted once).
 * out_sample_dev (nullable): spp*3 doubles per pixel, per sample and channel
 *         the largest change of the contribution over the conditioning runs
 *         (every ray and sigma g perturbed at FP32 rounding scale; 0 when
 *         prm->fp32_eps or prm->cond_tol is 0); +inf on every channel when a
 *         run changes a discrete outcome along the path (a blended surfel, a
 *         bounce, a roulette decision). */
int ora_render(const ora_scene* sc, const ora_camera* cam, const ora_params* prm, int32_t kind,
               int32_t spp, int32_t max_bounces, int32_t rr_start, uint64_t seed,
               const int32_t* pixels, int64_t n_pix, double* out_rgb, double* out_samples,
               uint32_t* out_sample_flags, int64_t* out_segments, double* out_sample_dev,
               int32_t n_threads);

/* Path tracing (kind 1, Eq. 8) with a level of detail: the primary segment
 * and the bounce segments k < lod_from trace sc, the bounce segments
 * k >= lod_from (k = 1 is the segment after the first reflection) trace
 * lod_sc (the merged surfels of the level-of-detail reading).  Everything
 * else as in ora_render; emitter sampling (prm->mis) is not supported
 * (returns -1). */
int ora_render_lod(const ora_scene* sc, const ora_scene* lod_sc, int32_t lod_from, const ora_camera* cam,
                   const ora_params* prm, int32_t spp, int32_t max_bounces, int32_t rr_start, uint64_t seed,
                   const int32_t* pixels, int64_t n_pix, double* out_rgb, double* out_samples,
                   uint32_t* out_sample_flags, int64_t* out_segments, double* out_sample_dev,
                   int32_t n_threads);

/* Gradient of L = sum_p sum_c dL_drgb[p][c] * I[p][c] for the single-bounce
 * render of the listed pixels, with respect to every surfel parameter.
 * grad: 16 doubles per surfel, accumulated (+=):
 *   [0..2] centre p, [3..6] quaternion q (raw), [7..8] scales, [9] opacity,
 *   [10..12] albedo, [13..15] radiance.  (The emissive term enters only
 *   through threshold tests, so its derivative is zero almost everywhere.)
 * out_flags (nullable): per pixel OR of sample flags.
 * run: 0 for the gradient; r > 0 for conditioning run r, which evaluates the
 * same gradient with the primary direction, every secondary ray and every
 * sigma g perturbed at FP32 rounding scale (the perturbations of ora_render's
 * conditioning runs): how far an entry moves under them estimates how well
 * an FP32 evaluation can resolve it. */
int ora_single_bounce_grad(const ora_scene* sc, const ora_camera* cam, const ora_params* prm,
                           int32_t spp, uint64_t seed, const int32_t* pixels, int64_t n_pix,
                           const double* dL_drgb, double* grad, uint32_t* out_flags,
                           int32_t n_threads, int32_t run);

/* Gradient of L = sum dL_drgb . I for the 0-bounce (radiance) render, whose
 * pixel value is the primary segment's blended radiance R (the radiant scene
 * of Sec. 3.2; light baking, Eq. 10).  Same layout and accumulation as
 * ora_single_bounce_grad. */
int ora_radiance_grad(const ora_scene* sc, const ora_camera* cam, const ora_params* prm, const int32_t* pixels,
                      int64_t n_pix, const double* dL_drgb, double* grad, uint32_t* out_flags, int32_t n_threads,
                      int32_t run);

#ifdef __cplusplus
}
#endif
#endif
