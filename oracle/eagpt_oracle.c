/* FP64 brute-force oracle for emission-aware 2D Gaussian surfel path tracing.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU baseline
 * leg of the benchmark are the only users.  It shares no code with the CUDA
 * path and is deliberately plain: every segment tests every surfel, hits are
 * collected and sorted, then blended front to back exactly as written in the
 * paper (Sec. 3.1, Eq. 1-3), the bounce follows Sec. 3.1 "Light Bouncing",
 * the single-bounce estimator is Eq. 6 and the path tracer is Eq. 8.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes): hits are ordered by (t, surfel index); the blend stops after the
 * hit that takes the transmittance below T_min; Gaussian support is
 * support_sigma standard deviations; alpha = min(sigma*g, alpha_max) and hits
 * with alpha < alpha_min are skipped; the blended normal faces the ray origin;
 * the primary ray goes through the pixel centre and is shared by all samples;
 * the new origin is offset by bounce_offset along the blended normal; the
 * cosine sample uses Duff et al.'s orthonormal basis; Russian roulette (not in
 * the paper) survives with probability min(1, max(beta)); random numbers are
 * Philox4x32-10 with counter (pixel, sample, bounce, 0) and key = seed.
 *
 * Near-boundary flags: every discrete decision records whether its FP64
 * margin is within an estimate of the error an FP32 evaluation could make
 * (scaled by fp32_eps); a flagged sample may legitimately differ.
 */
#include "eagpt_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

#define ERR_C 3.0   /* FP32 roundings assumed per estimated quantity */
#define FLAG_K 4.0  /* slack applied to the estimates at each decision */
/* Conditioning runs per sample: the largest deviation over these runs
 * estimates how far FP32 rounding can move the sample (two runs missed
 * samples that four catch). */
#define ORA_COND_RUNS 4
#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): 10 rounds of the 4x32 S-box with multipliers     */
/* 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.   */
/* ------------------------------------------------------------------------ */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Uniform in [0,1) from the top 24 bits (exactly representable in FP32). */
static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

static void draws_w(uint64_t seed, int64_t pixel, int32_t sample, int32_t bounce, uint32_t word, double u[4]) {
  uint32_t ctr[4] = {(uint32_t)pixel, (uint32_t)sample, (uint32_t)bounce, word};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  ora_philox4x32_10(ctr, key, o);
  for (int i = 0; i < 4; ++i) u[i] = u24(o[i]);
}

static void draws(uint64_t seed, int64_t pixel, int32_t sample, int32_t bounce, double u[4]) {
  uint32_t ctr[4] = {(uint32_t)pixel, (uint32_t)sample, (uint32_t)bounce, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  ora_philox4x32_10(ctr, key, o);
  for (int i = 0; i < 4; ++i) u[i] = u24(o[i]);
}

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
static double amax3(const double* a) {
  double m = fabs(a[0]);
  if (fabs(a[1]) > m) m = fabs(a[1]);
  if (fabs(a[2]) > m) m = fabs(a[2]);
  return m;
}

/* Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin:
 * "Building an Orthonormal Basis, Revisited" (JCGT 2017). */
static void onb(const double n[3], double b1[3], double b2[3]) {
  double sgn = copysign(1.0, n[2]);
  double a = -1.0 / (sgn + n[2]);
  double b = n[0] * n[1] * a;
  b1[0] = 1.0 + sgn * n[0] * n[0] * a;
  b1[1] = sgn * b;
  b1[2] = -sgn * n[0];
  b2[0] = b;
  b2[1] = sgn + n[1] * n[1] * a;
  b2[2] = -n[1];
}

/* Local cosine-weighted direction: radius sqrt(u0), angle 2*pi*u1, height
 * sqrt(1-u0) (Malley's method; pdf cos(theta)/pi). */
static void cosine_local(double u0, double u1, double l[3]) {
  double r = sqrt(u0), phi = 2.0 * ORA_PI * u1;
  l[0] = r * cos(phi);
  l[1] = r * sin(phi);
  l[2] = sqrt(fmax(0.0, 1.0 - u0));
}

void ora_cosine_direction(const double n[3], double u0, double u1, double out[3]) {
  double b1[3], b2[3], l[3];
  onb(n, b1, b2);
  cosine_local(u0, u1, l);
  for (int i = 0; i < 3; ++i) out[i] = l[0] * b1[i] + l[1] * b2[i] + l[2] * n[i];
}

/* ------------------------------------------------------------------------ */
/* surfel frame (Eq. 1): rotation of the normalised quaternion; t_u, t_v are   */
/* its first two columns and n = t_u x t_v its third.                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  double p[3], tu[3], tv[3], n[3];
  double su, sv, sigma;
  double rho[3], r[3], e;
} surfel64;

static void quat_frame(const double* q_raw, double tu[3], double tv[3], double n[3]) {
  double qn = sqrt(q_raw[0] * q_raw[0] + q_raw[1] * q_raw[1] + q_raw[2] * q_raw[2] + q_raw[3] * q_raw[3]);
  double w = q_raw[0] / qn, x = q_raw[1] / qn, y = q_raw[2] / qn, z = q_raw[3] / qn;
  tu[0] = 1 - 2 * (y * y + z * z);
  tu[1] = 2 * (x * y + w * z);
  tu[2] = 2 * (x * z - w * y);
  tv[0] = 2 * (x * y - w * z);
  tv[1] = 1 - 2 * (x * x + z * z);
  tv[2] = 2 * (y * z + w * x);
  /* n = t_u x t_v */
  n[0] = tu[1] * tv[2] - tu[2] * tv[1];
  n[1] = tu[2] * tv[0] - tu[0] * tv[2];
  n[2] = tu[0] * tv[1] - tu[1] * tv[0];
}

static surfel64* load_surfels(const ora_scene* sc) {
  surfel64* s = (surfel64*)malloc(sizeof(surfel64) * (size_t)(sc->n > 0 ? sc->n : 1));
  if (!s) return NULL;
  for (int64_t i = 0; i < sc->n; ++i) {
    surfel64* g = &s[i];
    for (int k = 0; k < 3; ++k) {
      g->p[k] = sc->pos[3 * i + k];
      g->rho[k] = sc->albedo[3 * i + k];
      g->r[k] = sc->radiance[3 * i + k];
    }
    quat_frame(&sc->quat[4 * i], g->tu, g->tv, g->n);
    g->su = sc->scale[2 * i];
    g->sv = sc->scale[2 * i + 1];
    g->sigma = sc->opacity[i];
    g->e = sc->emissive[i];
  }
  return s;
}

/* ------------------------------------------------------------------------ */
/* one segment: brute force over all surfels, sort, blend (Eq. 1-3)           */
/* ------------------------------------------------------------------------ */
typedef struct {
  double t, alpha, g, sg, u, v, d, q, rel_alpha, dt;
  int64_t idx;
  int clamped;
} hit64;

typedef struct {
  hit64* h;
  int64_t n, cap;
} hitbuf;

static int hb_push(hitbuf* b, const hit64* x) {
  if (b->n == b->cap) {
    int64_t nc = b->cap ? 2 * b->cap : 256;
    hit64* nh = (hit64*)realloc(b->h, sizeof(hit64) * (size_t)nc);
    if (!nh) return -1;
    b->h = nh;
    b->cap = nc;
  }
  b->h[b->n++] = *x;
  return 0;
}

static int hit_cmp(const void* a, const void* b) {
  const hit64* x = (const hit64*)a;
  const hit64* y = (const hit64*)b;
  if (x->t < y->t) return -1;
  if (x->t > y->t) return 1;
  return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

typedef struct {
  const surfel64* s;
  int64_t n;
  const ora_params* prm;
  uint32_t ajit; /* conditioning run r > 0: every sigma g is perturbed by a
                    reproducible relative +-4 FP32 ulps (its FP32 rounding) */
  /* level of detail: bounce segments k >= lod_from trace these surfels
   * instead (NULL: no level of detail) */
  const surfel64* s_lod;
  int64_t n_lod;
  int32_t lod_from;
} world;

/* splitmix64 finaliser (Steele, Lea, Flood: "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) */
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* uniform in [-1, 1) from (surfel, run) */
static double ajit_draw(int64_t idx, uint32_t run) {
  const uint64_t z = mix64((uint64_t)idx * 0x9E3779B97F4A7C15ull + (uint64_t)run * 0xD1B54A32D192ED03ull);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

/* the discrete outcome of a traced segment: its blended surfels in order */
static uint64_t hits_signature(const hitbuf* b) {
  uint64_t h = mix64(0x9E3779B97F4A7C15ull ^ (uint64_t)b->n);
  for (int64_t k = 0; k < b->n; ++k) h = mix64(h ^ (uint64_t)b->h[k].idx);
  return h;
}

/* Collects every blended hit of the segment in order (after the stop) into
 * b, fills seg, returns 0.  mode 1 masks the radiance of non-emitters.
 *
 * eO, eW: first-order estimates of the error an FP32 evaluation carries in
 * the ray origin (absolute length) and direction (radians) when it reaches
 * this segment.  Together with the segment's own FP32 rounding (fp32_eps
 * times the magnitudes involved, times the slack FLAG_K) they give the error
 * of each hit's local coordinates, hence of its alpha, and the near-boundary
 * margins of every decision; the segment's outputs carry the propagated
 * errors (eN, eD, eR, eP, eE) to the next bounce.  Only the flags and these
 * estimates depend on them; the traced values do not. */
static int segment(const world* W, const double O[3], const double w[3], double t_lo, int mode, double eO,
                   double eW, hitbuf* b, ora_segment* seg) {
  const ora_params* prm = W->prm;
  const double eps = prm->fp32_eps;
  const double S2 = prm->support_sigma * prm->support_sigma;
  uint32_t flags = 0;
  b->n = 0;
  double Omax = amax3(O);
  for (int64_t i = 0; i < W->n; ++i) {
    const surfel64* g = &W->s[i];
    double d = dot3(w, g->n);
    if (fabs(d) < 1e-12) continue;
    double pO[3] = {g->p[0] - O[0], g->p[1] - O[1], g->p[2] - O[2]};
    double t = dot3(pO, g->n) / d;
    /* x - p = (O - p) + t w */
    double dx[3] = {-pO[0] + t * w[0], -pO[1] + t * w[1], -pO[2] + t * w[2]};
    double u = dot3(dx, g->tu) / g->su;
    double v = dot3(dx, g->tv) / g->sv;
    double q = u * u + v * v;
    /* position error at the hit: own rounding of coordinates of magnitude L
     * plus the incoming ray error; 1/|d| through the plane intersection,
     * divided by the scale in u, v */
    double L = Omax + amax3(g->p) + fabs(t);
    double ep = eps > 0 ? ERR_C * eps * L + eO + fabs(t) * eW : 0.0;
    double dt = ep / fabs(d);
    double smin = g->su < g->sv ? g->su : g->sv;
    double du = ep / (fabs(d) * smin);
    double dq = 2.0 * sqrt(2.0 * (q > S2 ? q : S2)) * du + ERR_C * eps * S2;
    double sg = g->sigma * exp(-0.5 * q);
    if (W->ajit) sg *= 1.0 + 4.0 * eps * ajit_draw(i, W->ajit);
    double rel_a = sqrt(2.0 * q) * du + ERR_C * eps;
    int in_support = q <= S2;
    int near_support = eps > 0 && fabs(q - S2) <= FLAG_K * dq;
    int ahead = t > t_lo;
    int near_tlo = eps > 0 && fabs(t - t_lo) <= FLAG_K * dt;
    double alpha = sg < prm->alpha_max ? sg : prm->alpha_max;
    int big = alpha >= prm->alpha_min;
    int near_amin = eps > 0 && fabs(sg - prm->alpha_min) <= FLAG_K * (sg * rel_a + ERR_C * eps * prm->alpha_min);
    /* flags only matter for surfels that are, or could be, accepted */
    if ((in_support || near_support) && (ahead || near_tlo) && (big || near_amin)) {
      if (near_support) flags |= ORA_FLAG_SUPPORT;
      if (near_tlo) flags |= ORA_FLAG_TLO;
      if (near_amin) flags |= ORA_FLAG_AMIN;
      if (eps > 0 && fabs(sg - prm->alpha_max) <= FLAG_K * (sg * rel_a + ERR_C * eps)) flags |= ORA_FLAG_AMAX;
      if (eps > 0 && fabs(d) < FLAG_K * eps) flags |= ORA_FLAG_GRAZE;
    }
    if (!(in_support && ahead && big)) continue;
    hit64 h;
    h.t = t;
    h.alpha = alpha;
    h.g = exp(-0.5 * q);
    h.sg = sg;
    h.u = u;
    h.v = v;
    h.d = d;
    h.q = q;
    h.rel_alpha = sg >= prm->alpha_max ? ERR_C * eps : rel_a;
    h.dt = dt;
    h.idx = i;
    h.clamped = sg >= prm->alpha_max;
    if (hb_push(b, &h)) return -1;
  }
  qsort(b->h, (size_t)b->n, sizeof(hit64), hit_cmp);

  memset(seg, 0, sizeof(*seg));
  double T = 1.0, relT = 0.0;
  int64_t used = 0;
  for (int64_t k = 0; k < b->n; ++k) {
    const hit64* h = &b->h[k];
    const surfel64* g = &W->s[h->idx];
    double wgt = T * h->alpha;
    double sgn = h->d > 0 ? -1.0 : 1.0; /* normal facing the ray origin */
    double remit = (mode == 1 && !(g->e > prm->tau_E)) ? 0.0 : 1.0;
    for (int c = 0; c < 3; ++c) {
      seg->N[c] += wgt * sgn * g->n[c];
      seg->R[c] += wgt * remit * g->r[c];
      seg->P[c] += wgt * g->rho[c];
    }
    seg->D += wgt * h->t;
    seg->E += wgt * g->e;
    T *= (1.0 - h->alpha);
    relT += h->alpha / (1.0 - h->alpha) * h->rel_alpha;
    used = k + 1;
    if (eps > 0) {
      if (fabs(T - prm->T_min) <= FLAG_K * (relT * T + ERR_C * eps * prm->T_min)) flags |= ORA_FLAG_TSTOP;
      if (k + 1 < b->n) {
        const hit64* h2 = &b->h[k + 1];
        if (fabs(h2->t - h->t) <= FLAG_K * (h->dt + h2->dt)) flags |= ORA_FLAG_ORDER;
      }
    }
    if (T < prm->T_min) break;
  }
  b->n = used;
  seg->A = 1.0 - T;
  seg->n_hits = (int32_t)used;
  if (used > 0) {
    double nn = norm3(seg->N);
    for (int c = 0; c < 3; ++c) seg->Nn[c] = seg->N[c] / nn;
    seg->Dn = seg->D / seg->A;
  }
  /* propagated errors of the blended values (first order in the weight errors) */
  if (eps > 0 && used > 0) {
    double Tb = 1.0, rT = 0.0, eR = 0.0, eP = 0.0, eE = 0.0, eN = 0.0, eD = 0.0;
    for (int64_t k = 0; k < used; ++k) {
      const hit64* h = &b->h[k];
      const surfel64* g = &W->s[h->idx];
      const double wgt = Tb * h->alpha, rw = h->rel_alpha + rT;
      const double sgn = h->d > 0 ? -1.0 : 1.0;
      const double remit = (mode == 1 && !(g->e > prm->tau_E)) ? 0.0 : 1.0;
      double rmax = remit * amax3(g->r), pmax = amax3(g->rho);
      eR += wgt * rw * rmax;
      eP += wgt * rw * pmax;
      eE += wgt * rw * fabs(g->e);
      double nf[3] = {sgn * g->n[0], sgn * g->n[1], sgn * g->n[2]};
      double c = dot3(nf, seg->Nn);
      double perp[3] = {nf[0] - c * seg->Nn[0], nf[1] - c * seg->Nn[1], nf[2] - c * seg->Nn[2]};
      eN += wgt * rw * norm3(perp);
      eD += wgt * (rw * fabs(h->t - seg->Dn) + h->dt);
      rT += h->alpha / (1.0 - h->alpha) * h->rel_alpha;
      Tb *= 1.0 - h->alpha;
    }
    double Rm = amax3(seg->R), Pm = amax3(seg->P);
    seg->eR = Rm > 0 ? eR / Rm + ERR_C * eps : 0.0;
    seg->eP = Pm > 0 ? eP / Pm + ERR_C * eps : 0.0;
    seg->eE = eE + ERR_C * eps;
    seg->eN = eN / norm3(seg->N) + ERR_C * eps;
    seg->eD = eD / seg->A + seg->Dn * (T * rT) / seg->A + ERR_C * eps * seg->Dn;
  }
  if (eps > 0 && fabs(seg->E - prm->tau_E) <= FLAG_K * seg->eE) flags |= ORA_FLAG_EMIT;
  seg->flags = flags;
  return 0;
}

int ora_trace_segment(const ora_scene* sc, const ora_params* prm, const double O[3], const double w[3],
                      double t_lo, int32_t mode, ora_segment* out, int32_t* hit_idx, int32_t max_hits) {
  surfel64* s = load_surfels(sc);
  if (!s) return -1;
  world W = {s, sc->n, prm};
  hitbuf b = {0, 0, 0};
  int rc = segment(&W, O, w, t_lo, mode, 0.0, 0.0, &b, out);
  if (hit_idx)
    for (int32_t k = 0; k < max_hits; ++k) hit_idx[k] = k < b.n ? (int32_t)b.h[k].idx : -1;
  free(b.h);
  free(s);
  return rc;
}

static void write_rec(const ora_segment* g, double* rec) {
  rec[0] = g->Nn[0];
  rec[1] = g->Nn[1];
  rec[2] = g->Nn[2];
  rec[3] = g->Dn;
  rec[4] = g->R[0];
  rec[5] = g->R[1];
  rec[6] = g->R[2];
  rec[7] = g->E;
  rec[8] = g->P[0];
  rec[9] = g->P[1];
  rec[10] = g->P[2];
  rec[11] = g->A;
}

/* ------------------------------------------------------------------------ */
/* camera: OpenCV pinhole ray through the pixel centre                        */
/* ------------------------------------------------------------------------ */
static void primary_ray(const ora_camera* cam, int64_t pixel, double O[3], double w[3]) {
  int64_t x = pixel % cam->width, y = pixel / cam->width;
  double dc[3] = {((double)x + 0.5 - cam->cx) / cam->fx, ((double)y + 0.5 - cam->cy) / cam->fy, 1.0};
  for (int r = 0; r < 3; ++r) {
    O[r] = cam->c2w[4 * r + 3];
    w[r] = cam->c2w[4 * r + 0] * dc[0] + cam->c2w[4 * r + 1] * dc[1] + cam->c2w[4 * r + 2] * dc[2];
  }
  double l = norm3(w);
  for (int r = 0; r < 3; ++r) w[r] /= l;
}

/* ------------------------------------------------------------------------ */
/* threading: a shared atomic work counter over items                        */
/* ------------------------------------------------------------------------ */
typedef struct job job;
typedef int (*item_fn)(job* jb, int64_t item, hitbuf* b);
struct job {
  world W;
  item_fn fn;
  int64_t n_items;
  atomic_llong next;
  atomic_int err;
  void* ctx;
};

static void* worker(void* arg) {
  job* jb = (job*)arg;
  hitbuf b = {0, 0, 0};
  for (;;) {
    int64_t i = atomic_fetch_add(&jb->next, 1);
    if (i >= jb->n_items) break;
    if (jb->fn(jb, i, &b)) atomic_store(&jb->err, 1);
  }
  free(b.h);
  return NULL;
}

static int run_job(job* jb, int32_t n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  atomic_store(&jb->next, 0);
  atomic_store(&jb->err, 0);
  pthread_t th[256];
  int started = 0;
  for (int i = 1; i < n_threads; ++i) {
    if (pthread_create(&th[i], NULL, worker, jb) == 0) started = i;
    else break;
  }
  worker(jb);
  for (int i = 1; i <= started; ++i) pthread_join(th[i], NULL);
  return atomic_load(&jb->err) ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* batch of rays                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  const double* rays;
  int32_t mode, max_hits;
  double* out_rec;
  int32_t* out_nhits;
  uint32_t* out_flags;
  int32_t* hit_idx;
  double* out_dev;
} rays_ctx;

static void jitter_ray(double O[3], double w[3], uint64_t seed, int64_t pix, int32_t s, int32_t k, int32_t run,
                       double mag);

static int rays_item(job* jb, int64_t i, hitbuf* b) {
  rays_ctx* c = (rays_ctx*)jb->ctx;
  const double* r = &c->rays[6 * i];
  ora_segment g;
  if (segment(&jb->W, r, r + 3, 0.0, c->mode, 0.0, 0.0, b, &g)) return -1;
  write_rec(&g, &c->out_rec[12 * i]);
  if (c->out_nhits) c->out_nhits[i] = g.n_hits;
  if (c->hit_idx)
    for (int32_t k = 0; k < c->max_hits; ++k) c->hit_idx[i * c->max_hits + k] = k < b->n ? (int32_t)b->h[k].idx : -1;
  /* a single segment is ill-conditioned in FP32 when re-tracing it with the
   * ray perturbed at FP32 rounding scale (and every sigma g by +-4 ulps), as
   * the render's conditioning runs do for whole samples, changes its blended
   * surfel list or moves a blended value by more than cond_tol: R, P, E and A
   * relative to the value, N~ by cond_tol / 5 absolute (the comparison's
   * 2e-5 on a unit vector, with the same margin), D~ relative */
  const ora_params* prm = jb->W.prm;
  double* dv = c->out_dev ? &c->out_dev[12 * i] : NULL;
  if (dv)
    for (int k = 0; k < 12; ++k) dv[k] = 0.0;
  if (prm->fp32_eps > 0 && prm->cond_tol > 0 && g.n_hits > 0) {
    const uint64_t sig = hits_signature(b);
    double rec0[12];
    write_rec(&g, rec0);
    /* with out_dev both runs are taken, so the spread covers both; the flag
     * is the same either way */
    for (int run = 1; run <= 2 && (dv || !(g.flags & ORA_FLAG_COND)); ++run) {
      world Wj = jb->W;
      Wj.ajit = (uint32_t)run;
      double Oj[3] = {r[0], r[1], r[2]}, wj[3] = {r[3], r[4], r[5]};
      jitter_ray(Oj, wj, 0x9E3779B97F4A7C15ull, i, -2, 0, run, 2.0 * prm->fp32_eps);
      ora_segment gj;
      if (segment(&Wj, Oj, wj, 0.0, c->mode, 0.0, 0.0, b, &gj)) return -1;
      int ill = hits_signature(b) != sig;
      const double tol = prm->cond_tol;
      for (int k = 0; k < 3 && !ill; ++k) {
        ill |= fabs(gj.R[k] - g.R[k]) > tol * fabs(g.R[k]);
        ill |= fabs(gj.P[k] - g.P[k]) > tol * fabs(g.P[k]);
        ill |= fabs(gj.Nn[k] - g.Nn[k]) > tol / 5.0;
      }
      ill |= fabs(gj.E - g.E) > tol * fabs(g.E);
      ill |= fabs(gj.A - g.A) > tol * fabs(g.A);
      ill |= fabs(gj.Dn - g.Dn) > tol * fabs(g.Dn);
      if (ill) g.flags |= ORA_FLAG_COND;
      if (dv) {
        /* per record column, the largest change over the runs; +inf on
         * every column when a run changes the blended surfel list */
        const int discrete = hits_signature(b) != sig;
        double recj[12];
        write_rec(&gj, recj);
        for (int k = 0; k < 12; ++k) {
          const double d = discrete ? INFINITY : fabs(recj[k] - rec0[k]);
          if (d > dv[k]) dv[k] = d;
        }
      }
    }
  }
  if (c->out_flags) c->out_flags[i] = g.flags;
  return 0;
}

int ora_trace_rays(const ora_scene* sc, const ora_params* prm, const double* rays, int64_t n_rays,
                   int32_t mode, double* out_rec, int32_t* out_nhits, uint32_t* out_flags, int32_t* hit_idx,
                   int32_t max_hits, double* out_dev, int32_t n_threads) {
  surfel64* s = load_surfels(sc);
  if (!s) return -1;
  rays_ctx c = {rays, mode, max_hits, out_rec, out_nhits, out_flags, hit_idx, out_dev};
  job jb;
  memset(&jb, 0, sizeof(jb)); /* W.ajit = 0: the exact evaluation, no perturbation */
  jb.W.s = s;
  jb.W.n = sc->n;
  jb.W.prm = prm;
  jb.fn = rays_item;
  jb.n_items = n_rays;
  jb.ctx = &c;
  int rc = run_job(&jb, n_threads);
  free(s);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* primary records                                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
  const ora_camera* cam;
  int32_t mode;
  const int32_t* pixels;
  double* out_rec;
  uint32_t* out_flags;
} prim_ctx;

static int prim_item(job* jb, int64_t i, hitbuf* b) {
  prim_ctx* c = (prim_ctx*)jb->ctx;
  double O[3], w[3];
  primary_ray(c->cam, c->pixels[i], O, w);
  ora_segment g;
  if (segment(&jb->W, O, w, 0.0, c->mode, 0.0, ERR_C * jb->W.prm->fp32_eps, b, &g)) return -1;
  write_rec(&g, &c->out_rec[12 * i]);
  if (c->out_flags) c->out_flags[i] = g.flags;
  return 0;
}

int ora_primary(const ora_scene* sc, const ora_camera* cam, const ora_params* prm, int32_t mode,
                const int32_t* pixels, int64_t n_pix, double* out_rec, uint32_t* out_flags, int32_t n_threads) {
  surfel64* s = load_surfels(sc);
  if (!s) return -1;
  prim_ctx c = {cam, mode, pixels, out_rec, out_flags};
  job jb;
  memset(&jb, 0, sizeof(jb)); /* W.ajit = 0: the exact evaluation, no perturbation */
  jb.W.s = s;
  jb.W.n = sc->n;
  jb.W.prm = prm;
  jb.fn = prim_item;
  jb.n_items = n_pix;
  jb.ctx = &c;
  int rc = run_job(&jb, n_threads);
  free(s);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* emitter sampling with multiple importance sampling (path tracing, mis = 1)
 *
 * The paper names emitter importance sampling with MIS as future work
 * (Sec. 5 and Appendix D, on sampling); this is one exact form of it.  The
 * blended radiance of a segment is a sum of per-surfel terms, R = sum_i w_i
 * r~_i (Eq. 2, w_i = T_{i-1} alpha_i), and each emitter term of the
 * one-bounce integral is estimated by two strategies combined with the power
 * heuristic: the cosine-sampled continuation (pdf p_B = cos / pi) and
 * sampling a point on that emitter surfel (pdf p_L,i = q_i g_i(u, v) t^2 /
 * |w . n_i| in solid angle, q_i the selection probability and g_i the
 * truncated Gaussian density on the surfel plane).  Both pdfs are local to
 * the hit, so no other surfel is involved.                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t n_e;   /* emitters with a positive weight                       */
  int64_t* idx;  /* surfel index of the k-th emitter, ascending           */
  double* cdf;   /* running sum of the weights in that order              */
  double total;
  double* q;     /* per surfel: selection probability (0: not an emitter) */
  double norm;   /* 2 pi (1 - exp(-S^2 / 2)): the truncated Gaussian's mass */
} emitters;

/* selection weight: mean radiance x opacity x scale area (e_i > tau_E) */
static double emitter_weight(const surfel64* g, const ora_params* prm) {
  if (!(g->e > prm->tau_E)) return 0.0;
  double m = (g->r[0] + g->r[1]) + g->r[2];
  m = m / 3.0;
  return ((m * g->sigma) * g->su) * g->sv;
}

static int build_emitters(const world* W, emitters* em) {
  memset(em, 0, sizeof(*em));
  const ora_params* prm = W->prm;
  em->norm = 2.0 * ORA_PI * (1.0 - exp(-0.5 * prm->support_sigma * prm->support_sigma));
  em->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(W->n > 0 ? W->n : 1));
  em->cdf = (double*)malloc(sizeof(double) * (size_t)(W->n > 0 ? W->n : 1));
  em->q = (double*)calloc((size_t)(W->n > 0 ? W->n : 1), sizeof(double));
  if (!em->idx || !em->cdf || !em->q) return -1;
  double run = 0.0;
  for (int64_t i = 0; i < W->n; ++i) {
    double w = emitter_weight(&W->s[i], prm);
    if (w > 0.0) {
      run += w;
      em->idx[em->n_e] = i;
      em->cdf[em->n_e] = run;
      ++em->n_e;
    }
  }
  em->total = run;
  for (int64_t k = 0; k < em->n_e; ++k) {
    const int64_t i = em->idx[k];
    em->q[i] = emitter_weight(&W->s[i], prm) / run;
  }
  return 0;
}

static void free_emitters(emitters* em) {
  free(em->idx);
  free(em->cdf);
  free(em->q);
}

/* the k-th emitter for a draw u in [0, 1): smallest k with cdf_k > u total */
static int64_t select_emitter(const emitters* em, double u) {
  const double x = u * em->total;
  int64_t lo = 0, hi = em->n_e - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (em->cdf[mid] > x) hi = mid;
    else lo = mid + 1;
  }
  return em->idx[lo];
}

/* a point of the emitter's support disc with the truncated standard 2D
 * Gaussian density: radius by the inverse of its CDF, uniform angle */
static void emitter_point(const surfel64* g, double S2, double u1, double u2, double y[3]) {
  double rho = sqrt(-2.0 * log(1.0 - u1 * (1.0 - exp(-0.5 * S2))));
  double phi = 2.0 * ORA_PI * u2;
  double a = rho * cos(phi), b = rho * sin(phi);
  for (int k = 0; k < 3; ++k) y[k] = g->p[k] + a * g->su * g->tu[k] + b * g->sv * g->tv[k];
}

/* solid-angle density of the emitter strategy for a hit of surfel g */
static double light_pdf_hit(const emitters* em, const surfel64* g, double qsel, const hit64* h) {
  return qsel * exp(-0.5 * h->q) / (em->norm * g->su * g->sv) * h->t * h->t / fabs(h->d);
}

int ora_light_pdf(const ora_scene* sc, const ora_params* prm, const double O[3], const double w[3],
                  double* out_pdf) {
  surfel64* s = load_surfels(sc);
  if (!s) return -1;
  world W = {s, sc->n, prm};
  emitters em;
  if (build_emitters(&W, &em)) {
    free(s);
    free_emitters(&em);
    return -1;
  }
  const double S2 = prm->support_sigma * prm->support_sigma;
  double sum = 0.0;
  int count = 0;
  for (int64_t i = 0; i < sc->n; ++i) {
    if (!(em.q[i] > 0.0)) continue;
    const surfel64* g = &s[i];
    double d = dot3(w, g->n);
    if (fabs(d) < 1e-12) continue;
    double pO[3] = {g->p[0] - O[0], g->p[1] - O[1], g->p[2] - O[2]};
    double t = dot3(pO, g->n) / d;
    if (!(t > 0.0)) continue;
    double dx[3] = {-pO[0] + t * w[0], -pO[1] + t * w[1], -pO[2] + t * w[2]};
    double u = dot3(dx, g->tu) / g->su, v = dot3(dx, g->tv) / g->sv;
    hit64 h;
    h.q = u * u + v * v;
    if (h.q > S2) continue;
    h.t = t;
    h.d = d;
    sum += light_pdf_hit(&em, g, em.q[i], &h);
    ++count;
  }
  *out_pdf = sum;
  free_emitters(&em);
  free(s);
  return count;
}

/* ------------------------------------------------------------------------ */
/* rendering (Eq. 6 and Eq. 8)                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  const ora_camera* cam;
  int32_t kind, spp, max_bounces, rr_start;
  uint64_t seed;
  const int32_t* pixels;
  double* out_rgb;
  double* out_samples;
  uint32_t* out_sample_flags;
  int64_t* out_segments;
  const emitters* em; /* emitter sampling (path tracing with mis), else NULL */
  double* out_sample_dev;
} render_ctx;

/* Perturbs a ray at FP32 rounding scale for the conditioning estimate:
 * every origin component by up to mag * max|O|, every direction component by
 * up to mag, then renormalises.  Counter-based, so the perturbation of a
 * (pixel, sample, bounce, run) is reproducible. */
static void jitter_ray(double O[3], double w[3], uint64_t seed, int64_t pix, int32_t s, int32_t k, int32_t run,
                       double mag) {
  uint32_t key[2] = {(uint32_t)seed ^ 0x5bd1e995u, (uint32_t)(seed >> 32) ^ 0x1b873593u};
  uint32_t c1[4] = {(uint32_t)pix, (uint32_t)s, (uint32_t)k, 0x40000000u | (uint32_t)run};
  uint32_t c2[4] = {(uint32_t)pix, (uint32_t)s, (uint32_t)k, 0x20000000u | (uint32_t)run};
  uint32_t o1[4], o2[4];
  ora_philox4x32_10(c1, key, o1);
  ora_philox4x32_10(c2, key, o2);
  double om = amax3(O);
  if (om < 1e-3) om = 1e-3;
  for (int j = 0; j < 3; ++j) {
    O[j] += mag * om * (2.0 * u24(o1[j]) - 1.0);
    w[j] += mag * (2.0 * u24(o2[j]) - 1.0);
  }
  double l = norm3(w);
  for (int j = 0; j < 3; ++j) w[j] /= l;
}

/* One sample's path from the pixel's primary segment g1 (Eq. 6 for kind 0,
 * Eq. 8 for kind 1).  run > 0 perturbs every secondary ray (conditioning
 * estimate); run 0 is the exact evaluation and also collects the flags.
 * *psig accumulates the path's discrete outcome: each traced segment's
 * blended surfels and each bounce entered. */
static int path_sample(job* jb, const render_ctx* c, hitbuf* b, int64_t pix, int32_t s, const double O[3],
                       const double w[3], const ora_segment* g1, int32_t run, double contrib[3], uint32_t* sflags,
                       int64_t* segments, uint64_t* psig) {
  const ora_params* prm = jb->W.prm;
  const double eps = prm->fp32_eps;
  const int pt = c->kind == 1;
  const int seg_mode = pt ? 1 : 0;
  const int reflect_all = prm->emitters_reflect != 0;
  contrib[0] = contrib[1] = contrib[2] = 0.0;
  if (g1->n_hits == 0) return 0; /* primary miss: no light (no environment) */
  if (g1->E > prm->tau_E && !reflect_all) {
    for (int k = 0; k < 3; ++k) contrib[k] = g1->R[k]; /* Eq. 4: L_o = L_e = R */
    return 0;
  }
  double beta[3], X[3], Nn[3], rel = g1->eP, eN = g1->eN;
  if (reflect_all)
    for (int k = 0; k < 3; ++k) contrib[k] = g1->R[k];
  for (int k = 0; k < 3; ++k) {
    beta[k] = g1->P[k]; /* f cos / p = (P/pi) cos / (cos/pi) = P */
    X[k] = O[k] + g1->Dn * w[k];
    Nn[k] = g1->Nn[k];
  }
  const int B = pt ? c->max_bounces : 1;
  for (int32_t k = 1; k <= B; ++k) {
    double u[4];
    draws(c->seed, pix, s, k, u);
    if (pt && !reflect_all && k >= c->rr_start) {
      double q = beta[0];
      if (beta[1] > q) q = beta[1];
      if (beta[2] > q) q = beta[2];
      if (q > 1.0) q = 1.0;
      if (eps > 0 && fabs(u[2] - q) <= FLAG_K * (rel * q + ERR_C * eps)) *sflags |= ORA_FLAG_RR;
      if (!(u[2] < q)) return 0; /* terminated, contributes 0 */
      for (int j = 0; j < 3; ++j) beta[j] /= q;
    }
    if (eps > 0 && fabs(Nn[2]) <= FLAG_K * eN) *sflags |= ORA_FLAG_ONB;
    *psig = mix64(*psig ^ (0x100u + (uint32_t)k));
    double w2[3], O2[3];
    ora_cosine_direction(Nn, u[0], u[1], w2);
    for (int j = 0; j < 3; ++j) O2[j] = X[j] + prm->bounce_offset * Nn[j];
    const emitters* em = c->em;
    /* the normal the MIS pdfs use: with emitter sampling the blended normal
     * enters the sample directly (p_B = cos / pi, the emitter sample's cos),
     * so the conditioning runs also perturb it by its propagated FP32 error
     * estimate */
    double Nm[3] = {Nn[0], Nn[1], Nn[2]};
    if (em && em->n_e > 0 && run > 0) {
      double Oz[3] = {0, 0, 0};
      jitter_ray(Oz, Nm, c->seed, pix, s, k + (2 << 20), run, eN + ERR_C * eps);
    }
    if (em && em->n_e > 0) {
      /* emitter sample from this vertex: draws (pixel, sample, k, 1) */
      double v4[4], y[3], wl[3], Ol[3] = {O2[0], O2[1], O2[2]};
      draws_w(c->seed, pix, s, k, 1u, v4);
      const int64_t it = select_emitter(em, v4[0]);
      const surfel64* gt = &jb->W.s[it];
      emitter_point(gt, prm->support_sigma * prm->support_sigma, v4[1], v4[2], y);
      double dl[3] = {y[0] - O2[0], y[1] - O2[1], y[2] - O2[2]};
      const double dist = norm3(dl);
      for (int j = 0; j < 3; ++j) wl[j] = dl[j] / dist;
      const double cosx = dot3(wl, Nm);
      if (eps > 0 && fabs(cosx) <= FLAG_K * (eN + ERR_C * eps * (1.0 + amax3(O2) / dist))) *sflags |= ORA_FLAG_HEMI;
      if (cosx > 0.0) {
        /* the FP32 emitter point comes from three transcendental evaluations
         * (log, sqrt, sincos): its rays are perturbed at four times the scale
         * of the other rays in the conditioning runs */
        if (run > 0) jitter_ray(Ol, wl, c->seed, pix, s, k + (1 << 20), run, 8.0 * eps);
        ora_segment g3;
        if (segment(&jb->W, Ol, wl, 0.0, 1, ERR_C * eps * amax3(Ol), ERR_C * eps, b, &g3)) return -1;
        *psig = mix64(*psig ^ hits_signature(b));
        ++*segments;
        *sflags |= g3.flags;
        if (g3.n_hits > 0 && g3.E > prm->tau_E) {
          double T = 1.0;
          for (int64_t h = 0; h < b->n; ++h) {
            const hit64* hh = &b->h[h];
            if (hh->idx == it) {
              const double wi = T * hh->alpha;
              const double pl = light_pdf_hit(em, gt, em->q[it], hh), pb = cosx / ORA_PI;
              const double f = wi * pb * pl / (pl * pl + pb * pb);
              for (int j = 0; j < 3; ++j) contrib[j] += beta[j] * gt->r[j] * f;
              break;
            }
            T *= 1.0 - hh->alpha;
          }
        }
      }
    }
    if (run > 0) jitter_ray(O2, w2, c->seed, pix, s, k, run, 2.0 * eps);
    ora_segment g2;
    /* the surfels this bounce segment traces: the merged ones from bounce
     * lod_from on */
    world Wk = jb->W;
    if (Wk.s_lod && k >= Wk.lod_from) {
      Wk.s = Wk.s_lod;
      Wk.n = Wk.n_lod;
    }
    /* margins at this segment's own FP32 rounding scale */
    if (segment(&Wk, O2, w2, 0.0, seg_mode, ERR_C * eps * amax3(O2), ERR_C * eps, b, &g2)) return -1;
    *psig = mix64(*psig ^ hits_signature(b));
    ++*segments;
    *sflags |= g2.flags;
    if (g2.n_hits == 0) return 0; /* miss: no light */
    if (reflect_all) {
      for (int j = 0; j < 3; ++j) contrib[j] += beta[j] * g2.R[j];
    } else if (!pt) {
      /* Eq. 6: the secondary's accumulated radiance is the cache */
      for (int j = 0; j < 3; ++j) contrib[j] = beta[j] * g2.R[j];
      return 0;
    } else if (g2.E > prm->tau_E) {
      /* Eq. 8: first emissive vertex within the bounce limit; with emitter
       * sampling each emitter term carries its power-heuristic weight */
      if (em && em->n_e > 0) {
        const double pb = dot3(w2, Nm) / ORA_PI;
        double T = 1.0;
        for (int64_t h = 0; h < b->n; ++h) {
          const hit64* hh = &b->h[h];
          const surfel64* g = &jb->W.s[hh->idx];
          const double wk = T * hh->alpha;
          if (em->q[hh->idx] > 0.0) {
            const double pl = light_pdf_hit(em, g, em->q[hh->idx], hh);
            const double f = wk * pb * pb / (pb * pb + pl * pl);
            for (int j = 0; j < 3; ++j) contrib[j] += beta[j] * g->r[j] * f;
          }
          T *= 1.0 - hh->alpha;
        }
      } else {
        for (int j = 0; j < 3; ++j) contrib[j] = beta[j] * g2.R[j];
      }
      return 0;
    }
    if (k == B) return 0; /* bounce limit exceeded: discarded (or done) */
    for (int j = 0; j < 3; ++j) {
      beta[j] *= g2.P[j];
      X[j] = O2[j] + g2.Dn * w2[j];
      Nn[j] = g2.Nn[j];
    }
    rel += g2.eP;
    eN = g2.eN;
  }
  return 0;
}

static int render_item(job* jb, int64_t i, hitbuf* b) {
  render_ctx* c = (render_ctx*)jb->ctx;
  const ora_params* prm = jb->W.prm;
  const double eps = prm->fp32_eps;
  const int64_t pix = c->pixels[i];
  const int seg_mode = c->kind == 1 ? 1 : 0;
  double O[3], w[3];
  primary_ray(c->cam, pix, O, w);
  ora_segment g1;
  if (segment(&jb->W, O, w, 0.0, seg_mode, 0.0, ERR_C * eps, b, &g1)) return -1;
  const uint64_t sig1 = hits_signature(b);
  int64_t segments = 1;
  double acc[3] = {0, 0, 0};
  /* conditioning runs: the whole sample (primary direction included) is
   * re-evaluated with every ray perturbed at FP32 scale */
  const int n_runs = (prm->cond_tol > 0 && eps > 0) ? ORA_COND_RUNS : 0;
  double* dev = NULL;
  double* mag = NULL;
  if (n_runs) {
    dev = (double*)calloc((size_t)c->spp * 3, sizeof(double));
    mag = (double*)calloc((size_t)c->spp * 3, sizeof(double));
    if (!dev || !mag) {
      free(dev);
      free(mag);
      return -1;
    }
  }
  ora_segment gj[ORA_COND_RUNS];
  double wj[ORA_COND_RUNS][3];
  uint64_t sigj[ORA_COND_RUNS];
  job jr[ORA_COND_RUNS];
  for (int r = 0; r < n_runs; ++r) {
    jr[r] = *jb;
    jr[r].W.ajit = (uint32_t)(r + 1);
    double Oj[3] = {O[0], O[1], O[2]};
    for (int k = 0; k < 3; ++k) wj[r][k] = w[k];
    jitter_ray(Oj, wj[r], c->seed, pix, -1, 0, r + 1, 2.0 * eps);
    if (segment(&jr[r].W, O, wj[r], 0.0, seg_mode, 0.0, ERR_C * eps, b, &gj[r])) {
      free(dev);
      free(mag);
      return -1;
    }
    sigj[r] = hits_signature(b);
  }
  for (int32_t s = 0; s < c->spp; ++s) {
    uint32_t sflags = g1.flags;
    double contrib[3];
    uint64_t sig0 = sig1;
    if (path_sample(jb, c, b, pix, s, O, w, &g1, 0, contrib, &sflags, &segments, &sig0)) {
      free(dev);
      free(mag);
      return -1;
    }
    for (int r = 0; r < n_runs; ++r) {
      double cj[3];
      uint32_t fj = 0;
      int64_t sj = 0;
      uint64_t sigr = sigj[r];
      if (path_sample(&jr[r], c, b, pix, s, O, wj[r], &gj[r], r + 1, cj, &fj, &sj, &sigr)) {
        free(dev);
        free(mag);
        return -1;
      }
      for (int k = 0; k < 3; ++k) {
        double d = fabs(cj[k] - contrib[k]);
        if (d > dev[3 * s + k]) dev[3 * s + k] = d;
      }
      /* a discrete outcome along the path (a blended surfel, a bounce) that
       * FP32-scale perturbations change makes the sample ill-conditioned even
       * when this run's value happens to agree */
      if (sigr != sig0) dev[3 * s] = INFINITY;
    }
    for (int k = 0; k < 3; ++k) acc[k] += contrib[k];
    if (mag)
      for (int k = 0; k < 3; ++k) mag[3 * s + k] = fabs(contrib[k]);
    if (c->out_samples)
      for (int k = 0; k < 3; ++k) c->out_samples[(i * c->spp + s) * 3 + k] = contrib[k];
    if (c->out_sample_flags) c->out_sample_flags[i * c->spp + s] = sflags;
  }
  for (int k = 0; k < 3; ++k) c->out_rgb[3 * i + k] = c->spp > 0 ? acc[k] / c->spp : 0.0;
  if (c->out_sample_dev)
    for (int32_t s = 0; s < c->spp; ++s) {
      /* a discrete change is reported on every channel */
      const int discrete = n_runs && isinf(dev[3 * s]);
      for (int k = 0; k < 3; ++k)
        c->out_sample_dev[(i * c->spp + s) * 3 + k] = !n_runs ? 0.0 : discrete ? INFINITY : dev[3 * s + k];
    }
  if (n_runs && c->out_sample_flags) {
    /* a sample is ill-conditioned when FP32-scale perturbations move any of
     * its channels by more than cond_tol of that channel's value (the
     * comparison's tolerance is per channel; radiance is non-negative, so a
     * mean of unflagged samples keeps that relative bound) or change a
     * discrete outcome along its path */
    for (int32_t s = 0; s < c->spp; ++s)
      for (int k = 0; k < 3; ++k)
        if (dev[3 * s + k] > prm->cond_tol * mag[3 * s + k]) c->out_sample_flags[i * c->spp + s] |= ORA_FLAG_COND;
  }
  free(dev);
  free(mag);
  if (c->out_segments) c->out_segments[i] = segments;
  return 0;
}

int ora_render(const ora_scene* sc, const ora_camera* cam, const ora_params* prm, int32_t kind, int32_t spp,
               int32_t max_bounces, int32_t rr_start, uint64_t seed, const int32_t* pixels, int64_t n_pix,
               double* out_rgb, double* out_samples, uint32_t* out_sample_flags, int64_t* out_segments,
               double* out_sample_dev, int32_t n_threads) {
  surfel64* s = load_surfels(sc);
  if (!s) return -1;
  render_ctx c = {cam, kind, spp, max_bounces, rr_start, seed, pixels, out_rgb, out_samples, out_sample_flags,
                  out_segments, NULL, out_sample_dev};
  job jb;
  memset(&jb, 0, sizeof(jb)); /* W.ajit = 0: the exact evaluation, no perturbation */
  jb.W.s = s;
  jb.W.n = sc->n;
  jb.W.prm = prm;
  jb.fn = render_item;
  jb.n_items = n_pix;
  jb.ctx = &c;
  emitters em;
  memset(&em, 0, sizeof(em));
  if (prm->mis && kind == 1) {
    if (prm->emitters_reflect || build_emitters(&jb.W, &em)) {
      free_emitters(&em);
      free(s);
      return -1;
    }
    c.em = &em;
  }
  int rc = run_job(&jb, n_threads);
  free_emitters(&em);
  free(s);
  return rc;
}

int ora_render_lod(const ora_scene* sc, const ora_scene* lod_sc, int32_t lod_from, const ora_camera* cam,
                   const ora_params* prm, int32_t spp, int32_t max_bounces, int32_t rr_start, uint64_t seed,
                   const int32_t* pixels, int64_t n_pix, double* out_rgb, double* out_samples,
                   uint32_t* out_sample_flags, int64_t* out_segments, double* out_sample_dev,
                   int32_t n_threads) {
  if (prm->mis || !lod_sc || lod_from < 1) return -1;
  surfel64* s = load_surfels(sc);
  surfel64* sl = load_surfels(lod_sc);
  if (!s || !sl) {
    free(s);
    free(sl);
    return -1;
  }
  render_ctx c = {cam, 1, spp, max_bounces, rr_start, seed, pixels, out_rgb, out_samples, out_sample_flags,
                  out_segments, NULL, out_sample_dev};
  job jb;
  memset(&jb, 0, sizeof(jb));
  jb.W.s = s;
  jb.W.n = sc->n;
  jb.W.prm = prm;
  jb.W.s_lod = sl;
  jb.W.n_lod = lod_sc->n;
  jb.W.lod_from = lod_from;
  jb.fn = render_item;
  jb.n_items = n_pix;
  jb.ctx = &c;
  int rc = run_job(&jb, n_threads);
  free(sl);
  free(s);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* adjoint of the single-bounce render                                       */
/* ------------------------------------------------------------------------ */

/* dL/d(q_raw) from dL/d(t_u, t_v, n) for the normalised-quaternion frame. */
static void quat_frame_adjoint(const double* q_raw, const double a[3], const double bb[3], const double c[3],
                               double dq[4]) {
  double qn = sqrt(q_raw[0] * q_raw[0] + q_raw[1] * q_raw[1] + q_raw[2] * q_raw[2] + q_raw[3] * q_raw[3]);
  double w = q_raw[0] / qn, x = q_raw[1] / qn, y = q_raw[2] / qn, z = q_raw[3] / qn;
  /* n is written as t_u x t_v in the forward pass; for a unit quaternion it
   * equals the third rotation column, whose partials are used here. */
  double gw = a[1] * 2 * z - a[2] * 2 * y - bb[0] * 2 * z + bb[2] * 2 * x + c[0] * 2 * y - c[1] * 2 * x;
  double gx = a[1] * 2 * y + a[2] * 2 * z + bb[0] * 2 * y - bb[1] * 4 * x + bb[2] * 2 * w + c[0] * 2 * z -
              c[1] * 2 * w - c[2] * 4 * x;
  double gy = -a[0] * 4 * y + a[1] * 2 * x - a[2] * 2 * w + bb[0] * 2 * x + bb[2] * 2 * z + c[0] * 2 * w +
              c[1] * 2 * z - c[2] * 4 * y;
  double gz = -a[0] * 4 * z + a[1] * 2 * w + a[2] * 2 * x - bb[0] * 2 * w - bb[1] * 4 * z + bb[2] * 2 * y +
              c[0] * 2 * x + c[1] * 2 * y;
  double qh[4] = {w, x, y, z}, g[4] = {gw, gx, gy, gz};
  double proj = qh[0] * g[0] + qh[1] * g[1] + qh[2] * g[2] + qh[3] * g[3];
  for (int k = 0; k < 4; ++k) dq[k] = (g[k] - qh[k] * proj) / qn;
}

/* gradient record of one surfel touched by a sample */
typedef struct {
  int64_t idx;
  double g[16];
} grad_entry;

typedef struct {
  grad_entry* e;
  int64_t n, cap;
} gradbuf;

static int gb_push(gradbuf* b, const grad_entry* x) {
  if (b->n == b->cap) {
    int64_t nc = b->cap ? 2 * b->cap : 1024;
    grad_entry* ne = (grad_entry*)realloc(b->e, sizeof(grad_entry) * (size_t)nc);
    if (!ne) return -1;
    b->e = ne;
    b->cap = nc;
  }
  b->e[b->n++] = *x;
  return 0;
}

/* Adjoint of one segment.  Inputs: the blended hits (in order) and the
 * segment, adjoints of the raw composites gN, gD, gR, gP, gA (E and the
 * emissive term carry none).  Accumulates surfel gradients into gb and
 * dL/dO, dL/dw of the ray. */
static int segment_adjoint(const world* W, const ora_scene* sc, const double O[3], const double w[3], int mode,
                           const hitbuf* b, const ora_segment* seg, const double gN[3], double gD,
                           const double gR[3], const double gP[3], double gA, gradbuf* gb, double dO[3],
                           double dw[3]) {
  const ora_params* prm = W->prm;
  const int64_t nh = b->n;
  if (nh == 0) return 0;
  const double Tn = 1.0 - seg->A;
  /* suffix sums S_i = sum_{j>i} w_j v_j, built back to front */
  double SN[3] = {0, 0, 0}, SD = 0, SR[3] = {0, 0, 0}, SP[3] = {0, 0, 0};
  /* transmittance before each hit */
  double* Tb = (double*)malloc(sizeof(double) * (size_t)nh);
  if (!Tb) return -1;
  double T = 1.0;
  for (int64_t k = 0; k < nh; ++k) {
    Tb[k] = T;
    T *= 1.0 - b->h[k].alpha;
  }
  for (int64_t k = nh - 1; k >= 0; --k) {
    const hit64* h = &b->h[k];
    const surfel64* g = &W->s[h->idx];
    const double a = h->alpha, Tp = Tb[k], wgt = Tp * a;
    const double sgn = h->d > 0 ? -1.0 : 1.0;
    const double remit = (mode == 1 && !(g->e > prm->tau_E)) ? 0.0 : 1.0;
    double vN[3] = {sgn * g->n[0], sgn * g->n[1], sgn * g->n[2]};
    double vR[3] = {remit * g->r[0], remit * g->r[1], remit * g->r[2]};
    /* dL/dalpha_i (Eq. 2): T_{i-1} v_i - S_i / (1 - alpha_i), and dA/dalpha_i */
    double da = gA * Tn / (1.0 - a);
    for (int c = 0; c < 3; ++c) {
      da += gN[c] * (Tp * vN[c] - SN[c] / (1.0 - a));
      da += gR[c] * (Tp * vR[c] - SR[c] / (1.0 - a));
      da += gP[c] * (Tp * g->rho[c] - SP[c] / (1.0 - a));
    }
    da += gD * (Tp * h->t - SD / (1.0 - a));
    /* update suffix sums to include hit k for the next (earlier) hit */
    for (int c = 0; c < 3; ++c) {
      SN[c] += wgt * vN[c];
      SR[c] += wgt * vR[c];
      SP[c] += wgt * g->rho[c];
    }
    SD += wgt * h->t;

    grad_entry ge;
    memset(&ge, 0, sizeof(ge));
    ge.idx = h->idx;
    /* albedo and radiance */
    for (int c = 0; c < 3; ++c) {
      ge.g[10 + c] = wgt * gP[c];
      ge.g[13 + c] = wgt * gR[c] * remit;
    }
    /* alpha = sigma * g (unclamped) */
    double dG = 0.0;
    if (!h->clamped) {
      ge.g[9] = da * h->g;
      dG = da * g->sigma;
    }
    double du = -dG * h->g * h->u;
    double dv = -dG * h->g * h->v;
    double Dx[3] = {O[0] - g->p[0] + h->t * w[0], O[1] - g->p[1] + h->t * w[1], O[2] - g->p[2] + h->t * w[2]};
    double dDx[3], dtu[3], dtv[3], dn[3];
    for (int c = 0; c < 3; ++c) {
      dDx[c] = du * g->tu[c] / g->su + dv * g->tv[c] / g->sv;
      dtu[c] = du * Dx[c] / g->su;
      dtv[c] = dv * Dx[c] / g->sv;
      dn[c] = wgt * gN[c] * sgn; /* from the facing normal */
    }
    ge.g[7] = -du * h->u / g->su;
    ge.g[8] = -dv * h->v / g->sv;
    double dt = wgt * gD + dot3(dDx, w);
    /* Dx = O - p + t w */
    for (int c = 0; c < 3; ++c) {
      dO[c] += dDx[c];
      ge.g[c] -= dDx[c];
      dw[c] += h->t * dDx[c];
    }
    /* t = ((p - O) . n) / (w . n) */
    double pO[3] = {g->p[0] - O[0], g->p[1] - O[1], g->p[2] - O[2]};
    for (int c = 0; c < 3; ++c) {
      ge.g[c] += dt * g->n[c] / h->d;
      dO[c] -= dt * g->n[c] / h->d;
      dn[c] += dt * (pO[c] - h->t * w[c]) / h->d;
      dw[c] -= dt * h->t * g->n[c] / h->d;
    }
    quat_frame_adjoint(&sc->quat[4 * h->idx], dtu, dtv, dn, &ge.g[3]);
    if (gb_push(gb, &ge)) {
      free(Tb);
      return -1;
    }
  }
  free(Tb);
  return 0;
}

/* dL/dn of w' = l0 b1(n) + l1 b2(n) + l2 n (Duff basis, branch held fixed) */
static void cosine_direction_adjoint(const double n[3], const double l[3], const double dw[3], double dn[3]) {
  double sgn = copysign(1.0, n[2]);
  double a = -1.0 / (sgn + n[2]);
  double a2 = a * a;
  /* Jacobians of b1 and b2 (rows: components; cols: n_x, n_y, n_z) */
  double J1[3][3] = {{2 * sgn * n[0] * a, 0, sgn * n[0] * n[0] * a2},
                     {sgn * n[1] * a, sgn * n[0] * a, sgn * n[0] * n[1] * a2},
                     {-sgn, 0, 0}};
  double J2[3][3] = {{n[1] * a, n[0] * a, n[0] * n[1] * a2}, {0, 2 * n[1] * a, n[1] * n[1] * a2}, {0, -1, 0}};
  for (int c = 0; c < 3; ++c) {
    dn[c] = l[2] * dw[c];
    for (int r = 0; r < 3; ++r) dn[c] += l[0] * J1[r][c] * dw[r] + l[1] * J2[r][c] * dw[r];
  }
}

typedef struct {
  const ora_scene* sc;
  const ora_camera* cam;
  int32_t spp;
  uint64_t seed;
  const int32_t* pixels;
  const double* dL;
  uint32_t* out_flags;
  gradbuf* per_thread;
  int32_t n_threads;
  int32_t radiance_only; /* 0-bounce render: I = R_1 for every pixel */
  int32_t run;           /* > 0: a conditioning run (rays and sigma g perturbed at FP32 scale, as in ora_render) */
} grad_ctx;

static int grad_pixel(const world* W, grad_ctx* c, int64_t i, hitbuf* b1, hitbuf* b2, gradbuf* gb) {
  const ora_params* prm = W->prm;
  const int64_t pix = c->pixels[i];
  const double* gI = &c->dL[3 * i];
  double O[3], w[3];
  primary_ray(c->cam, pix, O, w);
  if (c->run > 0) {
    double Oj[3] = {O[0], O[1], O[2]};
    jitter_ray(Oj, w, c->seed, pix, -1, 0, c->run, 2.0 * prm->fp32_eps);
  }
  ora_segment g1;
  if (segment(W, O, w, 0.0, 0, 0.0, ERR_C * prm->fp32_eps, b1, &g1)) return -1;
  uint32_t flags = g1.flags;
  double zero3[3] = {0, 0, 0};
  double dO[3] = {0, 0, 0}, dw[3] = {0, 0, 0};
  if (g1.n_hits == 0) {
    if (c->out_flags) c->out_flags[i] = flags;
    return 0;
  }
  if (c->radiance_only || g1.E > prm->tau_E) {
    /* 0-bounce render, or emitter pixel: I = R_1 */
    int rc = segment_adjoint(W, c->sc, O, w, 0, b1, &g1, zero3, 0.0, gI, zero3, 0.0, gb, dO, dw);
    if (c->out_flags) c->out_flags[i] = flags;
    return rc;
  }
  const double invS = 1.0 / c->spp;
  double gP1[3] = {0, 0, 0}, gNn1[3] = {0, 0, 0}, gDn1 = 0.0;
  double X[3];
  for (int k = 0; k < 3; ++k) X[k] = O[k] + g1.Dn * w[k];
  for (int32_t s = 0; s < c->spp; ++s) {
    double u[4], l[3], w2[3], O2[3];
    draws(c->seed, pix, s, 1, u);
    const double eps = prm->fp32_eps;
    if (eps > 0 && fabs(g1.Nn[2]) <= FLAG_K * g1.eN) flags |= ORA_FLAG_ONB;
    cosine_local(u[0], u[1], l);
    ora_cosine_direction(g1.Nn, u[0], u[1], w2);
    for (int k = 0; k < 3; ++k) O2[k] = X[k] + prm->bounce_offset * g1.Nn[k];
    if (c->run > 0) jitter_ray(O2, w2, c->seed, pix, s, 1, c->run, 2.0 * eps);
    const double eO2 = ERR_C * eps * amax3(O2);
    ora_segment g2;
    if (segment(W, O2, w2, 0.0, 0, eO2, ERR_C * eps, b2, &g2)) return -1;
    flags |= g2.flags;
    if (g2.n_hits == 0) continue;
    double gR2[3];
    for (int k = 0; k < 3; ++k) {
      gP1[k] += invS * gI[k] * g2.R[k];
      gR2[k] = invS * gI[k] * g1.P[k];
    }
    double dO2[3] = {0, 0, 0}, dw2[3] = {0, 0, 0};
    if (segment_adjoint(W, c->sc, O2, w2, 0, b2, &g2, zero3, 0.0, gR2, zero3, 0.0, gb, dO2, dw2)) return -1;
    /* O2 = O + Dn1 w + eps Nn1 ; w2 = basis(Nn1) l */
    gDn1 += dot3(dO2, w);
    double dn[3];
    cosine_direction_adjoint(g1.Nn, l, dw2, dn);
    for (int k = 0; k < 3; ++k) gNn1[k] += prm->bounce_offset * dO2[k] + dn[k];
  }
  /* normalisations: Nn = N/|N|, Dn = D/A */
  double nn = norm3(g1.N);
  double proj = dot3(g1.Nn, gNn1);
  double gN1[3];
  for (int k = 0; k < 3; ++k) gN1[k] = (gNn1[k] - g1.Nn[k] * proj) / nn;
  double gD1 = gDn1 / g1.A;
  double gA1 = -gDn1 * g1.D / (g1.A * g1.A);
  if (segment_adjoint(W, c->sc, O, w, 0, b1, &g1, gN1, gD1, zero3, gP1, gA1, gb, dO, dw)) return -1;
  if (c->out_flags) c->out_flags[i] = flags;
  return 0;
}

typedef struct {
  const world* W;
  grad_ctx* c;
  int64_t n_pix;
  int32_t tid;
  int err;
} gthread;

static void* gworker(void* arg) {
  gthread* t = (gthread*)arg;
  hitbuf b1 = {0, 0, 0}, b2 = {0, 0, 0};
  for (int64_t i = t->tid; i < t->n_pix; i += t->c->n_threads)
    if (grad_pixel(t->W, t->c, i, &b1, &b2, &t->c->per_thread[t->tid])) t->err = 1;
  free(b1.h);
  free(b2.h);
  return NULL;
}

static int grad_common(const ora_scene* sc, const ora_camera* cam, const ora_params* prm, int32_t spp,
                       uint64_t seed, const int32_t* pixels, int64_t n_pix, const double* dL_drgb, double* grad,
                       uint32_t* out_flags, int32_t n_threads, int32_t radiance_only, int32_t run);

int ora_single_bounce_grad(const ora_scene* sc, const ora_camera* cam, const ora_params* prm, int32_t spp,
                           uint64_t seed, const int32_t* pixels, int64_t n_pix, const double* dL_drgb,
                           double* grad, uint32_t* out_flags, int32_t n_threads, int32_t run) {
  return grad_common(sc, cam, prm, spp, seed, pixels, n_pix, dL_drgb, grad, out_flags, n_threads, 0, run);
}

int ora_radiance_grad(const ora_scene* sc, const ora_camera* cam, const ora_params* prm, const int32_t* pixels,
                      int64_t n_pix, const double* dL_drgb, double* grad, uint32_t* out_flags, int32_t n_threads,
                      int32_t run) {
  return grad_common(sc, cam, prm, 1, 0, pixels, n_pix, dL_drgb, grad, out_flags, n_threads, 1, run);
}

static int grad_common(const ora_scene* sc, const ora_camera* cam, const ora_params* prm, int32_t spp,
                       uint64_t seed, const int32_t* pixels, int64_t n_pix, const double* dL_drgb, double* grad,
                       uint32_t* out_flags, int32_t n_threads, int32_t radiance_only, int32_t run) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  surfel64* s = load_surfels(sc);
  if (!s) return -1;
  world W = {s, sc->n, prm, (uint32_t)(run > 0 ? run : 0)};
  gradbuf* per = (gradbuf*)calloc((size_t)n_threads, sizeof(gradbuf));
  gthread* th = (gthread*)calloc((size_t)n_threads, sizeof(gthread));
  pthread_t* pt = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!per || !th || !pt) {
    free(s);
    free(per);
    free(th);
    free(pt);
    return -1;
  }
  grad_ctx c = {sc, cam, spp, seed, pixels, dL_drgb, out_flags, per, n_threads, radiance_only, run};
  int started = 0;
  for (int t = 0; t < n_threads; ++t) {
    th[t].W = &W;
    th[t].c = &c;
    th[t].n_pix = n_pix;
    th[t].tid = t;
    th[t].err = 0;
  }
  for (int t = 1; t < n_threads; ++t) {
    if (pthread_create(&pt[t], NULL, gworker, &th[t]) != 0) break;
    started = t;
  }
  /* threads that failed to start: do their share here */
  gworker(&th[0]);
  for (int t = started + 1; t < n_threads; ++t) gworker(&th[t]);
  for (int t = 1; t <= started; ++t) pthread_join(pt[t], NULL);
  int err = 0;
  for (int t = 0; t < n_threads; ++t) {
    err |= th[t].err;
    for (int64_t k = 0; k < per[t].n; ++k) {
      const grad_entry* e = &per[t].e[k];
      for (int j = 0; j < 16; ++j) grad[16 * e->idx + j] += e->g[j];
    }
    free(per[t].e);
  }
  free(per);
  free(th);
  free(pt);
  free(s);
  return err ? -1 : 0;
}
