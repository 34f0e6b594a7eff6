/*
 * FP64 CPU oracle for the mixture-of-media random walk.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * What it computes (paper, Sec. 4.1):
 *   - the BSSRDF as a path integral over paths whose contribution is the
 *     product of boundary terms, transmittances T and albedo-scaled phase
 *     functions alpha*sigma_t*pf (the display defining f_SSS after Eq. 2);
 *   - its radial form under normal incidence, R_d(r) = R * P_d(r) (Eq. 3);
 *   - the K-media mixture S = sum_k w_k S_k with sum_k w_k = 1 (Eq. 4),
 *     estimated by picking ONE medium per path, with probability w_k, before
 *     the walk starts (Sec. 4.1 last paragraph, Sec. 6 "each photon randomly
 *     selects a medium", Sec. 7 "select the medium ... adjust the pdf").
 *
 * The estimator is the textbook analog / weighted random walk, written step
 * by step in double precision:
 *   select medium -> enter (weight 1-R0) -> loop { exponential flight with
 *   sigma_t; if the flight reaches a face, smooth-dielectric Fresnel
 *   reflect-or-exit; otherwise a collision: albedo weighting with Russian
 *   roulette (or analog absorption), Henyey-Greenstein scattering with g }
 *   -> tally the exit weight into R, the radial histogram, R_k, R1, T.
 *
 * Random numbers: both this oracle and the CUDA path implement ONE
 * counter-based generator, Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11), from its published
 * definition, with the same counter layout:
 *     key     = (seed_lo, seed_hi)
 *     counter = (step, path, instance, tag)   tag 0 = walk step, 1 = selection
 * and the same 23-bit uniform u = ((x >> 9) + 0.5) * 2^-23 in (0,1), which
 * is exact in binary32 as well as binary64 (a 24-bit version would round
 * to 1.0 in binary32 at the top of its range).
 * Everything else (flights, Fresnel, HG, rotation, weights, tallies) is
 * double precision here, so GPU-vs-oracle differences come only from the
 * kernel's binary32 rounding.  The one integer decision that floating point
 * takes before any other (which medium a path uses) is taken in binary32,
 * the kernel's precision, on both sides.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_KMAX 4
#define ORC_NBINS_MAX 4096
#define ORC_NV_MAX (ORC_NBINS_MAX + 1 + ORC_KMAX + 5)
#define ORC_CHUNK 1024

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): 10 rounds of the 4x32 S-box with a Weyl key bump. */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u; /* round multipliers */
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u; /* key schedule (golden ratio) */
static const uint32_t PHILOX_W1 = 0xBB67AE85u; /* key schedule (sqrt(3)-1) */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 23-bit uniform strictly inside (0,1): never 0 (so -ln u is finite), never 1. */
static double u23(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

static void draw4(uint64_t seed, uint32_t step, uint32_t path, uint32_t inst,
                  uint32_t tag, double u[4]) {
  uint32_t ctr[4] = {step, path, inst, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  oracle_philox4x32_10(ctr, key, x);
  for (int i = 0; i < 4; ++i) u[i] = u23(x[i]);
}

/* ------------------------------------------------------------------------ */
/* Physics helpers (exported so the tests can check them one by one).        */
/* ------------------------------------------------------------------------ */

/* Unpolarised Fresnel reflectance of a smooth dielectric interface, light
 * going from the medium (index n) to the outside (index 1), incidence cosine
 * cos_i.  Total internal reflection when n*sin_i >= 1.  (Sec. 8: smooth
 * Fresnel boundary.) */
double oracle_fresnel(double cos_i, double n) {
  if (n == 1.0) return 0.0;
  if (cos_i > 1.0) cos_i = 1.0;
  double sin_i = sqrt(fmax(0.0, 1.0 - cos_i * cos_i));
  double sin_t = n * sin_i;
  if (sin_t >= 1.0) return 1.0;
  double cos_t = sqrt(1.0 - sin_t * sin_t);
  double rs = (n * cos_i - cos_t) / (n * cos_i + cos_t);
  double rp = (cos_i - n * cos_t) / (cos_i + n * cos_t);
  return 0.5 * (rs * rs + rp * rp);
}

/* Henyey-Greenstein cosine by inversion of its CDF (isotropic at g = 0). */
double oracle_hg_mu(double g, double u) {
  double mu;
  if (g == 0.0) {
    mu = 2.0 * u - 1.0;
  } else {
    double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
    mu = (1.0 + g * g - t * t) / (2.0 * g);
  }
  if (mu > 1.0) mu = 1.0;
  if (mu < -1.0) mu = -1.0;
  return mu;
}

/* d/dg log p_HG(mu; g), p_HG(mu) = (1-g^2) / (2 (1+g^2-2 g mu)^{3/2}). */
double oracle_hg_dlogp_dg(double g, double mu) {
  return -2.0 * g / (1.0 - g * g) - 3.0 * (g - mu) / (1.0 + g * g - 2.0 * g * mu);
}

/* Rotate direction u by polar cosine mu and azimuth phi (spherical frame
 * about the current direction; special case when u is nearly along z). */
void oracle_rotate(double u[3], double mu, double phi) {
  double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  double cp = cos(phi), sp = sin(phi);
  double ux = u[0], uy = u[1], uz = u[2];
  double nx, ny, nz;
  if (fabs(uz) > 1.0 - 1e-6) {
    nx = st * cp;
    ny = st * sp;
    nz = (uz >= 0.0 ? 1.0 : -1.0) * mu;
  } else {
    double tmp = sqrt(1.0 - uz * uz);
    nx = st * (ux * uz * cp - uy * sp) / tmp + ux * mu;
    ny = st * (uy * uz * cp + ux * sp) / tmp + uy * mu;
    nz = -st * cp * tmp + uz * mu;
  }
  double nrm = sqrt(nx * nx + ny * ny + nz * nz);
  u[0] = nx / nrm; u[1] = ny / nrm; u[2] = nz / nrm;
}

/* Medium choice with probability w_k / sum(w): the first k whose running
 * CDF exceeds u, the last medium taking any round-off remainder.  Taken in
 * binary32 (the kernel's precision) so both sides make the same choice. */
int oracle_select_medium(const float* w, int K, double u) {
  float total = 0.0f;
  for (int k = 0; k < K; ++k) total += w[k];
  float inv = 1.0f / total;
  float us = (float)u;
  float cdf = 0.0f;
  for (int k = 0; k < K - 1; ++k) {
    cdf += w[k] * inv;
    if (us < cdf) return k;
  }
  return K - 1;
}

/* ------------------------------------------------------------------------ */
/* One path.                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int nbins;
  double r_max_mm;
  int mode;            /* 0 = albedo weighting + Russian roulette, 1 = analog */
  double rr_threshold; /* W_th; 0 disables roulette (weight mode only) */
  int entry_fresnel;   /* 1: entry weight 1 - F (specular excluded) */
  uint32_t max_steps;
  uint64_t seed;
  int incidence;       /* 0 = normal, 1 = cosine-weighted lobe */
  double log_r_min_mm; /* 0: linear bins; > 0: bin 0 = [0, r_min), then
                          logarithmic edges r_min q^(b-1), q = (r_max/r_min)^(1/(nbins-1)) */
  int select_pdf;      /* 0: medium k with probability w_k / sum(w) (Sec. 7);
                          1: uniformly, with path weight K w_k / sum(w) */
} oracle_opts;

/* Optional second layer under the chosen medium (two-layer slab, Sec. 3):
 * the chosen medium fills 0 <= z < d1, this layer fills d1 <= z < thickness
 * (semi-infinite when the thickness is +inf).  Arrays are [n_inst]. */
typedef struct {
  const float *alpha2, *sigma_t2, *g2, *d1;
} oracle_layer2;

typedef struct {
  int exit_kind;    /* 0 top, 1 bottom, 2 absorbed/roulette, 3 truncated */
  int medium;
  int bin;          /* top exits: bin index, nbins = overflow */
  double weight;    /* exit weight (0 unless exit_kind is 0 or 1) */
  double absorbed;  /* weight deposited by collisions */
  uint32_t steps;   /* random-number draws used by the loop */
  uint32_t n_coll;  /* collisions (scattering or absorption events) */
  double length;    /* total distance travelled inside the medium, mm */
  double dlogp_dg;  /* sum over scatterings of d log p_HG / dg */
  double x, y;      /* exit point on the face */
  /* the parts of n_coll, length and dlogp_dg spent in the second layer of a
   * two-layer slab (0 otherwise) */
  uint32_t n_coll2;
  double length2, dlogp_dg2;
} oracle_path;

/* inst indexes the parameter arrays; rng_inst is the instance number the
 * random-number counters use (the same unless a subset of a larger batch is
 * being re-walked). */
void oracle_trace_path_layered(const float* alpha, const float* sigma_t, const float* g,
                               const float* w, int K, int64_t n_inst, int64_t inst,
                               uint32_t rng_inst, uint32_t path, double thickness_mm,
                               double n_rel, const oracle_opts* o, const oracle_layer2* l2,
                               oracle_path* res) {
  double u[4];
  memset(res, 0, sizeof(*res));
  /* Medium selection once per path, before the walk (Eq. 4, Sec. 7). */
  float wk[ORC_KMAX];
  for (int k = 0; k < K; ++k) wk[k] = w[(int64_t)k * n_inst + inst];
  draw4(o->seed, 0u, path, rng_inst, 1u, u);
  int k;
  double w_sel = 1.0; /* w_k / (p_k sum(w)): the estimator weight of the choice */
  if (o->select_pdf == 1) {
    /* another selection pdf (Sec. 7 samples by w_k and leaves others
     * open): uniform over the K media, reweighted so that the mixture
     * of Eq. 4 is still estimated without bias */
    k = (int)floor(u[0] * (double)K);
    if (k > K - 1) k = K - 1;
    double tot = 0.0;
    for (int j = 0; j < K; ++j) tot += (double)wk[j];
    w_sel = (double)K * (double)wk[k] / tot;
  } else {
    k = oracle_select_medium(wk, K, u[0]);
  }
  res->medium = k;
  double a = alpha[(int64_t)k * n_inst + inst];
  double st = sigma_t[(int64_t)k * n_inst + inst];
  double gg = g[(int64_t)k * n_inst + inst];
  /* optics of the other layer, swapped in when the path crosses z = d1 */
  double a_o = 0.0, st_o = 1.0, g_o = 0.0, d1 = INFINITY;
  if (l2) {
    a_o = l2->alpha2[inst];
    st_o = l2->sigma_t2[inst];
    g_o = l2->g2[inst];
    d1 = l2->d1[inst];
  }
  int layer = 0;

  /* Entry at the origin.  Normal incidence (Eq. 3), or a cosine-weighted
   * incident lobe (the fitting assumption of Sec. 8): outside cosine
   * sqrt(u), azimuth 2 pi u', refracted into the medium by Snell's law.
   * The weight after the entry BTDF is 1 - F at the refracted angle (the
   * reflectance is the same from either side). */
  double pos[3] = {0.0, 0.0, 0.0};
  double dir[3] = {0.0, 0.0, 1.0};
  if (o->incidence == 1) {
    double v[4];
    draw4(o->seed, 0u, path, rng_inst, 2u, v);
    const double mu_o = sqrt(v[0]);
    const double sin_o = sqrt(fmax(0.0, 1.0 - mu_o * mu_o));
    const double sin_i = sin_o / n_rel;
    const double phi = 2.0 * M_PI * v[1];
    dir[0] = sin_i * cos(phi);
    dir[1] = sin_i * sin(phi);
    dir[2] = sqrt(1.0 - sin_i * sin_i);
  }
  double W = (o->entry_fresnel ? 1.0 - oracle_fresnel(dir[2], n_rel) : 1.0) * w_sel;
  double d = thickness_mm; /* +inf: semi-infinite */

  uint32_t step = 0;
  for (;;) {
    if (step >= o->max_steps) { res->exit_kind = 3; break; }
    draw4(o->seed, step, path, rng_inst, 0u, u);
    step++;
    double s = -log(u[0]) / st; /* exponential free flight (transmittance T) */
    /* the planes bounding the current layer */
    const double ztop = layer == 0 ? 0.0 : d1;
    const double zbot = (l2 && layer == 0) ? d1 : d;
    double db = INFINITY;
    if (dir[2] < 0.0) db = (ztop - pos[2]) / dir[2];
    else if (dir[2] > 0.0) db = (zbot - pos[2]) / dir[2];
    if (db <= s) {
      pos[0] += db * dir[0];
      pos[1] += db * dir[1];
      int top = dir[2] < 0.0;
      res->length += db;
      if (layer == 1) res->length2 += db;
      if (l2 && ((top && layer == 1) || (!top && layer == 0))) {
        /* Internal interface (index matched): cross into the other layer
         * and draw a fresh flight there (flights are memoryless). */
        pos[2] = d1;
        layer ^= 1;
        double t;
        t = a; a = a_o; a_o = t;
        t = st; st = st_o; st_o = t;
        t = gg; gg = g_o; g_o = t;
        continue;
      }
      /* Reaches an outer face: move there, then smooth-dielectric Fresnel. */
      pos[2] = top ? 0.0 : d;
      double F = oracle_fresnel(fabs(dir[2]), n_rel);
      if (u[1] < F) { dir[2] = -dir[2]; continue; }
      res->exit_kind = top ? 0 : 1;
      res->weight = W;
      res->x = pos[0];
      res->y = pos[1];
      if (top) {
        double r = sqrt(pos[0] * pos[0] + pos[1] * pos[1]);
        double fb;
        if (o->log_r_min_mm > 0.0) {
          fb = r < o->log_r_min_mm
                   ? 0.0
                   : 1.0 + floor(log(r / o->log_r_min_mm) /
                                 (log(o->r_max_mm / o->log_r_min_mm) / (o->nbins - 1)));
        } else {
          fb = floor(r * (double)o->nbins / o->r_max_mm);
        }
        res->bin = fb >= (double)o->nbins ? o->nbins : (int)fb;
      }
      break;
    }
    /* Collision inside the medium. */
    for (int i = 0; i < 3; ++i) pos[i] += s * dir[i];
    res->length += s;
    res->n_coll++;
    if (layer == 1) {
      res->length2 += s;
      res->n_coll2++;
    }
    if (o->mode == 0) {
      res->absorbed += W * (1.0 - a);
      W *= a;
      if (W < o->rr_threshold) {
        if (u[3] < W / o->rr_threshold) W = o->rr_threshold;
        else { res->exit_kind = 2; break; }
      }
    } else {
      if (u[3] >= a) { res->absorbed += W; res->exit_kind = 2; break; }
    }
    double mu = oracle_hg_mu(gg, u[1]);
    const double dl = oracle_hg_dlogp_dg(gg, mu);
    res->dlogp_dg += dl;
    if (layer == 1) res->dlogp_dg2 += dl;
    oracle_rotate(dir, mu, 2.0 * M_PI * u[2]);
  }
  res->steps = step;
}

void oracle_trace_path(const float* alpha, const float* sigma_t, const float* g,
                       const float* w, int K, int64_t n_inst, int64_t inst,
                       uint32_t rng_inst, uint32_t path, double thickness_mm, double n_rel,
                       const oracle_opts* o, oracle_path* res) {
  oracle_trace_path_layered(alpha, sigma_t, g, w, K, n_inst, inst, rng_inst, path,
                            thickness_mm, n_rel, o, NULL, res);
}

/* ------------------------------------------------------------------------ */
/* Batched forward tallies.                                                   */
/* ------------------------------------------------------------------------ */
/* Outputs, all per instance, NULL allowed for any of them:
 *   R, T, A, overflow, R1, truncated : [n_inst]
 *   bins : [n_inst][nbins]      R_k : [n_inst][K]
 *   se_R, se_T, se_A, se_R1 : [n_inst]   se_bins : [n_inst][nbins]
 *   se_R_k : [n_inst][K]
 * Each tally is the mean over the instance's N paths of the per-path
 * contribution (a fraction of the incident power); se_* is the sample
 * standard error of that mean.  inst_ids (or NULL) gives the instance number
 * each array column had in the batch it was drawn from, for the counters. */
typedef struct {
  double *R, *T, *A, *bins, *overflow, *R_k, *R1, *truncated;
  double *se_R, *se_T, *se_A, *se_bins, *se_R_k, *se_R1;
  double *steps; /* mean random-number draws per path */
} oracle_out;

static double se_of(double s, double s2, double n) {
  if (n < 2.0) return 0.0;
  double m = s / n;
  double v = (s2 / n - m * m) * n / (n - 1.0);
  return v > 0.0 ? sqrt(v / n) : 0.0;
}

int oracle_walk(int64_t n_inst, int K, const float* alpha, const float* sigma_t,
                const float* g, const float* w, const uint32_t* n_paths,
                const float* thickness_mm, double n_rel, const oracle_opts* o,
                uint32_t path_offset, const int64_t* inst_ids, const oracle_layer2* l2,
                oracle_out* out) {
  if (K < 1 || K > ORC_KMAX || o->nbins < 1 || o->nbins > ORC_NBINS_MAX) return 1;
  const int nb = o->nbins;
  /* per-path vector: [bins nb][overflow][R_k K][R1][T][A][trunc][steps] */
  const int nv = nb + 1 + K + 5;
  for (int64_t i = 0; i < n_inst; ++i) {
    const uint32_t N = n_paths[i];
    const double d = thickness_mm ? (double)thickness_mm[i] : INFINITY;
    /* Fixed chunks of paths, each summed in path order, then the chunks in
     * chunk order: the result does not depend on the thread count. */
    const int64_t nch = ((int64_t)N + ORC_CHUNK - 1) / ORC_CHUNK;
    double* ps = calloc((size_t)(nch > 0 ? nch : 1) * 2 * (size_t)nv, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nch; ++ch) {
      double* ls = ps + (size_t)ch * 2 * (size_t)nv;
      double* ls2 = ls + nv;
      double c[ORC_NV_MAX];
      const int64_t p1 = (ch + 1) * ORC_CHUNK < (int64_t)N ? (ch + 1) * ORC_CHUNK : (int64_t)N;
      for (int64_t p = ch * ORC_CHUNK; p < p1; ++p) {
        oracle_path r;
        oracle_trace_path_layered(alpha, sigma_t, g, w, K, n_inst, i,
                                  inst_ids ? (uint32_t)inst_ids[i] : (uint32_t)i,
                                  path_offset + (uint32_t)p, d, n_rel, o, l2, &r);
        memset(c, 0, sizeof(double) * (size_t)nv);
        if (r.exit_kind == 0) {
          c[r.bin] = r.weight; /* bin or overflow slot */
          c[nb + 1 + r.medium] = r.weight;
          if (r.n_coll == 1) c[nb + 1 + K] = r.weight;
        } else if (r.exit_kind == 1) {
          c[nb + 1 + K + 1] = r.weight;
        } else if (r.exit_kind == 3) {
          c[nb + 1 + K + 3] = 1.0;
        }
        c[nb + 1 + K + 2] = r.absorbed;
        c[nb + 1 + K + 4] = (double)r.steps;
        for (int j = 0; j < nv; ++j) { ls[j] += c[j]; ls2[j] += c[j] * c[j]; }
      }
    }
    double* s = calloc((size_t)nv, sizeof(double));
    double* s2 = calloc((size_t)nv, sizeof(double));
    for (int64_t ch = 0; ch < nch; ++ch)
      for (int j = 0; j < nv; ++j) {
        s[j] += ps[(size_t)ch * 2 * (size_t)nv + (size_t)j];
        s2[j] += ps[(size_t)ch * 2 * (size_t)nv + (size_t)nv + (size_t)j];
      }
    free(ps);
    const double n = (double)N;
    double sR = 0.0, s2R = 0.0;
    for (int b = 0; b <= nb; ++b) { sR += s[b]; s2R += s2[b]; }
    /* a path exits through at most one slot, so sum of squares adds up */
    if (out->R) out->R[i] = sR / n;
    if (out->se_R) out->se_R[i] = se_of(sR, s2R, n);
    for (int b = 0; b < nb; ++b) {
      if (out->bins) out->bins[i * nb + b] = s[b] / n;
      if (out->se_bins) out->se_bins[i * nb + b] = se_of(s[b], s2[b], n);
    }
    if (out->overflow) out->overflow[i] = s[nb] / n;
    for (int k = 0; k < K; ++k) {
      if (out->R_k) out->R_k[i * K + k] = s[nb + 1 + k] / n;
      if (out->se_R_k) out->se_R_k[i * K + k] = se_of(s[nb + 1 + k], s2[nb + 1 + k], n);
    }
    const int o1 = nb + 1 + K;
    if (out->R1) out->R1[i] = s[o1] / n;
    if (out->se_R1) out->se_R1[i] = se_of(s[o1], s2[o1], n);
    if (out->T) out->T[i] = s[o1 + 1] / n;
    if (out->se_T) out->se_T[i] = se_of(s[o1 + 1], s2[o1 + 1], n);
    if (out->A) out->A[i] = s[o1 + 2] / n;
    if (out->se_A) out->se_A[i] = se_of(s[o1 + 2], s2[o1 + 2], n);
    if (out->truncated) out->truncated[i] = s[o1 + 3];
    if (out->steps) out->steps[i] = s[o1 + 4] / n;
    free(s); free(s2);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Hero-wavelength walk: one path geometry shared by C bands of a texel.      */
/* ------------------------------------------------------------------------ */
/* Hero-wavelength spectral sampling (Wilkie et al., EGSR 2014; the paper's
 * related work names hero-wavelength tracking), applied to the mixture walk.
 * Instances are texels x nb bands, band fastest.  With C dividing nb, the
 * bands of a texel fall into nb/C groups whose members share path
 * geometries: blocks of C adjacent bands, or (orbits = 1) Wilkie et al.'s
 * rotation orbits {o, o + nb/C, ..., o + (C-1) nb/C}.  The estimate is
 * unbiased for any partition, since given its group a path's hero is
 * uniform over the members; adjacent bands have close optics, so their
 * balance weights stay near 1/C and the variance near that of separate
 * walks.  Path p of a
 * group samples everything (medium choice, flights, Henyey-Greenstein
 * cosines, roulette) with the optics of its hero member h = p mod C, so each
 * member is the hero of N/C of the paths.  Member j then scores the
 * one-sample balance-heuristic estimate
 *     F_j = f_j(x) / ((1/C) sum_i p_i(x)) = W_j C / sum_i exp(L_i - L_j),
 * where p_i is the density of the path's sampling decisions under member i's
 * optics (selection probability of the chosen medium, exp(-sigma s) and
 * sigma per collision, p_HG(mu) per scattering; Fresnel choices are the same
 * for every member and cancel), L_i = log p_i, and W_j = f_j / p_j is the
 * member's albedo-weighted throughput (entry weight, w_k / selection
 * probability, alpha_j per collision, and the roulette boosts, shared by the
 * members and decided on their largest weight).  Weight mode only;
 * absorption (A) is not scored.  Counters: (step, path, first member + offset, tag). */
static double hg_logpdf(double g, double mu) {
  /* density of mu = cos(theta) on [-1, 1] */
  return log(0.5 * (1.0 - g * g)) - 1.5 * log(1.0 + g * g - 2.0 * g * mu);
}

typedef struct {
  int exit_kind;          /* 0 top, 1 bottom, 2 roulette, 3 truncated */
  int medium, bin;
  uint32_t steps, n_coll;
  double F[ORC_KMAX];     /* per member: the balance-heuristic exit weight */
} oracle_hero_path;

static void trace_hero(const float* alpha, const float* sigma_t, const float* g, const float* w,
                       int K, int64_t n_inst, const int64_t* mem, int C, int h,
                       uint32_t rng_inst, uint32_t path, double d, double n_rel,
                       const oracle_opts* o, oracle_hero_path* res) {
  double u[4];
  memset(res, 0, sizeof(*res));
  float wk[ORC_KMAX];
  for (int k = 0; k < K; ++k) wk[k] = w[(int64_t)k * n_inst + mem[h]];
  draw4(o->seed, 0u, path, rng_inst, 1u, u);
  int k;
  if (o->select_pdf == 1) {
    k = (int)floor(u[0] * (double)K);
    if (k > K - 1) k = K - 1;
  } else {
    k = oracle_select_medium(wk, K, u[0]);
  }
  res->medium = k;
  double a[ORC_KMAX], st[ORC_KMAX], gg[ORC_KMAX], L[ORC_KMAX], W[ORC_KMAX];
  for (int i = 0; i < C; ++i) {
    a[i] = alpha[(int64_t)k * n_inst + mem[i]];
    st[i] = sigma_t[(int64_t)k * n_inst + mem[i]];
    gg[i] = g[(int64_t)k * n_inst + mem[i]];
    double tot = 0.0;
    for (int j = 0; j < K; ++j) tot += (double)w[(int64_t)j * n_inst + mem[i]];
    const double mix = (double)w[(int64_t)k * n_inst + mem[i]] / tot; /* Eq. 4 weight */
    const double sel = o->select_pdf == 1 ? 1.0 / (double)K : mix; /* its choice prob. */
    L[i] = log(sel);
    W[i] = mix / sel;
  }
  double pos[3] = {0.0, 0.0, 0.0};
  double dir[3] = {0.0, 0.0, 1.0};
  if (o->incidence == 1) {
    double v[4];
    draw4(o->seed, 0u, path, rng_inst, 2u, v);
    const double mu_o = sqrt(v[0]);
    const double sin_i = sqrt(fmax(0.0, 1.0 - mu_o * mu_o)) / n_rel;
    const double phi = 2.0 * M_PI * v[1];
    dir[0] = sin_i * cos(phi);
    dir[1] = sin_i * sin(phi);
    dir[2] = sqrt(1.0 - sin_i * sin_i);
  }
  const double W0 = o->entry_fresnel ? 1.0 - oracle_fresnel(dir[2], n_rel) : 1.0;
  for (int i = 0; i < C; ++i) W[i] *= W0;

  uint32_t step = 0;
  for (;;) {
    if (step >= o->max_steps) { res->exit_kind = 3; break; }
    draw4(o->seed, step, path, rng_inst, 0u, u);
    step++;
    const double s = -log(u[0]) / st[h];
    double db = INFINITY;
    if (dir[2] < 0.0) db = -pos[2] / dir[2];
    else if (dir[2] > 0.0) db = (d - pos[2]) / dir[2];
    if (db <= s) {
      /* no collision over db: probability exp(-sigma db) under each member */
      for (int i = 0; i < C; ++i) L[i] += -st[i] * db;
      pos[0] += db * dir[0];
      pos[1] += db * dir[1];
      const int top = dir[2] < 0.0;
      pos[2] = top ? 0.0 : d;
      const double F = oracle_fresnel(fabs(dir[2]), n_rel);
      if (u[1] < F) { dir[2] = -dir[2]; continue; }
      res->exit_kind = top ? 0 : 1;
      if (top) {
        const double r = sqrt(pos[0] * pos[0] + pos[1] * pos[1]);
        double fb;
        if (o->log_r_min_mm > 0.0) {
          fb = r < o->log_r_min_mm
                   ? 0.0
                   : 1.0 + floor(log(r / o->log_r_min_mm) /
                                 (log(o->r_max_mm / o->log_r_min_mm) / (o->nbins - 1)));
        } else {
          fb = floor(r * (double)o->nbins / o->r_max_mm);
        }
        res->bin = fb >= (double)o->nbins ? o->nbins : (int)fb;
      }
      for (int j = 0; j < C; ++j) {
        double den = 0.0;
        for (int i = 0; i < C; ++i) den += exp(L[i] - L[j]);
        res->F[j] = W[j] * (double)C / den;
      }
      break;
    }
    /* collision after s: density sigma exp(-sigma s) under each member */
    for (int i = 0; i < C; ++i) L[i] += log(st[i]) - st[i] * s;
    for (int i = 0; i < 3; ++i) pos[i] += s * dir[i];
    res->n_coll++;
    for (int i = 0; i < C; ++i) W[i] *= a[i];
    /* roulette on the largest member weight Wr (survival probability > 0
     * whenever any member still carries weight); survivors of every member
     * are boosted by the same factor rr / Wr */
    double Wr = 0.0;
    for (int i = 0; i < C; ++i) Wr = fmax(Wr, W[i]);
    if (Wr < o->rr_threshold) {
      if (u[3] < Wr / o->rr_threshold) {
        const double boost = o->rr_threshold / Wr;
        for (int i = 0; i < C; ++i) W[i] = W[i] == Wr ? o->rr_threshold : W[i] * boost;
      } else {
        res->exit_kind = 2;
        break;
      }
    }
    const double mu = oracle_hg_mu(gg[h], u[1]);
    for (int i = 0; i < C; ++i) L[i] += hg_logpdf(gg[i], mu);
    oracle_rotate(dir, mu, 2.0 * M_PI * u[2]);
  }
  res->steps = step;
}

/* Tallies per member instance, as oracle_walk's (A and se_A stay 0).
 * N paths per group; thickness_mm (or NULL) is read at each group's first
 * member and shared by the group. */
int oracle_walk_hero(int64_t n_inst, int K, const float* alpha, const float* sigma_t,
                     const float* g, const float* w, uint32_t N, const float* thickness_mm,
                     double n_rel, const oracle_opts* o, int C, int nb_texel, int orbits,
                     uint32_t inst_offset, oracle_out* out) {
  if (K < 1 || K > ORC_KMAX || o->nbins < 1 || o->nbins > ORC_NBINS_MAX) return 1;
  if (C < 1 || C > ORC_KMAX || nb_texel < C || nb_texel % C || n_inst % nb_texel) return 1;
  if (o->mode != 0) return 1;
  const int nb = o->nbins;
  const int nv = nb + 1 + K + 4; /* [bins][overflow][R_k][R1][T][trunc][steps] */
  const int64_t per_texel = nb_texel / C;  /* groups per texel */
  const int64_t n_groups = n_inst / C;
  for (int64_t grp = 0; grp < n_groups; ++grp) {
    /* orbits: {q, q + nb/C, ...}; otherwise blocks of C adjacent bands */
    const int64_t q = grp % per_texel;
    const int64_t stride = orbits ? per_texel : 1;
    const int64_t first = (grp / per_texel) * nb_texel + (orbits ? q : q * C);
    int64_t mem[ORC_KMAX];
    for (int j = 0; j < C; ++j) mem[j] = first + j * stride;
    const double d = thickness_mm ? (double)thickness_mm[first] : INFINITY;
    const int64_t nch = ((int64_t)N + ORC_CHUNK - 1) / ORC_CHUNK;
    const size_t per = 2 * (size_t)nv * (size_t)C;
    double* ps = calloc((size_t)(nch > 0 ? nch : 1) * per, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nch; ++ch) {
      double* ls = ps + (size_t)ch * per;  /* [C][nv] sums, then [C][nv] squares */
      double c[ORC_NV_MAX];
      const int64_t p1 = (ch + 1) * ORC_CHUNK < (int64_t)N ? (ch + 1) * ORC_CHUNK : (int64_t)N;
      for (int64_t p = ch * ORC_CHUNK; p < p1; ++p) {
        oracle_hero_path r;
        trace_hero(alpha, sigma_t, g, w, K, n_inst, mem, C, (int)(p % C),
                   (uint32_t)(first + inst_offset), (uint32_t)p, d, n_rel, o, &r);
        for (int j = 0; j < C; ++j) {
          memset(c, 0, sizeof(double) * (size_t)nv);
          if (r.exit_kind == 0) {
            c[r.bin] = r.F[j];
            c[nb + 1 + r.medium] = r.F[j];
            if (r.n_coll == 1) c[nb + 1 + K] = r.F[j];
          } else if (r.exit_kind == 1) {
            c[nb + 2 + K] = r.F[j];
          } else if (r.exit_kind == 3) {
            c[nb + 3 + K] = 1.0;
          }
          c[nb + 4 + K] = (double)r.steps;
          double* lj = ls + (size_t)j * nv;
          double* l2j = ls + (size_t)C * nv + (size_t)j * nv;
          for (int q = 0; q < nv; ++q) { lj[q] += c[q]; l2j[q] += c[q] * c[q]; }
        }
      }
    }
    for (int j = 0; j < C; ++j) {
      const int64_t i = mem[j];
      double s[ORC_NV_MAX] = {0}, s2[ORC_NV_MAX] = {0};
      for (int64_t ch = 0; ch < nch; ++ch)
        for (int q = 0; q < nv; ++q) {
          s[q] += ps[(size_t)ch * per + (size_t)j * nv + (size_t)q];
          s2[q] += ps[(size_t)ch * per + (size_t)C * nv + (size_t)j * nv + (size_t)q];
        }
      const double n = (double)N;
      double sR = 0.0, s2R = 0.0;
      for (int b = 0; b <= nb; ++b) { sR += s[b]; s2R += s2[b]; }
      if (out->R) out->R[i] = sR / n;
      if (out->se_R) out->se_R[i] = se_of(sR, s2R, n);
      for (int b = 0; b < nb; ++b) {
        if (out->bins) out->bins[i * nb + b] = s[b] / n;
        if (out->se_bins) out->se_bins[i * nb + b] = se_of(s[b], s2[b], n);
      }
      if (out->overflow) out->overflow[i] = s[nb] / n;
      for (int k = 0; k < K; ++k) {
        if (out->R_k) out->R_k[i * K + k] = s[nb + 1 + k] / n;
        if (out->se_R_k) out->se_R_k[i * K + k] = se_of(s[nb + 1 + k], s2[nb + 1 + k], n);
      }
      if (out->R1) out->R1[i] = s[nb + 1 + K] / n;
      if (out->se_R1) out->se_R1[i] = se_of(s[nb + 1 + K], s2[nb + 1 + K], n);
      if (out->T) out->T[i] = s[nb + 2 + K] / n;
      if (out->se_T) out->se_T[i] = se_of(s[nb + 2 + K], s2[nb + 2 + K], n);
      if (out->A) out->A[i] = 0.0;
      if (out->se_A) out->se_A[i] = 0.0;
      if (out->truncated) out->truncated[i] = s[nb + 3 + K];
      if (out->steps) out->steps[i] = s[nb + 4 + K] / n;
    }
    free(ps);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Score-function gradient (differentiating the path contribution f_SSS of  */
/* Sec. 4.1 and the mixture of Eq. 4).                                        */
/* ------------------------------------------------------------------------ */
/* For a path that chose medium k, made n collisions, travelled L and
 * scattered with cosines mu_i, the log-density of its geometry and its
 * throughput alpha^n give
 *   d/d alpha_k   :  n / alpha_k
 *   d/d sigma_t,k :  n / sigma_t,k - L
 *   d/d g_k       :  sum_i d log p_HG(mu_i; g_k) / d g_k
 *   d/d w_k       :  1 / p_k with p_k = w_k / sum(w)   (the partial of
 *                     sum_k w_k S_k with the others held fixed, i.e. S_k)
 * each multiplied by the path's exit weight and by the upstream derivative
 * of the loss with respect to the tally the path landed in:
 *   top exit   : grad_R + grad_bins[bin] (0 for overflow) + grad_R_k[k]
 *   bottom exit: grad_T
 * Roulette and analog absorption change only the sampling of the weight,
 * whose conditional mean given the geometry is the analog throughput, so
 * they add no score term.  Outputs d_* are [K][n_inst] and hold the mean
 * over the instance's N paths. */
/* With a second layer (l2 non-NULL), the score terms above take only the
 * collisions, length and scatterings of the top layer (the chosen medium),
 * and the layer's own optics get the same three terms from its part of the
 * path: d_alpha2, d_sigma_t2, d_g2 and their standard errors se_d_*2
 * ([n_inst] each, or NULL). */
#define ORC_NG (4 * ORC_KMAX + 3) /* per-path score vector: [4][K] then 3 for layer 2 */
int oracle_walk_grad(int64_t n_inst, int K, const float* alpha, const float* sigma_t,
                     const float* g, const float* w, const uint32_t* n_paths,
                     const float* thickness_mm, double n_rel, const oracle_opts* o,
                     const int64_t* inst_ids, const oracle_layer2* l2,
                     const double* grad_R, const double* grad_bins,
                     const double* grad_R_k, const double* grad_T,
                     double* d_alpha, double* d_sigma_t, double* d_g, double* d_w,
                     double* se_d_alpha, double* se_d_sigma_t, double* se_d_g,
                     double* se_d_w, double* d_alpha2, double* d_sigma_t2, double* d_g2,
                     double* se_d_alpha2, double* se_d_sigma_t2, double* se_d_g2) {
  if (K < 1 || K > ORC_KMAX || o->nbins < 1) return 1;
  const int nb = o->nbins;
  const int ng = 4 * K + 3;
  for (int64_t i = 0; i < n_inst; ++i) {
    const uint32_t N = n_paths[i];
    const double d = thickness_mm ? (double)thickness_mm[i] : INFINITY;
    double wsum = 0.0;
    float wk[ORC_KMAX];
    for (int k = 0; k < K; ++k) { wk[k] = w[(int64_t)k * n_inst + i]; wsum += wk[k]; }
    const int64_t nch = ((int64_t)N + ORC_CHUNK - 1) / ORC_CHUNK;
    double* ps = calloc((size_t)(nch > 0 ? nch : 1) * 2 * ORC_NG, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < nch; ++ch) {
      double* ls = ps + (size_t)ch * 2 * ORC_NG;
      double* ls2 = ls + ORC_NG;
      const int64_t p1 = (ch + 1) * ORC_CHUNK < (int64_t)N ? (ch + 1) * ORC_CHUNK : (int64_t)N;
      for (int64_t p = ch * ORC_CHUNK; p < p1; ++p) {
        oracle_path r;
        oracle_trace_path_layered(alpha, sigma_t, g, w, K, n_inst, i,
                                  inst_ids ? (uint32_t)inst_ids[i] : (uint32_t)i, (uint32_t)p,
                                  d, n_rel, o, l2, &r);
        double v = 0.0;
        if (r.exit_kind == 0) {
          if (grad_R) v += grad_R[i];
          if (grad_bins && r.bin < nb) v += grad_bins[i * nb + r.bin];
          if (grad_R_k) v += grad_R_k[i * K + r.medium];
        } else if (r.exit_kind == 1) {
          if (grad_T) v += grad_T[i];
        }
        double c[ORC_NG] = {0};
        if (v != 0.0 && r.weight != 0.0) {
          const int k = r.medium;
          const double a = alpha[(int64_t)k * n_inst + i];
          const double st = sigma_t[(int64_t)k * n_inst + i];
          const double Wv = r.weight * v;
          /* top layer (the whole path without a second layer) */
          const double n1 = (double)(r.n_coll - r.n_coll2);
          c[0 * K + k] = Wv * n1 / a;
          c[1 * K + k] = Wv * (n1 / st - (r.length - r.length2));
          c[2 * K + k] = Wv * (r.dlogp_dg - r.dlogp_dg2);
          c[3 * K + k] = Wv * wsum / (double)wk[k];
          if (l2) {
            const double n2 = (double)r.n_coll2;
            c[4 * K + 0] = Wv * n2 / (double)l2->alpha2[i];
            c[4 * K + 1] = Wv * (n2 / (double)l2->sigma_t2[i] - r.length2);
            c[4 * K + 2] = Wv * r.dlogp_dg2;
          }
        }
        for (int j = 0; j < ng; ++j) { ls[j] += c[j]; ls2[j] += c[j] * c[j]; }
      }
    }
    double s[ORC_NG] = {0}, s2[ORC_NG] = {0};
    for (int64_t ch = 0; ch < nch; ++ch)
      for (int j = 0; j < ng; ++j) {
        s[j] += ps[(size_t)ch * 2 * ORC_NG + (size_t)j];
        s2[j] += ps[(size_t)ch * 2 * ORC_NG + ORC_NG + (size_t)j];
      }
    free(ps);
    const double n = (double)N;
    if (d_alpha2) d_alpha2[i] = s[4 * K + 0] / n;
    if (d_sigma_t2) d_sigma_t2[i] = s[4 * K + 1] / n;
    if (d_g2) d_g2[i] = s[4 * K + 2] / n;
    if (se_d_alpha2) se_d_alpha2[i] = se_of(s[4 * K + 0], s2[4 * K + 0], n);
    if (se_d_sigma_t2) se_d_sigma_t2[i] = se_of(s[4 * K + 1], s2[4 * K + 1], n);
    if (se_d_g2) se_d_g2[i] = se_of(s[4 * K + 2], s2[4 * K + 2], n);
    double* outs[4] = {d_alpha, d_sigma_t, d_g, d_w};
    double* ses[4] = {se_d_alpha, se_d_sigma_t, se_d_g, se_d_w};
    for (int q = 0; q < 4; ++q)
      for (int k = 0; k < K; ++k) {
        if (outs[q]) outs[q][(int64_t)k * n_inst + i] = s[q * K + k] / n;
        if (ses[q]) ses[q][(int64_t)k * n_inst + i] = se_of(s[q * K + k], s2[q * K + k], n);
      }
  }
  return 0;
}

/* Per-path trace for a list of (instance, path) pairs: lets tests compare a
 * sampled subset of a full-size run one path at a time. */
int oracle_trace_many(int64_t n_inst, int K, const float* alpha, const float* sigma_t,
                      const float* g, const float* w, const float* thickness_mm,
                      double n_rel, const oracle_opts* o, int64_t n_query,
                      const int64_t* q_inst, const uint32_t* q_path, oracle_path* res) {
  if (K < 1 || K > ORC_KMAX) return 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < n_query; ++q) {
    const int64_t i = q_inst[q];
    const double d = thickness_mm ? (double)thickness_mm[i] : INFINITY;
    oracle_trace_path(alpha, sigma_t, g, w, K, n_inst, i, (uint32_t)i, q_path[q], d, n_rel, o,
                      &res[q]);
  }
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
