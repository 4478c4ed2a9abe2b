/*
 * imask_oracle.c -- plain FP64 CPU oracle for the ImaSk hot path.
 *
 * TEST INFRASTRUCTURE ONLY: it is loaded by the tests, by the smoke check and
 * by the CPU-baseline legs of the benchmark, never by the product path.  It is
 * deliberately slow and literal: single-threaded loops in double precision,
 * each function following the passage of the paper named above it, with no
 * blocking, fusion or reordering beyond what that passage states.
 *
 * Readings of points the paper leaves open (all restated in the design notes):
 *  - Level index ell = 0..r-1: ell = 0 is the compensated full-resolution
 *    sketch (the paper's i = r), ell >= 1 halves the grid ell times.
 *  - T_ell is the 2^ell x 2^ell block mean; the paper's "adjoint" T_ell^* is
 *    replication (Sec. 4.1), so S_ell = T_ell^* T_ell is the orthogonal
 *    projector onto block-constant images and the true transpose of T_ell is
 *    4^-ell T_ell^*.
 *  - R_ell is the same projector on the coarse grid (pixel width 2^ell h).
 *  - The projector is Joseph's method: along the major axis of each ray, one
 *    linear interpolation between the two nearest pixel centres per column
 *    (or row), scaled by the pixel width over the major direction cosine.
 *  - Level draw: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) at stream
 *    position k, compared with integer thresholds from the cumulative p.
 *  - Alg. 1 is run with its self-consistent update lines: phi holds K_i^T y
 *    (image space), psi holds K_i x (measurement space); the sums use the
 *    tables before the update.
 */
#include "imask_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* small helpers                                                              */
/* ------------------------------------------------------------------------ */

static int32_t n_levels(const orc_desc *d) { return d->levels < 1 ? 1 : d->levels; }

static double prob(const orc_desc *d, int32_t ell) {
  if (d->probs) return d->probs[ell];
  return 1.0 / (double)n_levels(d);
}

static int64_t n_meas(const orc_desc *d) { return (int64_t)d->n_angles * d->n_det; }
static int64_t n_pix(const orc_desc *d) { return (int64_t)d->n * d->n; }

static double *dalloc(int64_t n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

static double dot(const double *a, const double *b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* ------------------------------------------------------------------------ */
/* Level draw -- Alg. 1, "sample i_k at random with probability p".          */
/* ------------------------------------------------------------------------ */

/* Output number k (0-based) of SplitMix64 started from state `seed`:
 * the state advances by the golden-gamma 0x9E3779B97F4A7C15 and the output is
 * the published 64-bit finaliser of the new state. */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* thr[ell] = round(2^53 * (p_0 + ... + p_ell)) * 2^11 for ell = 0..r-2; a draw
 * u lands on the level equal to the number of thresholds that are <= u. */
void orc_level_thresholds(const orc_desc *d, uint64_t *thr) {
  int32_t r = n_levels(d);
  double cum = 0.0;
  for (int32_t ell = 0; ell + 1 < r; ++ell) {
    cum += prob(d, ell);
    double scaled = cum * 9007199254740992.0; /* 2^53 */
    long long v = llround(scaled);
    if (v >= 9007199254740992LL)
      thr[ell] = UINT64_MAX;
    else if (v <= 0)
      thr[ell] = 0;
    else
      thr[ell] = ((uint64_t)v) << 11;
  }
}

int32_t orc_level(const orc_desc *d, uint64_t seed, uint64_t k) {
  int32_t r = n_levels(d);
  uint64_t thr[64];
  orc_level_thresholds(d, thr);
  uint64_t u = orc_splitmix64_at(seed, k);
  int32_t ell = 0;
  for (int32_t t = 0; t + 1 < r; ++t)
    if (u >= thr[t]) ell += 1;
  return ell;
}

void orc_levels(const orc_desc *d, uint64_t seed, uint64_t k0, int64_t n, int32_t *out) {
  for (int64_t t = 0; t < n; ++t) out[t] = orc_level(d, seed, k0 + (uint64_t)t);
}

/* ------------------------------------------------------------------------ */
/* Acquisition geometry (Sec. 4.1: K traces X-rays from source to detector).  */
/* ------------------------------------------------------------------------ */

/* Default bin pitch: the full-resolution pixel width h for parallel beam; for
 * fan beam h magnified to the detector, h (D_so + D_od) / D_so. */
double orc_det_spacing(const orc_desc *d) {
  if (d->det_spacing > 0.0) return d->det_spacing;
  double h = d->fov / (double)d->n;
  if (d->geometry == 0) return h;
  return h * (d->src_dist + d->det_dist) / d->src_dist;
}

/* Ray (a, j): a point p0 on it and an (unnormalised) direction.
 * Parallel: view angle th, ray {P : <P, (cos th, sin th)> = s_j}, direction
 *   (-sin th, cos th), point s_j (cos th, sin th).
 * Fan: source S = D_so (cos b, sin b); bin centre
 *   D_j = -D_od (cos b, sin b) + u_j (-sin b, cos b); p0 = S, dir = D_j - S.
 * s_j and u_j are (j - (n_det - 1)/2) times the bin pitch. */
void orc_ray(const orc_desc *d, int32_t a, int32_t j, double p0[2], double dir[2]) {
  double ang = d->angle_start + d->angle_span * (double)a / (double)d->n_angles;
  double s = ((double)j - 0.5 * (double)(d->n_det - 1)) * orc_det_spacing(d);
  double ca = cos(ang), sa = sin(ang);
  if (d->geometry == 0) {
    p0[0] = s * ca;
    p0[1] = s * sa;
    dir[0] = -sa;
    dir[1] = ca;
  } else {
    double sx = d->src_dist * ca;
    double sy = d->src_dist * sa;
    double dx = -d->det_dist * ca - s * sa;
    double dy = -d->det_dist * sa + s * ca;
    p0[0] = sx;
    p0[1] = sy;
    dir[0] = dx - sx;
    dir[1] = dy - sy;
  }
}

/* Major axis of a ray: x-major when |dir_x| >= |dir_y| (ties go to x). */
int32_t orc_ray_is_xmajor(const orc_desc *d, int32_t a, int32_t j) {
  double p0[2], dir[2];
  orc_ray(d, a, j, p0, dir);
  return fabs(dir[0]) >= fabs(dir[1]) ? 1 : 0;
}

static double pixel(const double *img, int32_t nl, int32_t i, int32_t c) {
  if (i < 0 || i >= nl || c < 0 || c >= nl) return 0.0;
  return img[(int64_t)i * nl + c];
}

/* Joseph's method on the grid of side nl (pixel width hl = W / nl).
 * x-major: at every column centre x_c the ray height y is converted to the
 * fractional row q = (y + W/2) / hl - 1/2; the image is interpolated linearly
 * between rows floor(q) and floor(q) + 1 (rows off the grid count as zero);
 * the sum over columns is scaled by hl / |cos| = hl sqrt(1 + (dy/dx)^2).
 * y-major is the same with rows and columns exchanged. */
double orc_joseph_ray(const orc_desc *d, int32_t nl, const double *img, int32_t a, int32_t j) {
  double p0[2], dir[2];
  orc_ray(d, a, j, p0, dir);
  const double W = d->fov;
  const double hl = W / (double)nl;
  double sum = 0.0;
  if (fabs(dir[0]) >= fabs(dir[1])) {
    double t = dir[1] / dir[0];
    for (int32_t c = 0; c < nl; ++c) {
      double xc = -0.5 * W + ((double)c + 0.5) * hl;
      double y = p0[1] + (xc - p0[0]) * t;
      double q = (y + 0.5 * W) / hl - 0.5;
      if (q < -2.0 || q > (double)nl + 1.0) continue; /* both rows off the grid */
      double fl = floor(q);
      int32_t i0 = (int32_t)fl;
      double f = q - fl;
      sum += (1.0 - f) * pixel(img, nl, i0, c) + f * pixel(img, nl, i0 + 1, c);
    }
    return sum * hl * sqrt(1.0 + t * t);
  } else {
    double t = dir[0] / dir[1];
    for (int32_t i = 0; i < nl; ++i) {
      double yi = -0.5 * W + ((double)i + 0.5) * hl;
      double x = p0[0] + (yi - p0[1]) * t;
      double q = (x + 0.5 * W) / hl - 0.5;
      if (q < -2.0 || q > (double)nl + 1.0) continue;
      double fl = floor(q);
      int32_t c0 = (int32_t)fl;
      double f = q - fl;
      sum += (1.0 - f) * pixel(img, nl, i, c0) + f * pixel(img, nl, i, c0 + 1);
    }
    return sum * hl * sqrt(1.0 + t * t);
  }
}

void orc_joseph_fp(const orc_desc *d, int32_t nl, const double *img, double *sino) {
  for (int32_t a = 0; a < d->n_angles; ++a)
    for (int32_t j = 0; j < d->n_det; ++j)
      sino[(int64_t)a * d->n_det + j] = orc_joseph_ray(d, nl, img, a, j);
}

static void scatter(double *img, int32_t nl, int32_t i, int32_t c, double v) {
  if (i < 0 || i >= nl || c < 0 || c >= nl) return;
  img[(int64_t)i * nl + c] += v;
}

/* The transpose of orc_joseph_fp: every weight that the forward projection
 * multiplies a pixel by is used here to scatter the ray's value back. */
void orc_joseph_bp(const orc_desc *d, int32_t nl, const double *sino, double *img) {
  const double W = d->fov;
  const double hl = W / (double)nl;
  memset(img, 0, sizeof(double) * (size_t)nl * (size_t)nl);
  for (int32_t a = 0; a < d->n_angles; ++a) {
    for (int32_t j = 0; j < d->n_det; ++j) {
      double p0[2], dir[2];
      orc_ray(d, a, j, p0, dir);
      double yv = sino[(int64_t)a * d->n_det + j];
      if (fabs(dir[0]) >= fabs(dir[1])) {
        double t = dir[1] / dir[0];
        double scale = hl * sqrt(1.0 + t * t);
        for (int32_t c = 0; c < nl; ++c) {
          double xc = -0.5 * W + ((double)c + 0.5) * hl;
          double y = p0[1] + (xc - p0[0]) * t;
          double q = (y + 0.5 * W) / hl - 0.5;
          if (q < -2.0 || q > (double)nl + 1.0) continue;
          double fl = floor(q);
          int32_t i0 = (int32_t)fl;
          double f = q - fl;
          scatter(img, nl, i0, c, (1.0 - f) * scale * yv);
          scatter(img, nl, i0 + 1, c, f * scale * yv);
        }
      } else {
        double t = dir[0] / dir[1];
        double scale = hl * sqrt(1.0 + t * t);
        for (int32_t i = 0; i < nl; ++i) {
          double yi = -0.5 * W + ((double)i + 0.5) * hl;
          double x = p0[0] + (yi - p0[1]) * t;
          double q = (x + 0.5 * W) / hl - 0.5;
          if (q < -2.0 || q > (double)nl + 1.0) continue;
          double fl = floor(q);
          int32_t c0 = (int32_t)fl;
          double f = q - fl;
          scatter(img, nl, i, c0, (1.0 - f) * scale * yv);
          scatter(img, nl, i, c0 + 1, f * scale * yv);
        }
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Image-domain sketches -- Sec. 4.1, decimator T_i, its "adjoint", S_r.      */
/* ------------------------------------------------------------------------ */

/* T_ell: mean over each 2^ell x 2^ell block; output side n / 2^ell. */
void orc_block_mean(int32_t n, int32_t ell, const double *x, double *out) {
  int32_t b = 1 << ell, nl = n / b;
  for (int32_t I = 0; I < nl; ++I)
    for (int32_t J = 0; J < nl; ++J) {
      double s = 0.0;
      for (int32_t u = 0; u < b; ++u)
        for (int32_t v = 0; v < b; ++v) s += x[(int64_t)(I * b + u) * n + (J * b + v)];
      out[(int64_t)I * nl + J] = s / (double)(b * b);
    }
}

/* T_ell^*: every fine pixel takes the value of the coarse pixel that holds it. */
void orc_replicate(int32_t n, int32_t ell, const double *c, double *out) {
  int32_t nl = n >> ell;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) out[(int64_t)i * n + j] = c[(int64_t)(i >> ell) * nl + (j >> ell)];
}

/* S_r = p_r^{-1} (I - sum_{i<r} p_i T_i^* T_i), in the level index ell = 0. */
void orc_compensate(const orc_desc *d, const double *x, double *out) {
  const int32_t n = d->n, r = n_levels(d);
  const int64_t np = n_pix(d);
  double *coarse = dalloc(np), *fine = dalloc(np);
  for (int64_t t = 0; t < np; ++t) out[t] = x[t];
  for (int32_t ell = 1; ell < r; ++ell) {
    orc_block_mean(n, ell, x, coarse);
    orc_replicate(n, ell, coarse, fine);
    for (int64_t t = 0; t < np; ++t) out[t] -= prob(d, ell) * fine[t];
  }
  for (int64_t t = 0; t < np; ++t) out[t] /= prob(d, 0);
  free(coarse);
  free(fine);
}

/* K_ell x, eq. CT_sketches: ell >= 1: R_ell (T_ell x); ell = 0: K (S_r x);
 * ell = -1: K x. */
void orc_apply_K(const orc_desc *d, int32_t ell, const double *x, double *sino) {
  const int32_t n = d->n;
  if (ell < 0) {
    orc_joseph_fp(d, n, x, sino);
  } else if (ell == 0) {
    double *s = dalloc(n_pix(d));
    orc_compensate(d, x, s);
    orc_joseph_fp(d, n, s, sino);
    free(s);
  } else {
    int32_t nl = n >> ell;
    double *c = dalloc((int64_t)nl * nl);
    orc_block_mean(n, ell, x, c);
    orc_joseph_fp(d, nl, c, sino);
    free(c);
  }
}

/* K_ell^T y: ell >= 1: 4^-ell T_ell^* (R_ell^T y); ell = 0: S_r (K^T y)
 * (S_r is symmetric); ell = -1: K^T y. */
void orc_apply_KT(const orc_desc *d, int32_t ell, const double *y, double *img) {
  const int32_t n = d->n;
  const int64_t np = n_pix(d);
  if (ell < 0) {
    orc_joseph_bp(d, n, y, img);
  } else if (ell == 0) {
    double *g = dalloc(np);
    orc_joseph_bp(d, n, y, g);
    orc_compensate(d, g, img);
    free(g);
  } else {
    int32_t nl = n >> ell;
    double *g = dalloc((int64_t)nl * nl);
    orc_joseph_bp(d, nl, y, g);
    orc_replicate(n, ell, g, img);
    double s = 1.0 / (double)((int64_t)1 << (2 * ell));
    for (int64_t t = 0; t < np; ++t) img[t] *= s;
    free(g);
  }
}

/* ------------------------------------------------------------------------ */
/* Regulariser and its prox -- eq. prox_op; TV prox by FISTA as in Sec. 4.5.  */
/* ------------------------------------------------------------------------ */

/* Forward differences with zero difference on the last row / column. */
static void grad_fwd(int32_t n, const double *x, double *g1, double *g2) {
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) {
      int64_t p = (int64_t)i * n + j;
      g1[p] = (i + 1 < n) ? x[p + n] - x[p] : 0.0;
      g2[p] = (j + 1 < n) ? x[p + 1] - x[p] : 0.0;
    }
}

/* Transpose of grad_fwd applied to (w1, w2), accumulated into out. */
static void grad_fwd_T(int32_t n, const double *w1, const double *w2, double *out) {
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < n; ++j) {
      int64_t p = (int64_t)i * n + j;
      if (i + 1 < n) {
        out[p + n] += w1[p];
        out[p] -= w1[p];
      }
      if (j + 1 < n) {
        out[p + 1] += w2[p];
        out[p] -= w2[p];
      }
    }
}

/* R(x) = mu/2 |x|^2 (+ lambda sum_p sqrt(|grad x|_p^2 + eps^2) when reg = 1);
 * reg = 2: lambda sum_p |grad x|_p (TV with a nonnegativity constraint). */
double orc_regulariser(const orc_desc *d, const double *x) {
  const int64_t np = n_pix(d);
  if (d->reg == 2) {
    /* lambda |grad x|_{1,2}; the nonnegativity indicator is not evaluated
     * (the iterates are nonnegative by construction of the prox) */
    double *g1 = dalloc(np), *g2 = dalloc(np);
    grad_fwd(d->n, x, g1, g2);
    double tv = 0.0;
    for (int64_t p = 0; p < np; ++p) tv += sqrt(g1[p] * g1[p] + g2[p] * g2[p]);
    free(g1);
    free(g2);
    return d->tv_lambda * tv;
  }
  double r = 0.5 * d->mu * dot(x, x, np);
  if (d->reg == 1) {
    double *g1 = dalloc(np), *g2 = dalloc(np);
    grad_fwd(d->n, x, g1, g2);
    double tv = 0.0;
    for (int64_t p = 0; p < np; ++p) tv += sqrt(g1[p] * g1[p] + g2[p] * g2[p] + d->tv_eps * d->tv_eps);
    r += d->tv_lambda * tv;
    free(g1);
    free(g2);
  }
  return r;
}

/* argmin_{x >= 0} 1/2 |x - v|^2 + alpha |grad x|_{1,2} (Sec. 4.5: TV with a
 * nonnegativity constraint, prox by FISTA) by exactly tv_inner iterations of
 * the fast gradient projection on the dual (Beck & Teboulle, IEEE TIP 2009):
 * for a dual field p = (p1, p2) with |p_j| <= 1 the primal point is
 * x(p) = P_{>=0}(v - alpha grad^T p); a projected gradient step on the dual
 * is p <- P_{|.|<=1}(r + grad x(r) / (8 alpha)) (|grad|^2 <= 8), with Nesterov
 * extrapolation r = p_k + (t_k - 1)/t_{k+1} (p_k - p_{k-1}), starting from
 * p = r = 0, t_1 = 1.  The result is x(p_N).  alpha = 0 or tv_inner = 0
 * gives the projection P_{>=0}(v). */
static void prox_tv_nonneg(const orc_desc *d, double alpha, const double *v, double *out) {
  const int32_t n = d->n;
  const int64_t np = n_pix(d);
  if (!(alpha > 0.0) || d->tv_inner <= 0) {
    for (int64_t p = 0; p < np; ++p) out[p] = v[p] > 0.0 ? v[p] : 0.0;
    return;
  }
  double *p1 = dalloc(np), *p2 = dalloc(np), *q1 = dalloc(np), *q2 = dalloc(np);
  double *r1 = dalloc(np), *r2 = dalloc(np), *x = dalloc(np), *dt = dalloc(np);
  double *g1 = dalloc(np), *g2 = dalloc(np);
  double t = 1.0;
  for (int32_t k = 0; k < d->tv_inner; ++k) {
    /* x(r) = P_{>=0}(v - alpha grad^T r) */
    for (int64_t p = 0; p < np; ++p) dt[p] = 0.0;
    grad_fwd_T(n, r1, r2, dt);
    for (int64_t p = 0; p < np; ++p) {
      const double u = v[p] - alpha * dt[p];
      x[p] = u > 0.0 ? u : 0.0;
    }
    /* p_k = P(r + grad x / (8 alpha)) */
    grad_fwd(n, x, g1, g2);
    for (int64_t p = 0; p < np; ++p) {
      q1[p] = p1[p];   /* p_{k-1} */
      q2[p] = p2[p];
      const double a = r1[p] + g1[p] / (8.0 * alpha);
      const double b = r2[p] + g2[p] / (8.0 * alpha);
      const double nrm = sqrt(a * a + b * b);
      const double sc = nrm > 1.0 ? 1.0 / nrm : 1.0;
      p1[p] = a * sc;
      p2[p] = b * sc;
    }
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const double beta = (t - 1.0) / tn;
    for (int64_t p = 0; p < np; ++p) {
      r1[p] = p1[p] + beta * (p1[p] - q1[p]);
      r2[p] = p2[p] + beta * (p2[p] - q2[p]);
    }
    t = tn;
  }
  for (int64_t p = 0; p < np; ++p) dt[p] = 0.0;
  grad_fwd_T(n, p1, p2, dt);
  for (int64_t p = 0; p < np; ++p) {
    const double u = v[p] - alpha * dt[p];
    out[p] = u > 0.0 ? u : 0.0;
  }
  free(p1);
  free(p2);
  free(q1);
  free(q2);
  free(r1);
  free(r2);
  free(x);
  free(dt);
  free(g1);
  free(g2);
}

/* prox_{tau R}(v) = argmin_x 1/2 |x - v|^2 + tau R(x).
 * Quadratic R: v / (1 + tau mu).
 * Quadratic + smoothed TV: exactly tv_inner FISTA steps (Beck & Teboulle) on
 * F(x) = 1/2|x - v|^2 + tau mu/2 |x|^2 + tau lambda TV_eps(x), started at v,
 * with step 1/L_in, L_in = 1 + tau mu + 8 tau lambda / eps (|grad|^2 <= 8). */
void orc_prox(const orc_desc *d, double tau, const double *v, double *out) {
  const int64_t np = n_pix(d);
  if (d->reg == 2) {
    prox_tv_nonneg(d, tau * d->tv_lambda, v, out);
    return;
  }
  if (d->reg != 1) {
    for (int64_t p = 0; p < np; ++p) out[p] = v[p] / (1.0 + tau * d->mu);
    return;
  }
  const int32_t n = d->n;
  const double lam = d->tv_lambda, eps = d->tv_eps;
  const double Lin = 1.0 + tau * d->mu + 8.0 * tau * lam / eps;
  double *x = dalloc(np), *xprev = dalloc(np), *z = dalloc(np), *grad = dalloc(np);
  double *g1 = dalloc(np), *g2 = dalloc(np);
  for (int64_t p = 0; p < np; ++p) x[p] = z[p] = v[p];
  double t = 1.0;
  for (int32_t it = 0; it < d->tv_inner; ++it) {
    /* gradient of F at z */
    grad_fwd(n, z, g1, g2);
    for (int64_t p = 0; p < np; ++p) {
      double nrm = sqrt(g1[p] * g1[p] + g2[p] * g2[p] + eps * eps);
      g1[p] /= nrm;
      g2[p] /= nrm;
    }
    for (int64_t p = 0; p < np; ++p) grad[p] = 0.0;
    grad_fwd_T(n, g1, g2, grad);
    for (int64_t p = 0; p < np; ++p) grad[p] = (z[p] - v[p]) + tau * d->mu * z[p] + tau * lam * grad[p];
    /* gradient step and Nesterov extrapolation */
    for (int64_t p = 0; p < np; ++p) {
      xprev[p] = x[p];
      x[p] = z[p] - grad[p] / Lin;
    }
    double tnext = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    double beta = (t - 1.0) / tnext;
    for (int64_t p = 0; p < np; ++p) z[p] = x[p] + beta * (x[p] - xprev[p]);
    t = tnext;
  }
  for (int64_t p = 0; p < np; ++p) out[p] = x[p];
  free(x);
  free(xprev);
  free(z);
  free(grad);
  free(g1);
  free(g2);
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 (ImaSk).                                                            */
/* ------------------------------------------------------------------------ */

int32_t orc_imask_run(const orc_desc *d, const double *b, uint64_t seed, int64_t k0,
                      int32_t iters, double *x, double *y, double *phi, double *psi,
                      int32_t *levels_out) {
  const int32_t r = n_levels(d);
  const int64_t np = n_pix(d), m = n_meas(d);
  const double sigma = d->sigma, mu = d->mu;
  if (!(sigma > 0.0) || !(mu > 0.0)) return 1;
  double *phi_new = dalloc(np), *psi_new = dalloc(m);
  double *xi = dalloc(np), *zeta = dalloc(m), *v = dalloc(np), *xn = dalloc(np);
  for (int32_t it = 0; it < iters; ++it) {
    const uint64_t k = (uint64_t)(k0 + it);
    /* line 2: sample i_k */
    const int32_t l = orc_level(d, seed, k);
    if (levels_out) levels_out[it] = l;
    /* lines 3-4: refreshed table entries K_l^T y^k and K_l x^k */
    orc_apply_KT(d, l, y, phi_new);
    orc_apply_K(d, l, x, psi_new);
    /* line 5: xi = phi_new - phi_l + sum_i p_i phi_i (tables before the update) */
    for (int64_t p = 0; p < np; ++p) {
      double s = 0.0;
      for (int32_t i = 0; i < r; ++i) s += prob(d, i) * phi[(int64_t)i * np + p];
      xi[p] = phi_new[p] - phi[(int64_t)l * np + p] + s;
    }
    /* line 6: zeta = psi_new - psi_l + sum_i p_i psi_i */
    for (int64_t q = 0; q < m; ++q) {
      double s = 0.0;
      for (int32_t i = 0; i < r; ++i) s += prob(d, i) * psi[(int64_t)i * m + q];
      zeta[q] = psi_new[q] - psi[(int64_t)l * m + q] + s;
    }
    /* line 7: x^{k+1} = prox_{sigma/mu R}(x^k - sigma/mu xi) */
    for (int64_t p = 0; p < np; ++p) v[p] = x[p] - (sigma / mu) * xi[p];
    orc_prox(d, sigma / mu, v, xn);
    /* line 8: y^{k+1} = (y^k + sigma zeta - sigma b) / (1 + sigma) */
    for (int64_t q = 0; q < m; ++q) y[q] = (y[q] + sigma * zeta[q] - sigma * b[q]) / (1.0 + sigma);
    for (int64_t p = 0; p < np; ++p) x[p] = xn[p];
    /* table updates of lines 3-4 take effect for the next iteration */
    memcpy(phi + (int64_t)l * np, phi_new, sizeof(double) * (size_t)np);
    memcpy(psi + (int64_t)l * m, psi_new, sizeof(double) * (size_t)m);
  }
  free(phi_new);
  free(psi_new);
  free(xi);
  free(zeta);
  free(v);
  free(xn);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 7 (ImaSk-Seq): the dual step first, on the extrapolated iterate; the  */
/* primal step with the new dual iterate; then the extrapolation.             */
/* ------------------------------------------------------------------------ */

int32_t orc_imask_seq_run(const orc_desc *d, const double *b, uint64_t seed, int64_t k0,
                          int32_t iters, double theta, double *x, double *xbar, double *y,
                          double *phi, double *psi, int32_t *levels_out) {
  const int32_t r = n_levels(d);
  const int64_t np = n_pix(d), m = n_meas(d);
  const double sigma = d->sigma, mu = d->mu;
  if (!(sigma > 0.0) || !(mu > 0.0)) return 1;
  double *phi_new = dalloc(np), *psi_new = dalloc(m);
  double *xi = dalloc(np), *zeta = dalloc(m), *v = dalloc(np), *xn = dalloc(np);
  for (int32_t it = 0; it < iters; ++it) {
    const uint64_t k = (uint64_t)(k0 + it);
    /* sample i_k */
    const int32_t l = orc_level(d, seed, k);
    if (levels_out) levels_out[it] = l;
    /* psi_l refreshed with K_l xbar^k */
    orc_apply_K(d, l, xbar, psi_new);
    /* zeta = psi_new - psi_l + sum_i p_i psi_i (tables before the update) */
    for (int64_t q = 0; q < m; ++q) {
      double s = 0.0;
      for (int32_t i = 0; i < r; ++i) s += prob(d, i) * psi[(int64_t)i * m + q];
      zeta[q] = psi_new[q] - psi[(int64_t)l * m + q] + s;
    }
    /* dual update y^{k+1} = (y^k + sigma zeta - sigma b) / (1 + sigma) */
    for (int64_t q = 0; q < m; ++q) y[q] = (y[q] + sigma * zeta[q] - sigma * b[q]) / (1.0 + sigma);
    /* phi_l refreshed with K_l^T y^{k+1}, the new dual iterate */
    orc_apply_KT(d, l, y, phi_new);
    /* xi = phi_new - phi_l + sum_i p_i phi_i */
    for (int64_t p = 0; p < np; ++p) {
      double s = 0.0;
      for (int32_t i = 0; i < r; ++i) s += prob(d, i) * phi[(int64_t)i * np + p];
      xi[p] = phi_new[p] - phi[(int64_t)l * np + p] + s;
    }
    /* x^{k+1} = prox_{sigma/mu R}(x^k - sigma/mu xi) */
    for (int64_t p = 0; p < np; ++p) v[p] = x[p] - (sigma / mu) * xi[p];
    orc_prox(d, sigma / mu, v, xn);
    /* extrapolation xbar^{k+1} = x^{k+1} + theta (x^{k+1} - x^k) */
    for (int64_t p = 0; p < np; ++p) {
      xbar[p] = xn[p] + theta * (xn[p] - x[p]);
      x[p] = xn[p];
    }
    memcpy(phi + (int64_t)l * np, phi_new, sizeof(double) * (size_t)np);
    memcpy(psi + (int64_t)l * m, psi_new, sizeof(double) * (size_t)m);
  }
  free(phi_new);
  free(psi_new);
  free(xi);
  free(zeta);
  free(v);
  free(xn);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Variants of Alg. 1 / Alg. 7 on one loop:                                   */
/*  - sequential: Alg. 7's order and extrapolation (else Alg. 1's);           */
/*  - snapshots: the measurement-side tables are kept as the projector inputs */
/*    of each level's last refresh (the remark after Alg. 3: store x instead  */
/*    of A_i x, same number of products by linearity), with the running sum   */
/*    sum_i p_i psi_i kept as its own m-vector;                               */
/*  - independent: the primal level (back-projector, phi tables) is drawn     */
/*    from a second stream, the dual level (projector, psi tables) from the   */
/*    first (the separate primal and dual samples named as an open question   */
/*    in the discussion, Sec. 6).                                              */
/* ------------------------------------------------------------------------ */

/* Nearest representable value with RNE: the quantum is 2^(e - bits + 1) for a
 * value in [2^e, 2^(e+1)), with e clamped below at emin (subnormals); ties go
 * to the even multiple (nearbyint in the default rounding mode).  Overflow is
 * not modelled (the tables stay far below both formats' largest values). */
double orc_round_format(double v, int32_t bits, int32_t emin) {
  if (v == 0.0 || !isfinite(v)) return v;
  int e2 = 0;
  frexp(v, &e2);          /* |v| = f 2^e2, f in [0.5, 1) */
  int ex = e2 - 1;        /* |v| in [2^ex, 2^(ex+1)) */
  if (ex < emin) ex = emin;
  const double q = ldexp(1.0, ex - (bits - 1));
  return nearbyint(v / q) * q;
}

static double store_table(const orc_variant *var, double v) {
  if (var->storage == 1) return orc_round_format(v, 8, -126);
  if (var->storage == 2) return orc_round_format(v, 11, -14);
  return v;
}

uint64_t orc_primal_seed(uint64_t seed) {
  /* the SplitMix64 finaliser applied to the seed itself */
  uint64_t z = seed;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

int32_t orc_imask_variant_run(const orc_desc *d, const orc_variant *var, const double *b,
                              uint64_t seed, int64_t k0, int32_t iters, double *x, double *xbar,
                              double *y, double *phi, double *psi, double *snap,
                              double *psi_mean, int32_t *levels_dual, int32_t *levels_primal) {
  const int32_t r = n_levels(d);
  const int64_t np = n_pix(d), m = n_meas(d);
  const double sigma = d->sigma, mu = d->mu;
  if (!(sigma > 0.0) || !(mu > 0.0)) return 1;
  if (var->sequential && !xbar) return 2;
  if (var->snapshots ? (!snap || !psi_mean) : !psi) return 2;
  const uint64_t seed_x = var->independent ? orc_primal_seed(seed) : seed;
  double *phi_new = dalloc(np), *kx = dalloc(m), *delta = dalloc(m), *diff = dalloc(np);
  double *u = dalloc(np), *xi = dalloc(np), *zeta = dalloc(m), *v = dalloc(np), *xn = dalloc(np);
  double *yn = dalloc(m);
  for (int32_t it = 0; it < iters; ++it) {
    const uint64_t k = (uint64_t)(k0 + it);
    const int32_t ld = orc_level(d, seed, k);   /* dual level: projector, psi tables */
    const int32_t lp = orc_level(d, seed_x, k); /* primal level: back-projector, phi tables */
    if (levels_dual) levels_dual[it] = ld;
    if (levels_primal) levels_primal[it] = lp;
    /* projector input: x^k (Alg. 1) or xbar^k (Alg. 7) */
    memcpy(u, var->sequential ? xbar : x, sizeof(double) * (size_t)np);
    /* delta = (refreshed psi_ld) - psi_ld and zeta = delta + sum_i p_i psi_i */
    if (var->snapshots) {
      for (int64_t p = 0; p < np; ++p) diff[p] = u[p] - snap[(int64_t)ld * np + p];
      orc_apply_K(d, ld, diff, delta);
      for (int64_t q = 0; q < m; ++q) zeta[q] = delta[q] + psi_mean[q];
    } else {
      orc_apply_K(d, ld, u, kx);
      for (int64_t q = 0; q < m; ++q) {
        double s = 0.0;
        for (int32_t i = 0; i < r; ++i) s += prob(d, i) * psi[(int64_t)i * m + q];
        delta[q] = kx[q] - psi[(int64_t)ld * m + q];
        zeta[q] = delta[q] + s;
      }
      /* 16-bit tables: the refreshed entry is stored rounded (the sum above
       * always runs over the stored values) */
      for (int64_t q = 0; q < m; ++q) kx[q] = store_table(var, kx[q]);
    }
    /* Alg. 1 back-projects y^k; Alg. 7 back-projects y^{k+1} */
    for (int64_t q = 0; q < m; ++q) yn[q] = (y[q] + sigma * zeta[q] - sigma * b[q]) / (1.0 + sigma);
    orc_apply_KT(d, lp, var->sequential ? yn : y, phi_new);
    for (int64_t p = 0; p < np; ++p) {
      double s = 0.0;
      for (int32_t i = 0; i < r; ++i) s += prob(d, i) * phi[(int64_t)i * np + p];
      xi[p] = phi_new[p] - phi[(int64_t)lp * np + p] + s;
    }
    for (int64_t p = 0; p < np; ++p) v[p] = x[p] - (sigma / mu) * xi[p];
    orc_prox(d, sigma / mu, v, xn);
    if (var->sequential)
      for (int64_t p = 0; p < np; ++p) xbar[p] = xn[p] + var->theta * (xn[p] - x[p]);
    memcpy(x, xn, sizeof(double) * (size_t)np);
    memcpy(y, yn, sizeof(double) * (size_t)m);
    /* table updates (16-bit tables: the refreshed image-side entry is stored
     * rounded too; xi above took the refreshed value itself) */
    for (int64_t p = 0; p < np; ++p) phi[(int64_t)lp * np + p] = store_table(var, phi_new[p]);
    if (var->snapshots) {
      for (int64_t q = 0; q < m; ++q) psi_mean[q] += prob(d, ld) * delta[q];
      memcpy(snap + (int64_t)ld * np, u, sizeof(double) * (size_t)np);
    } else {
      memcpy(psi + (int64_t)ld * m, kx, sizeof(double) * (size_t)m);
    }
  }
  free(phi_new);
  free(kx);
  free(delta);
  free(diff);
  free(u);
  free(xi);
  free(zeta);
  free(v);
  free(xn);
  free(yn);
  return 0;
}

static void apply_Kbar(const orc_desc *d, const double *x, double *out);
static void apply_KbarT(const orc_desc *d, const double *y, double *out);

/* ------------------------------------------------------------------------ */
/* PDHG (Chambolle & Pock 2011), the comparison method and x_nat generator of */
/* Sec. 5, on min_x 1/2 |Kbar x - b|^2 + R(x) with Kbar = sum_l p_l K_l:     */
/*   y+ = prox_{s f*}(y + s Kbar xbar) = (y + s Kbar xbar - s b) / (1 + s)     */
/*   x+ = prox_{t R}(x - t Kbar^T y+),  xbar = x+ + theta (x+ - x).            */
/* ------------------------------------------------------------------------ */

/* The parameters printed with the comparison of Sec. 5 for a mu-strongly
 * convex R: kappa = sqrt(1 + |K|^2 / (mu rho^2)), s = 1/(kappa - 1),
 * t = 1/((kappa - 1) mu), theta = 1 - 2/(1 + kappa).  out = {s, t, theta}. */
void orc_pdhg_params(double norm_K, double mu, double rho, double out[3]) {
  const double kappa = sqrt(1.0 + norm_K * norm_K / (mu * rho * rho));
  out[0] = 1.0 / (kappa - 1.0);
  out[1] = 1.0 / ((kappa - 1.0) * mu);
  out[2] = 1.0 - 2.0 / (1.0 + kappa);
}

int32_t orc_pdhg_run(const orc_desc *d, const double *b, int32_t iters, double s, double t,
                     double theta, double *x, double *xbar, double *y) {
  const int64_t np = n_pix(d), m = n_meas(d);
  if (!(s > 0.0) || !(t > 0.0)) return 1;
  double *kx = dalloc(m), *kty = dalloc(np), *v = dalloc(np), *xn = dalloc(np);
  for (int32_t it = 0; it < iters; ++it) {
    apply_Kbar(d, xbar, kx);
    for (int64_t q = 0; q < m; ++q) y[q] = (y[q] + s * kx[q] - s * b[q]) / (1.0 + s);
    apply_KbarT(d, y, kty);
    for (int64_t p = 0; p < np; ++p) v[p] = x[p] - t * kty[p];
    orc_prox(d, t, v, xn);
    for (int64_t p = 0; p < np; ++p) {
      xbar[p] = xn[p] + theta * (xn[p] - x[p]);
      x[p] = xn[p];
    }
  }
  free(kx);
  free(kty);
  free(v);
  free(xn);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Step-size constants -- Sec. 3.4 (B, Bbar, Bbar_p with A_i = p_i K_i and the */
/* normalisation of Sec. 3.3 by sqrt(mu)), estimated by the power method.     */
/* ------------------------------------------------------------------------ */

typedef void (*level_op)(const void *ctx, int32_t ell, int32_t transpose, const double *in,
                         double *out);

typedef struct {
  level_op op;
  const void *ctx;
  int32_t r;
  const double *w;
  int64_t dim_x, dim_y;
  int32_t cross, transposed;
} power_ctx;

/* One application of the symmetric operator selected in power_ctx. */
static void power_apply(const power_ctx *pc, const double *in, double *out) {
  const int64_t nx = pc->dim_x, ny = pc->dim_y;
  if (pc->cross) {
    /* (sum w_l K_l)^T (sum w_l K_l) in = sum_l w_l K_l^T (sum_k w_k K_k in) */
    double *acc = dalloc(ny), *tmp = dalloc(ny), *tx = dalloc(nx);
    for (int32_t l = 0; l < pc->r; ++l) {
      pc->op(pc->ctx, l, 0, in, tmp);
      for (int64_t q = 0; q < ny; ++q) acc[q] += pc->w[l] * tmp[q];
    }
    for (int64_t p = 0; p < nx; ++p) out[p] = 0.0;
    for (int32_t l = 0; l < pc->r; ++l) {
      pc->op(pc->ctx, l, 1, acc, tx);
      for (int64_t p = 0; p < nx; ++p) out[p] += pc->w[l] * tx[p];
    }
    free(acc);
    free(tmp);
    free(tx);
  } else if (!pc->transposed) {
    /* sum_l w_l K_l^T K_l in  (image space) */
    double *tmp = dalloc(ny), *tx = dalloc(nx);
    for (int64_t p = 0; p < nx; ++p) out[p] = 0.0;
    for (int32_t l = 0; l < pc->r; ++l) {
      pc->op(pc->ctx, l, 0, in, tmp);
      pc->op(pc->ctx, l, 1, tmp, tx);
      for (int64_t p = 0; p < nx; ++p) out[p] += pc->w[l] * tx[p];
    }
    free(tmp);
    free(tx);
  } else {
    /* sum_l w_l K_l K_l^T in  (measurement space) */
    double *tmp = dalloc(nx), *ty = dalloc(ny);
    for (int64_t q = 0; q < ny; ++q) out[q] = 0.0;
    for (int32_t l = 0; l < pc->r; ++l) {
      pc->op(pc->ctx, l, 1, in, tmp);
      pc->op(pc->ctx, l, 0, tmp, ty);
      for (int64_t q = 0; q < ny; ++q) out[q] += pc->w[l] * ty[q];
    }
    free(tmp);
    free(ty);
  }
}

/* Power method (Golub & Van Loan): v <- M v / |M v| from a fixed start vector;
 * returns the Rayleigh quotient of the last iterate. */
static double power_method(const power_ctx *pc, int32_t iters) {
  const int64_t n = (pc->cross || !pc->transposed) ? pc->dim_x : pc->dim_y;
  double *v = dalloc(n), *w = dalloc(n);
  for (int64_t i = 0; i < n; ++i) v[i] = 1.0 + 0.5 * cos(0.7 * (double)i);
  double nv = sqrt(dot(v, v, n));
  for (int64_t i = 0; i < n; ++i) v[i] /= nv;
  double lam = 0.0;
  for (int32_t it = 0; it < iters; ++it) {
    power_apply(pc, v, w);
    lam = dot(v, w, n);
    double nw = sqrt(dot(w, w, n));
    if (!(nw > 0.0)) {
      lam = 0.0;
      break;
    }
    for (int64_t i = 0; i < n; ++i) v[i] = w[i] / nw;
  }
  free(v);
  free(w);
  return lam;
}

static void desc_op(const void *ctx, int32_t ell, int32_t transpose, const double *in, double *out) {
  const orc_desc *d = (const orc_desc *)ctx;
  if (transpose)
    orc_apply_KT(d, ell, in, out);
  else
    orc_apply_K(d, ell, in, out);
}

typedef struct {
  const double *mats;
  int64_t dim_x, dim_y;
} dense_ctx;

static void dense_op(const void *ctx, int32_t ell, int32_t transpose, const double *in, double *out) {
  const dense_ctx *c = (const dense_ctx *)ctx;
  const double *A = c->mats + (int64_t)ell * c->dim_x * c->dim_y;
  if (!transpose) {
    for (int64_t i = 0; i < c->dim_y; ++i) {
      double s = 0.0;
      for (int64_t j = 0; j < c->dim_x; ++j) s += A[i * c->dim_x + j] * in[j];
      out[i] = s;
    }
  } else {
    for (int64_t j = 0; j < c->dim_x; ++j) out[j] = 0.0;
    for (int64_t i = 0; i < c->dim_y; ++i)
      for (int64_t j = 0; j < c->dim_x; ++j) out[j] += A[i * c->dim_x + j] * in[i];
  }
}

double orc_power_eig(const orc_desc *d, const double *w, int32_t cross, int32_t transposed,
                     int32_t iters) {
  power_ctx pc = {desc_op, d, n_levels(d), w, n_pix(d), n_meas(d), cross, transposed};
  return power_method(&pc, iters);
}

/* L = |sum_l p_l K_l| / sqrt(mu);
 * Lbar^2   = max(lmax(sum p_l^2 K_l^T K_l), lmax(sum p_l^2 K_l K_l^T)) / mu;
 * Lbar_p^2 = max(lmax(sum p_l   K_l^T K_l), lmax(sum p_l   K_l K_l^T)) / mu. */
static void constants_from(level_op op, const void *ctx, int32_t r, const double *p, int64_t nx,
                           int64_t ny, double mu, int32_t iters, double out[3]) {
  double w1[64], w2[64];
  for (int32_t l = 0; l < r; ++l) {
    w1[l] = p[l];
    w2[l] = p[l] * p[l];
  }
  power_ctx c_cross = {op, ctx, r, w1, nx, ny, 1, 0};
  power_ctx c_bar_x = {op, ctx, r, w2, nx, ny, 0, 0};
  power_ctx c_bar_y = {op, ctx, r, w2, nx, ny, 0, 1};
  power_ctx c_p_x = {op, ctx, r, w1, nx, ny, 0, 0};
  power_ctx c_p_y = {op, ctx, r, w1, nx, ny, 0, 1};
  double lc = power_method(&c_cross, iters);
  double lb = fmax(power_method(&c_bar_x, iters), power_method(&c_bar_y, iters));
  double lp = fmax(power_method(&c_p_x, iters), power_method(&c_p_y, iters));
  out[0] = sqrt(lc / mu);
  out[1] = sqrt(lb / mu);
  out[2] = sqrt(lp / mu);
}

void orc_constants_dense(const double *mats, int32_t r, const double *p, int32_t dim_x,
                         int32_t dim_y, double mu, int32_t iters, double out[3]) {
  dense_ctx c = {mats, dim_x, dim_y};
  constants_from(dense_op, &c, r, p, dim_x, dim_y, mu, iters, out);
}

void orc_constants(const orc_desc *d, int32_t iters, double out[3]) {
  int32_t r = n_levels(d);
  double p[64];
  for (int32_t l = 0; l < r; ++l) p[l] = prob(d, l);
  constants_from(desc_op, d, r, p, n_pix(d), n_meas(d), d->mu, iters, out);
}

/* ||K|| for the plain full-resolution operator (ell = -1), power method on K^T K. */
double orc_norm_K(const orc_desc *d, int32_t iters) {
  const int64_t nx = n_pix(d), ny = n_meas(d);
  double *v = dalloc(nx), *t = dalloc(ny), *u = dalloc(nx);
  for (int64_t i = 0; i < nx; ++i) v[i] = 1.0 + 0.5 * cos(0.7 * (double)i);
  double nv = sqrt(dot(v, v, nx));
  for (int64_t i = 0; i < nx; ++i) v[i] /= nv;
  double lam = 0.0;
  for (int32_t it = 0; it < iters; ++it) {
    orc_apply_K(d, -1, v, t);
    orc_apply_KT(d, -1, t, u);
    lam = dot(v, u, nx);
    double nu = sqrt(dot(u, u, nx));
    if (!(nu > 0.0)) break;
    for (int64_t i = 0; i < nx; ++i) v[i] = u[i] / nu;
  }
  free(v);
  free(t);
  free(u);
  return sqrt(lam);
}

/* ------------------------------------------------------------------------ */
/* Optimal step size -- Sec. 3.5 (eq. theta, phi_psi, alpha) and Thm. 3.      */
/* ------------------------------------------------------------------------ */

/* alpha^{-1} = Lbar^2 / (rho c) * (1 - (1 + L^2) c) / (1 - (1 + L^2 + Lbar_p^2) c) */
static double alpha_inv(double c, double rho, double L, double Lbar, double Lbar_p) {
  double num = 1.0 - (1.0 + L * L) * c;
  double den = 1.0 - (1.0 + L * L + Lbar_p * Lbar_p) * c;
  return Lbar * Lbar / (rho * c) * num / den;
}

/* theta_{c,rho}(eta) = max(phi, psi) with
 * phi = (eta - c)^2 / c + 1 - (1 - rho) c,  psi = alpha^{-1} eta^2 + 1 - min p. */
double orc_theta(double eta, double c, double rho, double L, double Lbar, double Lbar_p,
                 double pmin) {
  double phi = (eta - c) * (eta - c) / c + 1.0 - (1.0 - rho) * c;
  double psi = alpha_inv(c, rho, L, Lbar, Lbar_p) * eta * eta + 1.0 - pmin;
  return phi > psi ? phi : psi;
}

/* Thm. 3: eta* = c under eq. opt:cond, else the crossing of eq. eta_opt. */
double orc_eta_opt(double c, double rho, double L, double Lbar, double Lbar_p, double pmin) {
  double ai = alpha_inv(c, rho, L, Lbar, Lbar_p);
  double cond_rhs = (Lbar * Lbar / rho * (1.0 - (1.0 + L * L) * c) /
                         (1.0 - (1.0 + L * L + Lbar_p * Lbar_p) * c) +
                     1.0 - rho) *
                    c;
  if (pmin > cond_rhs) return c;
  double D = ai - 1.0 / c;
  return (sqrt(1.0 + D * (pmin + rho * c)) - 1.0) / D;
}

/* Minimise theta*(c, rho) = theta_{c,rho}(eta*) over the grid
 * c = cbar (i + 1/2) / G, rho = (j + 1/2) / G, cbar = 1 / (1 + L^2 + Lbar_p^2);
 * sigma = eta / (1 - eta). */
void orc_optimal_step(double L, double Lbar, double Lbar_p, double pmin, int32_t grid,
                      double out[4]) {
  double cbar = 1.0 / (1.0 + L * L + Lbar_p * Lbar_p);
  double best = INFINITY, best_eta = 0.0, best_c = 0.0, best_rho = 0.0;
  for (int32_t i = 0; i < grid; ++i) {
    double c = cbar * ((double)i + 0.5) / (double)grid;
    for (int32_t j = 0; j < grid; ++j) {
      double rho = ((double)j + 0.5) / (double)grid;
      double eta = orc_eta_opt(c, rho, L, Lbar, Lbar_p, pmin);
      double th = orc_theta(eta, c, rho, L, Lbar, Lbar_p, pmin);
      if (th < best) {
        best = th;
        best_eta = eta;
        best_c = c;
        best_rho = rho;
      }
    }
  }
  out[0] = best_eta / (1.0 - best_eta);
  out[1] = best;
  out[2] = best_c;
  out[3] = best_rho;
}

/* ------------------------------------------------------------------------ */
/* Fixed point of the sketched problem (eq. min_obj_new) and metrics.          */
/* ------------------------------------------------------------------------ */

/* Kbar x = sum_l p_l K_l x */
static void apply_Kbar(const orc_desc *d, const double *x, double *out) {
  const int64_t m = n_meas(d);
  double *t = dalloc(m);
  for (int64_t q = 0; q < m; ++q) out[q] = 0.0;
  for (int32_t l = 0; l < n_levels(d); ++l) {
    orc_apply_K(d, l, x, t);
    for (int64_t q = 0; q < m; ++q) out[q] += prob(d, l) * t[q];
  }
  free(t);
}

static void apply_KbarT(const orc_desc *d, const double *y, double *out) {
  const int64_t np = n_pix(d);
  double *t = dalloc(np);
  for (int64_t p = 0; p < np; ++p) out[p] = 0.0;
  for (int32_t l = 0; l < n_levels(d); ++l) {
    orc_apply_KT(d, l, y, t);
    for (int64_t p = 0; p < np; ++p) out[p] += prob(d, l) * t[p];
  }
  free(t);
}

/* Conjugate gradients on (Kbar^T Kbar + mu I) x = Kbar^T b from x = 0, stopped
 * when the residual falls below tol times the right-hand side. */
int32_t orc_solve_quadratic(const orc_desc *d, const double *b, int32_t max_iter, double tol,
                            double *x) {
  const int64_t np = n_pix(d), m = n_meas(d);
  double *rhs = dalloc(np), *r = dalloc(np), *p = dalloc(np), *Ap = dalloc(np), *t = dalloc(m);
  apply_KbarT(d, b, rhs);
  for (int64_t i = 0; i < np; ++i) {
    x[i] = 0.0;
    r[i] = rhs[i];
    p[i] = r[i];
  }
  double rr = dot(r, r, np), r0 = sqrt(dot(rhs, rhs, np));
  int32_t it = 0;
  for (; it < max_iter && sqrt(rr) > tol * r0; ++it) {
    apply_Kbar(d, p, t);
    apply_KbarT(d, t, Ap);
    for (int64_t i = 0; i < np; ++i) Ap[i] += d->mu * p[i];
    double alpha = rr / dot(p, Ap, np);
    for (int64_t i = 0; i < np; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    double rr2 = dot(r, r, np);
    for (int64_t i = 0; i < np; ++i) p[i] = r[i] + (rr2 / rr) * p[i];
    rr = rr2;
  }
  free(rhs);
  free(r);
  free(p);
  free(Ap);
  free(t);
  return it;
}

/* 1/2 |Kbar x - b|^2 + R(x), the objective of eq. min_obj_new. */
double orc_objective(const orc_desc *d, const double *b, const double *x) {
  const int64_t m = n_meas(d);
  double *t = dalloc(m);
  apply_Kbar(d, x, t);
  double s = 0.0;
  for (int64_t q = 0; q < m; ++q) s += (t[q] - b[q]) * (t[q] - b[q]);
  free(t);
  return 0.5 * s + orc_regulariser(d, x);
}
