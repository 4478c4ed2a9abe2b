/*
 * imask_oracle.h -- plain FP64 CPU oracle for the ImaSk hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the smoke check and the CPU-baseline legs of
 * the benchmark do.  It shares no header, helper, table or constant with the
 * CUDA library; the two agree only because both follow the same definitions.
 *
 * Paper: A. Perelli, C.-B. Schoenlieb, M. J. Ehrhardt, "ImaSk: Stochastic
 * Multiresolution Image Sketching for Inverse Imaging Problems".
 *
 * Conventions (level index ell = 0..r-1):
 *   ell = 0      the full-resolution compensated sketch (the paper's i = r):
 *                K_0 = K S_r,  S_r = p_0^{-1} (I - sum_{ell>=1} p_ell T_ell^* T_ell)
 *   ell >= 1     the paper's i = ell: K_ell = R_ell T_ell on the grid of side
 *                N / 2^ell (Sec. 4.1, eq. CT_sketches)
 *   ell = -1     the plain full-resolution operator K (no sketch)
 * Images are row-major [N][N]; pixel (i, c) is centred at
 * (x_c, y_i) = (-W/2 + (c + 1/2) h, -W/2 + (i + 1/2) h), h = W / N.
 * Sinograms are row-major [n_angles][n_det].
 */
#ifndef IMASK_ORACLE_H
#define IMASK_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n;            /* full image side N */
  int32_t n_angles;     /* number of views */
  int32_t n_det;        /* detector bins per view */
  int32_t geometry;     /* 0 parallel beam, 1 fan beam with a flat detector */
  double fov;           /* field-of-view width W */
  double det_spacing;   /* bin pitch; <= 0 selects the default rule */
  double angle_start;   /* first view angle (radians) */
  double angle_span;    /* views are angle_start + angle_span * a / n_angles */
  double src_dist;      /* fan: source to centre */
  double det_dist;      /* fan: centre to detector */
  int32_t levels;       /* r */
  const double *probs;  /* p_ell, ell = 0..r-1; NULL selects uniform 1/r */
  int32_t reg;          /* 0: R = mu/2 |x|^2; 1: plus lambda * smoothed TV;
                           2: lambda * TV with x >= 0 (no quadratic term) */
  double mu;            /* strong convexity of R */
  double tv_lambda;     /* smoothed-TV weight */
  double tv_eps;        /* smoothed-TV epsilon */
  int32_t tv_inner;     /* FISTA steps used for the TV prox */
  double sigma;         /* step size of Alg. 1 */
} orc_desc;

/* ---- level draw (Alg. 1, sampling step) ---- */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t k);
void orc_level_thresholds(const orc_desc *d, uint64_t *thr /* r-1 entries */);
int32_t orc_level(const orc_desc *d, uint64_t seed, uint64_t k);
void orc_levels(const orc_desc *d, uint64_t seed, uint64_t k0, int64_t n, int32_t *out);

/* ---- geometry and Joseph projector (Sec. 4.1 / 4.2) ---- */
double orc_det_spacing(const orc_desc *d);
void orc_ray(const orc_desc *d, int32_t a, int32_t j, double p0[2], double dir[2]);
int32_t orc_ray_is_xmajor(const orc_desc *d, int32_t a, int32_t j);
double orc_joseph_ray(const orc_desc *d, int32_t nl, const double *img, int32_t a, int32_t j);
void orc_joseph_fp(const orc_desc *d, int32_t nl, const double *img, double *sino);
void orc_joseph_bp(const orc_desc *d, int32_t nl, const double *sino, double *img);

/* ---- image-domain sketches (Sec. 4.1) ---- */
void orc_block_mean(int32_t n, int32_t ell, const double *x, double *out);   /* T_ell */
void orc_replicate(int32_t n, int32_t ell, const double *c, double *out);    /* T_ell^* */
void orc_compensate(const orc_desc *d, const double *x, double *out);        /* S_r */
void orc_apply_K(const orc_desc *d, int32_t ell, const double *x, double *sino);
void orc_apply_KT(const orc_desc *d, int32_t ell, const double *y, double *img);

/* ---- prox of tau * R (eq. prox_op; Sec. 4.5 for the TV part) ---- */
void orc_prox(const orc_desc *d, double tau, const double *v, double *out);
double orc_regulariser(const orc_desc *d, const double *x);

/* ---- Alg. 1 ---- */
/* Runs iterations k0 .. k0+iters-1 of Alg. 1 in place on the state
 * (x[d], y[m], phi[r*d], psi[r*m]); all-zero arrays are the defaults of Alg. 1.
 * levels_out (may be NULL) receives the drawn levels.  Returns 0 on success. */
int32_t orc_imask_run(const orc_desc *d, const double *b, uint64_t seed, int64_t k0,
                      int32_t iters, double *x, double *y, double *phi, double *psi,
                      int32_t *levels_out);

/* ---- Alg. 7 (ImaSk-Seq) ---- */
/* Iterations k0 .. k0+iters-1 of Alg. 7 in place on (x[d], xbar[d], y[m],
 * phi[r*d], psi[r*m]); theta is the extrapolation weight.  Returns 0. */
int32_t orc_imask_seq_run(const orc_desc *d, const double *b, uint64_t seed, int64_t k0,
                          int32_t iters, double theta, double *x, double *xbar, double *y,
                          double *phi, double *psi, int32_t *levels_out);

/* ---- variants on one loop ---- */
typedef struct {
  int32_t sequential;  /* 0: Alg. 1 order; 1: Alg. 7 order with extrapolation */
  double theta;        /* Alg. 7 extrapolation weight */
  int32_t snapshots;   /* 1: dual tables kept as projector-input snapshots */
  int32_t independent; /* 1: primal level drawn from the stream of orc_primal_seed(seed) */
  int32_t storage;     /* SAGA tables (measurement- and image-side) held as 0 FP64,
                          1 bfloat16, 2 binary16 */
} orc_variant;

/* Round-to-nearest-even of v to a binary format with `bits` significant bits
 * and minimum normal exponent emin (bfloat16: 8, -126; binary16: 11, -14). */
double orc_round_format(double v, int32_t bits, int32_t emin);

uint64_t orc_primal_seed(uint64_t seed);
/* State: x[d], xbar[d] (sequential), y[m], phi[r*d], and either psi[r*m]
 * (snapshots = 0) or snap[r*d] with psi_mean[m] (snapshots = 1); unused
 * arrays may be NULL.  levels_dual / levels_primal may be NULL.  Returns 0,
 * 1 for a non-positive sigma or mu, 2 for a missing array. */
int32_t orc_imask_variant_run(const orc_desc *d, const orc_variant *var, const double *b,
                              uint64_t seed, int64_t k0, int32_t iters, double *x, double *xbar,
                              double *y, double *phi, double *psi, double *snap,
                              double *psi_mean, int32_t *levels_dual, int32_t *levels_primal);

/* ---- PDHG (Sec. 5 comparison, x_nat generator) on Kbar = sum_l p_l K_l ---- */
void orc_pdhg_params(double norm_K, double mu, double rho, double out[3]);
int32_t orc_pdhg_run(const orc_desc *d, const double *b, int32_t iters, double s, double t,
                     double theta, double *x, double *xbar, double *y);

/* ---- step-size theory (Sec. 3.4-3.6, Thm. 3) ---- */
/* Power method on sum_l w_l K_l^T K_l (transposed=0, size d) or
 * sum_l w_l K_l K_l^T (transposed=1, size m); cross=1 applies
 * (sum_l w_l K_l)^T (sum_l w_l K_l) instead.  Returns the largest eigenvalue. */
double orc_power_eig(const orc_desc *d, const double *w, int32_t cross, int32_t transposed,
                     int32_t iters);
/* The same three operator norms for r dense matrices mats[l] (dim_y x dim_x,
 * row-major), so that the Remark on identical operators can pin the code. */
void orc_constants_dense(const double *mats, int32_t r, const double *p, int32_t dim_x,
                         int32_t dim_y, double mu, int32_t iters, double out[3]);
void orc_constants(const orc_desc *d, int32_t iters, double out[3]);   /* L, Lbar, Lbar_p */
double orc_norm_K(const orc_desc *d, int32_t iters);                   /* ||K||, ell = -1 */
double orc_theta(double eta, double c, double rho, double L, double Lbar, double Lbar_p,
                 double pmin);
double orc_eta_opt(double c, double rho, double L, double Lbar, double Lbar_p, double pmin);
void orc_optimal_step(double L, double Lbar, double Lbar_p, double pmin, int32_t grid,
                      double out[4] /* sigma, theta, c, rho */);

/* ---- fixed point and metrics ---- */
/* x_nat = argmin 1/2 |Kbar x - b|^2 + mu/2 |x|^2 (quadratic R only) by CG. */
int32_t orc_solve_quadratic(const orc_desc *d, const double *b, int32_t max_iter, double tol,
                            double *x);
double orc_objective(const orc_desc *d, const double *b, const double *x);

#ifdef __cplusplus
}
#endif
#endif
