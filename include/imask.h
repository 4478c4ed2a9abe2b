/*
 * imask.h -- C ABI of libimask.so, the GB300 (sm_103a) hot path of ImaSk.
 *
 * ImaSk (A. Perelli, C.-B. Schoenlieb, M. J. Ehrhardt, "ImaSk: Stochastic
 * Multiresolution Image Sketching for Inverse Imaging Problems") solves
 *     min_x 1/2 |K x - b|^2 + R(x)                            (eq. min_obj)
 * through the sketched problem min_x 1/2 |sum_i p_i K_i x - b|^2 + R(x)
 * (eq. min_obj_new) with the SAGA-type primal-dual iteration of Alg. 1: at
 * every iteration one resolution level is drawn at random and only that
 * level's operator K_i and its adjoint are applied.
 *
 * Levels.  ell = 0..levels-1.  ell = 0 is the full-resolution compensated
 * sketch K_0 = K S_r with S_r = p_0^{-1}(I - sum_{ell>=1} p_ell T_ell^* T_ell)
 * (the paper's i = r, Sec. 4.1); ell >= 1 is K_ell = R_ell T_ell, the block
 * mean over 2^ell x 2^ell blocks followed by the projector on the grid of side
 * n / 2^ell (eq. CT_sketches).  ell = -1 selects the plain operator K.
 *
 * Layouts.  Images are row-major float[n][n]; pixel (i, c) is centred at
 * (x_c, y_i) = (-W/2 + (c + 1/2) h, -W/2 + (i + 1/2) h) with h = W / n.
 * Sinograms are row-major float[n_angles][n_det].  The projector is Joseph's
 * method (linear interpolation along the major axis of every ray); the
 * back-projector is its exact transpose: every pixel's owner thread applies
 * the rays crossing its tile into private shared-memory accumulators, no
 * atomics, partial images added in a fixed order (parallel-beam plans may
 * instead gather over bins pixel by pixel: imask_desc.bp_gather).
 *
 * Conventions.
 *  - Pointers named *_dev are device pointers owned by the caller; the library
 *    never frees them.  Plans and states own their internal buffers.
 *  - Every call is asynchronous and ordered on the stream it is given (a
 *    cudaStream_t passed as void*; NULL is the legacy default stream), except
 *    where a call says it synchronises.
 *  - Functions never abort.  On error they return a status other than
 *    IMASK_OK, record a message readable with imask_last_error() in the
 *    calling thread, and leave their outputs unspecified.
 *  - A plan is read-only after creation and may be shared between threads.
 *    A state belongs to one caller at a time.
 *  - n must be a multiple of 2^(levels-1) (IMASK_ERR_SHAPE otherwise); the
 *    paper assumes power-of-two sides (Sec. 4.1), multiples suffice here.
 */
#ifndef IMASK_H
#define IMASK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IMASK_OK = 0,
  IMASK_ERR_INVALID = 1,   /* bad argument or descriptor field */
  IMASK_ERR_SHAPE = 2,     /* n not a multiple of 2^(levels-1), sizes out of range */
  IMASK_ERR_OOM = 3,       /* device or host allocation failed */
  IMASK_ERR_CUDA = 4,      /* a CUDA runtime call failed */
  IMASK_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
  IMASK_ERR_NONFINITE = 6  /* a reduction met NaN or Inf */
} imask_status;

typedef struct imask_plan_s *imask_plan_t;   /* immutable geometry, levels, step size */
typedef struct imask_state_s *imask_state_t; /* one solve: x, y, SAGA tables, counter */
typedef struct imask_batch_s *imask_batch_t; /* states advanced together by CUDA graphs */

/* Problem description.  Geometry (Sec. 4.1-4.2): parallel beam, or fan beam
 * with a flat detector.  View a is at angle angle_start + angle_span*a/n_angles.
 * Bin j sits at offset (j - (n_det-1)/2) * det_spacing; det_spacing <= 0 picks
 * h for parallel beam and h (src_dist + det_dist) / src_dist for fan beam.
 * Parallel ray (a, j): {P : <P, (cos, sin)> = offset}.  Fan ray (a, j): from the
 * source src_dist (cos, sin) to the bin centre -det_dist (cos, sin) +
 * offset (-sin, cos).  probs[ell] (NULL: uniform) are the p_ell of Alg. 1.
 * R(x) = mu/2 |x|^2 (reg 0) or mu/2 |x|^2 + tv_lambda sum sqrt(|grad x|^2 +
 * tv_eps^2) with forward differences (reg 1, prox by tv_inner FISTA steps),
 * or tv_lambda sum |grad x| restricted to x >= 0 (reg 2, the non-smooth TV
 * with nonnegativity of Sec. 4.5; prox by tv_inner steps of the fast gradient
 * projection on the dual; no quadratic term, mu only scales the primal step
 * sigma/mu -- the paper uses the TV weight itself there).
 * mu <= 0 picks mu = |K|^2 / 2.46^2; sigma <= 0 picks a step from power-method
 * estimates of L, Lbar, Lbar_p (Sec. 3.4-3.6) by step_rule: 0 the Thm. 3
 * optimum sigma*, 1 half of sigma*, 2 sigma_B = 1/(L^2 + 3 Lbar^2) (the comparison
 * step of Sec. 3.6); for variant 1 sigma <= 0 picks 0.05, the value the paper
 * found by grid search for Alg. 7.
 *
 * Iteration options (a zero-filled tail selects plain Alg. 1):
 *  variant      0: Alg. 1 (parallel primal and dual updates);
 *               1: Alg. 7, ImaSk-Seq: the dual update first (projector on the
 *               extrapolated iterate xbar), the back-projector on the new dual
 *               iterate, then xbar = x+ + theta (x+ - x).
 *  theta        the extrapolation weight of Alg. 7 (the paper uses 1).
 *  dual_tables  0: the measurement-side tables psi_l = K_l x (levels * m
 *               floats); 1: per level the sketched projector input of its
 *               last refresh (n^2 + sum_{l>=1} (n/2^l)^2 floats; the remark
 *               after Alg. 3), the projector then applies K_l to the
 *               difference.  Same iterates up to rounding.
 *  storage      format of the SAGA tables of Alg. 1: the measurement-side
 *               tables psi_l (dual_tables 0), the largest arrays of a solve,
 *               and the image-side tables phi_l (level 0 on the full grid,
 *               levels >= 1 on their own grids): 0 fp32, 1 bfloat16,
 *               2 binary16 (round to nearest even on store; all arithmetic in
 *               fp32, the projector and back-projector accumulating in fp32;
 *               xi and zeta take the refreshed value, the running means move
 *               by the stored value's change, so they stay the p-weighted
 *               sums of the stored tables).  Rounded tables move the fixed
 *               point by about the format's precision;
 *               imask_state_set_storage(state, 0, ...) switches a state to
 *               fp32 tables for a refinement sweep.
 *  bp_gather    1 (parallel beam, geometry 0, only; else IMASK_ERR_INVALID):
 *               the back-projector of every call and solve of the plan is
 *               pixel-driven -- each pixel adds Lambda(q - i) g y over the
 *               few bins of every view whose ray passes within one pixel of
 *               it (Joseph's weights, the transpose of the projector up to
 *               fp32 rounding of the pixel's local offsets, a few 1e-6 of a
 *               weight) -- instead of owner-computes (exact to the last bit).
 *               Fused batches (imask_batch_create_fused) refuse such plans;
 *               IMASK_ERR_SHAPE when a level's ray window per 16 x 32-pixel tile
 *               would exceed the kernel's staging (detector pitch far below
 *               the pixel width at coarse levels).  -1: for parallel beam the
 *               faster of the two forms -- with autotune = 1 both are timed
 *               at plan time (each with its own tuned splits, weighted by the
 *               level probabilities), else the pixel-driven one -- falling
 *               back to the owners where the windows do not fit; for fan beam
 *               the owners.  imask_plan_info.bp_gather reports the form.
 *  draws        0: one level per iteration (Alg. 1); 1: the primal level
 *               (back-projector, image-side tables) is drawn from a second
 *               SplitMix64 stream whose seed is the SplitMix64 finaliser of
 *               the seed, the dual level (projector) from the first
 *               (independent primal and dual samples, an open question of the
 *               paper's discussion, Sec. 6). */
typedef struct {
  int32_t n, n_angles, n_det, geometry;  /* geometry: 0 parallel, 1 fan */
  double fov, det_spacing, angle_start, angle_span, src_dist, det_dist;
  int32_t levels;                        /* r, 1..8 */
  const double *probs;                   /* host array of r entries, or NULL */
  int32_t reg;                           /* 0 quadratic, 1 + smoothed TV, 2 TV, x >= 0 */
  double mu, tv_lambda, tv_eps;
  int32_t tv_inner;
  double sigma;
  int32_t storage;                       /* tables: 0 fp32, 1 bf16, 2 fp16 (see below) */
  int32_t variant;                       /* 0 Alg. 1, 1 Alg. 7 */
  double theta;                          /* Alg. 7 extrapolation */
  int32_t dual_tables;                   /* 0 K_l x tables, 1 input snapshots */
  int32_t draws;                         /* 0 common level, 1 independent primal/dual */
  int32_t step_rule;                     /* sigma <= 0: 0 sigma*, 1 half, 2 sigma_B */
  int32_t power_iters;                   /* power-method iterations; 0 picks 100 */
  int32_t autotune;                      /* 1: time, per level at plan time, the
                                            back-projector's view-group split and
                                            the projector's strip height */
  int32_t bp_gather;                     /* parallel beam only: 1 computes K_l^T
                                            pixel by pixel (see below), 0 by the
                                            owners of tile segments, -1 picks */
} imask_desc;

/* Constants of a plan (Sec. 3.4-3.6): L = |sum p K_l| / sqrt(mu), Lbar,
 * Lbar_p; sigma, and theta, the contraction factor of Thm. 3 for that sigma
 * (0 when sigma was given or for variant 1). */
typedef struct {
  double mu, sigma, theta, L, Lbar, Lbar_p, norm_K;
  int64_t n_meas, n_pix;
  int32_t levels, n_xmajor_views_split; /* views whose rays change major axis */
  int64_t n_xmajor_rays;
  int64_t state_bytes;                  /* device bytes one imask_state_create allocates */
  int64_t plan_bytes;                   /* device bytes the plan holds */
  int32_t autotuned;                    /* 1 when the choices below were measured */
  int32_t bp_view_groups[8];            /* back-projector view groups per level */
  int32_t fp_strip_lines[8];            /* projector strip height (lines) per level */
  int32_t bp_gather;                    /* back-projector form in use: 1 pixel-driven, 0 owners */
} imask_plan_info;

/* Creates a plan: validates the descriptor, builds the per-ray geometry tables
 * in FP64 on the host, uploads them, and (when mu or sigma are <= 0) runs the
 * FP64 power method on the device and the Thm. 3 solver on the host.
 * Synchronises.  Errors: INVALID, SHAPE, OOM, CUDA. */
imask_status imask_plan(const imask_desc *desc, imask_plan_t *plan_out);
/* Frees a plan.  Synchronises the device first (states of the plan may have
 * work in flight on any stream); destroy the plan's states before it. */
imask_status imask_plan_destroy(imask_plan_t plan);
imask_status imask_plan_get_info(imask_plan_t plan, imask_plan_info *info);

/* Synchronises the device and reports IMASK_ERR_TIMEOUT if a projector
 * launch of this plan gave up a bounded wait for its image strips since the
 * last check (the flag is then cleared).  A library built with
 * -DIMASK_BOUNDS_CHECK also checks the kernels' computed indices, skips an
 * access out of its buffer and records it; such a record (of any plan) is
 * reported here as IMASK_ERR_INVALID and cleared. */
imask_status imask_plan_check(imask_plan_t plan);

/* Host copy of the per-view major-axis split that the plan uses: for view a,
 * rays j < split[a] are x-major iff first_x[a] != 0, the others the opposite
 * (x-major: |dir_x| >= |dir_y| in FP64).  Arrays of n_angles entries. */
imask_status imask_plan_axis_split(imask_plan_t plan, int32_t *split, int32_t *first_x);

/* Same tables computed on the host alone, without a device (for testing the
 * host geometry).  Errors: INVALID, SHAPE. */
imask_status imask_geometry_axis_split(const imask_desc *desc, int32_t *split, int32_t *first_x);

/* The back-projector's view groups, on the host alone: the views holding rays
 * of one major axis (role 0 x-major, 1 y-major) in increasing order, into
 * views[0 .. *n_views) (n_angles entries of room), and their split into
 * n_groups consecutive groups of about equal numbers of such rays, group g
 * being views[bounds[g] .. bounds[g + 1]) (n_groups + 1 entries; a view goes to
 * the group that holds the midpoint of its rays in the running count; groups
 * may be empty).  Plans use these groups for their per-level split counts.
 * Errors: INVALID, SHAPE. */
imask_status imask_geometry_view_groups(const imask_desc *desc, int32_t role, int32_t n_groups,
                                        int32_t *views, int32_t *n_views, int32_t *bounds);

/* Thm. 3 step size from given constants (host FP64, grid x grid search over
 * (c, rho) in (0, cbar) x (0, 1)): out = {sigma, theta, c, rho}. */
imask_status imask_optimal_step(double L, double Lbar, double Lbar_p, double p_min,
                                int32_t grid, double out[4]);

/* sino_dev[n_angles*n_det] = K_level x_dev[n*n] (eq. CT_sketches; level -1:
 * plain K).  Allocates its temporary images with cudaMallocAsync on stream. */
imask_status imask_project(imask_plan_t plan, int32_t level, const float *x_dev,
                           float *sino_dev, void *stream);

/* img_dev[n*n] = K_level^T y_dev: level >= 1: 4^-level T^*(R_level^T y);
 * level 0: S_r (K^T y); level -1: K^T y.  Owner-computes: each thread owns a
 * line segment of a tile and applies the rays crossing the tile to it in
 * private shared-memory accumulators (no atomics); the partial images of the
 * view groups are added in a fixed order (deterministic).
 * Allocates its coarse temporary with cudaMallocAsync on stream. */
imask_status imask_backproject(imask_plan_t plan, int32_t level, const float *y_dev,
                               float *img_dev, void *stream);

/* Same result as imask_backproject, without allocating: no cudaMalloc,
 * cudaMallocAsync or cudaFree, for callers that cannot allocate device memory
 * while they run (their own allocator has reserved the device memory, or an
 * allocation could stall or fail inside a latency-bound loop).  The paper has
 * no counterpart; this is a deployment variant.  The back-projector's partial
 * sums go to one fixed array inside the library (16 MiB of device memory,
 * 4 Mi floats, held by every GPU that loads the library until the process
 * exits); a plan whose scratch need exceeds it gets IMASK_ERR_SHAPE.  The
 * first call on each device looks up that array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is kept per device and CUDA context: after a cudaDeviceReset
 * (which also invalidates every plan) the first call in the new context
 * looks it up again.  All calls share the array and it keeps the last call's contents: calls
 * that may overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller. */
imask_status imask_backproject_noalloc(imask_plan_t plan, int32_t level, const float *y_dev,
                                       float *img_dev, void *stream);

/* The level stream of Alg. 1 (sampling step): out_dev[t] = ell_{k0+t} drawn on
 * the device from SplitMix64 output k0+t of `seed` against thresholds
 * round(2^53 * cumsum(p)) * 2^11.  Bit-exact with any other implementation of
 * that definition. */
imask_status imask_levels(imask_plan_t plan, uint64_t seed, int64_t k0, int64_t n,
                          int32_t *out_dev, void *stream);

/* Creates the state of one solve (Alg. 1 defaults: x = y = 0, tables 0, k = 0)
 * and copies b_dev[n_angles*n_det] (sinogram order, view-major).  Inside the
 * state the measurement-space vectors (b, y, the tables psi_l and their mean)
 * are kept in the plan's ray-list order, which the projector's epilogue
 * reads and writes without an index; imask_state_get returns them in
 * sinogram order.  Allocates with cudaMallocAsync on stream. */
imask_status imask_state_create(imask_plan_t plan, const float *b_dev, uint64_t seed,
                                imask_state_t *state_out, void *stream);
/* Advances the state by n_iters iterations (Alg. 1, or the plan's variant) on
 * stream.  Every call that takes a state and a stream (step, batch step, get,
 * save, load, set_storage) is ordered after the state's previous call even
 * when that one used another stream (an event joins the two), unless either
 * stream is being captured into a graph.  For Alg. 1 the state's own two side streams run the projector and
 * the back-projector concurrently with each other and with the previous
 * update, ordered by events as the data require; all work is joined into
 * `stream` before the call's last iteration ends, so later work on `stream`
 * sees the result.  Runs of 8 or more iterations replay a captured CUDA graph
 * of four iterations (as imask_batch_step does for a batch of this state
 * alone; the first such call captures it).  With kernel profiling at a period
 * of 4 or more, the profiled iterations are launched kernel by kernel and in
 * order on `stream` (so that their events time each kernel alone) and the
 * iterations between them replay the graph; at periods 1 to 3 every
 * iteration is launched kernel by kernel.  Results are the same either way. */
imask_status imask_step(imask_state_t state, int32_t n_iters, void *stream);

/* Batches of independent solves (the paper has no counterpart; this is the
 * batched form of the same iteration).  A batch holds n_states distinct
 * states, of the same or of different plans.  imask_batch_step advances every
 * state by n_iters iterations with the same result as imask_step on each:
 * four iterations of all states are captured once as one CUDA graph, each
 * state on its own branches so that the solves overlap on the device, and the
 * graph is replayed n_iters / 4 times on stream (the iteration counter is read
 * from a device copy held by each state); the remaining iterations run with
 * plain launches.  The graph is captured again when a state's dual ping-pong
 * parity differs from the captured one (after an odd number of steps) or its
 * buffers moved (imask_state_set_storage).
 * Capture happens inside the call, on a stream the batch owns (relaxed
 * capture mode); the graph is then launched on `stream`, which may be the
 * legacy default stream.  Profiling events are not recorded in graphs.
 * Destroy a batch before its states.  Errors: INVALID, OOM, CUDA. */
imask_status imask_batch_create(const imask_state_t *states, int32_t n_states,
                                imask_batch_t *batch_out);
/* A fused batch: the same results as imask_batch_create's (bit for bit: the
 * same per-solve work in the same order), with one projector, one
 * back-projector and one update launch per iteration for all n_states
 * states, whose sizes, view counts and level sets may all differ.  The
 * projector and update grids are the solves' own grids one after the other;
 * the back-projector runs resident CTAs that take (solve, tile, view group)
 * items from a device counter, the solves' items listed at the levels drawn
 * for the iteration (a one-CTA planner launch writes the list), so that the
 * coarse levels of some solves fill the GPU beside the fine levels of
 * others.  Four iterations of these launches are captured as one CUDA graph
 * and replayed, as for imask_batch_create.  The states must use the quadratic
 * regulariser (reg = 0); at most 1024 states.  Errors: INVALID, OOM, CUDA. */
imask_status imask_batch_create_fused(const imask_state_t *states, int32_t n_states,
                                      imask_batch_t *batch_out);
imask_status imask_batch_step(imask_batch_t batch, int32_t n_iters, void *stream);
imask_status imask_batch_destroy(imask_batch_t batch);
/* Iteration counter k of the state (host value, no synchronisation). */
int64_t imask_state_iteration(imask_state_t state);
/* Copies a part of the state into dst_dev (float): what = 0 x[n*n], 1 y[m],
 * 2 the running mean sum_l p_l phi_l [n*n], 3 the running mean sum_l p_l psi_l [m]
 * (the measurement-space parts 1 and 3 in sinogram order). */
imask_status imask_state_get(imask_state_t state, int32_t what, float *dst_dev, void *stream);
imask_status imask_state_get_x(imask_state_t state, float *x_dev, void *stream);
/* Checkpoints.  imask_state_save writes the whole state (iterates, tables,
 * running means, sketch images, b, the iteration counter, the seeds and the
 * dual ping-pong parity) into dst_dev, a device buffer of
 * imask_state_checkpoint_bytes(state) bytes, ordered after the state's work
 * and on stream; the state's later calls, on any stream, come after the
 * copy.  The header carries a fingerprint of the saving state's plan: the
 * descriptor, the derived mu, sigma and theta, and every level's
 * back-projector split and partial-image size.  imask_state_load restores
 * such a checkpoint into a state of the same plan, or of a plan with the same
 * fingerprint (built from the same descriptor on the same kind of device,
 * with the same autotuned splits); it synchronises stream and the state's
 * stream.  Stepping then continues exactly as the saved state would have, the
 * level streams being counter-based.  INVALID for a checkpoint of a plan with
 * another fingerprint or storage format, or for a state whose tables changed
 * storage (imask_state_set_storage). */
int64_t imask_state_checkpoint_bytes(imask_state_t state);
imask_status imask_state_save(imask_state_t state, void *dst_dev, void *stream);
imask_status imask_state_load(imask_state_t state, const void *src_dev, void *stream);
/* Converts the state's SAGA tables (measurement- and image-side) to another
 * storage format (0 fp32, 1 bf16, 2 fp16) and re-forms their running means
 * from the converted tables; later iterations use the new format (widening to
 * fp32 is exact: the refinement sweep of a 16-bit solve).  Allocates the new
 * tables with cudaMallocAsync on stream.  INVALID for a snapshot-form state
 * (no measurement-side tables) unless storage is 0.  Graphs captured for the state (its own, or a batch's) are
 * captured again at their next step.  Not to be called while a batch holding
 * the state is being stepped from another thread. */
imask_status imask_state_set_storage(imask_state_t state, int32_t storage, void *stream);
/* Frees the state's buffers (stream-ordered on the stream last used). */
imask_status imask_state_destroy(imask_state_t state);

/* Whole solve: state_create, iters steps, copy x to x_dev, destroy. */
imask_status imask_solve(imask_plan_t plan, const float *b_dev, uint64_t seed, int32_t iters,
                         float *x_dev, void *stream);

/* PDHG (Chambolle & Pock 2011), the comparison method of Sec. 5 and a
 * generator of reference solutions, on the plan's sketched problem
 * min_x 1/2 |Kbar x - b|^2 + R(x), Kbar = sum_l p_l K_l (= K for one level):
 *   y+ = (y + s (Kbar xbar - b)) / (1 + s);  x+ = prox_{t R}(x - t Kbar^T y+);
 *   xbar = x+ + theta (x+ - x), from x = xbar = y = 0.
 * Every iteration applies every level's projector and back-projector.
 * x_dev[n*n] receives x after iters iterations.  Allocates its work buffers
 * with cudaMallocAsync on stream.  Errors: INVALID, OOM, CUDA. */
imask_status imask_pdhg(imask_plan_t plan, const float *b_dev, int32_t iters, double s,
                        double t, double theta, float *x_dev, void *stream);
/* The PDHG parameters printed with that comparison (for a mu-strongly convex
 * R): kappa = sqrt(1 + norm_K^2 / (mu rho^2)), s = 1/(kappa - 1),
 * t = 1/((kappa - 1) mu), theta = 1 - 2/(1 + kappa); the paper uses rho = 0.99.
 * out = {s, t, theta}.  Host only. */
imask_status imask_pdhg_params(double norm_K, double mu, double rho, double out[3]);

/* Metrics in FP64 on the device (synchronise; results on the host).
 * Objective of eq. min_obj_new: 1/2 |sum_l p_l K_l x - b|^2 + R(x). */
imask_status imask_objective(imask_plan_t plan, const float *x_dev, const float *b_dev,
                             double *out, void *stream);
/* |a - b|^2 / |b|^2 over n floats (IMASK_ERR_NONFINITE on NaN/Inf). */
imask_status imask_rel_distance(int64_t n, const float *a_dev, const float *b_dev, double *out,
                                void *stream);

/* Kernel timing for roofline reports.  While enabled (period >= 1), the
 * projector, back-projector and update launches of every period-th iteration
 * of imask_step (iteration counter k with k % period == 0), and every launch
 * of imask_project / imask_backproject, are bracketed by CUDA events on their
 * stream; period 0 disables.  Sampling keeps the events' own cost out of most
 * iterations.  imask_profile_read synchronises those events and returns, per
 * kind (0 forward projection, 1 back-projection, 2 primal update) and level
 * (0..7), the total milliseconds and launch counts accumulated since the last
 * reset: ms[kind*8 + level], count[kind*8 + level]. */
imask_status imask_profile_enable(int32_t period);
imask_status imask_profile_read(double ms[24], int64_t count[24], int32_t reset);
/* Failure-detection self-test (the paper has no counterpart): one projector
 * launch whose first image strip is never requested, so that every CTA's
 * bounded wait for it runs out; the CTAs record the failure in the plan's
 * error flag, let their other copies land and return.  The next
 * imask_plan_check reports IMASK_ERR_TIMEOUT (and clears the flag); the plan
 * stays usable.  No GPU fault or hang is involved.  Allocates scratch with
 * cudaMallocAsync on stream. */
imask_status imask_selftest_projector_timeout(imask_plan_t plan, void *stream);

/* Measured shared-memory ceilings of the current GPU, for roofline reports
 * (the paper has no counterpart): out[0] = GB/s of conflict-free 32-bit loads,
 * out[1] = GB/s (read + write bytes) of read-modify-writes of private slots,
 * the back-projector's access pattern; every SM runs 8 CTAs of 256 threads
 * with 8 independent access chains each, best of 3 timed launches.
 * Synchronises.  Errors: INVALID, CUDA. */
imask_status imask_probe_smem(double out[2], void *stream);
/* Number of kernels this library has launched in the process so far. */
int64_t imask_launch_count(void);

const char *imask_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
