// imask_internal.h -- structures shared by the kernels and the host side of
// libimask.so.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/imask.h"

#define IMASK_MAX_LEVELS 8
#define IMASK_PAD 34           // zero entries before every padded image line
#define IMASK_PAD_END 18       // zero entries after every padded image line
#define FP_THREADS 512         // forward projector: threads per CTA
#define FP_RAYS 4              // forward projector: rays per thread
#define FP_CHUNK (FP_THREADS * FP_RAYS)
#define FP_STAGES 3            // TMA strip pipeline depth
#define FP_STAGE_FLOATS 9216   // 36 KB per strip buffer (4 lines of a 2048-wide level)
#ifndef BP_THREADS
#define BP_THREADS 256         // back-projector: threads per CTA
#endif
#define BP_W 16                // back-projector tile: lines along the major axis
#ifndef BP_SEG
#define BP_SEG 32              // back-projector tile: lines across (one owner segment)
#endif
#ifndef BP_SLOTS
#define BP_SLOTS 512           // back-projector: ray slots per staged chunk (2 per thread)
#endif
#define LBLOCK 16              // lines per local interpolation frame (see block_origin);
                               // equal to BP_W so a back-projector tile is one block
#define GW_TY 16               // gather back-projector: tile rows
#define GW_TX 32               // gather back-projector: tile columns
#ifndef GW_PR
#define GW_PR 1                // gather back-projector: pixel rows per thread
#endif
#ifndef GW_PC
#define GW_PC 2                // gather back-projector: pixel columns per thread
#endif
#define GW_THREADS ((GW_TY / GW_PR) * (GW_TX / GW_PC))
#define GW_SLOTS 4096          // gather back-projector: staged bins per chunk of views
#ifndef UPD_THREADS
#define UPD_THREADS 256        // sketch / update kernels: threads per CTA
#endif

// Per-view data for the back-projector's ray windows (32 bytes).
struct ViewInfo {
  float c, s;       // cos / sin of the view angle
  int xj0, xj1;     // x-major rays of the view: j in [xj0, xj1)
  int xoff;         // ray-list index of ray (a, xj0)
  int yj0, yj1;     // y-major rays: j in [yj0, yj1)
  int yoff;         // ray-list index of ray (a, yj0)
};

// Geometry of one level grid.  Index 0 of the tables below is the plain
// full-resolution grid (level -1), index ell + 1 is level ell.
struct LevelGeom {
  int nl;          // grid side
  int ls;          // padded line stride, nl + IMASK_PAD + IMASK_PAD_END
  int lines;       // lines allocated (a multiple of tc)
  int tc;          // lines per TMA strip
  float inv2l;     // 2^-ell (1 for level -1)
  float scale2l;   // 2^ell
  float hl;        // pixel width fov / nl
  float cmid;      // (nl - 1) / 2
  int bp_nm;       // back-projector tiles along the major axis (BP_W lines each)
  int bp_nc;       // back-projector tiles across it (BP_SEG lines each)
  int bp_vgo;      // back-projector view groups per major axis (partial sums)
  int bp_nv;       // largest number of views handled by one CTA
  int bp_order_off;  // this level's entries in DevPlan::bp_order
  int gw_max;      // gather back-projector: most bins of one view that cross a tile
  int gw_vc;       // gather back-projector: views staged together (GW_SLOTS / gw_max)
  int gw_nc;       // gather back-projector: most bins with weight per pixel and view
};

// Everything the kernels need about a plan (passed by value).
struct DevPlan {
  int n, n_angles, n_det, geometry, levels;
  int m, d;          // measurement and pixel counts
  int m_x;           // x-major rays (the first m_x entries of the ray list)
  float fov, inv_pitch, center, src_dist, sd_dist;
  float probs[IMASK_MAX_LEVELS];
  unsigned long long thr[IMASK_MAX_LEVELS];   // level thresholds (r - 1 used)
  LevelGeom lg[IMASK_MAX_LEVELS + 1];
  int upd_tile;      // fine-pixel tile side of the sketch / update kernels
  int bp_gather;     // 1: the pixel-driven back-projector (parallel beam), 0: owner scatter
  const float *view_da;   // parallel beam: per view, the change of a from one bin to the next
  int fp_chunk_x;    // projector: x-major rays per CTA (<= FP_CHUNK)
  int fp_chunk_y;    // projector: y-major rays per CTA (<= FP_CHUNK)
  const float4 *rays;      // ray list: (a_hi, t_hi, g, sino index bits)
  const float2 *rays_lo;   // ray list: (a_lo, t_lo), the low words of a and t
  const ViewInfo *views;   // per view
  // back-projector CTA order per level: (role * tiles + tile) codes, heaviest
  // (most rays to apply) first; the view groups of one code are adjacent
  const int *bp_order;
  // back-projector view groups.  bp_views[role * n_angles + i] lists the views
  // holding rays of that major axis (role 0: x-major); for level index li the
  // view group vg of a role covers list positions [b[vg], b[vg + 1]) with
  // b = bp_vb + (li * 2 + role) * (n_angles + 1), the groups holding about
  // equal numbers of rays
  const int *bp_views;
  const int *bp_vb;
};

// Padded level images: for every level index li (0: level -1, ell + 1: ell),
// an x-major copy (lines = columns, "T") and a y-major copy (lines = rows, "R").
struct PadSet {
  float *T[IMASK_MAX_LEVELS + 1];
  float *R[IMASK_MAX_LEVELS + 1];
};

// Level selection for a launch: fixed >= -1 uses that level, otherwise the
// level is drawn on the device from (seed, k) for the projector side and from
// (seed_x, k) for the back-projector / image side (seed_x = seed unless the
// primal and dual levels are drawn independently).
// The iteration counter is k, or *k_dev + k_add when k_dev is set (a
// device-resident counter, so that captured CUDA graphs can be replayed).
struct LevelSel {
  int fixed;
  unsigned long long seed;
  unsigned long long seed_x;
  long long k;
  const long long *k_dev;
  int k_add;
};

// Snapshot form of the measurement-side tables: per level the sketched
// projector input of its last refresh, level ell at snap + snap_off[ell]
// (n*n floats for ell = 0, (n >> ell)^2 for ell >= 1).  snap == nullptr: the
// sketch is written as is.
struct SnapArgs {
  float *snap;
  long long snap_off[IMASK_MAX_LEVELS];
};

// Projector input of Alg. 7: xbar = x + theta (x - x_prev); x_prev == nullptr
// (and theta unused) gives x itself.
struct ExtrapArgs {
  const float *x_prev;
  float theta;
};

// Dual epilogue (Alg. 1, the zeta and y updates) fused into the projector.
// A solve keeps its measurement-space vectors (y, b, the tables psi and their
// mean) in ray-list order: entry i belongs to ray i of DevPlan::rays.
struct DualArgs {
  int on;
  const float *y_in;
  float *y_out;
  const float *b;
  void *psi;         // table base, level ell at entry ell * m; nullptr: the
                     // projector output is already the table difference
  int psi_fmt;       // table entries: 0 float, 1 bfloat16, 2 binary16
  float *psi_mean;   // sum_l p_l psi_l
  float sigma, inv_1ps;
};

// Primal epilogue (Alg. 1, the xi and x updates) in the update kernel.
struct PrimalArgs {
  const float *g;    // R_ell^T y on the level grid as bp_vgo partial sums
  float *x;          // iterate, updated in place
  void *phi0;        // table entry of level 0 (n*n)
  void *phic;        // tables of levels >= 1, stored on their own grids, level
  long long phic_off[IMASK_MAX_LEVELS];   // ell at entry phic_off[ell]
  int phi_fmt;       // table entries: 0 float, 1 bfloat16, 2 binary16
  float *phi_mean;   // sum_l p_l phi_l (n*n)
  float tau;         // sigma / mu
  float inv_1ps;     // 1 / (1 + sigma)
  int prox_in_place; // 1: quadratic prox here; 0: store v, a TV prox follows
  float *x_prev;     // nullptr, or receives x^k (Alg. 7 with a TV prox)
  int extrapolate;   // 1: the fused sketch is of x+ + theta (x+ - x^k) (Alg. 7)
  float theta;
  SnapArgs snap;
};

// One solve of a fused batch: everything the projector, back-projector and
// update launches of one iteration need for it (the device copy of its plan
// and its buffers for the iteration's ping-pong parity).  A fused launch
// covers every solve of the batch, the CTAs of solve s after those of solves
// 0..s-1.
struct FusedSlice {
  DevPlan P;
  LevelSel sel;        // seed, device iteration counter and offset
  PadSet pads_fp;      // sketch images the projector reads
  PadSet pads_upd;     // sketch images the update writes
  DualArgs D;          // projector epilogue
  const float *y_bp;   // back-projector input (ray-list order)
  float *g;            // back-projector partial images
  PrimalArgs A;        // update
  unsigned int *err;
  int n_cta_x;         // projector CTAs of x-major rays
};
#define IMASK_MAX_FUSED 1024   // solves per fused batch

// ---- kernel launchers (kernels.cu) -------------------------------------------
extern "C++" {
int lvl_host_draw(const DevPlan &P, unsigned long long seed, long long k);
cudaError_t launch_levels(const DevPlan &P, unsigned long long seed, long long k0, long long n,
                          int *out, cudaStream_t st);
cudaError_t launch_sketch(const DevPlan &P, LevelSel sel, const float *x, PadSet pads,
                          ExtrapArgs ex, SnapArgs snap, cudaStream_t st);
unsigned long long primal_seed(unsigned long long seed);
cudaError_t launch_fp(const DevPlan &P, LevelSel sel, PadSet pads, float *sino, DualArgs dual,
                      int n_cta_x, int n_cta_y, unsigned int *err, cudaStream_t st,
                      int test_skip_first_strip = 0);
// y_list: y in ray-list order (a state's dual iterate) rather than (view, bin)
// order
cudaError_t launch_bp(const DevPlan &P, LevelSel sel, const float *y, int y_list, float *g,
                      unsigned int *err, cudaStream_t st);
// dst = src moved from (view, bin) order to ray-list order (to_list = 1) or back
cudaError_t launch_sino_order(const DevPlan &P, const float *src, float *dst, int to_list,
                              cudaStream_t st);
long long bp_smem_bytes(const DevPlan &P);
int bp_blocks_per_sm(long long dyn_smem);
cudaError_t launch_adjsketch(const DevPlan &P, int ell, const float *g, float *img,
                             cudaStream_t st);
cudaError_t launch_update(const DevPlan &P, LevelSel sel, PrimalArgs pa, int write_sketch,
                          PadSet pads, cudaStream_t st);
// Fused batches: one launch of each kernel for all n_slices solves.
// fp_start / upd_start[s] (device, n_slices + 1 entries): the first CTA of
// solve s.  The back-projector launches a one-CTA planner that writes the
// solves' item offsets at their drawn levels into bp_start (device,
// n_slices + 1 ints) and zeroes bp_counter (device int), then `grid` resident
// CTAs that take items from the counter.  smem sizes and nv_cap are the
// largest over the solves.
cudaError_t launch_fp_multi(const FusedSlice *recs, const int *fp_start, int n_slices,
                            int total_ctas, cudaStream_t st);
// max_items > 0: one CTA per item over a grid of max_items CTAs (those past
// the iteration's list return at once) instead of `grid` resident CTAs
cudaError_t launch_bp_multi(const FusedSlice *recs, int n_slices, int *bp_start, int *bp_counter,
                            int nv_cap, long long smem, int grid, int max_items,
                            cudaStream_t st);
int bp_multi_blocks_per_sm(long long dyn_smem);
cudaError_t launch_update_multi(const FusedSlice *recs, const int *upd_start, int n_slices,
                                int total_ctas, int smem, cudaStream_t st);
int upd_smem_bytes_of(const DevPlan &P);
// *k_dev += delta for the iteration counter of every solve (recs[s].sel.k_dev)
cudaError_t launch_counter_multi(const FusedSlice *recs, int n_slices, long long delta,
                                 cudaStream_t st);
cudaError_t launch_tv_prox(const DevPlan &P, float tau, float mu, float lam, float eps, int inner,
                           float *x, float *work, cudaStream_t st);
cudaError_t launch_tv_nonneg_prox(const DevPlan &P, float alpha, int inner, float *x, float *work,
                                  cudaStream_t st);
cudaError_t launch_pdhg_dual(long long m, const float *kx, const float *b, float s, float *y,
                             cudaStream_t st);
cudaError_t launch_pdhg_primal(long long d, float scale, float theta, float *xn, float *x,
                               float *xbar, cudaStream_t st);
cudaError_t launch_axpy(long long n, float alpha, const float *x, float *y, cudaStream_t st);
// *k_dev += delta (one thread), or *k_dev = value when set_value != 0
cudaError_t launch_counter(long long *k_dev, long long delta, int set_value, cudaStream_t st);
// dst[i] = src[i] converted between the table formats (0 float, 1 bfloat16, 2 binary16)
cudaError_t launch_convert(long long n, const void *src, int src_fmt, void *dst, int dst_fmt,
                           cudaStream_t st);
// flags of the index checks of a checked build (0 in the normal build)
cudaError_t read_index_check_flag(unsigned int *flags, bool clear);
// shared-memory bandwidth probe: blocks x 256 threads x iters x 8 accesses
cudaError_t launch_probe_smem(int blocks, int iters, int rmw, float *sink, cudaStream_t st);
// psi_mean = sum_l p_l psi_l over the level tables
cudaError_t launch_table_mean(const DevPlan &P, const void *psi, int fmt, float *psi_mean,
                              cudaStream_t st);
// phi_mean = sum_l p_l phi_l on the fine grid (level ell >= 1 replicated from
// its grid), phi0 / phic as in PrimalArgs
cudaError_t launch_phi_mean(const DevPlan &P, const void *phi0, const void *phic,
                            const long long *phic_off, int fmt, float *phi_mean,
                            cudaStream_t st);
cudaError_t launch_scale(long long n, float alpha, float *x, cudaStream_t st);
cudaError_t launch_fill(long long n, float v, float *x, cudaStream_t st);
cudaError_t launch_copy(long long n, const float *x, float *y, cudaStream_t st);
// FP64 reductions: out[0] = sum a*b (b may equal a), or sum (a-b)^2 and sum b^2.
cudaError_t launch_dot64(long long n, const float *a, const float *b, double *partial,
                         double *out, cudaStream_t st);
cudaError_t launch_diff64(long long n, const float *a, const float *b, double *partial,
                          double *out, cudaStream_t st);
cudaError_t launch_tv_value64(const DevPlan &P, const float *x, float eps, double *partial,
                              double *out, cudaStream_t st);
int reduce_blocks();
long long fp_smem_bytes();
int64_t launch_counter();
void count_launch();
void add_launches(int64_t n);   // may be negative (captured launches that did not run)
}
