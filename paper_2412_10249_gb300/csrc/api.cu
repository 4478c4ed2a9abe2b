// api.cu -- host side of libimask.so: the C ABI declared in include/imask.h.
//
// Plan creation builds the acquisition geometry in FP64 on the host (ray list
// with per-ray interpolation parameters, per-view major-axis split), uploads
// it, and estimates the step-size constants of Sec. 3.4 with the power method
// on the device (FP32 operators, FP64 reductions) before solving Thm. 3 on the
// host.  States hold one solve of Alg. 1; imask_step launches the three
// kernels of every iteration (see kernels.cu).
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "imask_internal.h"

// ===================================================================================
// errors
// ===================================================================================
namespace {

thread_local std::string t_err;

imask_status fail(imask_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return s;
}

imask_status cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(IMASK_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(IMASK_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
  } while (0)

inline size_t align64(size_t n) { return (n + 63) & ~(size_t)63; }

// NVTX range for tools that record them (header-only; no cost without a tool)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// ===================================================================================
// profiling: CUDA events around projector / back-projector / update launches
// ===================================================================================
struct ProfRec {
  int kind, level;
  cudaEvent_t a, b;
};

struct Profiler {
  std::mutex mu;
  std::atomic<bool> on{false};
  std::atomic<int> period{0};   // imask_step times the iterations with k % period == 0
  std::vector<cudaEvent_t> pool;
  std::vector<ProfRec> pending;
  double ms[24] = {0};
  int64_t count[24] = {0};

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
};

Profiler g_prof;

// Opens a timed region for (kind, level) on stream st; returns false when off.
struct ProfScope {
  bool active = false;
  ProfRec rec{};
  cudaStream_t st = nullptr;
  ProfScope(int kind, int level, cudaStream_t s, bool sampled = true) : st(s) {
    if (!sampled) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!g_prof.on || level < 0 || level > 7) return;
    rec.kind = kind;
    rec.level = level;
    rec.a = g_prof.get();
    rec.b = g_prof.get();
    if (!rec.a || !rec.b) return;
    active = cudaEventRecord(rec.a, st) == cudaSuccess;
  }
  ~ProfScope() {
    if (!active) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (cudaEventRecord(rec.b, st) == cudaSuccess) g_prof.pending.push_back(rec);
  }
};

}  // namespace

// ===================================================================================
// plan and state
// ===================================================================================
struct imask_plan_s {
  imask_desc desc{};
  std::vector<double> probs;
  DevPlan dp{};
  float4 *d_rays = nullptr;
  float2 *d_rays_lo = nullptr;
  ViewInfo *d_views = nullptr;
  int *d_bp_order = nullptr;
  float *d_view_da = nullptr;   // per view, a's step from one bin to the next (parallel)
  int *d_bp_views = nullptr;    // per role, the views holding rays of that role
  int *d_bp_vb = nullptr;       // per level and role, the view-group bounds
  std::vector<int> role_rays[2];   // rays of the role in each listed view
  size_t gcap = 0;   // floats of the back-projector's partial-sum buffer
  unsigned int *d_err = nullptr;
  std::vector<int> split, first_x;
  int n_cta_x = 0, n_cta_y = 0;
  int n_split_views = 0;
  double mu = 0, sigma = 0, theta = 0, L = 0, Lbar = 0, Lbar_p = 0, norm_K = 0;
  bool autotuned = false;
  // hash of everything that decides how a state's block is laid out and read
  // (descriptor, derived step size, per-level back-projector splits); a
  // checkpoint loads only into a state of a plan with the same value
  uint64_t fingerprint = 0;
};

struct imask_state_s {
  imask_plan_t plan = nullptr;
  unsigned long long seed = 0;
  long long k = 0;
  int cur = 0;
  cudaStream_t stream = nullptr;
  float *block = nullptr;
  unsigned long long seed_x = 0;   // primal level stream (= seed unless draws = 1)
  void *psi = nullptr;        // measurement-side tables (format psi_fmt), or nullptr
  int psi_fmt = 0;            // 0 float, 1 bfloat16, 2 binary16
  void *psi_block = nullptr;  // separate table allocation after a storage change
  void *phi_block = nullptr;  // idem for the image-side tables
  int phi_fmt = 0;            // image-side tables: 0 float, 1 bfloat16, 2 binary16
  float *x = nullptr, *y[2] = {nullptr, nullptr}, *b = nullptr,
        *psi_mean = nullptr, *phi_mean = nullptr, *g = nullptr,
        *tv = nullptr, *x_prev = nullptr;
  // image-side tables: level 0 at phi0 (n*n entries), level ell >= 1 on its
  // own grid at entry phic_off[ell] of phic (phic == phi0: one region)
  void *phi0 = nullptr, *phic = nullptr;
  long long phic_off[IMASK_MAX_LEVELS] = {0};
  SnapArgs snap{};   // dual_tables = 1: sketched projector inputs per level
  // padded sketch images: the projector of iteration k reads pads[k % 2], the
  // update writes the next sketch into pads[(k + 1) % 2] (one set, both
  // entries equal, for Alg. 7, whose launches run in order anyway)
  PadSet pads[2] = {};
  // Alg. 1: the projector runs on aux, concurrently with the back-projector
  // and the update on the caller's stream (fork / join events)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_fp = nullptr;
  // Alg. 1 across iterations: the back-projector of k + 1 runs on aux2 as soon
  // as the projector of k is done, beside the update of k; its partial images
  // alternate between g and g2 so the update of k can still read its own
  cudaStream_t aux2 = nullptr;
  cudaEvent_t ev_start = nullptr, ev_bp = nullptr, ev_upd[2] = {nullptr, nullptr};
  float *g2 = nullptr;
  long long *k_dev = nullptr;   // device copy of k for graph replays
  bool k_dev_stale = true;      // k advanced by eager launches since the last sync
  struct imask_batch_s *self_batch = nullptr;   // graph replays of this state alone
  int gen = 0;                  // bumped when buffers move; captured graphs go stale
  cudaEvent_t ev_order = nullptr;   // orders a call on a new stream after the last one
};

struct imask_batch_s {
  std::vector<imask_state_s *> states;
  cudaStream_t origin = nullptr;       // capture origin (the legacy stream cannot capture)
  std::vector<cudaStream_t> streams;   // capture branches, one per state
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> cur_at_capture;     // ping-pong parity the graph was captured for
  std::vector<int> gen_at_capture;     // state buffer generations it was captured with
  int unroll = 0;                      // iterations per replay (even)
  int64_t kernels_per_replay = 0;
  // fused mode: one projector, one back-projector and one update launch per
  // iteration for every state (see kernels.cu, k_fp_multi and friends)
  bool fused = false;
  std::vector<int> order;              // states by decreasing size (launch order)
  FusedSlice *d_recs = nullptr;        // [unroll][n] iteration records
  int *d_fp_start = nullptr;           // [n + 1] first projector CTA of each state
  int *d_upd_start = nullptr;          // [n + 1] first update CTA of each state
  int *d_bp_start = nullptr;           // [unroll][n + 1] back-projector item offsets
  int *d_bp_counter = nullptr;         // [unroll] back-projector work counters
  int fp_total = 0, upd_total = 0, upd_smem = 0, bp_grid = 0, nv_cap = 0;
  int bp_max_items = 0;   // one back-projector CTA per item (0: resident CTAs)
  long long bp_smem = 0;
  bool any_seq = false;                // some state runs Alg. 7
  cudaStream_t f_fp = nullptr, f_bp = nullptr;   // capture branches of the fused launches
  std::vector<cudaEvent_t> f_ev;       // [3 * unroll]: projector, back-projector, update done
};

namespace {

// ---------------------------------------------------------------------------------
// descriptor validation and host geometry (FP64)
// ---------------------------------------------------------------------------------
double pitch_of(const imask_desc &d) {
  if (d.det_spacing > 0.0) return d.det_spacing;
  double h = d.fov / (double)d.n;
  if (d.geometry == 0) return h;
  return h * (d.src_dist + d.det_dist) / d.src_dist;
}

imask_status validate(const imask_desc *d) {
  if (!d) return fail(IMASK_ERR_INVALID, "descriptor is NULL");
  if (d->n < 1 || d->n > 2048) return fail(IMASK_ERR_SHAPE, "n = %d outside [1, 2048]", d->n);
  if (d->n_angles < 1 || d->n_det < 1)
    return fail(IMASK_ERR_SHAPE, "n_angles and n_det must be positive");
  if ((long long)d->n_angles * d->n_det >= (1LL << 30))
    return fail(IMASK_ERR_SHAPE, "n_angles * n_det too large");
  if (d->geometry != 0 && d->geometry != 1)
    return fail(IMASK_ERR_INVALID, "geometry must be 0 (parallel) or 1 (fan)");
  if (!(d->fov > 0.0) || !isfinite(d->fov)) return fail(IMASK_ERR_INVALID, "fov must be > 0");
  if (d->levels < 1 || d->levels > IMASK_MAX_LEVELS)
    return fail(IMASK_ERR_INVALID, "levels = %d outside [1, %d]", d->levels, IMASK_MAX_LEVELS);
  if (d->n % (1 << (d->levels - 1)) != 0)
    return fail(IMASK_ERR_SHAPE, "n = %d is not a multiple of 2^(levels-1) = %d", d->n,
                1 << (d->levels - 1));
  if (d->probs) {
    double s = 0.0;
    for (int l = 0; l < d->levels; ++l) {
      if (!(d->probs[l] > 0.0 && d->probs[l] <= 1.0))
        return fail(IMASK_ERR_INVALID, "probs[%d] = %g outside (0, 1]", l, d->probs[l]);
      s += d->probs[l];
    }
    if (fabs(s - 1.0) > 1e-9) return fail(IMASK_ERR_INVALID, "probs sum to %.17g, not 1", s);
  }
  if (d->reg < 0 || d->reg > 2) return fail(IMASK_ERR_INVALID, "reg must be 0, 1 or 2");
  if (d->reg == 1 && (!(d->tv_eps > 0.0) || d->tv_lambda < 0.0 || d->tv_inner < 0))
    return fail(IMASK_ERR_INVALID, "smoothed TV needs tv_eps > 0, tv_lambda >= 0, tv_inner >= 0");
  if (d->reg == 2 && (!(d->tv_lambda >= 0.0) || d->tv_inner < 0))
    return fail(IMASK_ERR_INVALID, "TV with nonnegativity needs tv_lambda >= 0, tv_inner >= 0");
  if (d->storage < 0 || d->storage > 2)
    return fail(IMASK_ERR_INVALID, "storage must be 0 (fp32), 1 (bf16) or 2 (fp16)");
  if (d->storage != 0 && d->dual_tables == 1)
    return fail(IMASK_ERR_INVALID, "16-bit storage applies to the measurement-side tables, "
                                   "which the snapshot form does not keep");
  if (d->variant != 0 && d->variant != 1)
    return fail(IMASK_ERR_INVALID, "variant must be 0 (Alg. 1) or 1 (Alg. 7)");
  if (d->variant == 1 && !isfinite(d->theta))
    return fail(IMASK_ERR_INVALID, "theta must be finite");
  if (d->dual_tables != 0 && d->dual_tables != 1)
    return fail(IMASK_ERR_INVALID, "dual_tables must be 0 or 1");
  if (d->draws != 0 && d->draws != 1) return fail(IMASK_ERR_INVALID, "draws must be 0 or 1");
  if (d->step_rule < 0 || d->step_rule > 2)
    return fail(IMASK_ERR_INVALID, "step_rule must be 0, 1 or 2");
  if (d->autotune != 0 && d->autotune != 1) return fail(IMASK_ERR_INVALID, "autotune must be 0 or 1");
  if (d->bp_gather < -1 || d->bp_gather > 1)
    return fail(IMASK_ERR_INVALID, "bp_gather must be -1, 0 or 1");
  if (d->bp_gather == 1 && d->geometry != 0)
    return fail(IMASK_ERR_INVALID, "the pixel-driven back-projector (bp_gather) is for parallel "
                                   "beam only");
  if (d->power_iters < 0 || d->power_iters > 100000)
    return fail(IMASK_ERR_INVALID, "power_iters must be in [0, 100000]");
  if (d->geometry == 1) {
    if (!(d->src_dist > 0.5 * d->fov * 1.4142135623730951))
      return fail(IMASK_ERR_INVALID, "fan source must lie outside the field of view");
    if (d->det_dist < 0.0) return fail(IMASK_ERR_INVALID, "det_dist must be >= 0");
  }
  if (!(pitch_of(*d) > 0.0)) return fail(IMASK_ERR_INVALID, "detector pitch must be > 0");
  return IMASK_OK;
}

// Ray (a, j) as a point and a direction, in the same operation order as the
// definition in imask.h (the major-axis decision depends on the last bit).
void ray_geom(const imask_desc &d, double pitch, int a, int j, double p0[2], double dir[2],
              double *ca_out, double *sa_out) {
  double ang = d.angle_start + d.angle_span * (double)a / (double)d.n_angles;
  double s = ((double)j - 0.5 * (double)(d.n_det - 1)) * pitch;
  double ca = cos(ang), sa = sin(ang);
  if (d.geometry == 0) {
    p0[0] = s * ca;
    p0[1] = s * sa;
    dir[0] = -sa;
    dir[1] = ca;
  } else {
    double sx = d.src_dist * ca;
    double sy = d.src_dist * sa;
    double dx = -d.det_dist * ca - s * sa;
    double dy = -d.det_dist * sa + s * ca;
    p0[0] = sx;
    p0[1] = sy;
    dir[0] = dx - sx;
    dir[1] = dy - sy;
  }
  if (ca_out) *ca_out = ca;
  if (sa_out) *sa_out = sa;
}

// Per-view split: rays j < split[a] have major axis first_x[a] (1: x-major).
imask_status axis_split(const imask_desc &d, std::vector<int> &split, std::vector<int> &first_x) {
  const double pitch = pitch_of(d);
  split.assign(d.n_angles, d.n_det);
  first_x.assign(d.n_angles, 1);
  for (int a = 0; a < d.n_angles; ++a) {
    int first = -1, sp = d.n_det;
    for (int j = 0; j < d.n_det; ++j) {
      double p0[2], dir[2];
      ray_geom(d, pitch, a, j, p0, dir, nullptr, nullptr);
      int xm = fabs(dir[0]) >= fabs(dir[1]) ? 1 : 0;
      if (j == 0) {
        first = xm;
      } else if (xm != first && sp == d.n_det) {
        sp = j;
      } else if (sp != d.n_det && xm == first) {
        return fail(IMASK_ERR_INVALID,
                    "view %d: rays change major axis more than once (fan wider than 90 degrees)",
                    a);
      }
    }
    split[a] = sp;
    first_x[a] = first;
  }
  return IMASK_OK;
}

// thr[l] = round(2^53 * (p_0 + ... + p_l)) * 2^11, l = 0..r-2.
void level_thresholds(const std::vector<double> &p, unsigned long long *thr) {
  double cum = 0.0;
  for (size_t l = 0; l + 1 < p.size(); ++l) {
    cum += p[l];
    long long v = llround(cum * 9007199254740992.0);
    if (v >= 9007199254740992LL)
      thr[l] = ~0ull;
    else if (v <= 0)
      thr[l] = 0ull;
    else
      thr[l] = ((unsigned long long)v) << 11;
  }
}

LevelGeom level_geom(const imask_desc &d, int ell) {
  LevelGeom g{};
  const int sh = ell > 0 ? ell : 0;
  g.nl = d.n >> sh;
  g.ls = g.nl + IMASK_PAD + IMASK_PAD_END;
  // lines per TMA strip: a multiple of 4 that fits a stage buffer; among those,
  // the one with the least padding (every padded line is a full line of
  // samples for all rays) plus half a line per strip hand-over
  const int tmax = std::min(32, std::max(4, (FP_STAGE_FLOATS / g.ls) & ~3));
  int tc = tmax;
  double best = 1e30;
  for (int t = tmax; t >= 4; t -= 4) {
    const int strips = (g.nl + t - 1) / t;
    const double cost = (double)strips * t + 0.5 * strips;
    if (cost < best - 1e-9) {
      best = cost;
      tc = t;
    }
  }
  g.tc = tc;
  g.lines = (g.nl + tc - 1) / tc * tc;
  g.inv2l = (float)ldexp(1.0, -sh);
  g.scale2l = (float)ldexp(1.0, sh);
  g.hl = (float)(d.fov / (double)g.nl);
  g.cmid = 0.5f * (float)(g.nl - 1);
  g.bp_nm = (g.nl + BP_W - 1) / BP_W;
  g.bp_nc = (g.nl + BP_SEG - 1) / BP_SEG;
  g.bp_vgo = 1;   // chosen per device in imask_plan
  return g;
}

#ifndef IMASK_UPD_TILE_CAP
#define IMASK_UPD_TILE_CAP 32
#endif

// The largest power of two that divides n, is at least the coarsest block
// (2^(levels-1), which divides n) and at most the cap: the kernels index tile
// pixels with shifts and masks.  The tile size does not change any result
// (block means are over aligned blocks inside one tile whatever its size).
int update_tile(int n, int levels) {
  const int blk = 1 << (levels - 1);
  const int cap = std::max(IMASK_UPD_TILE_CAP, blk);
  int best = blk;
  while (2 * best <= cap && n % (2 * best) == 0) best *= 2;
  return best;
}

size_t pad_floats(const LevelGeom &g) { return align64((size_t)g.lines * g.ls); }

// Host copy of one state-or-scratch allocation plan.
struct Carve {
  size_t off = 0;
  size_t take(size_t n) {
    size_t o = off;
    off += align64(n);
    return o;
  }
};

// ---------------------------------------------------------------------------------
// scratch for the bare operators (padded images of every level + coarse output)
// ---------------------------------------------------------------------------------
struct Scratch {
  float *block = nullptr;
  PadSet pads{};
  float *g = nullptr;
  cudaStream_t st = nullptr;
};

// levels_mask bit li (level li-1) selects which padded images to allocate.
imask_status scratch_alloc(const imask_plan_s *p, unsigned levels_mask, bool with_g, cudaStream_t st,
                           Scratch &s) {
  Carve cv;
  size_t offT[IMASK_MAX_LEVELS + 1] = {0}, offR[IMASK_MAX_LEVELS + 1] = {0};
  for (int li = 0; li <= p->desc.levels; ++li) {
    if (!(levels_mask & (1u << li))) continue;
    const size_t f = pad_floats(p->dp.lg[li]);
    offT[li] = cv.take(f);
    offR[li] = cv.take(f);
  }
  size_t offg = with_g ? cv.take(p->gcap) : 0;
  const size_t total = std::max<size_t>(cv.off, 64);
  void *mem = nullptr;
  CK(cudaMallocAsync(&mem, total * sizeof(float), st), "cudaMallocAsync(scratch)");
  s.block = (float *)mem;
  s.st = st;
  CK(cudaMemsetAsync(mem, 0, total * sizeof(float), st), "cudaMemsetAsync(scratch)");
  for (int li = 0; li <= p->desc.levels; ++li) {
    if (!(levels_mask & (1u << li))) continue;
    s.pads.T[li] = s.block + offT[li];
    s.pads.R[li] = s.block + offR[li];
  }
  s.g = with_g ? s.block + offg : nullptr;
  return IMASK_OK;
}

void scratch_free(Scratch &s) {
  if (s.block) cudaFreeAsync(s.block, s.st);
  s.block = nullptr;
}

LevelSel fixed_level(int ell) {
  LevelSel s{};
  s.fixed = ell;
  return s;
}

DualArgs no_dual() {
  DualArgs d{};
  d.on = 0;
  return d;
}

// x <- prox_{tau R}(x) for the TV regularisers (x holds the prox input v);
// work: 5 n^2 floats.
cudaError_t launch_reg_prox(const imask_plan_s *p, float tau, float *x, float *work,
                            cudaStream_t st) {
  if (p->desc.reg == 1)
    return launch_tv_prox(p->dp, tau, (float)p->mu, (float)p->desc.tv_lambda,
                          (float)p->desc.tv_eps, p->desc.tv_inner, x, work, st);
  return launch_tv_nonneg_prox(p->dp, tau * (float)p->desc.tv_lambda, p->desc.tv_inner, x, work,
                               st);
}

// K_ell x -> sino using scratch pads (level index ell + 1 allocated).
imask_status apply_K(const imask_plan_s *p, int ell, const float *x, float *sino, Scratch &s,
                     cudaStream_t st) {
  const LevelSel sel = fixed_level(ell);
  CK(launch_sketch(p->dp, sel, x, s.pads, ExtrapArgs{}, SnapArgs{}, st), "sketch launch");
  {
    ProfScope ps(0, ell < 0 ? 0 : ell, st);
    CK(launch_fp(p->dp, sel, s.pads, sino, no_dual(), p->n_cta_x, p->n_cta_y, p->d_err, st),
       "projector launch");
  }
  return IMASK_OK;
}

imask_status apply_KT(const imask_plan_s *p, int ell, const float *y, float *img, Scratch &s,
                      cudaStream_t st) {
  const LevelSel sel = fixed_level(ell);
  {
    ProfScope ps(1, ell < 0 ? 0 : ell, st);
    CK(launch_bp(p->dp, sel, y, 0, s.g, p->d_err, st), "back-projector launch");
  }
  CK(launch_adjsketch(p->dp, ell, s.g, img, st), "adjoint sketch launch");
  return IMASK_OK;
}

// ---------------------------------------------------------------------------------
// Back-projector view groups: the views holding rays of one major axis are
// split into vgo consecutive groups of about equal numbers of rays (a view
// goes to the group that holds the midpoint of its rays in the running
// count).  Writes bounds[0..vgo] (positions in the role's view list) and
// returns the largest group.  Groups may be empty.
// ---------------------------------------------------------------------------------
// Per major axis (role 0: x-major), the views that hold rays of that axis and
// their ray counts, from the per-view split of the ray list.
void bp_role_lists(const std::vector<int> &split, const std::vector<int> &first_x, int n_det,
                   std::vector<int> views[2], std::vector<int> rays[2]) {
  for (int role = 0; role < 2; ++role) {
    views[role].clear();
    rays[role].clear();
  }
  for (int a = 0; a < (int)split.size(); ++a) {
    const int nx = first_x[a] ? split[a] : n_det - split[a];
    const int nr[2] = {nx, n_det - nx};
    for (int role = 0; role < 2; ++role)
      if (nr[role] > 0) {
        views[role].push_back(a);
        rays[role].push_back(nr[role]);
      }
  }
}

int bp_group_bounds(const std::vector<int> &rays, int vgo, int *bounds) {
  const int nv = (int)rays.size();
  long long tot = 0;
  for (int w : rays) tot += w;
  int g = 0, largest = 0, start = 0;
  bounds[0] = 0;
  long long acc = 0;
  for (int i = 0; i < nv; ++i) {
    const int gi = tot > 0 ? (int)std::min<long long>(vgo - 1, ((2 * acc + rays[i]) * vgo) / (2 * tot))
                           : 0;
    while (g < gi) {
      bounds[++g] = i;
      largest = std::max(largest, i - start);
      start = i;
    }
    acc += rays[i];
  }
  while (g < vgo) {
    bounds[++g] = nv;
    largest = std::max(largest, nv - start);
    start = nv;
  }
  return largest;
}

// Bounds of both roles for level index li into the plan's device table (on
// st), and the level's largest group.
imask_status upload_bp_groups(imask_plan_s *p, int li, cudaStream_t st) {
  LevelGeom &g = p->dp.lg[li];
  const int na = p->desc.n_angles;
  std::vector<int> b(2 * (size_t)(na + 1), 0);
  int largest = 1;
  for (int role = 0; role < 2; ++role)
    largest = std::max(largest, bp_group_bounds(p->role_rays[role], g.bp_vgo,
                                                b.data() + role * (na + 1)));
  g.bp_nv = largest;
  if (p->d_bp_vb)
    CK(cudaMemcpyAsync(p->d_bp_vb + (size_t)li * 2 * (na + 1), b.data(), b.size() * sizeof(int),
                       cudaMemcpyHostToDevice, st),
       "upload view groups");
  return IMASK_OK;
}

// ---------------------------------------------------------------------------------
// Plan-time autotuning of the back-projector's view-group split: for every
// level, K_ell^T (back-projector and the partial-image sum that consumes its
// output) is timed with CUDA events for split counts around the occupancy
// heuristic's choice, and the fastest is kept.
// ---------------------------------------------------------------------------------
imask_status autotune_bp(imask_plan_s *p, cudaStream_t st,
                         std::vector<float> *best_ms_out = nullptr) {
  DevPlan &dp = p->dp;
  if (best_ms_out) best_ms_out->assign(IMASK_MAX_LEVELS + 1, 0.0f);
  const int r = p->desc.levels, na = p->desc.n_angles;
  std::vector<int> cand[IMASK_MAX_LEVELS + 1];
  size_t gmax = p->gcap;
  for (int li = 0; li <= r; ++li) {
    const int base = dp.lg[li].bp_vgo;
    for (int v : {base, std::max(1, base / 2), std::max(1, (2 * base) / 3), (3 * base + 1) / 2,
                  2 * base}) {
      v = std::min(v, na);
      if (std::find(cand[li].begin(), cand[li].end(), v) == cand[li].end()) cand[li].push_back(v);
      gmax = std::max(gmax, (size_t)2 * v * dp.lg[li].nl * dp.lg[li].nl);
    }
  }
  const size_t d = dp.d, m = dp.m;
  Scratch sc;
  sc.st = st;
  Carve cv;
  const size_t o_g = cv.take(gmax), o_y = cv.take(m), o_img = cv.take(d);
  void *mem = nullptr;
  CK(cudaMallocAsync(&mem, cv.off * sizeof(float), st), "cudaMallocAsync(autotune)");
  float *B = (float *)mem;
  sc.g = B + o_g;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  imask_status rc = IMASK_OK;
  cudaError_t e = cudaMemsetAsync(mem, 0, cv.off * sizeof(float), st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int li = 1; li <= r && e == cudaSuccess && rc == IMASK_OK; ++li) {
    const int ell = li - 1;
    float best_ms = 1e30f;
    int best_v = dp.lg[li].bp_vgo;
    for (int v : cand[li]) {
      LevelGeom &g = dp.lg[li];
      g.bp_vgo = v;
      if ((rc = upload_bp_groups(p, li, st)) != IMASK_OK) break;
      if (bp_smem_bytes(dp) > 160 * 1024) continue;
      float ms = 0.0f, tot = 0.0f;
      for (int rep = 0; rep < 4 && rc == IMASK_OK && e == cudaSuccess; ++rep) {
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
        rc = apply_KT(p, ell, B + o_y, B + o_img, sc, st);
        if (rc != IMASK_OK) break;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        if (rep > 0) tot += ms;   // the first launch warms up
      }
      if (rc != IMASK_OK || e != cudaSuccess) break;
      if (tot < best_ms) {
        best_ms = tot;
        best_v = v;
      }
    }
    dp.lg[li].bp_vgo = best_v;
    if (best_ms_out) (*best_ms_out)[li] = best_ms;
    if (rc == IMASK_OK) rc = upload_bp_groups(p, li, st);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(mem, st);
  if (rc != IMASK_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  p->gcap = 0;
  for (int li = 0; li <= r; ++li)
    p->gcap = std::max(p->gcap, (size_t)2 * dp.lg[li].bp_vgo * dp.lg[li].nl * dp.lg[li].nl);
  p->autotuned = true;
  return IMASK_OK;
}

// ---------------------------------------------------------------------------------
// Plan-time autotuning of the projector's strip height: for every level the
// bare projector K_ell is timed with CUDA events for every strip height (a
// multiple of 4 lines) that fits a stage buffer, and the fastest is kept.  The
// strip height changes only how the image streams through shared memory (and
// how many zero lines pad the last strip), never a sample's value.
// ---------------------------------------------------------------------------------
imask_status autotune_fp(imask_plan_s *p, cudaStream_t st) {
  DevPlan &dp = p->dp;
  const int r = p->desc.levels;
  float *sino = nullptr;
  CK(cudaMallocAsync((void **)&sino, (size_t)dp.m * sizeof(float), st), "cudaMallocAsync(autotune)");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  imask_status rc = IMASK_OK;
  for (int li = 1; li <= r && e == cudaSuccess && rc == IMASK_OK; ++li) {
    LevelGeom &g = dp.lg[li];
    const int tmax = std::min(32, std::max(4, (FP_STAGE_FLOATS / g.ls) & ~3));
    const int t0 = g.tc;
    float best_ms = 1e30f;
    int best_t = t0;
    for (int t = 4; t <= tmax && e == cudaSuccess && rc == IMASK_OK; t += 4) {
      g.tc = t;
      g.lines = (g.nl + t - 1) / t * t;
      Scratch sc;
      if ((rc = scratch_alloc(p, 1u << li, false, st, sc)) != IMASK_OK) break;
      float ms = 0.0f, tot = 0.0f;
      for (int rep = 0; rep < 4; ++rep) {
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
        if ((e = launch_fp(dp, fixed_level(li - 1), sc.pads, sino, no_dual(), p->n_cta_x,
                           p->n_cta_y, p->d_err, st)) != cudaSuccess)
          break;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        if (rep > 0) tot += ms;   // the first launch warms up
      }
      scratch_free(sc);
      if (e == cudaSuccess && tot < best_ms) {
        best_ms = tot;
        best_t = t;
      }
    }
    g.tc = best_t;
    g.lines = (g.nl + best_t - 1) / best_t * best_t;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(sino, st);
  if (rc != IMASK_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "autotune (projector)");
  return IMASK_OK;
}

// ---------------------------------------------------------------------------------
// FP64 power method on the device (Sec. 3.6): largest eigenvalue of
// sum_l w_l K_l^T K_l (image space), sum_l w_l K_l K_l^T (measurement space), or
// (sum_l w_l K_l)^T (sum_l w_l K_l) (cross); level -1 alone when plain = true.
// ---------------------------------------------------------------------------------
struct PowerBuf {
  float *v = nullptr, *u = nullptr, *ti = nullptr, *tm = nullptr, *acc = nullptr;
  double *part = nullptr, *res = nullptr;
};

imask_status device_dot(const float *a, const float *b, long long n, PowerBuf &pb, cudaStream_t st,
                        double *out) {
  CK(launch_dot64(n, a, b, pb.part, pb.res, st), "dot launch");
  CK(cudaMemcpyAsync(out, pb.res, sizeof(double), cudaMemcpyDeviceToHost, st), "copy dot");
  CK(cudaStreamSynchronize(st), "sync dot");
  return IMASK_OK;
}

imask_status power_method(const imask_plan_s *p, const double *w, bool cross, bool meas_space,
                          bool plain, int iters, Scratch &s, PowerBuf &pb, cudaStream_t st,
                          double *lam_out) {
  const long long d = p->dp.d, m = p->dp.m;
  const long long n = (cross || !meas_space) ? d : m;
  const int r = plain ? 1 : p->desc.levels;
  // start vector 1 + cos(0.7 i) / 2, normalised
  std::vector<float> h(n);
  double nrm = 0.0;
  for (long long i = 0; i < n; ++i) {
    double v = 1.0 + 0.5 * cos(0.7 * (double)i);
    nrm += v * v;
    h[i] = (float)v;
  }
  nrm = sqrt(nrm);
  for (long long i = 0; i < n; ++i) h[i] = (float)((double)h[i] / nrm);
  CK(cudaMemcpyAsync(pb.v, h.data(), n * sizeof(float), cudaMemcpyHostToDevice, st), "upload v");
  double lam = 0.0;
  imask_status rc;
  for (int it = 0; it < iters; ++it) {
    CK(launch_fill(n, 0.0f, pb.u, st), "fill");
    if (cross) {
      CK(launch_fill(m, 0.0f, pb.acc, st), "fill");
      for (int l = 0; l < r; ++l) {
        if ((rc = apply_K(p, plain ? -1 : l, pb.v, pb.tm, s, st)) != IMASK_OK) return rc;
        CK(launch_axpy(m, (float)w[l], pb.tm, pb.acc, st), "axpy");
      }
      for (int l = 0; l < r; ++l) {
        if ((rc = apply_KT(p, plain ? -1 : l, pb.acc, pb.ti, s, st)) != IMASK_OK) return rc;
        CK(launch_axpy(d, (float)w[l], pb.ti, pb.u, st), "axpy");
      }
    } else if (!meas_space) {
      for (int l = 0; l < r; ++l) {
        if ((rc = apply_K(p, plain ? -1 : l, pb.v, pb.tm, s, st)) != IMASK_OK) return rc;
        if ((rc = apply_KT(p, plain ? -1 : l, pb.tm, pb.ti, s, st)) != IMASK_OK) return rc;
        CK(launch_axpy(d, (float)w[l], pb.ti, pb.u, st), "axpy");
      }
    } else {
      for (int l = 0; l < r; ++l) {
        if ((rc = apply_KT(p, plain ? -1 : l, pb.v, pb.ti, s, st)) != IMASK_OK) return rc;
        if ((rc = apply_K(p, plain ? -1 : l, pb.ti, pb.tm, s, st)) != IMASK_OK) return rc;
        CK(launch_axpy(m, (float)w[l], pb.tm, pb.u, st), "axpy");
      }
    }
    double vu = 0.0, uu = 0.0;
    if ((rc = device_dot(pb.v, pb.u, n, pb, st, &vu)) != IMASK_OK) return rc;
    if ((rc = device_dot(pb.u, pb.u, n, pb, st, &uu)) != IMASK_OK) return rc;
    if (!isfinite(vu) || !isfinite(uu))
      return fail(IMASK_ERR_NONFINITE, "power method met a non-finite value");
    lam = vu;
    if (!(uu > 0.0)) break;
    CK(launch_copy(n, pb.u, pb.v, st), "copy");
    CK(launch_scale(n, (float)(1.0 / sqrt(uu)), pb.v, st), "scale");
  }
  *lam_out = lam;
  return IMASK_OK;
}

imask_status plan_constants(imask_plan_s *p, cudaStream_t st) {
  const bool need_mu = !(p->desc.mu > 0.0);
  p->mu = p->desc.mu;
  p->sigma = p->desc.sigma;
  // Alg. 7 has no step-size theory; the paper tuned sigma = 0.05 by grid search
  if (p->desc.variant == 1 && !(p->sigma > 0.0)) p->sigma = 0.05;
  const bool need_sigma = !(p->sigma > 0.0);
  if (!need_mu && !need_sigma) return IMASK_OK;
  const int iters = p->desc.power_iters > 0 ? p->desc.power_iters : 100;
  const long long d = p->dp.d, m = p->dp.m;
  Scratch s;
  unsigned mask = 0;
  for (int li = 0; li <= p->desc.levels; ++li) mask |= 1u << li;
  imask_status rc = scratch_alloc(p, mask, true, st, s);
  if (rc != IMASK_OK) return rc;
  PowerBuf pb;
  void *mem = nullptr;
  // v, u: max(d, m) each; ti: d; tm, acc: m
  const size_t big = std::max(align64(d), align64(m));
  const size_t fl = 2 * big + align64(d) + 2 * align64(m);
  cudaError_t e = cudaMallocAsync(&mem, fl * sizeof(float) + 2048 * sizeof(double), st);
  if (e != cudaSuccess) {
    scratch_free(s);
    return cuda_fail(e, "cudaMallocAsync(power)");
  }
  float *f = (float *)mem;
  pb.v = f;
  pb.u = pb.v + big;
  pb.ti = pb.u + big;
  pb.tm = pb.ti + align64(d);
  pb.acc = pb.tm + align64(m);
  pb.part = (double *)((char *)mem + fl * sizeof(float));
  pb.res = pb.part + 1024;
  do {
    double one = 1.0, lam = 0.0;
    if ((rc = power_method(p, &one, true, false, true, iters, s, pb, st, &lam)) != IMASK_OK) break;
    p->norm_K = sqrt(lam);
    if (need_mu) p->mu = p->norm_K * p->norm_K / (2.46 * 2.46);
    if (!(p->mu > 0.0)) {
      rc = fail(IMASK_ERR_INVALID, "derived mu is not positive");
      break;
    }
    if (!need_sigma) break;
    const int r = p->desc.levels;
    double w1[IMASK_MAX_LEVELS], w2[IMASK_MAX_LEVELS];
    for (int l = 0; l < r; ++l) {
      w1[l] = p->probs[l];
      w2[l] = p->probs[l] * p->probs[l];
    }
    double lc = 0, lbx = 0, lby = 0, lpx = 0, lpy = 0;
    if ((rc = power_method(p, w1, true, false, false, iters, s, pb, st, &lc)) != IMASK_OK) break;
    if ((rc = power_method(p, w2, false, false, false, iters, s, pb, st, &lbx)) != IMASK_OK) break;
    if ((rc = power_method(p, w2, false, true, false, iters, s, pb, st, &lby)) != IMASK_OK) break;
    if ((rc = power_method(p, w1, false, false, false, iters, s, pb, st, &lpx)) != IMASK_OK) break;
    if ((rc = power_method(p, w1, false, true, false, iters, s, pb, st, &lpy)) != IMASK_OK) break;
    p->L = sqrt(lc / p->mu);
    p->Lbar = sqrt(std::max(lbx, lby) / p->mu);
    p->Lbar_p = sqrt(std::max(lpx, lpy) / p->mu);
    double pmin = 1.0;
    for (int l = 0; l < r; ++l) pmin = std::min(pmin, p->probs[l]);
    double out[4];
    imask_optimal_step(p->L, p->Lbar, p->Lbar_p, pmin, 200, out);
    p->sigma = out[0];
    p->theta = out[1];
    if (p->desc.step_rule == 1) {
      p->sigma = 0.5 * out[0];
      p->theta = 0.0;
    } else if (p->desc.step_rule == 2) {
      // the step of the SAGA primal-dual method the paper compares with
      p->sigma = 1.0 / (p->L * p->L + 3.0 * p->Lbar * p->Lbar);
      p->theta = 0.0;
    }
  } while (false);
  cudaFreeAsync(mem, st);
  scratch_free(s);
  if (rc == IMASK_OK) {
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e2 != cudaSuccess) return cuda_fail(e2, "plan constants");
  }
  if (rc == IMASK_OK && !(p->sigma > 0.0)) rc = fail(IMASK_ERR_INVALID, "no admissible step size");
  return rc;
}

}  // namespace

namespace {

// Float offsets of the parts of a state's single device allocation.
struct StateLayout {
  size_t x = 0, y0 = 0, y1 = 0, b = 0, psi = 0, psim = 0, phi0 = 0, phim = 0, xprev = 0, kdev = 0,
         g = 0, g2 = 0, tv = 0, total = 0;
  size_t snap[IMASK_MAX_LEVELS] = {0}, phic[IMASK_MAX_LEVELS] = {0};
  size_t T[IMASK_MAX_LEVELS + 1] = {0}, R[IMASK_MAX_LEVELS + 1] = {0};
  size_t T2[IMASK_MAX_LEVELS + 1] = {0}, R2[IMASK_MAX_LEVELS + 1] = {0};   // Alg. 1 only
};

StateLayout state_layout(const imask_plan_s *p) {
  StateLayout L;
  const int r = p->desc.levels;
  const size_t d = p->dp.d, m = p->dp.m;
  const bool snapshots = p->desc.dual_tables == 1;
  const bool seq = p->desc.variant == 1;
  Carve cv;
  L.x = cv.take(d);   // first: offset 0 marks "absent" for the optional parts below
  L.y0 = cv.take(m);
  L.y1 = cv.take(m);
  L.b = cv.take(m);
  const size_t esize = p->desc.storage != 0 ? 2 : 4;   // bytes per table entry
  L.psi = snapshots ? 0 : cv.take((m * r * esize + 3) / 4);
  L.psim = cv.take(m);
  // image-side tables, level 0 and then the coarse levels, in one region
  size_t phi_entries = d;
  for (int l = 1; l < r; ++l) phi_entries += (size_t)p->dp.lg[l + 1].nl * p->dp.lg[l + 1].nl;
  L.phi0 = cv.take((phi_entries * esize + 3) / 4);
  L.phim = cv.take(d);
  if (snapshots)
    for (int l = 0; l < r; ++l) {
      const size_t nl = (size_t)p->dp.lg[l + 1].nl;
      L.snap[l] = cv.take(nl * nl);
    }
  L.xprev = (seq && p->desc.reg != 0) ? cv.take(d) : 0;
  L.kdev = cv.take(2);   // one 64-bit counter
  L.g = cv.take(p->gcap);
  L.g2 = seq ? 0 : cv.take(p->gcap);
  L.tv = p->desc.reg != 0 ? cv.take(5 * d) : 0;
  for (int li = 1; li <= r; ++li) {
    L.T[li] = cv.take(pad_floats(p->dp.lg[li]));
    L.R[li] = cv.take(pad_floats(p->dp.lg[li]));
    if (!seq) {
      L.T2[li] = cv.take(pad_floats(p->dp.lg[li]));
      L.R2[li] = cv.take(pad_floats(p->dp.lg[li]));
    }
  }
  L.total = cv.off;
  return L;
}

}  // namespace

namespace {

// Back-projector CTA order per level (only the order changes, not the result):
// every (role, tile) is weighted by the rays its windows hold over a sample of
// the views, computed in FP64 with the kernel's window rule (bins of the tile
// box's corners, widened by one pixel across), and sorted heaviest first.
std::vector<int> bp_tile_order(const DevPlan &dp, const std::vector<ViewInfo> &views,
                               const imask_desc &d) {
  std::vector<int> all;
  const int na = d.n_angles;
  const int stride = std::max(1, na / 90);
  const double pitch = 1.0 / (double)dp.inv_pitch, center = dp.center;
  auto bin = [&](double c, double s, double x, double y) {
    if (d.geometry == 0) return (x * c + y * s) / pitch + center;
    const double num = -x * s + y * c, den = d.src_dist - (x * c + y * s);
    return (d.src_dist + d.det_dist) * num / den / pitch + center;
  };
  for (int li = 0; li <= d.levels; ++li) {
    const LevelGeom &g = dp.lg[li];
    const int nm = g.bp_nm, nc = g.bp_nc, ntile = nm * nc;
    const double W = d.fov, hl = W / (double)g.nl;
    std::vector<std::pair<double, int>> wts;
    for (int role = 0; role < 2; ++role)
      for (int tile = 0; tile < ntile; ++tile) {
        const int mb = tile % nm, cb = tile / nm;
        const int m0 = mb * BP_W, m1 = std::min(m0 + BP_W, g.nl) - 1;
        const int c0 = cb * BP_SEG, c1 = std::min(c0 + BP_SEG, g.nl) - 1;
        const double mlo = -0.5 * W + (m0 + 0.5) * hl, mhi = -0.5 * W + (m1 + 0.5) * hl;
        const double clo = -0.5 * W + (c0 + 0.5) * hl - hl, chi = -0.5 * W + (c1 + 0.5) * hl + hl;
        double w = 0.0;
        for (int a = 0; a < na; a += stride) {
          const ViewInfo &V = views[a];
          double mn = 1e30, mx = -1e30;
          for (int k = 0; k < 4; ++k) {
            const double mc = (k & 1) ? mhi : mlo, cc = (k & 2) ? chi : clo;
            const double j = role == 0 ? bin(V.c, V.s, mc, cc) : bin(V.c, V.s, cc, mc);
            mn = std::min(mn, j);
            mx = std::max(mx, j);
          }
          const int j0 = role == 0 ? V.xj0 : V.yj0, j1 = role == 0 ? V.xj1 : V.yj1;
          const double lo = std::max(std::ceil(mn), (double)j0);
          const double hi = std::min(std::floor(mx), (double)(j1 - 1));
          if (hi >= lo) w += hi - lo + 1.0;
        }
        wts.push_back(std::make_pair(-w, role * ntile + tile));
      }
    std::stable_sort(wts.begin(), wts.end());
    for (auto &e : wts) all.push_back(e.second);
  }
  return all;
}

}  // namespace

namespace {

// FNV-1a (64-bit) over the bytes of the values that fix a state's layout and
// meaning: the descriptor's scalars, the level probabilities, the derived mu,
// sigma and theta, and every level's back-projector split and the size of its
// partial-image buffer.
struct Fnv64 {
  uint64_t h = 0xcbf29ce484222325ull;
  void bytes(const void *p, size_t n) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 0x100000001b3ull;
  }
  template <class T> void add(const T &v) { bytes(&v, sizeof(T)); }
};

uint64_t plan_fingerprint(const imask_plan_s *p) {
  const imask_desc &d = p->desc;
  Fnv64 f;
  f.add(d.n); f.add(d.n_angles); f.add(d.n_det); f.add(d.geometry);
  f.add(d.fov); f.add(d.det_spacing); f.add(d.angle_start); f.add(d.angle_span);
  f.add(d.src_dist); f.add(d.det_dist); f.add(d.levels);
  f.add(d.reg); f.add(d.tv_lambda); f.add(d.tv_eps); f.add(d.tv_inner);
  f.add(d.storage); f.add(d.variant); f.add(d.dual_tables); f.add(d.draws); f.add(d.step_rule);
  for (double v : p->probs) f.add(v);
  f.add(p->mu); f.add(p->sigma); f.add(p->theta);
  for (int li = 0; li <= d.levels; ++li) {
    f.add(p->dp.lg[li].bp_vgo);
    f.add(p->dp.lg[li].tc);
  }
  f.add((uint64_t)p->gcap);
  return f.h;
}

// Orders the work that a call is about to enqueue on st after the state's
// earlier work, which ran on s->stream (the stream of its last call), when
// the two differ; the state then belongs to st.  Skipped while either stream
// is being captured into a graph (the capture's own dependencies order it).
imask_status state_use_stream(imask_state_s *s, cudaStream_t st) {
  if (s->stream == st) return IMASK_OK;
  cudaStreamCaptureStatus c0 = cudaStreamCaptureStatusNone, c1 = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &c0) == cudaSuccess &&
      cudaStreamIsCapturing(s->stream, &c1) == cudaSuccess &&
      c0 == cudaStreamCaptureStatusNone && c1 == cudaStreamCaptureStatusNone) {
    if (!s->ev_order)
      CK(cudaEventCreateWithFlags(&s->ev_order, cudaEventDisableTiming), "state order event");
    CK(cudaEventRecord(s->ev_order, s->stream), "state order");
    CK(cudaStreamWaitEvent(st, s->ev_order, 0), "state order");
  } else {
    cudaGetLastError();   // a failed query leaves no sticky error behind
  }
  s->stream = st;
  return IMASK_OK;
}

}  // namespace

// ===================================================================================
// C ABI
// ===================================================================================
extern "C" {

const char *imask_last_error(void) { return t_err.c_str(); }

int64_t imask_launch_count(void) { return launch_counter(); }

imask_status imask_geometry_axis_split(const imask_desc *desc, int32_t *split, int32_t *first_x) {
  imask_status rc = validate(desc);
  if (rc != IMASK_OK) return rc;
  if (!split || !first_x) return fail(IMASK_ERR_INVALID, "NULL output");
  std::vector<int> s, f;
  if ((rc = axis_split(*desc, s, f)) != IMASK_OK) return rc;
  for (int a = 0; a < desc->n_angles; ++a) {
    split[a] = s[a];
    first_x[a] = f[a];
  }
  return IMASK_OK;
}

imask_status imask_geometry_view_groups(const imask_desc *desc, int32_t role, int32_t n_groups,
                                        int32_t *views, int32_t *n_views, int32_t *bounds) {
  imask_status rc = validate(desc);
  if (rc != IMASK_OK) return rc;
  if (!views || !n_views || !bounds) return fail(IMASK_ERR_INVALID, "NULL output");
  if (role != 0 && role != 1) return fail(IMASK_ERR_INVALID, "role must be 0 or 1");
  if (n_groups < 1) return fail(IMASK_ERR_INVALID, "n_groups must be >= 1");
  std::vector<int> s, f;
  if ((rc = axis_split(*desc, s, f)) != IMASK_OK) return rc;
  std::vector<int> lists[2], rays[2];
  bp_role_lists(s, f, desc->n_det, lists, rays);
  std::vector<int> b((size_t)n_groups + 1);
  bp_group_bounds(rays[role], n_groups, b.data());
  *n_views = (int32_t)lists[role].size();
  for (size_t i = 0; i < lists[role].size(); ++i) views[i] = lists[role][i];
  for (int g = 0; g <= n_groups; ++g) bounds[g] = b[g];
  return IMASK_OK;
}

// Thm. 3 on the grid c = cbar (i + 1/2)/G, rho = (j + 1/2)/G: eta* = c when
// p_min > (Lbar^2/rho (1 - (1+L^2)c) / (1 - (1+L^2+Lbar_p^2)c) + 1 - rho) c,
// else the crossing (sqrt(1 + D (p_min + rho c)) - 1) / D, D = 1/alpha - 1/c;
// theta = max(phi(eta*), psi(eta*)); the best (c, rho) wins; sigma = eta/(1-eta).
imask_status imask_optimal_step(double L, double Lbar, double Lbar_p, double p_min, int32_t grid,
                                double out[4]) {
  if (!out) return fail(IMASK_ERR_INVALID, "NULL output");
  if (!(L > 0) || !(Lbar > 0) || !(Lbar_p > 0) || !(p_min > 0) || p_min > 1 || grid < 1)
    return fail(IMASK_ERR_INVALID, "optimal_step: invalid constants");
  const double L2 = L * L, Lb2 = Lbar * Lbar, Lp2 = Lbar_p * Lbar_p;
  const double cbar = 1.0 / (1.0 + L2 + Lp2);
  double best = INFINITY, best_eta = 0, best_c = 0, best_rho = 0;
  for (int i = 0; i < grid; ++i) {
    const double c = cbar * ((double)i + 0.5) / (double)grid;
    for (int j = 0; j < grid; ++j) {
      const double rho = ((double)j + 0.5) / (double)grid;
      const double ratio = (1.0 - (1.0 + L2) * c) / (1.0 - (1.0 + L2 + Lp2) * c);
      const double ainv = Lb2 / (rho * c) * ratio;
      double eta;
      if (p_min > (Lb2 / rho * ratio + 1.0 - rho) * c) {
        eta = c;
      } else {
        const double D = ainv - 1.0 / c;
        eta = (sqrt(1.0 + D * (p_min + rho * c)) - 1.0) / D;
      }
      const double phi = (eta - c) * (eta - c) / c + 1.0 - (1.0 - rho) * c;
      const double psi = ainv * eta * eta + 1.0 - p_min;
      const double th = phi > psi ? phi : psi;
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
  return IMASK_OK;
}

imask_status imask_plan(const imask_desc *desc, imask_plan_t *plan_out) {
  NvtxRange nv("imask_plan");
  if (!plan_out) return fail(IMASK_ERR_INVALID, "plan_out is NULL");
  *plan_out = nullptr;
  imask_status rc = validate(desc);
  if (rc != IMASK_OK) return rc;
  imask_plan_s *p = new (std::nothrow) imask_plan_s();
  if (!p) return fail(IMASK_ERR_OOM, "host allocation");
  p->desc = *desc;
  const int r = desc->levels;
  for (int l = -1; l < r; ++l) {
    const LevelGeom g = level_geom(*desc, l);
    if (g.tc * g.ls > FP_STAGE_FLOATS) {
      delete p;
      return fail(IMASK_ERR_SHAPE, "level %d is too wide for the projector's strip buffer", l);
    }
  }
  p->probs.resize(r);
  for (int l = 0; l < r; ++l) p->probs[l] = desc->probs ? desc->probs[l] : 1.0 / (double)r;
  p->desc.probs = nullptr;  // never keep the caller's pointer

  if ((rc = axis_split(*desc, p->split, p->first_x)) != IMASK_OK) {
    delete p;
    return rc;
  }
  // ray list: x-major rays in sinogram order, then y-major rays
  const int na = desc->n_angles, nd = desc->n_det;
  const double pitch = pitch_of(*desc);
  const double W = desc->fov, h = W / (double)desc->n;
  std::vector<float4> rays((size_t)na * nd);
  std::vector<float2> rays_lo((size_t)na * nd);
  std::vector<ViewInfo> views(na);
  std::vector<float> view_da(na, 0.0f);   // parallel beam: a's step per bin, per view
  std::vector<float> view_t(na, 0.0f);    // parallel beam: the view's slope
  std::vector<double> view_a0(na, 0.0);   // a of the view's first bin
  int m_x = 0;
  for (int a = 0; a < na; ++a) {
    const int sp = p->split[a];
    const bool fx = p->first_x[a] != 0;
    const int xs = fx ? 0 : sp, xe = fx ? sp : nd;
    m_x += xe - xs;
    if (sp > 0 && sp < nd) p->n_split_views++;
  }
  int xi = 0, yi = m_x;
  for (int a = 0; a < na; ++a) {
    const int sp = p->split[a];
    const bool fx = p->first_x[a] != 0;
    ViewInfo v{};
    v.xj0 = fx ? 0 : sp;
    v.xj1 = fx ? sp : nd;
    v.yj0 = fx ? sp : 0;
    v.yj1 = fx ? nd : sp;
    v.xoff = xi;
    v.yoff = yi;
    double ca = 0, sa = 0;
    for (int j = 0; j < nd; ++j) {
      double p0[2], dir[2];
      ray_geom(*desc, pitch, a, j, p0, dir, &ca, &sa);
      const bool xm = (j < sp) == fx;
      double t, c0;
      if (xm) {
        t = dir[1] / dir[0];
        c0 = p0[1] + (0.0 - p0[0]) * t;   // ray height at x = 0
      } else {
        t = dir[0] / dir[1];
        c0 = p0[0] + (0.0 - p0[1]) * t;   // ray abscissa at y = 0
      }
      // a = (cross coordinate at the centre line + W/2) / h, split into two
      // floats, and the slope t likewise (see block_origin in kernels.cu)
      const double av = (c0 + 0.5 * W) / h;
      if (j == 0) {
        view_t[a] = (float)t;
        view_a0[a] = av;
        view_da[a] = 1.0f;   // one bin: any step
      } else if (j == 1) {
        view_da[a] = (float)(av - view_a0[a]);
      }
      float4 e;
      e.x = (float)av;
      e.y = (float)t;
      e.z = (float)(h * sqrt(1.0 + t * t));
      int sidx = a * nd + j;
      memcpy(&e.w, &sidx, sizeof(int));
      float2 lo;
      lo.x = (float)(av - (double)e.x);
      lo.y = (float)(t - (double)e.y);
      const int slot = xm ? xi++ : yi++;
      rays[slot] = e;
      rays_lo[slot] = lo;
    }
    v.c = (float)ca;
    v.s = (float)sa;
    views[a] = v;
  }

  DevPlan &dp = p->dp;
  dp.n = desc->n;
  dp.n_angles = na;
  dp.n_det = nd;
  dp.geometry = desc->geometry;
  dp.levels = r;
  dp.m = na * nd;
  dp.d = desc->n * desc->n;
  dp.m_x = m_x;
  dp.fov = (float)W;
  dp.inv_pitch = (float)(1.0 / pitch);
  dp.center = (float)(0.5 * (double)(nd - 1));
  dp.src_dist = (float)desc->src_dist;
  dp.sd_dist = (float)(desc->src_dist + desc->det_dist);
  for (int l = 0; l < IMASK_MAX_LEVELS; ++l) dp.probs[l] = l < r ? (float)p->probs[l] : 0.0f;
  level_thresholds(p->probs, dp.thr);
  dp.lg[0] = level_geom(*desc, -1);
  for (int l = 0; l < r; ++l) dp.lg[l + 1] = level_geom(*desc, l);
  dp.upd_tile = update_tile(desc->n, r);
  // pixel-driven back-projector: per level, the most bins of one view that
  // cross a GW_TY x GW_TX tile (the tile widened by one pixel across the
  // rays' major axis, the slope's drift along it), and the views staged at once
  // (bp_gather = -1, parallel beam: the form is chosen below; the bounds are
  // needed in case the pixel-driven one is)
  dp.bp_gather = desc->bp_gather == 1 ? 1 : 0;
  bool gather_possible = desc->geometry == 0 && desc->bp_gather != 0;
  if (gather_possible) {
    for (int li = 0; li <= r && gather_possible; ++li) {
      LevelGeom &g = dp.lg[li];
      double wmax = 1.0;
      int ncmax = 1;
      for (int a = 0; a < na; ++a) {
        // the kernel's count, in the same float operations
        const float Df = view_da[a] * g.inv2l;
        const float inv = 1.0f / Df;
        ncmax = std::max(ncmax, (int)floorf(2.0f * fabsf(inv)) + 1);
        const double D = fabs((double)view_da[a]) * (double)g.inv2l;
        // cross extent (lines + 1) plus the march extent's drift, for either
        // orientation of the tile
        const double at = fabs((double)view_t[a]);
        const double span = std::max((GW_TY + 1) + (GW_TX - 1) * at, (GW_TX + 1) + (GW_TY - 1) * at);
        const double b = nd > 1 ? ceil(span / std::max(D, 1e-9)) + 3.0 : 1.0;
        wmax = std::max(wmax, std::min(b, (double)nd));
      }
      if (wmax > GW_SLOTS - 18) {   // a window and its zero padding must fit
        if (desc->bp_gather == -1) {   // chosen automatically: keep the owner-computes form
          gather_possible = false;
          break;
        }
        imask_plan_destroy(p);
        return fail(IMASK_ERR_SHAPE,
                    "pixel-driven back-projector: %d bins of one view cross a tile at level "
                    "%d, more than the %d it stages", (int)wmax, li - 1, GW_SLOTS - 18);
      }
      g.gw_max = (int)wmax;
      g.gw_nc = ncmax;
      g.gw_vc = std::max(1, std::min(128, GW_SLOTS / (g.gw_max + 18)));
    }
  }
  // Grid sizes from the SM count: the projector runs exactly one wave of
  // 2 CTAs per SM (ray chunks shrink below FP_CHUNK to fill it); the
  // back-projector's view groups are chosen for the best last-wave fill at
  // the resident CTAs per SM that an undivided view range allows (a lower
  // bound: split ranges need less shared memory), and the plan-time
  // autotuner, when asked for, times the splits around that choice.
  int n_sm = 152;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
        n_sm = v;
    }
  }
  {
    const int m_y = dp.m - m_x;
    const int target = 2 * n_sm;
    int cx = m_x > 0 ? std::max(1, (int)std::lround((double)target * m_x / dp.m)) : 0;
    int cy = m_y > 0 ? std::max(1, target - cx) : 0;
    cx = std::max(cx, (m_x + FP_CHUNK - 1) / FP_CHUNK);
    cy = std::max(cy, (m_y + FP_CHUNK - 1) / FP_CHUNK);
    dp.fp_chunk_x = cx > 0 ? (m_x + cx - 1) / cx : 1;
    dp.fp_chunk_y = cy > 0 ? (m_y + cy - 1) / cy : 1;
    p->n_cta_x = cx > 0 ? (m_x + dp.fp_chunk_x - 1) / dp.fp_chunk_x : 0;
    p->n_cta_y = cy > 0 ? (m_y + dp.fp_chunk_y - 1) / dp.fp_chunk_y : 0;
  }
  {
    // resident back-projector CTAs per SM, for the largest per-CTA view range
    for (int li = 0; li <= r; ++li) dp.lg[li].bp_nv = desc->n_angles;
    const int occ = bp_blocks_per_sm(bp_smem_bytes(dp));
    const double slots = (double)occ * n_sm;
    for (int li = 0; li <= r; ++li) {
      LevelGeom &g = dp.lg[li];
      const int tiles = 2 * g.bp_nm * g.bp_nc;   // x- and y-major CTAs per view group
      const int vmax = std::max(1, std::min(desc->n_angles, (int)std::ceil(8.0 * slots / tiles)));
      // at least two waves where the views allow it, then the fullest last wave
      double best = -1.0;
      int bv = 1;
      for (int v = 1; v <= vmax; ++v) {
        const double waves = tiles * (double)v / slots;
        const double eff = (waves / std::ceil(waves)) * std::min(1.0, waves / 2.0);
        if (eff > best + 0.03) {   // a larger split must buy a clearly better fill
          best = eff;
          bv = v;
        }
      }
      g.bp_vgo = bv;
    }
  }
  std::vector<int> role_views;   // role 0 list, then role 1 list, each padded to na
  role_views.assign(2 * (size_t)na, 0);
  {
    std::vector<int> lists[2];
    bp_role_lists(p->split, p->first_x, nd, lists, p->role_rays);
    for (int role = 0; role < 2; ++role)
      std::copy(lists[role].begin(), lists[role].end(), role_views.begin() + (size_t)role * na);
  }
  p->gcap = 0;
  for (int li = 0; li <= r; ++li) {
    LevelGeom &g = dp.lg[li];
    upload_bp_groups(p, li, nullptr);   // bounds and bp_nv only (no table yet)
    p->gcap = std::max(p->gcap, (size_t)2 * g.bp_vgo * g.nl * g.nl);
  }
  if (bp_smem_bytes(dp) > 160 * 1024) {
    imask_plan_destroy(p);
    return fail(IMASK_ERR_SHAPE, "too many views per back-projector CTA for shared memory");
  }
  const std::vector<int> order = bp_tile_order(dp, views, *desc);
  {
    int off = 0;
    for (int li = 0; li <= r; ++li) {
      dp.lg[li].bp_order_off = off;
      off += 2 * dp.lg[li].bp_nm * dp.lg[li].bp_nc;
    }
  }

  cudaError_t e;
  if ((e = cudaMalloc(&p->d_rays, rays.size() * sizeof(float4))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_rays_lo, rays_lo.size() * sizeof(float2))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_views, views.size() * sizeof(ViewInfo))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_err, sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_bp_order, order.size() * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_view_da, view_da.size() * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_bp_views, role_views.size() * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_bp_vb, (size_t)(r + 1) * 2 * (na + 1) * sizeof(int))) !=
          cudaSuccess) {
    imask_plan_destroy(p);
    return cuda_fail(e, "cudaMalloc(plan)");
  }
  // Every upload and every launch of the plan's set-up goes to one
  // non-blocking stream, which is synchronised before the plan is returned:
  // a copy on the legacy stream would not be ordered before work on a
  // non-blocking stream, and a pageable cudaMemcpy may return before its
  // transfer has landed.
  cudaStream_t st = nullptr;
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
    imask_plan_destroy(p);
    return cuda_fail(e, "cudaStreamCreate");
  }
  if ((e = cudaMemcpyAsync(p->d_rays, rays.data(), rays.size() * sizeof(float4),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(p->d_rays_lo, rays_lo.data(), rays_lo.size() * sizeof(float2),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(p->d_views, views.data(), views.size() * sizeof(ViewInfo),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(p->d_bp_order, order.data(), order.size() * sizeof(int),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(p->d_view_da, view_da.data(), view_da.size() * sizeof(float),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(p->d_bp_views, role_views.data(), role_views.size() * sizeof(int),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(p->d_err, 0, sizeof(unsigned int), st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    imask_plan_destroy(p);
    return cuda_fail(e, "upload plan");
  }
  dp.rays = p->d_rays;
  dp.rays_lo = p->d_rays_lo;
  dp.views = p->d_views;
  dp.bp_order = p->d_bp_order;
  dp.view_da = p->d_view_da;
  dp.bp_views = p->d_bp_views;
  dp.bp_vb = p->d_bp_vb;
  for (int li = 0; li <= r && rc == IMASK_OK; ++li) rc = upload_bp_groups(p, li, st);

  if (rc == IMASK_OK && p->desc.autotune) {
    if (gather_possible && p->desc.bp_gather == -1) {
      // both back-projector forms, each with its own tuned splits; the one
      // with the smaller expected time per iteration (sum of p_l times the
      // level's time) is kept
      double t_form[2] = {0.0, 0.0};
      int vgo_form[2][IMASK_MAX_LEVELS + 1];
      int vgo0[IMASK_MAX_LEVELS + 1];
      for (int li = 0; li <= r; ++li) vgo0[li] = dp.lg[li].bp_vgo;
      for (int form = 0; form < 2 && rc == IMASK_OK; ++form) {
        dp.bp_gather = form;
        for (int li = 0; li <= r; ++li) dp.lg[li].bp_vgo = vgo0[li];
        std::vector<float> ms;
        rc = autotune_bp(p, st, &ms);
        for (int li = 1; li <= r && rc == IMASK_OK; ++li)
          t_form[form] += p->probs[li - 1] * (double)ms[li];
        for (int li = 0; li <= r; ++li) vgo_form[form][li] = dp.lg[li].bp_vgo;
      }
      if (rc == IMASK_OK) {
        dp.bp_gather = t_form[1] < t_form[0] ? 1 : 0;
        p->gcap = 0;
        for (int li = 0; li <= r && rc == IMASK_OK; ++li) {
          dp.lg[li].bp_vgo = vgo_form[dp.bp_gather][li];
          p->gcap = std::max(p->gcap, (size_t)2 * dp.lg[li].bp_vgo * dp.lg[li].nl * dp.lg[li].nl);
          rc = upload_bp_groups(p, li, st);
        }
      }
    } else {
      rc = autotune_bp(p, st);
    }
  } else if (rc == IMASK_OK && gather_possible && p->desc.bp_gather == -1) {
    dp.bp_gather = 1;   // not timed: the pixel-driven form (the faster one measured)
  }
  if (rc == IMASK_OK && p->desc.autotune) rc = autotune_fp(p, st);
  if (rc == IMASK_OK) rc = plan_constants(p, st);
  e = cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (rc == IMASK_OK && e != cudaSuccess) rc = cuda_fail(e, "plan set-up");
  if (rc != IMASK_OK) {
    imask_plan_destroy(p);
    return rc;
  }
  p->fingerprint = plan_fingerprint(p);
  *plan_out = p;
  return IMASK_OK;
}

imask_status imask_plan_destroy(imask_plan_t p) {
  if (!p) return IMASK_OK;
  cudaDeviceSynchronize();
  if (p->d_rays) cudaFree(p->d_rays);
  if (p->d_rays_lo) cudaFree(p->d_rays_lo);
  if (p->d_views) cudaFree(p->d_views);
  if (p->d_err) cudaFree(p->d_err);
  if (p->d_bp_order) cudaFree(p->d_bp_order);
  if (p->d_view_da) cudaFree(p->d_view_da);
  if (p->d_bp_views) cudaFree(p->d_bp_views);
  if (p->d_bp_vb) cudaFree(p->d_bp_vb);
  delete p;
  return IMASK_OK;
}

imask_status imask_plan_get_info(imask_plan_t p, imask_plan_info *info) {
  if (!p || !info) return fail(IMASK_ERR_INVALID, "NULL argument");
  memset(info, 0, sizeof *info);
  info->mu = p->mu;
  info->sigma = p->sigma;
  info->theta = p->theta;
  info->L = p->L;
  info->Lbar = p->Lbar;
  info->Lbar_p = p->Lbar_p;
  info->norm_K = p->norm_K;
  info->n_meas = p->dp.m;
  info->n_pix = p->dp.d;
  info->levels = p->desc.levels;
  info->n_xmajor_views_split = p->n_split_views;
  info->n_xmajor_rays = p->dp.m_x;
  info->state_bytes = (int64_t)(state_layout(p).total * sizeof(float));
  info->autotuned = p->autotuned ? 1 : 0;
  info->bp_gather = p->dp.bp_gather;
  for (int l = 0; l < IMASK_MAX_LEVELS; ++l)
    info->bp_view_groups[l] = l < p->desc.levels ? p->dp.lg[l + 1].bp_vgo : 0;
  for (int l = 0; l < 8; ++l)
    info->fp_strip_lines[l] = l < p->desc.levels ? p->dp.lg[l + 1].tc : 0;
  int64_t n_order = 0;
  for (int li = 0; li <= p->desc.levels; ++li) n_order += 2 * p->dp.lg[li].bp_nm * p->dp.lg[li].bp_nc;
  const int64_t na = p->dp.n_angles;
  info->plan_bytes = (int64_t)(p->dp.m * (sizeof(float4) + sizeof(float2)) +
                               na * sizeof(ViewInfo) + sizeof(unsigned int)) +
                     n_order * (int64_t)sizeof(int) +
                     (2 * na + (int64_t)(p->desc.levels + 1) * 2 * (na + 1)) *
                         (int64_t)sizeof(int);   // view lists and view-group bounds
  return IMASK_OK;
}

imask_status imask_plan_axis_split(imask_plan_t p, int32_t *split, int32_t *first_x) {
  if (!p || !split || !first_x) return fail(IMASK_ERR_INVALID, "NULL argument");
  for (int a = 0; a < p->desc.n_angles; ++a) {
    split[a] = p->split[a];
    first_x[a] = p->first_x[a];
  }
  return IMASK_OK;
}

imask_status imask_plan_check(imask_plan_t p) {
  if (!p) return fail(IMASK_ERR_INVALID, "NULL plan");
  CK(cudaDeviceSynchronize(), "synchronise");
  unsigned int idx_flags = 0;
  CK(read_index_check_flag(&idx_flags, true), "read index-check flag");
  if (idx_flags)
    return fail(IMASK_ERR_INVALID,
                "an index check of the checked build failed (flags 0x%x: 2 projector line, "
                "4 back-projector staging, 8 sketch writes)", idx_flags);
  unsigned int flag = 0;
  CK(cudaMemcpy(&flag, p->d_err, sizeof flag, cudaMemcpyDeviceToHost), "read error flag");
  if (flag) {
    // cleared before returning, so no later launch can race with the reset
    cudaMemset(p->d_err, 0, sizeof flag);
    cudaDeviceSynchronize();
    return fail(IMASK_ERR_TIMEOUT, "a projector launch gave up waiting for its image strips");
  }
  return IMASK_OK;
}

imask_status imask_project(imask_plan_t p, int32_t level, const float *x_dev, float *sino_dev,
                           void *stream) {
  if (!p || !x_dev || !sino_dev) return fail(IMASK_ERR_INVALID, "NULL argument");
  if (level < -1 || level >= p->desc.levels)
    return fail(IMASK_ERR_INVALID, "level %d outside [-1, %d]", level, p->desc.levels - 1);
  cudaStream_t st = (cudaStream_t)stream;
  Scratch s;
  imask_status rc = scratch_alloc(p, 1u << (level + 1), false, st, s);
  if (rc != IMASK_OK) return rc;
  rc = apply_K(p, level, x_dev, sino_dev, s, st);
  scratch_free(s);
  return rc;
}

imask_status imask_backproject(imask_plan_t p, int32_t level, const float *y_dev, float *img_dev,
                               void *stream) {
  if (!p || !y_dev || !img_dev) return fail(IMASK_ERR_INVALID, "NULL argument");
  if (level < -1 || level >= p->desc.levels)
    return fail(IMASK_ERR_INVALID, "level %d outside [-1, %d]", level, p->desc.levels - 1);
  cudaStream_t st = (cudaStream_t)stream;
  Scratch s;
  imask_status rc = scratch_alloc(p, 0u, true, st, s);
  if (rc != IMASK_OK) return rc;
  rc = apply_KT(p, level, y_dev, img_dev, s, st);
  scratch_free(s);
  return rc;
}

// Allocation-free back-projection.  The partial sums that imask_backproject
// keeps in a buffer obtained with cudaMallocAsync live here in one fixed
// device array instead, for callers that must not allocate device memory
// once they are running: a host whose own allocator has reserved the device
// memory, a latency-bound loop where an allocation could stall or fail, or a
// process that may only allocate at start-up.  The array is part of the
// library image, so every GPU that loads the library holds its 16 MiB until
// the process exits.
#define IMASK_NOALLOC_FLOATS (4u << 20)
static __device__ __align__(256) float g_noalloc_scratch[IMASK_NOALLOC_FLOATS];

namespace {
// Device address of the array per device, looked up once per CUDA context
// (a cudaDeviceReset ends the context; the module is loaded again, possibly
// at another address, in the next one).  The context is identified through
// the driver's cuCtxGetCurrent / cuCtxGetId, reached via the runtime.
std::mutex g_noalloc_mu;
struct NoallocAddr {
  unsigned long long ctx_id = 0;
  bool known = false;
  float *ptr = nullptr;
};
NoallocAddr g_noalloc_addr[256];
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_ctx_fns_tried = false;

// Identifier of the calling thread's current context; 0 if it cannot be read
// (the address is then looked up on every call).
unsigned long long current_ctx_id() {
  if (!g_ctx_fns_tried) {
    g_ctx_fns_tried = true;
    void *f0 = nullptr, *f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) ==
            cudaSuccess &&
        q0 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess) {
      g_ctx_get_current = (CtxGetCurrentFn)f0;
      g_ctx_get_id = (CtxGetIdFn)f1;
    }
    cudaGetLastError();
  }
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}
}  // namespace

imask_status imask_backproject_noalloc(imask_plan_t p, int32_t level, const float *y_dev,
                                       float *img_dev, void *stream) {
  if (!p || !y_dev || !img_dev) return fail(IMASK_ERR_INVALID, "NULL argument");
  if (level < -1 || level >= p->desc.levels)
    return fail(IMASK_ERR_INVALID, "level %d outside [-1, %d]", level, p->desc.levels - 1);
  if (p->gcap > IMASK_NOALLOC_FLOATS)
    return fail(IMASK_ERR_SHAPE,
                "imask_backproject_noalloc: this plan needs %zu floats of scratch, above the "
                "fixed %u (16 MiB); use imask_backproject",
                p->gcap, (unsigned)IMASK_NOALLOC_FLOATS);
  int dev = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(IMASK_ERR_INVALID, "device index %d out of range", dev);
  float *ptr = nullptr;
  {
    // first call on this device (in this context): look up the array's
    // device address (in host code the array's name is only a host-side
    // stand-in)
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    const unsigned long long ctx = current_ctx_id();
    NoallocAddr &a = g_noalloc_addr[dev];
    if (!a.known || ctx == 0 || a.ctx_id != ctx) {
      void *addr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
      a.ptr = (float *)addr;
      a.ctx_id = ctx;
      a.known = true;
    }
    ptr = a.ptr;
  }
  // every scratch element read below is written earlier in the same call,
  // so nothing is cleared
  Scratch s;
  s.g = ptr;
  return apply_KT(p, level, y_dev, img_dev, s, (cudaStream_t)stream);
}

imask_status imask_levels(imask_plan_t p, uint64_t seed, int64_t k0, int64_t n, int32_t *out_dev,
                          void *stream) {
  if (!p || (!out_dev && n > 0)) return fail(IMASK_ERR_INVALID, "NULL argument");
  if (n < 0 || k0 < 0) return fail(IMASK_ERR_INVALID, "negative range");
  CK(launch_levels(p->dp, seed, k0, n, out_dev, (cudaStream_t)stream), "levels launch");
  return IMASK_OK;
}

imask_status imask_state_create(imask_plan_t p, const float *b_dev, uint64_t seed,
                                imask_state_t *state_out, void *stream) {
  if (!p || !b_dev || !state_out) return fail(IMASK_ERR_INVALID, "NULL argument");
  *state_out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  imask_state_s *s = new (std::nothrow) imask_state_s();
  if (!s) return fail(IMASK_ERR_OOM, "host allocation");
  s->plan = p;
  s->seed = seed;
  s->stream = st;
  const int r = p->desc.levels;
  const size_t m = p->dp.m;
  const bool snapshots = p->desc.dual_tables == 1;
  const StateLayout L = state_layout(p);
  const size_t o_x = L.x, o_y0 = L.y0, o_y1 = L.y1, o_b = L.b, o_psi = L.psi, o_psim = L.psim,
               o_phi0 = L.phi0, o_phim = L.phim, o_xprev = L.xprev, o_kdev = L.kdev, o_g = L.g,
               o_tv = L.tv;
  const size_t *o_snap = L.snap, *o_T = L.T, *o_R = L.R;
  Carve cv;
  cv.off = L.total;
  void *mem = nullptr;
  cudaError_t e = cudaMallocAsync(&mem, cv.off * sizeof(float), st);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaMallocAsync(state)");
  }
  float *B = (float *)mem;
  s->block = B;
  s->x = B + o_x;
  s->y[0] = B + o_y0;
  s->y[1] = B + o_y1;
  s->b = B + o_b;
  s->psi = snapshots ? nullptr : (void *)(B + o_psi);
  s->psi_fmt = p->desc.storage;
  s->psi_mean = B + o_psim;
  s->seed_x = p->desc.draws == 1 ? primal_seed(seed) : seed;
  if (snapshots) {
    s->snap.snap = B;
    for (int l = 0; l < r; ++l) s->snap.snap_off[l] = (long long)o_snap[l];
  }
  s->x_prev = o_xprev ? B + o_xprev : nullptr;
  s->k_dev = (long long *)(B + o_kdev);
  s->phi0 = (void *)(B + o_phi0);
  s->phi_fmt = p->desc.storage;
  s->phi_mean = B + o_phim;
  s->g = B + o_g;
  s->g2 = L.g2 ? B + L.g2 : s->g;
  s->phic = s->phi0;
  {
    long long off = (long long)p->dp.d;
    for (int l = 1; l < r; ++l) {
      s->phic_off[l] = off;
      off += (long long)p->dp.lg[l + 1].nl * p->dp.lg[l + 1].nl;
    }
  }
  s->tv = p->desc.reg != 0 ? B + o_tv : nullptr;
  for (int li = 1; li <= r; ++li) {
    s->pads[0].T[li] = B + o_T[li];
    s->pads[0].R[li] = B + o_R[li];
    s->pads[1].T[li] = L.T2[li] ? B + L.T2[li] : s->pads[0].T[li];
    s->pads[1].R[li] = L.R2[li] ? B + L.R2[li] : s->pads[0].R[li];
  }
  if ((e = cudaMemsetAsync(mem, 0, cv.off * sizeof(float), st)) != cudaSuccess ||
      (e = launch_sino_order(p->dp, b_dev, s->b, 1, st)) != cudaSuccess) {
    cudaFreeAsync(mem, st);
    delete s;
    return cuda_fail(e, "state init");
  }
  if (p->desc.variant == 0 &&
      ((e = cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking)) != cudaSuccess ||
       (e = cudaStreamCreateWithFlags(&s->aux2, cudaStreamNonBlocking)) != cudaSuccess ||
       (e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
       (e = cudaEventCreateWithFlags(&s->ev_fp, cudaEventDisableTiming)) != cudaSuccess ||
       (e = cudaEventCreateWithFlags(&s->ev_start, cudaEventDisableTiming)) != cudaSuccess ||
       (e = cudaEventCreateWithFlags(&s->ev_bp, cudaEventDisableTiming)) != cudaSuccess ||
       (e = cudaEventCreateWithFlags(&s->ev_upd[0], cudaEventDisableTiming)) != cudaSuccess ||
       (e = cudaEventCreateWithFlags(&s->ev_upd[1], cudaEventDisableTiming)) != cudaSuccess)) {
    imask_state_destroy(s);
    return cuda_fail(e, "state streams");
  }
  *state_out = s;
  return IMASK_OK;
}

namespace {

// Enqueues one iteration of the state's algorithm on stream st, reading and
// writing the dual iterate pair selected by `cur`.  graph: the kernels take the
// iteration counter from the state's device counter plus k_add (for captured
// graphs) and no profiling events are recorded; otherwise the counter is k.
//
// Alg. 1 runs on three streams of the state: the projector of k on aux, its
// back-projector on aux2, the update on st.  Within a sequence of iterations
// (pos 0 .. last) the projector of k waits for the update of k - 1 (its sketch),
// the back-projector of k for the projector of k - 1 (y^k) and for the update
// of k - 2 (which read the partial-image buffer it overwrites), the update of k
// for the back-projector of k; the sequence starts after everything before it
// on st and ends with st joined to both side streams.  Profiled iterations run
// in order on st (one-iteration sequences).
imask_status enqueue_iteration(const imask_state_s *s, cudaStream_t st, int cur, long long k,
                               bool graph, int k_add, int pos = 0, bool last = true) {
  const imask_plan_s *p = s->plan;
  const DevPlan &P = p->dp;
  const bool seq = p->desc.variant == 1;
  const float sigma = (float)p->sigma;
  const float inv_1ps = (float)(1.0 / (1.0 + p->sigma));
  const float tau = (float)(p->sigma / p->mu);
  const float theta = (float)p->desc.theta;
  LevelSel sel{};
  sel.fixed = -2;
  sel.seed = s->seed;
  sel.seed_x = s->seed_x;
  sel.k = k;
  sel.k_dev = graph ? s->k_dev : nullptr;
  sel.k_add = k_add;
  const int pp = g_prof.period.load();
  const bool prof = !graph && g_prof.on.load() && pp > 0 && k % pp == 0;
  const int lvl = prof ? lvl_host_draw(P, s->seed, k) : 0;
  const int lvl_x = prof ? lvl_host_draw(P, s->seed_x, k) : 0;
  const bool fork = !seq && s->aux && !prof;
  if (prof) {
    pos = 0;
    last = true;
  }
  const cudaStream_t sfp = fork ? s->aux : st, sbp = fork ? s->aux2 : st;
  // partial images of this iteration's back-projection (alternating with the
  // iteration parity, which equals cur, in Alg. 1)
  float *g = cur != 0 ? s->g2 : s->g;
  if (fork) {
    if (pos == 0) {
      CK(cudaEventRecord(s->ev_start, st), "fork");
      CK(cudaStreamWaitEvent(s->aux, s->ev_start, 0), "fork");
      CK(cudaStreamWaitEvent(s->aux2, s->ev_start, 0), "fork");
    } else {
      // projector of k - 1 done (y^k); update of k - 2 done with the buffer g
      // (when k - 2 is in this sequence; earlier work is behind the start)
      CK(cudaStreamWaitEvent(s->aux2, s->ev_fp, 0), "order");
      if (pos >= 2) CK(cudaStreamWaitEvent(s->aux2, s->ev_upd[cur], 0), "order");
      // update of k - 1 done (the sketch the projector reads)
      CK(cudaEventRecord(s->ev_fork, st), "order");
      CK(cudaStreamWaitEvent(s->aux, s->ev_fork, 0), "order");
    }
  }
  // dual half: projector on the sketch of x^k (Alg. 1) or xbar^k (Alg. 7)
  // prepared by the previous iteration, fused with the zeta and y updates
  DualArgs D{};
  D.on = 1;
  D.y_in = s->y[cur];
  D.y_out = s->y[1 - cur];
  D.b = s->b;
  D.psi = s->psi;
  D.psi_fmt = s->psi_fmt;
  D.psi_mean = s->psi_mean;
  D.sigma = sigma;
  D.inv_1ps = inv_1ps;
  {
    ProfScope ps(0, lvl, sfp, prof);
    CK(launch_fp(P, sel, s->pads[cur], nullptr, D, p->n_cta_x, p->n_cta_y, p->d_err, sfp),
       "projector launch");
  }
  if (fork) CK(cudaEventRecord(s->ev_fp, s->aux), "order");
  // primal half: Alg. 1 back-projects y^k, Alg. 7 the new y^{k+1}
  {
    ProfScope ps(1, lvl_x, sbp, prof);
    CK(launch_bp(P, sel, seq ? s->y[1 - cur] : s->y[cur], 1, g, p->d_err, sbp),
       "back-projector launch");
  }
  if (fork) {
    CK(cudaEventRecord(s->ev_bp, s->aux2), "order");
    CK(cudaStreamWaitEvent(st, s->ev_bp, 0), "order");
  }
  PrimalArgs A{};
  A.g = g;
  A.x = s->x;
  A.phi0 = s->phi0;
  A.phic = s->phic;
  for (int l = 0; l < IMASK_MAX_LEVELS; ++l) A.phic_off[l] = s->phic_off[l];
  A.phi_fmt = s->phi_fmt;
  A.phi_mean = s->phi_mean;
  A.tau = tau;
  A.inv_1ps = inv_1ps;
  A.prox_in_place = p->desc.reg == 0 ? 1 : 0;
  A.x_prev = p->desc.reg == 0 ? nullptr : s->x_prev;
  A.extrapolate = seq ? 1 : 0;
  A.theta = theta;
  A.snap = s->snap;
  {
    ProfScope ps(2, lvl_x, st, prof);
    CK(launch_update(P, sel, A, p->desc.reg == 0 ? 1 : 0, s->pads[1 - cur], st),
       "update launch");
  }
  if (p->desc.reg != 0) {
    CK(launch_reg_prox(p, tau, s->x, s->tv, st), "TV prox launch");
    LevelSel nxt = sel;
    nxt.k = k + 1;
    nxt.k_add = k_add + 1;
    ExtrapArgs ex{};
    if (seq) {
      ex.x_prev = s->x_prev;
      ex.theta = theta;
    }
    CK(launch_sketch(P, nxt, s->x, s->pads[1 - cur], ex, s->snap, st), "sketch launch");
  }
  if (fork) {
    CK(cudaEventRecord(s->ev_upd[cur], st), "order");
    if (last) CK(cudaStreamWaitEvent(st, s->ev_fp, 0), "join");
  }
  return IMASK_OK;
}

// Iterations per captured graph (even, so that the dual ping-pong returns to
// its start).  Within a graph the back-projector of one iteration overlaps the
// update of the previous one; replays are serialised, so longer graphs keep
// that overlap for more of the iterations.
#ifndef IMASK_GRAPH_UNROLL
#define IMASK_GRAPH_UNROLL 4
#endif
constexpr int kGraphUnroll = IMASK_GRAPH_UNROLL;
static_assert(kGraphUnroll % 2 == 0, "graphs hold an even number of iterations");

void batch_release_graph(imask_batch_s *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->cur_at_capture.clear();
  b->gen_at_capture.clear();
}

// Captures `unroll` iterations of every state of the batch, each state on its
// own branch, as one CUDA graph.
imask_status batch_capture(imask_batch_s *b, int unroll) {
  batch_release_graph(b);
  cudaStream_t origin = b->origin;
  const int64_t c0 = launch_counter();
  CK(cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed), "begin capture");
  imask_status rc = IMASK_OK;
  cudaError_t e = cudaEventRecord(b->fork, origin);
  for (size_t i = 0; i < b->states.size() && e == cudaSuccess && rc == IMASK_OK; ++i) {
    imask_state_s *s = b->states[i];
    cudaStream_t bs = b->streams[i];
    if ((e = cudaStreamWaitEvent(bs, b->fork, 0)) != cudaSuccess) break;
    int cur = s->cur;
    for (int u = 0; u < unroll && rc == IMASK_OK; ++u) {
      rc = enqueue_iteration(s, bs, cur, 0, true, u, u, u == unroll - 1);
      cur = 1 - cur;
    }
    if (rc != IMASK_OK) break;
    if ((e = launch_counter(s->k_dev, unroll, 0, bs)) != cudaSuccess) break;
    if ((e = cudaEventRecord(b->joins[i], bs)) != cudaSuccess) break;
    e = cudaStreamWaitEvent(origin, b->joins[i], 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
  const int64_t captured = launch_counter() - c0;
  add_launches(-captured);   // captured, not run
  if (rc != IMASK_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(e, "graph capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_fail(e, "graph instantiate");
  }
  b->unroll = unroll;
  b->kernels_per_replay = captured;
  b->cur_at_capture.clear();
  b->gen_at_capture.clear();
  for (auto *s : b->states) {
    b->cur_at_capture.push_back(s->cur);
    b->gen_at_capture.push_back(s->gen);
  }
  return IMASK_OK;
}

// The iteration records of a fused batch for `unroll` iterations starting at
// the states' current ping-pong parity, in launch order (states by decreasing
// size).  Mirrors the arguments enqueue_iteration gives the three kernels.
std::vector<FusedSlice> fused_records(const imask_batch_s *b, int unroll) {
  const int n = (int)b->states.size();
  std::vector<FusedSlice> recs((size_t)unroll * n);
  for (int pos = 0; pos < unroll; ++pos)
    for (int i = 0; i < n; ++i) {
      const imask_state_s *s = b->states[b->order[i]];
      const imask_plan_s *p = s->plan;
      const bool seq = p->desc.variant == 1;
      const int cur = s->cur ^ (pos & 1);
      FusedSlice &R = recs[(size_t)pos * n + i];
      memset(&R, 0, sizeof(R));
      R.P = p->dp;
      R.sel.fixed = -2;
      R.sel.seed = s->seed;
      R.sel.seed_x = s->seed_x;
      R.sel.k = 0;
      R.sel.k_dev = s->k_dev;
      R.sel.k_add = pos;
      R.pads_fp = s->pads[cur];
      R.pads_upd = s->pads[1 - cur];
      R.D.on = 1;
      R.D.y_in = s->y[cur];
      R.D.y_out = s->y[1 - cur];
      R.D.b = s->b;
      R.D.psi = s->psi;
      R.D.psi_fmt = s->psi_fmt;
      R.D.psi_mean = s->psi_mean;
      R.D.sigma = (float)p->sigma;
      R.D.inv_1ps = (float)(1.0 / (1.0 + p->sigma));
      R.y_bp = seq ? s->y[1 - cur] : s->y[cur];
      R.g = cur != 0 ? s->g2 : s->g;
      R.A.g = R.g;
      R.A.x = s->x;
      R.A.phi0 = s->phi0;
      R.A.phic = s->phic;
      for (int l = 0; l < IMASK_MAX_LEVELS; ++l) R.A.phic_off[l] = s->phic_off[l];
      R.A.phi_fmt = s->phi_fmt;
      R.A.phi_mean = s->phi_mean;
      R.A.tau = (float)(p->sigma / p->mu);
      R.A.inv_1ps = (float)(1.0 / (1.0 + p->sigma));
      R.A.prox_in_place = 1;
      R.A.x_prev = nullptr;
      R.A.extrapolate = seq ? 1 : 0;
      R.A.theta = (float)p->desc.theta;
      R.A.snap = s->snap;
      R.err = p->d_err;
      R.n_cta_x = p->n_cta_x;
    }
  return recs;
}

// Captures `unroll` iterations of a fused batch: per iteration one projector,
// one back-projector (with its planner) and one update launch for all states,
// then one launch that advances every state's device iteration counter.  The
// launches are ordered as Alg. 1's data require, on three capture branches,
// so that the projector of k runs beside the back-projector of k and the
// back-projector of k + 1 beside the update of k: the projector of k after
// the update of k - 1 (the sketch it reads), the back-projector of k after
// the projector of k - 1 (y^k; Alg. 7: of k, whose y^{k+1} it reads) and the
// update of k - 2 (which read the partial images it overwrites), the update
// of k after the back-projector of k.
imask_status batch_capture_fused(imask_batch_s *b, int unroll) {
  batch_release_graph(b);
  const int n = (int)b->states.size();
  const std::vector<FusedSlice> recs = fused_records(b, unroll);
  cudaStream_t origin = b->origin;
  CK(cudaMemcpyAsync(b->d_recs, recs.data(), recs.size() * sizeof(FusedSlice),
                     cudaMemcpyHostToDevice, origin),
     "fused records");
  CK(cudaStreamSynchronize(origin), "fused records");
  if ((int)b->f_ev.size() < 3 * unroll) {
    while ((int)b->f_ev.size() < 3 * unroll) {
      cudaEvent_t ev = nullptr;
      CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "fused events");
      b->f_ev.push_back(ev);
    }
  }
  if (!b->f_fp) CK(cudaStreamCreateWithFlags(&b->f_fp, cudaStreamNonBlocking), "fused streams");
  if (!b->f_bp) CK(cudaStreamCreateWithFlags(&b->f_bp, cudaStreamNonBlocking), "fused streams");
  cudaEvent_t *ev_fp = b->f_ev.data(), *ev_bp = ev_fp + unroll, *ev_upd = ev_bp + unroll;
  const int64_t c0 = launch_counter();
  CK(cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed), "begin capture");
  cudaError_t e = cudaEventRecord(b->fork, origin);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->f_fp, b->fork, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->f_bp, b->fork, 0);
  for (int pos = 0; pos < unroll && e == cudaSuccess; ++pos) {
    const FusedSlice *r = b->d_recs + (size_t)pos * n;
    if (pos > 0 && (e = cudaStreamWaitEvent(b->f_fp, ev_upd[pos - 1], 0)) != cudaSuccess) break;
    if ((e = launch_fp_multi(r, b->d_fp_start, n, b->fp_total, b->f_fp)) != cudaSuccess) break;
    if ((e = cudaEventRecord(ev_fp[pos], b->f_fp)) != cudaSuccess) break;
    if (b->any_seq) {
      if ((e = cudaStreamWaitEvent(b->f_bp, ev_fp[pos], 0)) != cudaSuccess) break;
    } else if (pos > 0 && (e = cudaStreamWaitEvent(b->f_bp, ev_fp[pos - 1], 0)) != cudaSuccess) {
      break;
    }
    if (pos >= 2 && (e = cudaStreamWaitEvent(b->f_bp, ev_upd[pos - 2], 0)) != cudaSuccess) break;
    if ((e = launch_bp_multi(r, n, b->d_bp_start + (size_t)pos * (n + 1), b->d_bp_counter + pos,
                             b->nv_cap, b->bp_smem, b->bp_grid, b->bp_max_items, b->f_bp)) !=
        cudaSuccess)
      break;
    if ((e = cudaEventRecord(ev_bp[pos], b->f_bp)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(origin, ev_bp[pos], 0)) != cudaSuccess) break;
    if ((e = launch_update_multi(r, b->d_upd_start, n, b->upd_total, b->upd_smem, origin)) !=
        cudaSuccess)
      break;
    e = cudaEventRecord(ev_upd[pos], origin);
  }
  // join both branches: the last projector (y of the next iteration) and the
  // last back-projector (ordered before the last update already)
  if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, ev_fp[unroll - 1], 0);
  if (e == cudaSuccess) e = launch_counter_multi(b->d_recs, n, unroll, origin);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
  const int64_t captured = launch_counter() - c0;
  add_launches(-captured);   // captured, not run
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(e, "fused graph capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_fail(e, "graph instantiate");
  }
  b->unroll = unroll;
  b->kernels_per_replay = captured;
  b->cur_at_capture.clear();
  b->gen_at_capture.clear();
  for (auto *s : b->states) {
    b->cur_at_capture.push_back(s->cur);
    b->gen_at_capture.push_back(s->gen);
  }
  return IMASK_OK;
}

}  // namespace

imask_status imask_step(imask_state_t s, int32_t n_iters, void *stream) {
  NvtxRange nv("imask_step");
  if (!s) return fail(IMASK_ERR_INVALID, "NULL state");
  if (n_iters < 0) return fail(IMASK_ERR_INVALID, "n_iters < 0");
  cudaStream_t st = (cudaStream_t)stream;
  imask_status rc0 = state_use_stream(s, st);
  if (rc0 != IMASK_OK) return rc0;
  // Runs of several iterations replay a captured two-iteration graph (same
  // kernels, fewer launch gaps).  With kernel profiling every period-th
  // iteration is launched on its own so that its events are recorded, and the
  // pairs in between still replay the graph.
  bool prof_on;
  int period;
  {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    prof_on = g_prof.on.load();
    period = g_prof.period.load();
  }
  if (n_iters >= 8 && (!prof_on || period >= 4)) {
    if (!s->self_batch) {
      imask_state_t one[1] = {s};
      imask_status rc = imask_batch_create(one, 1, &s->self_batch);
      if (rc != IMASK_OK) return rc;
    }
    if (!prof_on) return imask_batch_step(s->self_batch, n_iters, stream);
    int left = n_iters;
    while (left > 0) {
      const int into = (int)(s->k % period);
      int run = into == 0 ? 1 : std::min(left, period - into);   // up to the next profiled k
      imask_status rc = IMASK_OK;
      if (into == 0) {
        rc = enqueue_iteration(s, st, s->cur, s->k, false, 0);
        if (rc == IMASK_OK) {
          s->cur = 1 - s->cur;
          s->k += 1;
          s->k_dev_stale = true;
        }
      } else {
        const int units = run / kGraphUnroll;
        if (units > 0) rc = imask_batch_step(s->self_batch, kGraphUnroll * units, stream);
        for (int i = kGraphUnroll * units; i < run && rc == IMASK_OK; ++i) {
          rc = enqueue_iteration(s, st, s->cur, s->k, false, 0);
          s->cur = 1 - s->cur;
          s->k += 1;
          s->k_dev_stale = true;
        }
      }
      if (rc != IMASK_OK) return rc;
      left -= run;
    }
    return IMASK_OK;
  }
  for (int it = 0; it < n_iters; ++it) {
    imask_status rc = enqueue_iteration(s, st, s->cur, s->k, false, 0);
    if (rc != IMASK_OK) return rc;
    s->cur = 1 - s->cur;
    s->k += 1;
    s->k_dev_stale = true;
  }
  return IMASK_OK;
}

imask_status imask_batch_create(const imask_state_t *states, int32_t n_states,
                                imask_batch_t *batch_out) {
  if (!states || !batch_out || n_states < 1) return fail(IMASK_ERR_INVALID, "bad argument");
  *batch_out = nullptr;
  for (int i = 0; i < n_states; ++i) {
    if (!states[i]) return fail(IMASK_ERR_INVALID, "state %d is NULL", i);
    for (int j = 0; j < i; ++j)
      if (states[j] == states[i]) return fail(IMASK_ERR_INVALID, "state %d appears twice", i);
  }
  imask_batch_s *b = new (std::nothrow) imask_batch_s();
  if (!b) return fail(IMASK_ERR_OOM, "host allocation");
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  for (int i = 0; i < n_states && e == cudaSuccess; ++i) {
    b->states.push_back(states[i]);
    cudaStream_t bs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking)) != cudaSuccess) break;
    b->streams.push_back(bs);
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) break;
    b->joins.push_back(ev);
  }
  if (e != cudaSuccess) {
    imask_batch_destroy(b);
    return cuda_fail(e, "batch streams");
  }
  *batch_out = b;
  return IMASK_OK;
}

imask_status imask_batch_create_fused(const imask_state_t *states, int32_t n_states,
                                      imask_batch_t *batch_out) {
  if (!states || !batch_out || n_states < 1) return fail(IMASK_ERR_INVALID, "bad argument");
  if (n_states > IMASK_MAX_FUSED)
    return fail(IMASK_ERR_INVALID, "a fused batch holds at most %d states", IMASK_MAX_FUSED);
  for (int i = 0; i < n_states; ++i) {
    if (states[i] && states[i]->plan->desc.reg != 0)
      return fail(IMASK_ERR_INVALID,
                  "state %d: fused batches take the quadratic regulariser (reg = 0) only", i);
    if (states[i] && states[i]->plan->dp.bp_gather != 0)
      return fail(IMASK_ERR_INVALID,
                  "state %d: fused batches run the owner-computes back-projector, not the "
                  "pixel-driven one (bp_gather)", i);
  }
  imask_status rc = imask_batch_create(states, n_states, batch_out);
  if (rc != IMASK_OK) return rc;
  imask_batch_s *b = *batch_out;
  const int n = n_states;
  b->fused = true;
  for (int i = 0; i < n_states; ++i) b->any_seq = b->any_seq || b->states[i]->plan->desc.variant == 1;
  // launch order: largest solves first, so that the back-projector's dynamic
  // item list ends with the small ones
  b->order.resize(n);
  for (int i = 0; i < n; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) {
    const DevPlan &A = b->states[a]->plan->dp, &C = b->states[c]->plan->dp;
    return (long long)A.m * A.n > (long long)C.m * C.n;
  });
  std::vector<int> fp_start(n + 1, 0), upd_start(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const imask_plan_s *p = b->states[b->order[i]]->plan;
    const DevPlan &P = p->dp;
    fp_start[i + 1] = fp_start[i] + p->n_cta_x + p->n_cta_y;
    upd_start[i + 1] = upd_start[i] + (P.n / P.upd_tile) * (P.n / P.upd_tile);
    b->bp_smem = std::max(b->bp_smem, bp_smem_bytes(P));
    b->upd_smem = std::max(b->upd_smem, upd_smem_bytes_of(P));
    for (int li = 0; li <= P.levels; ++li) b->nv_cap = std::max(b->nv_cap, P.lg[li].bp_nv);
    int most = 0;
    for (int li = 1; li <= P.levels; ++li)
      most = std::max(most, 2 * P.lg[li].bp_nm * P.lg[li].bp_nc * P.lg[li].bp_vgo);
    b->bp_max_items += most;
  }
  b->fp_total = fp_start[n];
  b->upd_total = upd_start[n];
  int n_sm = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n_sm = v;
  }
  b->bp_grid = bp_multi_blocks_per_sm(b->bp_smem) * n_sm;
  const int unroll = kGraphUnroll;
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_recs, (size_t)unroll * n * sizeof(FusedSlice))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_fp_start, (n + 1) * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_upd_start, (n + 1) * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_bp_start, (size_t)unroll * (n + 1) * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_bp_counter, unroll * sizeof(int))) != cudaSuccess ||
      (e = cudaMemcpyAsync(b->d_fp_start, fp_start.data(), (n + 1) * sizeof(int),
                           cudaMemcpyHostToDevice, b->origin)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b->d_upd_start, upd_start.data(), (n + 1) * sizeof(int),
                           cudaMemcpyHostToDevice, b->origin)) != cudaSuccess ||
      (e = cudaStreamSynchronize(b->origin)) != cudaSuccess) {
    imask_batch_destroy(b);
    *batch_out = nullptr;
    return cuda_fail(e, "fused batch buffers");
  }
  return IMASK_OK;
}

imask_status imask_batch_step(imask_batch_t b, int32_t n_iters, void *stream) {
  NvtxRange nv("imask_batch_step");
  if (!b) return fail(IMASK_ERR_INVALID, "NULL batch");
  if (n_iters < 0) return fail(IMASK_ERR_INVALID, "n_iters < 0");
  cudaStream_t st = (cudaStream_t)stream;
  const int unroll = kGraphUnroll;
  const int replays = n_iters / unroll;
  for (auto *s : b->states) {
    imask_status rc = state_use_stream(s, st);
    if (rc != IMASK_OK) return rc;
  }
  if (replays > 0) {
    // bring the device counters up to date with eager steps taken meanwhile
    for (auto *s : b->states)
      if (s->k_dev_stale) {
        CK(launch_counter(s->k_dev, s->k, 1, st), "counter set");
        s->k_dev_stale = false;
      }
    bool match = b->exec && b->unroll == unroll && b->cur_at_capture.size() == b->states.size();
    for (size_t i = 0; match && i < b->states.size(); ++i)
      match = b->cur_at_capture[i] == b->states[i]->cur &&
              b->gen_at_capture[i] == b->states[i]->gen;
    if (!match) {
      imask_status rc = b->fused ? batch_capture_fused(b, unroll) : batch_capture(b, unroll);
      if (rc != IMASK_OK) return rc;
    }
    for (int r = 0; r < replays; ++r) {
      CK(cudaGraphLaunch(b->exec, st), "graph launch");
      add_launches(b->kernels_per_replay);
    }
    for (auto *s : b->states) {
      s->k += (long long)replays * unroll;   // unroll is even: cur is unchanged
      s->stream = st;
    }
  }
  // the odd remainder runs eagerly, state by state
  for (int it = replays * unroll; it < n_iters; ++it)
    for (auto *s : b->states) {
      imask_status rc = imask_step(s, 1, stream);
      if (rc != IMASK_OK) return rc;
    }
  return IMASK_OK;
}

imask_status imask_batch_destroy(imask_batch_t b) {
  if (!b) return IMASK_OK;
  batch_release_graph(b);
  for (auto st : b->streams) cudaStreamDestroy(st);
  if (b->origin) cudaStreamDestroy(b->origin);
  for (auto ev : b->joins) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto ev : b->f_ev) cudaEventDestroy(ev);
  if (b->f_fp) cudaStreamDestroy(b->f_fp);
  if (b->f_bp) cudaStreamDestroy(b->f_bp);
  for (void *ptr : {(void *)b->d_recs, (void *)b->d_fp_start, (void *)b->d_upd_start,
                    (void *)b->d_bp_start, (void *)b->d_bp_counter})
    if (ptr) cudaFree(ptr);
  delete b;
  return IMASK_OK;
}

int64_t imask_state_iteration(imask_state_t s) { return s ? s->k : -1; }

imask_status imask_state_get(imask_state_t s, int32_t what, float *dst, void *stream) {
  if (!s || !dst) return fail(IMASK_ERR_INVALID, "NULL argument");
  const imask_plan_s *p = s->plan;
  const float *src = nullptr;
  size_t n = 0;
  switch (what) {
    case 0: src = s->x; n = p->dp.d; break;
    case 1: src = s->y[s->cur]; n = p->dp.m; break;
    case 2: src = s->phi_mean; n = p->dp.d; break;
    case 3: src = s->psi_mean; n = p->dp.m; break;
    default: return fail(IMASK_ERR_INVALID, "unknown state part %d", what);
  }
  imask_status rc = state_use_stream(s, (cudaStream_t)stream);
  if (rc != IMASK_OK) return rc;
  if (what == 1 || what == 3) {
    // measurement-space parts are kept in ray-list order: back to (view, bin)
    CK(launch_sino_order(p->dp, src, dst, 0, (cudaStream_t)stream), "copy state");
  } else {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream),
       "copy state");
  }
  return IMASK_OK;
}

imask_status imask_state_get_x(imask_state_t s, float *x_dev, void *stream) {
  return imask_state_get(s, 0, x_dev, stream);
}

namespace {

// Header of a state checkpoint, followed by the state's device block.
struct CheckpointHeader {
  uint64_t magic;          // kCheckpointMagic
  uint64_t block_floats;   // size of the state's block
  int64_t k;               // iteration counter
  uint64_t seed, seed_x;   // level streams
  int32_t cur;             // dual ping-pong parity
  int32_t psi_fmt;         // storage format of the tables
  uint64_t plan_fp;        // fingerprint of the saving state's plan
  uint64_t reserved;
};
constexpr uint64_t kCheckpointMagic = 0x31504b43534b4d49ull;   // "IMSKCKP1"

size_t state_block_floats(const imask_state_s *s) { return state_layout(s->plan).total; }

}  // namespace

int64_t imask_state_checkpoint_bytes(imask_state_t s) {
  if (!s) return -1;
  return (int64_t)(sizeof(CheckpointHeader) + state_block_floats(s) * sizeof(float));
}

imask_status imask_state_save(imask_state_t s, void *dst, void *stream) {
  if (!s || !dst) return fail(IMASK_ERR_INVALID, "NULL argument");
  if (s->psi_block || s->phi_block)
    return fail(IMASK_ERR_INVALID, "a state whose tables changed storage cannot be saved");
  cudaStream_t st = (cudaStream_t)stream;
  CheckpointHeader h{};
  h.magic = kCheckpointMagic;
  h.block_floats = state_block_floats(s);
  h.k = s->k;
  h.seed = s->seed;
  h.seed_x = s->seed_x;
  h.cur = s->cur;
  h.psi_fmt = s->psi_fmt;
  h.plan_fp = s->plan->fingerprint;
  // the copy comes after the state's earlier work (its side streams are joined
  // into its stream after every step), and the state's later calls, on any
  // stream, come after the copy: the state now belongs to st
  imask_status rc = state_use_stream(s, st);
  if (rc != IMASK_OK) return rc;
  CK(cudaMemcpyAsync(dst, &h, sizeof(h), cudaMemcpyHostToDevice, st), "checkpoint header");
  CK(cudaMemcpyAsync((char *)dst + sizeof(h), s->block, h.block_floats * sizeof(float),
                     cudaMemcpyDeviceToDevice, st),
     "checkpoint block");
  return IMASK_OK;
}

imask_status imask_state_load(imask_state_t s, const void *src, void *stream) {
  if (!s || !src) return fail(IMASK_ERR_INVALID, "NULL argument");
  if (s->psi_block || s->phi_block)
    return fail(IMASK_ERR_INVALID, "a state whose tables changed storage cannot be loaded");
  cudaStream_t st = (cudaStream_t)stream;
  CheckpointHeader h{};
  CK(cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDeviceToHost, st), "checkpoint header");
  CK(cudaStreamSynchronize(st), "checkpoint header");
  if (h.magic != kCheckpointMagic) return fail(IMASK_ERR_INVALID, "not a state checkpoint");
  if (h.block_floats != state_block_floats(s) || h.psi_fmt != s->psi_fmt)
    return fail(IMASK_ERR_INVALID, "checkpoint of a state of another plan or storage");
  if (h.plan_fp != s->plan->fingerprint)
    return fail(IMASK_ERR_INVALID,
                "checkpoint of a state of another plan (descriptor, step size or "
                "back-projector splits differ)");
  // the state's own pending work comes first
  CK(cudaStreamSynchronize(s->stream), "checkpoint order");
  CK(cudaMemcpyAsync(s->block, (const char *)src + sizeof(h), h.block_floats * sizeof(float),
                     cudaMemcpyDeviceToDevice, st),
     "checkpoint block");
  s->k = h.k;
  s->seed = h.seed;
  s->seed_x = h.seed_x;
  s->cur = h.cur;
  s->stream = st;
  s->k_dev_stale = true;   // the device counter is set again before the next replay
  s->gen += 1;             // graphs captured before the load are captured again
  return IMASK_OK;
}

imask_status imask_state_set_storage(imask_state_t s, int32_t storage, void *stream) {
  if (!s) return fail(IMASK_ERR_INVALID, "NULL state");
  if (storage < 0 || storage > 2) return fail(IMASK_ERR_INVALID, "storage must be 0, 1 or 2");
  if (!s->psi && storage != 0)
    return fail(IMASK_ERR_INVALID, "the snapshot form keeps no measurement-side tables");
  const bool psi_change = s->psi && storage != s->psi_fmt;
  const bool phi_change = storage != s->phi_fmt;
  if (!psi_change && !phi_change) return IMASK_OK;
  cudaStream_t st = (cudaStream_t)stream;
  imask_status rc = state_use_stream(s, st);
  if (rc != IMASK_OK) return rc;
  const imask_plan_s *p = s->plan;
  const size_t esz = storage != 0 ? 2 : 4;
  void *psi_mem = nullptr, *phi_mem = nullptr;
  cudaError_t e = cudaSuccess;
  // measurement-side tables, and their running mean re-formed from the
  // converted tables so that it stays their p-weighted sum
  if (psi_change) {
    const long long n = (long long)p->dp.m * p->desc.levels;
    if ((e = cudaMallocAsync(&psi_mem, (size_t)n * esz, st)) == cudaSuccess &&
        (e = launch_convert(n, s->psi, s->psi_fmt, psi_mem, storage, st)) == cudaSuccess)
      e = launch_table_mean(p->dp, psi_mem, storage, s->psi_mean, st);
  }
  // image-side tables (level 0 and the coarse levels, one region), likewise
  if (e == cudaSuccess && phi_change) {
    long long n = (long long)p->dp.d;
    for (int l = 1; l < p->desc.levels; ++l)
      n += (long long)p->dp.lg[l + 1].nl * p->dp.lg[l + 1].nl;
    if ((e = cudaMallocAsync(&phi_mem, (size_t)n * esz, st)) == cudaSuccess &&
        (e = launch_convert(n, s->phi0, s->phi_fmt, phi_mem, storage, st)) == cudaSuccess)
      e = launch_phi_mean(p->dp, phi_mem, phi_mem, s->phic_off, storage, s->phi_mean, st);
  }
  if (e != cudaSuccess) {
    if (psi_mem) cudaFreeAsync(psi_mem, st);
    if (phi_mem) cudaFreeAsync(phi_mem, st);
    return cuda_fail(e, "table conversion");
  }
  if (psi_change) {
    if (s->psi_block) cudaFreeAsync(s->psi_block, st);
    s->psi_block = psi_mem;
    s->psi = psi_mem;
    s->psi_fmt = storage;
  }
  if (phi_change) {
    if (s->phi_block) cudaFreeAsync(s->phi_block, st);
    s->phi_block = phi_mem;
    s->phi0 = phi_mem;
    s->phic = phi_mem;
    s->phi_fmt = storage;
  }
  s->stream = st;
  s->gen += 1;   // graphs captured with the old tables are captured again
  return IMASK_OK;
}

imask_status imask_state_destroy(imask_state_t s) {
  if (!s) return IMASK_OK;
  if (s->self_batch) imask_batch_destroy(s->self_batch);
  // the work on aux and aux2 is joined into s->stream at the end of every
  // step, so the frees below, ordered on s->stream, come after it
  if (s->aux) cudaStreamDestroy(s->aux);
  if (s->aux2) cudaStreamDestroy(s->aux2);
  for (cudaEvent_t ev : {s->ev_fork, s->ev_fp, s->ev_start, s->ev_bp, s->ev_upd[0], s->ev_upd[1],
                        s->ev_order})
    if (ev) cudaEventDestroy(ev);
  if (s->psi_block) cudaFreeAsync(s->psi_block, s->stream);
  if (s->phi_block) cudaFreeAsync(s->phi_block, s->stream);
  if (s->block) cudaFreeAsync(s->block, s->stream);
  delete s;
  return IMASK_OK;
}

imask_status imask_solve(imask_plan_t p, const float *b_dev, uint64_t seed, int32_t iters,
                         float *x_dev, void *stream) {
  if (!p || !b_dev || !x_dev) return fail(IMASK_ERR_INVALID, "NULL argument");
  if (iters < 0) return fail(IMASK_ERR_INVALID, "iters < 0");
  imask_state_t s = nullptr;
  imask_status rc = imask_state_create(p, b_dev, seed, &s, stream);
  if (rc != IMASK_OK) return rc;
  rc = imask_step(s, iters, stream);
  if (rc == IMASK_OK) rc = imask_state_get_x(s, x_dev, stream);
  imask_state_destroy(s);
  return rc;
}

imask_status imask_rel_distance(int64_t n, const float *a_dev, const float *b_dev, double *out,
                                void *stream) {
  if (!a_dev || !b_dev || !out || n < 0) return fail(IMASK_ERR_INVALID, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  void *mem = nullptr;
  CK(cudaMallocAsync(&mem, (2 * reduce_blocks() + 2) * sizeof(double), st), "cudaMallocAsync");
  double *part = (double *)mem, *res = part + 2 * reduce_blocks();
  double h[2] = {0, 0};
  cudaError_t e = launch_diff64(n, a_dev, b_dev, part, res, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(mem, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "rel_distance");
  if (!isfinite(h[0]) || !isfinite(h[1])) return fail(IMASK_ERR_NONFINITE, "non-finite input");
  *out = h[1] > 0 ? h[0] / h[1] : h[0];
  return IMASK_OK;
}

imask_status imask_pdhg_params(double norm_K, double mu, double rho, double out[3]) {
  if (!out) return fail(IMASK_ERR_INVALID, "NULL argument");
  if (!(norm_K > 0.0) || !(mu > 0.0) || !(rho > 0.0 && rho <= 1.0))
    return fail(IMASK_ERR_INVALID, "need norm_K > 0, mu > 0, 0 < rho <= 1");
  const double kappa = sqrt(1.0 + norm_K * norm_K / (mu * rho * rho));
  out[0] = 1.0 / (kappa - 1.0);
  out[1] = 1.0 / ((kappa - 1.0) * mu);
  out[2] = 1.0 - 2.0 / (1.0 + kappa);
  return IMASK_OK;
}

imask_status imask_pdhg(imask_plan_t p, const float *b_dev, int32_t iters, double s_step,
                        double t_step, double theta, float *x_dev, void *stream) {
  NvtxRange nv("imask_pdhg");
  if (!p || !b_dev || !x_dev) return fail(IMASK_ERR_INVALID, "NULL argument");
  if (iters < 0) return fail(IMASK_ERR_INVALID, "iters < 0");
  if (!(s_step > 0.0) || !(t_step > 0.0) || !isfinite(theta))
    return fail(IMASK_ERR_INVALID, "PDHG needs s > 0, t > 0 and a finite theta");
  cudaStream_t st = (cudaStream_t)stream;
  const long long d = p->dp.d, m = p->dp.m;
  const int r = p->desc.levels;
  Scratch sc;
  unsigned mask = 0;
  for (int li = 1; li <= r; ++li) mask |= 1u << li;
  imask_status rc = scratch_alloc(p, mask, true, st, sc);
  if (rc != IMASK_OK) return rc;
  Carve cv;
  const size_t o_x = cv.take(d), o_xb = cv.take(d), o_xn = cv.take(d), o_kty = cv.take(d),
               o_ti = cv.take(d), o_y = cv.take(m), o_kx = cv.take(m), o_tm = cv.take(m),
               o_tv = p->desc.reg != 0 ? cv.take(5 * d) : 0;
  void *mem = nullptr;
  cudaError_t e = cudaMallocAsync(&mem, cv.off * sizeof(float), st);
  if (e != cudaSuccess) {
    scratch_free(sc);
    return cuda_fail(e, "cudaMallocAsync(pdhg)");
  }
  float *B = (float *)mem;
  float *x = B + o_x, *xb = B + o_xb, *xn = B + o_xn, *kty = B + o_kty, *ti = B + o_ti;
  float *y = B + o_y, *kx = B + o_kx, *tm = B + o_tm, *tv = p->desc.reg != 0 ? B + o_tv : nullptr;
  const float s = (float)s_step, t = (float)t_step, th = (float)theta;
  // quadratic prox folded into the extrapolation kernel's scale
  const float scale = p->desc.reg == 0 ? (float)(1.0 / (1.0 + t_step * p->mu)) : 1.0f;
  do {
    if ((e = cudaMemsetAsync(mem, 0, cv.off * sizeof(float), st)) != cudaSuccess) break;
    for (int it = 0; it < iters && rc == IMASK_OK && e == cudaSuccess; ++it) {
      // y <- (y + s (Kbar xbar - b)) / (1 + s)
      for (int l = 0; l < r && rc == IMASK_OK && e == cudaSuccess; ++l) {
        rc = apply_K(p, l, xb, l == 0 ? kx : tm, sc, st);
        if (rc != IMASK_OK) break;
        e = l == 0 ? launch_scale(m, (float)p->probs[0], kx, st)
                   : launch_axpy(m, (float)p->probs[l], tm, kx, st);
      }
      if (rc != IMASK_OK || e != cudaSuccess) break;
      if ((e = launch_pdhg_dual(m, kx, b_dev, s, y, st)) != cudaSuccess) break;
      // x+ = prox_{t R}(x - t Kbar^T y), xbar = x+ + theta (x+ - x)
      for (int l = 0; l < r && rc == IMASK_OK && e == cudaSuccess; ++l) {
        rc = apply_KT(p, l, y, l == 0 ? kty : ti, sc, st);
        if (rc != IMASK_OK) break;
        e = l == 0 ? launch_scale(d, (float)p->probs[0], kty, st)
                   : launch_axpy(d, (float)p->probs[l], ti, kty, st);
      }
      if (rc != IMASK_OK || e != cudaSuccess) break;
      if ((e = launch_copy(d, x, xn, st)) != cudaSuccess) break;
      if ((e = launch_axpy(d, -t, kty, xn, st)) != cudaSuccess) break;
      if (p->desc.reg != 0 && (e = launch_reg_prox(p, t, xn, tv, st)) != cudaSuccess) break;
      e = launch_pdhg_primal(d, scale, th, xn, x, xb, st);
    }
    if (rc == IMASK_OK && e == cudaSuccess)
      e = cudaMemcpyAsync(x_dev, x, d * sizeof(float), cudaMemcpyDeviceToDevice, st);
  } while (false);
  cudaFreeAsync(mem, st);
  scratch_free(sc);
  if (rc != IMASK_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "pdhg");
  return IMASK_OK;
}

imask_status imask_objective(imask_plan_t p, const float *x_dev, const float *b_dev, double *out,
                             void *stream) {
  if (!p || !x_dev || !b_dev || !out) return fail(IMASK_ERR_INVALID, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const long long d = p->dp.d, m = p->dp.m;
  Scratch s;
  unsigned mask = 0;
  for (int li = 1; li <= p->desc.levels; ++li) mask |= 1u << li;
  imask_status rc = scratch_alloc(p, mask, false, st, s);
  if (rc != IMASK_OK) return rc;
  void *mem = nullptr;
  cudaError_t e = cudaMallocAsync(
      &mem, (2 * align64(m)) * sizeof(float) + (2 * reduce_blocks() + 8) * sizeof(double), st);
  if (e != cudaSuccess) {
    scratch_free(s);
    return cuda_fail(e, "cudaMallocAsync(objective)");
  }
  float *kx = (float *)mem, *t = kx + align64(m);
  double *part = (double *)(t + align64(m)), *res = part + 2 * reduce_blocks();
  double h[4] = {0, 0, 0, 0};
  do {
    if ((e = launch_fill(m, 0.0f, kx, st)) != cudaSuccess) break;
    for (int l = 0; l < p->desc.levels && rc == IMASK_OK; ++l) {
      rc = apply_K(p, l, x_dev, t, s, st);
      if (rc == IMASK_OK) e = launch_axpy(m, (float)p->probs[l], t, kx, st);
      if (e != cudaSuccess) break;
    }
    if (rc != IMASK_OK || e != cudaSuccess) break;
    if ((e = launch_diff64(m, kx, b_dev, part, res, st)) != cudaSuccess) break;
    if ((e = launch_dot64(d, x_dev, x_dev, part, res + 2, st)) != cudaSuccess) break;
    if (p->desc.reg != 0 &&
        (e = launch_tv_value64(p->dp, x_dev, p->desc.reg == 1 ? (float)p->desc.tv_eps : 0.0f,
                               part, res + 3, st)) != cudaSuccess)
      break;
    e = cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, st);
  } while (false);
  cudaFreeAsync(mem, st);
  scratch_free(s);
  if (rc != IMASK_OK) return rc;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "objective");
  // reg 2 has no quadratic term; its nonnegativity indicator is not evaluated
  double obj = 0.5 * h[0] + (p->desc.reg == 2 ? 0.0 : 0.5 * p->mu * h[2]);
  if (p->desc.reg != 0) obj += p->desc.tv_lambda * h[3];
  if (!isfinite(obj)) return fail(IMASK_ERR_NONFINITE, "objective is not finite");
  *out = obj;
  return IMASK_OK;
}

imask_status imask_selftest_projector_timeout(imask_plan_t p, void *stream) {
  if (!p) return fail(IMASK_ERR_INVALID, "NULL plan");
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc;
  imask_status rc = scratch_alloc(p, 1u, false, st, sc);   // level -1 images (zeros)
  if (rc != IMASK_OK) return rc;
  void *sino = nullptr;
  cudaError_t e = cudaMallocAsync(&sino, (size_t)p->dp.m * sizeof(float), st);
  if (e == cudaSuccess)
    e = launch_fp(p->dp, fixed_level(-1), sc.pads, (float *)sino, no_dual(), p->n_cta_x,
                  p->n_cta_y, p->d_err, st, 1);
  if (sino) cudaFreeAsync(sino, st);
  scratch_free(sc);
  if (e != cudaSuccess) return cuda_fail(e, "self-test projector");
  return IMASK_OK;
}

imask_status imask_probe_smem(double out[2], void *stream) {
  if (!out) return fail(IMASK_ERR_INVALID, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, n_sm = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  const int blocks = 8 * n_sm, iters = 4096;
  void *mem = nullptr;
  CK(cudaMallocAsync(&mem, 256, st), "cudaMallocAsync(probe)");
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  for (int rmw = 0; rmw < 2 && e == cudaSuccess; ++rmw) {
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      float ms = 0.0f;
      if ((e = cudaEventRecord(a, st)) != cudaSuccess) break;
      if ((e = launch_probe_smem(blocks, iters, rmw, (float *)mem, st)) != cudaSuccess) break;
      if ((e = cudaEventRecord(b, st)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
      if ((e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) break;
      if (rep > 0 && ms < best) best = ms;   // the first launch warms up
    }
    // bytes moved through shared memory: 4 per load, 8 per read-modify-write
    const double bytes = (double)blocks * 256 * iters * 8 * (rmw ? 8.0 : 4.0);
    out[rmw] = bytes / (best * 1e-3) / 1e9;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFreeAsync(mem, st);
  if (e != cudaSuccess) return cuda_fail(e, "shared-memory probe");
  return IMASK_OK;
}

imask_status imask_profile_enable(int32_t period) {
  if (period < 0) return fail(IMASK_ERR_INVALID, "profile period must be >= 0");
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = period != 0;
  g_prof.period = period;
  return IMASK_OK;
}

imask_status imask_profile_read(double ms[24], int64_t count[24], int32_t reset) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  for (auto &r : g_prof.pending) {
    float t = 0.0f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      g_prof.ms[r.kind * 8 + r.level] += t;
      g_prof.count[r.kind * 8 + r.level] += 1;
    }
    g_prof.pool.push_back(r.a);
    g_prof.pool.push_back(r.b);
  }
  g_prof.pending.clear();
  for (int i = 0; i < 24; ++i) {
    if (ms) ms[i] = g_prof.ms[i];
    if (count) count[i] = g_prof.count[i];
  }
  if (reset) {
    for (int i = 0; i < 24; ++i) {
      g_prof.ms[i] = 0;
      g_prof.count[i] = 0;
    }
  }
  return IMASK_OK;
}

}  // extern "C"
