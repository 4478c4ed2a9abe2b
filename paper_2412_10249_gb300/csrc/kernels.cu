// kernels.cu -- device code of libimask.so (sm_103a).
//
// The hot path of one ImaSk iteration (Alg. 1) is three launches:
//   k_fp      forward projection K_ell x (Joseph, one ray per thread and slot)
//             over image strips staged in shared memory by TMA bulk copies,
//             with the dual SAGA update and dual prox fused into its epilogue;
//   k_bp      back-projection R_ell^T y on the level grid, owner-computes
//             (each thread owns a line segment of a tile and applies the rays
//             crossing the tile in private shared-memory accumulators; no
//             atomics), the exact transpose of k_fp's weights;
//   k_update  the image-side adjoint sketch (T_ell^T or S_r), the primal SAGA
//             update and prox, and the image-side sketch T_ell' / S_r of the
//             new iterate for the next drawn level (fused "sketch on load").
// The level of every launch is drawn on the device from (seed, k).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "imask_internal.h"

namespace {

std::atomic<int64_t> g_launches{0};

constexpr float kMagic = 12582912.0f;   // 1.5 * 2^23: floor via round-down add
constexpr int kMagicBits = 0x4B400000;
#define kMagic2 make_float2(kMagic, kMagic)
#define kNegMagic2 make_float2(-kMagic, -kMagic)
#define kMinusOne2 make_float2(-1.0f, -1.0f)
constexpr float kBpEps = 0.01f;          // slack (in bins) of the back-projector's ray range
constexpr int kWaitLimit = 1 << 20;      // bounded mbarrier polls before giving up

}  // namespace

// Index checks of a checked build (-DIMASK_BOUNDS_CHECK): a computed index
// outside its buffer sets a bit of this flag (1 projector image line, 2
// back-projector staging, 3 sketch / update writes, 4 pixel-driven
// back-projector views and windows) and the access is skipped
// or redirected to element 0; the host reads the flag in imask_plan_check.
// In the normal build the checks compile to nothing.
__device__ unsigned int g_index_check_flag = 0u;

namespace {

#ifdef IMASK_BOUNDS_CHECK
#define IMASK_INDEX_OK(cond, bit) \
  ((cond) ? true : (atomicOr(&g_index_check_flag, 1u << (bit)), false))
#else
#define IMASK_INDEX_OK(cond, bit) true
#endif

// ---------------------------------------------------------------------------------
// Level draw: SplitMix64 output k of `seed` against the integer thresholds of the
// cumulative probabilities (Alg. 1, sampling step).
// ---------------------------------------------------------------------------------
__host__ __device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                                     unsigned long long k) {
  unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ int draw_level(const DevPlan &P, unsigned long long seed,
                                                   long long k) {
  const unsigned long long u = splitmix64_at(seed, (unsigned long long)k);
  int l = 0;
  for (int t = 0; t + 1 < P.levels; ++t) l += (u >= P.thr[t]) ? 1 : 0;
  return l;
}

// Iteration counter of a launch.
__device__ __forceinline__ long long sel_k(const LevelSel &s) {
  return s.k_dev ? *s.k_dev + s.k_add : s.k;
}

// Projector-side (dual) level of a launch.
__device__ __forceinline__ int sel_level(const DevPlan &P, const LevelSel &s) {
  return s.fixed >= -1 ? s.fixed : draw_level(P, s.seed, sel_k(s));
}

// Back-projector / image-side (primal) level of a launch.
__device__ __forceinline__ int sel_level_x(const DevPlan &P, const LevelSel &s) {
  return s.fixed >= -1 ? s.fixed : draw_level(P, s.seed_x, sel_k(s));
}

// ---------------------------------------------------------------------------------
// mbarrier / TMA bulk-copy helpers (inline PTX)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One 1-D bulk copy global -> shared that completes a transaction on `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Polls the barrier phase `parity` at most kWaitLimit times.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = kWaitLimit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// ---------------------------------------------------------------------------------
// Local interpolation frames.
//
// Along its major axis a ray is sampled at lines (columns for x-major rays,
// rows for y-major rays) c = 0..nl-1 of the level grid, at the fractional
// cross coordinate q(c) = a 2^-ell - 1/2 + (c - (nl-1)/2) t.  In FP32, q of
// several hundred carries an absolute error of ~1e-5, which is the full error
// budget of the operators, so q is never formed: lines are grouped in blocks of
// LBLOCK, and for each (ray, block) the origin q(cB) = I + r is split into an
// integer I and a remainder |r| <~ 1 with double-float arithmetic from the
// two-word ray parameters a = a_hi + a_lo, t = t_hi + t_lo.  Inside the block
// q(cB + d) - I = r + d t_hi, a number below LBLOCK + 1, exact to ~1e-6.  The
// projector and the back-projector call the same function, so their weights
// agree to the last bit.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void block_origin(float a_hi, float a_lo, float t_hi, float t_lo,
                                             float s, float cc, int &I, float &r) {
  const float A = a_hi * s;                 // exact: s is a power of two
  const float Pp = cc * t_hi;
  const float E = fmaf(cc, t_hi, -Pp);      // exact rounding error of the product
  const float S = A + Pp;                   // two-sum S + e1 = A + Pp
  const float bb = S - A;
  const float e1 = (A - (S - bb)) + (Pp - bb);
  const float tq = S + kMagic;              // round to the nearest integer (|S| < 2^22)
  const float Sr = tq - kMagic;
  I = __float_as_int(tq) - kMagicBits;
  r = (S - Sr) + (e1 + E + fmaf(a_lo, s, fmaf(cc, t_lo, -0.5f)));
}

// Table entries in one of the storage formats (0 float, 1 bfloat16, 2 binary16):
// read as float; a store rounds to nearest even and returns the stored value.
__device__ __forceinline__ float tab_load(const void *t, size_t i, int fmt) {
  if (fmt == 1) return __bfloat162float(((const __nv_bfloat16 *)t)[i]);
  if (fmt == 2) return __half2float(((const __half *)t)[i]);
  return ((const float *)t)[i];
}

__device__ __forceinline__ float tab_store(void *t, size_t i, float v, int fmt) {
  if (fmt == 1) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    ((__nv_bfloat16 *)t)[i] = h;
    return __bfloat162float(h);
  }
  if (fmt == 2) {
    const __half h = __float2half_rn(v);
    ((__half *)t)[i] = h;
    return __half2float(h);
  }
  ((float *)t)[i] = v;
  return v;
}

// ---------------------------------------------------------------------------------
// Forward projector (Joseph) with the fused dual epilogue.
//
// Rays are listed x-major first, then y-major.  CTA b < n_cta_x takes x-major
// rays [b*fp_chunk_x, ...), the others y-major rays (chunks sized so that the
// grid fills the GPU in one wave).  An x-major ray marches over
// the columns of the x-major padded image (one line per column, rows
// contiguous) and interpolates linearly between the rows I + floor(r + d t) and
// the next one.  Strips of tc lines are streamed through FP_STAGES
// shared-memory buffers by cp.async.bulk.  Every line carries IMASK_PAD zeros
// before and IMASK_PAD_END after the grid rows.  Within one block of LBLOCK
// lines a ray moves by at most 16 rows (|slope| <= 1), so a block that touches
// the grid reads rows in [-18, nl + 16], inside the padding, and a block that
// misses the grid entirely is redirected into the leading zeros: no per-sample
// bounds check is needed.
// ---------------------------------------------------------------------------------
// Ray slot r of thread tid in a CTA whose rays start at `begin`.  Slots go in
// pairs: pair p of warp w covers the 64 consecutive list entries from
// begin + 2 p FP_THREADS + 64 w, lane l taking entries l and l + 32, so that
// the two rays of a pair are close bins of one view (they hit or miss the
// grid together) and the 32 lanes of a slot read 32 neighbouring rays' rows
// (no shared-memory bank conflicts).
__device__ __forceinline__ int fp_ray(int begin, int r, int tid) {
  return begin + (r >> 1) * (2 * FP_THREADS) + (tid >> 5) * 64 + (r & 1) * 32 + (tid & 31);
}

// One projector CTA (block `bid` of the plan's projector grid); the plan and
// the arguments may live in kernel parameters (k_fp) or in device memory
// (k_fp_multi, several solves in one launch).
__device__ __forceinline__ void fp_body(const DevPlan &P, const LevelSel &sel, const PadSet &pads,
                                        float *sino, const DualArgs &D, int n_cta_x,
                                        unsigned int *err, int test_skip_first_strip, int bid) {
  extern __shared__ __align__(128) float fp_smem[];
  __shared__ __align__(8) unsigned long long full_bar[FP_STAGES];
  __shared__ unsigned int released[FP_STAGES];   // warps done with each stage (monotone)
  __shared__ unsigned int issued[FP_STAGES];     // bulk loads issued into each stage

  const int ell = sel_level(P, sel);
  const LevelGeom G = P.lg[ell + 1];
  const bool xaxis = bid < n_cta_x;
  const int chunk = xaxis ? bid : bid - n_cta_x;
  const int csz = xaxis ? P.fp_chunk_x : P.fp_chunk_y;
  const int begin = xaxis ? chunk * csz : P.m_x + chunk * csz;
  const int end = xaxis ? min(begin + csz, P.m_x) : min(begin + csz, P.m);
  const float *img = xaxis ? pads.T[ell + 1] : pads.R[ell + 1];
  const int tid = threadIdx.x;

  static_assert(FP_RAYS % 2 == 0, "rays go in pairs");
  float ahi[FP_RAYS], alo[FP_RAYS], thi[FP_RAYS], tlo[FP_RAYS], rl[FP_RAYS], acc[FP_RAYS];
  int boff[FP_RAYS];
#pragma unroll
  for (int r = 0; r < FP_RAYS; ++r) {
    const int idx = fp_ray(begin, r, tid);
    acc[r] = 0.0f;
    rl[r] = 0.0f;
    boff[r] = 0;
    if (idx < end) {
      const float4 p = P.rays[idx];
      const float2 lo = P.rays_lo[idx];
      ahi[r] = p.x;
      thi[r] = p.y;
      alo[r] = lo.x;
      tlo[r] = lo.y;
    } else {
      ahi[r] = -16384.0f;  // far below the grid: the clamped index reads zeros
      thi[r] = 0.0f;
      alo[r] = 0.0f;
      tlo[r] = 0.0f;
    }
  }

  const int tc = G.tc, ls = G.ls;
  const int nstrips = G.lines / tc;
  const uint32_t strip_bytes = (uint32_t)(tc * ls) * 4u;
  if (tid == 0) {
    for (int s = 0; s < FP_STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      released[s] = 0u;
      issued[s] = 0u;
    }
    mbar_fence_init();
  }
  __syncthreads();
  // (test_skip_first_strip: a self-test leaves the first strip unrequested, so
  // that every warp's bounded wait for it runs out -- after a short limit)
  const int wait_limit = test_skip_first_strip ? 256 : kWaitLimit;
  if (tid == 0) {
    for (int s = test_skip_first_strip ? 1 : 0; s < FP_STAGES && s < nstrips; ++s) {
      bulk_load(smem_u32(fp_smem + s * FP_STAGE_FLOATS), img + (size_t)s * tc * ls, strip_bytes,
                smem_u32(&full_bar[s]));
      issued[s] += 1u;
    }
  }
  constexpr unsigned kWarps = FP_THREADS / 32;
  const int lane = tid & 31;

  // Warps move through the strips independently (up to FP_STAGES apart): a
  // warp releases a stage when it is done with it, and the warp that releases
  // it last refills it with the strip FP_STAGES further on.
  bool failed = false;
  unsigned act = 0u;   // ray slots with at least one on-grid ray in the warp (this block)
  // The strip loop, compiled for the common strip heights (a fixed trip
  // count through the strip, and block starts known at compile time when the
  // height is a multiple of LBLOCK) and once for any other height.
  auto strips = [&](auto tc_const) {
    constexpr int TC = decltype(tc_const)::value;
    const int tcv = TC > 0 ? TC : tc;
    for (int s = 0; s < nstrips; ++s) {
      const int st = s % FP_STAGES;
      const uint32_t parity = (uint32_t)((s / FP_STAGES) & 1);
      const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&full_bar[st]), parity, wait_limit));
      if (!ok) {
        failed = true;
        break;
      }
      const float *buf = fp_smem + st * FP_STAGE_FLOATS;
      float part[FP_RAYS];
  #pragma unroll
      for (int r = 0; r < FP_RAYS; ++r) part[r] = 0.0f;
  #pragma unroll
      for (int cc = 0; cc < tcv; cc += 4) {
        const int c = s * tcv + cc;
        if ((c & (LBLOCK - 1)) == 0) {
          const float ccm = (float)c - G.cmid;
          act = 0u;
  #pragma unroll
          for (int r = 0; r < FP_RAYS; ++r) {
            int I;
            block_origin(ahi[r], alo[r], thi[r], tlo[r], G.inv2l, ccm, I, rl[r]);
            // rows of the block's first and last sample
            const int f0 = __float_as_int(__fadd_rd(rl[r], kMagic)) - kMagicBits;
            const int f1 =
                __float_as_int(__fadd_rd(fmaf((float)(LBLOCK - 1), thi[r], rl[r]), kMagic)) -
                kMagicBits;
            const int lo = I + min(f0, f1), hi = I + max(f0, f1);
            // off the grid (no row in [0, nl-1] is read): land in the leading zeros
            const bool off = (hi + 1 < 0) || (lo > G.nl - 1);
            boff[r] = off ? (IMASK_PAD / 2) - f0 : IMASK_PAD + I;
            // a slot whose 32 rays all miss the grid in this block adds exactly
            // zero: the warp skips its samples (the branch is warp-uniform)
            act |= (__any_sync(0xffffffffu, !off) ? 1u : 0u) << r;
          }
        }
        const float d0 = (float)(c & (LBLOCK - 1));
        // Rays go in pairs through the packed FP32x2 instructions of sm_100+
        // (one issue slot for both rays; per component the rounding is that of
        // the scalar operation, so the samples are bit for bit those of
        // fmaf / __fadd_rd / subtraction).  A pair is skipped when neither of its
        // slots has a ray on the grid in this block.
  #pragma unroll
        for (int r = 0; r < FP_RAYS; r += 2) {
          if (!(act & (3u << r))) continue;
          const float2 t2 = make_float2(thi[r], thi[r + 1]);
          const float2 r2 = make_float2(rl[r], rl[r + 1]);
          float2 a[4];
  #pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float dcf = d0 + (float)u;
            const float *line = buf + (cc + u) * ls;
            const float2 q = __ffma2_rn(make_float2(dcf, dcf), t2, r2);
            const float2 tq = __fadd2_rd(q, kMagic2);
            int i0 = boff[r] + (__float_as_int(tq.x) - kMagicBits);
            int i1 = boff[r + 1] + (__float_as_int(tq.y) - kMagicBits);
            if (!IMASK_INDEX_OK(i0 >= 0 && i0 + 1 < ls, 1)) i0 = 0;
            if (!IMASK_INDEX_OK(i1 >= 0 && i1 + 1 < ls, 1)) i1 = 0;
            // f = q - (tq - magic), the subtraction as a fused multiply-add by -1
            const float2 f = __ffma2_rn(__fadd2_rn(tq, kNegMagic2), kMinusOne2, q);
            const float2 v0 = make_float2(line[i0], line[i1]);
            const float2 v1 = make_float2(line[i0 + 1], line[i1 + 1]);
            // independent samples, summed as a tree
            a[u] = __ffma2_rn(f, __ffma2_rn(v0, kMinusOne2, v1), v0);
          }
          const float2 sum = __fadd2_rn(__fadd2_rn(a[0], a[1]), __fadd2_rn(a[2], a[3]));
          part[r] += sum.x;
          part[r + 1] += sum.y;
        }
      }
  #pragma unroll
      for (int r = 0; r < FP_RAYS; ++r) acc[r] += part[r];
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();   // this warp's reads of the stage come first
        const unsigned n = atomicAdd(&released[st], 1u) + 1u;
        if (n % kWarps == 0u && s + FP_STAGES < nstrips) {
          fence_proxy_async();
          bulk_load(smem_u32(fp_smem + st * FP_STAGE_FLOATS),
                    img + (size_t)(s + FP_STAGES) * tcv * ls, strip_bytes, smem_u32(&full_bar[st]));
          issued[st] += 1u;   // only the last releaser of a stage issues its refill
        }
      }
    }
  };
  switch (tc) {
    case 16: strips(std::integral_constant<int, 16>{}); break;
    case 20: strips(std::integral_constant<int, 20>{}); break;
    case 32: strips(std::integral_constant<int, 32>{}); break;
    default: strips(std::integral_constant<int, 0>{}); break;
  }
  if (__syncthreads_or(failed)) {
    if (tid == 0) {
      atomicOr(err, 1u);
      // give the copies still in flight a bounded chance to land before exit:
      // at most one load per stage is outstanding, the latest issued one
      for (int s = 0; s < FP_STAGES; ++s)
        if (issued[s] > 0u) mbar_wait(smem_u32(&full_bar[s]), (issued[s] - 1u) & 1u);
    }
    return;
  }

  // Epilogue.  Every load of the four rays is issued before the first store
  // (two rounds of independent loads: the ray's sinogram index, then the
  // state it indexes), so that a warp waits for two memory latencies rather
  // than two per ray: the stores of one ray could alias the next ray's loads,
  // which would otherwise keep them in order.
  int qv[FP_RAYS];
  float gz[FP_RAYS];
#pragma unroll
  for (int r = 0; r < FP_RAYS; ++r) {
    const int idx = fp_ray(begin, r, tid);
    qv[r] = -1;
    gz[r] = 0.0f;
    if (idx >= end) continue;
    if (D.on) {
      // a solve's measurement-space vectors are kept in ray-list order: the
      // ray's entry is its own index (coalesced, no index load), and only the
      // ray's weight is read back
      qv[r] = idx;
      gz[r] = __ldg(&P.rays[idx].z) * G.scale2l;
    } else {
      // the bare operator writes the sinogram in (view, bin) order
      const float4 p = P.rays[idx];
      qv[r] = __float_as_int(p.w);
      gz[r] = p.z * G.scale2l;
    }
  }
  if (!D.on) {
#pragma unroll
    for (int r = 0; r < FP_RAYS; ++r)
      if (qv[r] >= 0) sino[qv[r]] = acc[r] * gz[r];
    return;
  }
  // Alg. 1: zeta = psi_new - psi_l + sum p psi; y+ = (y + s zeta - s b)/(1+s);
  // the running mean and the table entry take the refreshed value.  With
  // snapshot tables the projector already applied K_l to the input
  // difference, so v is psi_new - psi_l itself.  With 16-bit tables the
  // refreshed entry is stored rounded and the running mean moves by the
  // stored change, so that it stays the p-weighted sum of the stored tables.
  float old[FP_RAYS], pmv[FP_RAYS], bv[FP_RAYS], yv[FP_RAYS];
#pragma unroll
  for (int r = 0; r < FP_RAYS; ++r) {
    old[r] = pmv[r] = bv[r] = yv[r] = 0.0f;
    const int q = qv[r];
    if (q < 0) continue;
    if (D.psi) {
      const size_t qi = (size_t)ell * P.m + q;
      if (D.psi_fmt == 1)
        old[r] = __bfloat162float(((const __nv_bfloat16 *)D.psi)[qi]);
      else if (D.psi_fmt == 2)
        old[r] = __half2float(((const __half *)D.psi)[qi]);
      else
        old[r] = ((const float *)D.psi)[qi];
    }
    pmv[r] = D.psi_mean[q];
    bv[r] = D.b[q];
    yv[r] = D.y_in[q];
  }
#pragma unroll
  for (int r = 0; r < FP_RAYS; ++r) {
    const int q = qv[r];
    if (q < 0) continue;
    const float v = acc[r] * gz[r];
    float delta = v, dmean = v;
    if (D.psi) {
      const size_t qi = (size_t)ell * P.m + q;
      float stored = v;
      if (D.psi_fmt == 1) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        ((__nv_bfloat16 *)D.psi)[qi] = h;
        stored = __bfloat162float(h);
      } else if (D.psi_fmt == 2) {
        const __half h = __float2half_rn(v);
        ((__half *)D.psi)[qi] = h;
        stored = __half2float(h);
      } else {
        ((float *)D.psi)[qi] = v;
      }
      delta = v - old[r];
      dmean = stored - old[r];
    }
    const float zeta = delta + pmv[r];
    D.y_out[q] = fmaf(D.sigma, zeta - bv[r], yv[r]) * D.inv_1ps;
    D.psi_mean[q] = fmaf(P.probs[ell], dmean, pmv[r]);
  }
}

__global__ void __launch_bounds__(FP_THREADS, 2)
    k_fp(DevPlan P, LevelSel sel, PadSet pads, float *sino, DualArgs D, int n_cta_x,
         unsigned int *err, int test_skip_first_strip) {
  fp_body(P, sel, pads, sino, D, n_cta_x, err, test_skip_first_strip, (int)blockIdx.x);
}

// ---------------------------------------------------------------------------------
// Back-projector: g = R_ell^T y on the level grid, owner-computes (no atomics).
//
// The x-major and y-major rays go to separate CTAs.  An x-major CTA owns a tile
// of BP_W columns x BP_SEG rows of level pixels and one of bp_vgo groups of
// consecutive views that hold x-major rays, the groups holding about equal
// numbers of such rays (the consumer adds the partial images, 2 bp_vgo of
// them, in a fixed order).  CTAs take (role, tile) pairs from the plan's
// heaviest-first order, so that light tiles fill the last wave.  Thread t owns the column t % BP_W of the tile, a
// segment of BP_SEG rows with private accumulators in shared memory, and takes
// every (BP_THREADS / BP_W)-th staged ray.  y-major CTAs do the same with rows
// and columns exchanged.
//   prologue  each view of the range gets its ray window: the bins of the
//             corners of the tile box widened by one pixel across the major
//             axis (the bin map is affine for parallel beam and
//             linear-fractional for fan beam, so its extremes over the box
//             are at corners); window lengths are prefix-summed into one flat
//             ray list;
//   pipeline  the list is processed in chunks of BP_SLOTS entries; while
//             chunk k is scattered from one shared-memory buffer, the raw data
//             of chunk k+1 (parameters, low words, y) is loaded into registers
//             (each entry's view is found by galloping from the thread's
//             previous one), then converted to (r, t, g y, I') in the local
//             frame of the tile's line block (block_origin, as in k_fp) and
//             stored into the other buffer; one barrier per chunk;
//   scatter   a thread applies a ray to its segment exactly as k_fp samples
//             it: q = r + d t, row I + floor(q) gets (1 - f) g y and the next
//             row f g y, f = q - floor(q); rows outside the segment land in
//             guard slots (one unsigned clamp).  Only the owner ever touches a
//             slot.
//   epilogue  every pixel sums its BP_THREADS / BP_W owners' slots.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float bin_of(const DevPlan &P, float c, float s, float x, float y) {
  if (P.geometry == 0) return fmaf(fmaf(x, c, y * s), P.inv_pitch, P.center);
  const float num = fmaf(-x, s, y * c);
  const float den = P.src_dist - fmaf(x, c, y * s);
  return fmaf(P.sd_dist * __fdividef(num, den), P.inv_pitch, P.center);
}

__device__ __forceinline__ int floor_i(float v) {
  return __float_as_int(__fadd_rd(v, kMagic)) - kMagicBits;
}

__device__ __forceinline__ int ceil_i(float v) {
  return __float_as_int(__fadd_ru(v, kMagic)) - kMagicBits;
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) {
  return fminf(fmaxf(v, lo), hi);
}

#define BP_GROUPS (BP_THREADS / BP_W)   // ray residue classes per CTA
#ifndef BP_UNROLL
#define BP_UNROLL 8                      // unrolling of the scatter loop
#endif
#define IMASK_STR(x) #x
#define IMASK_UNROLL(n) _Pragma(IMASK_STR(unroll n))
#define BP_ACC (BP_SEG + 4)             // accumulator slots per segment: 2 guards each side

// shared-memory layout of k_bp (dynamic part): two buffers of BP_SLOTS
// converted window entries, then the per-view table of the CTA's range
__device__ __forceinline__ float4 *bp_win(float4 *raw, int b) { return raw + b * BP_SLOTS; }
__device__ __forceinline__ int2 *bp_vinfo(float4 *raw) { return (int2 *)(raw + 2 * BP_SLOTS); }

// Block-wide exclusive scan of n counters held in a[0..n) (in place); a[n]
// receives the total, which is also returned.
__device__ int scan_counts(int *a, int n) {
  __shared__ int wsum[BP_THREADS / 32];
  const int per = (n + BP_THREADS - 1) / BP_THREADS;
  const int v0 = threadIdx.x * per, v1 = min(v0 + per, n);
  int sa = 0;
  for (int v = v0; v < v1; ++v) sa += a[v];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int ia = sa;
  for (int o = 1; o < 32; o <<= 1) {
    const int ta = __shfl_up_sync(0xffffffffu, ia, o);
    if (lane >= o) ia += ta;
  }
  if (lane == 31) wsum[w] = ia;
  __syncthreads();
  int ba = 0, tot = 0;
  for (int k = 0; k < BP_THREADS / 32; ++k) {
    if (k < w) ba += wsum[k];
    tot += wsum[k];
  }
  int ra = ba + ia - sa;   // exclusive prefix of this thread's run
  for (int v = v0; v < v1; ++v) {
    const int ca = a[v];
    a[v] = ra;
    ra += ca;
  }
  if (threadIdx.x == 0) a[n] = tot;
  __syncthreads();
  return tot;
}

// One back-projector work item (block `bid` of the plan's grid at the drawn
// level); returns with every shared-memory read done except the last
// barrier's.
// y_list: y is in ray-list order (a solve's dual iterate) rather than in
// (view, bin) order (the bare operator's input).
__device__ __forceinline__ void bp_body(const DevPlan &P, const LevelSel &sel,
                                        const float *__restrict__ y, int y_list,
                                        float *__restrict__ gout, unsigned int *err, int nv_cap,
                                        int bid) {
  extern __shared__ __align__(16) float4 bp_raw[];
  // private accumulators: [slot][thread]; slots 0..BP_ACC-1 are cross lines
  // -2..BP_SEG+1 of the owner's segment
  __shared__ float acc_s[BP_ACC * BP_THREADS];
  const int ell = sel_level_x(P, sel);
  const LevelGeom G = P.lg[ell + 1];
  const int nm = G.bp_nm, nc = G.bp_nc, vgo = G.bp_vgo;
  const int ntile = nm * nc;
  // CTAs go heaviest (role, tile) first so that light tiles fill the last wave
  const int rank = bid / vgo, vg = bid % vgo;
  if (rank >= 2 * ntile) return;
  const int code = P.bp_order[G.bp_order_off + rank];
  const int role = code >= ntile ? 1 : 0;   // 0: x-major rays, 1: y-major
  const int tile = code - role * ntile;
  const int mb = tile % nm, cb = tile / nm;   // march block (BP_W lines), cross block (BP_SEG)
  const int tid = threadIdx.x;
  // this CTA's views: a group of the views holding rays of its major axis
  const int *vb = P.bp_vb + ((ell + 1) * 2 + role) * (P.n_angles + 1);
  const int a0 = vb[vg];
  const int nv = vb[vg + 1] - a0;
  const int *vlist = P.bp_views + role * P.n_angles + a0;
  const float hl = G.hl, W = P.fov;
  int2 *vinfo = bp_vinfo(bp_raw);   // per view: ray-list index and y index of the window start
  int *pref = (int *)(vinfo + nv_cap);   // nv_cap + 1 prefix counts

  // ---- prologue: ray windows of every view (this CTA's major axis only) ----
  {
    const int m0 = mb * BP_W, m1 = min(m0 + BP_W, G.nl) - 1;      // march lines
    const int c0 = cb * BP_SEG, c1 = min(c0 + BP_SEG, G.nl) - 1;  // cross lines
    const float mlo = -0.5f * W + ((float)m0 + 0.5f) * hl, mhi = -0.5f * W + ((float)m1 + 0.5f) * hl;
    const float clo = -0.5f * W + ((float)c0 + 0.5f) * hl - hl;
    const float chi = -0.5f * W + ((float)c1 + 0.5f) * hl + hl;
    for (int v = tid; v < nv; v += BP_THREADS) {
      const int a = vlist[v];
      if (!IMASK_INDEX_OK(a >= 0 && a < P.n_angles, 2)) {
        vinfo[v] = make_int2(0, 0);
        pref[v] = 0;
        continue;
      }
      const ViewInfo V = P.views[a];
      float mn = 1.0e30f, mx = -1.0e30f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float mcoord = (k & 1) ? mhi : mlo, ccoord = (k & 2) ? chi : clo;
        const float j = role == 0 ? bin_of(P, V.c, V.s, mcoord, ccoord)
                                  : bin_of(P, V.c, V.s, ccoord, mcoord);
        mn = fminf(mn, j);
        mx = fmaxf(mx, j);
      }
      const int j0 = role == 0 ? V.xj0 : V.yj0, j1 = role == 0 ? V.xj1 : V.yj1;
      const int lo = max(ceil_i(clampf(mn - kBpEps, -1.0e6f, 1.0e6f)), j0);
      const int hi = min(floor_i(clampf(mx + kBpEps, -1.0e6f, 1.0e6f)), j1 - 1);
      const int base = role == 0 ? V.xoff - V.xj0 : V.yoff - V.yj0;
      vinfo[v] = make_int2(base + lo, a * P.n_det + lo);
      pref[v] = max(hi - lo + 1, 0);
    }
    for (int k = tid; k < BP_ACC * BP_THREADS; k += BP_THREADS) acc_s[k] = 0.0f;
  }
  __syncthreads();
  const int NR = scan_counts(pref, nv);

  const int g = tid / BP_W;                          // ray residue class of this thread
  const float dseg = (float)(tid % BP_W);            // own march line inside the block
  const float cco = (float)(mb * BP_W) - G.cmid;     // line-block origin (march coordinate)
  const int cross0 = cb * BP_SEG;                    // first cross line of the segment
  float *acc = acc_s + tid;
  const int nch = (NR + BP_SLOTS - 1) / BP_SLOTS;

  // The flat ray list is processed in chunks of BP_SLOTS entries, each thread
  // holding BP_SPT of them.  While chunk k is scattered from one buffer, the
  // raw data of chunk k+1 (ray parameters, low words, y) is already loaded
  // into registers; after the scatter it is converted to the tile's local
  // frame (r, t, g y, I - cross0 + 2) and stored into the other buffer, and one
  // barrier per chunk orders both buffers.  The view of a list entry is found
  // by galloping forward from the thread's previous entry (entries only move
  // forward), then bisecting the last step.
  constexpr int BP_SPT = BP_SLOTS / BP_THREADS;
  static_assert(BP_SLOTS % BP_THREADS == 0, "a chunk is a whole number of entries per thread");
  int vs = 0;
  float4 rw[BP_SPT];
  float2 rlo[BP_SPT];
  float ry[BP_SPT];
  auto fetch = [&](int k) {
#pragma unroll
    for (int u = 0; u < BP_SPT; ++u) {
      const int e = k * BP_SLOTS + tid + u * BP_THREADS;
      rw[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      rlo[u] = make_float2(0.0f, 0.0f);
      ry[u] = 0.0f;
      if (e >= NR) continue;
      int step = 1;
      while (vs + step < nv && pref[vs + step] <= e) {
        vs += step;
        step <<= 1;
      }
      int hi = min(vs + step, nv) - 1;   // pref[hi + 1] > e or hi = nv - 1
      while (vs < hi) {
        const int mid = (vs + hi + 1) >> 1;
        if (pref[mid] <= e)
          vs = mid;
        else
          hi = mid - 1;
      }
      const int kk = e - pref[vs];
      const int2 vi = vinfo[vs];
      // (a checked build records an index outside the ray list and applies a
      // zero-weight entry instead)
      if (!IMASK_INDEX_OK(vi.x + kk >= 0 && vi.x + kk < P.m && vi.y + kk >= 0 &&
                              vi.y + kk < P.m, 2))
        continue;
      rw[u] = __ldg(P.rays + vi.x + kk);
      rlo[u] = __ldg(P.rays_lo + vi.x + kk);
      ry[u] = __ldg(y + (y_list ? vi.x : vi.y) + kk);
    }
  };
  auto put = [&](int k, int b) {
    float4 *win = bp_win(bp_raw, b);
#pragma unroll
    for (int u = 0; u < BP_SPT; ++u) {
      const int sl = tid + u * BP_THREADS;
      if (k * BP_SLOTS + sl >= NR) continue;
      int I;
      float r;
      block_origin(rw[u].x, rlo[u].x, rw[u].y, rlo[u].y, G.inv2l, cco, I, r);
      win[sl] = make_float4(r, rw[u].y, rw[u].z * ry[u], __int_as_float(I - cross0 + 2));
    }
  };

  if (nch > 0) {
    fetch(0);
    put(0, 0);
  }
  __syncthreads();
  for (int k = 0; k < nch; ++k) {
    const int b = k & 1;
    if (k + 1 < nch) fetch(k + 1);
    const float4 *win = bp_win(bp_raw, b);
    const int n = min(BP_SLOTS, NR - k * BP_SLOTS);
    auto apply = [&](int sl) {
      const float4 e = win[sl];
      const float q = fmaf(dseg, e.y, e.x);
      const float tq = __fadd_rd(q, kMagic);
      // one unsigned clamp: rows off the segment on either side (negative
      // slots wrap to large unsigned values) land in the top guard slots,
      // which the epilogue never reads
      const int slot = (int)min((unsigned)(__float_as_int(tq) - kMagicBits + __float_as_int(e.w)),
                                (unsigned)(BP_ACC - 2));
      const float f = q - (tq - kMagic);
      const float w1 = f * e.z;
      // plain read-modify-writes: shared-memory atomic adds on the same
      // private slots measured about 35% slower
      float *pa = acc + slot * BP_THREADS;
      pa[0] += e.z - w1;
      pa[BP_THREADS] += w1;
    };
    // a full chunk runs a fixed trip count (no per-entry bound test); the
    // last, partial chunk tests the bound
    if (n == BP_SLOTS) {
      IMASK_UNROLL(BP_UNROLL)
      for (int it = 0; it < BP_SLOTS / BP_GROUPS; ++it) apply(g + it * BP_GROUPS);
    } else {
      IMASK_UNROLL(BP_UNROLL)
      for (int sl = g; sl < n; sl += BP_GROUPS) apply(sl);
    }
    // buffer b ^ 1 was last read by the scatter of chunk k - 1, which ended
    // before the previous barrier
    if (k + 1 < nch) put(k + 1, b ^ 1);
    __syncthreads();
  }
  // ---- epilogue: every pixel of the tile sums its owners' slots ----
  float *plane = gout + (size_t)(role * vgo + vg) * G.nl * G.nl;
  for (int p = tid; p < BP_W * BP_SEG; p += BP_THREADS) {
    const int ml = p % BP_W, cl = p / BP_W;          // march, cross offsets
    const int mline = mb * BP_W + ml, cline = cross0 + cl;
    if (mline >= G.nl || cline >= G.nl) continue;
    float sum = 0.0f;
#pragma unroll
    for (int gg = 0; gg < BP_GROUPS; ++gg) sum += acc_s[(cl + 2) * BP_THREADS + ml + BP_W * gg];
    const int i = role == 0 ? cline : mline, c = role == 0 ? mline : cline;
    plane[(size_t)i * G.nl + c] = sum * G.scale2l;
  }
}

__global__ void __launch_bounds__(BP_THREADS, 4)
    k_bp(DevPlan P, LevelSel sel, const float *__restrict__ y, int y_list,
         float *__restrict__ gout, unsigned int *err, int nv_cap) {
  bp_body(P, sel, y, y_list, gout, err, nv_cap, (int)blockIdx.x);
}

// ---------------------------------------------------------------------------------
// Pixel-driven back-projector for parallel beam (plans with bp_gather = 1):
// g = R_ell^T y computed pixel by pixel, each pixel's sum in a register.
//
// Joseph's weight of ray j at pixel (i, c) is Lambda(q_j(c) - i) (x-major
// rays; q_j(c) the ray's cross coordinate at line c, Lambda(u) = max(0,
// 1 - |u|)), and Lambda(q_j(i) - c) for y-major rays -- the same weights the
// projector applies.  In parallel beam the rays of a view share their slope
// and their intercepts a_j step by a constant D per bin, so with the local
// frame (I, r) of one reference ray j0 at the tile's first line (block_origin,
// as in the projector) q_{j0+e}(m0 + d) = I + r + d t + e D 2^-ell, and a
// pixel finds the few bins with weight (|q - i| < 1) from one division-free
// estimate instead of visiting rays.
//
// CTA = a GW_TY x GW_TX tile of level pixels (GW_PR x GW_PC per thread,
// sharing the view parameters) and one view group vg; it covers that group's x-major views (partial image role 0) and
// y-major views (role 1), so it writes the same 2 bp_vgo partial images as the
// owner-computes back-projector and the consumer adds them the same way.
// Views go in chunks of gw_vc; for each the bins crossing the tile (the ray
// window of the scatter, from the bin map at the tile's corners) are staged
// as g y in shared memory, at most gw_max per view (plan-time bound), with
// kGwPad zeros on either side so that a fixed trip of bins needs no test.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(GW_THREADS)
    k_bp_gather(DevPlan P, LevelSel sel, const float *__restrict__ y, int y_list,
                float *__restrict__ gout, unsigned int *err) {
  constexpr int kThreads = GW_THREADS;
  // a thread's pixels: GW_PR rows GW_TY / GW_PR apart times GW_PC columns
  // GW_TX / GW_PC apart
  constexpr int kRs = GW_TY / GW_PR, kCs = GW_TX / GW_PC, kPix = GW_PR * GW_PC;
  static_assert(kRs * kCs == GW_THREADS, "the pixels of a tile fill the CTA");
  constexpr int kMaxVc = 128;
  constexpr int kGwPad = 9;   // zeros staged on either side of a view's window
  __shared__ float yg[GW_SLOTS];
  __shared__ float4 vf[kMaxVc];   // per staged view: (r, t, D_ell, 1 / D_ell)
  __shared__ int4 vi[kMaxVc];     // per staged view: (I, bins staged, candidates, y index)
  __shared__ float vw[kMaxVc];    // per staged view: the rays' weight g
  __shared__ float vx[kMaxVc];    // per staged view: I as a float (exact)
  const int ell = sel_level_x(P, sel);
  const LevelGeom G = P.lg[ell + 1];
  const int ntx = (G.nl + GW_TX - 1) / GW_TX, nty = (G.nl + GW_TY - 1) / GW_TY;
  const int vgo = G.bp_vgo;
  const int tile = (int)blockIdx.x / vgo, vg = (int)blockIdx.x % vgo;
  if (tile >= ntx * nty) return;
  const int i0 = (tile / ntx) * GW_TY, c0 = (tile % ntx) * GW_TX;
  const int tid = threadIdx.x;
  const int di = tid / kCs, dc = tid % kCs;
  const int wmax = G.gw_max, wstr = wmax + 2 * kGwPad;   // window and its stride
  // views staged together: the plan's count, at most one per thread (each
  // thread sets up one view) and what the staging buffer holds
  const int vc = max(1, min(min(min(G.gw_vc, kMaxVc), kThreads), GW_SLOTS / wstr));
  const float hl = G.hl, W = P.fov;
  float acc[2][kPix];   // [role][pixel]
#pragma unroll
  for (int k = 0; k < kPix; ++k) acc[0][k] = acc[1][k] = 0.0f;
#pragma unroll
  for (int role = 0; role < 2; ++role) {
    const int *vb = P.bp_vb + ((ell + 1) * 2 + role) * (P.n_angles + 1);
    const int a0 = vb[vg];
    const int nv = vb[vg + 1] - a0;
    const int *vlist = P.bp_views + role * P.n_angles + a0;
    // march lines (columns for x-major rays) and cross lines of the tile
    const int m0 = role == 0 ? c0 : i0, x0 = role == 0 ? i0 : c0;
    const int m1 = min(m0 + (role == 0 ? GW_TX : GW_TY), G.nl) - 1;
    const int x1 = min(x0 + (role == 0 ? GW_TY : GW_TX), G.nl) - 1;
    const float mlo = -0.5f * W + ((float)m0 + 0.5f) * hl, mhi = -0.5f * W + ((float)m1 + 0.5f) * hl;
    const float clo = -0.5f * W + ((float)x0 + 0.5f) * hl - hl;
    const float chi = -0.5f * W + ((float)x1 + 0.5f) * hl + hl;
    const float cco = (float)m0 - G.cmid;
    // own march offsets and cross lines in the tile (x-major rays march along
    // a row, across the columns; y-major rays down a column)
    float dmk[kPix], xok[kPix];   // (the cross lines as floats, exact)
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
      const int ri = di + (k / GW_PC) * kRs, ci = dc + (k % GW_PC) * kCs;
      dmk[k] = (float)(role == 0 ? ci : ri);
      xok[k] = (float)(role == 0 ? i0 + ri : c0 + ci);
    }
    for (int v0 = 0; v0 < nv; v0 += vc) {
      const int nvc = min(vc, nv - v0);
      __syncthreads();   // the previous chunk's reads are done
      if (tid < nvc) {
        const int a = vlist[v0 + tid];
        int len = 0, I = 0, nc = 0, ybase = 0;
        float gw = 0.0f;
        float4 f = make_float4(0.0f, 0.0f, 1.0f, 1.0f);
        if (IMASK_INDEX_OK(a >= 0 && a < P.n_angles, 4)) {
          const ViewInfo V = P.views[a];
          float mn = 1.0e30f, mx = -1.0e30f;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float mcoord = (k & 1) ? mhi : mlo, ccoord = (k & 2) ? chi : clo;
            const float j = role == 0 ? bin_of(P, V.c, V.s, mcoord, ccoord)
                                      : bin_of(P, V.c, V.s, ccoord, mcoord);
            mn = fminf(mn, j);
            mx = fmaxf(mx, j);
          }
          const int j0 = role == 0 ? V.xj0 : V.yj0, j1 = role == 0 ? V.xj1 : V.yj1;
          const int lo = max(ceil_i(clampf(mn - kBpEps, -1.0e6f, 1.0e6f)), j0);
          const int hi = min(floor_i(clampf(mx + kBpEps, -1.0e6f, 1.0e6f)), j1 - 1);
          len = max(hi - lo + 1, 0);
          // (the plan's bound; a checked build records a window beyond it)
          if (!IMASK_INDEX_OK(len <= wmax, 4)) len = wmax;
          if (len > 0) {
            const int list0 = (role == 0 ? V.xoff - V.xj0 : V.yoff - V.yj0) + lo;
            const float4 pr = P.rays[list0];
            const float2 pl = P.rays_lo[list0];
            float r;
            block_origin(pr.x, pl.x, pr.y, pl.y, G.inv2l, cco, I, r);
            const float D = P.view_da[a] * G.inv2l;
            const float inv = 1.0f / D;
            // the bins e with |q - i| < 1 lie within 1 / |D| of the estimate
            nc = (int)floorf(2.0f * fabsf(inv)) + 1;
            // (the plan's per-level bound; a checked build records a view beyond it)
            if (!IMASK_INDEX_OK(nc <= G.gw_nc, 4)) nc = G.gw_nc;
            f = make_float4(r, pr.y, D, inv);
            ybase = y_list ? list0 : a * P.n_det + lo;
            gw = pr.z;
          }
        }
        vf[tid] = f;
        vi[tid] = make_int4(I, len, nc, ybase);
        vw[tid] = gw;
        vx[tid] = (float)I;
      }
      __syncthreads();
      // stage g y of every view's window (a parallel view's rays share g),
      // kGwPad zeros on either side of it
      for (int k = tid; k < nvc * wstr; k += kThreads) {
        const int v = k / wstr, e = k - v * wstr - kGwPad;
        const int4 q = vi[v];
        yg[k] = (e >= 0 && e < q.y) ? __ldg(y + q.w + e) * vw[v] : 0.0f;
      }
      __syncthreads();
      // The level's largest bin count per pixel-view (plan time, the same
      // float arithmetic as nc above) picks a fixed, branch-free trip of 3, 5
      // or 9 bins for the whole chunk, else a bounded loop.  The padding
      // holds zeros for bins just outside a window (empty windows included),
      // and a start clamped into the padding only skips bins of zero weight
      // or outside the window.
      auto views = [&](auto nc_const) {
        constexpr int NC = decltype(nc_const)::value;   // 0: the bounded loop
        float av[kPix];
#pragma unroll
        for (int k = 0; k < kPix; ++k) av[k] = acc[role][k];
#pragma unroll 2
        for (int v = 0; v < nvc; ++v) {
          const int4 q = vi[v];
          const float4 f = vf[v];
          const float fx = vx[v];
          const float *yv = yg + v * wstr + kGwPad;
          // cross offset of the reference ray from the pixel at its line, the
          // estimate of the bin that passes through the pixel, and its bins
          auto pixel = [&](float dm, float xo, float &a) {
            // (fx - xo is a difference of small integers: exact)
            const float ep = (fx - xo) + fmaf(dm, f.y, f.x);
            const int elo = ceil_i(fmaf(-ep, f.w, -fabsf(f.w)));
            if constexpr (NC > 0) {
              const int eb = min(max(elo, -kGwPad), q.y + kGwPad - NC);
              const float d0 = fmaf((float)eb, f.z, ep);
#pragma unroll
              for (int k = 0; k < NC; ++k) {
                // 1 - |d| never exceeds 1, so clamping to [0, 1] is max(., 0)
                const float w = __saturatef(1.0f - fabsf(fmaf((float)k, f.z, d0)));
                a = fmaf(w, yv[eb + k], a);
              }
            } else {
              for (int k = 0; k < q.z; ++k) {
                const int e = elo + k;
                if ((unsigned)e < (unsigned)q.y) {
                  const float w = 1.0f - fabsf(fmaf((float)e, f.z, ep));
                  if (w > 0.0f) a = fmaf(w, yv[e], a);
                }
              }
            }
          };
#pragma unroll
          for (int k = 0; k < kPix; ++k) pixel(dmk[k], xok[k], av[k]);
        }
#pragma unroll
        for (int k = 0; k < kPix; ++k) acc[role][k] = av[k];
      };
      if (G.gw_nc <= 3) {
        views(std::integral_constant<int, 3>{});
      } else if (G.gw_nc <= 5) {
        views(std::integral_constant<int, 5>{});
      } else if (G.gw_nc <= 9) {
        views(std::integral_constant<int, 9>{});
      } else {
        views(std::integral_constant<int, 0>{});
      }
    }
  }
  const size_t plane = (size_t)G.nl * G.nl;
#pragma unroll
  for (int k = 0; k < kPix; ++k) {
    const int i = i0 + di + (k / GW_PC) * kRs, c = c0 + dc + (k % GW_PC) * kCs;
    if (i < G.nl && c < G.nl) {
#pragma unroll
      for (int role = 0; role < 2; ++role)
        gout[(size_t)(role * vgo + vg) * plane + (size_t)i * G.nl + c] = acc[role][k] * G.scale2l;
    }
  }
}

// The back-projector leaves 2 bp_vgo partial images (x- and y-major rays, one
// per view group), each of side nl; their sum in a fixed order is R_ell^T y.
// Sums planes v0, v0 + dv, ... (fewer than v1) at element idx in that order;
// the loads go in batches of kPlaneBatch, all in flight before the adds.
constexpr int kPlaneBatch = 8;
__device__ __forceinline__ float planes_sum(const float *g, int v0, int v1, int dv, size_t plane,
                                            size_t idx, float s) {
  for (int v = v0; v < v1; v += kPlaneBatch * dv) {
    float t[kPlaneBatch];
#pragma unroll
    for (int u = 0; u < kPlaneBatch; ++u) {
      const int w = v + u * dv;
      t[u] = w < v1 ? __ldg(g + (size_t)w * plane + idx) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kPlaneBatch; ++u)
      if (v + u * dv < v1) s += t[u];
  }
  return s;
}

__device__ __forceinline__ float g_sum(const float *g, int vgo, size_t plane, size_t idx) {
  return planes_sum(g, 1, vgo, 1, plane, idx, __ldg(g + idx));
}

// log2 of a power of two (tile and block sides of the update-side kernels,
// which index with shifts and masks instead of divisions)
__device__ __forceinline__ int lg2i(int x) { return __ffs(x) - 1; }

// Sum of the back-projector's npl partial planes for the cs x cs coarse pixels
// starting at (I0, J0) of a level grid of side nl, into out[cs * cs]: K lanes
// per pixel add planes k, k+K, ..., then the lanes are added in a fixed order.
// Ends with a barrier.
__device__ void coarse_planes_sum(const float *g, int npl, int nl, int I0, int J0, int cs,
                                  float *out) {
  __shared__ float red[UPD_THREADS];
  const int ncp = cs * cs;
  const int K = max(1, min(UPD_THREADS / ncp, npl));   // K = 1 when ncp >= UPD_THREADS
  const size_t plane = (size_t)nl * nl;
  const int lcs = lg2i(cs), lnp = 2 * lcs;
  if (K > 1) {
    for (int u = threadIdx.x; u < ncp * K; u += blockDim.x) {
      const int p = u & (ncp - 1), k = u >> lnp;
      const size_t gi = (size_t)(I0 + (p >> lcs)) * nl + J0 + (p & (cs - 1));
      red[u] = planes_sum(g, k, npl, K, plane, gi, 0.0f);
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < ncp; p += blockDim.x) {
    float sum = 0.0f;
    if (K > 1) {
      for (int k = 0; k < K; ++k) sum += red[k * ncp + p];
    } else {
      const size_t gi = (size_t)(I0 + (p >> lcs)) * nl + J0 + (p & (cs - 1));
      sum = planes_sum(g, 0, npl, 1, plane, gi, 0.0f);
    }
    out[p] = sum;
  }
  __syncthreads();
}

// Block means of the tile `src` (side ts) at levels 1..r-1, level l at
// pyr + pyr_off(l), side ts >> l.  Hierarchical 2x2 means.
__device__ __forceinline__ void tile_pyramid(const float *src, float *pyr, int ts, int r) {
  const float *prev = src;
  int ps = ts, off = 0;
  for (int l = 1; l < r; ++l) {
    const int s = ps >> 1, ls = lg2i(s);
    float *cur = pyr + off;
    for (int p = threadIdx.x; p < s * s; p += blockDim.x) {
      const int I = p >> ls, J = p & (s - 1);
      const float *q = prev + (2 * I) * ps + 2 * J;
      cur[p] = 0.25f * ((q[0] + q[1]) + (q[ps] + q[ps + 1]));
    }
    __syncthreads();
    prev = cur;
    ps = s;
    off += s * s;
  }
}

__device__ __forceinline__ int pyr_off(int ts, int l) {
  int off = 0;
  for (int k = 1; k < l; ++k) off += (ts >> k) * (ts >> k);
  return off;
}

// S_r v at tile pixel (li, lj): (v - sum_{l>=1} p_l mean_l) / p_0 (levels = r).
__device__ __forceinline__ float compensate_px(const DevPlan &P, float v, const float *pyr, int ts,
                                               int li, int lj, int levels) {
  float s = v;
  int off = 0;
  for (int l = 1; l < levels; ++l) {
    const int side = ts >> l;
    s = fmaf(-P.probs[l], pyr[off + (li >> l) * side + (lj >> l)], s);
    off += side * side;
  }
  return s / P.probs[0];
}

// Writes the tile's contribution to the padded images of level `ell`
// (-1: plain grid).  `vals` holds the level values of the tile (side `side`).
// With a snapshot array S of the level (ell >= 0) the images receive
// vals - S, S takes vals, and vals is overwritten with the difference.
__device__ __forceinline__ void write_padded(const DevPlan &P, const PadSet &pads, int ell,
                                             float *vals,
                             int side, int ti0, int tj0, float *S) {
  const int li = ell + 1;
  const LevelGeom G = P.lg[li];
  const int sh = ell > 0 ? ell : 0;
  const int I0 = ti0 >> sh, J0 = tj0 >> sh;
  float *R = pads.R[li];
  float *T = pads.T[li];
  const int lsd = lg2i(side), msd = side - 1;
  if (S) {
    for (int p = threadIdx.x; p < side * side; p += blockDim.x) {
      const size_t gi = (size_t)(I0 + (p >> lsd)) * G.nl + J0 + (p & msd);
      const float v = vals[p];
      vals[p] = v - S[gi];
      S[gi] = v;
    }
    __syncthreads();
  }
  for (int p = threadIdx.x; p < side * side; p += blockDim.x) {
    const int I = p >> lsd, J = p & msd;
    if (!IMASK_INDEX_OK(I0 + I < G.nl && J0 + J < G.nl, 3)) continue;
    R[(size_t)(I0 + I) * G.ls + IMASK_PAD + J0 + J] = vals[I * side + J];
  }
  for (int p = threadIdx.x; p < side * side; p += blockDim.x) {
    const int J = p >> lsd, I = p & msd;
    T[(size_t)(J0 + J) * G.ls + IMASK_PAD + I0 + I] = vals[I * side + J];
  }
}

// Sketch of the tile held in xs (fine values) for level ell; uses aux and pyr.
// S: the level's snapshot array (snapshot tables) or nullptr; levels = r.
__device__ __forceinline__ void sketch_tile(const DevPlan &P, const PadSet &pads, int ell,
                                            float *xs, float *aux, float *pyr, int ts, int ti0,
                                            int tj0, float *S, int levels) {
  if (ell < 0) {
    write_padded(P, pads, -1, xs, ts, ti0, tj0, nullptr);
    return;
  }
  if (levels > 1) tile_pyramid(xs, pyr, ts, levels);
  if (ell == 0) {
    for (int p = threadIdx.x; p < ts * ts; p += blockDim.x)
      aux[p] = compensate_px(P, xs[p], pyr, ts, p >> lg2i(ts), p & (ts - 1), levels);
    __syncthreads();
    write_padded(P, pads, 0, aux, ts, ti0, tj0, S);
  } else {
    write_padded(P, pads, ell, pyr + pyr_off(ts, ell), ts >> ell, ti0, tj0, S);
  }
}

// Sketch of x (or of Alg. 7's xbar = x + theta (x - x_prev)) for the
// projector-side level of sel.
__global__ void __launch_bounds__(UPD_THREADS)
    k_sketch(DevPlan P, LevelSel sel, const float *__restrict__ x, PadSet pads, ExtrapArgs ex,
             SnapArgs sn) {
  extern __shared__ __align__(16) float upd_smem[];
  const int ts = P.upd_tile, ntx = P.n / ts, lts = lg2i(ts);
  float *xs = upd_smem, *aux = xs + ts * ts, *pyr = aux + ts * ts;
  const int ti0 = (blockIdx.x / ntx) * ts, tj0 = (blockIdx.x % ntx) * ts;
  const int ell = sel_level(P, sel);
  for (int p = threadIdx.x; p < ts * ts; p += blockDim.x) {
    const size_t gp = (size_t)(ti0 + (p >> lts)) * P.n + tj0 + (p & (ts - 1));
    const float v = x[gp];
    xs[p] = ex.x_prev ? fmaf(ex.theta, v - ex.x_prev[gp], v) : v;
  }
  __syncthreads();
  float *S = (sn.snap && ell >= 0) ? sn.snap + sn.snap_off[ell] : nullptr;
  sketch_tile(P, pads, ell, xs, aux, pyr, ts, ti0, tj0, S, P.levels);
}

// img = K_ell^T-side image map of g: ell >= 1: 4^-ell T^* g; ell = 0: S_r g;
// ell = -1: g.
__global__ void __launch_bounds__(UPD_THREADS)
    k_adjsketch(DevPlan P, int ell, const float *__restrict__ g, float *__restrict__ img) {
  extern __shared__ __align__(16) float upd_smem[];
  const int ts = P.upd_tile, ntx = P.n / ts, lts = lg2i(ts);
  float *xs = upd_smem, *pyr = xs + 2 * ts * ts;
  const int ti0 = (blockIdx.x / ntx) * ts, tj0 = (blockIdx.x % ntx) * ts;
  const int n = P.n;
  const LevelGeom G = P.lg[ell + 1];
  const size_t plane = (size_t)G.nl * G.nl;
  if (ell < 0) {
    for (int p = threadIdx.x; p < ts * ts; p += blockDim.x) {
      const size_t gp = (size_t)(ti0 + (p >> lts)) * n + tj0 + (p & (ts - 1));
      img[gp] = g_sum(g, 2 * G.bp_vgo, plane, gp);
    }
    return;
  }
  if (ell >= 1) {
    const float s = G.inv2l * G.inv2l;
    const int cs = ts >> ell;
    coarse_planes_sum(g, 2 * G.bp_vgo, G.nl, ti0 >> ell, tj0 >> ell, cs, xs);
    for (int p = threadIdx.x; p < ts * ts; p += blockDim.x) {
      const int li = p >> lts, lj = p & (ts - 1);
      img[(size_t)(ti0 + li) * n + tj0 + lj] = xs[(li >> ell) * cs + (lj >> ell)] * s;
    }
    return;
  }
  for (int p = threadIdx.x; p < ts * ts; p += blockDim.x)
    xs[p] = g_sum(g, 2 * G.bp_vgo, plane, (size_t)(ti0 + (p >> lts)) * n + tj0 + (p & (ts - 1)));
  __syncthreads();
  if (P.levels > 1) tile_pyramid(xs, pyr, ts, P.levels);
  for (int p = threadIdx.x; p < ts * ts; p += blockDim.x)
    img[(size_t)(ti0 + (p >> lts)) * n + tj0 + (p & (ts - 1))] =
        compensate_px(P, xs[p], pyr, ts, p >> lts, p & (ts - 1), P.levels);
}

// Primal half of Alg. 1 on one tile, then the sketch of the new iterate for
// the next level.  phi_new = 4^-ell T^*(g) (ell >= 1, block-constant, kept on
// the level grid) or S_r g (ell = 0); xi = phi_new - phi_ell + sum p phi;
// x+ = prox(x - (sigma/mu) xi); the running mean and the table take phi_new.
// ts (the plan's update tile) and levels (r) come in as arguments, so that a
// call with constants compiles the tile loops for that shape.
__device__ __forceinline__ void update_body(const DevPlan &P, const LevelSel &sel,
                                            const PrimalArgs &A, int write_sketch,
                                            const PadSet &pads, int bid, int ts, int levels) {
  extern __shared__ __align__(16) float upd_smem[];
  const int ntx = P.n / ts, lts = lg2i(ts);
  float *xs = upd_smem, *aux = xs + ts * ts, *pyr = aux + ts * ts;
  float *dc = pyr + ts * ts / 2 + 4;
  float *dm = dc + ts * ts / 4 + 4;
  const int ti0 = (bid / ntx) * ts, tj0 = (bid % ntx) * ts;
  const int n = P.n;
  const int ell = sel_level_x(P, sel);
  const float pl = P.probs[ell];
  const int fmt = A.phi_fmt;

  // A thread's pixels go in groups of kUpdPix: every load of a group is
  // issued before its first store (a store to one pixel could alias the next
  // pixel's loads and would otherwise keep them waiting one by one).  When
  // one group covers the tile (the usual case) its loads are issued first of
  // all, so that they are in flight together with the partial-plane sums.
  constexpr int kUpdPix = 4;
  const bool one_group = ts * ts <= kUpdPix * (int)blockDim.x;
  float pmv[kUpdPix], xov[kUpdPix], ph0[kUpdPix];
  auto load_group = [&](int p0) {
#pragma unroll
    for (int u = 0; u < kUpdPix; ++u) {
      const int p = p0 + u * (int)blockDim.x;
      pmv[u] = xov[u] = ph0[u] = 0.0f;
      if (p >= ts * ts) continue;
      const size_t gp = (size_t)(ti0 + (p >> lts)) * n + tj0 + (p & (ts - 1));
      pmv[u] = A.phi_mean[gp];
      xov[u] = A.x[gp];
      if (ell < 1) ph0[u] = tab_load(A.phi0, gp, fmt);
    }
  };
  if (one_group) load_group(threadIdx.x);

  int cs = 0;
  if (ell >= 1) {
    const LevelGeom G = P.lg[ell + 1];
    cs = ts >> ell;
    const int I0 = ti0 >> ell, J0 = tj0 >> ell;
    const long long off = A.phic_off[ell];
    const float inv4l = G.inv2l * G.inv2l;
    auto table_index = [&](int p) {
      return (size_t)off + (size_t)(I0 + (p >> (lts - ell))) * G.nl + J0 + (p & (cs - 1));
    };
    // the table entry of the thread's first coarse pixel is loaded before the
    // plane sums, so that the two loads are in flight together
    const int p_first = (int)threadIdx.x;
    const float old_first = p_first < cs * cs ? tab_load(A.phic, table_index(p_first), fmt) : 0.0f;
    coarse_planes_sum(A.g, 2 * G.bp_vgo, G.nl, I0, J0, cs, dc);
    // xi takes the refreshed value's change, the running mean the stored
    // (rounded, with 16-bit tables) value's change, so that the mean stays the
    // p-weighted sum of the stored tables
    for (int p = threadIdx.x; p < cs * cs; p += blockDim.x) {
      const size_t gi = table_index(p);
      const float cnew = dc[p] * inv4l;
      const float old = p == p_first ? old_first : tab_load(A.phic, gi, fmt);
      const float stored = tab_store(A.phic, gi, cnew, fmt);
      dc[p] = cnew - old;
      dm[p] = stored - old;
    }
    __syncthreads();
  } else {
    // the partial planes of kUpdPix pixels per thread, kPlaneBatch planes of
    // each in flight at once, added per pixel in plane order
    const int vgo0 = 2 * P.lg[1].bp_vgo;
    const size_t plane = (size_t)n * n;
    for (int p0 = threadIdx.x; p0 < ts * ts; p0 += kUpdPix * blockDim.x) {
      size_t gi[kUpdPix];
      float sum[kUpdPix];
#pragma unroll
      for (int u = 0; u < kUpdPix; ++u) {
        const int p = p0 + u * (int)blockDim.x;
        gi[u] = p < ts * ts ? (size_t)(ti0 + (p >> lts)) * n + tj0 + (p & (ts - 1)) : 0;
        sum[u] = p < ts * ts ? __ldg(A.g + gi[u]) : 0.0f;
      }
      for (int v = 1; v < vgo0; v += kPlaneBatch) {
        float t[kUpdPix][kPlaneBatch];
#pragma unroll
        for (int u = 0; u < kUpdPix; ++u)
#pragma unroll
          for (int w = 0; w < kPlaneBatch; ++w)
            t[u][w] = v + w < vgo0 ? __ldg(A.g + (size_t)(v + w) * plane + gi[u]) : 0.0f;
#pragma unroll
        for (int u = 0; u < kUpdPix; ++u)
#pragma unroll
          for (int w = 0; w < kPlaneBatch; ++w)
            if (v + w < vgo0) sum[u] += t[u][w];
      }
#pragma unroll
      for (int u = 0; u < kUpdPix; ++u) {
        const int p = p0 + u * (int)blockDim.x;
        if (p < ts * ts) aux[p] = sum[u];
      }
    }
    __syncthreads();
    if (levels > 1) tile_pyramid(aux, pyr, ts, levels);
  }

  for (int p0 = threadIdx.x; p0 < ts * ts; p0 += kUpdPix * blockDim.x) {
    if (!one_group) load_group(p0);
#pragma unroll
    for (int u = 0; u < kUpdPix; ++u) {
      const int p = p0 + u * (int)blockDim.x;
      if (p >= ts * ts) continue;
      const int li = p >> lts, lj = p & (ts - 1);
      const size_t gp = (size_t)(ti0 + li) * n + tj0 + lj;
      float delta, dmean;
      if (ell >= 1) {
        delta = dc[(li >> ell) * cs + (lj >> ell)];
        dmean = dm[(li >> ell) * cs + (lj >> ell)];
      } else {
        const float s0 = compensate_px(P, aux[p], pyr, ts, li, lj, levels);
        delta = s0 - ph0[u];
        dmean = tab_store(A.phi0, gp, s0, fmt) - ph0[u];
      }
      const float pm = pmv[u];
      const float xi = delta + pm;
      const float xo = xov[u];
      const float v = fmaf(-A.tau, xi, xo);
      A.phi_mean[gp] = fmaf(pl, dmean, pm);
      const float xn = A.prox_in_place ? v * A.inv_1ps : v;
      A.x[gp] = xn;
      if (A.x_prev) A.x_prev[gp] = xo;
      // the next projector input: x+ (Alg. 1) or x+ + theta (x+ - x) (Alg. 7)
      xs[p] = A.extrapolate ? fmaf(A.theta, xn - xo, xn) : xn;
    }
  }
  if (!write_sketch) return;
  __syncthreads();
  const int elln = draw_level(P, sel.seed, sel_k(sel) + 1);
  float *S = A.snap.snap ? A.snap.snap + A.snap.snap_off[elln] : nullptr;
  sketch_tile(P, pads, elln, xs, aux, pyr, ts, ti0, tj0, S, levels);
}

__global__ void __launch_bounds__(UPD_THREADS)
    k_update(DevPlan P, LevelSel sel, PrimalArgs A, int write_sketch, PadSet pads) {
  // the 32-pixel tile of a four-level plan compiled on its own, any other shape
  // with runtime loops
  if (P.upd_tile == 32 && P.levels == 4)
    update_body(P, sel, A, write_sketch, pads, (int)blockIdx.x, 32, 4);
  else
    update_body(P, sel, A, write_sketch, pads, (int)blockIdx.x, P.upd_tile, P.levels);
}

// ---------------------------------------------------------------------------------
// Fused batches: one launch of each kernel runs one iteration of every solve.
// The projector and update grids are the solves' own grids one after the other
// (their sizes do not depend on the drawn level).  The back-projector's work
// depends on each solve's level, so its CTAs stay resident and take items
// (one (role, tile, view group) each, heaviest first within a solve, the
// solves largest first) from a device counter until the iteration's items
// run out; no CTA ever waits for another.
// ---------------------------------------------------------------------------------
// Index s with start[s] <= b < start[s + 1] (start ascending, start[0] = 0).
__device__ __forceinline__ int slice_of(const int *start, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(FP_THREADS, 2)
    k_fp_multi(const FusedSlice *__restrict__ recs, const int *__restrict__ fp_start, int n) {
  const int b = (int)blockIdx.x;
  const int s = slice_of(fp_start, n, b);
  const FusedSlice &R = recs[s];
  fp_body(R.P, R.sel, R.pads_fp, nullptr, R.D, R.n_cta_x, R.err, 0, b - fp_start[s]);
}

__global__ void __launch_bounds__(UPD_THREADS, 3)
    k_update_multi(const FusedSlice *__restrict__ recs, const int *__restrict__ upd_start, int n) {
  const int b = (int)blockIdx.x;
  const int s = slice_of(upd_start, n, b);
  const FusedSlice &R = recs[s];
  update_body(R.P, R.sel, R.A, 1, R.pads_upd, b - upd_start[s], R.P.upd_tile, R.P.levels);
}

// Items of every solve's back-projection at its drawn level, as offsets into
// one list (start[n] = total), and the work counter reset for the launch that
// follows.  One CTA.
__global__ void __launch_bounds__(BP_THREADS)
    k_bp_plan(const FusedSlice *__restrict__ recs, int n, int *__restrict__ start, int *counter) {
  __shared__ int cnt[IMASK_MAX_FUSED + 1];
  for (int s = threadIdx.x; s < n; s += BP_THREADS) {
    const FusedSlice &R = recs[s];
    const int ell = sel_level_x(R.P, R.sel);
    const LevelGeom &G = R.P.lg[ell + 1];
    cnt[s] = 2 * G.bp_nm * G.bp_nc * G.bp_vgo;
  }
  __syncthreads();
  scan_counts(cnt, n);   // ends with a barrier
  for (int s = threadIdx.x; s <= n; s += BP_THREADS) start[s] = cnt[s];
  if (threadIdx.x == 0) *counter = 0;
}

// One item per CTA: the grid covers the most items the solves can have at
// any level, CTAs past the iteration's list return at once.  Unlike resident
// CTAs, these leave SMs to the projector's CTAs as they finish.
__global__ void __launch_bounds__(BP_THREADS, 4)
    k_bp_items(const FusedSlice *__restrict__ recs, int n, const int *__restrict__ start,
               int nv_cap) {
  const int it = (int)blockIdx.x;
  if (it >= start[n]) return;
  const int s = slice_of(start, n, it);
  const FusedSlice &R = recs[s];
  bp_body(R.P, R.sel, R.y_bp, 1, R.g, R.err, nv_cap, it - start[s]);
}

__global__ void __launch_bounds__(BP_THREADS, 4)
    k_bp_multi(const FusedSlice *__restrict__ recs, int n, const int *__restrict__ start,
               int *counter, int nv_cap) {
  __shared__ int item;
  const int total = start[n];
  // thread 0 asks for the next item while the current one runs, so that the
  // counter's round trip is hidden behind the work
  int next = 0;
  if (threadIdx.x == 0) next = atomicAdd(counter, 1);
  for (;;) {
    if (threadIdx.x == 0) {
      item = next;
      if (next < total) next = atomicAdd(counter, 1);
    }
    __syncthreads();
    const int it = item;
    if (it >= total) break;
    const int s = slice_of(start, n, it);
    const FusedSlice &R = recs[s];
    bp_body(R.P, R.sel, R.y_bp, 1, R.g, R.err, nv_cap, it - start[s]);
    // every thread is done with the item's shared memory (and with `item`)
    // before the next item is published
    __syncthreads();
  }
}

__global__ void k_counter_multi(const FusedSlice *__restrict__ recs, int n, long long delta) {
  for (int s = (int)(blockIdx.x * blockDim.x + threadIdx.x); s < n; s += gridDim.x * blockDim.x)
    *const_cast<long long *>(recs[s].sel.k_dev) += delta;
}

// ---------------------------------------------------------------------------------
// Smoothed-TV prox by FISTA (fixed step count), global-memory kernels.
// F(x) = 1/2|x - v|^2 + tau mu/2 |x|^2 + tau lam sum sqrt(|grad x|^2 + eps^2)
// ---------------------------------------------------------------------------------
__global__ void k_tv_dual(int n, const float *__restrict__ z, float eps, float *__restrict__ w1,
                          float *__restrict__ w2) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)n * n) return;
  const int i = (int)(p / n), j = (int)(p % n);
  const float zp = z[p];
  const float g1 = (i + 1 < n) ? z[p + n] - zp : 0.0f;
  const float g2 = (j + 1 < n) ? z[p + 1] - zp : 0.0f;
  const float inv = rsqrtf(fmaf(g1, g1, fmaf(g2, g2, eps * eps)));
  w1[p] = g1 * inv;
  w2[p] = g2 * inv;
}

__global__ void k_tv_step(int n, const float *__restrict__ v, float *__restrict__ xk,
                          float *__restrict__ z, const float *__restrict__ w1,
                          const float *__restrict__ w2, float tau_mu, float tau_lam, float inv_L,
                          float beta, float *__restrict__ out) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)n * n) return;
  const int i = (int)(p / n), j = (int)(p % n);
  // transpose of the forward differences applied to (w1, w2)
  float div = 0.0f;
  if (i + 1 < n) div -= w1[p];
  if (i >= 1) div += w1[p - n];
  if (j + 1 < n) div -= w2[p];
  if (j >= 1) div += w2[p - 1];
  const float zp = z[p];
  const float grad = (zp - v[p]) + tau_mu * zp + tau_lam * div;
  const float xn = zp - grad * inv_L;
  const float xo = xk[p];
  xk[p] = xn;
  z[p] = fmaf(beta, xn - xo, xn);
  if (out) out[p] = xn;
}

// ---------------------------------------------------------------------------------
// TV prox with nonnegativity: fast gradient projection on the dual (fixed step
// count).  argmin_{x >= 0} 1/2|x - v|^2 + alpha |grad x|_{1,2};
// x(r) = max(0, v - alpha grad^T r); p <- P_{|.|<=1}(r + grad x / (8 alpha));
// r <- p + beta (p - p_old).
// ---------------------------------------------------------------------------------
__global__ void k_fgp_primal(int n, const float *__restrict__ v, const float *__restrict__ r1,
                             const float *__restrict__ r2, float alpha, float *__restrict__ x) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)n * n) return;
  const int i = (int)(p / n), j = (int)(p % n);
  // transpose of the forward differences applied to (r1, r2)
  float dt = 0.0f;
  if (i + 1 < n) dt -= r1[p];
  if (i >= 1) dt += r1[p - n];
  if (j + 1 < n) dt -= r2[p];
  if (j >= 1) dt += r2[p - 1];
  x[p] = fmaxf(0.0f, fmaf(-alpha, dt, v[p]));
}

__global__ void k_fgp_dual(int n, const float *__restrict__ x, float inv8a, float beta,
                           float *__restrict__ p1, float *__restrict__ p2, float *__restrict__ r1,
                           float *__restrict__ r2) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)n * n) return;
  const int i = (int)(p / n), j = (int)(p % n);
  const float xp = x[p];
  const float g1 = (i + 1 < n) ? x[p + n] - xp : 0.0f;
  const float g2 = (j + 1 < n) ? x[p + 1] - xp : 0.0f;
  const float a = fmaf(g1, inv8a, r1[p]);
  const float b = fmaf(g2, inv8a, r2[p]);
  const float nrm = sqrtf(fmaf(a, a, b * b));
  const float sc = nrm > 1.0f ? 1.0f / nrm : 1.0f;
  const float n1 = a * sc, n2 = b * sc;
  const float o1 = p1[p], o2 = p2[p];
  p1[p] = n1;
  p2[p] = n2;
  r1[p] = fmaf(beta, n1 - o1, n1);
  r2[p] = fmaf(beta, n2 - o2, n2);
}

__global__ void k_relu(long long n, float *x) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] = fmaxf(0.0f, x[t]);
}

// ---------------------------------------------------------------------------------
// PDHG helpers: dual prox of f = 1/2|. - b|^2 and the primal extrapolation.
// ---------------------------------------------------------------------------------
__global__ void k_pdhg_dual(long long m, const float *__restrict__ kx, const float *__restrict__ b,
                            float s, float inv_1ps, float *__restrict__ y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = fmaf(s, kx[t] - b[t], y[t]) * inv_1ps;
}

// xn holds x - t Kbar^T y on entry for the quadratic prox (scaled here) or
// the prox result already; xbar = xn + theta (xn - x); x = xn.
__global__ void k_pdhg_primal(long long d, float scale, float theta, float *__restrict__ xn,
                              float *__restrict__ x, float *__restrict__ xbar) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < d;
       t += (long long)gridDim.x * blockDim.x) {
    const float v = xn[t] * scale;
    const float xo = x[t];
    xbar[t] = fmaf(theta, v - xo, v);
    x[t] = v;
  }
}

// ---------------------------------------------------------------------------------
// Elementwise helpers and FP64 reductions
// ---------------------------------------------------------------------------------
__global__ void k_levels(DevPlan P, unsigned long long seed, long long k0, long long n, int *out) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = draw_level(P, seed, k0 + t);
}

__device__ __forceinline__ float load_fmt(const void *p, long long i, int fmt) {
  if (fmt == 1) return __bfloat162float(((const __nv_bfloat16 *)p)[i]);
  if (fmt == 2) return __half2float(((const __half *)p)[i]);
  return ((const float *)p)[i];
}

__global__ void k_convert(long long n, const void *src, int sf, void *dst, int df) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const float v = load_fmt(src, t, sf);
    if (df == 1)
      ((__nv_bfloat16 *)dst)[t] = __float2bfloat16_rn(v);
    else if (df == 2)
      ((__half *)dst)[t] = __float2half_rn(v);
    else
      ((float *)dst)[t] = v;
  }
}

// Shared-memory ceilings for roofline reports: conflict-free 32-bit loads
// (every warp reads 32 consecutive words) and read-modify-writes of private
// slots (the back-projector's access pattern).  Eight independent chains per
// thread; volatile keeps every access.
constexpr int kProbeWords = 8192;
__global__ void __launch_bounds__(256) k_probe_smem(int iters, int rmw, float *sink) {
  __shared__ float buf[kProbeWords];
  for (int i = threadIdx.x; i < kProbeWords; i += blockDim.x) buf[i] = (float)i;
  __syncthreads();
  volatile float *vb = buf;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.0f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      // word (row, lane): rows cycle through the array, 32 consecutive words per warp
      const int row = (w * 8 + u + it * 3) & (kProbeWords / 32 - 1);
      const int a = row * 32 + lane;
      if (rmw)
        vb[a] = vb[a] + 1.0f;
      else
        acc[u] += vb[a];
    }
  }
  float t = 0.0f;
#pragma unroll
  for (int u = 0; u < 8; ++u) t += acc[u];
  if (t == -1.0f) sink[0] = t;   // never true; keeps the loads
}

// psi_mean[q] = sum_l p_l psi_l[q], levels in order
__global__ void k_table_mean(DevPlan P, const void *psi, int fmt, float *psi_mean) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < P.m;
       q += (long long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int l = 0; l < P.levels; ++l) s = fmaf(P.probs[l], load_fmt(psi, (long long)l * P.m + q, fmt), s);
    psi_mean[q] = s;
  }
}

// phi_mean[p] = sum_l p_l phi_l[p], levels in order, level ell >= 1 read at
// the block of p on its own grid
__global__ void k_phi_mean(DevPlan P, const void *phi0, const void *phic, PrimalArgs offs,
                           int fmt, float *phi_mean) {
  const long long d = (long long)P.n * P.n;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < d;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q / P.n), j = (int)(q % P.n);
    float s = P.probs[0] * tab_load(phi0, (size_t)q, fmt);
    for (int l = 1; l < P.levels; ++l) {
      const int nl = P.n >> l;
      const size_t gi = (size_t)offs.phic_off[l] + (size_t)(i >> l) * nl + (j >> l);
      s = fmaf(P.probs[l], tab_load(phic, gi, fmt), s);
    }
    phi_mean[q] = s;
  }
}

// Measurement-space vectors between (view, bin) order and ray-list order:
// entry i of the list is sinogram entry rays[i].w.
__global__ void k_sino_order(DevPlan P, const float *__restrict__ src, float *__restrict__ dst,
                             int to_list) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.m;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = __float_as_int(__ldg(&P.rays[i].w));
    if (to_list)
      dst[i] = src[q];
    else
      dst[q] = src[i];
  }
}

__global__ void k_counter(long long *k, long long delta, int set_value) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *k = set_value ? delta : *k + delta;
}

__global__ void k_axpy(long long n, float a, const float *__restrict__ x, float *__restrict__ y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = fmaf(a, x[t], y[t]);
}

__global__ void k_scale(long long n, float a, float *x) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] *= a;
}

__global__ void k_fill(long long n, float v, float *x) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    x[t] = v;
}

__global__ void k_copy(long long n, const float *__restrict__ x, float *__restrict__ y) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = x[t];
}

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kRedThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kRedThreads / 32; ++w) s += sh[w];
  __syncthreads();
  return s;
}

__global__ void __launch_bounds__(kRedThreads)
    k_dot64(long long n, const float *__restrict__ a, const float *__restrict__ b, double *part) {
  double s = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    s = fma((double)a[t], (double)b[t], s);
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads)
    k_diff64(long long n, const float *__restrict__ a, const float *__restrict__ b, double *part) {
  double s = 0.0, q = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const double d = (double)a[t] - (double)b[t];
    s = fma(d, d, s);
    q = fma((double)b[t], (double)b[t], q);
  }
  s = block_sum(s);
  q = block_sum(q);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s;
    part[2 * blockIdx.x + 1] = q;
  }
}

__global__ void __launch_bounds__(kRedThreads)
    k_tv64(int n, const float *__restrict__ x, double eps, double *part) {
  double s = 0.0;
  const long long d = (long long)n * n;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < d;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p / n), j = (int)(p % n);
    const double g1 = (i + 1 < n) ? (double)x[p + n] - (double)x[p] : 0.0;
    const double g2 = (j + 1 < n) ? (double)x[p + 1] - (double)x[p] : 0.0;
    s += sqrt(g1 * g1 + g2 * g2 + eps * eps);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Deterministic final sum of `nb` partials with stride `stride` (component `comp`).
__global__ void k_final64(const double *part, int nb, int stride, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int c = 0; c < stride; ++c) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b * stride + c];
    out[c] = s;
  }
}

inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 4096) b = 4096;
  if (b < 1) b = 1;
  return (int)b;
}

inline int upd_smem_bytes(const DevPlan &P) {
  const int ts = P.upd_tile;
  return (int)sizeof(float) * (ts * ts * 2 + ts * ts / 2 + 4 + 2 * (ts * ts / 4 + 4));
}

}  // namespace

// ===================================================================================
// launchers
// ===================================================================================
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_counter() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int reduce_blocks() { return kRedBlocks; }
long long fp_smem_bytes() { return (long long)FP_STAGES * FP_STAGE_FLOATS * (long long)sizeof(float); }

int lvl_host_draw(const DevPlan &P, unsigned long long seed, long long k) {
  return draw_level(P, seed, k);
}

// Seed of the primal stream when the levels are drawn independently: the
// SplitMix64 finaliser applied to the seed.
unsigned long long primal_seed(unsigned long long seed) {
  unsigned long long z = seed;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

cudaError_t launch_levels(const DevPlan &P, unsigned long long seed, long long k0, long long n,
                          int *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  k_levels<<<grid_for(n, 256), 256, 0, st>>>(P, seed, k0, n, out);
  return cudaGetLastError();
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes`.  The
// limit is process-wide and only ever raised, so that plans of different sizes
// launching from several threads never see it lowered under them.
static cudaError_t set_smem(const void *fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, int> limit;   // (device, kernel) -> bytes
  int dev = 0;
  const cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess) return ed;
  std::lock_guard<std::mutex> lk(mu);
  int &cur = limit[std::make_pair(dev, fn)];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

cudaError_t launch_sketch(const DevPlan &P, LevelSel sel, const float *x, PadSet pads,
                          ExtrapArgs ex, SnapArgs snap, cudaStream_t st) {
  const int nt = P.n / P.upd_tile;
  const int sm = upd_smem_bytes(P);
  cudaError_t e = set_smem((const void *)k_sketch, sm);
  if (e != cudaSuccess) return e;
  count_launch();
  k_sketch<<<nt * nt, UPD_THREADS, sm, st>>>(P, sel, x, pads, ex, snap);
  return cudaGetLastError();
}

cudaError_t launch_fp(const DevPlan &P, LevelSel sel, PadSet pads, float *sino, DualArgs dual,
                      int n_cta_x, int n_cta_y, unsigned int *err, cudaStream_t st,
                      int test_skip_first_strip) {
  const int sm = (int)fp_smem_bytes();
  cudaError_t e = set_smem((const void *)k_fp, sm);
  if (e != cudaSuccess) return e;
  if (n_cta_x + n_cta_y == 0) return cudaSuccess;
  count_launch();
  k_fp<<<n_cta_x + n_cta_y, FP_THREADS, sm, st>>>(P, sel, pads, sino, dual, n_cta_x, err,
                                                  test_skip_first_strip);
  return cudaGetLastError();
}

static int bp_nv_cap(const DevPlan &P) {
  int nv = 0;
  for (int li = 0; li <= P.levels; ++li) nv = max(nv, P.lg[li].bp_nv);
  return nv;
}

// Resident back-projector CTAs per SM for a given dynamic shared-memory size.
int bp_blocks_per_sm(long long dyn_smem) {
  if (set_smem((const void *)k_bp, (int)dyn_smem) != cudaSuccess) return 1;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bp, BP_THREADS, (size_t)dyn_smem) !=
          cudaSuccess ||
      n < 1)
    return 1;
  return n;
}

long long bp_smem_bytes(const DevPlan &P) {   // dynamic part only
  return 2LL * BP_SLOTS * 16 + (long long)bp_nv_cap(P) * 8 +
         (long long)(bp_nv_cap(P) + 1) * 4;
}

cudaError_t launch_bp(const DevPlan &P, LevelSel sel, const float *y, int y_list, float *g,
                      unsigned int *err, cudaStream_t st) {
  // the grid covers the level with the most (tile, view group) pairs; extra
  // CTAs return at once
  if (P.bp_gather) {
    // pixel-driven form: (tile, view group) CTAs of GW_TY x GW_TX pixels
    auto gctas = [&](int li) {
      const int nl = P.lg[li].nl;
      return ((nl + GW_TX - 1) / GW_TX) * ((nl + GW_TY - 1) / GW_TY) * P.lg[li].bp_vgo;
    };
    int most = 0;
    for (int li = 0; li <= P.levels; ++li) most = max(most, gctas(li));
    if (sel.fixed >= -1) most = gctas(sel.fixed + 1);
    count_launch();
    k_bp_gather<<<most, GW_THREADS, 0, st>>>(P, sel, y, y_list, g, err);
    return cudaGetLastError();
  }
  auto ctas = [&](int li) { return 2 * P.lg[li].bp_nm * P.lg[li].bp_nc * P.lg[li].bp_vgo; };
  int most = 0;
  for (int li = 0; li <= P.levels; ++li) most = max(most, ctas(li));
  if (sel.fixed >= -1) most = ctas(sel.fixed + 1);
  const int sm = (int)bp_smem_bytes(P);
  cudaError_t e = set_smem((const void *)k_bp, sm);
  if (e != cudaSuccess) return e;
  count_launch();
  k_bp<<<most, BP_THREADS, sm, st>>>(P, sel, y, y_list, g, err, bp_nv_cap(P));
  return cudaGetLastError();
}

cudaError_t launch_adjsketch(const DevPlan &P, int ell, const float *g, float *img,
                             cudaStream_t st) {
  const int nt = P.n / P.upd_tile;
  const int sm = upd_smem_bytes(P);
  cudaError_t e = set_smem((const void *)k_adjsketch, sm);
  if (e != cudaSuccess) return e;
  count_launch();
  k_adjsketch<<<nt * nt, UPD_THREADS, sm, st>>>(P, ell, g, img);
  return cudaGetLastError();
}

cudaError_t launch_update(const DevPlan &P, LevelSel sel, PrimalArgs pa, int write_sketch,
                          PadSet pads, cudaStream_t st) {
  const int nt = P.n / P.upd_tile;
  const int sm = upd_smem_bytes(P);
  cudaError_t e = set_smem((const void *)k_update, sm);
  if (e != cudaSuccess) return e;
  count_launch();
  k_update<<<nt * nt, UPD_THREADS, sm, st>>>(P, sel, pa, write_sketch, pads);
  return cudaGetLastError();
}

int upd_smem_bytes_of(const DevPlan &P) { return upd_smem_bytes(P); }

cudaError_t launch_fp_multi(const FusedSlice *recs, const int *fp_start, int n_slices,
                            int total_ctas, cudaStream_t st) {
  const int sm = (int)fp_smem_bytes();
  cudaError_t e = set_smem((const void *)k_fp_multi, sm);
  if (e != cudaSuccess) return e;
  if (total_ctas <= 0) return cudaSuccess;
  count_launch();
  k_fp_multi<<<total_ctas, FP_THREADS, sm, st>>>(recs, fp_start, n_slices);
  return cudaGetLastError();
}

int bp_multi_blocks_per_sm(long long dyn_smem) {
  if (set_smem((const void *)k_bp_multi, (int)dyn_smem) != cudaSuccess) return 1;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bp_multi, BP_THREADS,
                                                    (size_t)dyn_smem) != cudaSuccess ||
      n < 1)
    return 1;
  return n;
}

cudaError_t launch_bp_multi(const FusedSlice *recs, int n_slices, int *bp_start, int *bp_counter,
                            int nv_cap, long long smem, int grid, int max_items,
                            cudaStream_t st) {
  if (n_slices < 1 || n_slices > IMASK_MAX_FUSED) return cudaErrorInvalidValue;
  const void *fn = max_items > 0 ? (const void *)k_bp_items : (const void *)k_bp_multi;
  cudaError_t e = set_smem(fn, (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  k_bp_plan<<<1, BP_THREADS, 0, st>>>(recs, n_slices, bp_start, bp_counter);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  count_launch();
  if (max_items > 0)
    k_bp_items<<<max_items, BP_THREADS, smem, st>>>(recs, n_slices, bp_start, nv_cap);
  else
    k_bp_multi<<<grid, BP_THREADS, smem, st>>>(recs, n_slices, bp_start, bp_counter, nv_cap);
  return cudaGetLastError();
}

cudaError_t launch_update_multi(const FusedSlice *recs, const int *upd_start, int n_slices,
                                int total_ctas, int smem, cudaStream_t st) {
  cudaError_t e = set_smem((const void *)k_update_multi, smem);
  if (e != cudaSuccess) return e;
  if (total_ctas <= 0) return cudaSuccess;
  count_launch();
  k_update_multi<<<total_ctas, UPD_THREADS, smem, st>>>(recs, upd_start, n_slices);
  return cudaGetLastError();
}

cudaError_t launch_counter_multi(const FusedSlice *recs, int n_slices, long long delta,
                                 cudaStream_t st) {
  count_launch();
  k_counter_multi<<<(n_slices + 255) / 256, 256, 0, st>>>(recs, n_slices, delta);
  return cudaGetLastError();
}

// work: 4 * n*n floats (v, x_k, z, w1 | w2 uses the 5th block: caller passes 5 n*n).
cudaError_t launch_tv_prox(const DevPlan &P, float tau, float mu, float lam, float eps, int inner,
                           float *x, float *work, cudaStream_t st) {
  const long long d = (long long)P.n * P.n;
  float *v = work, *xk = work + d, *z = work + 2 * d, *w1 = work + 3 * d, *w2 = work + 4 * d;
  const int blocks = (int)((d + 255) / 256);
  count_launch();
  k_copy<<<grid_for(d, 256), 256, 0, st>>>(d, x, v);
  count_launch();
  k_copy<<<grid_for(d, 256), 256, 0, st>>>(d, x, xk);
  count_launch();
  k_copy<<<grid_for(d, 256), 256, 0, st>>>(d, x, z);
  const float L = 1.0f + tau * mu + 8.0f * tau * lam / eps;
  double t = 1.0;
  for (int it = 0; it < inner; ++it) {
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const float beta = (float)((t - 1.0) / tn);
    t = tn;
    count_launch();
    k_tv_dual<<<blocks, 256, 0, st>>>(P.n, z, eps, w1, w2);
    count_launch();
    k_tv_step<<<blocks, 256, 0, st>>>(P.n, v, xk, z, w1, w2, tau * mu, tau * lam, 1.0f / L, beta,
                                      it + 1 == inner ? x : nullptr);
  }
  if (inner <= 0) {
    count_launch();
    k_copy<<<grid_for(d, 256), 256, 0, st>>>(d, v, x);
  }
  return cudaGetLastError();
}

cudaError_t launch_tv_nonneg_prox(const DevPlan &P, float alpha, int inner, float *x, float *work,
                                  cudaStream_t st) {
  const long long d = (long long)P.n * P.n;
  if (!(alpha > 0.0f) || inner <= 0) {
    count_launch();
    k_relu<<<grid_for(d, 256), 256, 0, st>>>(d, x);
    return cudaGetLastError();
  }
  float *v = work, *p1 = work + d, *p2 = work + 2 * d, *r1 = work + 3 * d, *r2 = work + 4 * d;
  const int blocks = (int)((d + 255) / 256);
  count_launch();
  k_copy<<<grid_for(d, 256), 256, 0, st>>>(d, x, v);
  cudaError_t e = cudaMemsetAsync(p1, 0, 4 * d * sizeof(float), st);
  if (e != cudaSuccess) return e;
  const float inv8a = 1.0f / (8.0f * alpha);
  double t = 1.0;
  for (int it = 0; it < inner; ++it) {
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const float beta = (float)((t - 1.0) / tn);
    t = tn;
    count_launch();
    k_fgp_primal<<<blocks, 256, 0, st>>>(P.n, v, r1, r2, alpha, x);
    count_launch();
    k_fgp_dual<<<blocks, 256, 0, st>>>(P.n, x, inv8a, beta, p1, p2, r1, r2);
  }
  count_launch();
  k_fgp_primal<<<blocks, 256, 0, st>>>(P.n, v, p1, p2, alpha, x);
  return cudaGetLastError();
}

cudaError_t launch_pdhg_dual(long long m, const float *kx, const float *b, float s, float *y,
                             cudaStream_t st) {
  count_launch();
  k_pdhg_dual<<<grid_for(m, 256), 256, 0, st>>>(m, kx, b, s, 1.0f / (1.0f + s), y);
  return cudaGetLastError();
}

cudaError_t launch_pdhg_primal(long long d, float scale, float theta, float *xn, float *x,
                               float *xbar, cudaStream_t st) {
  count_launch();
  k_pdhg_primal<<<grid_for(d, 256), 256, 0, st>>>(d, scale, theta, xn, x, xbar);
  return cudaGetLastError();
}

cudaError_t read_index_check_flag(unsigned int *flags, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(flags, g_index_check_flag, sizeof(unsigned int));
  if (e == cudaSuccess && clear && *flags) {
    const unsigned int zero = 0u;
    e = cudaMemcpyToSymbol(g_index_check_flag, &zero, sizeof(unsigned int));
  }
  return e;
}

cudaError_t launch_counter(long long *k_dev, long long delta, int set_value, cudaStream_t st) {
  count_launch();
  k_counter<<<1, 32, 0, st>>>(k_dev, delta, set_value);
  return cudaGetLastError();
}

cudaError_t launch_convert(long long n, const void *src, int src_fmt, void *dst, int dst_fmt,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  k_convert<<<grid_for(n, 256), 256, 0, st>>>(n, src, src_fmt, dst, dst_fmt);
  return cudaGetLastError();
}

cudaError_t launch_probe_smem(int blocks, int iters, int rmw, float *sink, cudaStream_t st) {
  count_launch();
  k_probe_smem<<<blocks, 256, 0, st>>>(iters, rmw, sink);
  return cudaGetLastError();
}

cudaError_t launch_table_mean(const DevPlan &P, const void *psi, int fmt, float *psi_mean,
                              cudaStream_t st) {
  count_launch();
  k_table_mean<<<grid_for(P.m, 256), 256, 0, st>>>(P, psi, fmt, psi_mean);
  return cudaGetLastError();
}

cudaError_t launch_phi_mean(const DevPlan &P, const void *phi0, const void *phic,
                            const long long *phic_off, int fmt, float *phi_mean,
                            cudaStream_t st) {
  PrimalArgs offs{};
  for (int l = 0; l < IMASK_MAX_LEVELS; ++l) offs.phic_off[l] = phic_off[l];
  count_launch();
  k_phi_mean<<<grid_for((long long)P.n * P.n, 256), 256, 0, st>>>(P, phi0, phic, offs, fmt,
                                                                 phi_mean);
  return cudaGetLastError();
}

cudaError_t launch_sino_order(const DevPlan &P, const float *src, float *dst, int to_list,
                              cudaStream_t st) {
  count_launch();
  k_sino_order<<<grid_for(P.m, 256), 256, 0, st>>>(P, src, dst, to_list);
  return cudaGetLastError();
}

cudaError_t launch_axpy(long long n, float alpha, const float *x, float *y, cudaStream_t st) {
  count_launch();
  k_axpy<<<grid_for(n, 256), 256, 0, st>>>(n, alpha, x, y);
  return cudaGetLastError();
}
cudaError_t launch_scale(long long n, float alpha, float *x, cudaStream_t st) {
  count_launch();
  k_scale<<<grid_for(n, 256), 256, 0, st>>>(n, alpha, x);
  return cudaGetLastError();
}
cudaError_t launch_fill(long long n, float v, float *x, cudaStream_t st) {
  count_launch();
  k_fill<<<grid_for(n, 256), 256, 0, st>>>(n, v, x);
  return cudaGetLastError();
}
cudaError_t launch_copy(long long n, const float *x, float *y, cudaStream_t st) {
  count_launch();
  k_copy<<<grid_for(n, 256), 256, 0, st>>>(n, x, y);
  return cudaGetLastError();
}

cudaError_t launch_dot64(long long n, const float *a, const float *b, double *partial, double *out,
                         cudaStream_t st) {
  count_launch();
  k_dot64<<<kRedBlocks, kRedThreads, 0, st>>>(n, a, b, partial);
  count_launch();
  k_final64<<<1, 32, 0, st>>>(partial, kRedBlocks, 1, out);
  return cudaGetLastError();
}

cudaError_t launch_diff64(long long n, const float *a, const float *b, double *partial,
                          double *out, cudaStream_t st) {
  count_launch();
  k_diff64<<<kRedBlocks, kRedThreads, 0, st>>>(n, a, b, partial);
  count_launch();
  k_final64<<<1, 32, 0, st>>>(partial, kRedBlocks, 2, out);
  return cudaGetLastError();
}

cudaError_t launch_tv_value64(const DevPlan &P, const float *x, float eps, double *partial,
                              double *out, cudaStream_t st) {
  count_launch();
  k_tv64<<<kRedBlocks, kRedThreads, 0, st>>>(P.n, x, (double)eps, partial);
  count_launch();
  k_final64<<<1, 32, 0, st>>>(partial, kRedBlocks, 1, out);
  return cudaGetLastError();
}
