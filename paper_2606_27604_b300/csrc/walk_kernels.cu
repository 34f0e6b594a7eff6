// walk_kernels.cu -- device kernels of the mixture-of-media random walk.
//
//   validate_params   : one thread per instance; flags out-of-range media.
//   units_count/scan  : per-instance work-unit counts -> exclusive prefix
//                       (uneven path budgets only).
//   walk_persistent<ADJ> : persistent batched walk.  Each warp takes work
//                       units (instance, range of paths) from a global
//                       counter; its lanes each run one path and, as soon as
//                       enough lanes are idle, are refilled from the warp's
//                       current unit (path regrouping).  A warp holds two
//                       units at once (double-buffered slots) so the tail of
//                       one unit overlaps the start of the next.  Tallies are
//                       64-bit fixed point (weight * 2^32), summed with
//                       shared-memory atomics per slot and flushed with one
//                       global atomic per nonzero entry when a unit is done:
//                       integer sums do not depend on order, so a rerun is
//                       bit-identical whatever the launch shape.
//                       ADJ = true is the path-replay adjoint: it re-runs
//                       the same paths and accumulates score-weighted
//                       upstream derivatives instead of tallies.
//   walk_plain        : baseline: one thread per path of one instance.
//   finalize_*        : fixed point -> float64 means / standard errors.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "walk_core.cuh"
#include "walk_kernels.cuh"

#include "hero.cuh"

namespace sss {

static constexpr unsigned kFull = 0xffffffffu;

// -------------------------------------------------------------- validate --
__global__ void validate_params_kernel(WalkConst c, unsigned int* status) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.n_inst) return;
  bool bad = false;
  float wsum = 0.0f;
  for (int k = 0; k < c.K; ++k) {
    const size_t o = (size_t)k * c.n_inst + i;
    const float a = c.alpha[o], s = c.sigma_t[o], g = c.g[o], w = c.w[o];
    bad |= !(a >= 0.0f && a <= 1.0f);
    bad |= !(s > 0.0f && s < __int_as_float(0x7f800000));
    bad |= !(g > -1.0f && g < 1.0f);
    bad |= !(w >= 0.0f && w <= 1.0f + 1e-5f);
    wsum += w;
  }
  bad |= !(fabsf(wsum - 1.0f) <= 1e-5f);
  const float d = c.thickness ? c.thickness[i] : __int_as_float(0x7f800000);
  if (c.thickness) bad |= !(d > 0.0f);  // +inf allowed, NaN and <= 0 rejected
  if (c.alpha2) {
    const float a = c.alpha2[i], s = c.sigma_t2[i], g = c.g2[i], d1 = c.d1[i];
    bad |= !(a >= 0.0f && a <= 1.0f);
    bad |= !(s > 0.0f && s < __int_as_float(0x7f800000));
    bad |= !(g > -1.0f && g < 1.0f);
    bad |= !(d1 > 0.0f && d1 <= d);
  }
  if (bad) atomicOr(status, SSS_DEV_FLAG_PARAM);
}

// -------------------------------------------------------- unit prefix sum --
// counts[i] = ceil(N_i / C); prefix[i] = sum_{j<i} counts[j]; prefix[n] = total.
// Three passes: per-block sums, one-block scan of the block sums, fix-up.
__global__ void unit_block_sums_kernel(const uint32_t* n_paths, uint32_t n, uint32_t C,
                                       unsigned long long* block_sums) {
  __shared__ unsigned long long red[32];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = i < n ? (unsigned long long)((n_paths[i] + (uint64_t)C - 1) / C) : 0ull;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = v;
  }
}

__global__ void unit_scan_block_sums_kernel(unsigned long long* block_sums, uint32_t nblocks,
                                            unsigned long long* total) {
  // single block of 1024 threads; sequential over chunks of 1024
  __shared__ unsigned long long buf[1024];
  unsigned long long carry = 0;
  for (uint32_t base = 0; base < nblocks; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    buf[threadIdx.x] = i < nblocks ? block_sums[i] : 0ull;
    __syncthreads();
    // Hillis-Steele inclusive scan
    for (int o = 1; o < 1024; o <<= 1) {
      unsigned long long t = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0ull;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    const unsigned long long incl = buf[threadIdx.x];
    const unsigned long long excl = incl - (i < nblocks ? block_sums[i] : 0ull);
    __syncthreads();
    if (i < nblocks) block_sums[i] = carry + excl;
    carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void unit_prefix_kernel(const uint32_t* n_paths, uint32_t n, uint32_t C,
                                   const unsigned long long* block_offsets,
                                   const unsigned long long* total,
                                   unsigned long long* prefix) {
  __shared__ unsigned long long warp_tot[32];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned long long v =
      i < n ? (unsigned long long)((n_paths[i] + (uint64_t)C - 1) / C) : 0ull;
  unsigned long long incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    unsigned long long t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
    unsigned long long ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(kFull, ti, o);
      if (lane >= o) ti += u;
    }
    warp_tot[lane] = ti - t;  // exclusive
  }
  __syncthreads();
  if (i < n) prefix[i] = block_offsets[blockIdx.x] + warp_tot[wid] + incl - v;
  if (i == 0) prefix[n] = *total;
}

// ------------------------------------------------------------- persistent --
struct UnitRange {
  uint32_t inst, p0, p1;
  bool ok;
};

__device__ __forceinline__ UnitRange unit_lookup(const WalkSched& s, const WalkConst& c,
                                                 unsigned long long u) {
  UnitRange r;
  r.ok = s.prefix == nullptr ? u < s.total_units : u < s.prefix[c.n_inst];
  if (!r.ok) return r;
  uint32_t inst;
  unsigned long long first;
  if (s.prefix == nullptr) {
    inst = (uint32_t)(u / s.units_per_inst);
    first = (unsigned long long)inst * s.units_per_inst;
  } else {
    // largest i with prefix[i] <= u (instances with no units are skipped)
    uint32_t lo = 0, hi = c.n_inst;  // prefix[lo] <= u < prefix[hi]
    while (hi - lo > 1) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      if (s.prefix[mid] <= u) lo = mid;
      else hi = mid;
    }
    inst = lo;
    first = s.prefix[lo];
  }
  const uint32_t N = c.n_paths ? c.n_paths[inst] : c.uniform_paths;
  const unsigned long long chunk = u - first;
  r.inst = inst;
  r.p0 = (uint32_t)(chunk * s.unit_paths);
  const unsigned long long e = (chunk + 1) * s.unit_paths;
  r.p1 = e < N ? (uint32_t)e : N;
  return r;
}

// Upstream-derivative scale of one instance for the adjoint: a power of two
// 2^E chosen so that |weight * upstream * score| < 2^20 * max|upstream| per
// path cannot overflow an int64 sum over N paths.
__device__ __forceinline__ int grad_exponent(const WalkConst& c, const GradIn& gi, uint32_t inst,
                                             int lane) {
  double vmax = 0.0;
  if (gi.grad_bins) {
    for (int b = lane; b < c.nbins; b += 32)
      vmax = fmax(vmax, fabs(gi.grad_bins[(size_t)inst * c.nbins + b]));
  }
  for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(kFull, vmax, o));
  double vk = 0.0;
  if (gi.grad_R_k)
    for (int k = 0; k < c.K; ++k) vk = fmax(vk, fabs(gi.grad_R_k[(size_t)inst * c.K + k]));
  double top = vmax + vk + (gi.grad_R ? fabs(gi.grad_R[inst]) : 0.0);
  double bot = gi.grad_T ? fabs(gi.grad_T[inst]) : 0.0;
  const double v = fmax(top, bot);
  if (!(v > 0.0)) return 0;
  const uint32_t N = c.n_paths ? c.n_paths[inst] : c.uniform_paths;
  const int lgN = N > 1 ? 32 - __clz(N - 1) : 0;
  int ev;
  frexp(v, &ev);  // v < 2^ev
  int E = 62 - 20 - lgN - ev;
  E = max(-100, min(100, E));
  return E;
}

// Warp-uniform state of one work unit held by a warp (kept in shared memory).
// `gl` holds the slot's generation (the number of its flushes) times two
// plus a live bit: a lane whose path outlives its unit (the slot was
// flushed, and perhaps refilled, meanwhile) sees another generation.  The
// first 16 bytes (inst, next, end, gl) are what the refill loop reads, in
// one vector load.
// A unit is one instance, so its media are staged here once, when the unit
// is taken: per medium (alpha, ln2 / sigma_t, g, sigma_t), the selection
// thresholds and weights, and a second layer's optics.  Paths then start
// from shared memory instead of re-reading and re-dividing per path.
struct SlotMeta {
  uint32_t inst, next, end, gl;
  float d, scale, lim, wsum;
  uint32_t spare0, spare1, spare2, spare3;
  float4 med[kKMax];     // alpha, ln2 / sigma_t, g, sigma_t per medium
  float cdf[kKMax];      // running sum of w_k / sum(w): first K - 1 used
  float wsel[kKMax];     // K w_k / sum(w) (uniform selection)
  float4 l2;             // second layer: alpha, ln2 / sigma_t, g, sigma_t
  float d1, pad3, pad4, pad5;
  float2 hgc[kKMax];     // hg_consts(g) per medium
};
static_assert(sizeof(SlotMeta) == kSlotMetaBytes, "slot header size");

// Per-warp buffer of medium choices: k[j] is the medium of path base + j of
// the warp's current unit (the buffer is invalidated whenever the warp takes
// a unit).  The 32 tag-1 Philox blocks are drawn by the whole warp at once,
// so the draw runs with every lane active instead of inside the refill's
// divergent block.
struct SelBuf {
  uint32_t base, valid, pad0, pad1;
  uint8_t k[32];
  uint32_t inst[32];  // instance of each lane's path (read only by a direct tally; the
                      // forward kernel keeps it here instead of in a register)
};
static_assert(sizeof(SelBuf) == kSelBufBytes, "selection buffer size");

// Loads the media of instance `inst` into slot header m: lane k < K reads
// medium k (one load per array per lane), lane 0 forms the selection
// thresholds in the order select_medium forms them, so a staged start is a
// global-memory start bit for bit.
template <bool LAYERED>
__device__ __forceinline__ void stage_media(const WalkConst& c, uint32_t inst, int lane,
                                            SlotMeta& m) {
  float w = 0.0f;
  if (lane < c.K) {
    const size_t off = (size_t)lane * c.n_inst + inst;
    const float a = __ldg(c.alpha + off), st = __ldg(c.sigma_t + off), g = __ldg(c.g + off);
    w = __ldg(c.w + off);
    m.med[lane] = make_float4(a, flight_scale(st), g, st);
    m.hgc[lane] = hg_consts(g);
  }
  float wk[kKMax];
#pragma unroll
  for (int k = 0; k < kKMax; ++k) wk[k] = __shfl_sync(kFull, w, k);
  if (lane == 0) {
    float total = 0.0f;
#pragma unroll
    for (int k = 0; k < kKMax; ++k)
      if (k < c.K) total = __fadd_rn(total, wk[k]);
    const float inv = __fdiv_rn(1.0f, total);
    float cdf = 0.0f;
#pragma unroll
    for (int k = 0; k < kKMax; ++k) {
      if (k < c.K) {
        cdf = __fadd_rn(cdf, __fmul_rn(wk[k], inv));
        m.cdf[k] = cdf;
        m.wsel[k] = __fmul_rn(__fmul_rn((float)c.K, wk[k]), inv);
      }
    }
    if (LAYERED) {
      const float st2 = __ldg(c.sigma_t2 + inst);
      m.l2 = make_float4(__ldg(c.alpha2 + inst), flight_scale(st2), __ldg(c.g2 + inst), st2);
      m.d1 = __ldg(c.d1 + inst);
    }
  }
}

// Medium of a path from its tag-1 uniform u: the first k whose threshold
// exceeds u (the last medium takes the remainder), or uniformly k = floor(u K).
__device__ __forceinline__ int staged_choice(const WalkConst& c, const SlotMeta& m, float u) {
  if (c.select_uniform) return min(c.K - 1, (int)__fmul_rn(u, (float)c.K));
  int k = c.K - 1;
#pragma unroll
  for (int j = kKMax - 2; j >= 0; --j)
    if (j < c.K - 1 && u < m.cdf[j]) k = j;
  return k;
}

// Starts path `path` with medium k of the unit (instance inst) staged in m:
// the arithmetic of path_init with the media read from shared memory.
template <bool LAYERED>
__device__ __forceinline__ void path_start(const WalkConst& c, const SlotMeta& m, uint32_t inst,
                                           int k, uint32_t path, Path& p) {
  const float4 md = m.med[k];
  p.k = k;
  p.alpha = md.x;
  p.fl = md.y;
  p.g = md.z;
  p.sigt = md.w;
  const float2 hc = m.hgc[k];
  p.hc1 = hc.x;
  p.hc2 = hc.y;
  p.ga = hg_dlogp_dg_const(p.g);
  p.d = m.d;
  p.x = 0.0f; p.y = 0.0f; p.z = 0.0f;
  p.ux = 0.0f; p.uy = 0.0f; p.uz = 1.0f;
  const float w_sel = c.select_uniform ? m.wsel[k] : 1.0f;
  p.W = __fmul_rn(c.W0, w_sel);
  if (c.incidence == 1) entry_lobe(c, path, inst + c.inst_offset, w_sel, p);
  p.Aacc = 0.0f;
  p.step = 0u;
  p.inst = inst;
  p.pc = philox_path(path, inst + c.inst_offset, c.rk);
  p.n_coll = 0u;
  p.L = 0.0f;
  p.G = 0.0f;
  if (LAYERED) {
    p.layer = 0;
    p.n2 = 0u;
    p.L2 = 0.0f;
    p.G2 = 0.0f;
    p.d1 = m.d1;
    p.a_o = m.l2.x;
    p.fl_o = m.l2.y;
    p.g_o = m.l2.z;
    p.sigt_o = m.l2.w;
  }
}

// Lane state: idle, running, or done with exit event e (state 1 + e, e >= 1),
// kept in one register.
enum : int { LANE_IDLE = 0, LANE_RUNNING = 1 };
__device__ __forceinline__ bool lane_done(int st) { return st > LANE_RUNNING; }

// Adds one finished path to its slot's shared accumulators, or, when the
// slot has moved on to another unit (`direct`), straight to the instance's
// global accumulators in the layout the slot flush uses.
template <bool ADJ, bool LAYERED>
__device__ __forceinline__ void tally_path(const WalkConst& c, const WalkSched& s,
                                           const GradIn& gi, const TallyOut& t, const Path& p,
                                           int ev, unsigned long long* m, bool direct) {
  auto add = [&](int j, unsigned long long v) {
    if (!direct) add64_shared(m + j, v);  // (two's complement: signed words too)
    else if (ADJ) atomicAdd(t.raw + (size_t)j * c.n_inst + p.inst, v);
    else atomicAdd(t.raw + (size_t)p.inst * s.slot_words + j, v);
  };
  if (!ADJ) {
    const int nb = c.nbins;
    if (ev == EV_TOP) {
      const int bin = exit_bin(c, p);
      const unsigned long long q = __float2ull_rn(__fmul_rn(p.W, kFix));
      add(bin, q);
      add(nb + 1 + p.k, q);
      if (p.n_coll == 1u) add(nb + 1 + c.K, q);
      if (s.want_sumsq)
        add(nb + 6 + c.K + bin, __float2ull_rn(__fmul_rn(__fmul_rn(p.W, p.W), kFix)));
    } else if (ev == EV_BOTTOM) {
      add(nb + 2 + c.K, __float2ull_rn(__fmul_rn(p.W, kFix)));
    } else if (ev == EV_TRUNC) {
      add(nb + 4 + c.K, 1ull);
    }
    if (p.Aacc > 0.0f) add(nb + 3 + c.K, __float2ull_rn(__fmul_rn(p.Aacc, kFix)));
    add(nb + 5 + c.K, (unsigned long long)p.step);
  } else {
    float v = 0.0f;
    if (ev == EV_TOP) {
      const int bin = exit_bin(c, p);
      double vd = 0.0;
      if (gi.grad_R) vd += gi.grad_R[p.inst];
      if (gi.grad_bins && bin < c.nbins) vd += gi.grad_bins[(size_t)p.inst * c.nbins + bin];
      if (gi.grad_R_k) vd += gi.grad_R_k[(size_t)p.inst * c.K + p.k];
      v = (float)vd;
    } else if (ev == EV_BOTTOM) {
      if (gi.grad_T) v = (float)gi.grad_T[p.inst];
    }
    if (v != 0.0f && p.W != 0.0f) {  // (W = 0: a zero-weight medium, chosen uniformly)
      const float Wv = __fmul_rn(__fmul_rn(p.W, v), p.gscale);
      // the top layer's optics (a path that ends in the second layer holds
      // them as the "other" layer's)
      const bool low = LAYERED && p.layer;
      const float a1 = low ? p.a_o : p.alpha, s1 = low ? p.sigt_o : p.sigt;
      const float nf = LAYERED ? (float)(p.n_coll - p.n2) : (float)p.n_coll;
      constexpr int NQ = LAYERED ? 7 : 4;
      float q[NQ];
      q[0] = __fmul_rn(Wv, __fdiv_rn(nf, a1));
      q[1] = __fmul_rn(Wv, __fsub_rn(__fdiv_rn(nf, s1), p.L));
      q[2] = __fmul_rn(Wv, p.G);
      q[3] = __fmul_rn(Wv, __fdiv_rn(p.wsum, __ldg(c.w + (size_t)p.k * c.n_inst + p.inst)));
      if constexpr (LAYERED) {
        const float a2 = low ? p.alpha : p.a_o, s2 = low ? p.sigt : p.sigt_o;
        const float n2 = (float)p.n2;
        q[4] = __fmul_rn(Wv, __fdiv_rn(n2, a2));
        q[5] = __fmul_rn(Wv, __fsub_rn(__fdiv_rn(n2, s2), p.L2));
        q[6] = __fmul_rn(Wv, p.G2);
      }
#pragma unroll
      for (int j = 0; j < NQ; ++j) {
        float x = q[j];
        if (!(fabsf(x) < p.glim)) {
          atomicOr(s.status, SSS_DEV_FLAG_OVERFLOW);
          x = (x != x) ? 0.0f : copysignf(p.glim, x);
        }
        // words [4][K] per medium, then 3 for the second layer
        add(j < 4 ? j * c.K + p.k : 4 * c.K + (j - 4), (unsigned long long)__float2ll_rn(x));
      }
    }
  }
  if (ev == EV_TRUNC) atomicOr(s.status, SSS_DEV_FLAG_STEP_LIMIT);
}

// Exact sum of v < 2^59 over the lanes of `mask` (every lane of the mask
// calls it): two 32-bit warp reductions of 27-bit pieces, which cannot wrap.
__device__ __forceinline__ unsigned long long warp_sum64(unsigned mask, unsigned long long v) {
  const uint32_t lo = __reduce_add_sync(mask, (uint32_t)(v & 0x7FFFFFFull));
  const uint32_t hi = __reduce_add_sync(mask, (uint32_t)(v >> 27));
  return (unsigned long long)lo + ((unsigned long long)hi << 27);
}

// Forward exit tally of the finishing lanes of a warp (one-layer or
// two-layer, no hero sharing).  Called by exactly the lanes of `done`.
//  * Words every finishing lane adds to (absorbed weight A and the step
//    count) are summed across the finishing lanes of each slot with warp
//    reductions first; one lane then adds the sum to the slot's word.
//  * Per-path words (radial bin, R_k, R1, T, squared weights) go to the
//    slot with native 32-bit shared atomics (add64_shared).
//  * A lane whose unit has been flushed meanwhile (`direct`) adds all its
//    words straight to the instance's global accumulators.
// Every word is an integer sum, so the result does not depend on how the
// additions are grouped.  (Fixed point uses the hardware conversion: a
// 64-bit integer construction from the binary32 encoding took more issue
// slots than the conversion's slow pipe cost, measured on the spectral field.)
__device__ __forceinline__ void tally_exit_warp(const WalkConst& c, const WalkSched& s,
                                                const TallyOut& t, const Path& p, int ev,
                                                unsigned long long* slot_mem, int myslot,
                                                bool direct, unsigned done, int lane,
                                                const uint32_t* lane_inst) {
  const int nb = c.nbins, K = c.K, sw = s.slot_words;
  const unsigned long long qa = p.Aacc > 0.0f ? __float2ull_rn(__fmul_rn(p.Aacc, kFix)) : 0ull;
  const unsigned long long qs = (unsigned long long)p.step;
  const int leader = __ffs(done) - 1;
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    const bool in = !direct && myslot == o;
    if (__ballot_sync(done, in) != 0u) {
      const unsigned long long sa = warp_sum64(done, in ? qa : 0ull);
      const unsigned long long ss = warp_sum64(done, in ? qs : 0ull);
      if (lane == leader) {
        unsigned long long* m = slot_mem + (size_t)o * sw;
        m[nb + 3 + K] += sa;
        m[nb + 5 + K] += ss;
      }
    }
  }
  if (!direct) {
    unsigned long long* m = slot_mem + (size_t)myslot * sw;
    if (ev == EV_TOP) {
      const int bin = exit_bin(c, p);
      const unsigned long long q = __float2ull_rn(__fmul_rn(p.W, kFix));
      add64_shared(m + bin, q);
      add64_shared(m + nb + 1 + p.k, q);
      if (p.n_coll == 1u) add64_shared(m + nb + 1 + K, q);
      if (s.want_sumsq) add64_shared(m + nb + 6 + K + bin, __float2ull_rn(__fmul_rn(__fmul_rn(p.W, p.W), kFix)));
    } else if (ev == EV_BOTTOM) {
      add64_shared(m + nb + 2 + K, __float2ull_rn(__fmul_rn(p.W, kFix)));
    } else if (ev == EV_TRUNC) {
      add64_shared(m + nb + 4 + K, 1ull);
    }
  } else {
    unsigned long long* g = t.raw + (size_t)lane_inst[lane] * sw;
    if (ev == EV_TOP) {
      const int bin = exit_bin(c, p);
      const unsigned long long q = __float2ull_rn(__fmul_rn(p.W, kFix));
      atomicAdd(g + bin, q);
      atomicAdd(g + nb + 1 + p.k, q);
      if (p.n_coll == 1u) atomicAdd(g + nb + 1 + K, q);
      if (s.want_sumsq) atomicAdd(g + nb + 6 + K + bin, __float2ull_rn(__fmul_rn(__fmul_rn(p.W, p.W), kFix)));
    } else if (ev == EV_BOTTOM) {
      atomicAdd(g + nb + 2 + K, __float2ull_rn(__fmul_rn(p.W, kFix)));
    } else if (ev == EV_TRUNC) {
      atomicAdd(g + nb + 4 + K, 1ull);
    }
    if (qa) atomicAdd(g + nb + 3 + K, qa);
    atomicAdd(g + nb + 5 + K, qs);
  }
  if (ev == EV_TRUNC) atomicOr(s.status, SSS_DEV_FLAG_STEP_LIMIT);
}

// The forward one-layer kernel is held to 48 registers: five 256-thread
// blocks per SM (40 warps) keep the issue slots busy.  HERO = C > 0: each
// scheduled "instance" is a hero group of C bands, and a slot holds the C
// members' accumulators.
// SEMI: every instance is a semi-infinite slab (no thickness array).
template <bool ADJ, bool LAYERED, int HERO, bool SEMI, int MODE>
__global__ void __launch_bounds__(256, (HERO >= 4 || (ADJ && LAYERED))
                                           ? 3 : ((ADJ || LAYERED || HERO) ? 4 : 5))
walk_persistent_kernel(WalkConst c, WalkSched s, TallyOut t, GradIn gi) {
  extern __shared__ __align__(16) unsigned long long smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int slot_words = (HERO > 0 ? HERO : 1) * s.slot_words;
  unsigned long long* slot_mem = smem + (size_t)wib * 2 * slot_words;
  SlotMeta* meta =
      reinterpret_cast<SlotMeta*>(smem + (size_t)nwarps * 2 * slot_words) + 2 * wib;
  SelBuf* sel = reinterpret_cast<SelBuf*>(reinterpret_cast<SlotMeta*>(
                    smem + (size_t)nwarps * 2 * slot_words) + 2 * nwarps) + wib;
  for (int j = lane; j < 2 * slot_words; j += 32) slot_mem[j] = 0ull;
  if (lane < 2) meta[lane].gl = 0u;  // generation 0, not live
  if (lane == 0) sel->valid = 0u;
  __syncwarp();

  int cur = 0;        // slot new paths are drawn from (warp-uniform)
  bool more = true;   // the global queue may still hold units (warp-uniform)

  int st = LANE_IDLE;
  uint32_t mytag = 0;  // slot of the lane's path (bit 0) and that slot's generation
  Path p;
  p.step = 0;
  HeroState<HERO> hs;

  // Takes the next unit from the global queue into slot o.
  auto fetch = [&](int o) -> bool {
    unsigned long long u = 0;
    if (lane == 0) u = atomicAdd(s.unit_counter, 1ull);
    u = __shfl_sync(kFull, u, 0);
    const UnitRange r = unit_lookup(s, c, u);
    if (!r.ok) return false;
    float scale = 1.0f, lim = 0.0f, wsum = 1.0f;
    if (ADJ) {
      const int E = grad_exponent(c, gi, r.inst, lane);
      scale = ldexpf(1.0f, E);
      const uint32_t N = c.n_paths ? c.n_paths[r.inst] : c.uniform_paths;
      const int lgN = N > 1 ? 32 - __clz(N - 1) : 0;
      lim = ldexpf(1.0f, 62 - lgN);
      wsum = 0.0f;
      for (int k = 0; k < c.K; ++k)
        wsum = __fadd_rn(wsum, __ldg(c.w + (size_t)k * c.n_inst + r.inst));
    }
    if constexpr (HERO == 0) stage_media<LAYERED>(c, r.inst, lane, meta[o]);
    if (lane == 0) {
      SlotMeta& sm = meta[o];
      sm.inst = r.inst;
      sm.next = r.p0;
      sm.end = r.p1;
      sm.gl |= 1u;         // live, same generation
      sel->valid = 0u;     // the choice buffer belonged to another unit
      uint32_t dinst = r.inst;
      if constexpr (HERO > 0) dinst = hero_group<HERO>(c, r.inst).first;
      sm.d = c.thickness ? __ldg(c.thickness + dinst) : __int_as_float(0x7f800000);
      sm.scale = scale;
      sm.lim = lim;
      sm.wsum = wsum;
    }
    __syncwarp();
    return true;
  };

  // Moves slot o's accumulators to global memory (one atomic per nonzero word).
  auto flush = [&](int o) {
    __syncwarp();
    unsigned long long* m = slot_mem + (size_t)o * slot_words;
    const uint32_t inst = meta[o].inst;
    for (int j = lane; j < slot_words; j += 32) {
      const unsigned long long v = m[j];
      if (v != 0ull) {
        if constexpr (ADJ) {
          atomicAdd(t.raw + (size_t)j * c.n_inst + inst, v);  // [4][K][n_inst]
        } else if constexpr (HERO > 0) {
          const int mem = j / s.slot_words;  // member, then its word
          const HeroGroup G = hero_group<HERO>(c, inst);
          const uint32_t mi = G.first + (uint32_t)mem * G.stride;
          atomicAdd(t.raw + (size_t)mi * s.slot_words + (j - mem * s.slot_words), v);
        } else {
          atomicAdd(t.raw + (size_t)inst * slot_words + j, v);
        }
        m[j] = 0ull;
      }
    }
    __syncwarp();
    if (lane == 0)  // next generation, not live: the unit's late paths tally directly
      meta[o].gl = ((meta[o].gl >> 1) + 1u) << 1;
    __syncwarp();
  };

  // Draws the medium choices of paths base .. base + 31 of slot o's unit.
  auto fill_choices = [&](int o, uint32_t base) {
    const uint4 r = philox4x32_10_rk(
        make_uint4(0u, c.path_offset + base + lane, meta[o].inst + c.inst_offset, 1u), c.rk);
    sel->k[lane] = (uint8_t)staged_choice(c, meta[o], u23(r.x));
    if (lane == 0) {
      sel->base = base;
      sel->valid = 1u;
    }
    __syncwarp();
  };

  if (!fetch(0)) more = false;

  while (true) {
    const unsigned not_running = __ballot_sync(kFull, st != LANE_RUNNING);
    const int n_nr = __popc(not_running);
    if (n_nr >= s.regroup) {  // (regroup <= 32: a warp with no running lane always enters)
      // ---- 1. finished lanes tally together (one divergent block) ----
      if constexpr (!ADJ && HERO == 0) {
        const unsigned done = __ballot_sync(kFull, lane_done(st));
        if (lane_done(st)) {
          const int myslot = (int)(mytag & 1u);
          tally_exit_warp(c, s, t, p, st - 1, slot_mem, myslot,
                          (meta[myslot].gl >> 1) != (mytag >> 1), done, lane, sel->inst);
          st = LANE_IDLE;
        }
      } else if (lane_done(st)) {
        const int myslot = (int)(mytag & 1u);
        const bool direct = (meta[myslot].gl >> 1) != (mytag >> 1);
        if constexpr (HERO > 0)
          tally_path_hero<HERO>(c, s, t, p, hs, st - 1, slot_mem + (size_t)myslot * slot_words,
                                direct);
        else
          tally_path<ADJ, LAYERED>(c, s, gi, t, p, st - 1,
                                   slot_mem + (size_t)myslot * slot_words, direct);
        st = LANE_IDLE;
      }
      // ---- 2. refill idle lanes from the current unit (regrouping) ----
      unsigned idle = __ballot_sync(kFull, st == LANE_IDLE);
      while (idle != 0u) {
        const uint4 mh = *reinterpret_cast<const uint4*>(meta + cur);  // inst, next, end, gl
        const uint32_t nxt = mh.y, end = mh.z;
        if ((mh.w & 1u) && nxt < end) {
          const uint32_t take = min((uint32_t)__popc(idle), end - nxt);
          const int rank = __popc(idle & ((1u << lane) - 1u));
          uint32_t base = 0;
          if constexpr (HERO == 0) {
            const uint4 sb = *reinterpret_cast<const uint4*>(sel);  // base, valid
            base = sb.x;
            if (!(sb.y && base <= nxt && nxt + take - base <= 32u)) {
              fill_choices(cur, nxt);
              base = nxt;
            }
          }
          __syncwarp();
          if (st == LANE_IDLE && (uint32_t)rank < take) {
            if constexpr (HERO > 0)
              hero_init<HERO>(c, mh.x, c.path_offset + nxt + rank, meta[cur].d, p, hs);
            else
              path_start<LAYERED>(c, meta[cur], mh.x, sel->k[nxt + rank - base],
                                  c.path_offset + nxt + rank, p);
            if (ADJ) {
              p.gscale = meta[cur].scale;
              p.glim = meta[cur].lim;
              p.wsum = meta[cur].wsum;
            }
            st = LANE_RUNNING;
            mytag = (mh.w & ~1u) | (uint32_t)cur;  // generation * 2 + slot
            if constexpr (HERO == 0) sel->inst[lane] = mh.x;
          }
          __syncwarp();
          if (lane == 0) meta[cur].next = nxt + take;
          __syncwarp();
          idle = __ballot_sync(kFull, st == LANE_IDLE);
        } else {
          if (!more) break;
          // The other slot is reused at once: its partial sums go to global
          // memory, and its paths still running tally there directly.
          const int o = cur ^ 1;
          if (meta[o].gl & 1u) flush(o);
          if (!fetch(o)) {
            more = false;
            break;
          }
          cur = o;
        }
      }
      // (without a refill fewer than `regroup` lanes are idle, so some run)
      if (__ballot_sync(kFull, st == LANE_RUNNING) == 0u) {
        if (!more) break;
        continue;
      }
    }
    // ---- advance every running path by one draw ----
    if (st == LANE_RUNNING) {
      const int ev = path_step<ADJ, LAYERED, HERO, SEMI, MODE>(c, p, hs);
      if (ev != EV_CONTINUE) st = LANE_RUNNING + ev;
    }
  }
  __syncwarp();
  for (int o = 0; o < 2; ++o)
    if (meta[o].gl & 1u) flush(o);
}

// ------------------------------------------------------------------ plain --
// One thread per path of a single instance; block-level shared tallies.
template <bool LAYERED>
__global__ void __launch_bounds__(256)
walk_plain_kernel(WalkConst c, WalkSched s, TallyOut t, uint32_t inst, uint32_t N) {
  extern __shared__ unsigned long long smem[];
  const int slot_words = s.slot_words;
  for (int j = threadIdx.x; j < slot_words; j += blockDim.x) smem[j] = 0ull;
  __syncthreads();
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) {
    Path p;
    HeroState<0> none;
    const float d = c.thickness ? c.thickness[inst] : __int_as_float(0x7f800000);
    path_init<LAYERED>(c, inst, c.path_offset + j, d, p);
    int ev;
    do {
      ev = path_step<false, LAYERED>(c, p, none);
    } while (ev == EV_CONTINUE);
    const int nb = c.nbins;
    if (ev == EV_TOP) {
      const int bin = exit_bin(c, p);
      const unsigned long long q = __float2ull_rn(__fmul_rn(p.W, kFix));
      atomicAdd(smem + bin, q);
      atomicAdd(smem + nb + 1 + p.k, q);
      if (p.n_coll == 1u) atomicAdd(smem + nb + 1 + c.K, q);
      if (s.want_sumsq)
        atomicAdd(smem + nb + 6 + c.K + bin, __float2ull_rn(__fmul_rn(__fmul_rn(p.W, p.W), kFix)));
    } else if (ev == EV_BOTTOM) {
      atomicAdd(smem + nb + 2 + c.K, __float2ull_rn(__fmul_rn(p.W, kFix)));
    } else if (ev == EV_TRUNC) {
      atomicAdd(smem + nb + 4 + c.K, 1ull);
      atomicOr(s.status, SSS_DEV_FLAG_STEP_LIMIT);
    }
    if (p.Aacc > 0.0f) atomicAdd(smem + nb + 3 + c.K, __float2ull_rn(__fmul_rn(p.Aacc, kFix)));
    atomicAdd(smem + nb + 5 + c.K, (unsigned long long)p.step);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < slot_words; k += blockDim.x) {
    const unsigned long long v = smem[k];
    if (v) atomicAdd(t.raw + (size_t)inst * slot_words + k, v);
  }
}

// --------------------------------------------------------------- finalize --
__device__ __forceinline__ double se_of(double s, double s2, double n) {
  if (n < 2.0) return 0.0;
  const double m = s / n;
  const double v = (s2 / n - m * m) * n / (n - 1.0);
  return v > 0.0 ? sqrt(v / n) : 0.0;
}

__global__ void finalize_tallies_kernel(WalkConst c, WalkSched s, TallyOut t) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.n_inst) return;
  const int nb = c.nbins, K = c.K, nt = s.slot_words;
  const unsigned long long* r = t.raw + (size_t)i * nt;
  const uint32_t N = c.n_paths ? c.n_paths[i] : c.uniform_paths;
  const double n = (double)N;
  const double inv = N ? kInvFix / n : 0.0;
  unsigned long long sR = 0, s2R = 0;
  for (int b = 0; b <= nb; ++b) {
    sR += r[b];
    if (s.want_sumsq) s2R += r[nb + 6 + K + b];
  }
  if (t.R) t.R[i] = (double)sR * inv;
  if (t.bins)
    for (int b = 0; b < nb; ++b) t.bins[(size_t)i * nb + b] = (double)r[b] * inv;
  if (t.overflow) t.overflow[i] = (double)r[nb] * inv;
  if (t.R_k)
    for (int k = 0; k < K; ++k) t.R_k[(size_t)i * K + k] = (double)r[nb + 1 + k] * inv;
  if (t.R1) t.R1[i] = (double)r[nb + 1 + K] * inv;
  if (t.T) t.T[i] = (double)r[nb + 2 + K] * inv;
  if (t.A) t.A[i] = (double)r[nb + 3 + K] * inv;
  if (t.truncated) t.truncated[i] = r[nb + 4 + K];
  if (t.steps) t.steps[i] = N ? (double)r[nb + 5 + K] / n : 0.0;
  if (s.want_sumsq && N) {
    if (t.stderr_R) t.stderr_R[i] = se_of((double)sR * kInvFix, (double)s2R * kInvFix, n);
    if (t.stderr_bins)
      for (int b = 0; b < nb; ++b)
        t.stderr_bins[(size_t)i * nb + b] =
            se_of((double)r[b] * kInvFix, (double)r[nb + 6 + K + b] * kInvFix, n);
  }
  if (t.raw_out)
    for (int j = 0; j < nt; ++j) t.raw_out[(size_t)i * nt + j] = r[j];
  if (t.profile) {  // P_d = bins / R (Eq. 3), from the exact integer sums
    const double inv_R = sR ? 1.0 / (double)sR : 0.0;
    for (int b = 0; b < nb; ++b) t.profile[(size_t)i * nb + b] = (double)r[b] * inv_R;
  }
}

__global__ void finalize_grads_kernel(WalkConst c, GradIn gi, const unsigned long long* raw,
                                      GradOut go) {
  // one warp per instance (grad_exponent reduces over the bins with shuffles)
  const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= c.n_inst) return;
  const int E = grad_exponent(c, gi, i, lane);
  if (lane != 0) return;
  const uint32_t N = c.n_paths ? c.n_paths[i] : c.uniform_paths;
  const double scale = N ? ldexp(1.0, -E) / (double)N : 0.0;
  double* outs[4] = {go.d_alpha, go.d_sigma_t, go.d_g, go.d_w};
  for (int q = 0; q < 4; ++q) {
    if (!outs[q]) continue;
    for (int k = 0; k < c.K; ++k) {
      const size_t o = (size_t)(q * c.K + k) * c.n_inst + i;
      outs[q][(size_t)k * c.n_inst + i] = (double)(long long)raw[o] * scale;
    }
  }
  if (go.d_w) {
    for (int k = 0; k < c.K; ++k)
      if (c.w[(size_t)k * c.n_inst + i] == 0.0f) atomicOr(go.status, SSS_DEV_FLAG_ZERO_WEIGHT);
  }
  if (c.alpha2) {  // second layer: words 4K .. 4K+2
    double* outs2[3] = {go.d_alpha2, go.d_sigma_t2, go.d_g2};
    for (int q = 0; q < 3; ++q)
      if (outs2[q])
        outs2[q][i] = (double)(long long)raw[(size_t)(4 * c.K + q) * c.n_inst + i] * scale;
  }
}

// ------------------------------------------------------------ diagnostics --
__global__ void philox_kernel(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n,
                              uint32_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 r = philox4x32_10(c, k0, k1);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

// ---------------------------------------------------------------- launch --
void launch_hero_logs(const WalkConst& c, float* logs, cudaStream_t st) {
  const size_t Kn = (size_t)c.K * c.n_inst;
  if (Kn == 0) return;
  const int block = 256;
  const int grid = (int)std::min<size_t>((Kn + block - 1) / block, 148 * 16);
  hero_logs_kernel<<<grid, block, 0, st>>>(c, logs);
}

void launch_validate(const WalkConst& c, unsigned int* status, cudaStream_t st) {
  if (c.n_inst == 0) return;
  validate_params_kernel<<<(c.n_inst + 255) / 256, 256, 0, st>>>(c, status);
}

void launch_unit_prefix(const uint32_t* n_paths, uint32_t n, uint32_t C,
                        unsigned long long* block_sums, unsigned long long* total,
                        unsigned long long* prefix, cudaStream_t st) {
  const uint32_t nb = (n + 255) / 256;
  if (n > 0) unit_block_sums_kernel<<<nb, 256, 0, st>>>(n_paths, n, C, block_sums);
  unit_scan_block_sums_kernel<<<1, 1024, 0, st>>>(block_sums, nb, total);
  if (n > 0) unit_prefix_kernel<<<nb, 256, 0, st>>>(n_paths, n, C, block_sums, total, prefix);
  else cudaMemcpyAsync(prefix, total, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
}

void launch_walk_persistent(bool adj, int grid, int block, size_t smem, const WalkConst& c,
                            const WalkSched& s, const TallyOut& t, const GradIn& gi,
                            cudaStream_t st) {
  const void* fn = persistent_kernel_ptr(adj, c.alpha2 != nullptr, c.hero,
                                         c.thickness == nullptr, c.mode);
  void* args[] = {const_cast<WalkConst*>(&c), const_cast<WalkSched*>(&s),
                  const_cast<TallyOut*>(&t), const_cast<GradIn*>(&gi)};
  cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

// Semi-infinite batches (no thickness array) take the SEMI instantiations;
// two-layer slabs keep the general one.  Single-layer walks in the default
// weighting mode take instantiations with the collision rule fixed at
// compile time (no uniform branch per collision); the rest read c.mode.
const void* persistent_kernel_ptr(bool adj, bool layered, int hero, bool semi, int mode) {
#define SSS_K(A, L, H) (semi ? (const void*)walk_persistent_kernel<A, L, H, true, -1> \
                             : (const void*)walk_persistent_kernel<A, L, H, false, -1>)
#define SSS_KW(A) (semi ? (const void*)walk_persistent_kernel<A, false, 0, true, 0> \
                        : (const void*)walk_persistent_kernel<A, false, 0, false, 0>)
  if (!layered && hero == 0 && mode == 0) return adj ? SSS_KW(true) : SSS_KW(false);
  if (adj)
    return layered ? (const void*)walk_persistent_kernel<true, true, 0, false, -1>
                   : SSS_K(true, false, 0);
  if (layered) return (const void*)walk_persistent_kernel<false, true, 0, false, -1>;
  switch (hero) {
    case 1: return SSS_K(false, false, 1);
    case 2: return SSS_K(false, false, 2);
    case 3: return SSS_K(false, false, 3);
    case 4: return SSS_K(false, false, 4);
    default: return SSS_K(false, false, 0);
  }
#undef SSS_K
#undef SSS_KW
}

void launch_walk_plain(const WalkConst& c, const WalkSched& s, const TallyOut& t, uint32_t inst,
                       uint32_t N, cudaStream_t st) {
  if (N == 0) return;
  if (c.alpha2)
    walk_plain_kernel<true><<<(N + 255) / 256, 256, (size_t)s.slot_words * 8, st>>>(c, s, t, inst, N);
  else
    walk_plain_kernel<false><<<(N + 255) / 256, 256, (size_t)s.slot_words * 8, st>>>(c, s, t, inst, N);
}

void launch_finalize_tallies(const WalkConst& c, const WalkSched& s, const TallyOut& t,
                             cudaStream_t st) {
  if (c.n_inst == 0) return;
  finalize_tallies_kernel<<<(c.n_inst + 127) / 128, 128, 0, st>>>(c, s, t);
}

void launch_finalize_grads(const WalkConst& c, const GradIn& gi, const unsigned long long* raw,
                           const GradOut& go, cudaStream_t st) {
  if (c.n_inst == 0) return;
  const uint64_t threads = (uint64_t)c.n_inst * 32;
  finalize_grads_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(c, gi, raw, go);
}

void launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out,
                   cudaStream_t st) {
  if (n <= 0) return;
  philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr, k0, k1, n, out);
}

}  // namespace sss
