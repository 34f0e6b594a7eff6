// walk_core.cuh -- one path of the mixture-of-media random walk, binary32.
//
// Shared, unchanged, by the forward kernels and the path-replay adjoint so a
// replayed path is the forward path bit for bit.  Every rounding step is
// spelled out with __f*_rn / __fmaf_rn intrinsics, which the compiler never
// contracts or reassociates, so the result of a step does not depend on the
// kernel it is inlined into.
//
// What a path does (paper Sec. 4.1, Eq. 2-4; Sec. 7):
//   1. pick medium k with probability w_k / sum(w), once, before the walk;
//   2. enter at the origin along +z (normal incidence, Eq. 3) with weight
//      1 - R0 (specular part excluded) or 1;
//   3. repeat: exponential flight with sigma_t,k (transmittance T);
//        flight reaches a face  -> smooth-dielectric Fresnel: reflect with
//                                  probability F, else leave (tally);
//        otherwise, a collision -> albedo weighting (W *= alpha_k) with
//                                  Russian roulette, or analog absorption;
//                                  then Henyey-Greenstein scattering with g_k.
// Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = 64-bit seed,
// counter = (step, path, instance, tag); tag 1 draws the medium, tag 0 one
// block of four uniforms per step (flight, Fresnel-or-HG cosine, azimuth,
// roulette/absorption).
#pragma once
#include <cstdint>

namespace sss {

// ---------------------------------------------------------------- Philox --
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The same block with the key schedule precomputed: rk[2r], rk[2r+1] are the
// round-r keys (k0 + r W0, k1 + r W1).  With rk in the kernel's parameter
// (constant) bank the XORs read it directly, so the key additions vanish.
// Each round's two products are taken as one 32x32->64 multiply each.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53ull;
    const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57ull;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1], (uint32_t)p0);
  }
  return c;
}

// A walk step's block, with its first two rounds partly done per path.  The
// step counter is (step, path, instance, 0).  In round 1 the product
// instance * M1 does not depend on the step, and neither does round 1's
// lane-x output x1 = hi(instance * M1) ^ path ^ k0; in round 2 the product
// x1 * M0 is then also a per-path constant.  So at the start of a path
//   b1 = lo(instance * M1),  e2 = hi(x1 * M0) ^ (round-2 key 1),  f2 = lo(x1 * M0)
// are formed once (philox_path), and a step (philox_step) computes rounds
// 1-2 from them and rounds 3-10 as usual: the same Philox4x32-10 block as
// philox4x32_10_rk, with two 32x32->64 products and one XOR fewer per draw.
struct PhiloxPath {
  uint32_t b1, e2, f2;
};

__device__ __forceinline__ PhiloxPath philox_path(uint32_t path, uint32_t cinst,
                                                  const uint32_t* rk) {
  const unsigned long long p1 = (unsigned long long)cinst * 0xCD9E8D57ull;
  const uint32_t x1 = (uint32_t)(p1 >> 32) ^ path ^ rk[0];
  const unsigned long long q0 = (unsigned long long)x1 * 0xD2511F53ull;
  PhiloxPath r;
  r.b1 = (uint32_t)p1;
  r.e2 = (uint32_t)(q0 >> 32) ^ rk[3];
  r.f2 = (uint32_t)q0;
  return r;
}

__device__ __forceinline__ uint4 philox_step(uint32_t step, const PhiloxPath& pc,
                                             const uint32_t* rk) {
  // round 1: (step, path, instance, 0) -> (x1, b1, z1, w1)
  const unsigned long long p0 = (unsigned long long)step * 0xD2511F53ull;
  const uint32_t z1 = (uint32_t)(p0 >> 32) ^ rk[1], w1 = (uint32_t)p0;
  // round 2: products x1 * M0 (per path) and z1 * M1
  const unsigned long long p1 = (unsigned long long)z1 * 0xCD9E8D57ull;
  uint4 c = make_uint4((uint32_t)(p1 >> 32) ^ pc.b1 ^ rk[2], (uint32_t)p1, pc.e2 ^ w1, pc.f2);
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    const unsigned long long q0 = (unsigned long long)c.x * 0xD2511F53ull;
    const unsigned long long q1 = (unsigned long long)c.z * 0xCD9E8D57ull;
    c = make_uint4((uint32_t)(q1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)q1,
                   (uint32_t)(q0 >> 32) ^ c.w ^ rk[2 * r + 1], (uint32_t)q0);
  }
  return c;
}

// 23 random bits k -> (k + 1/2) * 2^-23, exact in binary32, strictly in (0,1).
// The bits become the mantissa of 1 + k 2^-23 in [1, 2); subtracting
// 1 - 2^-24 (exact: both operands lie in [1/2, 2]) leaves (k + 1/2) 2^-23.
// The top 23 bits are taken as the high word of x * 2^23 plus the encoding
// of 1.0 in one integer multiply-add (the same bits as (x >> 9) | 0x3f800000,
// since x >> 9 < 2^23), which issues on the multiply-add pipe instead of two
// logic-unit operations.
__device__ __forceinline__ float u23(uint32_t x) {
  uint32_t y;
  asm("mad.hi.u32 %0, %1, 8388608, 1065353216;" : "=r"(y) : "r"(x));
  return __fsub_rn(__uint_as_float(y), 0.99999994039535522f);
}

// Two uniforms at once: the same values as u23(a), u23(b), with the two
// (exact) subtractions issued as one paired binary32 instruction.
__device__ __forceinline__ float2 u23x2(uint32_t a, uint32_t b) {
  uint32_t ya, yb;
  asm("mad.hi.u32 %0, %1, 8388608, 1065353216;" : "=r"(ya) : "r"(a));
  asm("mad.hi.u32 %0, %1, 8388608, 1065353216;" : "=r"(yb) : "r"(b));
  return __fadd2_rn(make_float2(__uint_as_float(ya), __uint_as_float(yb)),
                    make_float2(-0.99999994039535522f, -0.99999994039535522f));
}

// ------------------------------------------------------------ arguments --
struct WalkConst {
  const float* alpha;     // [K][n_inst]
  const float* sigma_t;   // [K][n_inst]
  const float* g;         // [K][n_inst]
  const float* w;         // [K][n_inst]
  const uint32_t* n_paths;  // [n_inst] or null
  const float* thickness;   // [n_inst] or null
  uint32_t uniform_paths;
  uint32_t n_inst;
  int K;
  float n_rel;
  float W0;          // entry weight
  int nbins;
  float bin_scale;   // nbins / r_max
  int mode;          // 0 weight + roulette, 1 analog
  float rr_th;       // roulette threshold
  float inv_rr_th;   // 1 / rr_th (exact for the power-of-two default)
  uint32_t max_steps;
  uint32_t key0, key1;
  uint32_t path_offset;
  uint32_t rk[20];   // Philox round keys derived from (key0, key1)
  uint32_t inst_offset;  // added to the instance index in the counters
  int incidence;         // 0 normal, 1 cosine-weighted lobe
  int entry_fresnel;
  // optional second layer (two-layer slab): [n_inst] each, or null
  const float *alpha2, *sigma_t2, *g2, *d1;
  // logarithmic radial bins: 1/r_min and 1/log2(q), or log_bins = 0
  int log_bins;
  float inv_rmin, inv_log2q;
  int select_uniform;  // 1: medium chosen uniformly, weight K w_k / sum(w)
  // hero-wavelength sharing: C bands per group (0 = off), bands per texel,
  // 1 = rotation orbits {q, q + nb/C, ...}, 0 = blocks of C adjacent bands
  int hero, hero_nb, hero_orbits;
  const float* hero_logs;  // [3][K][n_inst]: log2 sigma_t, log2(1 - g^2), log2 mixture weight
};

constexpr int kHeroMax = 4;

enum Event : int { EV_CONTINUE = 0, EV_TOP = 1, EV_BOTTOM = 2, EV_DEAD = 3, EV_TRUNC = 4 };

struct Path {
  float x, y, z, ux, uy, uz;
  float W;        // current weight
  float Aacc;     // weight deposited by collisions
  float alpha, sigt, fl, g, d;  // fl = ln(2) / sigma_t (flight scale for log2)
  uint32_t step, inst, n_coll;
  PhiloxPath pc;  // per-path constants of the step blocks' counters (philox_path)
  int k;
  float L;        // path length inside the medium (adjoint; top layer if layered)
  float G;        // sum of d log p_HG / d g (adjoint; top layer if layered)
  uint32_t n2;    // two-layer adjoint: collisions, length and HG score in the
  float L2, G2;   // second layer (n_coll counts both layers)
  // two-layer slab: optics of the other layer, interface depth, current layer
  float a_o, fl_o, g_o, sigt_o, d1;
  int layer;
  float gscale, glim, wsum;  // adjoint: fixed-point scale, per-path limit, sum(w)
  float hc1, hc2;  // Henyey-Greenstein constants of g (hg_consts)
  float ga;        // adjoint: -2g / (1 - g^2), the constant part of d log p_HG / d g
};

// The per-medium constants of the Henyey-Greenstein inversion (hg_mu):
// ((1 + g^2) / 2, g (3 - g^2) / 2), formed once per medium or path.
__device__ __forceinline__ float2 hg_consts(float g) {
  const float g2 = __fmul_rn(g, g);
  return make_float2(__fmaf_rn(g2, 0.5f, 0.5f), __fmul_rn(g, __fmaf_rn(g2, -0.5f, 1.5f)));
}

// Hero-wavelength sharing state of a path of a group of C members: the hero
// index h and, for the other members m (member (h + 1 + m) mod C), weight W,
// log2 path-density difference D to the hero, and their optics as alpha,
// (sigma_h - sigma) log2 e, log2(sigma / sigma_h), g and
// log2((1 - g^2) / (1 - g_h^2)).  Empty when sharing is off.
template <int C>
struct HeroState {
  int h;
  float W[C > 1 ? C - 1 : 1], D[C > 1 ? C - 1 : 1];
  float a[C > 1 ? C - 1 : 1], ds[C > 1 ? C - 1 : 1], ls[C > 1 ? C - 1 : 1],
      g[C > 1 ? C - 1 : 1], cg[C > 1 ? C - 1 : 1];
};
template <>
struct HeroState<0> {};

// Hardware approximations (one MUFU operation each, a few ulp).
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// The flush-to-zero forms of the other hardware approximations: the same
// results for normal operands and results (the only kind the walk produces),
// without the compiler's rescaling around them for subnormal ones.
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float div_approx(float a, float b) {
  float y;
  asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
  return y;
}
__device__ __forceinline__ void sincos_approx(float x, float* sp, float* cp) {
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*sp) : "f"(x));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*cp) : "f"(x));
}

// Paired binary32 arithmetic (one instruction for two lanes' worth of
// values); each half is rounded exactly like the scalar __f*_rn operation.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Unpolarised Fresnel reflectance, medium (index n) -> outside (index 1),
// without branches: total internal reflection (sin^2 t = n^2 sin^2 i >= 1)
// and n = 1 are selected at the end; the two quotients share one reciprocal.
// (Under total internal reflection 1 - sin^2 t < 0 and the arithmetic below
// is NaN, which the selection replaces by 1.)
// fresnel_parts: sin^2 t and the reflectance without the two selections.
__device__ __forceinline__ float fresnel_parts(float cos_i, float n, float* sin2_t_out) {
  const float sin2_t = __fmul_rn(__fmul_rn(n, n), __fmaf_rn(-cos_i, cos_i, 1.0f));
  const float cos_t = sqrt_approx(__fsub_rn(1.0f, sin2_t));
  const float2 nc = __fmul2_rn(f2(n, n), f2(cos_i, cos_t));  // (n cos_i, n cos_t)
  const float2 sp = __fadd2_rn(f2(nc.x, cos_i), f2(cos_t, nc.y));  // (sd, pd)
  const float inv = rcp_approx(__fmul_rn(sp.x, sp.y));
  const float2 df = __fadd2_rn(f2(nc.x, cos_i), f2(-cos_t, -nc.y));
  const float2 rr = __fmul2_rn(__fmul2_rn(df, f2(sp.y, sp.x)), f2(inv, inv));
  const float rs = rr.x, rp = rr.y;
  *sin2_t_out = sin2_t;
  return __fmul_rn(0.5f, __fmaf_rn(rs, rs, __fmul_rn(rp, rp)));
}
__device__ __forceinline__ float fresnel(float cos_i, float n) {
  float sin2_t;
  float F = fresnel_parts(cos_i, n, &sin2_t);
  F = sin2_t >= 1.0f ? 1.0f : F;
  return n == 1.0f ? 0.0f : F;
}
// The reflect-or-leave choice at a face, u < fresnel(cos_i, n), taken with
// predicates instead of the two selections: total internal reflection always
// reflects, n = 1 never does (cos_i = 0, where the two forms would differ for
// n = 1, never reaches a face).
__device__ __forceinline__ bool fresnel_reflects(float cos_i, float n, float u) {
  float sin2_t;
  const float F = fresnel_parts(cos_i, n, &sin2_t);
  return sin2_t >= 1.0f || (n != 1.0f && u < F);
}

// Medium choice: first k whose running binary32 CDF of w/sum(w) exceeds u.
__device__ __forceinline__ int select_medium(const WalkConst& c, uint32_t inst, float u) {
  float wk[4];
  float total = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    wk[k] = k < c.K ? __ldg(c.w + (size_t)k * c.n_inst + inst) : 0.0f;
    if (k < c.K) total = __fadd_rn(total, wk[k]);
  }
  const float inv = __fdiv_rn(1.0f, total);
  float cdf = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k < c.K - 1) {
      cdf = __fadd_rn(cdf, __fmul_rn(wk[k], inv));
      if (u < cdf) return k;
    }
  }
  return c.K - 1;
}

// d log p_HG(mu; g) / d g = -2g / (1 - g^2) - 3 (g - mu) / (1 + g^2 - 2 g mu).
// The first term is a constant of the medium (hg_dlogp_dg_const, formed once
// per path); the second is taken per scattering with the hardware reciprocal.
__device__ __forceinline__ float hg_dlogp_dg_const(float g) {
  return __fdiv_rn(__fmul_rn(-2.0f, g), __fmaf_rn(-g, g, 1.0f));
}
__device__ __forceinline__ float hg_dlogp_dg(float g, float ga, float mu) {
  const float den = __fmaf_rn(g, g, __fmaf_rn(-2.0f * g, mu, 1.0f));
  return __fmaf_rn(__fmul_rn(-3.0f, __fsub_rn(g, mu)), rcp_approx(den), ga);
}

// Cosine-weighted incident lobe (incidence = 1): outside cosine sqrt(u),
// azimuth 2 pi u', refracted by Snell's law; entry weight 1 - F at the
// refracted angle, times the selection weight w_sel.  One Philox block with
// tag 2 per path.
__device__ __forceinline__ void entry_lobe(const WalkConst& c, uint32_t path, uint32_t cinst,
                                           float w_sel, Path& p) {
  const uint4 e = philox4x32_10_rk(make_uint4(0u, path, cinst, 2u), c.rk);
  const float mu_o = sqrt_approx(u23(e.x));
  const float sin_i = div_approx(sqrt_approx(fmaxf(0.0f, __fmaf_rn(-mu_o, mu_o, 1.0f))),
                                 c.n_rel);
  float sp, cp;
  sincos_approx(__fmul_rn(6.2831853071795865f, __fsub_rn(u23(e.y), 0.5f)), &sp, &cp);
  p.ux = -__fmul_rn(sin_i, cp);
  p.uy = -__fmul_rn(sin_i, sp);
  p.uz = sqrt_approx(fmaxf(0.0f, __fmaf_rn(-sin_i, sin_i, 1.0f)));
  p.W = __fmul_rn(c.entry_fresnel ? __fsub_rn(1.0f, fresnel(p.uz, c.n_rel)) : 1.0f, w_sel);
}

// Flight scale ln(2) / sigma_t of a medium (exponential flights use log2).
__device__ __forceinline__ float flight_scale(float sigma_t) {
  return __fmul_rn(0.693147180559945309f, __fdiv_rn(1.0f, sigma_t));
}

// Starts a path from global memory (the plain kernel and hero-wavelength
// groups; the persistent kernel starts its paths from the media it staged
// per unit, with the same arithmetic).  inst indexes the parameter arrays;
// the random-number counters use instance number inst + instance_offset, or
// with OWN_CTR = false `ctr_inst` (a hero group's first member).
template <bool LAYERED = false, bool OWN_CTR = true>
__device__ __forceinline__ void path_init(const WalkConst& c, uint32_t inst, uint32_t path,
                                          float d, Path& p, uint32_t ctr_inst = 0) {
  // (the counter instance is spelled out at each use: naming it once costs
  // the adjoint kernel a register spill)
  const uint4 r = philox4x32_10_rk(
      make_uint4(0u, path, OWN_CTR ? inst + c.inst_offset : ctr_inst, 1u), c.rk);
  int k;
  float w_sel = 1.0f;  // w_k / (p_k sum(w)), the estimator weight of the choice
  if (!c.select_uniform) {
    k = select_medium(c, inst, u23(r.x));
  } else {
    // uniform choice (u K < K in binary32 for K <= 4), reweighted so the
    // mixture of Eq. 4 is still estimated without bias
    k = min(c.K - 1, (int)__fmul_rn(u23(r.x), (float)c.K));
    float total = 0.0f;
    for (int j = 0; j < c.K; ++j) total = __fadd_rn(total, __ldg(c.w + (size_t)j * c.n_inst + inst));
    w_sel = __fmul_rn(__fmul_rn((float)c.K, __ldg(c.w + (size_t)k * c.n_inst + inst)),
                      __fdiv_rn(1.0f, total));
  }
  const size_t off = (size_t)k * c.n_inst + inst;
  p.k = k;
  p.alpha = __ldg(c.alpha + off);
  p.sigt = __ldg(c.sigma_t + off);
  p.fl = flight_scale(p.sigt);
  p.g = __ldg(c.g + off);
  const float2 hc = hg_consts(p.g);
  p.hc1 = hc.x;
  p.hc2 = hc.y;
  p.ga = hg_dlogp_dg_const(p.g);
  p.d = d;
  p.x = 0.0f; p.y = 0.0f; p.z = 0.0f;
  p.ux = 0.0f; p.uy = 0.0f; p.uz = 1.0f;
  p.W = __fmul_rn(c.W0, w_sel);
  if (c.incidence == 1)
    entry_lobe(c, path, OWN_CTR ? inst + c.inst_offset : ctr_inst, w_sel, p);
  p.Aacc = 0.0f;
  p.step = 0u;
  p.inst = inst;
  p.pc = philox_path(path, OWN_CTR ? inst + c.inst_offset : ctr_inst, c.rk);
  p.n_coll = 0u;
  p.L = 0.0f;
  p.G = 0.0f;
  if (LAYERED) {
    p.layer = 0;
    p.n2 = 0u;
    p.L2 = 0.0f;
    p.G2 = 0.0f;
    p.d1 = __ldg(c.d1 + inst);
    p.a_o = __ldg(c.alpha2 + inst);
    p.sigt_o = __ldg(c.sigma_t2 + inst);
    p.fl_o = flight_scale(p.sigt_o);
    p.g_o = __ldg(c.g2 + inst);
  }
}

// Henyey-Greenstein cosine by CDF inversion.  With xi = 2u - 1, the textbook
// inverse  mu = (1 + g^2 - ((1-g^2)/(1+g xi))^2) / (2g)  is rewritten,
// multiplying out and dividing by g, as the branch-free
//   mu = ( (1 + g^2)/2 * xi (2 + g xi) + g (3 - g^2)/2 ) / (1 + g xi)^2,
// exact for every g in (-1, 1) (g = 0 gives mu = xi) and free of the
// 1/g cancellation of the textbook form at small g.  Lanes holding media
// with different g run the same instructions.  hc1, hc2 = hg_consts(g).
__device__ __forceinline__ float hg_mu(float g, float hc1, float hc2, float u) {
  const float xi = __fmaf_rn(2.0f, u, -1.0f);  // exact
  const float tx = __fmaf_rn(g, xi, 2.0f), ty = __fmaf_rn(g, xi, 1.0f);  // 2 + g xi, 1 + g xi
  const float num = __fmaf_rn(hc1, __fmul_rn(xi, tx), hc2);
  const float mu = div_approx(num, __fmul_rn(ty, ty));
  return fminf(1.0f, fmaxf(-1.0f, mu));
}


// New direction after a scattering with cosine mu and azimuth phi = 2 pi u:
// the standard frame rotation of (ux, uy, uz), with the pole |uz| ~ 1 taken
// in the fixed frame, renormalised.  phi is evaluated as phi - pi in
// (-pi, pi) and the sine and cosine negated.
__device__ __forceinline__ void scatter_direction(Path& p, float mu, float u) {
  float sp, cp;
  sincos_approx(__fmaf_rn(u, 6.2831853071795865f, -3.14159265358979324f), &sp, &cp);
  sp = -sp;
  cp = -cp;
  // mu is clamped to [-1, 1], so 1 - mu^2 (one rounding) is never negative
  const float st = sqrt_approx(__fmaf_rn(-mu, mu, 1.0f));
  const float s2 = __fmaf_rn(-p.uz, p.uz, 1.0f);
  const float itmp = rsqrt_approx(s2);
  const float2 ts = __fmul2_rn(make_float2(s2, st), make_float2(itmp, itmp));
  const float tmp = ts.x, sti = ts.y;
  const float uzcp = __fmul_rn(p.uz, cp);
  const bool polar = fabsf(p.uz) > 0.999999f;
  // (nx, ny) off the pole: sti (u_xy uz cp -+ u_yx sp) + u_xy mu, in pairs
  const float2 cross_sp = __fmul2_rn(f2(-p.uy, p.ux), f2(sp, sp));
  const float2 inner = __ffma2_rn(f2(p.ux, p.uy), f2(uzcp, uzcp), cross_sp);
  const float2 nxy = __ffma2_rn(f2(sti, sti), inner, __fmul2_rn(f2(p.ux, p.uy), f2(mu, mu)));
  const float2 pxy = __fmul2_rn(f2(st, st), f2(cp, sp));
  const float nx = polar ? pxy.x : nxy.x;
  const float ny = polar ? pxy.y : nxy.y;
  const float nz = polar ? (p.uz >= 0.0f ? mu : -mu)
                         : __fmaf_rn(-pxy.x, tmp, __fmul_rn(p.uz, mu));
  const float inr = rsqrt_approx(__fmaf_rn(nx, nx, __fmaf_rn(ny, ny, __fmul_rn(nz, nz))));
  const float2 uxy = __fmul2_rn(f2(nx, ny), f2(inr, inr));
  p.ux = uxy.x;
  p.uy = uxy.y;
  p.uz = __fmul_rn(nz, inr);
}

// One random-number draw of the walk.  Returns the event it ended in.
// The flight and face test are common; the face (Fresnel) and the collision
// (weighting, Henyey-Greenstein, rotation) are then two branches, so a warp
// runs each with the lanes that met that event.  SEMI = true compiles the
// semi-infinite slab (no far face: p.d is +inf), where only the entry face
// can be met; the results are those of the general form for d = +inf.
// MODE fixes the collision rule at compile time (0 albedo weighting with
// roulette, 1 analog absorption) or, at -1, takes it from c.mode.
template <bool ADJ, bool LAYERED = false, int HERO = 0, bool SEMI = false, int MODE = -1>
__device__ __forceinline__ int path_step(const WalkConst& c, Path& p, HeroState<HERO>& hs) {
  if (p.step >= c.max_steps) return EV_TRUNC;
  const uint4 r = philox_step(p.step, p.pc, c.rk);
  p.step++;
  const float2 u01 = u23x2(r.x, r.y), u23_ = u23x2(r.z, r.w);
  const float u0 = u01.x, u1 = u01.y, u2 = u23_.x, u3 = u23_.y;

  // Exponential free flight -ln(u0) / sigma_t, from the hardware log2
  // (absolute error <= 2^-22 mean free paths near u0 = 1, 2 ulp elsewhere).
  // |lg2 u0| = -lg2 u0 for u0 < 1; the absolute value (an operand modifier)
  // also keeps the flight non-negative where the approximation errs above 0.
  const float s = __fmul_rn(fabsf(lg2_approx(u0)), p.fl);
  // Distance to the face the path is heading to.
  const float iuz = rcp_approx(p.uz);
  const float inf = __int_as_float(0x7f800000);
  float db;
  bool cross = false;  // reaches the internal interface of a two-layer slab
  const bool top = p.uz < 0.0f;
  if (SEMI) {
    db = p.uz < 0.0f ? __fmul_rn(-p.z, iuz) : inf;
  } else if (!LAYERED) {
    db = p.uz < 0.0f ? __fmul_rn(-p.z, iuz)
                     : (p.uz > 0.0f ? __fmul_rn(__fsub_rn(p.d, p.z), iuz) : inf);
  } else {
    const float ztop = p.layer ? p.d1 : 0.0f;
    const float zbot = p.layer ? p.d : p.d1;
    db = p.uz < 0.0f ? __fmul_rn(__fsub_rn(ztop, p.z), iuz)
                     : (p.uz > 0.0f ? __fmul_rn(__fsub_rn(zbot, p.z), iuz) : inf);
  }
  const bool hit = db <= s;
  if (LAYERED) cross = hit && (top == (p.layer == 1));
  const float dist = hit ? db : s;
  const float2 xy = __ffma2_rn(f2(dist, dist), f2(p.ux, p.uy), f2(p.x, p.y));
  p.x = xy.x;
  p.y = xy.y;
  // the plane reached at a face (a semi-infinite slab has only the top face)
  const float zface = SEMI ? 0.0f : (cross ? p.d1 : (top ? 0.0f : p.d));
  if (ADJ) {
    if (LAYERED && p.layer) p.L2 = __fadd_rn(p.L2, dist);
    else p.L = __fadd_rn(p.L, dist);
  }

  bool reflect = false, dead = false;
  if constexpr (HERO <= 1) {
    // The face and the collision are separate branches, so each lane runs
    // only the arithmetic of the event it met.
    if (hit) {
      // Face: smooth-dielectric Fresnel, reflect with probability F.
      p.z = zface;
      reflect = !cross && fresnel_reflects(fabsf(p.uz), c.n_rel, u1);
      if (reflect) p.uz = -p.uz;
    } else {
      p.z = __fmaf_rn(dist, p.uz, p.z);
      // Collision: albedo weighting with roulette, or analog absorption.
      if (MODE < 0 ? c.mode == 0 : MODE == 0) {
        // the surviving weight W alpha and the deposit W - W alpha (one rounding)
        const float Wn = __fmul_rn(p.W, p.alpha);
        const float An = __fadd_rn(__fmaf_rn(p.W, -p.alpha, p.W), p.Aacc);
        const bool low = Wn < c.rr_th;
        dead = low && !(u3 < __fmul_rn(Wn, c.inv_rr_th));
        p.W = low ? c.rr_th : Wn;
        p.Aacc = An;
      } else {
        dead = u3 >= p.alpha;
        p.Aacc = dead ? __fadd_rn(p.Aacc, p.W) : p.Aacc;
      }
      p.n_coll += 1u;
      if (ADJ && LAYERED) p.n2 += p.layer ? 1u : 0u;
      // Henyey-Greenstein scattering with this medium's g.
      const float mu = hg_mu(p.g, p.hc1, p.hc2, u1);
      if (ADJ) {
        const float dl = dead ? 0.0f : hg_dlogp_dg(p.g, p.ga, mu);
        if (LAYERED && p.layer) p.G2 = __fadd_rn(p.G2, dl);
        else p.G = __fadd_rn(p.G, dl);
      }
      scatter_direction(p, mu, u2);
    }
  } else {
    // Hero-wavelength members (HERO = C > 1), the same two branches.  Every
    // draw adds each member's flight density term (sigma_h - sigma_m) dist
    // log2 e; a collision adds the members' log2(sigma_m / sigma_h), weights
    // and Henyey-Greenstein density ratios.
#pragma unroll
    for (int m = 0; m < HERO - 1; ++m) hs.D[m] = __fmaf_rn(hs.ds[m], dist, hs.D[m]);
    if (hit) {
      p.z = zface;
      reflect = !cross && fresnel_reflects(fabsf(p.uz), c.n_rel, u1);
      if (reflect) p.uz = -p.uz;
    } else {
      p.z = __fmaf_rn(dist, p.uz, p.z);
      // Roulette is decided on the largest member weight Wr and boosts every
      // member by rr_th / Wr.
      const float Wn = __fmul_rn(p.W, p.alpha);
      const float An = __fadd_rn(__fmaf_rn(p.W, -p.alpha, p.W), p.Aacc);
      float Wm[HERO > 1 ? HERO - 1 : 1];
      float Wr = Wn;
#pragma unroll
      for (int m = 0; m < HERO - 1; ++m) {
        hs.D[m] = __fadd_rn(hs.ls[m], hs.D[m]);
        Wm[m] = __fmul_rn(hs.W[m], hs.a[m]);
        Wr = fmaxf(Wr, Wm[m]);
      }
      const bool low = Wr < c.rr_th;
      dead = low && !(u3 < __fmul_rn(Wr, c.inv_rr_th));
      const float boost = __fmul_rn(c.rr_th, rcp_approx(Wr));
      p.W = low ? (Wn == Wr ? c.rr_th : __fmul_rn(Wn, boost)) : Wn;
#pragma unroll
      for (int m = 0; m < HERO - 1; ++m)
        hs.W[m] = low ? (Wm[m] == Wr ? c.rr_th : __fmul_rn(Wm[m], boost)) : Wm[m];
      p.Aacc = An;
      p.n_coll += 1u;
      // Henyey-Greenstein scattering with the hero's g, and the members'
      //   log2 p_HG(mu; g_m) - log2 p_HG(mu; g_h)
      //   = log2((1-g_m^2)/(1-g_h^2)) - 1.5 (log2(1+g_m^2-2 g_m mu) - log2(1+g_h^2-2 g_h mu))
      const float mu = hg_mu(p.g, p.hc1, p.hc2, u1);
      if (!dead) {
        const float lh =
            lg2_approx(__fmaf_rn(__fmul_rn(-2.0f, p.g), mu, __fmaf_rn(p.g, p.g, 1.0f)));
#pragma unroll
        for (int m = 0; m < HERO - 1; ++m) {
          const float gm = hs.g[m];
          const float lm =
              lg2_approx(__fmaf_rn(__fmul_rn(-2.0f, gm), mu, __fmaf_rn(gm, gm, 1.0f)));
          hs.D[m] = __fadd_rn(__fmaf_rn(-1.5f, __fsub_rn(lm, lh), hs.cg[m]), hs.D[m]);
        }
      }
      scatter_direction(p, mu, u2);
    }
  }

  if (LAYERED && cross) {  // continue in the other layer with a fresh flight
    float t;
    t = p.alpha; p.alpha = p.a_o; p.a_o = t;
    t = p.fl; p.fl = p.fl_o; p.fl_o = t;
    t = p.g; p.g = p.g_o; p.g_o = t;
    const float2 hc = hg_consts(p.g);  // the new layer's Henyey-Greenstein constants
    p.hc1 = hc.x;
    p.hc2 = hc.y;
    if (ADJ) p.ga = hg_dlogp_dg_const(p.g);
    t = p.sigt; p.sigt = p.sigt_o; p.sigt_o = t;
    p.layer ^= 1;
    return EV_CONTINUE;
  }
  if (dead) return EV_DEAD;
  if (hit && !reflect) return (SEMI || top) ? EV_TOP : EV_BOTTOM;
  return EV_CONTINUE;
}

// Radial bin of a top exit (nbins = overflow), linear or logarithmic.
__device__ __forceinline__ int exit_bin(const WalkConst& c, const Path& p) {
  const float rr = sqrt_approx(__fmaf_rn(p.x, p.x, __fmul_rn(p.y, p.y)));
  if (!c.log_bins) return (int)fminf(floorf(__fmul_rn(rr, c.bin_scale)), (float)c.nbins);
  const float t = __fmul_rn(rr, c.inv_rmin);
  if (t < 1.0f) return 0;
  return (int)fminf(1.0f + floorf(__fmul_rn(lg2_approx(t), c.inv_log2q)), (float)c.nbins);
}

}  // namespace sss
