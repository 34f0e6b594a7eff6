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

// 23 random bits k -> (k + 1/2) * 2^-23, exact in binary32, strictly in (0,1).
// The bits become the mantissa of 1 + k 2^-23 in [1, 2); subtracting
// 1 - 2^-24 (exact: both operands lie in [1/2, 2]) leaves (k + 1/2) 2^-23.
__device__ __forceinline__ float u23(uint32_t x) {
  return __fsub_rn(__uint_as_float(0x3f800000u | (x >> 9)), 0.99999994039535522f);
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
};

enum Event : int { EV_CONTINUE = 0, EV_TOP = 1, EV_BOTTOM = 2, EV_DEAD = 3, EV_TRUNC = 4 };

struct Path {
  float x, y, z, ux, uy, uz;
  float W;        // current weight
  float Aacc;     // weight deposited by collisions
  float alpha, sigt, inv_sigt, g, d;
  uint32_t step, path, inst, n_coll;
  int k;
  float L;        // path length inside the medium (adjoint)
  float G;        // sum of d log p_HG / d g (adjoint)
  int bin;        // exit bin on a top exit (nbins = overflow)
  float gscale, glim, wsum;  // adjoint: fixed-point scale, per-path limit, sum(w)
};

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

__device__ __forceinline__ void path_init(const WalkConst& c, uint32_t inst, uint32_t path,
                                          float d, Path& p) {
  const uint4 r = philox4x32_10(make_uint4(0u, path, inst, 1u), c.key0, c.key1);
  const int k = select_medium(c, inst, u23(r.x));
  const size_t off = (size_t)k * c.n_inst + inst;
  p.k = k;
  p.alpha = __ldg(c.alpha + off);
  p.sigt = __ldg(c.sigma_t + off);
  p.inv_sigt = __fdiv_rn(1.0f, p.sigt);
  p.g = __ldg(c.g + off);
  p.d = d;
  p.x = 0.0f; p.y = 0.0f; p.z = 0.0f;
  p.ux = 0.0f; p.uy = 0.0f; p.uz = 1.0f;
  p.W = c.W0;
  p.Aacc = 0.0f;
  p.step = 0u;
  p.path = path;
  p.inst = inst;
  p.n_coll = 0u;
  p.L = 0.0f;
  p.G = 0.0f;
  p.bin = 0;
}

// Unpolarised Fresnel reflectance, medium (index n) -> outside (index 1).
__device__ __forceinline__ float fresnel(float cos_i, float n) {
  if (n == 1.0f) return 0.0f;
  const float sin2_i = fmaxf(0.0f, __fmaf_rn(-cos_i, cos_i, 1.0f));
  const float sin_t = __fmul_rn(n, __fsqrt_rn(sin2_i));
  if (sin_t >= 1.0f) return 1.0f;
  const float cos_t = __fsqrt_rn(__fmaf_rn(-sin_t, sin_t, 1.0f));
  const float nci = __fmul_rn(n, cos_i);
  const float nct = __fmul_rn(n, cos_t);
  const float rs = __fdividef(__fsub_rn(nci, cos_t), __fadd_rn(nci, cos_t));
  const float rp = __fdividef(__fsub_rn(cos_i, nct), __fadd_rn(cos_i, nct));
  return __fmul_rn(0.5f, __fmaf_rn(rs, rs, __fmul_rn(rp, rp)));
}

// Henyey-Greenstein cosine by CDF inversion.  With xi = 2u - 1, the textbook
// inverse  mu = (1 + g^2 - ((1-g^2)/(1+g xi))^2) / (2g)  is rewritten,
// multiplying out and dividing by g, as the branch-free
//   mu = ((1 + g^2)(2 xi + g xi^2) + g (3 - g^2)) / (2 (1 + g xi)^2),
// exact for every g in (-1, 1) (g = 0 gives mu = xi) and free of the
// 1/g cancellation of the textbook form at small g.  Lanes holding media
// with different g run the same instructions.
__device__ __forceinline__ float hg_mu(float g, float u) {
  const float xi = __fsub_rn(__fmul_rn(2.0f, u), 1.0f);  // exact
  const float g2 = __fmul_rn(g, g);
  const float a = __fmaf_rn(g, __fmul_rn(xi, xi), __fmul_rn(2.0f, xi));  // 2 xi + g xi^2
  const float num = __fmaf_rn(__fadd_rn(1.0f, g2), a, __fmul_rn(g, __fsub_rn(3.0f, g2)));
  const float den = __fmaf_rn(g, xi, 1.0f);
  const float mu = __fdividef(num, __fmul_rn(2.0f, __fmul_rn(den, den)));
  return fminf(1.0f, fmaxf(-1.0f, mu));
}

__device__ __forceinline__ float hg_dlogp_dg(float g, float mu) {
  const float a = __fdiv_rn(__fmul_rn(-2.0f, g), __fmaf_rn(-g, g, 1.0f));
  const float den = __fmaf_rn(g, g, __fmaf_rn(-2.0f * g, mu, 1.0f));
  const float b = __fdiv_rn(__fmul_rn(-3.0f, __fsub_rn(g, mu)), den);
  return __fadd_rn(a, b);
}

// One random-number draw of the walk.  Returns the event it ended in.
template <bool ADJ>
__device__ __forceinline__ int path_step(const WalkConst& c, Path& p) {
  if (p.step >= c.max_steps) return EV_TRUNC;
  const uint4 r = philox4x32_10(make_uint4(p.step, p.path, p.inst, 0u), c.key0, c.key1);
  p.step++;
  const float u0 = u23(r.x), u1 = u23(r.y), u2 = u23(r.z), u3 = u23(r.w);

  // Exponential free flight (transmittance of the medium).
  const float s = __fmul_rn(-logf(u0), p.inv_sigt);
  // Distance to the face the path is heading to.
  float db = __int_as_float(0x7f800000);  // +inf
  const float iuz = __frcp_rn(p.uz);
  if (p.uz < 0.0f) db = __fmul_rn(-p.z, iuz);
  else if (p.uz > 0.0f) db = __fmul_rn(__fsub_rn(p.d, p.z), iuz);

  if (db <= s) {
    // Reaches the face: move onto it, then reflect or leave (Fresnel).
    p.x = __fmaf_rn(db, p.ux, p.x);
    p.y = __fmaf_rn(db, p.uy, p.y);
    const bool top = p.uz < 0.0f;
    p.z = top ? 0.0f : p.d;
    if (ADJ) p.L = __fadd_rn(p.L, db);
    const float F = fresnel(fabsf(p.uz), c.n_rel);
    if (u1 < F) {
      p.uz = -p.uz;
      return EV_CONTINUE;
    }
    if (!top) return EV_BOTTOM;
    const float rr = __fsqrt_rn(__fmaf_rn(p.x, p.x, __fmul_rn(p.y, p.y)));
    const float fb = fminf(floorf(__fmul_rn(rr, c.bin_scale)), (float)c.nbins);
    p.bin = (int)fb;
    return EV_TOP;
  }

  // Collision inside the medium.
  p.x = __fmaf_rn(s, p.ux, p.x);
  p.y = __fmaf_rn(s, p.uy, p.y);
  p.z = __fmaf_rn(s, p.uz, p.z);
  if (ADJ) p.L = __fadd_rn(p.L, s);
  p.n_coll++;
  if (c.mode == 0) {
    p.Aacc = __fmaf_rn(p.W, __fsub_rn(1.0f, p.alpha), p.Aacc);
    p.W = __fmul_rn(p.W, p.alpha);
    if (p.W < c.rr_th) {
      if (u3 < __fmul_rn(p.W, c.inv_rr_th)) p.W = c.rr_th;
      else return EV_DEAD;
    }
  } else {
    if (u3 >= p.alpha) {
      p.Aacc = __fadd_rn(p.Aacc, p.W);
      return EV_DEAD;
    }
  }

  // Henyey-Greenstein scattering with this medium's g.
  const float mu = hg_mu(p.g, u1);
  if (ADJ) p.G = __fadd_rn(p.G, hg_dlogp_dg(p.g, mu));
  // Azimuth phi = 2 pi u2; evaluated as phi - pi in (-pi, pi), then negated.
  float sp, cp;
  __sincosf(__fmul_rn(6.2831853071795865f, __fsub_rn(u2, 0.5f)), &sp, &cp);
  sp = -sp;
  cp = -cp;
  const float st = __fsqrt_rn(fmaxf(0.0f, __fmaf_rn(-mu, mu, 1.0f)));
  float nx, ny, nz;
  if (fabsf(p.uz) > 0.999999f) {
    nx = __fmul_rn(st, cp);
    ny = __fmul_rn(st, sp);
    nz = p.uz >= 0.0f ? mu : -mu;
  } else {
    const float s2 = __fmaf_rn(-p.uz, p.uz, 1.0f);
    const float itmp = rsqrtf(s2);
    const float tmp = __fmul_rn(s2, itmp);
    const float sti = __fmul_rn(st, itmp);
    const float uzcp = __fmul_rn(p.uz, cp);
    nx = __fmaf_rn(sti, __fmaf_rn(p.ux, uzcp, -__fmul_rn(p.uy, sp)), __fmul_rn(p.ux, mu));
    ny = __fmaf_rn(sti, __fmaf_rn(p.uy, uzcp, __fmul_rn(p.ux, sp)), __fmul_rn(p.uy, mu));
    nz = __fmaf_rn(-__fmul_rn(st, cp), tmp, __fmul_rn(p.uz, mu));
  }
  const float inr = rsqrtf(__fmaf_rn(nx, nx, __fmaf_rn(ny, ny, __fmul_rn(nz, nz))));
  p.ux = __fmul_rn(nx, inr);
  p.uy = __fmul_rn(ny, inr);
  p.uz = __fmul_rn(nz, inr);
  return EV_CONTINUE;
}

}  // namespace sss
