// hero.cuh -- hero-wavelength path sharing for the persistent walk kernel.
//
// Hero-wavelength spectral sampling (Wilkie et al., EGSR 2014; the paper's
// related work names hero-wavelength tracking among production random-walk
// techniques), applied to the mixture walk.  The bands of a texel form
// groups of C; path p of a group samples everything (medium choice, flights,
// Henyey-Greenstein cosines, roulette) with the optics of its hero member
// p mod C, and every member j scores the one-sample balance-heuristic
// estimate C f_j / sum_i p_i.  p_i is the density of the path's sampling
// decisions under member i's optics (selection probability, sigma exp(-sigma
// s) per collision or exp(-sigma s) per face flight, p_HG(mu) per
// scattering; the Fresnel choices are the same for every member and cancel),
// and f_j / p_j is member j's albedo-weighted weight.  The per-step part
// lives in path_step<..., HERO> (walk_core.cuh); this file holds the group
// layout, the start of a path and the exit tally.
#pragma once
#include <cstdint>

#include "walk_core.cuh"
#include "walk_kernels.cuh"

namespace sss {

// Members of hero group g: member j is first + j * stride, with groups as
// blocks of C adjacent bands of a texel, or the rotation orbits
// {q, q + nb/C, ...} (hero_orbits = 1).
struct HeroGroup {
  uint32_t first, stride;
};

template <int C>
__device__ __forceinline__ HeroGroup hero_group(const WalkConst& c, uint32_t g) {
  const uint32_t per = (uint32_t)c.hero_nb / C;  // groups per texel
  const uint32_t t = g / per, q = g - t * per;
  HeroGroup r;
  r.first = t * (uint32_t)c.hero_nb + (c.hero_orbits ? q : q * C);
  r.stride = c.hero_orbits ? per : 1u;
  return r;
}

// log2 sigma_t, log2(1 - g^2) and log2 of the mixture weight w_k / sum(w),
// for every (medium, instance): the constant parts of the members' density
// ratios, computed once per call instead of once per path.
__global__ void hero_logs_kernel(WalkConst c, float* logs) {
  const size_t n = c.n_inst, Kn = (size_t)c.K * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < Kn;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t i = idx % n;
    const float g = c.g[idx];
    float tot = 0.0f;
    for (int j = 0; j < c.K; ++j) tot = __fadd_rn(tot, c.w[(size_t)j * n + i]);
    logs[idx] = log2f(c.sigma_t[idx]);
    logs[Kn + idx] = log2f(__fmaf_rn(-g, g, 1.0f));
    logs[2 * Kn + idx] = log2f(__fdiv_rn(c.w[idx], tot));
  }
}

// Starts path `path` of hero group g: the hero member h = path mod C samples
// everything (path_init with its optics, under the counters of the group's
// first member); each other member starts with its weight (entry weight, or
// entry weight x K w_k / sum(w) under uniform selection) and the log2 ratio
// of its selection probability to the hero's.
template <int C>
__device__ __forceinline__ void hero_init(const WalkConst& c, uint32_t g, uint32_t path, float d,
                                          Path& p, HeroState<C>& hs) {
  const HeroGroup G = hero_group<C>(c, g);
  const int h = (int)(path % C);
  const uint32_t mh = G.first + (uint32_t)h * G.stride;
  path_init<false, false>(c, mh, path, d, p, G.first + c.inst_offset);
  hs.h = h;
  p.inst = g;
  const size_t Kn = (size_t)c.K * c.n_inst;
  const size_t ok = (size_t)p.k * c.n_inst;
  const float* lsig = c.hero_logs;
  const float* lg = c.hero_logs + Kn;
  const float* lmix = c.hero_logs + 2 * Kn;
  const float s_h = p.sigt, lsh = __ldg(lsig + ok + mh), lgh = __ldg(lg + ok + mh),
              lmh = __ldg(lmix + ok + mh);
  // the entry weight before the selection factor, as path_init forms it
  const float E = c.incidence == 1
                      ? (c.entry_fresnel ? __fsub_rn(1.0f, fresnel(p.uz, c.n_rel)) : 1.0f)
                      : c.W0;
#pragma unroll
  for (int m = 0; m < C - 1; ++m) {
    const uint32_t mj = G.first + (uint32_t)((h + 1 + m) % C) * G.stride;
    if (c.select_uniform) {
      // equal selection probabilities; weight E K w_k / sum(w) as path_init
      float tot = 0.0f;
      for (int j = 0; j < c.K; ++j) tot = __fadd_rn(tot, __ldg(c.w + (size_t)j * c.n_inst + mj));
      hs.W[m] = __fmul_rn(E, __fmul_rn(__fmul_rn((float)c.K, __ldg(c.w + ok + mj)),
                                       __fdiv_rn(1.0f, tot)));
      hs.D[m] = 0.0f;
    } else {
      // selection probability = mixture weight; weight E
      hs.W[m] = E;
      hs.D[m] = __fsub_rn(__ldg(lmix + ok + mj), lmh);
    }
    const float sj = __ldg(c.sigma_t + ok + mj);
    hs.a[m] = __ldg(c.alpha + ok + mj);
    hs.ds[m] = __fmul_rn(__fsub_rn(s_h, sj), 1.4426950408889634f);
    hs.ls[m] = __fsub_rn(__ldg(lsig + ok + mj), lsh);
    hs.g[m] = __ldg(c.g + ok + mj);
    hs.cg[m] = __fsub_rn(__ldg(lg + ok + mj), lgh);
  }
}

// Hero-wavelength exit: every member j of the group scores the one-sample
// balance-heuristic estimate F_j = W_j C 2^(D_j) / sum_i 2^(D_i), with D the
// log2 path density relative to the hero (D = 0 for the hero itself).  The
// slot holds the members' accumulators one after the other (member order);
// `direct` sends them to the members' global accumulators instead.
template <int C>
__device__ __forceinline__ void tally_path_hero(const WalkConst& c, const WalkSched& s,
                                                const TallyOut& t, const Path& p,
                                                const HeroState<C>& hs, int ev,
                                                unsigned long long* m, bool direct) {
  const int nb = c.nbins, sw = s.slot_words;
  const HeroGroup G = direct ? hero_group<C>(c, p.inst) : HeroGroup{0u, 0u};
  auto add = [&](int j, int w, unsigned long long v) {
    if (!direct) add64_shared(m + j * sw + w, v);
    else atomicAdd(t.raw + (size_t)(G.first + (uint32_t)j * G.stride) * sw + w, v);
  };
  float F[C];
  if (ev == EV_TOP || ev == EV_BOTTOM) {
    float dmax = 0.0f;
#pragma unroll
    for (int r = 0; r < C - 1; ++r) dmax = fmaxf(dmax, hs.D[r]);
    float E[C];
    E[0] = exp2f(-dmax);
    float S = E[0];
#pragma unroll
    for (int r = 0; r < C - 1; ++r) {
      E[r + 1] = exp2f(__fsub_rn(hs.D[r], dmax));
      S = __fadd_rn(S, E[r + 1]);
    }
    const float scale = __fdiv_rn((float)C, S);
    F[0] = __fmul_rn(__fmul_rn(p.W, E[0]), scale);
#pragma unroll
    for (int r = 0; r < C - 1; ++r) F[r + 1] = __fmul_rn(__fmul_rn(hs.W[r], E[r + 1]), scale);
  } else {
#pragma unroll
    for (int r = 0; r < C; ++r) F[r] = 0.0f;
  }
  const int bin = ev == EV_TOP ? exit_bin(c, p) : 0;
#pragma unroll
  for (int r = 0; r < C; ++r) {
    const int j = (hs.h + r) % C;  // r = 0 is the hero
    if (ev == EV_TOP) {
      const unsigned long long q = __float2ull_rn(__fmul_rn(F[r], kFix));
      add(j, bin, q);
      add(j, nb + 1 + p.k, q);
      if (p.n_coll == 1u) add(j, nb + 1 + c.K, q);
      if (s.want_sumsq)
        add(j, nb + 6 + c.K + bin, __float2ull_rn(__fmul_rn(__fmul_rn(F[r], F[r]), kFix)));
    } else if (ev == EV_BOTTOM) {
      add(j, nb + 2 + c.K, __float2ull_rn(__fmul_rn(F[r], kFix)));
    } else if (ev == EV_TRUNC) {
      add(j, nb + 4 + c.K, 1ull);
    }
    add(j, nb + 5 + c.K, (unsigned long long)p.step);
  }
  if (ev == EV_TRUNC) atomicOr(s.status, SSS_DEV_FLAG_STEP_LIMIT);
}

}  // namespace sss
