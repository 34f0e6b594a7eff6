// fit.cu -- batched LUT-based fit of K-media mixtures (paper Sec. 4.2).
//
// One warp per (tone, wavelength) problem.  Each Adam step evaluates
//   R_hat    = sum_k w_k R(alpha_k, g_k)                      (bilinear)
//   P_hat(r) = sum_k w_k sigma_k^2 p(sigma_k r | alpha_k, g_k) (trilinear, Eq. 5)
//   L = RMSE_j(log P_hat(r_j), log P_MC(r_j)) + lambda_R (R_hat - R_MC)^2
// (Eq. 6-9) over the radii with P_MC > 0, and its exact gradient through the
// piecewise-linear interpolation; lanes own radii, the per-medium gradient
// sums are reduced with warp shuffles, and every lane keeps the same copy of
// the 4K raw parameters.  Parameterisation: alpha and g squashed by a
// sigmoid into their table ranges, sigma_t = exp(raw), w = softmax(raw).
// Adam (0.9, 0.999, 1e-8) with lr_t = lr (1 + cos(pi t / S)) / 2.
#include <cuda_runtime.h>

#include <cstdint>

#include "fit_kernels.cuh"

namespace sss {
namespace fit {

constexpr unsigned kFull = 0xffffffffu;

struct Cell {
  int i;
  float f;
  bool inside;
};

__device__ __forceinline__ Cell cell(float x, float x0, float dx, int n) {
  const float u = (x - x0) / dx;
  Cell c;
  c.i = min(max((int)floorf(u), 0), n - 2);
  c.f = fminf(fmaxf(u - (float)c.i, 0.0f), 1.0f);
  c.inside = u >= 0.0f && u <= (float)(n - 1);
  return c;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Loss and gradient of one problem at raw parameters th[4K]; every lane
// returns the same values.  K is a template parameter so every per-medium
// array stays in registers.
template <int K>
__device__ float loss_grad(const LutView& L, const float* th, const float* r, int n_r,
                           const float* Pmc, float Rmc, float inv_n, const FitOpts& o,
                           float* grad, int lane) {
  float alpha[K], g[K], sig[K], w[K], sa[K], sg[K];
  float wmax = -3.0e38f;
#pragma unroll
  for (int k = 0; k < K; ++k) wmax = fmaxf(wmax, th[3 * K + k]);
  float wz = 0.0f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    sa[k] = 1.0f / (1.0f + __expf(-th[k]));
    sg[k] = 1.0f / (1.0f + __expf(-th[K + k]));
    alpha[k] = o.a_lo + (o.a_hi - o.a_lo) * sa[k];
    g[k] = o.g_lo + (o.g_hi - o.g_lo) * sg[k];
    sig[k] = __expf(th[2 * K + k]);
    w[k] = __expf(th[3 * K + k] - wmax);
    wz += w[k];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] /= wz;

  // R_hat and its partials (every lane, redundant)
  float Rk[K], dRa[K], dRg[K], Rhat = 0.0f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const Cell ca = cell(alpha[k], L.a0, L.da, L.na), cg = cell(g[k], L.g0, L.dg, L.ng);
    const float* R0 = L.R + (size_t)ca.i * L.ng + cg.i;
    const float c00 = R0[0], c01 = R0[1], c10 = R0[L.ng], c11 = R0[L.ng + 1];
    Rk[k] = (1 - ca.f) * (1 - cg.f) * c00 + ca.f * (1 - cg.f) * c10 + (1 - ca.f) * cg.f * c01 +
            ca.f * cg.f * c11;
    dRa[k] = ca.inside ? ((c10 - c00) * (1 - cg.f) + (c11 - c01) * cg.f) / L.da : 0.0f;
    dRg[k] = cg.inside ? ((c01 - c00) * (1 - ca.f) + (c11 - c10) * ca.f) / L.dg : 0.0f;
    Rhat += w[k] * Rk[k];
  }

  // profile terms for this lane's radii
  float Pk[2][K], dPa[2][K], dPg[2][K], dPs[2][K], e[2], Ph[2];
  bool valid[2];
  float se2 = 0.0f;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int t = lane + 32 * q;
    valid[q] = t < n_r && Pmc[t] > 0.0f;
    Ph[q] = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      Pk[q][k] = dPa[q][k] = dPg[q][k] = dPs[q][k] = 0.0f;
      if (!valid[q]) continue;
      const float rho = sig[k] * r[t];
      const Cell ca = cell(alpha[k], L.a0, L.da, L.na), cg = cell(g[k], L.g0, L.dg, L.ng);
      const Cell cb = cell(rho, 0.5f * L.drho, L.drho, L.nb);
      const float* base = L.p + ((size_t)ca.i * L.ng + cg.i) * L.nb + cb.i;
      const size_t sa_ = (size_t)L.ng * L.nb, sg_ = (size_t)L.nb;
      float c[2][2][2];
#pragma unroll
      for (int ia = 0; ia < 2; ++ia)
#pragma unroll
        for (int ig = 0; ig < 2; ++ig)
#pragma unroll
          for (int ib = 0; ib < 2; ++ib) c[ia][ig][ib] = base[ia * sa_ + ig * sg_ + ib];
      const float wa[2] = {1 - ca.f, ca.f}, wg[2] = {1 - cg.f, cg.f}, wb[2] = {1 - cb.f, cb.f};
      float v = 0.0f, va = 0.0f, vg = 0.0f, vb = 0.0f;
#pragma unroll
      for (int ia = 0; ia < 2; ++ia)
#pragma unroll
        for (int ig = 0; ig < 2; ++ig)
#pragma unroll
          for (int ib = 0; ib < 2; ++ib) v += wa[ia] * wg[ig] * wb[ib] * c[ia][ig][ib];
#pragma unroll
      for (int ig = 0; ig < 2; ++ig)
#pragma unroll
        for (int ib = 0; ib < 2; ++ib) va += wg[ig] * wb[ib] * (c[1][ig][ib] - c[0][ig][ib]);
#pragma unroll
      for (int ia = 0; ia < 2; ++ia)
#pragma unroll
        for (int ib = 0; ib < 2; ++ib) vg += wa[ia] * wb[ib] * (c[ia][1][ib] - c[ia][0][ib]);
#pragma unroll
      for (int ia = 0; ia < 2; ++ia)
#pragma unroll
        for (int ig = 0; ig < 2; ++ig) vb += wa[ia] * wg[ig] * (c[ia][ig][1] - c[ia][ig][0]);
      va = ca.inside ? va / L.da : 0.0f;
      vg = cg.inside ? vg / L.dg : 0.0f;
      vb = cb.inside ? vb / L.drho : 0.0f;
      const float s2 = sig[k] * sig[k];
      Pk[q][k] = s2 * v;
      dPa[q][k] = s2 * va;
      dPg[q][k] = s2 * vg;
      dPs[q][k] = 2.0f * sig[k] * v + s2 * r[t] * vb;
      Ph[q] += w[k] * Pk[q][k];
    }
    e[q] = valid[q] ? __logf(Ph[q]) - __logf(Pmc[t]) : 0.0f;
    se2 += e[q] * e[q];
  }
  const float Ls = sqrtf(warp_sum(se2) * inv_n);
  const float dR = Rhat - Rmc;
  const float loss = Ls + o.lambda_R * dR * dR;
  const float gR = 2.0f * o.lambda_R * dR;

  // per-medium sums over radii
  float sa_sum[K], sg_sum[K], ss_sum[K], sw_sum[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float a = 0.0f, b = 0.0f, s = 0.0f, ww = 0.0f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!valid[q] || Ls <= 0.0f) continue;
      const float gP = e[q] * inv_n / (Ls * Ph[q]);
      a += dPa[q][k] * gP;
      b += dPg[q][k] * gP;
      s += dPs[q][k] * gP;
      ww += Pk[q][k] * gP;
    }
    sa_sum[k] = warp_sum(a);
    sg_sum[k] = warp_sum(b);
    ss_sum[k] = warp_sum(s);
    sw_sum[k] = warp_sum(ww);
  }
  float dw[K], wdw = 0.0f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float d_alpha = w[k] * (sa_sum[k] + gR * dRa[k]);
    const float d_g = w[k] * (sg_sum[k] + gR * dRg[k]);
    const float d_sig = w[k] * ss_sum[k];
    dw[k] = sw_sum[k] + gR * Rk[k];
    wdw += w[k] * dw[k];
    grad[k] = d_alpha * (o.a_hi - o.a_lo) * sa[k] * (1.0f - sa[k]);
    grad[K + k] = d_g * (o.g_hi - o.g_lo) * sg[k] * (1.0f - sg[k]);
    grad[2 * K + k] = d_sig * sig[k];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) grad[3 * K + k] = w[k] * (dw[k] - wdw);
  return loss;
}

template <int K>
__global__ void __launch_bounds__(128)
lut_fit_kernel(LutView L, long long n_prob, const float* __restrict__ r, int n_r,
               const float* __restrict__ Pmc, const float* __restrict__ Rmc, FitOpts o,
               float* __restrict__ raw, float* __restrict__ loss_out,
               float* __restrict__ grad_out) {
  const long long prob = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (prob >= n_prob) return;  // whole warp leaves together
  constexpr int np = 4 * K;
  const float* P = Pmc + (size_t)prob * n_r;
  int nv = 0;
  for (int t = lane; t < n_r; t += 32) nv += P[t] > 0.0f ? 1 : 0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nv += __shfl_xor_sync(kFull, nv, off);
  const float inv_n = nv > 0 ? 1.0f / (float)nv : 0.0f;
  float th[np], m[np], v[np], gr[np];
#pragma unroll
  for (int j = 0; j < np; ++j) {
    th[j] = raw[(size_t)prob * np + j];
    m[j] = 0.0f;
    v[j] = 0.0f;
  }
  const float Rt = Rmc[prob];
  float b1t = 1.0f, b2t = 1.0f;
  for (int t = 1; t <= o.steps; ++t) {
    loss_grad<K>(L, th, r, n_r, P, Rt, inv_n, o, gr, lane);
    b1t *= 0.9f;
    b2t *= 0.999f;
    const float lr_t = o.lr * 0.5f * (1.0f + cospif((float)(t - 1) / (float)o.steps));
#pragma unroll
    for (int j = 0; j < np; ++j) {
      m[j] = 0.9f * m[j] + 0.1f * gr[j];
      v[j] = 0.999f * v[j] + 0.001f * gr[j] * gr[j];
      const float mh = m[j] / (1.0f - b1t), vh = v[j] / (1.0f - b2t);
      th[j] -= lr_t * mh / (sqrtf(vh) + 1e-8f);
    }
  }
  const float L_final = loss_grad<K>(L, th, r, n_r, P, Rt, inv_n, o, gr, lane);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < np; ++j) raw[(size_t)prob * np + j] = th[j];
    if (loss_out) loss_out[prob] = L_final;
    if (grad_out) {
#pragma unroll
      for (int j = 0; j < np; ++j) grad_out[(size_t)prob * np + j] = gr[j];
    }
  }
}

cudaError_t launch_lut_fit(const LutView& L, long long n_prob, const float* r, int n_r,
                           const float* Pmc, const float* Rmc, const FitOpts& o, float* raw,
                           float* loss, float* grad, cudaStream_t st) {
  if (n_prob <= 0) return cudaSuccess;
  const long long threads = n_prob * 32;
  const unsigned grid = (unsigned)((threads + 127) / 128);
  switch (o.K) {
    case 1: lut_fit_kernel<1><<<grid, 128, 0, st>>>(L, n_prob, r, n_r, Pmc, Rmc, o, raw, loss, grad); break;
    case 2: lut_fit_kernel<2><<<grid, 128, 0, st>>>(L, n_prob, r, n_r, Pmc, Rmc, o, raw, loss, grad); break;
    case 3: lut_fit_kernel<3><<<grid, 128, 0, st>>>(L, n_prob, r, n_r, Pmc, Rmc, o, raw, loss, grad); break;
    case 4: lut_fit_kernel<4><<<grid, 128, 0, st>>>(L, n_prob, r, n_r, Pmc, Rmc, o, raw, loss, grad); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fit
}  // namespace sss

// ------------------------------------------------------------------ C ABI --
#include "../../include/sss.h"

extern "C" sss_status sss_lut_fit(const sss_lut* lut, int64_t n_prob, const float* r_mm,
                                  int32_t n_r, const float* P_mc, const float* R_mc,
                                  const sss_fit_opts* o, float* raw, float* loss, float* grad,
                                  sss_stream_t stream) {
  if (!lut || !o || n_prob < 0) return SSS_ERR_INVALID_ARG;
  if (lut->na < 2 || lut->ng < 2 || lut->nb < 2 || !lut->R || !lut->p) return SSS_ERR_INVALID_ARG;
  if (!(lut->da > 0.0f) || !(lut->dg > 0.0f) || !(lut->drho > 0.0f)) return SSS_ERR_INVALID_ARG;
  if (o->K < 1 || o->K > 4 || o->steps < 0 || n_r < 1 || n_r > 64) return SSS_ERR_INVALID_ARG;
  if (n_prob > 0 && (!r_mm || !P_mc || !R_mc || !raw)) return SSS_ERR_INVALID_ARG;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      !(major == 10 && minor == 3))
    return SSS_ERR_UNSUPPORTED;
  sss::fit::LutView L{lut->R, lut->p, lut->na, lut->ng, lut->nb,
                      lut->a0, lut->da, lut->g0, lut->dg, lut->drho};
  sss::fit::FitOpts fo{o->K, o->steps, o->lr, o->lambda_R, o->a_lo, o->a_hi, o->g_lo, o->g_hi};
  cudaGetLastError();
  return sss::fit::launch_lut_fit(L, n_prob, r_mm, n_r, P_mc, R_mc, fo, raw, loss, grad,
                                  static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? SSS_OK
             : SSS_ERR_CUDA;
}
