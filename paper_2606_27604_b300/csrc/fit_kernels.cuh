// fit_kernels.cuh -- launch interface of the LUT fit (internal).
#pragma once
#include <cuda_runtime.h>

namespace sss {
namespace fit {

struct LutView {
  const float* R;  // [na][ng]
  const float* p;  // [na][ng][nb]
  int na, ng, nb;
  float a0, da, g0, dg, drho;
};

struct FitOpts {
  int K, steps;
  float lr, lambda_R;
  float a_lo, a_hi, g_lo, g_hi;
};

cudaError_t launch_lut_fit(const LutView& L, long long n_prob, const float* r, int n_r,
                           const float* Pmc, const float* Rmc, const FitOpts& o, float* raw,
                           float* loss, float* grad, cudaStream_t st);

}  // namespace fit
}  // namespace sss
