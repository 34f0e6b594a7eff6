// probe.cu -- sss_probe: issue-rate probes for the walk's roofline.
//
// The walk is bound by per-lane arithmetic issue (FP32, INT32 and the
// special-function unit), not by memory or tensor cores, so its roofline
// denominator is a per-SM instruction throughput.  These kernels measure
// that throughput for the instruction kinds a walk step is made of, each as
// eight independent dependency chains per thread (enough instruction-level
// parallelism that issue, not latency, limits them), with the iteration
// loop unrolled eightfold so loop control costs under 5% of the issue
// slots.  SSS_PROBE_PHILOX times whole Philox4x32-10 blocks, the integer
// half of a walk step.  The paper has no counterpart; this is measurement
// infrastructure.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/sss.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) probe_ffma(int64_t iters, float b, float c,
                                                       float* sink) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
#pragma unroll 8
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = __fmaf_rn(x[i], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) probe_ffma2(int64_t iters, float b, float c,
                                                        float* sink) {
  float2 x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i)
    x[i] = make_float2((float)(threadIdx.x + i) * 1e-3f, (float)(threadIdx.x - i) * 1e-3f);
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll 8
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], bb, cc);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
  sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) probe_imad(int64_t iters, uint32_t b, uint32_t c,
                                                       float* sink) {
  uint32_t x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = threadIdx.x * 7u + (uint32_t)i;
#pragma unroll 8
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = x[i] * b + c;
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s ^= x[i];
  sink[blockIdx.x * kThreads + threadIdx.x] = (float)s;
}

__global__ void __launch_bounds__(kThreads) probe_lop3(int64_t iters, uint32_t b, uint32_t c,
                                                       float* sink) {
  uint32_t x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = threadIdx.x * 13u + (uint32_t)i;
#pragma unroll 8
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (x[i] ^ b) & (x[i] | c);  // one 3-input logic op
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s ^= x[i];
  sink[blockIdx.x * kThreads + threadIdx.x] = (float)s;
}

__global__ void __launch_bounds__(kThreads) probe_mufu(int64_t iters, float b, float c,
                                                       float* sink) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 2.0f + (float)(threadIdx.x + i) * 1e-3f;
#pragma unroll 8
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      float y;
      asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[i]));
      x[i] = y + c;  // stays in [c, c + 2]: a positive, normal operand
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  sink[blockIdx.x * kThreads + threadIdx.x] = s + b;
}

// Whole Philox4x32-10 blocks (Salmon et al., SC'11) with the round keys in
// the kernel's parameter bank, the form the walk uses: four independent
// chains per thread, each block's output the next block's counter.
struct ProbeKeys {
  uint32_t rk[20];
};
constexpr int kPhiloxChains = 4;

__global__ void __launch_bounds__(kThreads) probe_philox(int64_t iters, ProbeKeys k,
                                                         float* sink) {
  uint4 x[kPhiloxChains];
#pragma unroll
  for (int i = 0; i < kPhiloxChains; ++i)
    x[i] = make_uint4(threadIdx.x, blockIdx.x, (uint32_t)i, 0u);
#pragma unroll 2
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kPhiloxChains; ++i) {
      uint4 c = x[i];
#pragma unroll
      for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53ull;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57ull;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.rk[2 * r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ k.rk[2 * r + 1], (uint32_t)p0);
      }
      x[i] = c;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kPhiloxChains; ++i) s ^= x[i].x ^ x[i].y ^ x[i].z ^ x[i].w;
  sink[blockIdx.x * kThreads + threadIdx.x] = (float)s;
}

}  // namespace

extern "C" {

sss_status sss_probe(int32_t kind, int64_t iters, int32_t blocks, float* sink,
                     sss_stream_t stream) {
  if (iters < 1 || blocks < 1 || !sink || kind < 0 || kind > 5) return SSS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  switch (kind) {
    case SSS_PROBE_FFMA: probe_ffma<<<blocks, kThreads, 0, st>>>(iters, 0.999f, 1e-3f, sink); break;
    case SSS_PROBE_FFMA2: probe_ffma2<<<blocks, kThreads, 0, st>>>(iters, 0.999f, 1e-3f, sink); break;
    case SSS_PROBE_IMAD: probe_imad<<<blocks, kThreads, 0, st>>>(iters, 1664525u, 1013904223u, sink); break;
    case SSS_PROBE_LOP3: probe_lop3<<<blocks, kThreads, 0, st>>>(iters, 0x9E3779B9u, 0x7F4A7C15u, sink); break;
    case SSS_PROBE_MUFU: probe_mufu<<<blocks, kThreads, 0, st>>>(iters, 0.0f, 2.0f, sink); break;
    default: {
      ProbeKeys k;
      for (int r = 0; r < 10; ++r) {  // key (0x12345678, 0x9abcdef0) and its schedule
        k.rk[2 * r] = 0x12345678u + (uint32_t)r * 0x9E3779B9u;
        k.rk[2 * r + 1] = 0x9abcdef0u + (uint32_t)r * 0xBB67AE85u;
      }
      probe_philox<<<blocks, kThreads, 0, st>>>(iters, k, sink);
      break;
    }
  }
  return cudaGetLastError() == cudaSuccess ? SSS_OK : SSS_ERR_CUDA;
}

int64_t sss_probe_ops_per_thread_iter(int32_t kind) {
  // (two lane ops per paired FMA; whole blocks for Philox)
  return kind == SSS_PROBE_FFMA2 ? 2 * kChains
                                 : (kind == SSS_PROBE_PHILOX ? kPhiloxChains : kChains);
}

}  // extern "C"
