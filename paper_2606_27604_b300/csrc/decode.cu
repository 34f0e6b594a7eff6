// decode.cu -- chained decoder MLP on the 5th-generation tensor cores.
//
// RGB albedo -> Enc -> p (5) -> Dec_R -> R_d (376 bands) -> Dec_T(R_d, p)
// -> theta(lambda) = {alpha_k, g_k, sigma_t,k, w_k}, K = 3 (paper Sec. 5.1,
// Eq. 10), resampled to the 81 visible bands and written as the walk's
// structure-of-arrays parameters.
//
// Every layer but the first is one GEMM  C = act(A B^T + bias)  with BF16
// operands and FP32 accumulation:
//   * operands are staged by TMA (cp.async.bulk.tensor, 128-byte swizzle)
//     into a 4-stage shared-memory ring guarded by mbarriers;
//   * one thread issues tcgen05.mma (M = 128, N = BN, K = 16 per issue)
//     with the accumulator in tensor memory (TMEM);
//   * four epilogue warps read their 32 TMEM lanes with tcgen05.ld, add the
//     bias, apply the activation and store: BF16 activations for hidden
//     layers, or, for Dec_T's last layer, the per-band sigmoid / softmax /
//     sigma_t map and the 376 -> 81 band resampling straight into the
//     float32 parameter arrays.
// The first layer (3 inputs) is a plain CUDA-core kernel.  Every wait on an
// mbarrier gives up after about a second of clock cycles, sets a status bit
// and lets the block finish.
#include <cuda.h>  // CUtensorMap and its enums (types only; no driver calls linked)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "decode_kernels.cuh"

namespace sss {
namespace dec {

constexpr int BM = 128;
constexpr int BK = 64;        // 64 bf16 = 128 bytes = one swizzle row
constexpr int STAGES = 4;
constexpr long long kWaitCycles = 2000000000ll;  // ~1 s at 2 GHz

// ------------------------------------------------------------- PTX glue --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kWaitCycles) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Tiled TMA store of one box from shared memory (bulk-group completion).
// Elements of the box outside the tensor are not written.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(src), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the thread's committed bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// the thread's committed bulk stores have completed
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// orders this thread's shared-memory writes before later async-proxy reads
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major tile whose rows are 128 bytes,
// 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride offset between 8-row groups
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major.
template <int N>
__device__ __forceinline__ constexpr uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t addr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sigmoid_fast(float x) {
  return __fmaf_rn(0.5f, tanh_fast(0.5f * x), 0.5f);
}

// One tanh.approx per element for either activation: sigmoid(x) is taken
// as (1 + tanh(x / 2)) / 2, the same operations as sigmoid_fast.
__device__ __forceinline__ float activate(float x, int act) {
  const float t = tanh_fast(act == ACT_SIGMOID ? 0.5f * x : x);
  return act == ACT_TANH ? t : act == ACT_SIGMOID ? __fmaf_rn(0.5f, t, 0.5f) : x;
}

template <int COLS>
struct TmemCols {
  // TMEM allocations are powers of two >= 32 columns
  static constexpr int value2 = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128
                              : COLS <= 256 ? 256 : 512;
};

// ------------------------------------------------------------- epilogues --
// Hidden layer: bias, activation, BF16 store of one 16-column chunk.
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a -> low half
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void epi_hidden_chunk(const float* v, int row, int col,
                                                 const float* sbias, const EpiParams& ep) {
  if (row >= ep.M || col >= ep.n_valid) return;
  uint32_t w[8];
#pragma unroll
  for (int j = 0; j < 8; ++j)
    w[j] = pack_bf16x2(activate(v[2 * j] + sbias[col + 2 * j], ep.act),
                       activate(v[2 * j + 1] + sbias[col + 2 * j + 1], ep.act));
  __nv_bfloat16* dst = ep.out + (size_t)row * ep.ldc + ep.col0 + col;
  if (col + 16 <= ep.n_valid && ((ep.col0 + col) & 7) == 0 && (ep.ldc & 7) == 0) {
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    d4[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d4[1] = make_uint4(w[4], w[5], w[6], w[7]);
  } else {
    uint16_t* d16 = reinterpret_cast<uint16_t*>(dst);
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (col + j < ep.n_valid) d16[j] = (uint16_t)(w[j >> 1] >> ((j & 1) * 16));
  }
}

// Hidden layer, TMA-store form: one 64-column block of a warp's 32 rows.
// The BF16 results go to the warp's 4 KB staging buffer in the 128-byte
// swizzled layout of the output tensor map (row r at r * 128 bytes, 16-byte
// chunk c at position c ^ (r & 7), so the eight rows of each store phase hit
// distinct banks), and one lane issues the tensor store.  The previous block's
// store must have finished reading the buffer before it is overwritten.
__device__ __forceinline__ void epi_hidden_block_tma(const float* v, const float* __restrict__ bias,
                                                     int col, int act, uint32_t stg, int lane,
                                                     const CUtensorMap* tmap_c, int y) {
  uint32_t w[32];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float4 b0 = __ldg(reinterpret_cast<const float4*>(bias + col + c * 8));
    const float4 b1 = __ldg(reinterpret_cast<const float4*>(bias + col + c * 8 + 4));
    const float* x = v + c * 8;
    w[4 * c + 0] = pack_bf16x2(activate(x[0] + b0.x, act), activate(x[1] + b0.y, act));
    w[4 * c + 1] = pack_bf16x2(activate(x[2] + b0.z, act), activate(x[3] + b0.w, act));
    w[4 * c + 2] = pack_bf16x2(activate(x[4] + b1.x, act), activate(x[5] + b1.y, act));
    w[4 * c + 3] = pack_bf16x2(activate(x[6] + b1.z, act), activate(x[7] + b1.w, act));
  }
  if (lane == 0) bulk_wait_read_all();
  __syncwarp();
  const uint32_t row = stg + (uint32_t)lane * 128u;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    st_shared_v4(row + ((uint32_t)(c ^ (lane & 7)) << 4), w[4 * c], w[4 * c + 1], w[4 * c + 2],
                 w[4 * c + 3]);
  fence_proxy_async_smem();
  __syncwarp();
  if (lane == 0) {
    tma_store_2d(tmap_c, stg, col, y);
    bulk_commit();
  }
}

// Dec_T's last layer, one group of 36 columns = 3 source bands x (K = 3
// media x 4 channels): the source band of even visible band 2P and the two
// source bands halfway around odd visible band 2P+1.  Channels: alpha, g,
// sigma_t (sigmoid; sigma_t = 10^(3 s)), w (softmax over the media).
__device__ __forceinline__ void epi_final_group(const float* v, int row, int P,
                                                const float* bp, const EpiParams& ep) {
  if (row >= ep.M || P >= ep.n_pairs) return;
  float a[3][3], gg[3][3], st[3][3], ww[3][3];  // [slot][k]
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    float m = -3.0e38f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int c = sl * 12 + k * 4;
      a[sl][k] = sigmoid_fast(v[c + 0] + bp[c + 0]);
      gg[sl][k] = sigmoid_fast(v[c + 1] + bp[c + 1]);
      st[sl][k] = exp2f(3.0f * 3.3219280948873623f * sigmoid_fast(v[c + 2] + bp[c + 2]));
      ww[sl][k] = v[c + 3] + bp[c + 3];
      m = fmaxf(m, ww[sl][k]);
    }
    float z = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ww[sl][k] = __expf(ww[sl][k] - m);
      z += ww[sl][k];
    }
    const float iz = __fdividef(1.0f, z);
#pragma unroll
    for (int k = 0; k < 3; ++k) ww[sl][k] *= iz;
  }
  const size_t T = (size_t)ep.T;
  const size_t nin = T * (size_t)ep.n_dst;
  const int je = 2 * P;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const size_t o = (size_t)k * nin + (size_t)je * T + row;
    ep.alpha[o] = a[0][k];
    ep.g[o] = gg[0][k];
    ep.sigma_t[o] = st[0][k];
    ep.w[o] = ww[0][k];
  }
  if (je + 1 < ep.n_dst) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const size_t o = (size_t)k * nin + (size_t)(je + 1) * T + row;
      ep.alpha[o] = 0.5f * (a[1][k] + a[2][k]);
      ep.g[o] = 0.5f * (gg[1][k] + gg[2][k]);
      ep.sigma_t[o] = 0.5f * (st[1][k] + st[2][k]);
      ep.w[o] = 0.5f * (ww[1][k] + ww[2][k]);
    }
  }
}

// ------------------------------------------------------------- the GEMM --
// Persistent: one CTA per SM walks the output tiles (n fastest, so the CTAs
// working at one time share rows of A in L2).  Warp 0 streams A/B k-blocks
// through the shared-memory ring without stopping between tiles; warp 1
// issues the MMAs into one of two TMEM accumulators; warps 2..9 drain the
// other accumulator (two warps per TMEM lane quarter), so a tile's epilogue
// overlaps the next tile's MMAs.  Hidden layers with N tiles of 64 columns
// or more split the quarter's columns into whole 64-column blocks, alternating
// between its two warps, write their BF16 output with TMA tensor stores from
// a 4 KB staging buffer per epilogue warp and read the bias through the
// read-only cache; the 16-column layer (alternate 16-column chunks) and the
// last layer (alternate column groups) stage the bias in shared memory and
// store from registers.  Every CTA
// loads its own A and B tiles with its own TMA copies into its own shared
// memory.
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kStagingBytes = 4096;  // per epilogue warp: 32 rows x 64 BF16 columns

template <int BN, int EPI>
struct GemmSmem {
  static constexpr bool kTmaStore = EPI == EPI_HIDDEN && BN >= 64;
  static constexpr int kStaging = kTmaStore ? kEpiWarps * kStagingBytes : 0;
};

template <int BN, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmap_a,
                 const __grid_constant__ CUtensorMap tmap_b,
                 const __grid_constant__ CUtensorMap tmap_c, int a_x0, int num_kb,
                 int n_tiles, long long m_tiles, const float* __restrict__ bias, EpiParams ep,
                 unsigned int* status) {
  constexpr int A_BYTES = BM * BK * 2;
  constexpr int B_BYTES = BN * BK * 2;
  constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr int TCOLS = TmemCols<2 * BN>::value2;
  constexpr int ACC_STRIDE = TCOLS / 2;  // TMEM columns between the two accumulators
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
  static_assert(B_BYTES % 1024 == 0, "tiles must stay 1024-byte aligned");
  constexpr bool kTmaStore = GemmSmem<BN, EPI>::kTmaStore;
  constexpr int STAGING = GemmSmem<BN, EPI>::kStaging;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* staging = smem + STAGES * STAGE_BYTES;  // kTmaStore: 1024-byte aligned
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + STAGING);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;   // accumulator b ready for the epilogue
  uint64_t* tempty = tfull + 2;       // accumulator b drained by the epilogue
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile uint32_t* abort_flag = tmem_slot + 1;
  float* sbias = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + STAGING + 256);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const long long first = (long long)blockIdx.x;
  const long long step = (long long)gridDim.x;
  const long long total = m_tiles * (long long)n_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);  // the MMA warp's commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);  // one arrival per epilogue warp
    }
    *abort_flag = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if constexpr (!kTmaStore)
    for (int j = threadIdx.x; j < n_tiles * BN; j += blockDim.x) sbias[j] = bias[j];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_a))
                   : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_b))
                   : "memory");
      if constexpr (kTmaStore)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_c))
                     : "memory");
      long long it = 0;
      for (long long t = first; t < total && !*abort_flag; t += step) {
        const int m_tile = (int)(t / n_tiles), n_tile = (int)(t % n_tiles);
        for (int kb = 0; kb < num_kb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u)) {
            atomicOr(status, DEC_FLAG_TIMEOUT);
            *abort_flag = 1u;
            break;
          }
          mbar_expect_tx(&full[s], STAGE_BYTES);  // A tile + B tile
          uint8_t* sa = smem + s * STAGE_BYTES;
          tma_load_2d(sa, &tmap_a, a_x0 + kb * BK, m_tile * BM, &full[s]);
          tma_load_2d(sa + A_BYTES, &tmap_b, kb * BK, n_tile * BN, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16<BN>();
      long long it = 0;
      int i = 0;
      for (long long t = first; t < total && !*abort_flag; t += step, ++i) {
        const int b = i & 1;
        if (!mbar_wait(&tempty[b], ((uint32_t)(i >> 1) & 1u) ^ 1u)) {
          atomicOr(status, DEC_FLAG_TIMEOUT);
          *abort_flag = 1u;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * ACC_STRIDE);
        for (int kb = 0; kb < num_kb; ++kb, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!mbar_wait(&full[s], ph)) {
            atomicOr(status, DEC_FLAG_TIMEOUT);
            *abort_flag = 1u;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES);
          const uint64_t da = smem_desc_sw128(a0), db = smem_desc_sw128(a0 + A_BYTES);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)  // K = 16 per MMA: advance 32 bytes
            umma_bf16(acc, da + 2 * k, db + 2 * k, idesc, (kb | k) != 0);
          // frees the stage once these MMAs have read it
          umma_commit(&empty[s]);
        }
        umma_commit(&tfull[b]);    // accumulator b complete
      }
    }
  } else {
    // ---------------------------- epilogue: warps 2..9 -------------------
    const int q = warp & 3;          // TMEM lane quarter this warp may read
    const int half = (warp - 2) >> 2;  // which alternate column chunks
    int i = 0;
    for (long long t = first; t < total; t += step, ++i) {
      const int m_tile = (int)(t / n_tiles), n_tile = (int)(t % n_tiles);
      const int b = i & 1;
      const bool ok = mbar_wait(&tfull[b], (uint32_t)(i >> 1) & 1u);
      if (!ok) {
        if (lane == 0) atomicOr(status, DEC_FLAG_TIMEOUT);
        *abort_flag = 1u;
        break;
      }
      tc_fence_after();
      const int row = m_tile * BM + q * 32 + lane;
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * ACC_STRIDE);
      if constexpr (kTmaStore) {
        // read this warp's 64-column blocks of the accumulator rows, release
        // TMEM, then activate and store block by block
        constexpr int NBLK = BN / 64;
        constexpr int MYB = (NBLK + 1) / 2;
        float v[MYB * 64];
#pragma unroll
        for (int j = 0; j < MYB; ++j) {
          const int blk = 2 * j + half;
          if (blk < NBLK) {
#pragma unroll
            for (int c = 0; c < 4; ++c) tmem_ld16(taddr + blk * 64 + c * 16, v + j * 64 + c * 16);
          }
        }
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                        smem_u32(&tempty[b]))
                                    : "memory");
        const int y = m_tile * BM + q * 32;
        if (y < ep.M) {  // (a box wholly below the last row writes nothing)
#pragma unroll
          for (int j = 0; j < MYB; ++j) {
            const int blk = 2 * j + half;
            if (blk < NBLK)
              epi_hidden_block_tma(v + j * 64, bias, n_tile * BN + blk * 64, ep.act,
                                   smem_u32(staging + (warp - 2) * kStagingBytes), lane,
                                   &tmap_c, y);
          }
        }
      } else if (EPI == EPI_HIDDEN) {
        // read this warp's chunks of the accumulator row, release TMEM, then
        // finish the math and the stores
        constexpr int NCH = BN / 16;
        constexpr int MY = (NCH + 1) / 2;
        float v[MY * 16];
#pragma unroll
        for (int j = 0; j < MY; ++j) {
          const int ch = 2 * j + half;
          if (ch < NCH) tmem_ld16(taddr + ch * 16, v + j * 16);
        }
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                        smem_u32(&tempty[b]))
                                    : "memory");
#pragma unroll
        for (int j = 0; j < MY; ++j) {
          const int ch = 2 * j + half;
          if (ch < NCH) epi_hidden_chunk(v + j * 16, row, n_tile * BN + ch * 16, sbias, ep);
        }
      } else {
        for (int gq = half; gq < BN / 36; gq += 2) {
          float v[36];
          tmem_ld16(taddr + gq * 36, v);
          tmem_ld16(taddr + gq * 36 + 16, v + 16);
          tmem_ld4(taddr + gq * 36 + 32, v + 32);
          tmem_wait_ld();
          epi_final_group(v, row, n_tile * (BN / 36) + gq, sbias + n_tile * BN + gq * 36, ep);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                        smem_u32(&tempty[b]))
                                    : "memory");
      }
    }
    // the staging buffers stay allocated until the warp's stores are done
    if constexpr (kTmaStore)
      if (lane == 0) bulk_wait_all();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TCOLS)
                 : "memory");
  }
}

// --------------------------------------------- first layer (CUDA cores) --
// h = tanh(W rgb + b), W [256][3] bf16, rgb float32 [T][3] -> bf16 [T][256].
__global__ void __launch_bounds__(256)
enc0_kernel(const float* __restrict__ rgb, long long T, const __nv_bfloat16* __restrict__ W,
            const float* __restrict__ b, __nv_bfloat16* __restrict__ out) {
  // one warp per texel row, each lane 8 outputs (16-byte store); a lane
  // computes the same 8 outputs for every row, so its 32 weights and biases
  // stay in registers; a grid of a few blocks per SM strides over the rows
  const int lane = threadIdx.x & 31;
  float w0[8], w1[8], w2[8], bb[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int o = lane * 8 + e;
    w0[e] = __bfloat162float(W[o * 3 + 0]);
    w1[e] = __bfloat162float(W[o * 3 + 1]);
    w2[e] = __bfloat162float(W[o * 3 + 2]);
    bb[e] = b[o];
  }
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long rowg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; rowg < T;
       rowg += warps) {
    const float r = rgb[rowg * 3 + 0], g = rgb[rowg * 3 + 1], bl = rgb[rowg * 3 + 2];
    uint32_t h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float z2[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int i = 2 * j + e;
        z2[e] = tanh_fast(__fmaf_rn(w0[i], r, __fmaf_rn(w1[i], g, __fmaf_rn(w2[i], bl, bb[i]))));
      }
      h[j] = pack_bf16x2(z2[0], z2[1]);
    }
    reinterpret_cast<uint4*>(out + rowg * 256)[lane] = make_uint4(h[0], h[1], h[2], h[3]);
  }
}

// --------------------------------------------------------------- packing --
// dst[r][c] (bf16, rows x cols) = src[rmap(r)][cmap(c)] or 0, for the layer
// layouts the GEMMs read (padding, Dec_T input order, last-layer grouping).
__global__ void pack_weights_kernel(const __nv_bfloat16* __restrict__ src, int src_rows,
                                    int src_cols, __nv_bfloat16* __restrict__ dst, int rows,
                                    int cols, int map_kind, const float* __restrict__ bsrc,
                                    float* __restrict__ bdst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)rows * cols) return;
  const int r = (int)(i / cols), c = (int)(i % cols);
  int sr = r, sc = c;
  if (map_kind == PACK_DECT_IN) {          // GPU order [R_d(376), p(5), 0...] <- paper [p, R_d]
    sc = c < 376 ? c + 5 : (c < 381 ? c - 376 : -1);
  } else if (map_kind == PACK_DECT_OUT) {  // grouped rows of the last layer
    sr = dect_out_source_row(r);
  }
  const bool ok = sr >= 0 && sr < src_rows && sc >= 0 && sc < src_cols;
  dst[i] = ok ? src[(size_t)sr * src_cols + sc] : __float2bfloat16_rn(0.0f);
  if (c == 0 && bdst) bdst[r] = (sr >= 0 && sr < src_rows) ? bsrc[sr] : 0.0f;
}

// ------------------------------------------------ bounded-wait self-test --
// One thread waits, with the pipeline's bounded wait, for a phase of an
// mbarrier that nothing completes; when the limit runs out it records the
// timeout in the status word exactly as the GEMM roles do, and returns.
__global__ void bounded_wait_selftest_kernel(unsigned int* status, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0u, limit)) atomicOr(status, DEC_FLAG_TIMEOUT);
  }
}

cudaError_t launch_bounded_wait_selftest(unsigned int* status, long long limit, cudaStream_t st) {
  bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(status, limit);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- launch --
template <int BN, int EPI>
static cudaError_t launch_gemm_t(const CUtensorMap& ta, const CUtensorMap& tb,
                                 const CUtensorMap& tc, int a_x0, int num_kb, int n_tiles,
                                 long long m_tiles, const float* bias, const EpiParams& ep,
                                 unsigned int* status, cudaStream_t st) {
  // at least half of the SM's shared memory, so exactly one CTA (and one
  // TMEM allocation of up to 512 columns) per SM; the largest case (N = 256,
  // TMA stores) is 192 + 32 + 1.25 KB of the 227 KB a block may have
  constexpr size_t ring = (size_t)STAGES * (BM * BK * 2 + BN * BK * 2);
  constexpr size_t staging = (size_t)GemmSmem<BN, EPI>::kStaging;
  const size_t smem = (ring > 120 * 1024 ? ring : 120 * 1024) + staging + 1024 + 256 +
                      (GemmSmem<BN, EPI>::kTmaStore ? 0 : (size_t)n_tiles * BN * sizeof(float));
  auto fn = gemm_bf16_kernel<BN, EPI>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long total = (long long)n_tiles * m_tiles;
  if (total == 0) return cudaSuccess;
  // persistent: one CTA per SM (its shared memory allows no second one)
  const long long ctas = total < sms ? total : sms;
  fn<<<(unsigned)ctas, kThreads, smem, st>>>(ta, tb, tc, a_x0, num_kb, n_tiles, m_tiles, bias,
                                             ep, status);
  return cudaGetLastError();
}

cudaError_t launch_gemm(int bn, int epi, const CUtensorMap& ta, const CUtensorMap& tb,
                        const CUtensorMap& tc, int a_x0, int num_kb, int n_tiles,
                        long long m_tiles, const float* bias, const EpiParams& ep,
                        unsigned int* status, cudaStream_t st) {
#define SSS_GEMM(BN_, EPI_) \
  return launch_gemm_t<BN_, EPI_>(ta, tb, tc, a_x0, num_kb, n_tiles, m_tiles, bias, ep, status, st)
  if (epi == EPI_FINAL && bn == kFinalBN) SSS_GEMM(kFinalBN, EPI_FINAL);
  if (epi == EPI_HIDDEN) {
    switch (bn) {
      case 16: SSS_GEMM(16, EPI_HIDDEN);
      case 192: SSS_GEMM(192, EPI_HIDDEN);
      case 256: SSS_GEMM(256, EPI_HIDDEN);
    }
  }
#undef SSS_GEMM
  return cudaErrorInvalidValue;
}

cudaError_t launch_enc0(const float* rgb, long long T, const __nv_bfloat16* W, const float* b,
                        __nv_bfloat16* out, cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long need = (T * 32 + 255) / 256;
  const long long grid = need < 8LL * sms ? need : 8LL * sms;
  enc0_kernel<<<(unsigned)grid, 256, 0, st>>>(rgb, T, W, b, out);
  return cudaGetLastError();
}

cudaError_t launch_pack(const __nv_bfloat16* src, int src_rows, int src_cols, __nv_bfloat16* dst,
                        int rows, int cols, int map_kind, const float* bsrc, float* bdst,
                        cudaStream_t st) {
  const long long n = (long long)rows * cols;
  pack_weights_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, src_rows, src_cols, dst, rows,
                                                                   cols, map_kind, bsrc, bdst);
  return cudaGetLastError();
}

}  // namespace dec
}  // namespace sss
