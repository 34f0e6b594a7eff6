// decode_kernels.cuh -- launch interface of the decoder kernels (internal).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace sss {
namespace dec {

enum : int { ACT_NONE = 0, ACT_TANH = 1, ACT_SIGMOID = 2 };
enum : int { EPI_HIDDEN = 0, EPI_FINAL = 1 };
enum : int { PACK_PLAIN = 0, PACK_DECT_IN = 1, PACK_DECT_OUT = 2 };
enum : unsigned int { DEC_FLAG_TIMEOUT = 0x10u };

// Dec_T's last layer, grouped for the epilogue: 41 groups of 36 rows (the
// source band of even visible band 2P, then the two source bands around odd
// visible band 2P+1, each 12 rows = 3 media x (alpha, g, sigma_t, w)),
// packed 7 groups (252 rows + 4 padding rows) to a 256-row tile: 6 tiles,
// so each 128-row block of activations is read 6 times per layer instead of
// the 11 times of 144-row tiles.  Visible band j (380 + 5j nm) sits at
// source index 65 + 2.5 j on the 250-1000 nm, 2 nm grid.
constexpr int kDstBands = 81;
constexpr int kPairs = 41;
constexpr int kFinalBN = 256;
constexpr int kGroupsPerTile = kFinalBN / 36;                            // 7
constexpr int kFinalTiles = (kPairs + kGroupsPerTile - 1) / kGroupsPerTile;  // 6
constexpr int kFinalRows = kFinalTiles * kFinalBN;                       // 1536

__host__ __device__ inline int dect_out_source_row(int r) {
  const int tile = r / kFinalBN, in_tile = r % kFinalBN;
  if (in_tile >= kGroupsPerTile * 36) return -1;  // padding rows of a tile
  const int P = tile * kGroupsPerTile + in_tile / 36, rem = in_tile % 36;
  const int slot = rem / 12, within = rem % 12;
  if (P >= kPairs) return -1;
  const int s = 65 + 5 * P + (slot == 0 ? 0 : (slot == 1 ? 2 : 3));
  return s * 12 + within;
}

struct EpiParams {
  // hidden layers
  __nv_bfloat16* out;
  int ldc, col0, n_valid, act;
  // last layer
  float *alpha, *g, *sigma_t, *w;
  long long T;
  int n_pairs, n_dst;
  // rows of A that exist
  long long M;
};

cudaError_t launch_bounded_wait_selftest(unsigned int* status, long long limit,
                                         cudaStream_t st);
// tc: the output tensor map of hidden layers with bn >= 64 (box 64 x 32,
// 128-byte swizzle), written by TMA stores; unused otherwise.
cudaError_t launch_gemm(int bn, int epi, const CUtensorMap& ta, const CUtensorMap& tb,
                        const CUtensorMap& tc, int a_x0, int num_kb, int n_tiles,
                        long long m_tiles, const float* bias, const EpiParams& ep,
                        unsigned int* status, cudaStream_t st);
cudaError_t launch_enc0(const float* rgb, long long T, const __nv_bfloat16* W, const float* b,
                        __nv_bfloat16* out, cudaStream_t st);
cudaError_t launch_pack(const __nv_bfloat16* src, int src_rows, int src_cols, __nv_bfloat16* dst,
                        int rows, int cols, int map_kind, const float* bsrc, float* bdst,
                        cudaStream_t st);

}  // namespace dec
}  // namespace sss
