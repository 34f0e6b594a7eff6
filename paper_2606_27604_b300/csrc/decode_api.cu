// decode_api.cu -- C ABI of the decoder (sss_decoder_pack, sss_decode).
//
// Host side only: packed-weight and workspace layouts, TMA tensor maps and
// the launch sequence.  The arithmetic runs in decode.cu's kernels.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/sss.h"
#include "decode_kernels.cuh"
#include "last_status.cuh"

using namespace sss::dec;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// The ten layers in the order of sss_decoder_weights.
struct LayerSpec {
  int src_rows, src_cols;   // natural [out][in]
  int rows, cols;           // packed (padded) [N][K]
  int map;                  // PACK_*
};
constexpr LayerSpec kLayers[10] = {
    {256, 3, 256, 3, PACK_PLAIN},         // enc0 (CUDA cores)
    {256, 256, 256, 256, PACK_PLAIN},     // enc1
    {5, 256, 16, 256, PACK_PLAIN},        // enc2
    {512, 5, 512, 64, PACK_PLAIN},        // dec_r0 (reads p from the Dec_T input)
    {512, 512, 512, 512, PACK_PLAIN},     // dec_r1
    {376, 512, 384, 512, PACK_PLAIN},     // dec_r2
    {768, 381, 768, 384, PACK_DECT_IN},   // dec_t0: columns reordered to [R_d, p]
    {768, 768, 768, 768, PACK_PLAIN},     // dec_t1
    {768, 768, 768, 768, PACK_PLAIN},     // dec_t2
    {4512, 768, kFinalRows, 768, PACK_DECT_OUT},  // dec_t3: grouped rows
};

struct PackedLayout {
  size_t w[10], b[10], total;
};

PackedLayout packed_layout() {
  PackedLayout L{};
  size_t off = 0;
  for (int i = 0; i < 10; ++i) {
    L.w[i] = off;
    off += align_up((size_t)kLayers[i].rows * kLayers[i].cols * 2);
    L.b[i] = off;
    off += align_up((size_t)kLayers[i].rows * 4);
  }
  L.total = off;
  return L;
}

// Activation buffers (bf16, row-major [T][cols]).
enum { BUF_R1, BUF_R2, BUF_T, BUF_A, BUF_B, NBUF };
constexpr int kBufCols[NBUF] = {512, 512, 384, 768, 768};

struct WsLayout {
  size_t header, buf[NBUF], total;
};

WsLayout ws_layout(int64_t T) {
  WsLayout L{};
  size_t off = 0;
  L.header = off;
  off += kAlign;
  for (int i = 0; i < NBUF; ++i) {
    L.buf[i] = off;
    off += align_up((size_t)T * kBufCols[i] * 2);
  }
  L.total = off;
  return L;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2-D bf16 tensor map over [rows][cols] with a row pitch of `pitch` elements
// (0: cols), box 64 x box_rows, 128-byte swizzle; loads outside the tensor
// return zeros and stores outside it write nothing.
bool make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows,
              uint64_t pitch = 0) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {(pitch ? pitch : cols) * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool device_is_sm103() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
    return false;
  return major == 10 && minor == 3;
}

}  // namespace

extern "C" {

size_t sss_decoder_packed_size(void) { return packed_layout().total; }

size_t sss_decode_workspace_size(int64_t T) {
  if (T < 0) return 0;
  return ws_layout(T).total;
}

sss_status sss_decoder_pack(const sss_decoder_weights* w, void* packed, size_t packed_bytes,
                            sss_stream_t stream) {
  if (!w || !packed || (reinterpret_cast<uintptr_t>(packed) & (kAlign - 1)))
    return SSS_ERR_INVALID_ARG;
  for (int i = 0; i < 10; ++i)
    if (!w->W[i] || !w->b[i]) return SSS_ERR_INVALID_ARG;
  const PackedLayout L = packed_layout();
  if (packed_bytes < L.total) return SSS_ERR_WORKSPACE;
  if (!device_is_sm103()) return SSS_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(packed);
  for (int i = 0; i < 10; ++i) {
    const LayerSpec& s = kLayers[i];
    if (launch_pack(reinterpret_cast<const __nv_bfloat16*>(w->W[i]), s.src_rows, s.src_cols,
                    reinterpret_cast<__nv_bfloat16*>(base + L.w[i]), s.rows, s.cols, s.map,
                    w->b[i], reinterpret_cast<float*>(base + L.b[i]), st) != cudaSuccess)
      return SSS_ERR_CUDA;
  }
  return SSS_OK;
}

sss_status sss_selftest_bounded_wait(uint32_t* status, int64_t limit_cycles,
                                     sss_stream_t stream) {
  if (!status || (reinterpret_cast<uintptr_t>(status) & 3u) || limit_cycles < 1 ||
      limit_cycles > 4000000000LL)
    return SSS_ERR_INVALID_ARG;
  cudaGetLastError();
  return launch_bounded_wait_selftest(reinterpret_cast<unsigned int*>(status), limit_cycles,
                                      static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? SSS_OK
             : SSS_ERR_CUDA;
}

static sss_status decode_impl(const float* rgb, int64_t T, const void* packed, void* workspace,
                              size_t workspace_bytes, float* alpha, float* g, float* sigma_t,
                              float* w, sss_stream_t stream);

sss_status sss_decode(const float* rgb, int64_t T, const void* packed, void* workspace,
                      size_t workspace_bytes, float* alpha, float* g, float* sigma_t, float* w,
                      sss_stream_t stream) {
  const sss_status r =
      decode_impl(rgb, T, packed, workspace, workspace_bytes, alpha, g, sigma_t, w, stream);
  if (r == SSS_OK) sss::note_last_workspace(static_cast<cudaStream_t>(stream), workspace);
  return r;
}

static sss_status decode_impl(const float* rgb, int64_t T, const void* packed, void* workspace,
                              size_t workspace_bytes, float* alpha, float* g, float* sigma_t,
                              float* w, sss_stream_t stream) {
  if (T < 0 || T > ((int64_t)1 << 31) || !packed || !workspace) return SSS_ERR_INVALID_ARG;
  if (T > 0 && (!rgb || !alpha || !g || !sigma_t || !w)) return SSS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1)) ||
      (reinterpret_cast<uintptr_t>(packed) & (kAlign - 1)))
    return SSS_ERR_INVALID_ARG;
  const WsLayout WL = ws_layout(T);
  if (workspace_bytes < WL.total) return SSS_ERR_WORKSPACE;
  if (!device_is_sm103()) return SSS_ERR_UNSUPPORTED;
  if (!encode_fn()) return SSS_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  unsigned int* status = reinterpret_cast<unsigned int*>(ws + WL.header);
  if (cudaMemsetAsync(status, 0, kAlign, st) != cudaSuccess) return SSS_ERR_CUDA;
  if (T == 0) return SSS_OK;
  const PackedLayout PL = packed_layout();
  const char* pk = static_cast<const char*>(packed);
  auto W = [&](int i) { return reinterpret_cast<const __nv_bfloat16*>(pk + PL.w[i]); };
  auto B = [&](int i) { return reinterpret_cast<const float*>(pk + PL.b[i]); };
  __nv_bfloat16* buf[NBUF];
  for (int i = 0; i < NBUF; ++i) buf[i] = reinterpret_cast<__nv_bfloat16*>(ws + WL.buf[i]);
  // The encoder's two hidden layers use the Dec_R buffers (dead until then).
  __nv_bfloat16* X0 = buf[BUF_R1];
  __nv_bfloat16* X1 = buf[BUF_R2];
  // Columns 381..383 of the Dec_T input are padding and must read as zero.
  if (cudaMemset2DAsync(buf[BUF_T] + 376, 384 * 2, 0, 8 * 2, (size_t)T, st) != cudaSuccess)
    return SSS_ERR_CUDA;
  if (launch_enc0(rgb, T, W(0), B(0), X0, st) != cudaSuccess) return SSS_ERR_CUDA;

  const long long mt = (T + 127) / 128;
  struct Step {
    const __nv_bfloat16* a; int a_cols; int a_x0; int layer; int bn; int epi;
    __nv_bfloat16* out; int ldc; int col0; int n_valid; int act;
  };
  // enc1..dec_t2: hidden layers; dec_t3: the parameter epilogue.
  // X0 is [T][256] in BUF_R1 (row pitch 256), X1 likewise in BUF_R2.
  const Step steps[9] = {
      {X0, 256, 0, 1, 256, EPI_HIDDEN, X1, 256, 0, 256, ACT_TANH},
      {X1, 256, 0, 2, 16, EPI_HIDDEN, buf[BUF_T], 384, 376, 5, ACT_SIGMOID},
      {buf[BUF_T], 384, 376, 3, 256, EPI_HIDDEN, buf[BUF_R1], 512, 0, 512, ACT_TANH},
      {buf[BUF_R1], 512, 0, 4, 256, EPI_HIDDEN, buf[BUF_R2], 512, 0, 512, ACT_TANH},
      {buf[BUF_R2], 512, 0, 5, 192, EPI_HIDDEN, buf[BUF_T], 384, 0, 376, ACT_SIGMOID},
      {buf[BUF_T], 384, 0, 6, 256, EPI_HIDDEN, buf[BUF_A], 768, 0, 768, ACT_TANH},
      {buf[BUF_A], 768, 0, 7, 256, EPI_HIDDEN, buf[BUF_B], 768, 0, 768, ACT_TANH},
      {buf[BUF_B], 768, 0, 8, 256, EPI_HIDDEN, buf[BUF_A], 768, 0, 768, ACT_TANH},
      {buf[BUF_A], 768, 0, 9, kFinalBN, EPI_FINAL, nullptr, 0, 0, 0, ACT_NONE},
  };
  for (const Step& s : steps) {
    const LayerSpec& L = kLayers[s.layer];
    CUtensorMap ta, tb, tc;
    if (!make_map(&ta, s.a, (uint64_t)T, (uint64_t)s.a_cols, 128) ||
        !make_map(&tb, W(s.layer), (uint64_t)L.rows, (uint64_t)L.cols, (uint32_t)s.bn))
      return SSS_ERR_CUDA;
    // hidden layers with 64-column blocks store through an output map whose
    // width is the valid columns, so a ragged last block is clipped
    const bool tma_store = s.epi == EPI_HIDDEN && s.bn >= 64;
    if (tma_store) {
      if (s.col0 != 0 || !make_map(&tc, s.out, (uint64_t)T, (uint64_t)s.n_valid, 32,
                                   (uint64_t)s.ldc))
        return SSS_ERR_CUDA;
    } else {
      tc = tb;  // not read
    }
    EpiParams ep{};
    ep.out = s.out;
    ep.ldc = s.ldc;
    ep.col0 = s.col0;
    ep.n_valid = s.n_valid;
    ep.act = s.act;
    ep.alpha = alpha;
    ep.g = g;
    ep.sigma_t = sigma_t;
    ep.w = w;
    ep.T = T;
    ep.n_pairs = kPairs;
    ep.n_dst = kDstBands;
    ep.M = T;
    const int num_kb = (L.cols + 63) / 64;
    const int n_tiles = L.rows / s.bn;
    if (launch_gemm(s.bn, s.epi, ta, tb, tc, s.a_x0, num_kb, n_tiles, mt, B(s.layer), ep,
                    status, st) != cudaSuccess)
      return SSS_ERR_CUDA;
  }
  return SSS_OK;
}

}  // extern "C"
