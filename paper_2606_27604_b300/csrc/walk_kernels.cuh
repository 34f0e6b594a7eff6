// walk_kernels.cuh -- host-visible launch interface of the walk kernels
// (internal to libsss; the public C ABI is include/sss.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "walk_core.cuh"

namespace sss {

// Device status-word bits; equal to SSS_FLAG_* of the public header.
enum : unsigned int {
  SSS_DEV_FLAG_PARAM = 0x1u,
  SSS_DEV_FLAG_STEP_LIMIT = 0x2u,
  SSS_DEV_FLAG_OVERFLOW = 0x4u,
  SSS_DEV_FLAG_ZERO_WEIGHT = 0x8u,
};

// Tallies are fixed point: an exit weight W adds round(W 2^32) to a uint64
// word, so sums do not depend on the order of the atomics.
constexpr float kFix = 4294967296.0f;  // 2^32
constexpr double kInvFix = 1.0 / 4294967296.0;

// Media per mixture the kernels support (SSS_KMAX of the public header).
constexpr int kKMax = 4;

// Bytes of the per-slot header (SlotMeta, with the unit's staged media)
// after a warp's two slots of shared accumulators, and of the per-warp
// buffer of medium choices (SelBuf) after the headers.
constexpr int kSlotMetaBytes = 208;
constexpr int kSelBufBytes = 176;

// 64-bit shared-memory accumulation from native 32-bit atomics: the low
// word's atomic returns its old value, so each adder sees whether its own
// addition wrapped and carries it into the high word.  The 64-bit sum of a
// word is exact once the adders are done (only the warp that owns the slot
// touches it, and it reads the pair back after a __syncwarp).
__device__ __forceinline__ void add64_shared(unsigned long long* a, unsigned long long v) {
  uint32_t* w = reinterpret_cast<uint32_t*>(a);
  const uint32_t lo = (uint32_t)v;
  uint32_t hi = (uint32_t)(v >> 32);
  if (lo != 0u) {
    const uint32_t old = atomicAdd(w, lo);
    hi += (uint32_t)(old + lo) < old ? 1u : 0u;
  }
  if (hi != 0u) atomicAdd(w + 1, hi);
}

struct WalkSched {
  unsigned long long* unit_counter;      // global work-queue head (zeroed per call)
  const unsigned long long* prefix;      // [n_inst+1] unit prefix, or null (uniform)
  unsigned long long total_units;
  unsigned long long units_per_inst;     // uniform budgets only
  uint32_t unit_paths;                   // paths per unit
  int regroup;                           // refill when this many lanes are idle
  int slot_words;                        // uint64 words per slot (tallies or grads)
  int want_sumsq;
  unsigned int* status;
};

struct TallyOut {
  unsigned long long* raw;   // fixed-point sums (forward: [n_inst][nt]; adjoint: [4][K][n_inst])
  double *R, *T, *A, *bins, *overflow, *R_k, *R1, *stderr_R, *stderr_bins, *steps;
  unsigned long long* truncated;
  unsigned long long* raw_out;
  double* profile;   // bins / R (Eq. 3), or null
};

struct GradIn {
  const double *grad_R, *grad_bins, *grad_R_k, *grad_T;
};

struct GradOut {
  double *d_alpha, *d_sigma_t, *d_g, *d_w;
  double *d_alpha2, *d_sigma_t2, *d_g2;  // second layer of a two-layer slab
  unsigned int* status;
};

void launch_validate(const WalkConst& c, unsigned int* status, cudaStream_t st);
// Fills the [3][K][n_inst] log table of hero-wavelength sharing (c.hero > 0).
void launch_hero_logs(const WalkConst& c, float* logs, cudaStream_t st);
void launch_unit_prefix(const uint32_t* n_paths, uint32_t n, uint32_t C,
                        unsigned long long* block_sums, unsigned long long* total,
                        unsigned long long* prefix, cudaStream_t st);
void launch_walk_persistent(bool adj, int grid, int block, size_t smem, const WalkConst& c,
                            const WalkSched& s, const TallyOut& t, const GradIn& gi,
                            cudaStream_t st);
const void* persistent_kernel_ptr(bool adj, bool layered, int hero, bool semi, int mode);
void launch_walk_plain(const WalkConst& c, const WalkSched& s, const TallyOut& t, uint32_t inst,
                       uint32_t N, cudaStream_t st);
void launch_finalize_tallies(const WalkConst& c, const WalkSched& s, const TallyOut& t,
                             cudaStream_t st);
void launch_finalize_grads(const WalkConst& c, const GradIn& gi, const unsigned long long* raw,
                           const GradOut& go, cudaStream_t st);
void launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out,
                   cudaStream_t st);

}  // namespace sss
