/*
 * sss.h -- C ABI of libsss: the mixture-of-media subsurface random walk on
 * NVIDIA B300 (sm_103a).
 *
 * The library evaluates, for many independent instances (texel x
 * wavelength), the radial subsurface profile of a K-media mixture
 * (paper: Sec. 4.1, Eq. 3 radial form R_d(r) = R * P_d(r) under normal
 * incidence; Eq. 4 mixture S = sum_k w_k S_k with sum_k w_k = 1), by a Monte
 * Carlo random walk that picks one medium per path with probability w_k
 * before the walk starts (Sec. 4.1, Sec. 6, Sec. 7).  Media are given by
 * single-scattering albedo alpha, extinction sigma_t and Henyey-Greenstein
 * anisotropy g (the parameter set theta(lambda) of Sec. 5.1, Eq. 10).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every pointer named "device" must point to memory of the CUDA device
 *    that is current on the calling thread.  The library never allocates
 *    device memory: the caller owns every buffer, including the workspace.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and runs asynchronously: results are valid once the stream has
 *    reached the call's end.  (Exceptions, each stated where it applies:
 *    the status reads, and the plain schedule with per-instance budgets.)
 *  - Errors a host can see (NULL pointer where one is required, sizes out of
 *    range, misaligned pointers, too small workspace) are returned at once
 *    and nothing is enqueued.  Errors only the device can see (invalid
 *    parameter values, step-cap truncation, fixed-point overflow) set bits
 *    of a status word kept in the workspace; read it with sss_read_status.
 *    No kernel traps and no kernel waits on another kernel.
 *  - When a status other than SSS_OK is returned or flagged, the outputs
 *    are undefined.
 *  - Calls that share a workspace must not overlap on the GPU.
 */
#ifndef SSS_H_
#define SSS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SSS_ABI_VERSION 3
#define SSS_KMAX 4          /* media per mixture supported (the paper uses 3) */
#define SSS_NBINS_MAX 1024  /* radial bins supported */

typedef enum {
  SSS_OK = 0,
  SSS_ERR_INVALID_ARG = 1,  /* host-detected bad argument */
  SSS_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  SSS_ERR_WORKSPACE = 3,    /* workspace smaller than sss_*_workspace_size */
  SSS_ERR_STEP_LIMIT = 4,   /* device: some paths hit the step cap */
  SSS_ERR_OVERFLOW = 5,     /* device: a fixed-point accumulator saturated */
  SSS_ERR_DEVICE_PARAM = 6, /* device: a parameter value is out of range */
  SSS_ERR_UNSUPPORTED = 7,  /* no sm_103a device, or a feature not built */
  SSS_ERR_TIMEOUT = 8,      /* device: a bounded wait gave up (decoder pipeline) */
  SSS_ERR_TOO_LARGE = 9     /* needs more scratch than sss_walk_noalloc's built-in array */
} sss_status;

/* Device status word bits (sss_read_status). */
#define SSS_FLAG_PARAM 0x1u      /* alpha, sigma_t, g, w or thickness invalid */
#define SSS_FLAG_STEP_LIMIT 0x2u /* at least one path was truncated */
#define SSS_FLAG_OVERFLOW 0x4u   /* a gradient accumulator saturated */
#define SSS_FLAG_ZERO_WEIGHT 0x8u /* a medium with w_k = 0 got a zero gradient */
#define SSS_FLAG_TIMEOUT 0x10u    /* a pipeline wait gave up (outputs undefined) */

typedef void* sss_stream_t; /* cudaStream_t */

/* Per-instance media.  Arrays are structure-of-arrays [K][n_inst], float32,
 * device, 4-byte aligned: element (k, i) is at [k * n_inst + i].
 *   alpha   in [0, 1]          single-scattering albedo
 *   sigma_t > 0, finite        extinction, mm^-1 (positions are in mm)
 *   g       in (-1, 1)         Henyey-Greenstein mean cosine
 *   w       >= 0, sum_k w = 1 (within 1e-5)   mixture weight (Eq. 4)
 * n_paths: device uint32 [n_inst] path budget per instance, or NULL to use
 *          uniform_paths for every instance.
 * thickness_mm: device float32 [n_inst] slab thickness (> 0; +inf for a
 *          semi-infinite slab), or NULL for all semi-infinite.
 * n_rel:   refractive index of the media relative to the outside (>= 1).
 * K in [1, SSS_KMAX]; n_inst in [0, 2^32).
 * alpha2, sigma_t2, g2, d1_mm: NULL, or device float32 [n_inst] each for a
 *          two-layer slab (the skin model of Sec. 3): the chosen medium fills
 *          the top layer 0 <= z < d1_mm, this second layer fills
 *          d1_mm <= z < thickness (semi-infinite if thickness is +inf).  The
 *          interface is index matched: a flight that reaches it stops there
 *          and continues with a fresh flight in the other layer.
 *          sss_walk_bwd gives the second layer's gradients in
 *          sss_grad_out.d_alpha2 / d_sigma_t2 / d_g2. */
typedef struct {
  const float* alpha;
  const float* sigma_t;
  const float* g;
  const float* w;
  const uint32_t* n_paths;
  uint32_t uniform_paths;
  const float* thickness_mm;
  float n_rel;
  int32_t K;
  int64_t n_inst;
  const float* alpha2;
  const float* sigma_t2;
  const float* g2;
  const float* d1_mm;
} sss_params;

/* Walk options (a zero-filled struct is NOT valid: call sss_walk_opts_default).
 *   nbins, r_max_mm : linear radial bins over [0, r_max) in the entry face;
 *                     exits at r >= r_max go to the overflow tally.
 *   mode            : 0 = albedo weighting with Russian roulette (default),
 *                     1 = analog absorption.
 *   rr_threshold    : roulette weight W_th (mode 0); a path whose weight
 *                     falls below it survives with probability W/W_th at
 *                     weight W_th.  0 disables roulette.
 *   entry_fresnel   : 1 = entry weight 1 - R0, R0 = ((n-1)/(n+1))^2: the
 *                     specular reflection is excluded from every tally.
 *   max_steps       : cap on random-number draws per path (a path that hits
 *                     it is dropped and counted in `truncated`).
 *   seed            : 64-bit Philox key.
 *   path_offset     : index of the first path of each instance; runs over
 *                     [0, M) and [M, N) add up bit-exactly to [0, N).
 *   want_sumsq      : 1 = also tally squared exit weights (standard errors).
 *   schedule        : 0 = persistent batched kernel over all instances;
 *                     1 = plain baseline, one launch per instance, one thread
 *                     per path, no regrouping.  With per-instance budgets
 *                     (n_paths non-NULL) the plain baseline is the one
 *                     synchronous case: sss_walk copies the budgets to the
 *                     host and waits for `stream` before it launches (each
 *                     launch's grid depends on its budget), and it cannot be
 *                     graph-captured (use_graph = 1: SSS_ERR_INVALID_ARG).
 *   use_graph       : 1 = capture the call's launches once in a CUDA graph
 *                     (cached per argument set, at most 64 plans, the oldest
 *                     dropped first) and replay it.
 *   block_threads, unit_paths, regroup : launch shape of the persistent
 *                     kernel (0 = built-in defaults); results do not depend
 *                     on them.
 *   instance_offset : number added to each instance's index in the random-
 *                     number counters, so a shard [b, e) of a larger batch,
 *                     walked with instance_offset = b, reproduces that
 *                     batch's instances bit for bit (multi-GPU sharding).
 *   log_r_min_mm    : 0 = linear bins (default).  > 0: logarithmic bins as
 *                     in the paper's dataset generator (Sec. 3): bin 0 is
 *                     [0, r_min), bin b >= 1 is [r_min q^(b-1), r_min q^b)
 *                     with q = (r_max / r_min)^(1 / (nbins - 1)).
 *                     Negative, non-finite, >= r_max_mm, or with nbins < 2:
 *                     SSS_ERR_INVALID_ARG.
 *   incidence       : 0 = normal incidence at the origin (Eq. 3, default);
 *                     1 = cosine-weighted incident lobe (the fitting
 *                     illumination of Sec. 8): outside cosine sqrt(u),
 *                     azimuth 2 pi u' from a third Philox draw per path
 *                     (tag 2), refracted by Snell's law, entry weight 1 - F
 *                     at the refracted angle when entry_fresnel = 1.
 *   select_pdf      : how a path picks its medium, once, before the walk.
 *                     0 = with probability w_k / sum(w) (Sec. 7, default);
 *                     1 = uniformly among the K media, the path weight
 *                     multiplied by K w_k / sum(w) so the mixture of Eq. 4
 *                     is estimated without bias (Sec. 7 leaves other
 *                     choices open).  Other values: SSS_ERR_INVALID_ARG.
 *   hero_bands      : 0 = off (default).  C in [1, 4]: hero-wavelength
 *                     sharing (Wilkie et al. 2014; the paper's related work
 *                     names hero-wavelength tracking).  Instances are texels
 *                     of hero_texel_bands consecutive bands; each texel's
 *                     bands form groups of C (blocks of C adjacent bands, or
 *                     with hero_orbits = 1 the rotation orbits {q, q + nb/C,
 *                     ...}).  Path p of a group samples with the optics of
 *                     member p mod C (counters: step, p, the group's first
 *                     member + instance_offset, tag) and every member scores
 *                     the balance-heuristic estimate C f_j / sum_i p_i, so a
 *                     group walks n_paths paths and each member gets an
 *                     n_paths-sample estimate.  Roulette is decided on the
 *                     largest member weight.  Requires mode 0, hero_texel_bands
 *                     a multiple of C, n_inst a multiple of hero_texel_bands
 *                     and uniform budgets (n_paths NULL), else
 *                     SSS_ERR_INVALID_ARG; the plain schedule, the adjoint
 *                     and two-layer slabs return SSS_ERR_UNSUPPORTED.  The
 *                     slab thickness is the group's first member's.  A (the
 *                     absorbed fraction) is not scored and reads 0.
 */
typedef struct {
  int32_t nbins;
  float r_max_mm;
  int32_t mode;
  float rr_threshold;
  int32_t entry_fresnel;
  uint32_t max_steps;
  uint64_t seed;
  uint32_t path_offset;
  int32_t want_sumsq;
  int32_t schedule;
  int32_t use_graph;
  int32_t block_threads;
  int32_t unit_paths;
  int32_t regroup;
  uint32_t instance_offset;
  int32_t incidence;
  float log_r_min_mm;
  int32_t select_pdf;
  int32_t hero_bands;
  int32_t hero_texel_bands;
  int32_t hero_orbits;
} sss_walk_opts;

/* Forward outputs, all float64 device arrays owned by the caller; any may be
 * NULL.  Each tally is the mean over the instance's N paths of that path's
 * exit weight (a fraction of the incident power):
 *   R [n_inst]         diffuse reflectance through the entry face (= sum of
 *                      bins + overflow), the "R" of Eq. 3
 *   T [n_inst]         transmittance through the far face of a finite slab
 *   A [n_inst]         absorbed weight
 *   bins [n_inst][nbins]  radial exit histogram (R * P_d(r) integrated over
 *                      each annulus)
 *   overflow [n_inst]  exits at r >= r_max
 *   R_k [n_inst][K]    reflectance carried by paths that chose medium k
 *   R1 [n_inst]        reflectance of paths with exactly one collision
 *   stderr_R, stderr_bins: standard errors (need want_sumsq = 1)
 *   truncated [n_inst] uint64 count of paths cut by max_steps
 *   steps [n_inst]     mean random-number draws (walk steps) per path
 *   raw [n_inst][sss_tally_count(nbins, K, want_sumsq)] uint64: the exact
 *                      fixed-point sums (weight * 2^32) in the order
 *                      bins, overflow, R_k, R1, T, A, then the plain counts
 *                      truncated and steps, then [sumsq bins, sumsq overflow]
 *                      (squared weights * 2^32).
 *   profile [n_inst][nbins]  the normalised radial profile P_d(r) of Eq. 3
 *                      (R_d(r) = R * P_d(r)): bins / R, the fraction of R
 *                      leaving through each annulus; 0 where R = 0.  The
 *                      scale-free tables of Sec. 4.2 are this profile at
 *                      sigma_t = 1. */
typedef struct {
  double* R;
  double* T;
  double* A;
  double* bins;
  double* overflow;
  double* R_k;
  double* R1;
  double* stderr_R;
  double* stderr_bins;
  uint64_t* truncated;
  double* steps;
  uint64_t* raw;
  double* profile;
} sss_tallies;

/* Upstream derivatives d(loss)/d(tally) for sss_walk_bwd; float64 device,
 * any may be NULL (= zero):  grad_R [n_inst], grad_bins [n_inst][nbins],
 * grad_R_k [n_inst][K], grad_T [n_inst]. */
typedef struct {
  const double* grad_R;
  const double* grad_bins;
  const double* grad_R_k;
  const double* grad_T;
} sss_grad_in;

/* Parameter gradients, float64 device [K][n_inst], any may be NULL.
 * d_w is the partial derivative of sum_k w_k S_k with the other weights
 * held fixed (Eq. 4), i.e. the medium's own contribution S_k; project onto
 * the simplex (subtract the w-weighted mean) for a constrained step.
 * Two-layer slabs: d_alpha .. d_w cover the top layer (the chosen medium),
 * and d_alpha2, d_sigma_t2, d_g2 ([n_inst] float64 device, any may be NULL)
 * the second layer's optics; those three are ignored without a second
 * layer. */
typedef struct {
  double* d_alpha;
  double* d_sigma_t;
  double* d_g;
  double* d_w;
  double* d_alpha2;
  double* d_sigma_t2;
  double* d_g2;
} sss_grad_out;

/* Fill *o with the defaults: 64 bins over 10 mm, mode 0, W_th = 1/16,
 * entry_fresnel 1, max_steps 65536, seed 0, want_sumsq 1, schedule 0,
 * use_graph 0, automatic launch shape. */
void sss_walk_opts_default(sss_walk_opts* o);

/* Number of uint64 tallies per instance in the raw layout above. */
int32_t sss_tally_count(int32_t nbins, int32_t K, int32_t want_sumsq);

/* Workspace bytes sss_walk / sss_walk_bwd need for these arguments
 * (256-byte aligned device memory; contents need not be initialised).
 * Returns 0 if the arguments are invalid. */
size_t sss_walk_workspace_size(const sss_params* p, const sss_walk_opts* o);
size_t sss_walk_bwd_workspace_size(const sss_params* p, const sss_walk_opts* o);

/* Forward walk (Sec. 4.1 Eq. 2-4; medium choice per Sec. 7).  Enqueues
 * parameter validation, the walk and the float64 finalisation on `stream`.
 * Results are bit-identical for identical arguments, whatever the launch
 * shape.  Returns SSS_ERR_INVALID_ARG / SSS_ERR_WORKSPACE / SSS_ERR_CUDA /
 * SSS_ERR_UNSUPPORTED as described above; device-side problems are
 * reported through sss_read_status. */
sss_status sss_walk(const sss_params* p, const sss_walk_opts* o, void* workspace,
                    size_t workspace_bytes, sss_tallies* out, sss_stream_t stream);

/* Path-replay adjoint of sss_walk: re-runs every path from its Philox
 * counters (no stored path state) and accumulates, for each path, its exit
 * weight times the upstream derivative of the tally it landed in times the
 * score of the path density (differentiating f_SSS of Sec. 4.1 and the
 * mixture of Eq. 4):
 *   d/d alpha_k : n / alpha_k           (n collisions)
 *   d/d sigma_t,k : n / sigma_t,k - L   (L = path length inside)
 *   d/d g_k     : sum_i d log p_HG(mu_i; g_k) / d g_k
 *   d/d w_k     : sum(w) / w_k          (paths that chose k)
 * Must get the same p and o (seed, path_offset, ...) as the forward call.
 * Requires mode 0 or 1; roulette is allowed. */
sss_status sss_walk_bwd(const sss_params* p, const sss_walk_opts* o, void* workspace,
                        size_t workspace_bytes, const sss_grad_in* gin,
                        sss_grad_out* gout, sss_stream_t stream);

/* Waits for `stream`, then returns the status word the last call that used
 * `workspace` left (SSS_FLAG_* bits) in *flags and maps it to a status:
 * SSS_ERR_TIMEOUT, SSS_ERR_DEVICE_PARAM, SSS_ERR_OVERFLOW, SSS_ERR_STEP_LIMIT
 * or SSS_OK (in that order of precedence). */
sss_status sss_read_status(const void* workspace, sss_stream_t stream, uint32_t* flags);

/* The same for the workspace of the last successful sss_walk, sss_walk_bwd,
 * sss_walk_noalloc or sss_decode call enqueued on `stream` (the library
 * remembers one per stream; thread-safe).  SSS_ERR_INVALID_ARG if no such
 * call was made on the stream or `flags` is NULL. */
sss_status sss_last_device_status(sss_stream_t stream, uint32_t* flags);

/* Philox4x32-10 blocks computed by the device code the walk uses
 * (diagnostic): out[4*i .. 4*i+3] = Philox(ctr[4*i .. 4*i+3], key).
 * ctr, out: device uint32 arrays of 4*n words. */
sss_status sss_philox(const uint32_t* ctr, uint64_t key, int64_t n, uint32_t* out,
                      sss_stream_t stream);

/* ------------------------------------------------------------------------
 * Chained decoder (paper Sec. 5.1, Eq. 10): RGB albedo -> Enc -> p (5) ->
 * Dec_R -> R_d (376 bands, 250-1000 nm at 2 nm) -> Dec_T(p, R_d) ->
 * theta(lambda) = {alpha_k, g_k, sigma_t,k, w_k}, K = 3, then resampled
 * linearly to the 81 visible bands 380-780 nm at 5 nm.  BF16 operands on the
 * tensor cores, FP32 accumulation, BF16 hidden activations.
 * Layers (natural layout W [out][in], bf16 bits as uint16, device; b [out]
 * float32, device), in this order:
 *   0 enc0  3 -> 256 tanh      1 enc1 256 -> 256 tanh   2 enc2 256 -> 5 sigmoid
 *   3 dec_r0 5 -> 512 tanh     4 dec_r1 512 -> 512 tanh 5 dec_r2 512 -> 376 sigmoid
 *   6 dec_t0 381 -> 768 tanh (input order: p then R_d)
 *   7 dec_t1 768 -> 768 tanh   8 dec_t2 768 -> 768 tanh
 *   9 dec_t3 768 -> 376*12, output index  band*12 + k*4 + c  with channel c
 *     0 alpha (sigmoid), 1 g (sigmoid), 2 sigma_t = 10^(3 sigmoid) mm^-1,
 *     3 w (softmax over k).
 * The Enc / Dec_R widths are stand-ins (the paper defers them to a cited
 * work); Dec_T's are the paper's. */
typedef struct {
  const uint16_t* W[10];
  const float* b[10];
} sss_decoder_weights;

/* Bytes of the packed (padded, reordered) weights sss_decode reads. */
size_t sss_decoder_packed_size(void);

/* Packs the natural-layout weights into `packed` (device, 256-byte aligned,
 * sss_decoder_packed_size() bytes) with kernels on `stream`. */
sss_status sss_decoder_pack(const sss_decoder_weights* w, void* packed, size_t packed_bytes,
                            sss_stream_t stream);

/* Workspace bytes sss_decode needs for T texels (activation buffers). */
size_t sss_decode_workspace_size(int64_t T);

/* Decodes T texels: rgb float32 [T][3] (device) -> float32 alpha, g,
 * sigma_t, w, each [3][81 * T] (device, caller-owned), in the walk's
 * sss_params layout with instance i = band * T + texel (band-major).
 * workspace: 256-byte aligned, sss_decode_workspace_size(T) bytes; its first
 * word is the status word (sss_read_status: SSS_FLAG_TIMEOUT). */
sss_status sss_decode(const float* rgb, int64_t T, const void* packed, void* workspace,
                      size_t workspace_bytes, float* alpha, float* g, float* sigma_t, float* w,
                      sss_stream_t stream);

/* Self-test of the decoder's failure detection (no counterpart in the
 * paper).  Launches one block whose first thread waits, with the same
 * bounded mbarrier wait the decoder's pipeline roles use, for a barrier
 * phase that nothing completes.  After limit_cycles SM clock cycles
 * (1 <= limit_cycles <= 4e9, about 2 s at most) it gives up, sets
 * SSS_FLAG_TIMEOUT in the word at `status` (device, 4-byte aligned, caller
 * owned; a decode workspace's first word works), and returns: the context
 * stays usable and sss_read_status on that word reports SSS_ERR_TIMEOUT.
 * Errors: SSS_ERR_INVALID_ARG for a null or misaligned pointer or a limit
 * out of range; SSS_ERR_CUDA if the launch fails. */
sss_status sss_selftest_bounded_wait(uint32_t* status, int64_t limit_cycles,
                                     sss_stream_t stream);

/* ------------------------------------------------------------------------
 * LUT-based mixture fit (paper Sec. 4.2, Eq. 6-9).  Tables of a homogeneous
 * semi-infinite medium at sigma_t = 1 (built with sss_walk, K = 1):
 *   R  [na][ng]      total reflectance R(alpha_i, g_j)
 *   p  [na][ng][nb]  radial exit density (per unit area, mfp^-2) at the bin
 *                    centres rho_b = (b + 1/2) drho
 * on alpha_i = a0 + i da, g_j = g0 + j dg (float32, device).  Lookups are
 * bilinear in (alpha, g) and linear in rho, clamped to the grid; extinction
 * rescales the radial axis: P(r | alpha, g, sigma_t) = sigma_t^2 p(sigma_t r).
 * For each problem (tone x wavelength) the fit minimises
 *   L = RMSE_j(log P_hat(r_j), log P_MC(r_j)) + lambda_R (R_hat - R_MC)^2,
 *   R_hat = sum_k w_k R(alpha_k, g_k),  P_hat(r) = sum_k w_k P(r | theta_k),
 * over the radii with P_MC > 0, by Adam (0.9, 0.999, 1e-8) with learning
 * rate lr (1 + cos(pi (t-1) / steps)) / 2.  Raw parameters per problem,
 * [4K] float32, in/out: [alpha_raw K][g_raw K][log sigma_t K][w_raw K] with
 * alpha = a_lo + (a_hi - a_lo) sigmoid(raw), g likewise, sigma_t = exp(raw),
 * w = softmax(raw).  One warp per problem. */
typedef struct {
  const float* R;
  const float* p;
  int32_t na, ng, nb;
  float a0, da, g0, dg, drho;
} sss_lut;

typedef struct {
  int32_t K;        /* media, 1..4 */
  int32_t steps;    /* Adam steps (0: only evaluate loss and gradient) */
  float lr;         /* 1e-2 in the paper */
  float lambda_R;   /* 5 in the paper */
  float a_lo, a_hi, g_lo, g_hi;
} sss_fit_opts;

/* r_mm [n_r] radii (mm, n_r <= 64), P_mc [n_prob][n_r] target profile
 * densities (mm^-2; entries <= 0 are ignored), R_mc [n_prob] target
 * reflectances, raw [n_prob][4K] in/out, loss [n_prob] out (may be NULL),
 * grad [n_prob][4K] out: gradient at the returned parameters (may be NULL).
 * All device pointers. */
sss_status sss_lut_fit(const sss_lut* lut, int64_t n_prob, const float* r_mm, int32_t n_r,
                       const float* P_mc, const float* R_mc, const sss_fit_opts* o, float* raw,
                       float* loss, float* grad, sss_stream_t stream);

/* Profiling hook.  With both events non-NULL (cudaEvent_t handles created by
 * the caller), each following sss_walk / sss_walk_bwd issued from this host
 * thread records `start` right before and `stop` right after its main walk
 * kernel, on the call's stream, so the caller can time that kernel alone.
 * Pass NULL, NULL to stop.  Ignored for calls replayed from a cached graph. */
void sss_profile_events(void* start, void* stop);

/* Forward walk for callers that cannot allocate device memory.  The paper
 * has no counterpart to this entry point; it exists for hosts that own every
 * device allocation themselves (a renderer plug-in inside an application
 * with its own memory pool) or that must not call cudaMalloc on the calling
 * thread (it can synchronise the device, and is not allowed while a stream is
 * being captured).  It computes exactly what sss_walk computes, but its
 * scratch lives in a fixed array inside the library:
 *  - the array holds SSS_NOALLOC_SCRATCH_BYTES (16 MiB) on every GPU that
 *    loads the library, until the process exits; calls whose
 *    sss_walk_workspace_size exceeds it return SSS_ERR_TOO_LARGE (at 64 bins,
 *    K = 3 and standard errors that is about 15,000 instances);
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current, and so does the first
 *    call after the device's context has changed (cudaDeviceReset); make
 *    those calls before any stream capture on that device;
 *  - every call shares the one array, which keeps the last call's contents:
 *    each call clears what must start at zero, but calls that overlap on
 *    the GPU (other streams, other threads) race and must be serialised;
 *  - it allocates nothing: no cudaMalloc / cudaFree and no allocating
 *    library routine; schedule must be 0 and use_graph 0 (otherwise
 *    SSS_ERR_INVALID_ARG).
 * `out` as for sss_walk.  status_flags: NULL, or a host word that receives
 * the device status word (the call then waits for `stream`, as
 * sss_read_status does, and returns the mapped status). */
#define SSS_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
sss_status sss_walk_noalloc(const sss_params* p, const sss_walk_opts* o, sss_tallies* out,
                            uint32_t* status_flags, sss_stream_t stream);

/* Drops every cached CUDA graph (use_graph = 1). */
void sss_release_plans(void);

/* Static text for a status code. */
const char* sss_status_string(sss_status s);

/* ------------------------------------------------------------------------ */
/* Issue-rate probes (no counterpart in the paper: measurement of the        */
/* per-SM arithmetic throughput that bounds the walk, for its roofline).     */
/* ------------------------------------------------------------------------ */
enum {
  SSS_PROBE_FFMA = 0,   /* binary32 fused multiply-add                        */
  SSS_PROBE_FFMA2 = 1,  /* paired binary32 fused multiply-add (two lanes' ops) */
  SSS_PROBE_IMAD = 2,   /* 32-bit integer multiply-add                        */
  SSS_PROBE_LOP3 = 3,   /* 32-bit three-input logic operation                 */
  SSS_PROBE_MUFU = 4,   /* special-function unit (lg2.approx)                 */
  SSS_PROBE_PHILOX = 5  /* whole Philox4x32-10 blocks, as the walk draws them  */
};

/* Launches `blocks` blocks of 256 threads on `stream`, each thread running
 * `iters` iterations of eight independent chains of the probed operation
 * (four chains of whole blocks for SSS_PROBE_PHILOX, each block's output
 * the next block's counter, round keys in the kernel's parameter bank as
 * the walk holds them), and writes one float per thread to sink[blocks *
 * 256] (device, caller owned) so nothing is optimised away.  Asynchronous: time it with events
 * on the stream.  Operations executed = blocks * 256 * iters *
 * sss_probe_ops_per_thread_iter(kind).  Errors: SSS_ERR_INVALID_ARG for a
 * bad kind, iters < 1, blocks < 1 or a null sink; SSS_ERR_CUDA if the
 * launch fails. */
sss_status sss_probe(int32_t kind, int64_t iters, int32_t blocks, float* sink,
                     sss_stream_t stream);
int64_t sss_probe_ops_per_thread_iter(int32_t kind);

/* SSS_ABI_VERSION of the loaded library. */
int32_t sss_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SSS_H_ */
