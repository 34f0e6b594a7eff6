// api.cu -- the C ABI of libsss (declared in include/sss.h).
//
// Host-side argument checks, workspace layout, launch shapes and the
// CUDA-graph cache.  Every step of the walk itself runs in the kernels of
// walk_kernels.cu; nothing here computes on the host.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sss.h"
#include "last_status.cuh"
#include "walk_kernels.cuh"

using namespace sss;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t header = 0;       // status u32 @0, unit counter u64 @8, total units u64 @16
  size_t block_sums = 0;   // uneven budgets: per-256-instance unit sums
  size_t prefix = 0;       // uneven budgets: [n_inst+1] unit prefix
  size_t hero = 0;         // hero-wavelength sharing: [3][K][n_inst] float log table
  size_t acc = 0;          // fixed-point accumulators
  size_t total = 0;
  int acc_words = 0;       // per instance (forward) or per slot (adjoint)
};

int tally_count(int nbins, int K, int sumsq) { return nbins + 6 + K + (sumsq ? nbins + 1 : 0); }

bool params_ok(const sss_params* p) {
  if (!p) return false;
  if (p->K < 1 || p->K > SSS_KMAX) return false;
  if (p->n_inst < 0 || p->n_inst > (int64_t)0xffffffffLL) return false;
  if (p->n_inst > 0 && (!p->alpha || !p->sigma_t || !p->g || !p->w)) return false;
  if (!(p->n_rel >= 1.0f) || !std::isfinite(p->n_rel)) return false;
  const bool l2 = p->alpha2 || p->sigma_t2 || p->g2 || p->d1_mm;
  if (l2 && !(p->alpha2 && p->sigma_t2 && p->g2 && p->d1_mm)) return false;  // all or none
  const void* ptrs[] = {p->alpha, p->sigma_t, p->g, p->w, p->n_paths, p->thickness_mm,
                        p->alpha2, p->sigma_t2, p->g2, p->d1_mm};
  for (const void* q : ptrs)
    if (q && (reinterpret_cast<uintptr_t>(q) & 3u)) return false;
  return true;
}

bool opts_ok(const sss_walk_opts* o) {
  if (!o) return false;
  if (o->nbins < 1 || o->nbins > SSS_NBINS_MAX) return false;
  if (!(o->r_max_mm > 0.0f) || !std::isfinite(o->r_max_mm)) return false;
  if (o->mode != 0 && o->mode != 1) return false;
  if (o->mode == 0 && !(o->rr_threshold >= 0.0f && o->rr_threshold <= 1.0f)) return false;
  if (o->entry_fresnel != 0 && o->entry_fresnel != 1) return false;
  if (o->max_steps < 1) return false;
  if (o->schedule != 0 && o->schedule != 1) return false;
  if (o->block_threads != 0 &&
      (o->block_threads < 32 || o->block_threads > 256 || o->block_threads % 32)) return false;
  if (o->unit_paths < 0 || o->regroup < 0 || o->regroup > 32) return false;
  if (o->incidence != 0 && o->incidence != 1) return false;
  if (o->select_pdf != 0 && o->select_pdf != 1) return false;
  if (o->hero_bands < 0 || o->hero_bands > kHeroMax) return false;
  if (o->hero_orbits != 0 && o->hero_orbits != 1) return false;
  if (o->hero_bands > 0 &&
      (o->hero_texel_bands < o->hero_bands || o->hero_texel_bands % o->hero_bands != 0 ||
       o->mode != 0))
    return false;
  if (o->log_r_min_mm < 0.0f || !std::isfinite(o->log_r_min_mm)) return false;
  if (o->log_r_min_mm > 0.0f && (o->log_r_min_mm >= o->r_max_mm || o->nbins < 2)) return false;
  return true;
}

Layout make_layout(const sss_params* p, const sss_walk_opts* o, bool adj) {
  Layout L;
  const size_t n = (size_t)p->n_inst;
  size_t off = 0;
  L.header = off;
  off += kAlign;
  if (p->n_paths) {
    L.block_sums = off;
    off += align_up(((n + 255) / 256 + 1) * 8);
    L.prefix = off;
    off += align_up((n + 1) * 8);
  }
  if (!adj && o->hero_bands > 0) {
    L.hero = off;
    off += align_up((size_t)3 * p->K * n * 4);
  }
  L.acc = off;
  if (adj) {
    // [4][K] per-medium gradient words, then 3 for a second layer's optics
    L.acc_words = 4 * p->K + (p->alpha2 ? 3 : 0);
    off += align_up((size_t)L.acc_words * n * 8);
  } else {
    L.acc_words = tally_count(o->nbins, p->K, o->want_sumsq);
    off += align_up((size_t)L.acc_words * n * 8);
  }
  L.total = off;
  return L;
}

struct DevInfo {
  bool checked = false;
  bool ok = false;
  int sms = 0;
};
std::mutex g_mu;
std::map<int, DevInfo> g_dev;

bool device_ok(int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  DevInfo& d = g_dev[dev];
  if (!d.checked) {
    int major = 0, minor = 0;
    d.checked = true;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
      d.ok = (major == 10 && minor == 3);
    }
  }
  if (sms) *sms = d.sms;
  return d.ok;
}

WalkConst make_const(const sss_params* p, const sss_walk_opts* o) {
  WalkConst c;
  c.alpha = p->alpha;
  c.sigma_t = p->sigma_t;
  c.g = p->g;
  c.w = p->w;
  c.n_paths = p->n_paths;
  c.thickness = p->thickness_mm;
  c.uniform_paths = p->uniform_paths;
  c.n_inst = (uint32_t)p->n_inst;
  c.K = p->K;
  c.n_rel = p->n_rel;
  const double n = p->n_rel;
  const double r0 = ((n - 1.0) / (n + 1.0)) * ((n - 1.0) / (n + 1.0));
  c.W0 = o->entry_fresnel ? (float)(1.0 - r0) : 1.0f;
  c.nbins = o->nbins;
  c.bin_scale = (float)((double)o->nbins / (double)o->r_max_mm);
  c.mode = o->mode;
  c.rr_th = o->mode == 0 ? o->rr_threshold : 0.0f;
  c.inv_rr_th = c.rr_th > 0.0f ? (float)(1.0 / (double)c.rr_th) : 0.0f;
  c.max_steps = o->max_steps;
  c.key0 = (uint32_t)(o->seed & 0xffffffffull);
  c.key1 = (uint32_t)(o->seed >> 32);
  c.path_offset = o->path_offset;
  c.inst_offset = o->instance_offset;
  c.incidence = o->incidence;
  c.entry_fresnel = o->entry_fresnel;
  c.select_uniform = o->select_pdf == 1;
  c.hero = o->hero_bands;
  c.hero_nb = o->hero_texel_bands;
  c.hero_orbits = o->hero_orbits;
  c.hero_logs = nullptr;  // set by enqueue_walk (workspace)
  c.log_bins = o->log_r_min_mm > 0.0f;
  c.inv_rmin = c.log_bins ? (float)(1.0 / (double)o->log_r_min_mm) : 0.0f;
  c.inv_log2q = c.log_bins && o->nbins > 1
                    ? (float)((double)(o->nbins - 1) /
                              std::log2((double)o->r_max_mm / (double)o->log_r_min_mm))
                    : 0.0f;
  c.alpha2 = p->alpha2;
  c.sigma_t2 = p->sigma_t2;
  c.g2 = p->g2;
  c.d1 = p->d1_mm;
  for (int r = 0; r < 10; ++r) {
    c.rk[2 * r] = c.key0 + (uint32_t)r * 0x9E3779B9u;
    c.rk[2 * r + 1] = c.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  return c;
}

// Profiling events (per host thread).
thread_local cudaEvent_t g_ev_start = nullptr, g_ev_stop = nullptr;

// Graph cache: one instantiated graph per exact argument set, at most
// kMaxGraphs of them (the oldest is dropped first).
constexpr size_t kMaxGraphs = 64;
std::map<std::string, cudaGraphExec_t> g_graphs;
std::vector<std::string> g_graph_order;          // insertion order, oldest first
std::map<cudaStream_t, const void*> g_last_ws;  // guarded by g_mu

// Keys are built member by member (never from raw struct bytes, whose
// padding is indeterminate), so equal arguments always give equal keys.
template <class T>
void put(std::string& k, const T& v) {
  k.append(reinterpret_cast<const char*>(&v), sizeof(T));
}

void put_params(std::string& k, const sss_params* p) {
  put(k, p->alpha); put(k, p->sigma_t); put(k, p->g); put(k, p->w);
  put(k, p->n_paths); put(k, p->uniform_paths); put(k, p->thickness_mm); put(k, p->n_rel);
  put(k, p->K); put(k, p->n_inst);
  put(k, p->alpha2); put(k, p->sigma_t2); put(k, p->g2); put(k, p->d1_mm);
}

void put_opts(std::string& k, const sss_walk_opts* o) {
  put(k, o->nbins); put(k, o->r_max_mm); put(k, o->mode); put(k, o->rr_threshold);
  put(k, o->entry_fresnel); put(k, o->max_steps); put(k, o->seed); put(k, o->path_offset);
  put(k, o->want_sumsq); put(k, o->schedule); put(k, o->use_graph); put(k, o->block_threads);
  put(k, o->unit_paths); put(k, o->regroup); put(k, o->instance_offset); put(k, o->incidence);
  put(k, o->log_r_min_mm); put(k, o->select_pdf); put(k, o->hero_bands);
  put(k, o->hero_texel_bands); put(k, o->hero_orbits);
}

// `ptrs` / `nptrs`: the output or gradient pointers of the call (structs of
// pointers only, so their bytes have no padding).
std::string graph_key(int tag, const sss_params* p, const sss_walk_opts* o, const void* ws,
                      size_t wsb, const void* const* ptrs, size_t nptrs, sss_stream_t st) {
  std::string k;
  int dev = 0;
  cudaGetDevice(&dev);
  put(k, tag);
  put(k, dev);
  put_params(k, p);
  put_opts(k, o);
  put(k, ws);
  put(k, wsb);
  for (size_t i = 0; i < nptrs; ++i) put(k, ptrs[i]);
  put(k, st);
  return k;
}

// Launch configuration of the persistent kernel.
struct Shape {
  int block, grid, regroup;
  uint32_t unit_paths;
  size_t smem;
};

sss_status persistent_shape(bool adj, const sss_params* p, const sss_walk_opts* o, int acc_words,
                            int sms, Shape* sh) {
  constexpr size_t kSmemLimit = 200 * 1024;
  sh->block = o->block_threads ? o->block_threads : 256;
  sh->regroup = o->regroup ? o->regroup : 8;
  sh->unit_paths = o->unit_paths ? (uint32_t)o->unit_paths : 1024u;
  // two slots of accumulators per warp; shrink the block for wide histograms
  // a hero group's slot holds its C members' accumulators
  const size_t members = o->hero_bands > 0 ? (size_t)o->hero_bands : 1;
  const size_t per_warp =
      (size_t)2 * members * acc_words * 8 + 2 * kSlotMetaBytes + kSelBufBytes;
  if (per_warp > kSmemLimit) return SSS_ERR_INVALID_ARG;
  const int max_warps = (int)(kSmemLimit / per_warp);
  if (sh->block / 32 > max_warps) sh->block = max_warps * 32;
  sh->smem = (size_t)(sh->block / 32) * per_warp;
  const void* fn = persistent_kernel_ptr(adj, p->alpha2 != nullptr, o->hero_bands,
                                         p->thickness_mm == nullptr, o->mode);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit) !=
      cudaSuccess)
    return SSS_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, sh->block, sh->smem) !=
      cudaSuccess)
    return SSS_ERR_CUDA;
  if (per_sm < 1) return SSS_ERR_INVALID_ARG;
  sh->grid = sms * per_sm;
  (void)p;
  return SSS_OK;
}

sss_status enqueue_walk(bool adj, const sss_params* p, const sss_walk_opts* o, void* ws,
                        const Layout& L, sss_tallies* out, const sss_grad_in* gin,
                        sss_grad_out* gout, int sms, cudaStream_t st) {
  char* base = static_cast<char*>(ws);
  unsigned int* status = reinterpret_cast<unsigned int*>(base + L.header);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(base + L.header + 8);
  unsigned long long* total = reinterpret_cast<unsigned long long*>(base + L.header + 16);
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(base + L.acc);
  WalkConst c = make_const(p, o);
  if (c.hero > 0) c.hero_logs = reinterpret_cast<const float*>(base + L.hero);

  // zero the header and the accumulators
  if (cudaMemsetAsync(base + L.header, 0, kAlign, st) != cudaSuccess) return SSS_ERR_CUDA;
  if (L.total > L.acc && cudaMemsetAsync(acc, 0, L.total - L.acc, st) != cudaSuccess)
    return SSS_ERR_CUDA;
  launch_validate(c, status, st);
  if (c.hero > 0) launch_hero_logs(c, reinterpret_cast<float*>(base + L.hero), st);

  Shape sh{};
  if (o->schedule == 0 || adj) {
    sss_status r = persistent_shape(adj, p, o, L.acc_words, sms, &sh);
    if (r != SSS_OK) return r;
  }
  WalkSched s{};
  s.unit_counter = counter;
  s.unit_paths = sh.unit_paths ? sh.unit_paths : 1024u;
  s.regroup = sh.regroup;
  s.slot_words = L.acc_words;
  s.want_sumsq = o->want_sumsq;
  s.status = status;
  if (p->n_paths) {
    unsigned long long* bsum = reinterpret_cast<unsigned long long*>(base + L.block_sums);
    unsigned long long* prefix = reinterpret_cast<unsigned long long*>(base + L.prefix);
    launch_unit_prefix(p->n_paths, (uint32_t)p->n_inst, s.unit_paths, bsum, total, prefix, st);
    s.prefix = prefix;
    // total units are read on the device: pass an upper bound and let the
    // lookup reject units past prefix[n_inst]
    s.total_units = ~0ull;
  } else {
    s.prefix = nullptr;
    s.units_per_inst = (p->uniform_paths + (unsigned long long)s.unit_paths - 1) / s.unit_paths;
    // hero-wavelength sharing schedules groups of hero_bands instances
    const unsigned long long n_sched =
        o->hero_bands > 0 ? (unsigned long long)p->n_inst / o->hero_bands
                          : (unsigned long long)p->n_inst;
    s.total_units = s.units_per_inst * n_sched;
  }

  TallyOut t{};
  t.raw = acc;
  GradIn gi{};
  if (gin) {
    gi.grad_R = gin->grad_R;
    gi.grad_bins = gin->grad_bins;
    gi.grad_R_k = gin->grad_R_k;
    gi.grad_T = gin->grad_T;
  }
  if (!adj && out) {
    t.R = out->R; t.T = out->T; t.A = out->A; t.bins = out->bins; t.overflow = out->overflow;
    t.R_k = out->R_k; t.R1 = out->R1; t.stderr_R = out->stderr_R;
    t.stderr_bins = out->stderr_bins;
    t.steps = out->steps;
    t.truncated = reinterpret_cast<unsigned long long*>(out->truncated);
    t.raw_out = reinterpret_cast<unsigned long long*>(out->raw);
    t.profile = out->profile;
  }

  if (p->n_inst > 0) {
    const bool prof = g_ev_start && g_ev_stop && !o->use_graph;
    if (prof) cudaEventRecord(g_ev_start, st);
    if (adj || o->schedule == 0) {
      launch_walk_persistent(adj, sh.grid, sh.block, sh.smem, c, s, t, gi, st);
    } else {
      std::vector<uint32_t> N((size_t)p->n_inst, p->uniform_paths);
      if (p->n_paths) {
        if (cudaMemcpyAsync(N.data(), p->n_paths, N.size() * 4, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
          return SSS_ERR_CUDA;
      }
      for (int64_t i = 0; i < p->n_inst; ++i) launch_walk_plain(c, s, t, (uint32_t)i, N[i], st);
    }
    if (prof) cudaEventRecord(g_ev_stop, st);
  }
  if (adj) {
    GradOut go{};
    if (gout) {
      go.d_alpha = gout->d_alpha; go.d_sigma_t = gout->d_sigma_t;
      go.d_g = gout->d_g; go.d_w = gout->d_w;
      if (p->alpha2) {
        go.d_alpha2 = gout->d_alpha2; go.d_sigma_t2 = gout->d_sigma_t2; go.d_g2 = gout->d_g2;
      }
    }
    go.status = status;
    launch_finalize_grads(c, gi, acc, go, st);
  } else {
    launch_finalize_tallies(c, s, t, st);
  }
  return cudaGetLastError() == cudaSuccess ? SSS_OK : SSS_ERR_CUDA;
}

sss_status run_impl(bool adj, const sss_params* p, const sss_walk_opts* o, void* ws, size_t wsb,
                    sss_tallies* out, const sss_grad_in* gin, sss_grad_out* gout,
                    sss_stream_t stream);

sss_status run(bool adj, const sss_params* p, const sss_walk_opts* o, void* ws, size_t wsb,
               sss_tallies* out, const sss_grad_in* gin, sss_grad_out* gout,
               sss_stream_t stream) {
  const sss_status r = run_impl(adj, p, o, ws, wsb, out, gin, gout, stream);
  if (r == SSS_OK) note_last_workspace(static_cast<cudaStream_t>(stream), ws);
  return r;
}

sss_status run_impl(bool adj, const sss_params* p, const sss_walk_opts* o, void* ws, size_t wsb,
                    sss_tallies* out, const sss_grad_in* gin, sss_grad_out* gout,
                    sss_stream_t stream) {
  if (!params_ok(p) || !opts_ok(o)) return SSS_ERR_INVALID_ARG;
  if ((uint64_t)o->instance_offset + (uint64_t)p->n_inst > 0x100000000ull)
    return SSS_ERR_INVALID_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1))) return SSS_ERR_INVALID_ARG;
  if (adj && !gout) return SSS_ERR_INVALID_ARG;
  if (o->hero_bands > 0) {
    // hero-wavelength sharing: forward, persistent schedule, one layer,
    // uniform path budgets, whole texels
    if (adj || o->schedule != 0 || p->alpha2) return SSS_ERR_UNSUPPORTED;
    if (p->n_paths || p->n_inst % o->hero_texel_bands != 0) return SSS_ERR_INVALID_ARG;
  }
  const Layout L = make_layout(p, o, adj);
  if (wsb < L.total) return SSS_ERR_WORKSPACE;
  int sms = 0;
  if (!device_ok(&sms)) return SSS_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // clear a stale error from unrelated work

  if (!o->use_graph) return enqueue_walk(adj, p, o, ws, L, out, gin, gout, sms, st);
  if (o->schedule == 1 && p->n_paths) return SSS_ERR_INVALID_ARG;  // needs a host sync

  std::string key;
  if (adj) {
    const void* ptrs[] = {gin ? gin->grad_R : nullptr, gin ? gin->grad_bins : nullptr,
                          gin ? gin->grad_R_k : nullptr, gin ? gin->grad_T : nullptr,
                          gout->d_alpha, gout->d_sigma_t, gout->d_g, gout->d_w,
                          gout->d_alpha2, gout->d_sigma_t2, gout->d_g2};
    key = graph_key(2, p, o, ws, wsb, ptrs, sizeof(ptrs) / sizeof(ptrs[0]), stream);
  } else {
    sss_tallies none{};
    const sss_tallies* tt = out ? out : &none;
    const void* ptrs[] = {tt->R, tt->T, tt->A, tt->bins, tt->overflow, tt->R_k, tt->R1,
                          tt->stderr_R, tt->stderr_bins, tt->truncated, tt->steps, tt->raw,
                          tt->profile};
    key = graph_key(1, p, o, ws, wsb, ptrs, sizeof(ptrs) / sizeof(ptrs[0]), stream);
  }
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_graphs.find(key);
    if (it != g_graphs.end()) exec = it->second;
  }
  if (!exec) {
    cudaStream_t cap = st;
    bool own = false;
    if (cap == nullptr) {  // the legacy stream cannot be captured
      if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return SSS_ERR_CUDA;
      own = true;
    }
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      if (own) cudaStreamDestroy(cap);
      return SSS_ERR_CUDA;
    }
    sss_status r = enqueue_walk(adj, p, o, ws, L, out, gin, gout, sms, cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    if (own) cudaStreamDestroy(cap);
    if (r != SSS_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return r != SSS_OK ? r : SSS_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return SSS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_graphs.find(key);
    if (it != g_graphs.end()) {  // another thread built the same plan meanwhile
      cudaGraphExecDestroy(exec);
      exec = it->second;
    } else {
      if (g_graphs.size() >= kMaxGraphs) {  // drop the oldest plan
        auto old = g_graphs.find(g_graph_order.front());
        if (old != g_graphs.end()) {
          cudaGraphExecDestroy(old->second);
          g_graphs.erase(old);
        }
        g_graph_order.erase(g_graph_order.begin());
      }
      g_graphs[key] = exec;
      g_graph_order.push_back(key);
    }
  }
  return cudaGraphLaunch(exec, st) == cudaSuccess ? SSS_OK : SSS_ERR_CUDA;
}

}  // namespace

extern "C" {

void sss_walk_opts_default(sss_walk_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->nbins = 64;
  o->r_max_mm = 10.0f;
  o->mode = 0;
  o->rr_threshold = 1.0f / 16.0f;
  o->entry_fresnel = 1;
  o->max_steps = 1u << 16;
  o->seed = 0;
  o->path_offset = 0;
  o->want_sumsq = 1;
  o->schedule = 0;
  o->use_graph = 0;
}

int32_t sss_tally_count(int32_t nbins, int32_t K, int32_t want_sumsq) {
  return tally_count(nbins, K, want_sumsq);
}

size_t sss_walk_workspace_size(const sss_params* p, const sss_walk_opts* o) {
  if (!params_ok(p) || !opts_ok(o)) return 0;
  return make_layout(p, o, false).total;
}

size_t sss_walk_bwd_workspace_size(const sss_params* p, const sss_walk_opts* o) {
  if (!params_ok(p) || !opts_ok(o)) return 0;
  return make_layout(p, o, true).total;
}

sss_status sss_walk(const sss_params* p, const sss_walk_opts* o, void* workspace,
                    size_t workspace_bytes, sss_tallies* out, sss_stream_t stream) {
  return run(false, p, o, workspace, workspace_bytes, out, nullptr, nullptr, stream);
}

sss_status sss_walk_bwd(const sss_params* p, const sss_walk_opts* o, void* workspace,
                        size_t workspace_bytes, const sss_grad_in* gin, sss_grad_out* gout,
                        sss_stream_t stream) {
  return run(true, p, o, workspace, workspace_bytes, nullptr, gin, gout, stream);
}

sss_status sss_read_status(const void* workspace, sss_stream_t stream, uint32_t* flags) {
  if (!workspace || !flags) return SSS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned int h = 0;
  if (cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SSS_ERR_CUDA;
  *flags = h;
  if (h & SSS_FLAG_TIMEOUT) return SSS_ERR_TIMEOUT;
  if (h & SSS_FLAG_PARAM) return SSS_ERR_DEVICE_PARAM;
  if (h & SSS_FLAG_OVERFLOW) return SSS_ERR_OVERFLOW;
  if (h & SSS_FLAG_STEP_LIMIT) return SSS_ERR_STEP_LIMIT;
  return SSS_OK;
}

sss_status sss_last_device_status(sss_stream_t stream, uint32_t* flags) {
  if (!flags) return SSS_ERR_INVALID_ARG;
  const void* ws = last_workspace(static_cast<cudaStream_t>(stream));
  if (!ws) return SSS_ERR_INVALID_ARG;
  return sss_read_status(ws, stream, flags);
}

sss_status sss_philox(const uint32_t* ctr, uint64_t key, int64_t n, uint32_t* out,
                      sss_stream_t stream) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return SSS_ERR_INVALID_ARG;
  if (!device_ok(nullptr)) return SSS_ERR_UNSUPPORTED;
  launch_philox(ctr, (uint32_t)(key & 0xffffffffull), (uint32_t)(key >> 32), n, out,
                static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? SSS_OK : SSS_ERR_CUDA;
}

void sss_profile_events(void* start, void* stop) {
  g_ev_start = static_cast<cudaEvent_t>(start);
  g_ev_stop = static_cast<cudaEvent_t>(stop);
}

void sss_release_plans(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : g_graphs) cudaGraphExecDestroy(kv.second);
  g_graphs.clear();
  g_graph_order.clear();
}

const char* sss_status_string(sss_status s) {
  switch (s) {
    case SSS_OK: return "ok";
    case SSS_ERR_INVALID_ARG: return "invalid argument";
    case SSS_ERR_CUDA: return "CUDA runtime error";
    case SSS_ERR_WORKSPACE: return "workspace too small";
    case SSS_ERR_STEP_LIMIT: return "some paths hit the step cap";
    case SSS_ERR_OVERFLOW: return "fixed-point accumulator saturated";
    case SSS_ERR_DEVICE_PARAM: return "parameter value out of range";
    case SSS_ERR_UNSUPPORTED: return "unsupported device or feature";
    case SSS_ERR_TIMEOUT: return "a bounded device wait gave up";
    case SSS_ERR_TOO_LARGE:
      return "problem needs more scratch than the no-allocation entry point's built-in array";
  }
  return "unknown status";
}

int32_t sss_abi_version(void) { return SSS_ABI_VERSION; }

}  // extern "C"

namespace sss {
void note_last_workspace(cudaStream_t stream, const void* workspace) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_last_ws[stream] = workspace;
}
const void* last_workspace(cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_last_ws.find(stream);
  return it == g_last_ws.end() ? nullptr : it->second;
}
}  // namespace sss
