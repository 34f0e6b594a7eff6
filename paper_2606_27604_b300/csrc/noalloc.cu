// noalloc.cu -- sss_walk_noalloc: the forward walk for callers that cannot
// allocate device memory.
//
// Some hosts that embed this library cannot hand it a workspace: a renderer
// plug-in running inside an application that owns every device allocation
// through its own pool, or code on a real-time or capture-sensitive thread
// where a cudaMalloc (which may synchronise the device) is not allowed.  For
// them this entry point runs the same forward walk as sss_walk, with its
// scratch (status word, work-queue head, fixed-point accumulators) in a
// fixed array that lives in the library's own device memory.  The paper has
// no counterpart to this; it is a deployment convenience.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds SSS_NOALLOC_SCRATCH_BYTES of it until the process exits.  In
// host code its name is only a host-side stand-in, not a device address; the
// address is obtained with cudaGetSymbolAddress (with the device current) on
// the first call on a device and cached.  The cache is keyed by the CUDA
// context's unique id as well, so after a cudaDeviceReset (which ends the
// context and with it the array's old address) the next call looks the
// address up again instead of handing a stale one to the kernels.
#include <cuda.h>  // CUcontext / CUresult types only; driver calls go through entry points
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/sss.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SSS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx[kMaxDevices] = {0};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the current CUDA context, or 0 if there is none yet (or the
// driver does not report one).
unsigned long long current_context_id() {
  static std::once_flag once;
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array on the current device: looked up on
// the first call for that device (and again when its context has changed).
sss_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SSS_ERR_UNSUPPORTED;
  if (dev < 0 || dev >= kMaxDevices) return SSS_ERR_UNSUPPORTED;
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
      return SSS_ERR_CUDA;
    g_addr[dev] = p;
    g_ctx[dev] = ctx != 0 ? ctx : current_context_id();  // the lookup creates the context
  }
  *out = g_addr[dev];
  return SSS_OK;
}

}  // namespace

extern "C" sss_status sss_walk_noalloc(const sss_params* p, const sss_walk_opts* o,
                                       sss_tallies* out, uint32_t* status_flags,
                                       sss_stream_t stream) {
  if (!p || !o) return SSS_ERR_INVALID_ARG;
  // only the direct persistent path: the plain baseline copies budgets to a
  // host vector and the graph path instantiates graphs
  if (o->schedule != 0 || o->use_graph != 0) return SSS_ERR_INVALID_ARG;
  const size_t need = sss_walk_workspace_size(p, o);
  if (need == 0) return SSS_ERR_INVALID_ARG;
  if (need > (size_t)SSS_NOALLOC_SCRATCH_BYTES) return SSS_ERR_TOO_LARGE;
  void* scratch = nullptr;
  sss_status s = scratch_address(&scratch);
  if (s != SSS_OK) return s;
  // sss_walk clears the status word and the accumulators before it starts
  s = sss_walk(p, o, scratch, (size_t)SSS_NOALLOC_SCRATCH_BYTES, out, stream);
  if (s != SSS_OK || status_flags == nullptr) return s;
  return sss_read_status(scratch, stream, status_flags);
}
