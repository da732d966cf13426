// noalloc.cu -- bkfac_apply_noalloc: the damped inverse application with its
// scratch memory in a fixed device array owned by the library, for callers
// that cannot allocate device memory themselves.
//
// Some callers cannot call cudaMalloc (or hand a workspace to the library):
// code that runs while a stream is being captured into a CUDA graph in a mode
// that forbids calls which may synchronise the device; host frameworks whose
// device memory belongs to their own pool allocator and is not reachable
// through a plain C interface; and latency-critical loops where the implicit
// device-wide synchronisation of cudaMalloc / cudaFree is not acceptable.  For
// them this entry point runs bkfac_apply with the workspace placed in the
// file-scope array below, so the call allocates nothing.
//
// The array is a __device__ variable: every GPU that loads the library holds
// it (BKFAC_NOALLOC_SCRATCH_BYTES) until the process exits.  In host code its
// name is only a host-side stand-in, not a device address, so its device
// address is looked up with cudaGetSymbolAddress (with the device current) on
// the first call on each device and cached.  The cache is keyed on the device
// and on the unique id of its current context: a device reset destroys the
// context and the module with it, and the next call on that device looks the
// address up again in the new context.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"

namespace {

static __device__ __align__(256) unsigned char g_apply_scratch[BKFAC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// unique id of the calling thread's current context (0 when it cannot be read)
unsigned long long current_context_id() {
  static std::once_flag once;
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx) get_id(ctx, &id);
  return id;
}

// device address of g_apply_scratch on the current device (set up on first use in
// each context of the device)
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BKFAC_ECUDA;
  const unsigned long long ctx = current_context_id();  // 0 before the runtime's first use
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_apply_scratch) != cudaSuccess || !p) return BKFAC_ECUDA;
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = current_context_id();  // the context the lookup ran in
  }
  *out = g_scratch_ptr[dev];
  return BKFAC_OK;
}

}  // namespace

extern "C" int bkfac_apply_noalloc(const bkfac_factor* fA, const bkfac_factor* fG, double lamA, double lamG,
                                   const void* G, int64_t ldg, void* S, int64_t lds, uint32_t flags,
                                   bkfac_stream_t stream) {
  const size_t need = bkfac_apply_workspace_size(fA, fG);
  if (need == 0) return BKFAC_EINVAL;
  if (need > (size_t)BKFAC_NOALLOC_SCRATCH_BYTES) return BKFAC_EWORKSPACE;
  void* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != BKFAC_OK) return rc;
  // bkfac_apply writes every scratch byte it reads within the same call, so the
  // previous call's contents need no clearing.
  return bkfac_apply(fA, fG, lamA, lamG, G, ldg, S, lds, flags, scratch, (size_t)BKFAC_NOALLOC_SCRATCH_BYTES,
                     stream);
}
