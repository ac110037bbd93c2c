// kde_lscv_noalloc: LSCV_h selection for callers that cannot allocate device
// memory themselves.
//
// Who needs this: code that runs inside a host application or framework that
// owns the whole device heap (its allocator must be the only one), code on a
// latency-critical path where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable, and plain C callers with no tensor
// library to hand them a workspace.  They still pass their samples and read
// their results; only the scratch space (descriptor, prepared samples,
// partial sums) comes from a buffer compiled into this library.
//
// The buffer is a file-scope __device__ array of KDE_NOALLOC_MAX_BYTES bytes.
// Every GPU that loads the library holds it until the process exits.  Its
// device address is looked up once per CUDA context, with that context
// current, by the first call made in it (cudaGetSymbolAddress); make that
// first call before any stream capture.  The address belongs to the context
// that loaded the module: after cudaDeviceReset, or when the primary context
// is released and created again, the module can load at another address, so
// the cache is keyed on the context's unique ID (cuCtxGetId) and a call in a
// new context looks the address up again.  All calls share the one buffer and it keeps
// the previous call's contents; nothing in it needs to start at zero (every
// value the kernels read is written earlier in the same call).  Calls that
// overlap on the GPU (different streams, or host threads, without ordering
// between them) race on the buffer: serialise them.
#include <cuda.h>

#include <mutex>

#include "gbkde.h"
#include "host.hpp"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[KDE_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;

// One cached address per device slot, valid only for the context it was
// looked up in (context IDs are unique for the life of the process).
struct ScratchSlot {
  unsigned long long ctx_id;
  void* ptr;
};
ScratchSlot g_slot[kMaxDevices] = {};

// Driver entry points for the current context and its ID, resolved through
// the runtime so the library needs no link against the driver library.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

int resolve_driver_entry_points() {
  if (g_ctx_get_current && g_ctx_get_id) return KDE_OK;
  void* a = nullptr;
  void* b = nullptr;
  cudaDriverEntryPointQueryResult qa = cudaDriverEntryPointSymbolNotFound;
  cudaDriverEntryPointQueryResult qb = cudaDriverEntryPointSymbolNotFound;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
  if (e != cudaSuccess || qa != cudaDriverEntryPointSuccess || !a)
    return gbkde::cuda_fail(e, "cudaGetDriverEntryPointByVersion(cuCtxGetCurrent)");
  e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
  if (e != cudaSuccess || qb != cudaDriverEntryPointSuccess || !b)
    return gbkde::cuda_fail(e, "cudaGetDriverEntryPointByVersion(cuCtxGetId)");
  g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
  g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(b);
  return KDE_OK;
}

// ID of the context current on this thread; 0 when none is current yet.
int current_context_id(unsigned long long* id) {
  CUcontext ctx = nullptr;
  CUresult r = g_ctx_get_current(&ctx);
  if (r != CUDA_SUCCESS) return gbkde::fail(KDE_ECUDA, "cuCtxGetCurrent failed (%d)", (int)r);
  *id = 0;
  if (!ctx) return KDE_OK;
  r = g_ctx_get_id(ctx, id);
  if (r != CUDA_SUCCESS) return gbkde::fail(KDE_ECUDA, "cuCtxGetId failed (%d)", (int)r);
  return KDE_OK;
}

// Device address of the scratch array in the current context (set-up on the
// first call in each context).
int scratch_for_current_context(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gbkde::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return gbkde::fail(KDE_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = resolve_driver_entry_points();
  if (rc) return rc;
  unsigned long long id = 0;
  rc = current_context_id(&id);
  if (rc) return rc;
  if (id == 0 || g_slot[dev].ctx_id != id || !g_slot[dev].ptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the device's context current
    if (e != cudaSuccess || !p) return gbkde::cuda_fail(e, "cudaGetSymbolAddress");
    rc = current_context_id(&id);
    if (rc) return rc;
    if (id == 0) return gbkde::fail(KDE_ECUDA, "no current CUDA context after cudaGetSymbolAddress");
    g_slot[dev].ctx_id = id;
    g_slot[dev].ptr = p;
  }
  *out = g_slot[dev].ptr;
  return KDE_OK;
}

}  // namespace

extern "C" int kde_lscv_noalloc(const void* x_dev, int dtype, int64_t n, int d, const kde_grid* grid,
                                const kde_opts* opts, void* stream, double* g_host, double* h_host,
                                kde_result* out) {
  if (!grid) return gbkde::fail(KDE_EINVAL, "grid is NULL");
  size_t need = 0;
  int rc = kde_workspace_size(n, d, grid->n_h, opts, &need);
  if (rc) return rc;
  if (need > (size_t)KDE_NOALLOC_MAX_BYTES)
    return gbkde::fail(KDE_ENOMEM,
                       "kde_lscv_noalloc: n = %lld, d = %d, n_h = %d needs %zu bytes of scratch, more "
                       "than the built-in %d; use kde_lscv with a caller workspace",
                       (long long)n, d, grid->n_h, need, KDE_NOALLOC_MAX_BYTES);
  void* scratch = nullptr;
  rc = scratch_for_current_context(&scratch);
  if (rc) return rc;
  return kde_lscv(x_dev, dtype, n, d, grid, opts, scratch, (size_t)KDE_NOALLOC_MAX_BYTES, stream,
                  g_host, h_host, out);
}
