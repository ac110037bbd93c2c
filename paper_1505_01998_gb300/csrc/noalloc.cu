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
// device address is looked up once per device, with that device current, by
// the first call made on that device (cudaGetSymbolAddress); make that first
// call before any stream capture.  All calls share the one buffer and it keeps
// the previous call's contents; nothing in it needs to start at zero (every
// value the kernels read is written earlier in the same call).  Calls that
// overlap on the GPU (different streams, or host threads, without ordering
// between them) race on the buffer: serialise them.
#include <mutex>

#include "gbkde.h"
#include "host.hpp"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[KDE_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (set-up on the
// first call per device).
int scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gbkde::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return gbkde::fail(KDE_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return gbkde::cuda_fail(e, "cudaGetSymbolAddress");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
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
  rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  return kde_lscv(x_dev, dtype, n, d, grid, opts, scratch, (size_t)KDE_NOALLOC_MAX_BYTES, stream,
                  g_host, h_host, out);
}
