// rsvd_small_svd_noalloc: the small-SVD step with its scratch in a static
// device array instead of a caller workspace.
//
// Some callers cannot allocate device memory for us or hand us a workspace:
// cudaMalloc and cudaFree synchronise the whole device, which a caller running
// a latency-bound loop next to other streams cannot afford, and some host
// frameworks own the entire device-memory budget and forbid libraries from
// calling the CUDA allocator at all.  This entry point needs nothing but the
// input and output pointers: its scratch is a file-scope __device__ array of
// RSVD_NOALLOC_SCRATCH_BYTES that every GPU which loads the library keeps until
// the process exits.
//
// The array's name is only a host-side stand-in in host code; its device
// address is looked up once per device with cudaGetSymbolAddress, with that
// device current, on the first call made on that device (do that first call
// before any stream capture).  The address is cached for the life of the
// process: after a cudaDeviceReset the module, and with it the array, is
// reloaded elsewhere, so the entry point must not be called on that device
// again.  All calls share the one array and it keeps the
// last call's contents; calls that overlap on the GPU (different streams, or
// host threads racing) race on it and must be serialised by the caller.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = RSVD_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device (set up once).
rsvd_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RSVD_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return RSVD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RSVD_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return RSVD_OK;
}

}  // namespace

extern "C" rsvd_status rsvd_small_svd_noalloc(int l, int dtype, const void* M, int64_t ldm,
                                              void* Uh, int64_t lduh, double* Sh, void* Vh,
                                              int64_t ldvh, int* d_info, void* stream,
                                              const rsvd_opts* opts) {
  if (l < 1 || l > 1024 || (dtype != RSVD_F32 && dtype != RSVD_F64)) return RSVD_ERR_INVALID_ARG;
  if (!M || !Uh || !Sh || !Vh || ldm < l || lduh < l || ldvh < l) return RSVD_ERR_INVALID_ARG;
  const size_t need = rsvd_small_svd_workspace_size(l, dtype, opts);
  if (need == 0) return RSVD_ERR_INVALID_ARG;
  if (need > kScratchBytes) return RSVD_ERR_WORKSPACE;   // l too large for the static scratch
  void* scratch = nullptr;
  const rsvd_status st = scratch_address(&scratch);
  if (st != RSVD_OK) return st;
  // Nothing in the scratch needs to start at zero: every buffer carved from it
  // is written by a kernel of this call before any kernel reads it.
  return rsvd_small_svd(l, dtype, M, ldm, Uh, lduh, Sh, Vh, ldvh, scratch, kScratchBytes, d_info,
                        stream, opts);
}
