// fhe_mult_relin_rescale_noalloc: the multiplication entry point for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they multiply: real-time or embedded hosts that forbid allocation after
// start-up (an allocation can block or fail at a bad moment), and plug-ins of
// other runtimes that must not touch the process's device allocator (it
// belongs to the host runtime, which accounts for every byte itself).  This entry point gives them fhe_mult_relin_rescale without a
// caller workspace: its scratch is one file-scope device array of
// kNoAllocScratchBytes (32 MiB), which every GPU that loads this library
// holds until the process exits.  Nothing here allocates: no cudaMalloc, no
// cudaFree, no allocator callback.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

// The scratch.  Host code must not pass this symbol to a kernel: on the host
// it is a stand-in, not a device address.  Its device address comes from
// cudaGetSymbolAddress below, once per device.
__device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up on the
// first call per device, with that device current).
int scratch_address(void** out) {
  int dev = 0;
  FHE_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    fhe::set_error("noalloc: device %d beyond the supported %d", dev, kMaxDevices);
    return FHE_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      fhe::set_error("noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return FHE_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return FHE_OK;
}

}  // namespace

extern "C" {

int fhe_mult_relin_rescale_noalloc(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, int k, fhe_ct* out,
                                   void* stream) {
  if (!ctx || !a || !b || !out) {
    fhe::set_error("mult_relin_rescale_noalloc: null argument");
    return FHE_EINVAL;
  }
  // the same argument errors as fhe_mult_relin_rescale, before any size or device question
  if (ctx->prm.scheme != FHE_SCHEME_CKKS || k < 1) {
    fhe::set_error("mult_relin_rescale_noalloc: CKKS only, k >= 1 (k = %d)", k);
    return FHE_EINVAL;
  }
  int dev = -1;
  FHE_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev != ctx->device) {
    fhe::set_error("mult_relin_rescale_noalloc: the context's device %d is not current (%d)", ctx->device, dev);
    return FHE_EINVAL;
  }
  const size_t need = fhe_workspace_bytes(ctx, FHE_OP_MULT, a->logQ, a->cnum);
  if (need == 0) {
    fhe::set_error("mult_relin_rescale_noalloc: bad level or batch size");
    return FHE_EINVAL;
  }
  if (need > kNoAllocScratchBytes) {
    fhe::set_error("mult_relin_rescale_noalloc: needs %zu bytes of scratch, the static scratch holds %zu "
                   "(use fhe_mult_relin_rescale with a workspace)",
                   need, kNoAllocScratchBytes);
    return FHE_EINVAL;
  }
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != FHE_OK) return rc;
  // Every scratch region is written before it is read, so stale contents from
  // an earlier call need no clearing.
  return fhe_mult_relin_rescale(ctx, a, b, k, out, scratch, kNoAllocScratchBytes, stream);
}

}  // extern "C"
