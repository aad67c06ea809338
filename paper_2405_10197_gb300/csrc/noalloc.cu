// forte_sigma_fp64_noalloc: the FP64 sigma build for callers that must not
// allocate device memory during the call.
//
// Who needs it: code whose device memory belongs to another allocator (a
// framework's caching allocator that has reserved the GPU, or a process held
// to a fixed memory budget), and latency-critical loops in which a cudaMalloc
// or cudaFree -- which may synchronise the whole device -- is not acceptable.
// forte_sigma grows a per-context scratch buffer with cudaMalloc on demand;
// this variant instead uses one fixed array compiled into the library.
//
// The array below is a file-scope __device__ variable: every GPU on which the
// library is loaded holds its 16 MB until the process exits.  Host code cannot
// use the symbol's host-side name as a device address, so the first call on a
// device looks up the real address with cudaGetSymbolAddress (with that device
// current) and caches it; that first call should therefore come before any
// stream capture.  The cached address belongs to the device's primary context:
// after cudaDeviceReset (or any teardown of that context) it is stale and this
// entry point must not be called again in the process.  All calls share the
// array: calls that overlap on the GPU (e.g. issued concurrently on two streams)
// race on it.  Each call overwrites the scratch it reads, so nothing needs
// clearing between calls.  The kernels are those of forte_sigma in FP64 (one
// shared host body), traced like them when forte_profile_enable is on.
#include <mutex>

#include "forte_internal.h"

namespace {

constexpr long long kNoallocMaxElems = 1LL << 20;  // nvec * N_det per call (two arrays of this size)

__device__ __align__(256) double g_sigma_scratch[2 * kNoallocMaxElems];

std::mutex g_mu;
constexpr int kMaxDevices = 256;
double *g_addr[kMaxDevices] = {nullptr};

}  // namespace

using namespace forte;

extern "C" int forte_sigma_fp64_noalloc(forte_ctx *ctx, const double *C, double *S, int nvec) {
  if (!ctx) { set_error("NULL context"); return FORTE_ERR_ARG; }
  if (nvec < 0) { set_error("nvec < 0"); return FORTE_ERR_ARG; }
  if (nvec == 0) return FORTE_OK;
  if (!C || !S) { set_error("C and S must be device pointers"); return FORTE_ERR_ARG; }
  if ((long long)nvec * ctx->Ndet > kNoallocMaxElems) {
    set_error("forte_sigma_fp64_noalloc: nvec * N_det = %lld exceeds the built-in scratch limit of %lld",
              (long long)nvec * ctx->Ndet, kNoallocMaxElems);
    return FORTE_ERR_ARG;
  }
  const char *c0 = (const char *)C, *c1 = c0 + sizeof(double) * ctx->Ndet * nvec;
  const char *s0 = (const char *)S, *s1 = s0 + sizeof(double) * ctx->Ndet * nvec;
  if (c0 < s1 && s0 < c1) { set_error("S overlaps C"); return FORTE_ERR_ARG; }
  const int dev = ctx->device;
  if (dev < 0 || dev >= kMaxDevices) { set_error("device index %d out of range", dev); return FORTE_ERR_ARG; }
  double *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      int cur = -1;
      FORTE_CUDA_TRY(cudaGetDevice(&cur));
      if (cur != dev) FORTE_CUDA_TRY(cudaSetDevice(dev));
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_sigma_scratch);
      if (cur != dev) cudaSetDevice(cur);
      if (e != cudaSuccess || !p) {
        set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
        return FORTE_ERR_CUDA;
      }
      g_addr[dev] = (double *)p;
    }
    base = g_addr[dev];
  }
  return sigma_fp64_scratch(ctx, C, S, nvec, base, base + kNoallocMaxElems);
}
