// noalloc.cu -- fsp_rhs_noalloc: the right-hand side for callers that cannot allocate
// device memory.
//
// fsp_rhs needs scratch memory (the per-line maxima of the splitting and the xi-direction
// accumulator) and takes it from a workspace the caller allocates.  Some callers cannot do
// that: a solver plugin inside a host application that owns every device allocation (its
// own pool, no cudaMalloc allowed to the plugin), code in a real-time loop where a
// cudaMalloc/cudaFree would synchronise the device, or a caller with no allocator of its
// own at all.  For them this file keeps the scratch in one fixed array in device memory,
// declared here at file scope, so the call itself allocates nothing.
//
// The array is FSP_NOALLOC_SCRATCH_BYTES (8 MiB) and every GPU that loads the library
// holds it until the process exits.  All calls share it, so calls that overlap on the GPU
// (different streams, or different host threads on one device) race on it and must be
// serialised by the caller.  The array keeps the previous call's contents; the per-line
// maxima are cleared at the start of every call, and the accumulator is fully overwritten.
#include <mutex>

#include "fsp_internal.h"

namespace fsp {
namespace {

constexpr size_t kScratchBytes = FSP_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch.  Host code must not pass `scratch` itself to a kernel: on the host this
// name is only a stand-in for the device symbol, so its device address is looked up with
// cudaGetSymbolAddress once per device (scratch_address below).
static __device__ __align__(256) unsigned char scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of `scratch` on the current device, looked up on the first call per
// device (the lookup may load the module, so that first call must not be inside a stream
// capture).  The address is cached per device index for the primary context: a caller that
// resets the device (cudaDeviceReset) or switches to another context between calls would be
// handed a stale address, so such callers must not use this entry point across a reset.
fsp_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FSP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, scratch);
    if (e != cudaSuccess || !p) return FSP_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return FSP_OK;
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace fsp

using namespace fsp;

extern "C" fsp_status fsp_rhs_noalloc(const fsp_config* cfg, const fsp_block* blk,
                                      const double* metrics, const void* Q, void* dQdt,
                                      void* stream) {
  size_t ws_bytes = 0;
  if (fsp_status s = fsp_workspace_size(cfg, blk, &ws_bytes)) return s;  // checks cfg and blk
  if (!on_device(metrics) || !on_device(Q) || !on_device(dQdt) || Q == dQdt) return FSP_ERR_INVALID_ARG;
  if (cfg->precision != FSP_FP64) return FSP_ERR_UNSUPPORTED;

  // scratch layout: per-line maxima (nj + ni doubles), then the xi accumulator
  const size_t lam_bytes = ((size_t)blk->ni + blk->nj) * sizeof(double);
  const size_t acc_off = (lam_bytes + 255) / 256 * 256;
  const size_t acc_bytes = 4 * (size_t)blk->nj * (size_t)blk->ld * sizeof(double);
  if (acc_off + acc_bytes > kScratchBytes) return FSP_ERR_NOMEM;  // block too large for the array

  void* base = nullptr;
  if (fsp_status s = scratch_address(&base)) return s;
  double* lam = static_cast<double*>(base);
  void* acc = static_cast<char*>(base) + acc_off;

  const Params P = make_params(*cfg, *blk, metrics);

  cudaStream_t st = (cudaStream_t)stream;
  // the maxima are accumulated by atomic max and must start at zero on every call
  if (cudaMemsetAsync(lam, 0, lam_bytes, st) != cudaSuccess) return FSP_ERR_CUDA;
  if (launch_lambda(P, cfg->precision, Q, lam, lam + blk->nj, nullptr, st) != cudaSuccess) return FSP_ERR_CUDA;
  return rhs_status(launch_rhs(cfg->scheme, cfg->precision, P, Q, lam, lam + blk->nj, acc, dQdt, 0, nullptr,
                               0.0, 0.0, 0.0, st));
}
