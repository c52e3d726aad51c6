// Helmholtz mat-vec for callers that cannot allocate device memory.
//
// dg_apply_implicit needs one scratch buffer (the h-scaled gradient between
// its gradient and divergence launches); it takes it from the mesh.  This
// variant takes it instead from a fixed array in the library's own device
// image, so the call itself performs no allocation of any kind.  Callers that cannot call cudaMalloc -- code
// running under an allocator that forbids it, inside a memory budget that is
// already fully committed, or a host framework that owns every allocation --
// can still apply the operator.
#include <mutex>

#include "ops.h"

namespace {

// Maximum scratch per device: 4 MiB.  Every GPU that loads the library holds
// this array until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)4 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of g_noalloc_scratch on `device`.  In host code the array's
// name is only a host stand-in, never a device address, so it is never passed
// to a kernel.  The address is looked up with the device current on the first
// call, and again on every later call that is not being captured into a CUDA
// graph (a cheap lookup), so that a call after a device reset, which reloads
// the module, does not use a stale address; during a capture the address
// recorded before it is used.
int scratch_address(int device, cudaStream_t s, void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (device < 0 || device >= kMaxDevices) return dg::fail(DG_EINVAL, "device ordinal out of range");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (g_scratch_addr[device] && cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone) {
    *out = g_scratch_addr[device];
    return DG_OK;
  }
  int cur = 0;
  DG_CUDA(cudaGetDevice(&cur));
  if (cur != device) DG_CUDA(cudaSetDevice(device));
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (cur != device) cudaSetDevice(cur);
  if (e != cudaSuccess) return dg::cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
  g_scratch_addr[device] = p;
  *out = p;
  return DG_OK;
}

}  // namespace

using namespace dg;

extern "C" int dg_apply_implicit_noalloc(dg_ctx* ctx, const dg_mesh* m, const void* h, const void* p, void* Ap,
                                         double alpha, int precision, void* stream) {
  if (!ctx || !m || !h || !p || !Ap) return fail(DG_EINVAL, "null argument");
  if (precision != DG_FP64 && precision != DG_FP32) return fail(DG_EINVAL, "bad precision");
  const size_t elem = precision == DG_FP64 ? sizeof(double) : sizeof(float);
  const size_t need = (size_t)m->dim * m->Nn * elem;
  if (need > kNoAllocScratchBytes)
    return fail(DG_EINVAL, "mesh too large for dg_apply_implicit_noalloc: needs " + std::to_string(need) +
                               " bytes of scratch, the static maximum is " + std::to_string(kNoAllocScratchBytes));
  void* base = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = scratch_address(ctx->device, s, &base);
  if (rc != DG_OK) return rc;
  if (precision == DG_FP64)
    return op_helmholtz<double>(m, (const double*)h, (const double*)p, (double*)Ap, alpha, (double*)base, s,
                                nullptr);
  return op_helmholtz<float>(m, (const float*)h, (const float*)p, (float*)Ap, (float)alpha, (float*)base, s,
                             nullptr);
}
