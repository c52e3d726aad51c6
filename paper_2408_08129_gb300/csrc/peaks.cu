// Arithmetic-throughput probes of the GPU the library runs on: independent
// fused multiply-add chains in FP64 or FP32 on every SM, for the ALU peaks
// the operator kernels are measured against.  No counterpart in the paper.
#include "dg_internal.h"

namespace dg {
namespace {

constexpr int kChains = 16;  // independent FMA chains per thread

// Every thread runs kChains independent chains x <- x * a + b for iters steps;
// a = 1 - 2^-20 and b = 2^-30 keep the values bounded away from overflow and
// denormals.  The sum is written out so that nothing is optimised away.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* __restrict__ out, int64_t iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(1) + T(c) * T(1e-3) + T(threadIdx.x) * T(1e-6);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace dg

using namespace dg;

extern "C" int dg_peak_fma(int precision, int64_t iters, int blocks, void* out, void* stream, double* flops) {
  if (!out || !flops || iters < 1 || blocks < 1) return fail(DG_EINVAL, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == DG_FP64)
    fma_probe_kernel<double><<<blocks, 256, 0, s>>>((double*)out, iters, 1.0 - 0x1p-20, 0x1p-30);
  else if (precision == DG_FP32)
    fma_probe_kernel<float><<<blocks, 256, 0, s>>>((float*)out, iters, 1.0f - 0x1p-20f, 0x1p-30f);
  else
    return fail(DG_EINVAL, "bad precision");
  DG_CUDA(cudaGetLastError());
  *flops = 2.0 * kChains * (double)iters * 256.0 * (double)blocks;
  return DG_OK;
}
