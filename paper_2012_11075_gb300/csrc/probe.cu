// Measurement aid: the FP64 fused multiply-add rate of the device, the
// ceiling of the float64 step kernel (whose time goes to FP64 arithmetic, not
// to memory traffic).  The paper has no counterpart of this entry point.
//
// Every thread runs eight independent chains a <- a * m + c (m slightly below
// one, c small, so the values stay normal and bounded) and writes the sum of
// its chains, so that no chain can be removed.  One launch performs
// blocks * threads * iters * 8 fused multiply-adds (16 flops each pair).
#include <cuda_runtime.h>

#include "../../include/wblbe.h"
#include "lbm_kernels.cuh"

namespace {

__global__ void reciprocal_kernel(const double* __restrict__ x, double* __restrict__ seed,
                                  double* __restrict__ refined, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (seed) seed[i] = wblbe::recip_seed(x[i]);
  if (refined) refined[i] = wblbe::recip(x[i]);
}

constexpr int kChains = 8;

__global__ void __launch_bounds__(1024) fp64_fma_kernel(double* __restrict__ out, int iters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * k + 1e-9 * t;
  const double m = 0.9999999999, c = 1e-10;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[t] = s;
}

}  // namespace

extern "C" wblbe_status wblbe_probe_fp64_fma(double* out, int32_t blocks, int32_t threads,
                                             int32_t iters, void* cuda_stream) {
  if (!out || blocks < 1 || threads < 32 || threads > 1024 || (threads % 32) != 0 || iters < 1)
    return WBLBE_EINVAL;
  fp64_fma_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(out, iters);
  return cudaGetLastError() == cudaSuccess ? WBLBE_OK : WBLBE_ECUDA;
}

extern "C" wblbe_status wblbe_probe_reciprocal(const double* x, double* seed, double* refined,
                                               int64_t n, void* cuda_stream) {
  if (!x || n < 0 || (!seed && !refined)) return WBLBE_EINVAL;
  if (n == 0) return WBLBE_OK;
  const long long blocks = (n + 255) / 256;
  if (blocks > 0x7fffffffLL) return WBLBE_EINVAL;
  reciprocal_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      x, seed, refined, (long long)n);
  return cudaGetLastError() == cudaSuccess ? WBLBE_OK : WBLBE_ECUDA;
}
