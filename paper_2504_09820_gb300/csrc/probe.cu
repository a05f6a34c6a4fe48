// Plain FMA throughput probe (fpcg_fma_probe): measures what the CUDA cores
// sustain in fp32 and fp64, the denominator of the SIMT kernels' roofline
// (the fp32 plain-CG comparator's Gram runs on these units, not on the tensor
// cores).  Each thread runs eight independent FMA chains, so the launch is
// bound by FMA issue, not by latency.
#include <cuda_runtime.h>
#include <stdint.h>

#include "api_internal.cuh"
#include "fpcg.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(T* out, int64_t iters) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = (T)(tid + c) * (T)1e-9;
  const T a = (T)0.999999, b = (T)1e-7;
#pragma unroll 1
  for (int64_t i = 0; i < iters; i += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[tid] = s;  // keeps the chains alive
}

}  // namespace

extern "C" FPCG_API int fpcg_fma_probe(int32_t fp64, int64_t iters, void* out, int64_t out_len, double* flops,
                                       void* stream) {
  if (!out || out_len < kThreads || out_len % kThreads || iters < 4 || iters % 4) return FPCG_EINVAL;
  if (out_len / kThreads > 0x7fffffff) return FPCG_EINVAL;
  if (((uintptr_t)out % (fp64 ? 8 : 4)) != 0) return FPCG_EINVAL;
  const unsigned grid = (unsigned)(out_len / kThreads);
  cudaStream_t s = (cudaStream_t)stream;
  if (fp64) fma_probe_kernel<double><<<grid, kThreads, 0, s>>>((double*)out, iters);
  else fma_probe_kernel<float><<<grid, kThreads, 0, s>>>((float*)out, iters);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fpcg::cuda_error(e);
  if (flops) *flops = 2.0 * kChains * (double)iters * (double)out_len;
  return FPCG_OK;
}
