// Internal interface of the tensor-core Gram kernel.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tc_pipeline.cuh"

namespace fpcg {

struct GramTcParams {
  tcp::Pipe pipe;
  const double* sigma2;
  float2* A;        // [batch][K][K] row-major
  float2* b;        // [batch][K]
  int32_t* status;  // nullable: FPCG_ST_TIMEOUT for systems a timed-out CTA left
};

bool gram_tc_supported(int K);
size_t gram_tc_smem_bytes();
// The TMA pipeline needs N even and 16-byte aligned H and y.
bool tma_pipe_ok(const void* H, const void* y, int N);
// SM cycles a tensor-core pipeline wait may take (FPCG_TC_WAIT_CYCLES, else ~2 s).
long long wait_budget_cycles();
// Fill the pipeline description (tensor maps included); false if the driver
// refused a tensor map.
bool make_pipe(tcp::Pipe* p, const float2* H, const float2* y, int N, int K, int64_t batch, int bf16);
cudaError_t launch_gram_tc(const GramTcParams& P, int num_sms, cudaStream_t stream);

// K = 128 (gram_tc128.cu): one system per tile, the real and imaginary parts
// of A in two TMEM accumulators.
struct GramTc128Params {
  CUtensorMap tmH;  // FP32 view of H: dims {2N, batch*128}, box {64, 128}
  CUtensorMap tmY;  // FP32 view of y: dims {2N, batch}, box {64, 1}
  CUtensorMap tmA;  // FP32 view of A: dims {256, batch*128}, box {32, 128}, 128-byte swizzle (stores)
  const float2* H;
  const double* sigma2;
  float2* A;        // [batch][128][128] row-major
  float2* b;        // [batch][128]
  int32_t* status;  // nullable: FPCG_ST_TIMEOUT for systems a timed-out CTA left
  int N, nchunks;   // nchunks = ceil(N / 64)
  int64_t batch;
  int bf16;
};
bool make_gram_tc128(GramTc128Params* p, const float2* H, const float2* y, float2* A, int N, int64_t batch,
                     int bf16);
size_t gram_tc128_smem_bytes();
cudaError_t launch_gram_tc128(const GramTc128Params& P, int num_sms, cudaStream_t stream);

}  // namespace fpcg
