// Internal interface of the mma.sync Gram kernel (gram_mma.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fpcg {

struct GramMmaParams {
  const float2* H;       // [batch][K][N] complex64
  const float2* y;       // [batch][N]
  const double* sigma2;  // [batch]
  float2* A;             // [batch][K][K]
  float2* b;             // [batch][K]
  int N, K;
  int64_t batch;
};

bool gram_mma_supported(int K);  // K in {8, 16, 32, 64, 128} (8: padded to 16)
cudaError_t launch_gram_mma(const GramMmaParams& P, int bf16, cudaStream_t stream);

}  // namespace fpcg
