// Internal interface of the batched matched-filter kernel (mf_mma.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fpcg {

struct MfMmaParams {
  const float2* H;             // [n_groups][K][N] complex64
  const float2* y;             // [n_rhs][N], grouped
  const int64_t* group_start;  // device [n_groups + 1]
  float2* b;                   // [n_rhs][K] out
  int N, K;
  int64_t n_groups;
};

bool mf_mma_supported(int K);  // K in {8, 16, 32, 64, 128} (8: padded to 16)
cudaError_t launch_mf_mma(const MfMmaParams& P, int bf16, cudaStream_t stream);

}  // namespace fpcg
