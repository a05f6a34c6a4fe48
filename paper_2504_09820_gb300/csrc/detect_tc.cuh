// Internal interface of the fused tensor-core detector.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tc_pipeline.cuh"

namespace fpcg {

struct DetectTcParams {
  tcp::Pipe pipe;
  const double* sigma2;
  const int32_t* qam;
  int iters, L, refine_steps, refine_iters, alpha_num, ip, resid_comp;
  float2* x_hat;
  uint8_t* sym;
  double* rel_res;
  float* res_hist;
  const uint8_t* tx;
  unsigned long long* bit_errors;
  int32_t* status;
};

bool detect_tc_supported(int K, int L);
size_t detect_tc_smem_bytes(int K, int L);
cudaError_t launch_detect_tc(const DetectTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream);

}  // namespace fpcg
