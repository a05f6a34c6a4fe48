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
  int iters, L, refine_steps, refine_iters, alpha_num, ip;
  float2* x_hat;
  uint8_t* sym;
  double* rel_res;
  float* res_hist;
  const uint8_t* tx;
  unsigned long long* bit_errors;
  int32_t* status;
};

// Shared memory of one CG warpgroup (layout carved in detect_tc_impl.cuh):
// A [64][K+1], b/W/X/R [64], M_d [64][L+1] (c64), packed p [64] (u32), flags.
__host__ __device__ inline size_t cg_smem_bytes(int K, int L) {
  size_t s = 0;
  s += sizeof(float2) * 64 * (K + 1);
  s += sizeof(float2) * 64 * 4;
  s += sizeof(float2) * 64 * ((L > 0 ? L : 1) + 1);
  s += sizeof(uint32_t) * 64;
  s += sizeof(int) * 4;
  return (s + 127) & ~size_t(127);
}

// Offset of the first CG region after the stages, barriers and TMEM slot.
__host__ __device__ inline size_t cg_region_offset() {
  return (tcp::kPipeBytes + sizeof(tcp::Bars) + 16 + 127) & ~size_t(127);
}

inline size_t detect_tc_smem_bytes(int K, int L) {
  const size_t s = 1024 + cg_region_offset() + 2 * cg_smem_bytes(K, L);
  return s < 120 * 1024 ? 120 * 1024 : s;  // one CTA (one 512-column TMEM allocation) per SM
}

// K in {16, 32, 64}; L in {0 (FP-CG), 4, 8, 16}.
inline bool detect_tc_supported(int K, int L) {
  return (K == 16 || K == 32 || K == 64) && (L == 0 || L == 4 || L == 8 || L == 16);
}

template <int K>
cudaError_t launch_detect_tc_k(const DetectTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream);

inline cudaError_t launch_detect_tc(const DetectTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream) {
  switch (P.pipe.K) {
    case 64: return launch_detect_tc_k<64>(P, num_sms, mv_bf16, stream);
    case 32: return launch_detect_tc_k<32>(P, num_sms, mv_bf16, stream);
    case 16: return launch_detect_tc_k<16>(P, num_sms, mv_bf16, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpcg
