// Internal interface of the generic SIMT detector (one CTA per system).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fpcg {

struct SimtParams {
  const float2* H;          // [batch][K][N] c64, or null with Ain
  const float2* y;          // [batch][N] c64
  const double* sigma2;     // [batch]
  const int32_t* qam;       // [batch], may be null when sym and bit_errors are null
  const void* Ain;          // [batch][K][K] given Gram (fpcg_solve_gram) or null
  const void* bin;          // [batch][K] given right-hand side
  const int32_t* a_map;     // shared-Gram mode (with Ain, H, y): system i uses A and H number a_map[i]
  const int64_t* group_start;  //   or, grouped: the systems of group g are [group_start[g], group_start[g+1])
  int64_t n_shared;         //   number of shared Gram matrices (bound of a_map)
  int N, K, iters, L, refine_steps, refine_iters, alpha_num, gram, ip, resid_fp64;
  int64_t batch;
  void* x_hat;
  uint8_t* sym;
  double* rel_res;
  float* res_hist;
  const uint8_t* tx;
  unsigned long long* bit_errors;
  int32_t* status;
  void* A_out;              // gram-only mode: write A [batch][K][K] and b, then stop
  void* b_out;
  float* coeffs;            // [batch][2][iters] or null: alpha_j, beta_j of the main solve
};

size_t simt_smem_bytes(int fp64, int K, int L, int mv);
cudaError_t launch_detect_simt(const SimtParams& P, int fp64, int mv, cudaStream_t stream);

}  // namespace fpcg
