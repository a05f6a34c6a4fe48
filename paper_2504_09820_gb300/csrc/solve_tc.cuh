// Internal interface of the tensor-core solver for given Gram matrices.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "detect_tc.cuh"

namespace fpcg {

struct SolveTcParams {
  DetectTcParams D;           // iteration settings and outputs (D.pipe only gives N, K, batch)
  const float2* A;            // [n_groups][K][K] complex fp32: A_g + sigma_g^2 I
  const float2* b;            // [n][K] given right-hand sides, or null: matched filter from H, y
  const float2* H;            // [n_groups][K][N] complex64 (matched-filter mode)
  const float2* y;            // [n][N] complex64 (matched-filter mode)
  const int64_t* group_start; // device [n_groups + 1]: systems of group g are [start[g], start[g+1]);
                              // null: system s uses group s
  int64_t n, n_groups;
  int N, K, gram;             // gram: rounding of H and y in the matched filter
};

// K in {16, 32, 64, 128}, L in {0, 4, 8, 16}: the CG warp's configurations.
inline bool solve_tc_supported(int K, int L) {
  return (K == 16 || K == 32 || K == 64 || K == 128) && (L == 0 || L == 4 || L == 8 || L == 16);
}

constexpr int kSolveWarps = 8;  // CG warps per CTA (grouped mode, and independent systems for K <= 64)

// Independent systems: one slot per warp; K = 128 slots (~80 KB) allow two per CTA.
__host__ __device__ constexpr int solve_warps(int K) { return K == 128 ? 2 : kSolveWarps; }

inline size_t solve_tc_smem_bytes(int K, int L) { return 128 + solve_warps(K) * tc_slot_bytes(K, L); }

// Grouped mode (fpcg_detect_grouped): all warps of a CTA share one group's A
// and inverted blocks; each warp has its own b, matvec result and B fragments.
inline bool solve_grouped_supported(int K, int L) {
  return (K == 16 || K == 32 || K == 64 || K == 128) && (L == 0 || L == 4 || L == 8 || L == 16);
}

__host__ __device__ inline size_t md_bytes(int K, int L) {
  return L > 0 ? sizeof(float2) * (size_t)(K / L) * md_block_stride(L) : 16;
}

inline size_t solve_grouped_smem_bytes(int K, int L) {
  return 128 + 4 * (size_t)K * K + md_bytes(K, L) + kSolveWarps * (size_t)(16 * K + 12 * K) + 16;
}

template <int K>
cudaError_t launch_solve_grouped_k(const SolveTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream);
extern template cudaError_t launch_solve_grouped_k<16>(const SolveTcParams&, int, int, cudaStream_t);
extern template cudaError_t launch_solve_grouped_k<32>(const SolveTcParams&, int, int, cudaStream_t);
extern template cudaError_t launch_solve_grouped_k<64>(const SolveTcParams&, int, int, cudaStream_t);
extern template cudaError_t launch_solve_grouped_k<128>(const SolveTcParams&, int, int, cudaStream_t);

inline cudaError_t launch_solve_grouped(const SolveTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream) {
  switch (P.K) {
    case 128: return launch_solve_grouped_k<128>(P, num_sms, mv_bf16, stream);
    case 64: return launch_solve_grouped_k<64>(P, num_sms, mv_bf16, stream);
    case 32: return launch_solve_grouped_k<32>(P, num_sms, mv_bf16, stream);
    case 16: return launch_solve_grouped_k<16>(P, num_sms, mv_bf16, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <int K>
cudaError_t launch_solve_tc_k(const SolveTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream);
extern template cudaError_t launch_solve_tc_k<16>(const SolveTcParams&, int, int, cudaStream_t);
extern template cudaError_t launch_solve_tc_k<32>(const SolveTcParams&, int, int, cudaStream_t);
extern template cudaError_t launch_solve_tc_k<64>(const SolveTcParams&, int, int, cudaStream_t);
extern template cudaError_t launch_solve_tc_k<128>(const SolveTcParams&, int, int, cudaStream_t);

inline cudaError_t launch_solve_tc(const SolveTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream) {
  switch (P.K) {
    case 128: return launch_solve_tc_k<128>(P, num_sms, mv_bf16, stream);
    case 64: return launch_solve_tc_k<64>(P, num_sms, mv_bf16, stream);
    case 32: return launch_solve_tc_k<32>(P, num_sms, mv_bf16, stream);
    case 16: return launch_solve_tc_k<16>(P, num_sms, mv_bf16, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpcg
