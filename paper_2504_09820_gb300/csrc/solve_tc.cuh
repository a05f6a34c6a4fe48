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
                              // null: system s uses group s (or a_map[s])
  const int32_t* a_map;       // device [n] or null: group of system s (independent-systems kernel; an
                              // index outside [0, n_groups) gives x_hat = 0 and FPCG_ST_BAD_INDEX)
  int64_t n, n_groups;
  int N, K, gram;             // gram: rounding of H and y in the matched filter
};

// K in {8, 16, 32, 64, 128}, L in {0, 4, 8, 16} (L <= K): the CG warp's
// configurations.  K = 8 runs padded to 16: the slot holds diag(A, I) and b
// padded with zeros, so the padded rows of r, p, z and A p stay exactly zero
// and the iteration is that of the 8 x 8 system.
inline bool solve_tc_supported(int K, int L) {
  return (K == 8 || K == 16 || K == 32 || K == 64 || K == 128) && (L == 0 || L == 4 || L == 8 || L == 16) && L <= K;
}

// Size of the slot's matrix: K rounded up to the smallest CG warp (16).
__host__ __device__ constexpr int pad_k(int K) { return K < 16 ? 16 : K; }

constexpr int kSolveWarps = 8;  // CG warps per CTA (grouped mode, and independent systems for K <= 64)

// Independent systems, K <= 64: one slot per warp, eight warps per CTA (K = 128
// runs four warps per system: kSplitWarps below).
__host__ __device__ constexpr int solve_warps(int) { return kSolveWarps; }

inline size_t solve_tc_smem_bytes(int K, int L);

// K = 128: four warps per system, two systems per CTA; a system's group holds
// its slot and one K-entry staging buffer per warp.
constexpr int kSplitWarps = 4;
constexpr int kSplitGroups = 2;
__host__ __device__ inline size_t split_group_bytes(int K, int L) { return tc_slot_bytes(K, L) + kSplitWarps * sizeof(float2) * K; }
inline size_t solve_split_smem_bytes(int K, int L) { return 128 + kSplitGroups * split_group_bytes(K, L); }

inline size_t solve_tc_smem_bytes(int K, int L) {
  return K == 128 ? solve_split_smem_bytes(K, L) : 128 + kSolveWarps * tc_slot_bytes(pad_k(K), L);
}

// Grouped mode (fpcg_detect_grouped): all warps of a CTA share one group's A
// and inverted blocks; each warp has its own b, matvec result and B fragments.
inline bool solve_grouped_supported(int K, int L) { return solve_tc_supported(K, L); }

__host__ __device__ inline size_t md_bytes(int K, int L) {
  return L > 0 ? sizeof(float2) * (size_t)(K / L) * md_block_stride(L) : 16;
}

// Grouped mode, per vector: b and W (8K bytes each) and 64 bytes that put
// the W of vectors 4i .. 4i+3 on alternate half-bank windows (the stores of
// one output tile).  Shared B fragments: K/16 k-tiles x 8 n-tiles x 8 columns
// x 16 rows of 16-bit values.
__host__ __device__ constexpr int grouped_vec_bytes(int K) { return 16 * K + 64; }
__host__ __device__ constexpr int grouped_pk_bytes(int K) { return (K / 16) * 8 * 8 * 16 * 2; }

inline size_t solve_grouped_smem_bytes(int K, int L) {
  K = pad_k(K);
  return 128 + 4 * (size_t)K * K + md_bytes(K, L) + kSolveWarps * (size_t)grouped_vec_bytes(K) +
         grouped_pk_bytes(K) + 16;
}

template <int K>
cudaError_t launch_solve_grouped_k(const SolveTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream);
extern template cudaError_t launch_solve_grouped_k<8>(const SolveTcParams&, int, int, cudaStream_t);
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
    case 8: return launch_solve_grouped_k<8>(P, num_sms, mv_bf16, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <int K>
cudaError_t launch_solve_tc_k(const SolveTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream);
extern template cudaError_t launch_solve_tc_k<8>(const SolveTcParams&, int, int, cudaStream_t);
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
    case 8: return launch_solve_tc_k<8>(P, num_sms, mv_bf16, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpcg
