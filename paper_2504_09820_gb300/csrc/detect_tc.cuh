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
  int nslots;      // systems in flight per CTA (tc_num_slots)
  int ncg;         // CG warps (tc_cg_warps); the converters are the 10 - ncg warps after them
  int resid_gram;  // residuals against the fp32 Gram (fused kernel: remainder pieces in global scratch; solvers: the given A)
  int status_or;   // OR the status bits into status[] instead of storing them (a Gram pass wrote it first)
  float2* x_hat;
  uint8_t* sym;
  double* rel_res;
  float* res_hist;
  const uint8_t* tx;
  unsigned long long* bit_errors;
  int32_t* status;
};

// Layout of the diagonal blocks M_d in a slot: block b at b * md_block_stride
// (float2 units), row i of a block at i * md_row_stride.  Rows are padded to
// an even length (16-byte aligned rows for vector loads) and blocks by 4 more
// entries (successive blocks start on different banks).
// L = 4: unpadded rows (32 bytes) and blocks 18 entries apart, so the start of
// block b moves by one 16-byte chunk per block and the 32 lanes' row loads
// spread over all eight chunks of a 128-byte window.
__host__ __device__ constexpr int md_row_stride(int L) { return L == 4 ? 4 : L + 2; }
__host__ __device__ constexpr int md_block_stride(int L) { return L == 4 ? 18 : L * (L + 2) + 4; }

// One system slot in shared memory (carved in cg_warp.cuh): A + sigma^2 I in
// the matvec format, the fp32 diagonal blocks M_d, b and the matvec result [K]
// (c64) and the packed B fragments (3K words).  16-bit matvec: [Re A; Im A]
// (2K x K).  e4m3 matvec (f8): A as K rows of 2K bytes (Re, Im interleaved),
// its per-(row, 16-column block) fp32 scales [K][K/16], 6K more words of
// B fragments (x in six e4m3 pieces for the residual) and the K/16 block
// scales of the vector last packed.
__host__ __device__ inline size_t tc_slot_bytes(int K, int L, bool f8 = false) {
  size_t s = f8 ? 2 * (size_t)K * K + sizeof(float) * (size_t)K * (K / 16) : 4 * (size_t)K * K;
  s += sizeof(float2) * (L > 0 ? (size_t)(K / L) * md_block_stride(L) : 2);
  s += sizeof(float2) * K * 2;
  s += sizeof(uint32_t) * (f8 ? 9 : 3) * K + (f8 ? sizeof(float) * (K / 16) : 0);
  return (s + 127) & ~size_t(127);
}

// e4m3 kernel: the drain's staging of 16-bit remainder pieces, 1 KB per drain
// warp, after the slots.
constexpr size_t kTcF8StageBytes = 4 * 1024;

constexpr int kTcCgWarps = 8;       // CG warps, one slot each (at most)

// CG warps of the fused kernel, of its 16 warps: 4 drain the accumulator, 2
// feed the pipeline, the rest convert the FP32 stages.  A tile brings 64 x N
// complex entries of H whatever K is, and two converter warps keep up with
// N <= 128 only: 8 CG warps and 2 converters there for K <= 32 (more systems
// in flight; the CG warps are latency-bound), 6 and 4 otherwise (K = 64 has at
// most six slots).  Measured on GB300, 7 + 7 iterations, L = 4: K = 32,
// N = 128: 0.58 -> 0.47 ms for 32768 systems; N = 256: 0.62 -> 0.80 ms.
__host__ __device__ constexpr int tc_cg_warps(int K, int N) { return K <= 32 && N <= 128 ? 8 : 6; }
// The most CG warps (and slots) a CTA of this K can run.
__host__ __device__ constexpr int tc_cg_warps_max(int K) { return K <= 32 ? 8 : 6; }

// Remainder of the fp32 Gram matrix beyond its matvec-format copy, for the
// residual b - A x of the fused kernel: A - A16 as one more 16-bit piece
// (fp16: 11 + 11 significant bits of the 24) or two (bf16: 8 + 8 + 8), in
// mma.sync A-fragment order, kept in a device scratch pool (one region per
// resident CTA, at most one CTA per SM) instead of shared memory.  With an
// e4m3 matvec the remainder is A - A_mv, as two bf16 pieces (the first within
// 2^-4 of an entry, so 4 + 8 + 8 significant bits and a last error of
// 2^-22 of the entry).
constexpr int kTcScratchRegions = 160;  // >= SMs of the GPU (checked at launch)
__host__ __device__ constexpr int tc_rem_pieces(bool bf16) { return bf16 ? 2 : 1; }
__host__ __device__ constexpr size_t tc_rem_piece_bytes(int K) { return 4 * (size_t)K * K; }
__host__ __device__ constexpr size_t tc_rem_region_bytes(int K) {
  return (size_t)tc_cg_warps_max(K) * 2 * tc_rem_piece_bytes(K);
}
constexpr int kTcStages32 = 4;      // FP32 TMA ring depth of the fused kernel
constexpr size_t kTcSmemMax = 227 * 1024;

// FP32 stages of the fused kernel: y of the 64 / K systems of a tile only.
__host__ __device__ constexpr int tc_stage32_bytes(int K) { return tcp::stage32_bytes(64 / K); }

// Offset of the first slot after the stages, barriers, TMEM address and abort flag.
__host__ __device__ inline size_t tc_slots_offset(int K) {
  return (tcp::pipe_bytes(kTcStages32, tc_stage32_bytes(K)) + sizeof(tcp::Bars) + 2 * kTcCgWarps * sizeof(uint64_t) +
          16 + 127) &
         ~size_t(127);
}

// Systems in flight per CTA: as many slots as fit beside the pipeline, one per CG warp.
inline int tc_num_slots(int K, int L, bool f8 = false) {
  const size_t avail = kTcSmemMax - 1024 - tc_slots_offset(K) - (f8 ? kTcF8StageBytes : 0);
  const size_t n = avail / tc_slot_bytes(K, L, f8);
  return n < (size_t)tc_cg_warps_max(K) ? (int)n : tc_cg_warps_max(K);
}

inline size_t detect_tc_smem_bytes(int K, int L, bool f8 = false) {
  const size_t s =
      1024 + tc_slots_offset(K) + tc_num_slots(K, L, f8) * tc_slot_bytes(K, L, f8) + (f8 ? kTcF8StageBytes : 0);
  return s < 120 * 1024 ? 120 * 1024 : s;  // one CTA (one 512-column TMEM allocation) per SM
}

// K in {16, 32, 64}; L in {0 (FP-CG), 4, 8, 16}.
inline bool detect_tc_supported(int K, int L) {
  return (K == 16 || K == 32 || K == 64) && (L == 0 || L == 4 || L == 8 || L == 16) && tc_num_slots(K, L) >= 2;
}

// Up to kTcMultiMax classes of one fused launch (detect_tc_multi_kernel):
// each class's own parameters (tensor maps of its H and y, outputs, slots),
// the number of the class's first tile in the launch's running tile count,
// and the scratch pools of K = 16, 32, 64 (device addresses, tc_rem_pool).
constexpr int kTcMultiMax = 10;
struct MultiTcParams {
  int nclass;
  int64_t tile_base[kTcMultiMax];
  uint8_t* pool[3];
  int* busy[3];
  DetectTcParams cls[kTcMultiMax];
};

// Device address of the scratch pool of K (and its busy flags) on the
// current device.  Looked up outside stream captures and remembered per
// device: during a capture the address found earlier is used (a capture that
// comes first fails with the lookup's error).
template <int K>
cudaError_t tc_rem_pool(cudaStream_t stream, uint8_t** pool, int** busy);
extern template cudaError_t tc_rem_pool<16>(cudaStream_t, uint8_t**, int**);
extern template cudaError_t tc_rem_pool<32>(cudaStream_t, uint8_t**, int**);
extern template cudaError_t tc_rem_pool<64>(cudaStream_t, uint8_t**, int**);

// One launch over the classes of M (every class: K in {16, 32, 64}, the
// given block size L, matvec format and residual mode; cls[c] filled as for
// launch_detect_tc, pools set).  Instantiated per L in detect_tc_multi_l*.cu.
template <int LT>
cudaError_t launch_detect_tc_multi_l(MultiTcParams& M, int num_sms, int mv_bf16, int resid_gram, cudaStream_t s);
extern template cudaError_t launch_detect_tc_multi_l<0>(MultiTcParams&, int, int, int, cudaStream_t);
extern template cudaError_t launch_detect_tc_multi_l<4>(MultiTcParams&, int, int, int, cudaStream_t);
extern template cudaError_t launch_detect_tc_multi_l<8>(MultiTcParams&, int, int, int, cudaStream_t);
extern template cudaError_t launch_detect_tc_multi_l<16>(MultiTcParams&, int, int, int, cudaStream_t);

inline cudaError_t launch_detect_tc_multi(MultiTcParams& M, int num_sms, int L, int mv_bf16, int resid_gram,
                                          cudaStream_t s) {
  switch (L) {
    case 0: return launch_detect_tc_multi_l<0>(M, num_sms, mv_bf16, resid_gram, s);
    case 4: return launch_detect_tc_multi_l<4>(M, num_sms, mv_bf16, resid_gram, s);
    case 8: return launch_detect_tc_multi_l<8>(M, num_sms, mv_bf16, resid_gram, s);
    case 16: return launch_detect_tc_multi_l<16>(M, num_sms, mv_bf16, resid_gram, s);
    default: return cudaErrorInvalidValue;
  }
}

// mv: the matvec format (FPCG_BF16, FPCG_FP16 or FPCG_FP8E4M3 codes).
template <int K>
cudaError_t launch_detect_tc_k(const DetectTcParams& P, int num_sms, int mv, cudaStream_t stream);
// Each K is instantiated in its own translation unit (detect_tc_k{16,32,64}.cu).
extern template cudaError_t launch_detect_tc_k<16>(const DetectTcParams&, int, int, cudaStream_t);
extern template cudaError_t launch_detect_tc_k<32>(const DetectTcParams&, int, int, cudaStream_t);
extern template cudaError_t launch_detect_tc_k<64>(const DetectTcParams&, int, int, cudaStream_t);

inline cudaError_t launch_detect_tc(const DetectTcParams& P, int num_sms, int mv, cudaStream_t stream) {
  switch (P.pipe.K) {
    case 64: return launch_detect_tc_k<64>(P, num_sms, mv, stream);
    case 32: return launch_detect_tc_k<32>(P, num_sms, mv, stream);
    case 16: return launch_detect_tc_k<16>(P, num_sms, mv, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpcg
