// Host side of the TMA pipeline: tensor maps for H and y.
#include <cuda.h>
#include <stdlib.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <mutex>
#include <stdint.h>
#include <string.h>

#include "gram_tc.cuh"

namespace fpcg {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D fp32 tensor: inner dimension `inner` floats, `rows` rows of `inner`
// floats each (contiguous), box {64, box_rows}.
bool encode(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  auto fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {inner * 4};
  const cuuint32_t box[2] = {64, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D fp32 tensor with a 128-byte swizzle (box {32, box_rows}: 128-byte rows).
bool encode_sw128(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  auto fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {inner * 4};
  const cuuint32_t box[2] = {32, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

long long wait_budget_cycles() {
  // FPCG_TC_WAIT_CYCLES: diagnostic override of the bounded waits (a tiny value makes
  // every pipeline wait give up, which exercises the abort path); default ~2 s at 2 GHz.
  const char* v = getenv("FPCG_TC_WAIT_CYCLES");
  const long long c = v ? atoll(v) : 0;
  return c > 0 ? c : 4000000000LL;
}

bool tma_pipe_ok(const void* H, const void* y, int N) {
  return N % 2 == 0 && ((uintptr_t)H % 16) == 0 && ((uintptr_t)y % 16) == 0;
}

bool make_pipe(tcp::Pipe* p, const float2* H, const float2* y, int N, int K, int64_t batch, int bf16) {
  memset(p, 0, sizeof(*p));
  p->H = H;
  p->y = y;
  p->N = N;
  p->K = K;
  p->P = 64 / K;
  p->nchunks = (N + tcp::kChunk - 1) / tcp::kChunk;
  p->batch = batch;
  p->ntiles = (batch + p->P - 1) / p->P;
  p->bf16 = bf16;
  p->s32b = tcp::kStage32Bytes;
  p->budget = wait_budget_cycles();
  return encode(&p->tmH, H, 2ull * N, (uint64_t)batch * K, 64) &&
         encode(&p->tmY, y, 2ull * N, (uint64_t)batch, (uint32_t)p->P);
}

bool make_gram_tc128(GramTc128Params* p, const float2* H, const float2* y, float2* A, int N, int64_t batch,
                     int bf16) {
  if (((uintptr_t)A % 16) != 0) return false;
  p->H = H;
  p->A = A;
  p->N = N;
  p->nchunks = (N + tcp::kChunk - 1) / tcp::kChunk;
  p->batch = batch;
  p->bf16 = bf16;
  return encode(&p->tmH, H, 2ull * N, (uint64_t)batch * 128, 128) && encode(&p->tmY, y, 2ull * N, (uint64_t)batch, 1) &&
         encode_sw128(&p->tmA, A, 256, (uint64_t)batch * 128, 128);
}

}  // namespace fpcg
