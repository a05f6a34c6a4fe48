// Gram matrix and matched filter on the tensor cores (tcgen05, sm_103a):
// A = fl(H)^H fl(H) + sigma^2 I and b = fl(H)^H fl(y) with fl = bf16 or fp16
// rounding and fp32 accumulation (Section II, eq. inversion), written to
// global memory.  Persistent kernel, one CTA per SM, warp-specialised:
//   warp 0      TMEM allocation and the UMMA-issuing thread,
//   warp 1      TMA producer,
//   warps 4-7   drain warpgroup (TMEM -> combine -> A, b in global memory),
//   warps 8-15  converters (FP32 stages -> bf16/fp16 swizzled operand stages).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gram_tc.cuh"
#include "tc_pipeline.cuh"

namespace fpcg {

namespace {

constexpr int kThreads = 512;
constexpr int kConv = 8;  // converter warps 8-15

struct Smem {
  uint8_t* pipe;
  tcp::Bars* bars;
  uint32_t* tmem_slot;
  volatile int* abort;
};

__device__ inline Smem carve(uint8_t* raw) {
  Smem s;
  const uint32_t a = tc::smem_u32(raw);
  uint8_t* base = raw + ((1024u - (a & 1023u)) & 1023u);
  s.pipe = base;
  s.bars = reinterpret_cast<tcp::Bars*>(base + tcp::kPipeBytes);
  s.tmem_slot = reinterpret_cast<uint32_t*>(s.bars + 1);
  s.abort = reinterpret_cast<volatile int*>(s.tmem_slot + 1);
  return s;
}

__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(const __grid_constant__ GramTcParams P) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  Smem S = carve(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const tcp::Pipe& pp = P.pipe;

  for (int i = threadIdx.x; i < tcp::kStages * tcp::kStageBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(tcp::stage16(S.pipe, 0))[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    tcp::init_bars(*S.bars, kConv);
    *S.abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(S.tmem_slot, 2 * tcp::kAccCols);
  tc::fence_proxy_async();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *S.tmem_slot;
  const int64_t tile0 = blockIdx.x, tstep = gridDim.x;

  if (warp == 0) {
    if (lane == 0) tcp::mma_role(pp, S.pipe, *S.bars, S.abort, tmem, tile0, tstep);
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) tcp::producer_role(pp, S.pipe, *S.bars, S.abort, tile0, tstep);
    __syncwarp();
  } else if (warp >= 8) {
    tcp::converter_role<kConv>(pp, S.pipe, *S.bars, S.abort, tile0, tstep, warp - 8, lane);
  } else if (warp >= 4) {
    const int q = warp - 4;
    const int row = 32 * q + lane;
    const int twoK = 2 * pp.K;
    const int k = (row % twoK) >> 1;
    const int odd = row & 1;
    int64_t j = 0;
    int64_t tile = tile0;
    for (; tile < pp.ntiles; tile += tstep, ++j) {
      const uint32_t b = (uint32_t)(j & 1), qa = (uint32_t)(j >> 1);
      if (tc::bar_or(1, 128, !tc::mbar_wait(&S.bars->acc_full[b], qa & 1u, S.abort, P.pipe.budget))) {
        *S.abort = 1;  // the four drain warps leave together
        break;
      }
      tc::tc_fence_after();
      const int64_t sys = tile * pp.P + row / twoK;
      const bool valid = (row / twoK) < pp.P && sys < pp.batch;
      const float s2 = valid ? (float)P.sigma2[sys] : 0.f;
      float* Ag = reinterpret_cast<float*>(P.A) + (valid ? ((sys * pp.K + k) * pp.K) * 2 : 0);
      float* bg = reinterpret_cast<float*>(P.b) + (valid ? (sys * pp.K + k) * 2 : 0);
      tcp::drain_tile(
          pp, tmem + b * tcp::kAccCols, q, lane,
          [&](int l, float v) {
            if (!valid) return;
            if (l == k) v = odd ? 0.f : v + s2;
            Ag[2 * l + odd] = v;
          },
          [&](float v) {
            if (valid) bg[odd] = v;
          });
      tc::tc_fence_before();
      tc::bar_sync(1, 128);
      if (row == 0) tc::mbar_arrive(&S.bars->acc_empty[b]);
    }
    if (*S.abort && P.status) {  // report the systems this CTA did not finish
      for (; tile < pp.ntiles; tile += tstep)
        for (int i = row; i < pp.P; i += 128)
          if (tile * pp.P + i < pp.batch) P.status[tile * pp.P + i] |= 32;
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * tcp::kAccCols);
  }
}

}  // namespace

bool gram_tc_supported(int K) { return K == 8 || K == 16 || K == 32 || K == 64; }

size_t gram_tc_smem_bytes() {
  size_t s = 1024 + tcp::kPipeBytes + sizeof(tcp::Bars) + 16;
  // at least half of the SM's shared memory, so one CTA (and one 512-column
  // TMEM allocation) per SM
  return s < 120 * 1024 ? 120 * 1024 : s;
}

cudaError_t launch_gram_tc(const GramTcParams& P, int num_sms, cudaStream_t stream) {
  const size_t smem = gram_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = P.pipe.ntiles < num_sms ? P.pipe.ntiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  gram_tc_kernel<<<(unsigned)grid, kThreads, smem, stream>>>(P);
  return cudaGetLastError();
}

}  // namespace fpcg
