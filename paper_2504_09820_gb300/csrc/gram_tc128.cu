// Gram matrix and matched filter of K = 128 users on the tensor cores
// (tcgen05, sm_103a): A = fl(H)^H fl(H) + sigma2 I and b = fl(H)^H fl(y)
// (Section II, eq. inversion), fl = bf16 or fp16, fp32 accumulation.
//
// With X_r = Re H^T and X_i = Im H^T (128 users x N antennas, the reduction
// axis), A = X_r X_r^T + X_i X_i^T + i (X_r X_i^T - X_i X_r^T).  Two TMEM
// accumulators per system, four UMMAs (M = N = 128, K = 16) per 16 antennas:
//   D1 += S1 S1^T + S2 S2^T         -> Re A
//   D2 += S1 S2^T + S2 (-S1)^T      -> Im A
// with the operand stages S1 = X_r and S2 = X_i (16-bit, 128-byte swizzled,
// K-major); the minus is the instruction's negate-B bit (exact).  256 columns
// per system, so two systems' accumulators fit in TMEM and the UMMAs of the
// next system overlap the drain of this one.  b = fl(H)^H fl(y) is formed by
// the converter warps from the same rounded values (exact products, fp32
// sums), 16 rows per warp, reduced across lanes at the end of the system.
//
// Persistent kernel, one CTA per SM, one system per tile, warp-specialised:
//   warp 0      TMEM allocation and the UMMA-issuing thread,
//   warp 1      TMA producer (FP32 boxes of 32 antennas x 128 users, y),
//   warps 4-7   drain (TMEM lane k = user k: row k of A through a swizzled
//               staging tile and TMA stores),
//   warps 8-15  converters (two FP32 stages -> one S1/S2 operand stage; b).
// Every wait is bounded; a timeout raises the CTA's abort flag.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gram_tc.cuh"
#include "tc.cuh"
#include "tc_pipeline.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace fpcg {

namespace {

constexpr int kThreads = 512;
constexpr int kConv = 8;                      // converter warps 8-15
constexpr int kK = 128;                       // users
constexpr int kS32 = 4;                       // FP32 stages of 32 antennas
constexpr int kSt32H = kK * 64 * 4;           // 128 rows x 64 floats
constexpr int kSt32 = kSt32H + 64 * 4;        // + 64 floats of y
constexpr int kOpBytes = kK * 128;            // one operand (S1 or S2): 128 rows of 128 bytes
constexpr int kSt16 = 2 * kOpBytes;           // S1 then S2
constexpr int kStages = 2;
constexpr int kRing = kStages * kSt16 + kS32 * kSt32;
constexpr int kStgOff = (kRing + 1023) & ~1023;  // A staging tile, 1024-byte aligned for the swizzle
constexpr int kStgBytes = 128 * 128;          // 128 rows x 16 complex
constexpr int kPipe = kStgOff + kStgBytes;
constexpr uint32_t kNegateB = 1u << 14;       // instruction descriptor: negate the B operand
constexpr uint32_t kAccCols = 256;            // per system: Re A at +0, Im A at +128
constexpr uint32_t kTmemCols = 512;

struct Bars {
  uint64_t full32[kS32];
  uint64_t empty32[kS32];
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t done;
};

__device__ __forceinline__ float rnd16(float v, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : __half2float(__float2half_rn(v));
}

__device__ __forceinline__ uint8_t* st32(uint8_t* pipe, int s) { return pipe + kStages * kSt16 + s * kSt32; }
__device__ __forceinline__ uint8_t* st16(uint8_t* pipe, int t) { return pipe + t * kSt16; }

__global__ void __launch_bounds__(kThreads, 1) gram_tc128_kernel(const __grid_constant__ GramTc128Params P) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t a = tc::smem_u32(smem_raw);
  uint8_t* pipe = smem_raw + ((1024u - (a & 1023u)) & 1023u);
  Bars* B = reinterpret_cast<Bars*>(pipe + kPipe);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(B + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = P.nchunks;  // operand stages (64 antennas) per system

  if (threadIdx.x == 0) {
    for (int s = 0; s < kS32; ++s) {
      tc::mbar_init(&B->full32[s], 1);
      tc::mbar_init(&B->empty32[s], kConv);
    }
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&B->full[s], kConv);
      tc::mbar_init(&B->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&B->acc_full[b], 1);
      tc::mbar_init(&B->acc_empty[b], 1);
    }
    tc::mbar_init(&B->done, 1);
    *abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_proxy_async();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t sys0 = blockIdx.x, sstep = gridDim.x;

  if (warp == 0) {
    if (lane == 0) {  // UMMA issue
      const uint32_t id = tc::idesc_f16(128, 128, P.bf16 != 0);
      uint32_t u = 0;
      int64_t j = 0;
      for (int64_t sys = sys0; sys < P.batch; sys += sstep, ++j) {
        const uint32_t ab = (uint32_t)(j & 1), qa = (uint32_t)(j >> 1);
        if (qa > 0 && !tc::mbar_wait(&B->acc_empty[ab], (qa - 1) & 1u, abort)) {
          *abort = 1;
          break;
        }
        tc::tc_fence_after();
        const uint32_t d1t = tmem + ab * kAccCols, d2t = d1t + 128u;
        for (int c = 0; c < nch; ++c, ++u) {
          const uint32_t t = u % kStages, q = u / kStages;
          if (!tc::mbar_wait(&B->full[t], q & 1u, abort)) {
            *abort = 1;
            break;
          }
          tc::tc_fence_after();
          const uint64_t s1 = tc::sdesc_k_sw128(tc::smem_u32(st16(pipe, (int)t)));
          const uint64_t s2 = tc::sdesc_k_sw128(tc::smem_u32(st16(pipe, (int)t) + kOpBytes));
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t d1 = s1 + (uint64_t)(ks * 2), d2 = s2 + (uint64_t)(ks * 2);  // +32 bytes along K
            const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
            tc::mma_f16(d1t, d1, d1, id, acc);
            tc::mma_f16(d1t, d2, d2, id, 1u);
            tc::mma_f16(d2t, d1, d2, id, acc);
            tc::mma_f16(d2t, d2, d1, id | kNegateB, 1u);
          }
          tc::mma_commit(&B->empty[t]);
        }
        if (*abort) break;
        tc::mma_commit(&B->acc_full[ab]);
      }
      tc::mma_commit(&B->done);  // nothing in flight before the TMEM is released
      tc::mbar_wait_issued(&B->done, 0);  // no MMA may still write TMEM when it is freed
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // TMA producer
      constexpr uint32_t tx = kSt32H + 64 * 4;
      uint32_t u = 0;
      // No L2 prefetch ahead of the loads: measured at N = 512, pulling the next
      // system into L2 (512 KB per SM) cost a third of the bandwidth.
      for (int64_t sys = sys0; sys < P.batch && !*abort; sys += sstep) {
        for (int c = 0; c < 2 * nch; ++c, ++u) {
          const uint32_t s = u % kS32, q = u / kS32;
          if (q > 0 && !tc::mbar_wait(&B->empty32[s], (q - 1) & 1u, abort)) {
            *abort = 1;
            break;
          }
          if (*abort) break;
          uint8_t* st = st32(pipe, (int)s);
          tc::mbar_expect_tx(&B->full32[s], tx);
          tc::tma_load_2d(st, &P.tmH, 64 * c, (int)(sys * kK), &B->full32[s]);
          tc::tma_load_2d(st + kSt32H, &P.tmY, 64 * c, (int)sys, &B->full32[s]);
        }
      }
      if (*abort) tcp::wait_issued_loads<kS32>(B->full32, u);  // none may land after the CTA is gone
    }
    __syncwarp();
  } else if (warp >= 8) {  // converters: rows cw + 8m; lane l fills k-positions 2l, 2l+1
    const int cw = warp - 8;
    const int half = lane >> 4, ll = lane & 15;
    const uint32_t kpos = 2u * lane;
    const int bf = P.bf16;
    uint32_t u32 = 0, u16 = 0;
    for (int64_t sys = sys0; sys < P.batch; sys += sstep) {
      float bacc[2 * (kK / kConv)];  // (Re, Im) of b for rows cw + 8m, this lane's antennas
#pragma unroll
      for (int i = 0; i < 2 * (kK / kConv); ++i) bacc[i] = 0.f;
      for (int c = 0; c < nch; ++c, u32 += 2, ++u16) {
        const uint32_t s0 = u32 % kS32, q0 = u32 / kS32;
        const uint32_t s1 = (u32 + 1) % kS32, q1 = (u32 + 1) / kS32;
        const uint32_t t = u16 % kStages, qt = u16 / kStages;
        const bool ok = tc::mbar_wait(&B->full32[s0], q0 & 1u, abort) && tc::mbar_wait(&B->full32[s1], q1 & 1u, abort) &&
                        (qt == 0 || tc::mbar_wait(&B->empty[t], (qt - 1) & 1u, abort));
        if (!__all_sync(0xffffffffu, ok)) {  // the whole warp leaves together
          *abort = 1;
          break;
        }
        const float* src = reinterpret_cast<const float*>(st32(pipe, (int)(half ? s1 : s0)));
        uint8_t* o1 = st16(pipe, (int)t);
        uint8_t* o2 = o1 + kOpBytes;
        const float4 yv = *reinterpret_cast<const float4*>(src + kSt32H / 4 + 4 * ll);  // y of antennas 2ll, 2ll+1
        const float yr0 = rnd16(yv.x, bf), yi0 = rnd16(yv.y, bf), yr1 = rnd16(yv.z, bf), yi1 = rnd16(yv.w, bf);
#pragma unroll
        for (int m = 0; m < kK / kConv; ++m) {
          const int row = cw + kConv * m;
          const float4 v = *reinterpret_cast<const float4*>(src + row * 64 + 4 * ll);  // antennas 2ll, 2ll+1
          const float hr0 = rnd16(v.x, bf), hi0 = rnd16(v.y, bf), hr1 = rnd16(v.z, bf), hi1 = rnd16(v.w, bf);
          *reinterpret_cast<uint32_t*>(o1 + tc::sw128_offset(row, kpos)) = tcp::pack2(hr0, hr1, bf);
          *reinterpret_cast<uint32_t*>(o2 + tc::sw128_offset(row, kpos)) = tcp::pack2(hi0, hi1, bf);
          // conj(h) y over the two antennas (exact products of the rounded values)
          bacc[2 * m] = fmaf(hr0, yr0, fmaf(hi0, yi0, fmaf(hr1, yr1, fmaf(hi1, yi1, bacc[2 * m]))));
          bacc[2 * m + 1] = fmaf(hr0, yi0, fmaf(-hi0, yr0, fmaf(hr1, yi1, fmaf(-hi1, yr1, bacc[2 * m + 1]))));
        }
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
          tc::mbar_arrive(&B->full[t]);
          tc::mbar_arrive(&B->empty32[s0]);
          tc::mbar_arrive(&B->empty32[s1]);
        }
      }
      if (__any_sync(0xffffffffu, *abort != 0)) break;
      // sum the 32 values over the lanes; lane l ends with value l (reduce-scatter)
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
          const float send = up ? bacc[i] : bacc[i + o];
          const float keep = up ? bacc[i + o] : bacc[i];
          bacc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      reinterpret_cast<float*>(P.b)[(sys * kK + cw + kConv * (lane >> 1)) * 2 + (lane & 1)] = bacc[0];
    }
  } else if (warp >= 4) {  // drain: thread = TMEM lane = user k
    // 16 columns of A at a time: row k into the 128-byte-swizzled staging
    // tile, then one TMA store of the 128 x 16 block.
    const int q = warp - 4, k = 32 * q + lane;
    int64_t j = 0, sys = sys0;
    for (; sys < P.batch; sys += sstep, ++j) {
      const uint32_t ab = (uint32_t)(j & 1);
      if (tc::bar_or(1, 128, !tc::mbar_wait(&B->acc_full[ab], (uint32_t)((j >> 1) & 1), abort))) {
        *abort = 1;  // the four drain warps leave together
        break;
      }
      tc::tc_fence_after();
      const uint32_t lb = tmem + ab * kAccCols + ((uint32_t)(32 * q) << 16);
      const float s2 = (float)P.sigma2[sys];
      uint8_t* stg = pipe + kStgOff;
#pragma unroll 1
      for (int c0 = 0; c0 < kK; c0 += 16) {
        uint32_t re[16], im[16];
        tc::tmem_ld16_async(lb + (uint32_t)c0, re);
        tc::tmem_ld16_async(lb + 128u + (uint32_t)c0, im);
        if (k == 0) tc::bulk_wait_read<0>();  // the previous store has read the tile
        tc::bar_sync(1, 128);
        tc::tmem_wait_ld();
#pragma unroll
        for (int m = 0; m < 16; m += 2) {
          float r0 = __uint_as_float(re[m]), r1 = __uint_as_float(re[m + 1]);
          float i0 = __uint_as_float(im[m]), i1 = __uint_as_float(im[m + 1]);
          const int l = c0 + m;
          if (l == k) {
            r0 += s2;
            i0 = 0.f;
          }
          if (l + 1 == k) {
            r1 += s2;
            i1 = 0.f;
          }
          const int ch = m >> 1;  // 16-byte chunk of the 128-byte row
          *reinterpret_cast<float4*>(stg + k * 128 + ((ch ^ (k & 7)) << 4)) = make_float4(r0, i0, r1, i1);
        }
        tc::fence_proxy_async();  // the tile is visible to the bulk-copy engine
        tc::bar_sync(1, 128);
        if (k == 0) {
          tc::tma_store_2d(&P.tmA, stg, 2 * c0, (int)(sys * kK));
          tc::bulk_commit();
        }
      }
      tc::tc_fence_before();
      tc::bar_sync(1, 128);
      if (k == 0) tc::mbar_arrive(&B->acc_empty[ab]);
    }
    if (k == 0) tc::bulk_wait<0>();  // every store of A has landed
    if (*abort && P.status)  // report the systems this CTA did not finish
      for (; sys < P.batch; sys += sstep)
        if (k == 0) P.status[sys] |= 32;
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

size_t gram_tc128_smem_bytes() { return 1024 + kPipe + sizeof(Bars) + 16; }

cudaError_t launch_gram_tc128(const GramTc128Params& P, int num_sms, cudaStream_t stream) {
  const size_t smem = gram_tc128_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(gram_tc128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = P.batch < num_sms ? P.batch : num_sms;
  if (grid <= 0) return cudaSuccess;
  gram_tc128_kernel<<<(unsigned)grid, kThreads, smem, stream>>>(P);
  return cudaGetLastError();
}

}  // namespace fpcg
