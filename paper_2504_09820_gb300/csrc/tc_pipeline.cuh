// The tensor-core Gram pipeline shared by the Gram-only and the fused
// detection kernels.
//
// Real embedding.  For one system with N antennas and K users, the rows of
// the K-major operand are X^T[2k] = Re h_k and X^T[2k+1] = Im h_k (h_k = column
// k of H, length N, the reduction axis), and two more rows hold Re y and Im y.
// One UMMA product D = X^T [X | Y] (M = 128 rows, N_mma = 128 + 16 columns,
// K = antennas) then contains, with D[i][j] = sum_n row_i[n] row_j[n]:
//   Re A_kl = D[2k][2l] + D[2k+1][2l+1]      Im A_kl = D[2k][2l+1] - D[2k+1][2l]
//   Re b_k  = D[2k][Y0] + D[2k+1][Y1]        Im b_k  = D[2k][Y1]   - D[2k+1][Y0]
// (Section II, eq. inversion: A = H^H H, b = H^H y; sigma^2 is added after).
// Rows 2k and 2k+1 live in adjacent TMEM lanes, so one shuffle per column pair
// combines them.  P = floor(64/K) systems are packed into one 128-row tile
// (they are consecutive columns of the [batch*K][N] matrix); their cross blocks
// of D are ignored.  Operands are bf16 or fp16 (the u_gram rounding), the
// accumulator fp32.
//
// Data movement.  A producer thread streams H and y with 2-D TMA loads
// (cp.async.bulk.tensor, FP32 boxes of 32 antennas x 64 columns of the
// [batch*K][2N] real view of H, and 32 antennas x P systems of y) into a ring
// of FP32 stages, counted on `full32` by transaction bytes; out-of-range boxes
// read as zeros.  Converter warps turn two FP32 stages (64 antennas) into one
// bf16/fp16 operand stage: rows of 128 bytes in the 128B-swizzled K-major
// layout, 144 rows (128 of X, 16 of Y) = 18 KiB.  Roles:
//   producer:        wait `empty32`, expect_tx, two TMA loads into `full32`;
//   converter warps: wait `full32` (two) and `empty16`, read FP32, round,
//                    store swizzled, fence.proxy.async, arrive `full16` and
//                    release the FP32 stages (`empty32`);
//   MMA thread:      wait `full16`, 4 UMMAs (K = 16 each), commit to `empty16`;
//                    after a tile's last stage commit to `acc_full`;
//   drain warps:     wait `acc_full`, tcgen05.ld, combine, consume, arrive
//                    `acc_empty`.
// Every wait is bounded; a timeout raises the CTA's abort flag and all roles
// leave their loops.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "tc.cuh"

namespace fpcg {
namespace tcp {

constexpr int kStages32 = 4;                   // FP32 staging ring (at most; a kernel may use fewer)
constexpr int kChunk32 = 32;                   // antennas per FP32 stage
constexpr int kStage32HBytes = 64 * 64 * 4;    // 64 columns x 64 floats
constexpr int kStage32Bytes = kStage32HBytes + 8 * 64 * 4;  // + y of up to 8 systems (the largest stage)
// FP32 stage for P systems per tile (a multiple of 128 bytes).
__host__ __device__ constexpr int stage32_bytes(int P) { return kStage32HBytes + ((64 * 4 * P + 127) & ~127); }
constexpr int kStages = 2;                     // bf16/fp16 operand stages
constexpr int kStageRows = 144;
constexpr int kStageBytes = kStageRows * 128;  // 18432, a multiple of 1024
constexpr int kChunk = 64;                     // antennas per operand stage
constexpr int kMmaN = 144;
constexpr int kAccCols = 256;                  // TMEM columns per accumulator buffer
// Operand stages first (1024-byte aligned for the 128B swizzle), then the ring.
__host__ __device__ constexpr int pipe_bytes(int stages32, int s32b = kStage32Bytes) {
  return kStages * kStageBytes + stages32 * s32b;
}
constexpr int kPipeBytes = pipe_bytes(kStages32);

struct Pipe {
  CUtensorMap tmH;   // FP32 view of H: dims {2N, batch*K}, box {64, 64}
  CUtensorMap tmY;   // FP32 view of y: dims {2N, batch}, box {64, P}
  const float2* H;
  const float2* y;
  int N, K, P, nchunks;   // nchunks = operand stages per tile = ceil(N / 64)
  int64_t batch, ntiles;
  int bf16;
  int s32b;          // bytes per FP32 stage (stage32_bytes(P) or more)
  long long budget;  // SM cycles a pipeline wait may take before the CTA aborts
};

// Wait for the TMA loads still in flight when the producer stops: the last
// min(u, S) of the u loads it issued (load i went to stage i % S, phase i / S).
template <int S>
__device__ inline void wait_issued_loads(uint64_t* full, uint32_t u) {
  for (uint32_t i = u > (uint32_t)S ? u - S : 0; i < u; ++i) tc::mbar_wait_issued(&full[i % S], (i / S) & 1u);
}

struct Bars {
  uint64_t full32[kStages32];
  uint64_t empty32[kStages32];
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t done;
};

__device__ __forceinline__ uint32_t pack2(float a, float b, int bf16) {
  if (bf16) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ uint8_t* stage32(uint8_t* pipe_base, int s, int s32b) {
  return pipe_base + kStages * kStageBytes + s * s32b;
}
__device__ __forceinline__ uint8_t* stage16(uint8_t* pipe_base, int t) {
  return pipe_base + t * kStageBytes;
}

// Producer role (one thread): tiles this CTA owns are tile0, tile0 + tstep, ...
// S32 = FP32 stages in the ring (2..kStages32).  DRAIN: also wait for the last
// loads at the end (the shared memory is reused after the role ends).
template <int S32 = kStages32, bool DRAIN = false>
__device__ inline void producer_role(const Pipe& p, uint8_t* pipe_base, Bars& B, volatile int* abort,
                                     int64_t tile0, int64_t tstep) {
  const uint32_t tx = kStage32HBytes + 64 * 4 * p.P;
  const uint64_t once = tc::policy_evict_first();  // H and y are read once
  uint32_t u = 0;
  // No L2 prefetch of later tiles: measured on the N = 256, K = 64 batch it cost
  // 2% (and a third of the bandwidth with 512 KB systems); the ring of TMA
  // loads alone keeps enough bytes in flight.
  for (int64_t tile = tile0; tile < p.ntiles; tile += tstep) {
    for (int c = 0; c < 2 * p.nchunks; ++c, ++u) {
      const uint32_t s = u % S32, q = u / S32;
      if (q > 0 && !tc::mbar_wait(&B.empty32[s], (q - 1) & 1u, abort, p.budget)) {
        *abort = 1;
        wait_issued_loads<S32>(B.full32, u);  // none may land after the CTA is gone
        return;
      }
      uint8_t* st = stage32(pipe_base, (int)s, p.s32b);
      tc::mbar_expect_tx(&B.full32[s], tx);
      tc::tma_load_2d_hint(st, &p.tmH, 64 * c, (int)(tile * 64), &B.full32[s], once);
      tc::tma_load_2d_hint(st + kStage32HBytes, &p.tmY, 64 * c, (int)(tile * p.P), &B.full32[s], once);
    }
  }
  // the last loads have landed before this role ends, even where the consumers
  // left early (an abort raised after the last issue)
  if constexpr (DRAIN) wait_issued_loads<S32>(B.full32, u);
}

// Converter warp `cw` of NC: columns cl = cw + NC m of the tile and y of
// systems cw + NC m.  Lane l fills k-positions 2l, 2l+1 of the operand stage
// (antennas 2l, 2l+1 of the 64), read from FP32 stage l/16 at antenna 2(l%16).
template <int NC, int S32 = kStages32>
__device__ inline void converter_role(const Pipe& p, uint8_t* pipe_base, Bars& B, volatile int* abort,
                                      int64_t tile0, int64_t tstep, int cw, int lane) {
  constexpr int NM = (64 + NC - 1) / NC;
  uint32_t u32 = 0, u16 = 0;
  const int half = lane >> 4, ll = lane & 15;
  const uint32_t kpos = 2u * lane;
  for (int64_t tile = tile0; tile < p.ntiles; tile += tstep) {
    for (int c = 0; c < p.nchunks; ++c, u32 += 2, ++u16) {
      const uint32_t s0 = u32 % S32, q0 = u32 / S32;
      const uint32_t s1 = (u32 + 1) % S32, q1 = (u32 + 1) / S32;
      const uint32_t t = u16 % kStages, qt = u16 / kStages;
      const bool ok = tc::mbar_wait(&B.full32[s0], q0 & 1u, abort, p.budget) &&
                      tc::mbar_wait(&B.full32[s1], q1 & 1u, abort, p.budget) &&
                      (qt == 0 || tc::mbar_wait(&B.empty[t], (qt - 1) & 1u, abort, p.budget));
      if (!__all_sync(0xffffffffu, ok)) {  // the whole warp leaves together
        *abort = 1;
        return;
      }
      const float* src = reinterpret_cast<const float*>(stage32(pipe_base, (int)(half ? s1 : s0), p.s32b));
      uint8_t* dst = stage16(pipe_base, (int)t);
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const int cl = cw + NC * m;
        if (cl < p.P * p.K) {
          const float4 v = *reinterpret_cast<const float4*>(src + cl * 64 + 4 * ll);
          *reinterpret_cast<uint32_t*>(dst + tc::sw128_offset(2 * cl, kpos)) = pack2(v.x, v.z, p.bf16);
          *reinterpret_cast<uint32_t*>(dst + tc::sw128_offset(2 * cl + 1, kpos)) = pack2(v.y, v.w, p.bf16);
        }
      }
      const float* ysrc = src + kStage32HBytes / 4;
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int ps = cw + NC * m;
        if (ps < p.P) {
          const float4 v = *reinterpret_cast<const float4*>(ysrc + ps * 64 + 4 * ll);
          *reinterpret_cast<uint32_t*>(dst + tc::sw128_offset(128 + 2 * ps, kpos)) = pack2(v.x, v.z, p.bf16);
          *reinterpret_cast<uint32_t*>(dst + tc::sw128_offset(129 + 2 * ps, kpos)) = pack2(v.y, v.w, p.bf16);
        }
      }
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&B.full[t]);
        tc::mbar_arrive(&B.empty32[s0]);
        tc::mbar_arrive(&B.empty32[s1]);
      }
    }
  }
}

// MMA role (one thread).  DRAIN: also wait for the arrivals of the last
// commits at the end (the shared memory is reused after the role ends).
template <bool DRAIN = false>
__device__ inline void mma_role(const Pipe& p, uint8_t* pipe_base, Bars& B, volatile int* abort, uint32_t tmem,
                                int64_t tile0, int64_t tstep) {
  const uint32_t idesc = tc::idesc_f16(128, kMmaN, p.bf16 != 0);
  uint32_t u = 0, nacc = 0;
  int64_t j = 0;
  for (int64_t tile = tile0; tile < p.ntiles; tile += tstep, ++j) {
    const uint32_t b = (uint32_t)(j & 1), qa = (uint32_t)(j >> 1);
    if (qa > 0 && !tc::mbar_wait(&B.acc_empty[b], (qa - 1) & 1u, abort, p.budget)) {
      *abort = 1;
      break;
    }
    tc::tc_fence_after();
    const uint32_t dt = tmem + b * kAccCols;
    for (int c = 0; c < p.nchunks; ++c, ++u) {
      const uint32_t st = u % kStages, q = u / kStages;
      if (!tc::mbar_wait(&B.full[st], q & 1u, abort, p.budget)) {
        *abort = 1;
        break;
      }
      tc::tc_fence_after();
      const uint32_t sa = tc::smem_u32(stage16(pipe_base, (int)st));
      const uint64_t d0 = tc::sdesc_k_sw128(sa);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t d = d0 + (uint64_t)(ks * 2);  // +32 bytes along K
        tc::mma_f16(dt, d, d, idesc, (c > 0 || ks > 0) ? 1u : 0u);
      }
      tc::mma_commit(&B.empty[st]);
    }
    if (*abort) break;
    tc::mma_commit(&B.acc_full[b]);
    ++nacc;
  }
  // make sure nothing is in flight before the TMEM is released, and that the
  // last commits' arrivals (stages nobody waits for again, tiles an aborting
  // drain did not take) have landed before the barriers can be invalidated
  tc::mma_commit(&B.done);
  tc::mbar_wait_issued(&B.done, 0);
  if constexpr (DRAIN) {
    wait_issued_loads<kStages>(B.empty, u);
    wait_issued_loads<2>(B.acc_full, nacc);
  }
}

// Initialise the pipeline's barriers (one thread).
__device__ inline void init_bars(Bars& B, int nconv, int stages32 = kStages32) {
  for (int s = 0; s < stages32; ++s) {
    tc::mbar_init(&B.full32[s], 1);
    tc::mbar_init(&B.empty32[s], nconv);
  }
  for (int s = 0; s < kStages; ++s) {
    tc::mbar_init(&B.full[s], nconv);
    tc::mbar_init(&B.empty[s], 1);
  }
  for (int b = 0; b < 2; ++b) {
    tc::mbar_init(&B.acc_full[b], 1);
    tc::mbar_init(&B.acc_empty[b], 1);
  }
  tc::mbar_init(&B.done, 1);
}

// Invalidate the pipeline's barriers (one thread, every phase complete), so
// that their memory can be laid out anew.
__device__ inline void inval_bars(Bars& B, int stages32 = kStages32) {
  for (int s = 0; s < stages32; ++s) {
    tc::mbar_inval(&B.full32[s]);
    tc::mbar_inval(&B.empty32[s]);
  }
  for (int s = 0; s < kStages; ++s) {
    tc::mbar_inval(&B.full[s]);
    tc::mbar_inval(&B.empty[s]);
  }
  for (int b = 0; b < 2; ++b) {
    tc::mbar_inval(&B.acc_full[b]);
    tc::mbar_inval(&B.acc_empty[b]);
  }
  tc::mbar_inval(&B.done);
}

// Drain helper: for the calling thread (TMEM lane `row` of the tile) combine
// column pairs of its own system block into A entries.  `emit(l, value)` gets
// Re A[k][l] on even rows and Im A[k][l] on odd rows; `emit_b(value)` gets
// Re b_k / Im b_k.  Must be called by whole warps of a warpgroup (all lanes
// take part in the shuffles).
template <typename EmitA, typename EmitB>
__device__ __forceinline__ void drain_tile(const Pipe& p, uint32_t tmem_acc, int q, int lane, EmitA emit,
                                           EmitB emit_b) {
  const int row = 32 * q + lane;
  const int twoK = 2 * p.K;
  const int sys = row / twoK;         // system of this lane within the tile
  const int blk0 = sys * twoK;        // first column of its block
  const bool odd = row & 1;
  const uint32_t lane_base = tmem_acc + ((uint32_t)(32 * q) << 16);
  // columns the warp needs: its lanes' blocks
  int c_lo, c_hi;
  if (twoK >= 32) {
    c_lo = (32 * q / twoK) * twoK;
    c_hi = c_lo + twoK;
  } else {
    c_lo = 32 * q;
    c_hi = 32 * q + 32;
  }
  // 32 columns (2 loads) in flight per wait
  for (int cg = c_lo; cg < c_hi; cg += 32) {
    uint32_t r[2][16];
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (cg + 16 * u < c_hi) tc::tmem_ld16_async(lane_base + (uint32_t)(cg + 16 * u), r[u]);
    tc::tmem_wait_ld();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (cg + 16 * u >= c_hi) break;
#pragma unroll
      for (int m = 0; m < 16; m += 2) {
        const float vm = __uint_as_float(r[u][m]);
        const float other = __shfl_xor_sync(0xffffffffu, __uint_as_float(r[u][m + 1]), 1);
        const int j = cg + 16 * u + m;
        if (sys < p.P && j >= blk0 && j < blk0 + twoK) {
          const int l = (j - blk0) >> 1;
          emit(l, odd ? (other - vm) : (vm + other));
        }
      }
    }
  }
  {  // y columns 128 + 2 sys, 129 + 2 sys; a warp covers one or two systems
    const int s0 = (32 * q) / twoK;
    const int s1 = s0 + 1 < 8 ? s0 + 1 : s0;
    uint32_t v0[2], v1[2];
    tc::tmem_ld2_async(lane_base + 128u + 2u * (uint32_t)s0, v0);
    tc::tmem_ld2_async(lane_base + 128u + 2u * (uint32_t)s1, v1);
    tc::tmem_wait_ld();
    const float mine0 = __uint_as_float(sys == s0 ? v0[0] : v1[0]);
    const float mine1 = __uint_as_float(sys == s0 ? v0[1] : v1[1]);
    const float other = __shfl_xor_sync(0xffffffffu, mine1, 1);
    if (sys < p.P) emit_b(odd ? (other - mine0) : (mine0 + other));
  }
}

}  // namespace tcp
}  // namespace fpcg
