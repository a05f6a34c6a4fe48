#pragma once
// Fused tensor-core detector (kernel templates; instantiated per K by
// detect_tc_k{16,32,64}.cu): the whole path for K in {16, 32, 64} in one
// persistent launch (one CTA per SM, 16 warps).
//
//   warps 0-3    drain warpgroup: TMEM accumulator -> system slots
//   warps 4-9    CG warps (4-11 for K <= 32 and N <= 128: tc_cg_warps): warp
//                4+c runs every system that lands in slot c (as many slots as
//                shared memory holds)
//   warps 10-13  converters (12-13 with eight CG warps): FP32 stages ->
//                bf16/fp16 swizzled operand stages
//   warp 14      TMA producer of the FP32 stages
//   warp 15      TMEM allocation and the UMMA-issuing thread
//
// Gram + matched filter (Section II, eq. inversion) come out of the tcgen05
// pipeline of tc_pipeline.cuh.  The drain warpgroup turns a finished tile of
// P = 64/K systems into P slots in shared memory: A + sigma^2 I rounded to the
// matvec format (bf16/fp16, as [Re A; Im A] in a swizzled row-major layout
// that ldmatrix reads without bank conflicts), the fp32 diagonal blocks of A
// and the fp32 b.  One CG warp then runs the system alone, with no barrier:
//   * block-Jacobi setup (eq. pre_BJ): in-place Gauss-Jordan of the diagonal
//     blocks, each lane owning one or two block columns;
//   * A p (u_MV): ldmatrix + mma.sync m16n8k16 over [Re A; Im A] against the
//     B fragment [Re p, Im p, 0...] (products exact, fp32 sums), one m-tile at
//     a time; the result is redistributed through shared memory;
//   * Algorithm 2 / 3: one or two rows of every vector per lane, inner
//     products by warp shuffles (u_IP rounding), z = M_d r by shuffles within
//     the block's lanes, updates by FMA at u_W = fp32;
//   * refinement: r = b - A x on the tensor cores with x = x_hi + x_mid +
//     x_lo split over B columns and A the fp32 Gram matrix, as A16 plus its
//     16-bit remainder pieces (written by the drain into a global scratch
//     region of this CTA, read back by the residual trips; with resid_gram
//     off, A16 alone), a correction solve, x += d; rel_res (norms in fp64);
//     Gray-QAM decision; bit errors.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "cg_warp.cuh"
#include "common.cuh"
#include "detect_tc.cuh"
#include "tc_pipeline.cuh"

namespace fpcg {

namespace {

constexpr int kThreads = 16 * 32;
constexpr int kMmaWarp = 15;
constexpr int kProdWarp = 14;
constexpr int kCg0 = 4;                     // CG warps 4 .. 3 + ncg, then the converters

struct Bars2 {
  uint64_t slot_full[kTcCgWarps];    // drain -> CG warp
  uint64_t slot_empty[kTcCgWarps];   // CG warp -> drain
};

struct Smem {
  uint8_t* pipe;
  tcp::Bars* bars;
  Bars2* sbars;
  uint32_t* tmem_slot;
  volatile int* abort;
  int* region;       // this CTA's scratch region (-1: none)
  uint8_t* pool;     // the scratch pool of this K and its busy flags
  int* busy;
  uint8_t* slots;
  uint8_t* f8stage;  // e4m3 kernel: the drain's staging, 1 KB per drain warp
};

// Scratch pool of the remainder pieces: one region per resident CTA.  The
// kernel needs more than half of an SM's shared memory, so at most one of its
// CTAs (of any K) runs per SM, and kTcScratchRegions >= the SM count leaves a
// free region for every CTA that starts.  A CTA takes one with atomicCAS and
// gives it back before it exits.
template <int K>
__device__ __align__(256) uint8_t g_rem[(size_t)kTcScratchRegions * tc_rem_region_bytes(K)];
template <int K>
__device__ int g_rem_busy[kTcScratchRegions];

template <int K>
__device__ __forceinline__ uint8_t* rem_slot(uint8_t* pool, int region, int slot) {
  return pool + (size_t)region * tc_rem_region_bytes(K) + (size_t)slot * 2 * tc_rem_piece_bytes(K);
}

// Drain warpgroup: tile j of this CTA (TMEM buffer j & 1) holds systems
// seq = j*P + p, p < P, which go to slots seq % nslots.  Thread = TMEM lane =
// row 2k + odd of its system's block.
// F8: each 16-column block of row k (Re from thread 2k, Im from 2k + 1) is
// quantised with its own scale (e4m3_scale of the block's largest |component|)
// into 32 interleaved bytes of A8; with RG, the exact remainder A - A_mv goes
// to the scratch as two bf16 pieces.
template <int K, bool BF, int LT, int RG, int F8>
__device__ void drain_role(const DetectTcParams& P, const Smem& S, uint32_t tmem, int64_t tile0, int64_t tstep) {
  const tcp::Pipe& pp = P.pipe;
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * q + lane;
  constexpr int twoK = 2 * K;
  constexpr int PP = 64 / K;
  constexpr int MLD = md_row_stride(LT > 0 ? LT : 1), MBS = md_block_stride(LT > 0 ? LT : 1);
  const int ns = P.nslots;
  const int ps = row / twoK, k = (row % twoK) >> 1, odd = row & 1;
  const int blk0 = ps * twoK;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
  const size_t slot_bytes = tc_slot_bytes(K, LT, F8);
  const uint64_t keep = tc::policy_evict_last();  // remainder pieces: read back by the CG warps
  int64_t j = 0;
  for (int64_t tile = tile0; tile < pp.ntiles; tile += tstep, ++j) {
    const uint32_t b = (uint32_t)(j & 1), qa = (uint32_t)(j >> 1);
    const int64_t sys = tile * PP + ps;
    const bool valid = sys < pp.batch;
    const float s2 = valid ? (float)P.sigma2[sys] : 1.f;  // issued before the wait
    bool ok = tc::mbar_wait(&S.bars->acc_full[b], qa & 1u, S.abort, pp.budget);
    for (int p = 0; ok && p < PP; ++p) {
      const int64_t seq = j * PP + p;
      const uint32_t sl = (uint32_t)(seq % ns), use = (uint32_t)(seq / ns);
      if (use > 0) ok = tc::mbar_wait(&S.sbars->slot_empty[sl], (use - 1) & 1u, S.abort, pp.budget);
    }
    if (tc::bar_or(1, 128, !ok)) {  // the four drain warps leave together
      *S.abort = 1;
      break;
    }
    tc::tc_fence_after();
    const uint32_t tb = lane_base + b * (uint32_t)tcp::kAccCols;
    const int slot = (int)((j * PP + ps) % ns);
    Slot sl = slot_carve(S.slots + slot * slot_bytes, K, LT, F8);
    uint8_t* rem = (RG && *S.region >= 0) ? rem_slot<K>(S.pool, *S.region, slot) : nullptr;
    const int arow = odd ? K + k : k;           // row of [Re A; Im A]
    const int kb0 = (k / (LT > 0 ? LT : 1)) * LT;  // first column of k's diagonal block
#pragma unroll 1
    for (int cg = blk0; cg < blk0 + twoK; cg += 32) {
      uint32_t v[2][16];
      tc::tmem_ld16_async(tb + (uint32_t)cg, v[0]);
      tc::tmem_ld16_async(tb + (uint32_t)(cg + 16), v[1]);
      tc::tmem_wait_ld();
      float a[2][8];  // columns l0(u) .. l0(u) + 7 of row arow, u = 0, 1: one k-tile
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int l0 = (cg + 16 * u - blk0) >> 1;  // first of the 8 columns l of this chunk
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const float vm = __uint_as_float(v[u][2 * m]);
          const float other = __shfl_xor_sync(0xffffffffu, __uint_as_float(v[u][2 * m + 1]), 1);
          float val = odd ? (other - vm) : (vm + other);
          if (!valid) val = 0.f;
          if (l0 + m == k) val = odd ? 0.f : val + s2;
          a[u][m] = val;
        }
      }
      const int kt = (cg - blk0) >> 5, mt = (k & (K - 1)) >> 4;
      float lo[2][8];  // the first piece for the scratch
      if constexpr (F8) {
        float m = 0.f;
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int mm = 0; mm < 8; ++mm) m = fmaxf(m, fabsf(a[u][mm]));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));  // Re and Im of the block
        float inv;
        const float sc = e4m3_scale_inv(m, inv);  // powers of two
        uint32_t wq[4];  // e4m3 bytes of columns 4i .. 4i + 3 of this thread's part
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float* src = &a[i >> 1][4 * (i & 1)];
          wq[i] = tc::cvt_e4m3x4(src[0] * inv, src[1] * inv, src[2] * inv, src[3] * inv);
          if constexpr (RG) {  // a - sc q: exact (q sc is within a factor of two of a, or 0)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(wq[i] >> (16 * h)), __NV_E4M3);
              const float2 f = __half22float2(__half2(hr));
              lo[i >> 1][4 * (i & 1) + 2 * h] = src[2 * h] - f.x * sc;
              lo[i >> 1][4 * (i & 1) + 2 * h + 1] = src[2 * h + 1] - f.y * sc;
            }
          }
        }
        // thread 2k (Re) writes columns 0-7 of the block, thread 2k + 1 (Im) columns 8-15
        const uint32_t s0 = __shfl_xor_sync(0xffffffffu, odd ? wq[0] : wq[2], 1);
        const uint32_t s1 = __shfl_xor_sync(0xffffffffu, odd ? wq[1] : wq[3], 1);
        const uint32_t re0 = odd ? s0 : wq[0], re1 = odd ? s1 : wq[1];
        const uint32_t im0 = odd ? wq[2] : s0, im1 = odd ? wq[3] : s1;
        *reinterpret_cast<uint4*>(sl.A16 + a16_offset<K>(k, 2 * kt + odd)) =
            make_uint4(__byte_perm(re0, im0, 0x5140), __byte_perm(re0, im0, 0x7362), __byte_perm(re1, im1, 0x5140),
                       __byte_perm(re1, im1, 0x7362));
        if (!odd) sl.sA[k * (K / 16) + kt] = sc;
      } else if (RG) {
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int mm = 0; mm < 8; ++mm) lo[u][mm] = a[u][mm] - round16<BF>(a[u][mm]);  // exact
      }
      if (RG && rem) {
        // The scratch pieces in mma A-fragment order (rem_block): the warp owns
        // one m-tile (16 rows of Re A and of Im A); each piece of this k-tile
        // goes row-major through shared memory (the slot's A16 area, rewritten
        // below, or the e4m3 kernel's staging block of this warp) and comes
        // back by ldmatrix as fragments, one 16-byte store per lane.
        uint8_t* stg = F8 ? S.f8stage + q * 1024 : nullptr;
        const uint32_t abase = tc::smem_u32(F8 ? stg : sl.A16);
        const int lr = lane & 15, lc = lane >> 4;
        const int srow = odd * 16 + (k & 15);
#pragma unroll
        for (int pc = 0; pc < tc_rem_pieces(BF); ++pc) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            uint4 q;
            q.x = pk2<BF>(lo[u][0], lo[u][1]);
            q.y = pk2<BF>(lo[u][2], lo[u][3]);
            q.z = pk2<BF>(lo[u][4], lo[u][5]);
            q.w = pk2<BF>(lo[u][6], lo[u][7]);
            if (F8) *reinterpret_cast<uint4*>(stg + stg_offset(srow, u)) = q;
            else *reinterpret_cast<uint4*>(sl.A16 + a16_offset<K>(arow, 2 * kt + u)) = q;
#pragma unroll
            for (int mm = 0; mm < 8; ++mm) lo[u][mm] -= round16<BF>(lo[u][mm]);  // exact
          }
          __syncwarp();
#pragma unroll
          for (int pr = 0; pr < 2; ++pr) {
            uint32_t f[4];
            tc::ldmatrix_x4(f, abase + (F8 ? stg_offset(pr * 16 + lr, lc)
                                           : a16_offset<K>(pr * K + 16 * mt + lr, 2 * kt + lc)));
            tc::st_global_hint(rem + rem_block<K>(pc, pr, mt, kt) + 16 * lane, make_uint4(f[0], f[1], f[2], f[3]),
                               keep);
          }
          __syncwarp();
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int l0 = (cg + 16 * u - blk0) >> 1;
        if constexpr (!F8) {  // 8 columns -> one 16-byte chunk of row arow
          uint4 pkd;
          pkd.x = pk2<BF>(a[u][0], a[u][1]);
          pkd.y = pk2<BF>(a[u][2], a[u][3]);
          pkd.z = pk2<BF>(a[u][4], a[u][5]);
          pkd.w = pk2<BF>(a[u][6], a[u][7]);
          *reinterpret_cast<uint4*>(sl.A16 + a16_offset<K>(arow, l0 >> 3)) = pkd;
        }
        if constexpr (LT > 0) {
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const int l = l0 + m;
            if (l >= kb0 && l < kb0 + LT)
              reinterpret_cast<float*>(sl.Md + (k / LT) * MBS + (k % LT) * MLD + (l - kb0))[odd] = a[u][m];
          }
        }
      }
    }
    {  // b from the y columns 128 + 2ps, 129 + 2ps (ps is the same on the whole warp)
      uint32_t v[2];
      tc::tmem_ld2_async(tb + 128u + 2u * (uint32_t)ps, v);
      tc::tmem_wait_ld();
      const float mine0 = __uint_as_float(v[0]), mine1 = __uint_as_float(v[1]);
      const float other = __shfl_xor_sync(0xffffffffu, mine1, 1);
      reinterpret_cast<float*>(sl.b + k)[odd] = valid ? (odd ? (other - mine0) : (mine0 + other)) : 0.f;
    }
    tc::tc_fence_before();
    tc::bar_sync(1, 128);
    if (row == 0) tc::mbar_arrive(&S.bars->acc_empty[b]);
    if (row == 0)
      for (int p = 0; p < PP; ++p) tc::mbar_arrive(&S.sbars->slot_full[(j * PP + p) % ns]);
  }
}

// CG warp c: every system whose slot is c, in order.
template <int K, bool BF, int LT, int RG, int F8>
__device__ void cg_role(const DetectTcParams& P, const Smem& S, int c, int64_t tile0, int64_t tstep) {
  const tcp::Pipe& pp = P.pipe;
  const int lane = threadIdx.x & 31;
  constexpr int PP = 64 / K;
  const int ns = P.nslots;
  const int64_t nloc = tile0 < pp.ntiles ? (pp.ntiles - tile0 + tstep - 1) / tstep : 0;
  CgWarp<K, BF, LT, K, 1, 1, RG, F8> W(P, slot_carve(S.slots + c * tc_slot_bytes(K, LT, F8), K, LT, F8), lane);
  if constexpr (RG == 1)
    if (*S.region >= 0) W.rem = rem_slot<K>(S.pool, *S.region, c);
  int64_t seq = c;
  for (; seq / PP < nloc; seq += ns) {
    const uint32_t use = (uint32_t)(seq / ns);
    if (!__all_sync(0xffffffffu, tc::mbar_wait(&S.sbars->slot_full[c], use & 1u, S.abort, pp.budget))) {
      *S.abort = 1;
      break;
    }
    const int64_t tile = tile0 + (seq / PP) * tstep;
    const int64_t sys = tile * PP + seq % PP;
    W.detect(sys, sys < pp.batch, W.bj_setup());
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(&S.sbars->slot_empty[c]);
  }
  if (*S.abort && P.status && lane == 0) {  // systems this warp did not finish
    for (; seq / PP < nloc; seq += ns) {
      const int64_t sys = (tile0 + (seq / PP) * tstep) * PP + seq % PP;
      if (sys < pp.batch) P.status[sys] = 32;
    }
  }
}

// One batch of one (N, K) class by the whole CTA: barriers, scratch region,
// the roles over tiles tile0, tile0 + tstep, ... of P, and on the way out the
// region released.  MULTI (a class of a multi-class launch): the producer and
// the MMA thread also wait for their last TMA loads and commits, and the
// barriers are invalidated, since the next class lays shared memory out anew
// (a single-class launch ends with the CTA, and its abort path already waits
// for what it issued).  `base` is the 1024-byte
// aligned start of dynamic shared memory, `tmem` the CTA's 512 TMEM columns,
// `pool` / `busy` the scratch pool of this K.
// RG = 1: residuals against the fp32 Gram matrix (resid_gram), with the
// remainder pieces in a scratch region; RG = 0: against A16 alone (none of
// that code is compiled in).  F8 = 1 (with BF): the e4m3 matvec; RG then
// makes the residual's remainder A - A_mv.
template <int K, bool BF, int LT, int RG, int F8, bool MULTI>
__device__ __forceinline__ void detect_tc_body(const DetectTcParams& P, uint8_t* base, uint32_t tmem, int64_t tile0,
                                               int64_t tstep, uint8_t* pool, int* busy) {
  Smem S;
  S.pipe = base;
  S.bars = reinterpret_cast<tcp::Bars*>(base + tcp::pipe_bytes(kTcStages32, tc_stage32_bytes(K)));
  S.sbars = reinterpret_cast<Bars2*>(S.bars + 1);
  S.tmem_slot = reinterpret_cast<uint32_t*>(S.sbars + 1);
  S.abort = reinterpret_cast<volatile int*>(S.tmem_slot + 1);
  S.region = const_cast<int*>(reinterpret_cast<volatile int*>(S.abort + 1));
  S.pool = pool;
  S.busy = busy;
  S.slots = base + tc_slots_offset(K);
  S.f8stage = S.slots + (size_t)P.nslots * tc_slot_bytes(K, LT, F8);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const tcp::Pipe& pp = P.pipe;
  for (int i = threadIdx.x; i < tcp::kStages * tcp::kStageBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(tcp::stage16(S.pipe, 0))[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    tcp::init_bars(*S.bars, kProdWarp - kCg0 - P.ncg, kTcStages32);
    for (int i = 0; i < kTcCgWarps; ++i) {
      tc::mbar_init(&S.sbars->slot_full[i], 1);
      tc::mbar_init(&S.sbars->slot_empty[i], 1);
    }
    *S.abort = 0;
    int got = -1;
    if (RG) {
      for (int t = 0; t < 2 * kTcScratchRegions && got < 0; ++t) {
        const int c = (int)((blockIdx.x + t) % kTcScratchRegions);
        if (atomicCAS(&busy[c], 0, 1) == 0) got = c;
      }
      __threadfence();  // the previous holder's accesses happen before ours
      if (got < 0) *S.abort = 1;  // not expected (one CTA per SM): no work, status FPCG_ST_TIMEOUT
    }
    *S.region = got;
    tc::fence_mbar_init();
  }
  tc::fence_proxy_async();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();

  if (*S.abort) {  // no scratch region: nothing was started; this CTA's systems are reported
    if (warp == kCg0 && P.status)
      for (int64_t tile = tile0; tile < pp.ntiles; tile += tstep)
        for (int p = lane; p < 64 / K; p += 32)
          if (tile * (64 / K) + p < pp.batch) P.status[tile * (64 / K) + p] = 32;
  } else if (warp == kMmaWarp) {
    if (lane == 0) tcp::mma_role<MULTI>(pp, S.pipe, *S.bars, S.abort, tmem, tile0, tstep);
    __syncwarp();
  } else if (warp == kProdWarp) {
    if (lane == 0) tcp::producer_role<kTcStages32, MULTI>(pp, S.pipe, *S.bars, S.abort, tile0, tstep);
    __syncwarp();
  } else if (warp >= kCg0 + P.ncg) {
    const int cw = warp - kCg0 - P.ncg;
    if (K <= 32 && P.ncg == 8) tcp::converter_role<2, kTcStages32>(pp, S.pipe, *S.bars, S.abort, tile0, tstep, cw, lane);
    else tcp::converter_role<4, kTcStages32>(pp, S.pipe, *S.bars, S.abort, tile0, tstep, cw, lane);
  } else if (warp >= kCg0) {
    if (warp - kCg0 < P.nslots) cg_role<K, BF, LT, RG, F8>(P, S, warp - kCg0, tile0, tstep);
  } else {
    drain_role<K, BF, LT, RG, F8>(P, S, tmem, tile0, tstep);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (RG && *S.region >= 0) {  // every access of this CTA to its region is done
      __threadfence();
      atomicExch(&busy[*S.region], 0);
    }
    if constexpr (MULTI) {
      tcp::inval_bars(*S.bars, kTcStages32);
      for (int i = 0; i < kTcCgWarps; ++i) {
        tc::mbar_inval(&S.sbars->slot_full[i]);
        tc::mbar_inval(&S.sbars->slot_empty[i]);
      }
    }
  }
  if constexpr (MULTI) __syncthreads();
}

// The fused detector for one class: one CTA per SM, tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...
template <int K, bool BF, int LT, int RG, int F8>
__global__ void __launch_bounds__(kThreads, 1) detect_tc_kernel(const __grid_constant__ DetectTcParams P) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ uint32_t s_tmem;
  const uint32_t a = tc::smem_u32(smem_raw);
  uint8_t* base = smem_raw + ((1024u - (a & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5;
  if (warp == kMmaWarp) tc::tmem_alloc(&s_tmem, 2 * tcp::kAccCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = s_tmem;
  detect_tc_body<K, BF, LT, RG, F8, false>(P, base, tmem, blockIdx.x, gridDim.x, g_rem<K>, g_rem_busy<K>);
  if (warp == kMmaWarp) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * tcp::kAccCols);
  }
}

// The fused detector for up to kTcMultiMax classes (K in {16, 32, 64}, the
// same matvec format, residual and block size) in one persistent launch.  The
// classes' tiles are numbered on, class after class, and dealt round-robin
// over the CTAs, so a CTA whose share of one class ends early starts on the
// next while the last tiles of the first still run elsewhere.
template <bool BF, int LT, int RG>
__global__ void __launch_bounds__(kThreads, 1) detect_tc_multi_kernel(const __grid_constant__ MultiTcParams M) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ uint32_t s_tmem;
  const uint32_t a = tc::smem_u32(smem_raw);
  uint8_t* base = smem_raw + ((1024u - (a & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5;
  if (warp == kMmaWarp) tc::tmem_alloc(&s_tmem, 2 * tcp::kAccCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int64_t g = gridDim.x;
  for (int c = 0; c < M.nclass; ++c) {
    const DetectTcParams& P = M.cls[c];
    const int64_t tile0 = (((int64_t)blockIdx.x - M.tile_base[c]) % g + g) % g;
    switch (P.pipe.K) {
      case 16: detect_tc_body<16, BF, LT, RG, 0, true>(P, base, tmem, tile0, g, M.pool[0], M.busy[0]); break;
      case 32: detect_tc_body<32, BF, LT, RG, 0, true>(P, base, tmem, tile0, g, M.pool[1], M.busy[1]); break;
      case 64: detect_tc_body<64, BF, LT, RG, 0, true>(P, base, tmem, tile0, g, M.pool[2], M.busy[2]); break;
      default: break;
    }
  }
  if (warp == kMmaWarp) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * tcp::kAccCols);
  }
}

// The launch settings of one class: CG warps (a valid preset -- 6, or 8 for
// K <= 32 -- is kept, anything else replaced by tc_cg_warps), slots, FP32 stage size.
inline void class_settings(DetectTcParams& P, int K, bool f8) {
  if (!(P.ncg == 6 || (P.ncg == 8 && K <= 32))) P.ncg = tc_cg_warps(K, P.pipe.N);
  P.nslots = tc_num_slots(K, P.L, f8);
  if (P.nslots > P.ncg) P.nslots = P.ncg;
  P.pipe.s32b = tc_stage32_bytes(K);
}

template <int K, bool BF, int LT, int RG, int F8 = 0>
cudaError_t launch_k(DetectTcParams P, int num_sms, cudaStream_t stream) {
  const size_t smem = detect_tc_smem_bytes(K, P.L, F8);
  class_settings(P, K, F8);
  cudaError_t e = cudaFuncSetAttribute(detect_tc_kernel<K, BF, LT, RG, F8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = P.pipe.ntiles < num_sms ? P.pipe.ntiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  detect_tc_kernel<K, BF, LT, RG, F8><<<(unsigned)grid, kThreads, smem, stream>>>(P);
  return cudaGetLastError();
}

template <bool BF, int LT, int RG>
cudaError_t launch_multi(MultiTcParams& M, int num_sms, cudaStream_t stream) {
  size_t smem = 0;
  int64_t tiles = 0;
  for (int c = 0; c < M.nclass; ++c) {
    DetectTcParams& P = M.cls[c];
    const int K = P.pipe.K;
    if ((K != 16 && K != 32 && K != 64) || P.L != LT) return cudaErrorInvalidValue;
    class_settings(P, K, false);
    const size_t sm = detect_tc_smem_bytes(K, LT);
    smem = sm > smem ? sm : smem;
    M.tile_base[c] = tiles;
    tiles += P.pipe.ntiles;
  }
  cudaError_t e =
      cudaFuncSetAttribute(detect_tc_multi_kernel<BF, LT, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = tiles < num_sms ? tiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  detect_tc_multi_kernel<BF, LT, RG><<<(unsigned)grid, kThreads, smem, stream>>>(M);
  return cudaGetLastError();
}

}  // namespace

template <int LT>
cudaError_t launch_detect_tc_multi_l(MultiTcParams& M, int num_sms, int mv_bf16, int resid_gram, cudaStream_t s) {
  if (M.nclass < 1 || M.nclass > kTcMultiMax) return cudaErrorInvalidValue;
  switch ((mv_bf16 ? 2 : 0) + (resid_gram ? 1 : 0)) {
    case 0: return launch_multi<false, LT, 0>(M, num_sms, s);
    case 1: return launch_multi<false, LT, 1>(M, num_sms, s);
    case 2: return launch_multi<true, LT, 0>(M, num_sms, s);
    default: return launch_multi<true, LT, 1>(M, num_sms, s);
  }
}

template <int K>
cudaError_t tc_rem_pool(cudaStream_t stream, uint8_t** pool, int** busy) {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static void* addr[kMaxDev][2] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (cap == cudaStreamCaptureStatusNone || !addr[dev][0]) {
    e = cudaGetSymbolAddress(&addr[dev][0], g_rem<K>);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&addr[dev][1], g_rem_busy<K>);
    if (e != cudaSuccess) {
      addr[dev][0] = addr[dev][1] = nullptr;
      return e;
    }
  }
  *pool = static_cast<uint8_t*>(addr[dev][0]);
  *busy = static_cast<int*>(addr[dev][1]);
  return cudaSuccess;
}

template <int K>
cudaError_t launch_detect_tc_k(const DetectTcParams& P, int num_sms, int mv, cudaStream_t stream) {
  if (mv == E4M3) {  // the residual against A_mv, or with the remainder against the fp32 Gram
    switch (P.L * 2 + (P.resid_gram ? 1 : 0)) {
      case 0: return launch_k<K, true, 0, 0, 1>(P, num_sms, stream);
      case 1: return launch_k<K, true, 0, 1, 1>(P, num_sms, stream);
      case 8: return launch_k<K, true, 4, 0, 1>(P, num_sms, stream);
      case 9: return launch_k<K, true, 4, 1, 1>(P, num_sms, stream);
      case 16: return launch_k<K, true, 8, 0, 1>(P, num_sms, stream);
      case 17: return launch_k<K, true, 8, 1, 1>(P, num_sms, stream);
      case 32: return launch_k<K, true, 16, 0, 1>(P, num_sms, stream);
      case 33: return launch_k<K, true, 16, 1, 1>(P, num_sms, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  const int mv_bf16 = mv == BF16;
  switch ((P.L * 2 + (mv_bf16 ? 1 : 0)) * 2 + (P.resid_gram ? 1 : 0)) {
    case 0: return launch_k<K, false, 0, 0>(P, num_sms, stream);
    case 1: return launch_k<K, false, 0, 1>(P, num_sms, stream);
    case 2: return launch_k<K, true, 0, 0>(P, num_sms, stream);
    case 3: return launch_k<K, true, 0, 1>(P, num_sms, stream);
    case 16: return launch_k<K, false, 4, 0>(P, num_sms, stream);
    case 17: return launch_k<K, false, 4, 1>(P, num_sms, stream);
    case 18: return launch_k<K, true, 4, 0>(P, num_sms, stream);
    case 19: return launch_k<K, true, 4, 1>(P, num_sms, stream);
    case 32: return launch_k<K, false, 8, 0>(P, num_sms, stream);
    case 33: return launch_k<K, false, 8, 1>(P, num_sms, stream);
    case 34: return launch_k<K, true, 8, 0>(P, num_sms, stream);
    case 35: return launch_k<K, true, 8, 1>(P, num_sms, stream);
    case 64: return launch_k<K, false, 16, 0>(P, num_sms, stream);
    case 65: return launch_k<K, false, 16, 1>(P, num_sms, stream);
    case 66: return launch_k<K, true, 16, 0>(P, num_sms, stream);
    case 67: return launch_k<K, true, 16, 1>(P, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpcg
