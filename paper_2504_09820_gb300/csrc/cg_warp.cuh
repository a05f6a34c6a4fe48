// The CG warp: one warp detects one system from a shared-memory slot holding
// A + sigma^2 I in the matvec format, the fp32 diagonal blocks M_d and b.
// Used by the fused tensor-core detector (slots filled from the Gram
// accumulator) and by the solver for given Gram matrices (slots filled from
// global memory).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "detect_tc.cuh"
#include "tc.cuh"
#include "tc_pipeline.cuh"

namespace fpcg {
namespace {

// ---- one system slot in shared memory -----------------------------------------
struct Slot {
  uint8_t* A16;     // [2K][K] 16-bit, row r at r*2K bytes, 16-byte chunk c at (c ^ swz(r));
                    // e4m3 matvec: [K][2K] bytes in the same row geometry (rows 0..K-1)
  float* sA;        // e4m3 matvec: scale of row k, k-tile kt at k * (K/16) + kt
  float2* Md;       // diagonal blocks of A (fp32), inverted in place (md_*_stride layout)
  float2* b;        // [K]
  float2* W;        // [K] matvec result, redistributed
  uint32_t* Pk;     // [3K] packed B fragments
  uint32_t* Pk8;    // e4m3 matvec: [6K] B fragments of x in six e4m3 pieces
  float* sv;        // e4m3 matvec: [K/16] block scales of the vector last packed
};

__device__ inline Slot slot_carve(uint8_t* base, int K, int L, bool f8 = false) {
  Slot s;
  uint8_t* p = base;
  s.A16 = p;
  if (f8) {
    p += 2 * K * K;
    s.sA = (float*)p;
    p += sizeof(float) * K * (K / 16);
  } else {
    s.sA = nullptr;
    p += 4 * K * K;
  }
  s.Md = (float2*)p;
  p += sizeof(float2) * (L > 0 ? (K / L) * md_block_stride(L) : 2);
  s.b = (float2*)p;
  p += sizeof(float2) * K;
  s.W = (float2*)p;
  p += sizeof(float2) * K;
  s.Pk = (uint32_t*)p;
  s.Pk8 = f8 ? s.Pk + 3 * K : nullptr;
  s.sv = f8 ? reinterpret_cast<float*>(s.Pk + 9 * K) : nullptr;
  return s;
}

// 16-byte chunk swizzle of row r of a [2K][K] 16-bit matrix (K/8 chunks per
// row): eight consecutive rows at one chunk hit eight different 16-byte bank
// groups of a 128-byte window.
template <int K>
__device__ __forceinline__ uint32_t a16_offset(int r, int chunk) {
  constexpr int CPR = K / 8;                           // chunks per row: 16, 8, 4, 2
  constexpr int SH = CPR >= 8 ? 0 : CPR == 4 ? 1 : 2;  // rows per swizzle step
  constexpr int MASK = (CPR >= 8 ? 8 : CPR) - 1;        // within one 128-byte bank window
  return (uint32_t)(r * (2 * K) + ((chunk ^ ((r >> SH) & MASK)) << 4));
}

// Byte offset of the 512-byte block holding one m16n8k16 A fragment (lane l's
// four registers at 16 l) of remainder piece pc, part pr (0: Re A, 1: Im A),
// m-tile mt and k-tile kt of a [2K][K] 16-bit matrix.  Element (r, c) of the
// 16 x 16 tile sits in lane (r % 8) * 4 + (c % 8) / 2, register r / 8 + 2 (c / 8),
// half c % 2.
template <int K>
__device__ __forceinline__ uint32_t rem_block(int pc, int pr, int mt, int kt) {
  return (uint32_t)((((pc * 2 + pr) * (K / 16) + mt) * (K / 16) + kt) * 512);
}

// Byte offset of row r (0..31: 16 rows of Re A, then 16 of Im A, of one
// m-tile) and 16-byte chunk c (columns 8c..8c+7 of one k-tile) in a 1 KB
// staging block of 16-bit values: the chunk swaps every four rows, so the
// eight rows of one ldmatrix phase fall on eight different 16-byte bank groups.
__device__ __forceinline__ uint32_t stg_offset(int r, int c) {
  return (uint32_t)(r * 32 + ((c ^ ((r >> 2) & 1)) << 4));
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <bool BF>
__device__ __forceinline__ uint32_t pk2(float a, float b) {
  return tcp::pack2(a, b, BF ? 1 : 0);
}

template <bool BF>
__device__ __forceinline__ float round16(float v) {
  if (BF) return __bfloat162float(__float2bfloat16_rn(v));
  return __half2float(__float2half_rn(v));
}

template <bool BF>
__device__ __forceinline__ void mma16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if (BF) tc::mma_m16n8k16_bf16(d, a, b0, b1);
  else tc::mma_m16n8k16_f16(d, a, b0, b1);
}

// In-place Gauss-Jordan inversion, no pivoting, of the K/L diagonal blocks
// (Hermitian positive definite, L x L) of M_d by one warp: lane l owns columns
// c = c0 + l + 32e (e < NE, c < K) of their blocks.  Per pivot pv, with
// d = 1 / M[pv][pv] and f = column pv of the block:
//   M[pv][j] <- M[pv][j] d,  M[i][j] <- M[i][j] - f_i M[pv][j] d   (j != pv)
//   M[pv][pv] <- d,          M[i][pv] <- -f_i d                    (j == pv)
// (one branch-free update for both cases).  Returns nonzero (on every lane) if
// a pivot was not positive.
template <int K, int LT, int NE>
__device__ __forceinline__ int gj_blocks(float2* Md, int lane, int c0 = 0) {
  constexpr int LD = md_row_stride(LT), BS = md_block_stride(LT);
  float2* M[NE];
  int j[NE];
  bool on[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int c = c0 + lane + 32 * e;
    on[e] = c < K;
    M[e] = Md + (on[e] ? (c / LT) * BS : 0);
    j[e] = c % LT;
  }
  int fail = 0;
#pragma unroll 1
  for (int pv = 0; pv < LT; ++pv) {
    float2 dinv[NE], mj[NE], f[NE][LT];
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const float2 piv = M[e][pv * LD + pv];
      if (on[e] && !(piv.x > 0.f && isfinite(piv.x))) fail = 1;
      const float rd = 1.f / (piv.x * piv.x + piv.y * piv.y);
      dinv[e] = make_float2(piv.x * rd, -piv.y * rd);
#pragma unroll
      for (int i = 0; i < LT; ++i) f[e][i] = M[e][i * LD + pv];
      mj[e] = M[e][pv * LD + j[e]];
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      if (!on[e]) continue;
      const bool own = j[e] == pv;
      const float2 prow = cmul(mj[e], dinv[e]);
      const float2 s = own ? dinv[e] : prow;
#pragma unroll
      for (int i = 0; i < LT; ++i) {  // row pv is rewritten below
        const float2 a = cmul(f[e][i], s);
        const float2 v = M[e][i * LD + j[e]];
        M[e][i * LD + j[e]] = own ? make_float2(-a.x, -a.y) : make_float2(v.x - a.x, v.y - a.y);
      }
      M[e][pv * LD + j[e]] = s;
    }
    __syncwarp();
  }
  return __any_sync(0xffffffffu, fail);
}

// Rounding of an inner product to u_IP when it is not fp32 (out of line: the
// format switch is rare and would otherwise be inlined at every call).
__device__ __noinline__ float round_ip(float v, int fmt) { return round_to(v, fmt); }

// ---- the CG warp -------------------------------------------------------------------
// Code size matters here: the CG warps share each SM sub-partition's
// instruction cache with the drain, converter, producer and MMA warps, and code
// that runs once per system is fetched cold.  So every step exists once in the
// code: the solves of all passes and the refinement residuals run in one loop,
// whose trips are either A p (a CG iteration) or b - A x (a residual).
// KR <= K: the system's own size; rows KR..K-1 of the slot are padding
// (identity rows of A, zeros of b) and are neither read from nor written to
// global memory.
//
// NV = 1: the warp works alone on its slot.  NV = 8: the eight warps of a CTA
// detect eight systems with one shared A in lockstep, and every product with
// A is one CTA-wide product A [v_0 .. v_7]: each warp packs its vector into
// the shared B fragments (S.Pk: n-tile nt, column c of k-tile kt at words
// ((kt*8 + nt)*8 + c)*8), then computes the rows of one m-tile for a share of
// the n-tiles, so A is read from shared memory once per trip instead of once
// per system.  A CG iteration uses two n-tiles (vectors 4nt..4nt+3, columns
// re, im of each); a residual uses one n-tile per vector (its six columns).
// S.b and S.W of warp v are at vbase + v * vst (and + 8K bytes).
//
// NS > 1: NS warps detect one system from one slot.  Every warp keeps the
// whole iteration state and repeats the scalar steps (identical results);
// each product with A is split by m-tiles over the NS warps between two
// barriers (id bar_id), and warp sj packs and writes the rows lane + 32e with
// e % NS == sj.  The preconditioner stages r in a warp-private buffer (rst),
// since the slot's W is shared.
//
// RM = 1: a residual trip also applies the remainder A - A16 of the fp32 Gram
// matrix (tc_rem_pieces 16-bit pieces, fragment order, at `rem`; skipped while
// rem is null), so that b - A x is formed against the fp32 Gram to within
// about 2^-22 of |A||x| (fp16) instead of against A16.
//
// RM = 2: a residual trip reads the fp32 Gram matrix itself from global
// memory (`agram`, KR x KR row-major; skipped while agram is null): b - A x
// with x in fp32, fp32 products and sums (apply_gram), within
// (2E + 6) u32 (|A||x| + |b|) of the exact residual; NV = 8: one CTA-wide pass
// over A for the eight vectors (apply_gram_cta).  For the solvers of given
// Gram matrices, which keep no remainder pieces.
//
// F8 = 1 (with BF, NV = NS = 1): the matvec of a CG iteration runs in e4m3
// (mma.sync m16n8k32) on the slot's A8 = A / s_A with one power-of-two scale
// s_A per row and 16-column block, against p quantised with one scale s_p per
// 16-entry block (the blocks of 32 interleaved real components of
// quant_e4m3); each block's fp32 partial sum is scaled by s_A s_p (exact) and
// accumulated in fp32.  A residual trip forms b - A_mv x on the same A8 with x
// in six e4m3 pieces (pack8x), and with RM = 1 subtracts (A - A_mv) x from
// the two bf16 remainder pieces in the scratch.
template <int K, bool BF, int LT, int KR = K, int NV = 1, int NS = 1, int RM = 0, int F8 = 0>
struct CgWarp {
  static constexpr int KT = K / 16;          // k-tiles (16 users)
  static constexpr int MT = K / 16;          // m-tiles of Re A (and of Im A)
  static constexpr int E = K >= 32 ? K / 32 : 1;  // vector rows per lane
  static constexpr int NCOL = 6;             // B columns (re, im) x (hi, mid, lo)
  static_assert(NV == 1 || (NV == 8 && MT <= 8), "cooperative mode: eight warps");
  static_assert(NS == 1 || (NV == 1 && E % NS == 0 && MT % NS == 0), "split mode: rows and m-tiles per warp");
  static_assert(!F8 || (BF && NV == 1 && NS == 1), "e4m3 matvec: one warp per slot, bf16 remainder pieces");
  const DetectTcParams& P;
  Slot S;
  int lane, g, t;
  int ipf, alpha_num, iters, refine_steps, refine_iters;  // parameters kept in registers
  int vw = 0;                // NV = 8: this warp's vector (its warp index)
  uint8_t* vbase = nullptr;  // NV = 8: per-vector b, W
  int vst = 0;
  int sj = 0, bar_id = 0;    // NS > 1: this warp's index in its system's group, the group's barrier
  float2* rst = nullptr;     // NS > 1: warp-private staging of r for the preconditioner
  const uint8_t* rem = nullptr;  // RM = 1: this slot's remainder pieces (global scratch)
  const float2* agram = nullptr; // RM = 2: this system's fp32 A + sigma^2 I (global, KR x KR)

  // NS > 1: rows lane + 32e this warp writes (packs, outputs)
  __device__ __forceinline__ bool mine(int e) const { return NS == 1 || e % NS == sj; }
  __device__ __forceinline__ void gsync() const {
    if constexpr (NS > 1) tc::bar_sync(bar_id, NS * 32);
  }

  __device__ CgWarp(const DetectTcParams& P_, Slot S_, int lane_) : P(P_), S(S_), lane(lane_) {
    g = lane >> 2;
    t = lane & 3;
    ipf = P_.ip;
    alpha_num = P_.alpha_num;
    iters = P_.iters;
    refine_steps = P_.refine_steps;
    refine_iters = P_.refine_iters;
  }

  __device__ __forceinline__ bool vact() const { return lane < K; }
  // row lane + 32e belongs to the system (not padding)
  __device__ __forceinline__ bool vout(int e) const { return KR == K ? vact() : lane + 32 * e < KR; }
  __device__ __forceinline__ float rip(float v) { return ipf == F32 ? v : round_ip(v, ipf); }

  // Re sum conj(a) b and Re sum conj(c) d over the warp's rows.
  __device__ __forceinline__ void dot2(const float2 (&a)[E], const float2 (&b)[E], const float2 (&c)[E],
                                       const float2 (&d)[E], float& s1, float& s2) {
    s1 = 0.f;
    s2 = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      s1 += a[e].x * b[e].x + a[e].y * b[e].y;
      s2 += c[e].x * d[e].x + c[e].y * d[e].y;
    }
    if (!vact()) s1 = s2 = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
  }

  // Store vector v (rows lane + 32e) as m16n8k16 B fragments: word
  // ((kt*NCOL + col)*4 + tt)*2 + h holds rows 16kt + 8h + 2tt, +1 of column
  // col.  Columns (re, im) of v rounded to the 16-bit format, then of the two
  // remainders when `split` (three pieces carry all 24 bits of an fp32 value;
  // zeros otherwise).
  __device__ __forceinline__ void pack(const float2 (&v)[E], bool split) {
    if constexpr (F8) {
      if (!split) {
        pack8(v);
        return;
      }
      pack8x(v);
      if constexpr (RM == 0) return;  // the bf16 split feeds the remainder pieces only
    }
    if constexpr (NS > 1 && NS == E) {  // split mode: only rows lane + 32 sj
      float2 vs = v[0];
#pragma unroll
      for (int e = 1; e < E; ++e)
        if (e == sj) vs = v[e];
      const float2 one[1] = {vs};
      pack_rows<1>(one, split, sj);
      return;
    }
    pack_rows<E>(v, split, 0);
  }

  // Rows lane + 32 (e0 + e) of v[e], e < NR, as B fragments (see pack).
  template <int NR>
  __device__ __forceinline__ void pack_rows(const float2 (&v)[NR], bool split, int e0) {
#pragma unroll
    for (int e = 0; e < NR; ++e) {
      const float nx = __shfl_down_sync(0xffffffffu, v[e].x, 1);
      const float ny = __shfl_down_sync(0xffffffffu, v[e].y, 1);
      const int rl = lane + 32 * (e0 + e);
      if (vact() && (rl & 1) == 0 && (NR < E || mine(e))) {
        const int kt = rl >> 4, j = rl & 15, tt = (j & 7) >> 1, h = j >> 3;
        uint32_t* w = S.Pk + tt * 2 + h +
                      (NV == 1 ? kt * NCOL * 8
                               : (split ? (kt * 8 + vw) * 64 : ((kt * 8 + (vw >> 2)) * 8 + 2 * (vw & 3)) * 8));
        float a[4] = {v[e].x, nx, v[e].y, ny};
        if (!split) {  // columns 2..5 feed only outputs the matvec does not read
          w[0] = pk2<BF>(a[0], a[1]);
          w[8] = pk2<BF>(a[2], a[3]);
        } else {
#pragma unroll
          for (int s3 = 0; s3 < 3; ++s3) {
            float hh[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              hh[u] = round16<BF>(a[u]);
              a[u] -= hh[u];  // exact remainder of the rounding
            }
            w[(2 * s3) * 8] = pk2<BF>(hh[0], hh[1]);
            w[(2 * s3 + 1) * 8] = pk2<BF>(hh[2], hh[3]);
          }
        }
      }
    }
    __syncwarp();
  }

  // F8: v as e4m3 B fragments.  k-tile kt holds entries 16kt..16kt+15 (the
  // real components 32kt..32kt+31 of v, Re and Im interleaved), divided by
  // their block's scale S.sv[kt] (e4m3_scale of the block's largest |component|)
  // and rounded to e4m3.  Column 0 holds (Re v_l, -Im v_l) pairs and column 1
  // (Im v_l, Re v_l), so that a row of A8 (Re, Im interleaved) times them gives
  // Re and Im of (A v)_k.  Word ((kt*2 + col)*4 + tt)*2 + h holds rows
  // 16h + 4tt .. 16h + 4tt + 3 of the k-tile: entries 16kt + 8h + 2tt and + 1.
  // The scales go to S.sv.
  __device__ __forceinline__ void pack8(const float2 (&v)[E]) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      float inv;
      const float s = block_scale(v[e], inv);
      if ((lane & 15) == 0 && 2 * e + (lane >> 4) < KT) S.sv[2 * e + (lane >> 4)] = s;  // k-tile 2e + lane / 16
      put8(S.Pk, lane + 32 * e, 0, e4m3_pairs(tc::cvt_e4m3x2(v[e].x * inv, v[e].y * inv)));
    }
    __syncwarp();
  }

  // The e4m3 scale of the 16-entry block (16 lanes) holding this lane's entry v.
  __device__ __forceinline__ float block_scale(float2 v, float& inv) const {
    float m = vact() ? fmaxf(fabsf(v.x), fabsf(v.y)) : 0.f;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    return e4m3_scale_inv(m, inv);
  }

  // The two B-column byte pairs of one entry from its e4m3 bytes (Re in byte
  // 0, Im in byte 1): (Re, -Im) in the low half, (Im, Re) in the high half.
  __device__ __forceinline__ static uint32_t e4m3_pairs(uint32_t q) {
    const uint32_t c0 = (q & 0xffu) | ((q ^ 0x8000u) & 0xff00u);
    const uint32_t c1 = ((q >> 8) & 0xffu) | ((q & 0xffu) << 8);
    return c0 | (c1 << 16);
  }

  // Row rl's pairs (and row rl + 1's, from the next lane) into the words of
  // piece pc: word ((((kt * NP + pc) * 2 + col) * 4 + tt) * 2 + h, NP the
  // pieces of the array (1 for p, 6 for x).
  template <int NP = 1>
  __device__ __forceinline__ void put8(uint32_t* base, int rl, int pc, uint32_t mine) {
    const uint32_t nb = __shfl_down_sync(0xffffffffu, mine, 1);
    if (vact() && (rl & 1) == 0) {
      const int kt = rl >> 4, j = rl & 15, tt = (j & 7) >> 1, h = j >> 3;
      uint32_t* w = base + ((((kt * NP + pc) * 2) * 4 + tt) * 2 + h);
      w[0] = (mine & 0xffffu) | (nb << 16);
      w[8] = (mine >> 16) | (nb & 0xffff0000u);
    }
  }

  // F8 residual: x = s0 sum_i 2^(-4i) q_i, q_i in e4m3, six pieces per entry:
  // s0 = S.sv[kt] is the e4m3 scale of the block, and piece i + 1 quantises the
  // exact remainder of piece i in units 16 times smaller.  The remainder of an
  // e4m3 rounding is at most 2^-4 of the value (subnormals: 2^-10), so no
  // piece saturates, and what is left after six is below 2^-24 of the block's
  // largest entry.  Pieces go to S.Pk8 (put8 with NP = 6), s0 to S.sv.
  __device__ __forceinline__ void pack8x(const float2 (&v)[E]) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      float inv;
      const float s = block_scale(v[e], inv);
      if ((lane & 15) == 0 && 2 * e + (lane >> 4) < KT) S.sv[2 * e + (lane >> 4)] = s;
      float rx = v[e].x * inv, ry = v[e].y * inv;  // exact: inv is a power of two
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const uint32_t q = tc::cvt_e4m3x2(rx, ry);
        const float2 dq = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)q, __NV_E4M3)));
        rx = (rx - dq.x) * 16.f;  // exact
        ry = (ry - dq.y) * 16.f;
        put8<6>(S.Pk8, lane + 32 * e, i, e4m3_pairs(q));
      }
    }
    __syncwarp();
  }

  // F8: W = A8 v with the block scales, one m-tile (16 rows of A8) pair at a
  // time; every k-tile's mma starts from zero and its fp32 partial sums are
  // scaled by s_A s_p and added.  Lane (g, t = 0) holds rows g, g + 8 of the
  // columns Re, Im.
  __device__ __forceinline__ void apply8(float2 (&w)[E]) {
    uint32_t b0[KT], b1[KT];
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      b0[kt] = b1[kt] = 0u;
      if (g < 2) {
        const uint2 pw = *reinterpret_cast<const uint2*>(S.Pk + ((kt * 2 + g) * 4 + t) * 2);
        b0[kt] = pw.x;
        b1[kt] = pw.y;
      }
    }
    const uint32_t abase = tc::smem_u32(S.A16);
    const int lr = lane & 15, lc = lane >> 4;
    constexpr int MP = MT >= 2 ? 2 : 1;
    const float zero[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int mt0 = 0; mt0 < MT; mt0 += MP) {
      float acc[MP][4];
      float sa[MP][2][KT];
#pragma unroll
      for (int j = 0; j < MP; ++j) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int kt = 0; kt < KT; ++kt) sa[j][h][kt] = S.sA[(16 * (mt0 + j) + g + 8 * h) * KT + kt] * S.sv[kt];
      }
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
#pragma unroll
        for (int j = 0; j < MP; ++j) {
          uint32_t a[4];
          float c[4];
          tc::ldmatrix_x4(a, abase + a16_offset<K>(16 * (mt0 + j) + lr, 2 * kt + lc));
          tc::mma_m16n8k32_e4m3(c, a, b0[kt], b1[kt], zero);
          acc[j][0] = fmaf(c[0], sa[j][0][kt], acc[j][0]);
          acc[j][1] = fmaf(c[1], sa[j][0][kt], acc[j][1]);
          acc[j][2] = fmaf(c[2], sa[j][1][kt], acc[j][2]);
          acc[j][3] = fmaf(c[3], sa[j][1][kt], acc[j][3]);
        }
      }
      if (t == 0) {
#pragma unroll
        for (int j = 0; j < MP; ++j) {
          S.W[16 * (mt0 + j) + g] = make_float2(acc[j][0], acc[j][1]);
          S.W[16 * (mt0 + j) + g + 8] = make_float2(acc[j][2], acc[j][3]);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e) w[e] = vact() ? S.W[lane + 32 * e] : make_float2(0.f, 0.f);
    __syncwarp();
  }

  // F8 residual: S.W = b - A_mv x on A8, x from its six pieces in S.Pk8.
  // n-tile 0 holds pieces 0-3 and n-tile 1 pieces 4, 5 (column 2i + c: piece
  // i, column c of pack8), so lane (g, t) accumulates pieces t and 4 + t, each
  // in its own units; they are scaled by 2^(-4 piece) and summed over the
  // quad, smallest first.
  __device__ __forceinline__ void res8() {
    const uint32_t abase = tc::smem_u32(S.A16);
    const int lr = lane & 15, lc = lane >> 4;
    const float f0 = __uint_as_float((uint32_t)(127 - 4 * t) << 23);       // 2^(-4t)
    const float f1 = __uint_as_float((uint32_t)(127 - 16 - 4 * t) << 23);  // 2^(-4(4 + t))
    const float zero[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
      float acc[2][4], sa[2][KT];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[0][q] = acc[1][q] = 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) sa[h][kt] = S.sA[(16 * mt + g + 8 * h) * KT + kt] * S.sv[kt];
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
        uint32_t a[4];
        tc::ldmatrix_x4(a, abase + a16_offset<K>(16 * mt + lr, 2 * kt + lc));
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int pc = 4 * nt + (g >> 1);  // pieces 6, 7: zero columns
          const uint2 pw = pc < 6 ? *reinterpret_cast<const uint2*>(
                                        S.Pk8 + ((((kt * 6 + pc) * 2 + (g & 1)) * 4 + t) * 2))
                                  : make_uint2(0u, 0u);
          float c[4];
          tc::mma_m16n8k32_e4m3(c, a, pw.x, pw.y, zero);
          acc[nt][0] = fmaf(c[0], sa[0][kt], acc[nt][0]);
          acc[nt][1] = fmaf(c[1], sa[0][kt], acc[nt][1]);
          acc[nt][2] = fmaf(c[2], sa[1][kt], acc[nt][2]);
          acc[nt][3] = fmaf(c[3], sa[1][kt], acc[nt][3]);
        }
      }
      float v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[q] = fmaf(acc[0][q], f0, acc[1][q] * f1);
        v[q] += __shfl_xor_sync(0xffffffffu, v[q], 2);
        v[q] += __shfl_xor_sync(0xffffffffu, v[q], 1);
      }
      if (t == 0) {
        const float2 bb0 = S.b[16 * mt + g], bb8 = S.b[16 * mt + g + 8];
        S.W[16 * mt + g] = make_float2(bb0.x - v[0], bb0.y - v[1]);
        S.W[16 * mt + g + 8] = make_float2(bb8.x - v[2], bb8.y - v[3]);
      }
    }
  }

  // F8: a CG iteration's A p (apply8) or a residual (res8, then the
  // remainder pieces with RM = 1), then w = W.
  __device__ __forceinline__ void apply_f8(bool res, float2 (&w)[E]) {
    if (!res) {
      apply8(w);
      return;
    }
    res8();
    if constexpr (RM == 1)
      if (rem != nullptr) {
        uint32_t b0[KT], b1[KT];
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
          b0[kt] = b1[kt] = 0u;
          if (g < NCOL) {
            const uint2 pw = *reinterpret_cast<const uint2*>(S.Pk + ((kt * NCOL + g) * 4 + t) * 2);
            b0[kt] = pw.x;
            b1[kt] = pw.y;
          }
        }
        uint4 q[2][KT];
        rem_load(rem, 0, q);
        __syncwarp();
        rem_apply(rem, b0, b1, q);
      }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e) w[e] = vact() ? S.W[lane + 32 * e] : make_float2(0.f, 0.f);
    __syncwarp();
  }

  // Rows 16mt.. of W = A v (or b - A v) for the NMT m-tiles mt0.. from the B
  // fragments b0, b1: the m-tiles interleaved along k, two accumulator
  // chains (even / odd k-tile) per m-tile and part.
  template <int NMT>
  __device__ __forceinline__ void apply_mtiles(int mt0, bool res, const uint32_t (&b0)[KT], const uint32_t (&b1)[KT]) {
    const uint32_t abase = tc::smem_u32(S.A16);
    const int lr = lane & 15, lc = lane >> 4;
    float cr[NMT][2][4], ci[NMT][2][4];
#pragma unroll
    for (int j = 0; j < NMT; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 4; ++q) cr[j][h][q] = ci[j][h][q] = 0.f;
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
#pragma unroll
      for (int j = 0; j < NMT; ++j) {
        uint32_t ar[4], ai[4];
        tc::ldmatrix_x4(ar, abase + a16_offset<K>(16 * (mt0 + j) + lr, 2 * kt + lc));
        tc::ldmatrix_x4(ai, abase + a16_offset<K>(K + 16 * (mt0 + j) + lr, 2 * kt + lc));
        mma16<BF>(cr[j][kt & 1], ar, b0[kt], b1[kt]);
        mma16<BF>(ci[j][kt & 1], ai, b0[kt], b1[kt]);
      }
    }
#pragma unroll
    for (int j = 0; j < NMT; ++j) {
      const int mt = mt0 + j;
      float r[4], im[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        r[q] = cr[j][0][q] + cr[j][1][q];
        im[q] = ci[j][0][q] + ci[j][1][q];
      }
      if (res) {  // add the mid (t = 1) and lo (t = 2) column products into t = 0
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float r1 = __shfl_down_sync(0xffffffffu, r[q], 1);
          const float r2 = __shfl_down_sync(0xffffffffu, r[q], 2);
          const float i1 = __shfl_down_sync(0xffffffffu, im[q], 1);
          const float i2 = __shfl_down_sync(0xffffffffu, im[q], 2);
          r[q] += r1 + r2;
          im[q] += i1 + i2;
        }
      }
      if (t == 0) {
        // rows 16mt+g / +8: (Re A vr - Im A vi) + i (Re A vi + Im A vr)
        float2 w0 = make_float2(r[0] - im[1], r[1] + im[0]);
        float2 w8 = make_float2(r[2] - im[3], r[3] + im[2]);
        if (res) {
          const float2 bb0 = S.b[16 * mt + g], bb8 = S.b[16 * mt + g + 8];
          w0 = make_float2(bb0.x - w0.x, bb0.y - w0.y);
          w8 = make_float2(bb8.x - w8.x, bb8.y - w8.y);
        }
        S.W[16 * mt + g] = w0;
        S.W[16 * mt + g + 8] = w8;
      }
    }
  }

  // Remainder fragments of round i = piece * MT + m-tile (both parts), from
  // src: the global scratch, or the slot's A16 region once they are staged there.
  __device__ __forceinline__ void rem_load(const uint8_t* src, int i, uint4 (&q)[2][KT]) {
    const int pc = i / MT, mt = i % MT;
    if (src == rem) {  // global scratch
      const uint64_t keep = tc::policy_evict_last();
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
        q[0][kt] = tc::ld_global_hint(src + rem_block<K>(pc, 0, mt, kt) + 16 * lane, keep);
        q[1][kt] = tc::ld_global_hint(src + rem_block<K>(pc, 1, mt, kt) + 16 * lane, keep);
      }
    } else {  // staged in the slot
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
        q[0][kt] = *reinterpret_cast<const uint4*>(src + rem_block<K>(pc, 0, mt, kt) + 16 * lane);
        q[1][kt] = *reinterpret_cast<const uint4*>(src + rem_block<K>(pc, 1, mt, kt) + 16 * lane);
      }
    }
  }

  // W -= (A - A16) x after the A16 part of a residual trip: one m-tile (of
  // one remainder piece) per round, the next round's fragments loaded while
  // this round's products are combined.  Rows of W belong to the lanes t = 0
  // that wrote them.
  __device__ __forceinline__ void rem_apply(const uint8_t* src, const uint32_t (&b0)[KT], const uint32_t (&b1)[KT],
                                            uint4 (&q)[2][KT]) {
    constexpr int NR = tc_rem_pieces(BF) * MT;
#pragma unroll 1
    for (int i = 0; i < NR; ++i) {
      float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
        const uint32_t ar[4] = {q[0][kt].x, q[0][kt].y, q[0][kt].z, q[0][kt].w};
        const uint32_t ai[4] = {q[1][kt].x, q[1][kt].y, q[1][kt].z, q[1][kt].w};
        mma16<BF>(cr, ar, b0[kt], b1[kt]);
        mma16<BF>(ci, ai, b0[kt], b1[kt]);
      }
      if (i + 1 < NR) rem_load(src, i + 1, q);
#pragma unroll
      for (int u = 0; u < 4; ++u) {  // the mid (t = 1) and lo (t = 2) column products into t = 0
        cr[u] += __shfl_down_sync(0xffffffffu, cr[u], 1) + __shfl_down_sync(0xffffffffu, cr[u], 2);
        ci[u] += __shfl_down_sync(0xffffffffu, ci[u], 1) + __shfl_down_sync(0xffffffffu, ci[u], 2);
      }
      if (t == 0) {
        const int mt = i % MT;
        float2* w0 = S.W + 16 * mt + g;
        const float2 a0 = w0[0], a8 = w0[8];
        w0[0] = make_float2(a0.x - (cr[0] - ci[1]), a0.y - (cr[1] + ci[0]));
        w0[8] = make_float2(a8.x - (cr[2] - ci[3]), a8.y - (cr[3] + ci[2]));
      }
    }
  }

  // RM = 2: W = b - A x from the fp32 Gram matrix in global memory, then w = W
  // (x arrives in w); one warp (NS warps) per system, or (NV = 8) one
  // CTA-wide pass for the eight vectors.  Defined in gram_resid.cuh, which
  // the solvers for given Gram matrices include.
  __device__ __forceinline__ void apply_gram(float2 (&w)[E]);
  __device__ __forceinline__ void apply_gram_cta(float2 (&w)[E]);

  // W = A v (res = false) or W = b - A v (res = true: the three column pairs
  // of v are summed), one m-tile (16 rows of Re A and of Im A) at a time; lane
  // (g, t) holds C rows g, g+8 and columns 2t, 2t+1.  Then w = W in the vector
  // layout.
  // last: this residual is the system's final one (the slot's A16 is free afterwards).
  __device__ __forceinline__ void apply(bool res, float2 (&w)[E], bool last = false) {
    if constexpr (RM == 2)
      if (res && agram != nullptr) {  // the same on every warp of a CTA (NV > 1) or system (NS > 1)
        if constexpr (NV > 1) apply_gram_cta(w);
        else apply_gram(w);
        return;
      }
    if constexpr (NV > 1) {
      apply_cta(res, w);
      return;
    }
    if constexpr (F8) {
      apply_f8(res, w);
      return;
    }
    gsync();  // NS > 1: every warp's rows are packed
    uint32_t b0[KT], b1[KT];
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      b0[kt] = b1[kt] = 0u;
      if (g < NCOL) {
        const uint2 pw = *reinterpret_cast<const uint2*>(S.Pk + ((kt * NCOL + g) * 4 + t) * 2);
        b0[kt] = pw.x;
        b1[kt] = pw.y;
      }
    }
    if constexpr (NS > 1) {  // this warp's m-tiles interleaved along k
      apply_mtiles<MT / NS>(sj * (MT / NS), res, b0, b1);
    } else {  // m-tiles in pairs: more independent chains, a rolled loop keeps the code small
      constexpr int MP = MT >= 2 ? 2 : 1;
#pragma unroll 1
      for (int mt = 0; mt < MT; mt += MP) apply_mtiles<MP>(mt, res, b0, b1);
      if constexpr (RM == 1)
        if (res && rem != nullptr) {
          const uint8_t* src = rem;
          if (last && tc_rem_pieces(BF) == 1) {  // A16 (as large as one piece) is not read again:
            // stage the remainder there, one round trip from L2 for all of it
            constexpr int kChunks = (int)tc_rem_piece_bytes(K) / 512;
            const uint32_t dst = tc::smem_u32(S.A16);
            __syncwarp();  // every lane's reads of A16 come first
#pragma unroll 4
            for (int c = 0; c < kChunks; ++c) tc::cp_async16(dst + 512 * c + 16 * lane, rem + 512 * c + 16 * lane);
            tc::cp_async_wait_all();  // each lane reads back only the bytes it copied
            src = S.A16;
          }
          uint4 q[2][KT];
          rem_load(src, 0, q);
          __syncwarp();
          rem_apply(src, b0, b1, q);
        }
    }
    __syncwarp();
    gsync();  // NS > 1: every m-tile of W is written
#pragma unroll
    for (int e = 0; e < E; ++e) w[e] = vact() ? S.W[lane + 32 * e] : make_float2(0.f, 0.f);
    __syncwarp();
  }

  // NV = 8: n-tiles nt0 .. nt0 + NB - 1 of m-tile mt, A fragments loaded once
  // per k-tile; results into the W of their vectors.
  template <int NB>
  __device__ __forceinline__ void cta_tiles(int mt, int nt0, bool res) {
    float cr[NB][4], ci[NB][4];
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) cr[j][q] = ci[j][q] = 0.f;
    const uint32_t abase = tc::smem_u32(S.A16);
    const int lr = lane & 15, lc = lane >> 4;
    const bool bz = res && g >= NCOL;  // residual n-tiles: columns 6, 7 are zero
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      uint32_t ar[4], ai[4];
      tc::ldmatrix_x4(ar, abase + a16_offset<K>(16 * mt + lr, 2 * kt + lc));
      tc::ldmatrix_x4(ai, abase + a16_offset<K>(K + 16 * mt + lr, 2 * kt + lc));
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        uint2 pw = *reinterpret_cast<const uint2*>(S.Pk + ((kt * 8 + nt0 + j) * 8 + g) * 8 + 2 * t);
        if (bz) pw = make_uint2(0u, 0u);
        mma16<BF>(cr[j], ar, pw.x, pw.y);
        mma16<BF>(ci[j], ai, pw.x, pw.y);
      }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int nt = nt0 + j;
      if (res) {  // n-tile = vector nt: add the mid and lo column products into t = 0
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float r1 = __shfl_down_sync(0xffffffffu, cr[j][q], 1);
          const float r2 = __shfl_down_sync(0xffffffffu, cr[j][q], 2);
          const float i1 = __shfl_down_sync(0xffffffffu, ci[j][q], 1);
          const float i2 = __shfl_down_sync(0xffffffffu, ci[j][q], 2);
          cr[j][q] += r1 + r2;
          ci[j][q] += i1 + i2;
        }
      }
      if (!res || t == 0) {
        const int v = res ? nt : 4 * nt + t;
        float2* Wv = reinterpret_cast<float2*>(vbase + v * vst + 8 * K);
        float2 w0 = make_float2(cr[j][0] - ci[j][1], cr[j][1] + ci[j][0]);
        float2 w8 = make_float2(cr[j][2] - ci[j][3], cr[j][3] + ci[j][2]);
        if (res) {
          const float2* bv = reinterpret_cast<const float2*>(vbase + v * vst);
          const float2 bb0 = bv[16 * mt + g], bb8 = bv[16 * mt + g + 8];
          w0 = make_float2(bb0.x - w0.x, bb0.y - w0.y);
          w8 = make_float2(bb8.x - w8.x, bb8.y - w8.y);
        }
        Wv[16 * mt + g] = w0;
        Wv[16 * mt + g + 8] = w8;
      }
    }
  }

  // NV = 8: the CTA-wide product; warp vw takes m-tile vw / WPM and its share
  // of the n-tiles (2 for a CG iteration, 8 for a residual).
  __device__ __forceinline__ void apply_cta(bool res, float2 (&w)[E]) {
    constexpr int WPM = 8 / MT;                 // warps per m-tile
    constexpr int NPI = WPM >= 2 ? 1 : 2;       // iteration n-tiles per warp
    constexpr int NPR = 8 / WPM;                // residual n-tiles per warp
    constexpr int NBR = NPR > 2 ? 2 : NPR;      // residual n-tiles per pass over A (registers)
    const int mt = vw / WPM, sub = vw % WPM;
    __syncthreads();  // every vector is packed
    if (!res) {
      if (sub * NPI < 2) cta_tiles<NPI>(mt, sub * NPI, false);
    } else {
#pragma unroll
      for (int c = 0; c < NPR; c += NBR) cta_tiles<NBR>(mt, sub * NPR + c, true);
    }
    __syncthreads();  // every W is complete
#pragma unroll
    for (int e = 0; e < E; ++e) w[e] = vact() ? S.W[lane + 32 * e] : make_float2(0.f, 0.f);
  }

  // z = M_d r (z = r without a preconditioner): r is staged in W and each
  // lane reads its block's L entries of it (broadcast) and its row of M_d.
  __device__ __forceinline__ void precond(const float2 (&r)[E], float2 (&z)[E]) {
    if constexpr (LT == 0) {
#pragma unroll
      for (int e = 0; e < E; ++e) z[e] = r[e];
    } else {
      constexpr int MLD = md_row_stride(LT), MBS = md_block_stride(LT);
      float2* st = NS > 1 ? rst : S.W;
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (vact()) st[lane + 32 * e] = r[e];
      __syncwarp();
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = vact() ? lane + 32 * e : 0;
        const float4* rb = reinterpret_cast<const float4*>(st + (k & ~(LT - 1)));
        const float4* mr = reinterpret_cast<const float4*>(S.Md + (k / LT) * MBS + (k % LT) * MLD);
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < LT / 2; ++q) {  // entries 2q, 2q+1
          const float4 m = mr[q], v = rb[q];
          a0.x = fmaf(m.x, v.x, fmaf(-m.y, v.y, a0.x));
          a0.y = fmaf(m.x, v.y, fmaf(m.y, v.x, a0.y));
          a1.x = fmaf(m.z, v.z, fmaf(-m.w, v.w, a1.x));
          a1.y = fmaf(m.z, v.w, fmaf(m.w, v.z, a1.y));
        }
        z[e] = vact() ? make_float2(a0.x + a1.x, a0.y + a1.y) : make_float2(0.f, 0.f);
      }
      __syncwarp();
    }
  }

  // The whole detection of one system from its slot.  Pass 0 runs Algorithm 2
  // (LT == 0) or 3 on b from x0 = 0; each refinement pass runs it again on the
  // residual b - A x and adds the correction; the last trip is the final
  // residual.
  // Block-Jacobi setup (eq. pre_BJ) on the slot's M_d: FPCG_ST_BJ_FAIL (8) and
  // M_d = I if a diagonal block was not positive definite, else 0.
  __device__ int bj_setup() {
    if constexpr (LT > 0 && NS > 1) {  // warp sj inverts the blocks of columns 32 (sj + NS r) ..
      constexpr int MLD = md_row_stride(LT), MBS = md_block_stride(LT);
      int fail = 0;
#pragma unroll 1
      for (int c0 = 32 * sj; c0 < K; c0 += 32 * NS) fail |= gj_blocks<K, LT, 1>(S.Md, lane, c0);
      if (tc::bar_or(bar_id, NS * 32, fail)) {  // a failed block: M_d = I for the system
        for (int i = sj * 32 + lane; i < K * LT; i += NS * 32)
          S.Md[(i / LT / LT) * MBS + ((i / LT) % LT) * MLD + i % LT] =
              make_float2((i / LT) % LT == i % LT ? 1.f : 0.f, 0.f);
        gsync();
        return 8;
      }
      return 0;
    } else if constexpr (LT > 0) {
      constexpr int MLD = md_row_stride(LT), MBS = md_block_stride(LT);
      int fail;
      if constexpr (E <= 2) {
        fail = gj_blocks<K, LT, E>(S.Md, lane);
      } else {  // columns in rounds of 64 (a block never straddles two)
        fail = 0;
#pragma unroll 1
        for (int c0 = 0; c0 < K; c0 += 64) fail |= gj_blocks<K, LT, 2>(S.Md, lane, c0);
      }
      if (fail) {
        for (int i = lane; i < K * LT; i += 32)
          S.Md[(i / LT / LT) * MBS + ((i / LT) % LT) * MLD + i % LT] =
              make_float2((i / LT) % LT == i % LT ? 1.f : 0.f, 0.f);
        __syncwarp();
        return 8;
      }
    }
    return 0;
  }

  // A system whose group index is out of range: x_hat = 0, labels 0,
  // rel_res = 0, FPCG_ST_BAD_INDEX (64); no bit errors counted.
  __device__ void bad_index(int64_t sys) {
    if (NS > 1 && sj != 0) return;
    const int64_t base = sys * (int64_t)KR;
    for (int k = lane; k < KR; k += 32) {
      P.x_hat[base + k] = make_float2(0.f, 0.f);
      if (P.sym) P.sym[base + k] = 0;
    }
    if (lane == 0) {
      if (P.rel_res) P.rel_res[sys] = 0.0;
      if (P.status) P.status[sys] = 64;
    }
  }

  // st0: status bits already known for this system (from bj_setup).
  __device__ void detect(int64_t sys, bool valid, int st0) {
    int st = st0;
    // per-system inputs of the output stage, loaded now (their latency hides under the solve)
    const int64_t base = sys * (int64_t)KR;
    const bool want_sym = valid && (P.sym || P.bit_errors);
    const int M = want_sym ? P.qam[sys] : 0;
    int txv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) txv[e] = (want_sym && P.tx && vout(e) && mine(e)) ? P.tx[base + lane + 32 * e] : 0;
    float* hist = (P.res_hist && valid) ? P.res_hist + sys * (int64_t)(iters + 1) : nullptr;

    float2 x[E], d[E], r[E], p[E], z[E], w[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      x[e] = d[e] = p[e] = make_float2(0.f, 0.f);
      r[e] = vact() ? S.b[lane + 32 * e] : make_float2(0.f, 0.f);
    }
    int pass = 0, it = 0, iters_p = iters, mask = ~0;
    float rho = 0.f, rho_prev = 1.f, rr = 0.f;
    bool fresh = true;    // r is a new right-hand side: start a pass
    bool frozen = false;  // NV = 8: this pass broke down; its remaining trips change nothing
#pragma unroll 1
    while (true) {
      if (!fresh) {
        const bool rt = it >= iters_p;  // this trip: residual, else a CG iteration
        if (rt) {
#pragma unroll
          for (int e = 0; e < E; ++e) x[e] = make_float2(x[e].x + d[e].x, x[e].y + d[e].y);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) w[e] = rt ? x[e] : p[e];
        if (RM != 2 || !rt || agram == nullptr) pack(w, rt);  // RM = 2 residuals read x in fp32
        apply(rt, w, rt && pass >= refine_steps);
        if (rt) {
#pragma unroll
          for (int e = 0; e < E; ++e) r[e] = w[e];  // r = b - A x
          if (pass >= refine_steps) break;
          ++pass;
          iters_p = refine_iters;
          it = 0;
          mask = 1;  // a refinement pass reports breakdown only
          hist = nullptr;
#pragma unroll
          for (int e = 0; e < E; ++e) d[e] = make_float2(0.f, 0.f);
          fresh = true;
          frozen = false;
        } else {
          if (NV > 1 && frozen) {  // lockstep with the other warps: the trip is taken, nothing changes
            ++it;
            continue;
          }
          float phi, rp;
          dot2(p, w, r, p, phi, rp);
          phi = rip(phi);
          rho_prev = (LT > 0 && alpha_num == 0) ? rip(rp) : rho;
          int bad = 0;
          if (rho_prev == 0.f) bad = 2;
          else if (!(phi > 0.f) || !isfinite(phi) || !isfinite(rho_prev)) bad = 1;
          if (bad) {  // the pass stops here; the history repeats its last value
            st |= bad & mask;
            if (hist && lane == 0 && sj == 0)
              for (int k = it + 1; k <= iters_p; ++k) hist[k] = hist[it];
            if constexpr (NV > 1) {  // the other warps still take this pass's trips
              frozen = true;
#pragma unroll
              for (int e = 0; e < E; ++e) p[e] = make_float2(0.f, 0.f);  // packed from now on: finite
              ++it;
            } else {
              it = iters_p;
            }
            continue;
          }
          const float alpha = __fdividef(rho_prev, phi);  // within 2 ulp of fl(rho / phi)
#pragma unroll
          for (int e = 0; e < E; ++e) {
            d[e] = make_float2(fmaf(alpha, p[e].x, d[e].x), fmaf(alpha, p[e].y, d[e].y));
            r[e] = make_float2(fmaf(-alpha, w[e].x, r[e].x), fmaf(-alpha, w[e].y, r[e].y));
          }
          ++it;
        }
      }
      // z = M_d r, rho = r^H z, and the next direction
      precond(r, z);
      float rz;
      dot2(r, z, r, r, rz, rr);
      const float rho_new = rip(rz);
      const float beta = fresh ? 0.f : __fdividef(rho_new, rho_prev);
#pragma unroll
      for (int e = 0; e < E; ++e)
        p[e] = fresh ? z[e] : make_float2(fmaf(beta, p[e].x, z[e].x), fmaf(beta, p[e].y, z[e].y));
      rho = rho_new;
      if (hist && lane == 0 && sj == 0) hist[it] = sqrtf(rr);
      fresh = false;
    }

    if (!valid) return;
    float nr = 0.f, nb = 0.f;  // squared norms of the final residual and of b (the ratio in fp64)
    int nonfinite = 0;
    unsigned errs = 0;
    const int m = qam_sqrt(M);
    const float sc = m ? sqrtf((float)(2 * (M - 1) / 3)) : 0.f;  // 2(M-1)/3 is an integer here
    const int nb2 = m ? qam_bits_axis(m) : 0;
    if (vact()) {
#pragma unroll  // x, r, txv stay in registers only with static indices
      for (int e = 0; e < E; ++e) {
        const float2 bv = S.b[lane + 32 * e];
        nr = fmaf(r[e].x, r[e].x, fmaf(r[e].y, r[e].y, nr));
        nb = fmaf(bv.x, bv.x, fmaf(bv.y, bv.y, nb));
        const int k = lane + 32 * e;
        if (!(isfinite(x[e].x) && isfinite(x[e].y))) nonfinite = 1;
        if (!vout(e) || !mine(e)) continue;
        P.x_hat[base + k] = x[e];
        if (want_sym) {
          int lab = 0;
          if (m) lab = (gray(axis_level<float>(x[e].x, m, sc)) << nb2) | gray(axis_level<float>(x[e].y, m, sc));
          if (P.sym) P.sym[base + k] = (uint8_t)lab;
          if (P.tx && m) errs += __popc((unsigned)(lab ^ txv[e]));
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nr += __shfl_xor_sync(0xffffffffu, nr, o);
      nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    nonfinite = __any_sync(0xffffffffu, nonfinite);
    if (P.bit_errors && P.tx) {
      errs = __reduce_add_sync(0xffffffffu, errs);
      if (lane == 0 && errs) atomicAdd(P.bit_errors, (unsigned long long)errs);
    }
    if (lane == 0 && sj == 0) {
      if (P.rel_res) P.rel_res[sys] = nb > 0.f ? sqrt((double)nr / (double)nb) : 0.0;
      if (nonfinite) st |= 4;
      if (want_sym && m == 0) st |= 16;
      if (P.status) P.status[sys] = P.status_or ? (P.status[sys] | st) : st;
    }
  }
};

}  // namespace
}  // namespace fpcg
