#pragma once
// The residual b - A x against a given fp32 Gram matrix in global memory for
// the CG warp (CgWarp RM = 2): the solvers for given Gram matrices keep only
// the matvec copy of A in shared memory, so a residual trip reads A again
// (from L2: the slot's fill has just read it).  Included by the solvers only.
#include <cuda_runtime.h>

#include "cg_warp.cuh"

namespace fpcg {
namespace {

// RM = 2: W = b - A x from the fp32 Gram matrix in global memory, then
// w = W (x arrives in w).  Lane j holds x_j (j = lane + 32e), so the loads of
// one row are coalesced.  RB rows at a time: every lane sums its columns'
// products, then log2(RB) exchange steps (lane distance 16, 8, ...) each
// keep half of the rows and hand the other half to the partner lane, so
// that row i0 + r, r = the top log2(RB) bits of the lane, ends up summed
// over RB lanes, and plain shuffles add the remaining 32 / RB.  RB = 4 for
// K = 128 (fewer loads in flight, fewer registers).  NS > 1: the row blocks
// are split over the warps of the system.  Padding rows (KR..K-1) are zero.
template <int K, bool BF, int LT, int KR, int NV, int NS, int RM, int F8>
__device__ __forceinline__ void CgWarp<K, BF, LT, KR, NV, NS, RM, F8>::apply_gram(float2 (&w)[E]) {
  constexpr int RB = E >= 4 ? 4 : 8;   // rows per block
  constexpr int LB = RB == 8 ? 3 : 2;  // exchange steps
  constexpr int GU = E <= 2 ? 2 : 1;   // row blocks whose loads are in flight together
  gsync();  // NS > 1: every warp has read the previous trip's W
  const int r = lane >> (5 - LB);
#pragma unroll GU
  for (int i0 = RB * sj; i0 < KR; i0 += RB * NS) {
    float re[RB], im[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) re[u] = im[u] = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = lane + 32 * e;
      if (j < KR) {
        const float2 xv = w[e];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          const float2 a = __ldg(agram + (size_t)(i0 + u) * KR + j);
          re[u] = fmaf(a.x, xv.x, fmaf(-a.y, xv.y, re[u]));
          im[u] = fmaf(a.x, xv.y, fmaf(a.y, xv.x, im[u]));
        }
      }
    }
#pragma unroll
    for (int h = RB / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {  // keep h of 2h rows, send the others
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int u = 0; u < h; ++u) {
        const float sr = up ? re[u] : re[u + h], si = up ? im[u] : im[u + h];
        const float kr = up ? re[u + h] : re[u], ki = up ? im[u + h] : im[u];
        re[u] = kr + __shfl_xor_sync(0xffffffffu, sr, o);
        im[u] = ki + __shfl_xor_sync(0xffffffffu, si, o);
      }
    }
#pragma unroll
    for (int o = 16 >> LB; o > 0; o >>= 1) {
      re[0] += __shfl_xor_sync(0xffffffffu, re[0], o);
      im[0] += __shfl_xor_sync(0xffffffffu, im[0], o);
    }
    if ((lane & ((32 >> LB) - 1)) == 0) {
      const float2 bv = S.b[i0 + r];
      S.W[i0 + r] = make_float2(bv.x - re[0], bv.y - im[0]);
    }
  }
  __syncwarp();
  gsync();  // NS > 1: every row block of W is written
#pragma unroll
  for (int e = 0; e < E; ++e) w[e] = vout(e) ? S.W[lane + 32 * e] : make_float2(0.f, 0.f);
  __syncwarp();
}

// NV = 8, RM = 2: the eight vectors' residuals in one CTA-wide pass over the
// group's fp32 A, read once per trip instead of once per vector.  Every warp
// stages its x in the shared B-fragment area (a residual trip packs nothing
// there), then warp vw takes row blocks vw, vw + 8, ... of RP rows for all
// eight vectors: 8 RP sums per lane (row u of the block, vector v), log2(8 RP)
// exchange steps (lane distance 16, 8, ...) leave sum u * 8 + v = the top
// log2(8 RP) bits of the lane, summed over 8 RP lanes, and plain shuffles add
// the remaining 4 / RP.  RP = 1 at K = 128 (fewer registers).  Each warp
// then reads its own W.
template <int K, bool BF, int LT, int KR, int NV, int NS, int RM, int F8>
__device__ __forceinline__ void CgWarp<K, BF, LT, KR, NV, NS, RM, F8>::apply_gram_cta(float2 (&w)[E]) {
  constexpr int RP = E >= 4 ? 1 : 2;        // rows per block
  constexpr int NQ = 8 * RP;                // sums per lane
  constexpr int LB = RP == 2 ? 4 : 3;       // exchange steps
  float2* xs = reinterpret_cast<float2*>(S.Pk);  // [8][K]
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (vact()) xs[vw * K + lane + 32 * e] = w[e];
  __syncthreads();
  const int q = lane >> (5 - LB), ru = q >> 3, rv = q & 7;
  // the next block's entries of A are loaded while this block is formed (the
  // blocks of a warp would otherwise wait for L2 one after the other)
  float2 an[RP][E];
  auto load_block = [&](int i) {
#pragma unroll
    for (int u = 0; u < RP; ++u)
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int j = lane + 32 * e;
        an[u][e] = j < KR ? __ldg(agram + (size_t)(i + u) * KR + j) : make_float2(0.f, 0.f);
      }
  };
  if (RP * vw < KR) load_block(RP * vw);
#pragma unroll 1
  for (int i0 = RP * vw; i0 < KR; i0 += 8 * RP) {
    float2 ab[RP][E];
#pragma unroll
    for (int u = 0; u < RP; ++u)
#pragma unroll
      for (int e = 0; e < E; ++e) ab[u][e] = an[u][e];
    if (i0 + 8 * RP < KR) load_block(i0 + 8 * RP);
    float re[NQ], im[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) re[u] = im[u] = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = lane + 32 * e;
      if (j < KR) {
        float2 a[RP];
#pragma unroll
        for (int u = 0; u < RP; ++u) a[u] = ab[u][e];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const float2 xv = xs[v * K + j];
#pragma unroll
          for (int u = 0; u < RP; ++u) {
            re[8 * u + v] = fmaf(a[u].x, xv.x, fmaf(-a[u].y, xv.y, re[8 * u + v]));
            im[8 * u + v] = fmaf(a[u].x, xv.y, fmaf(a[u].y, xv.x, im[8 * u + v]));
          }
        }
      }
    }
#pragma unroll
    for (int h = NQ / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {  // keep h of 2h sums, send the others
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int u = 0; u < h; ++u) {
        const float sr = up ? re[u] : re[u + h], si = up ? im[u] : im[u + h];
        const float kr = up ? re[u + h] : re[u], ki = up ? im[u + h] : im[u];
        re[u] = kr + __shfl_xor_sync(0xffffffffu, sr, o);
        im[u] = ki + __shfl_xor_sync(0xffffffffu, si, o);
      }
    }
#pragma unroll
    for (int o = 16 >> LB; o > 0; o >>= 1) {
      re[0] += __shfl_xor_sync(0xffffffffu, re[0], o);
      im[0] += __shfl_xor_sync(0xffffffffu, im[0], o);
    }
    if ((lane & ((32 >> LB) - 1)) == 0) {
      const float2 bv = reinterpret_cast<const float2*>(vbase + rv * vst)[i0 + ru];
      reinterpret_cast<float2*>(vbase + rv * vst + 8 * K)[i0 + ru] = make_float2(bv.x - re[0], bv.y - im[0]);
    }
  }
  __syncthreads();  // every vector's W is complete (and xs is read)
#pragma unroll
  for (int e = 0; e < E; ++e) w[e] = vout(e) ? S.W[lane + 32 * e] : make_float2(0.f, 0.f);
}

}  // namespace
}  // namespace fpcg
