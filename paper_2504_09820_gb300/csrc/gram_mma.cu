// Gram matrix and matched filter on the tensor cores by mma.sync, for the Gram
// sizes the tcgen05 pipeline does not take (K = 128, or data the TMA path
// cannot address): A = fl(H)^H fl(H) + sigma^2 I, b = fl(H)^H fl(y) (Section II,
// eq. inversion) with fl = bf16 or fp16 (exact products, fp32 sums).
//
// One CTA per system (16 warps for K = 128, else 8); K = 8 runs as K = 16 with
// zero rows.  The antennas are consumed in chunks of 64:
// every thread rounds eight complex entries of H per row to the 16-bit format
// and stores the real and imaginary parts as rows of Xre, Xim (K x 64,
// 16-byte chunks swizzled by row), y likewise.  The warps own 16 x 8 tiles of
// A on or above the diagonal (tile (m, n): users 16m.., 8n..) and accumulate
//   Re A += Xre Xre^T + Xim Xim^T,   Im A += Xre Xim^T - Xim Xre^T
// with ldmatrix fragments (the minus is a sign flip of the 16-bit B values,
// exact); one more tile per m accumulates b from y.  The upper triangle is
// written with its Hermitian mirror, sigma^2 on the diagonal.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gram_mma.cuh"
#include "tc.cuh"

namespace fpcg {
namespace {

constexpr int kChunk = 64;  // antennas per stage

// 16 warps for K = 128 (72 tiles), 8 otherwise.
__host__ __device__ constexpr int gram_warps(int K) { return K >= 128 ? 16 : 8; }

__host__ __device__ constexpr int n_tiles(int K) {  // tiles (m, n) with n >= 2m
  return (K / 16) * (K / 8) - (K / 16) * (K / 16 - 1);
}

template <int K>
__device__ __forceinline__ uint32_t x_off(int row, int chunk) {  // bytes, 128-byte rows
  return (uint32_t)(row * 128 + ((chunk ^ (row & 7)) << 4));
}

template <bool BF>
__device__ __forceinline__ uint32_t pack16(float a, float b) {
  if (BF) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  }
  __half2 v = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

template <bool BF>
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if (BF) tc::mma_m16n8k16_bf16(d, a, b0, b1);
  else tc::mma_m16n8k16_f16(d, a, b0, b1);
}

__device__ __forceinline__ void ldmatrix_x2(uint32_t& r0, uint32_t& r1, uint32_t saddr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(saddr) : "memory");
}

// KR <= K users: rows KR..K-1 of the tiles are zero and not written out
// (A and b of the KR-user system, row stride KR).
//
// Software pipeline: every thread holds its share of the next chunk of H (and
// of y) in registers while the warps multiply the current chunk, so the DRAM
// latency of chunk c+1 hides under the products of chunk c.
template <int K, int KR, bool BF>
__global__ void __launch_bounds__(gram_warps(K) * 32, K >= 128 ? 1 : 2) gram_mma_kernel(const GramMmaParams P) {
  constexpr int NW = gram_warps(K);
  constexpr int NTH = NW * 32;
  constexpr int NT = n_tiles(K);
  constexpr int TPW = (NT + NW - 1) / NW;    // A tiles per warp
  constexpr int MB = K / 16;                 // b tiles (on the last MB warps)
  constexpr int ITEMS = K * (kChunk / 8);    // 8-antenna pieces of H rows per chunk
  constexpr int IPT = (ITEMS + NTH - 1) / NTH;
  __shared__ __align__(128) uint8_t Xre[K * 128];
  __shared__ __align__(128) uint8_t Xim[K * 128];
  __shared__ __align__(16) uint32_t ys[2][kChunk / 2];  // 16-bit pairs of Re y, Im y
  const int64_t sys = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int N = P.N;
  const float2* Hs = P.H + (size_t)sys * KR * N;
  const float2* yv = P.y + (size_t)sys * N;

  // this warp's tiles: list index w + NW i of the (m, n >= 2m) tiles in (m, n) order
  int tm[TPW], tn[TPW];
#pragma unroll
  for (int i = 0; i < TPW; ++i) {
    int idx = warp + NW * i, m = 0;
    while (m < K / 16 && idx >= K / 8 - 2 * m) {
      idx -= K / 8 - 2 * m;
      ++m;
    }
    tm[i] = m;  // m == K/16: no tile
    tn[i] = 2 * m + idx;
  }
  const int bm = NW - 1 - warp;  // b tile of this warp (if < MB)
  float are[TPW][4], aim[TPW][4], bb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < TPW; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) are[i][q] = aim[i][q] = 0.f;
  const uint32_t bre = tc::smem_u32(Xre), bim = tc::smem_u32(Xim);
  const int lr = lane & 15, lc = lane >> 4;  // ldmatrix.x4 row / chunk half
  const int lb = lane & 7, lh = (lane >> 3) & 1;  // ldmatrix.x2

  // 16-byte loads where every row starts 16-byte aligned
  const bool vec = (reinterpret_cast<uintptr_t>(P.H) & 15) == 0 && (N & 1) == 0;
  float2 hp[IPT][8], yp[2];
  auto load = [&](int n0) {
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      const int it = threadIdx.x + NTH * u;
      const int k = it / (kChunk / 8), q = it % (kChunk / 8);
      if (vec && it < ITEMS && k < KR && n0 + 8 * q + 8 <= N) {  // four 16-byte loads
        const float4* src = reinterpret_cast<const float4*>(Hs + (size_t)k * N + n0 + 8 * q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 v = src[j];
          hp[u][2 * j] = make_float2(v.x, v.y);
          hp[u][2 * j + 1] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n0 + 8 * q + j;
          hp[u][j] = (it < ITEMS && k < KR && n < N) ? Hs[(size_t)k * N + n] : make_float2(0.f, 0.f);
        }
      }
    }
    if (threadIdx.x < kChunk / 2) {
      const int n = n0 + 2 * threadIdx.x;
      yp[0] = n < N ? yv[n] : make_float2(0.f, 0.f);
      yp[1] = n + 1 < N ? yv[n + 1] : make_float2(0.f, 0.f);
    }
  };
  load(0);

  for (int n0 = 0; n0 < N; n0 += kChunk) {
    __syncthreads();  // the previous chunk is consumed
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      const int it = threadIdx.x + NTH * u;
      if (it < ITEMS) {
        const int k = it / (kChunk / 8), q = it % (kChunk / 8);
        const float2* h = hp[u];
        *reinterpret_cast<uint4*>(Xre + x_off<K>(k, q)) =
            make_uint4(pack16<BF>(h[0].x, h[1].x), pack16<BF>(h[2].x, h[3].x), pack16<BF>(h[4].x, h[5].x),
                       pack16<BF>(h[6].x, h[7].x));
        *reinterpret_cast<uint4*>(Xim + x_off<K>(k, q)) =
            make_uint4(pack16<BF>(h[0].y, h[1].y), pack16<BF>(h[2].y, h[3].y), pack16<BF>(h[4].y, h[5].y),
                       pack16<BF>(h[6].y, h[7].y));
      }
    }
    if (threadIdx.x < kChunk / 2) {
      ys[0][threadIdx.x] = pack16<BF>(yp[0].x, yp[1].x);
      ys[1][threadIdx.x] = pack16<BF>(yp[0].y, yp[1].y);
    }
    __syncthreads();
    if (n0 + kChunk < N) load(n0 + kChunk);  // in flight during the products below
#pragma unroll
    for (int ks = 0; ks < kChunk / 16; ++ks) {
#pragma unroll
      for (int i = 0; i < TPW; ++i) {
        if (tm[i] >= K / 16) continue;
        uint32_t ar[4], ai[4], r0, r1, i0, i1;
        tc::ldmatrix_x4(ar, bre + x_off<K>(16 * tm[i] + lr, 2 * ks + lc));
        tc::ldmatrix_x4(ai, bim + x_off<K>(16 * tm[i] + lr, 2 * ks + lc));
        ldmatrix_x2(r0, r1, bre + x_off<K>(8 * tn[i] + lb, 2 * ks + lh));
        ldmatrix_x2(i0, i1, bim + x_off<K>(8 * tn[i] + lb, 2 * ks + lh));
        mma<BF>(are[i], ar, r0, r1);
        mma<BF>(are[i], ai, i0, i1);
        mma<BF>(aim[i], ar, i0, i1);
        mma<BF>(aim[i], ai, r0 ^ 0x80008000u, r1 ^ 0x80008000u);
      }
      if (bm < MB) {  // b tile bm: columns (Re y, Im y) against Xre, (Im y, -Re y) against Xim
        uint32_t ar[4], ai[4];
        tc::ldmatrix_x4(ar, bre + x_off<K>(16 * bm + lr, 2 * ks + lc));
        tc::ldmatrix_x4(ai, bim + x_off<K>(16 * bm + lr, 2 * ks + lc));
        const int w0 = 8 * ks + t, w1 = 8 * ks + 4 + t;  // 16-bit pair index of antennas 16ks+2t, +8
        const uint32_t yr0 = ys[0][w0], yr1 = ys[0][w1], yi0 = ys[1][w0], yi1 = ys[1][w1];
        const uint32_t b0 = g == 0 ? yr0 : g == 1 ? yi0 : 0u, b1 = g == 0 ? yr1 : g == 1 ? yi1 : 0u;
        const uint32_t c0 = g == 0 ? yi0 : g == 1 ? (yr0 ^ 0x80008000u) : 0u;
        const uint32_t c1 = g == 0 ? yi1 : g == 1 ? (yr1 ^ 0x80008000u) : 0u;
        mma<BF>(bb, ar, b0, b1);
        mma<BF>(bb, ai, c0, c1);
      }
    }
  }

  // outputs: upper triangle and its mirror; sigma^2 on the diagonal
  const float s2 = (float)P.sigma2[sys];
  float2* Ao = P.A + (size_t)sys * KR * KR;
#pragma unroll
  for (int i = 0; i < TPW; ++i) {
    if (tm[i] >= K / 16) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 16 * tm[i] + g + 8 * (q >> 1), l = 8 * tn[i] + 2 * t + (q & 1);
      if (k > l || l >= KR) continue;
      if (k == l) {
        Ao[(size_t)k * KR + l] = make_float2(are[i][q] + s2, 0.f);
      } else {
        Ao[(size_t)k * KR + l] = make_float2(are[i][q], aim[i][q]);
        Ao[(size_t)l * KR + k] = make_float2(are[i][q], -aim[i][q]);
      }
    }
  }
  if (bm < MB && t == 0) {
    float2* bo = P.b + (size_t)sys * KR + 16 * bm;
    if (16 * bm + g < KR) bo[g] = make_float2(bb[0], bb[1]);
    if (16 * bm + g + 8 < KR) bo[g + 8] = make_float2(bb[2], bb[3]);
  }
}

template <int KR, bool BF>
cudaError_t launch_k(const GramMmaParams& P, cudaStream_t s) {
  if (P.batch <= 0) return cudaSuccess;
  constexpr int K = KR < 16 ? 16 : KR;
  gram_mma_kernel<K, KR, BF><<<(unsigned)P.batch, gram_warps(K) * 32, 0, s>>>(P);
  return cudaGetLastError();
}

}  // namespace

bool gram_mma_supported(int K) { return K == 8 || K == 16 || K == 32 || K == 64 || K == 128; }

cudaError_t launch_gram_mma(const GramMmaParams& P, int bf16, cudaStream_t s) {
  switch (P.K * 2 + (bf16 ? 1 : 0)) {
    case 16: return launch_k<8, false>(P, s);
    case 17: return launch_k<8, true>(P, s);
    case 32: return launch_k<16, false>(P, s);
    case 33: return launch_k<16, true>(P, s);
    case 64: return launch_k<32, false>(P, s);
    case 65: return launch_k<32, true>(P, s);
    case 128: return launch_k<64, false>(P, s);
    case 129: return launch_k<64, true>(P, s);
    case 256: return launch_k<128, false>(P, s);
    case 257: return launch_k<128, true>(P, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpcg
