// Matched filters of many received vectors per channel on the tensor cores:
// b_s = fl(H_g)^H fl(y_s) (Section II, eq. inversion) for all vectors s of a
// group g at once, a (2K x N) x (N x 2 n_g) product per group.
//
// One CTA (16 warps) per group; K = 8 runs as K = 16 with zero rows.  The
// group's vectors are taken 64 at a time; for each batch the antennas are
// consumed in chunks of 64: H rows as Re h_k and Im h_k (16-bit, like the
// Gram), and the batch's y as rows (Re y_0, Im y_0, Re y_1, Im y_1, ...).  The
// warps own 16 x 8 output tiles (16 users x 4 vectors; a warp's tiles share
// one m-tile, so its A fragments are loaded once per k-step) and accumulate
//   [Re b_s, Im b_s] += Re H^T [Re y_s, Im y_s] + Im H^T [Im y_s, -Re y_s],
// the second B fragment made from the first by swapping column pairs (a lane
// exchange) and negating one of them.  Every thread holds its share of the
// next (batch, chunk) step in registers while the current one is multiplied.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mf_mma.cuh"
#include "tc.cuh"

namespace fpcg {
namespace {

constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
constexpr int kChunk = 64;  // antennas per stage
constexpr int kBatch = 64;  // received vectors per pass

__device__ __forceinline__ uint32_t x_off(int row, int chunk) {  // 128-byte rows, swizzled chunks
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

template <bool BF>
__device__ __forceinline__ uint4 pack8(const float2 (&v)[8], bool im) {
  return im ? make_uint4(pack16<BF>(v[0].y, v[1].y), pack16<BF>(v[2].y, v[3].y), pack16<BF>(v[4].y, v[5].y),
                         pack16<BF>(v[6].y, v[7].y))
            : make_uint4(pack16<BF>(v[0].x, v[1].x), pack16<BF>(v[2].x, v[3].x), pack16<BF>(v[4].x, v[5].x),
                         pack16<BF>(v[6].x, v[7].x));
}

// KR <= K users: rows KR..K-1 of the tile are zero and not written out.
template <int K, int KR, bool BF>
__global__ void __launch_bounds__(kThreads, 1) mf_mma_kernel(const MfMmaParams P) {
  constexpr int MTL = K / 16;                  // m-tiles (16 users)
  constexpr int NTL = 2 * kBatch / 8;          // n-tiles (4 vectors, re and im)
  constexpr int TPW = MTL * NTL / kWarps;      // tiles per warp: n-tiles nt0.. of one m-tile
  constexpr int HI = K * (kChunk / 8);         // 8-antenna pieces of H rows per chunk
  constexpr int HPT = (HI + kThreads - 1) / kThreads;
  static_assert(MTL * NTL % kWarps == 0, "tiles must split evenly over the warps");
  static_assert(kBatch * (kChunk / 8) == kThreads, "one piece of y per thread");
  __shared__ __align__(128) uint8_t Xre[K * 128];
  __shared__ __align__(128) uint8_t Xim[K * 128];
  __shared__ __align__(128) uint8_t Y[2 * kBatch * 128];  // rows Re y_s, Im y_s
  const int64_t g = blockIdx.x;
  const int64_t s_begin = P.group_start[g], s_end = P.group_start[g + 1];
  if (s_end <= s_begin) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, t = lane & 3;
  const int N = P.N;
  const int nchunks = (N + kChunk - 1) / kChunk;
  const int64_t nsteps = (s_end - s_begin + kBatch - 1) / kBatch * nchunks;
  const float2* Hg = P.H + (size_t)g * KR * N;
  const uint32_t bre = tc::smem_u32(Xre), bim = tc::smem_u32(Xim), by = tc::smem_u32(Y);
  const int lr = lane & 15, lc = lane >> 4, lb = lane & 7, lh = (lane >> 3) & 1;
  const uint32_t neg = (gq & 1) ? 0x80008000u : 0u;  // column 2v+1 of (Im y, -Re y) is -Re y
  const int mt = warp / (NTL / TPW), nt0 = warp % (NTL / TPW) * TPW;

  // 16-byte loads where every row starts 16-byte aligned
  const bool vec = ((reinterpret_cast<uintptr_t>(P.H) | reinterpret_cast<uintptr_t>(P.y)) & 15) == 0 && (N & 1) == 0;
  float2 hp[HPT][8], yp[8];
  auto load = [&](int64_t step) {  // H and y of step (batch, chunk) into registers
    const int64_t s0 = s_begin + step / nchunks * kBatch;
    const int n0 = (int)(step % nchunks) * kChunk;
#pragma unroll
    for (int u = 0; u < HPT; ++u) {
      const int it = threadIdx.x + kThreads * u;
      const int k = it / (kChunk / 8), q = it % (kChunk / 8);
      if (vec && it < HI && k < KR && n0 + 8 * q + 8 <= N) {  // four 16-byte loads
        const float4* src = reinterpret_cast<const float4*>(Hg + (size_t)k * N + n0 + 8 * q);
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
          hp[u][j] = (it < HI && k < KR && n < N) ? Hg[(size_t)k * N + n] : make_float2(0.f, 0.f);
        }
      }
    }
    const int v = threadIdx.x / (kChunk / 8), q = threadIdx.x % (kChunk / 8);
    if (vec && s0 + v < s_end && n0 + 8 * q + 8 <= N) {
      const float4* src = reinterpret_cast<const float4*>(P.y + (size_t)(s0 + v) * N + n0 + 8 * q);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 w = src[j];
        yp[2 * j] = make_float2(w.x, w.y);
        yp[2 * j + 1] = make_float2(w.z, w.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = n0 + 8 * q + j;
        yp[j] = (s0 + v < s_end && n < N) ? P.y[(size_t)(s0 + v) * N + n] : make_float2(0.f, 0.f);
      }
    }
  };

  float acc[TPW][4];
#pragma unroll
  for (int i = 0; i < TPW; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
  load(0);
  for (int64_t step = 0; step < nsteps; ++step) {
    __syncthreads();  // the previous step is consumed
#pragma unroll
    for (int u = 0; u < HPT; ++u) {
      const int it = threadIdx.x + kThreads * u;
      if (it < HI) {
        const int k = it / (kChunk / 8), q = it % (kChunk / 8);
        *reinterpret_cast<uint4*>(Xre + x_off(k, q)) = pack8<BF>(hp[u], false);
        *reinterpret_cast<uint4*>(Xim + x_off(k, q)) = pack8<BF>(hp[u], true);
      }
    }
    {
      const int v = threadIdx.x / (kChunk / 8), q = threadIdx.x % (kChunk / 8);
      *reinterpret_cast<uint4*>(Y + x_off(2 * v, q)) = pack8<BF>(yp, false);
      *reinterpret_cast<uint4*>(Y + x_off(2 * v + 1, q)) = pack8<BF>(yp, true);
    }
    __syncthreads();
    if (step + 1 < nsteps) load(step + 1);  // in flight during the products below
#pragma unroll 1  // one k-step at a time: the next step's H and y occupy the registers
    for (int ks = 0; ks < kChunk / 16; ++ks) {
      uint32_t ar[4], ai[4];
      tc::ldmatrix_x4(ar, bre + x_off(16 * mt + lr, 2 * ks + lc));
      tc::ldmatrix_x4(ai, bim + x_off(16 * mt + lr, 2 * ks + lc));
#pragma unroll
      for (int i = 0; i < TPW; ++i) {
        uint32_t b0, b1;
        ldmatrix_x2(b0, b1, by + x_off(8 * (nt0 + i) + lb, 2 * ks + lh));
        // (Im y, -Re y): lane exchange of the column pairs (lanes 4 apart), sign of the odd column
        const uint32_t c0 = __shfl_xor_sync(0xffffffffu, b0, 4) ^ neg;
        const uint32_t c1 = __shfl_xor_sync(0xffffffffu, b1, 4) ^ neg;
        mma<BF>(acc[i], ar, b0, b1);
        mma<BF>(acc[i], ai, c0, c1);
      }
    }
    if (step % nchunks == nchunks - 1) {  // the batch is complete
      // tile (mt, nt): rows users 16mt + gq (+8), columns 2t, 2t+1 = (Re, Im) of vector 4nt + t
      const int64_t s0 = s_begin + step / nchunks * kBatch;
#pragma unroll
      for (int i = 0; i < TPW; ++i) {
        const int64_t s = s0 + 4 * (nt0 + i) + t;
        const int k = 16 * mt + gq;
        if (s < s_end) {
          float2* bo = P.b + (size_t)s * KR + k;
          if (k < KR) bo[0] = make_float2(acc[i][0], acc[i][1]);
          if (k + 8 < KR) bo[8] = make_float2(acc[i][2], acc[i][3]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
      }
    }
  }
}

template <int KR, bool BF>
cudaError_t launch_k(const MfMmaParams& P, cudaStream_t s) {
  if (P.n_groups <= 0) return cudaSuccess;
  mf_mma_kernel<(KR < 16 ? 16 : KR), KR, BF><<<(unsigned)P.n_groups, kThreads, 0, s>>>(P);
  return cudaGetLastError();
}

}  // namespace

bool mf_mma_supported(int K) { return K == 8 || K == 16 || K == 32 || K == 64 || K == 128; }

cudaError_t launch_mf_mma(const MfMmaParams& P, int bf16, cudaStream_t s) {
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
