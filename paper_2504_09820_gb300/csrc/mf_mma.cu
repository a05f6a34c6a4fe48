// Matched filters of many received vectors per channel on the tensor cores:
// b_s = fl(H_g)^H fl(y_s) (Section II, eq. inversion) for all vectors s of a
// group g at once, a (2K x N) x (N x 2 n_g) product per group.
//
// One CTA (8 warps) per group; K = 8 runs as K = 16 with zero rows.  The group's vectors are taken 32 at a time;
// for each batch the antennas are consumed in chunks of 64: H rows as Re h_k
// and Im h_k (16-bit, like the Gram), and the batch's y as rows
// (Re y_0, Im y_0, Re y_1, Im y_1, ...) and (Im y_0, -Re y_0, ...).  The warps
// own 16 x 8 output tiles (16 users x 4 vectors) and accumulate
//   [Re b_s, Im b_s] += Re H^T [Re y_s, Im y_s] + Im H^T [Im y_s, -Re y_s].
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mf_mma.cuh"
#include "tc.cuh"

namespace fpcg {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kChunk = 64;  // antennas per stage
constexpr int kBatch = 32;  // received vectors per pass

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

// KR <= K users: rows KR..K-1 of the tile are zero and not written out.
template <int K, int KR, bool BF>
__global__ void __launch_bounds__(kThreads) mf_mma_kernel(const MfMmaParams P) {
  constexpr int MTL = K / 16;                  // m-tiles (16 users)
  constexpr int NTL = 2 * kBatch / 8;          // n-tiles (4 vectors, re and im)
  constexpr int TPW = MTL * NTL / kWarps;      // tiles per warp
  static_assert(MTL * NTL % kWarps == 0, "tiles must split evenly over the warps");
  __shared__ __align__(128) uint8_t Xre[K * 128];
  __shared__ __align__(128) uint8_t Xim[K * 128];
  __shared__ __align__(128) uint8_t Y1[2 * kBatch * 128];  // rows Re y_s, Im y_s
  __shared__ __align__(128) uint8_t Y2[2 * kBatch * 128];  // rows Im y_s, -Re y_s
  const int64_t g = blockIdx.x;
  const int64_t s_begin = P.group_start[g], s_end = P.group_start[g + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, t = lane & 3;
  const int N = P.N;
  const float2* Hg = P.H + (size_t)g * KR * N;
  const uint32_t bre = tc::smem_u32(Xre), bim = tc::smem_u32(Xim), by1 = tc::smem_u32(Y1), by2 = tc::smem_u32(Y2);
  const int lr = lane & 15, lc = lane >> 4, lb = lane & 7, lh = (lane >> 3) & 1;

  for (int64_t s0 = s_begin; s0 < s_end; s0 += kBatch) {
    const int nb = (int)min((int64_t)kBatch, s_end - s0);
    float acc[TPW][4];
#pragma unroll
    for (int i = 0; i < TPW; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
    for (int n0 = 0; n0 < N; n0 += kChunk) {
      __syncthreads();  // the previous chunk is consumed
      for (int it = threadIdx.x; it < K * (kChunk / 8); it += kThreads) {
        const int k = it / (kChunk / 8), q = it % (kChunk / 8);
        float re[8], im[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n0 + 8 * q + j;
          const float2 h = (n < N && k < KR) ? Hg[(size_t)k * N + n] : make_float2(0.f, 0.f);
          re[j] = h.x;
          im[j] = h.y;
        }
        *reinterpret_cast<uint4*>(Xre + x_off(k, q)) =
            make_uint4(pack16<BF>(re[0], re[1]), pack16<BF>(re[2], re[3]), pack16<BF>(re[4], re[5]), pack16<BF>(re[6], re[7]));
        *reinterpret_cast<uint4*>(Xim + x_off(k, q)) =
            make_uint4(pack16<BF>(im[0], im[1]), pack16<BF>(im[2], im[3]), pack16<BF>(im[4], im[5]), pack16<BF>(im[6], im[7]));
      }
      for (int it = threadIdx.x; it < kBatch * (kChunk / 8); it += kThreads) {
        const int v = it / (kChunk / 8), q = it % (kChunk / 8);
        float re[8], im[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n0 + 8 * q + j;
          const float2 yy = (v < nb && n < N) ? P.y[(size_t)(s0 + v) * N + n] : make_float2(0.f, 0.f);
          re[j] = yy.x;
          im[j] = yy.y;
        }
        const uint4 pr = make_uint4(pack16<BF>(re[0], re[1]), pack16<BF>(re[2], re[3]), pack16<BF>(re[4], re[5]),
                                    pack16<BF>(re[6], re[7]));
        const uint4 pi = make_uint4(pack16<BF>(im[0], im[1]), pack16<BF>(im[2], im[3]), pack16<BF>(im[4], im[5]),
                                    pack16<BF>(im[6], im[7]));
        const uint4 nr = make_uint4(pr.x ^ 0x80008000u, pr.y ^ 0x80008000u, pr.z ^ 0x80008000u, pr.w ^ 0x80008000u);
        *reinterpret_cast<uint4*>(Y1 + x_off(2 * v, q)) = pr;
        *reinterpret_cast<uint4*>(Y1 + x_off(2 * v + 1, q)) = pi;
        *reinterpret_cast<uint4*>(Y2 + x_off(2 * v, q)) = pi;
        *reinterpret_cast<uint4*>(Y2 + x_off(2 * v + 1, q)) = nr;
      }
      __syncthreads();
#pragma unroll
      for (int ks = 0; ks < kChunk / 16; ++ks) {
#pragma unroll
        for (int i = 0; i < TPW; ++i) {
          const int tile = warp * TPW + i, mt = tile / NTL, nt = tile % NTL;
          uint32_t ar[4], ai[4], b10, b11, b20, b21;
          tc::ldmatrix_x4(ar, bre + x_off(16 * mt + lr, 2 * ks + lc));
          tc::ldmatrix_x4(ai, bim + x_off(16 * mt + lr, 2 * ks + lc));
          ldmatrix_x2(b10, b11, by1 + x_off(8 * nt + lb, 2 * ks + lh));
          ldmatrix_x2(b20, b21, by2 + x_off(8 * nt + lb, 2 * ks + lh));
          mma<BF>(acc[i], ar, b10, b11);
          mma<BF>(acc[i], ai, b20, b21);
        }
      }
    }
    // tile (mt, nt): rows users 16mt + gq (+8), columns 2t, 2t+1 = (Re, Im) of vector 4nt + t
#pragma unroll
    for (int i = 0; i < TPW; ++i) {
      const int tile = warp * TPW + i, mt = tile / NTL, nt = tile % NTL;
      const int v = 4 * nt + t;
      if (v < nb) {
        const int k = 16 * mt + gq;
        float2* bo = P.b + (size_t)(s0 + v) * KR + k;
        if (k < KR) bo[0] = make_float2(acc[i][0], acc[i][1]);
        if (k + 8 < KR) bo[8] = make_float2(acc[i][2], acc[i][3]);
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
