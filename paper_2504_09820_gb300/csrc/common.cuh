// Device helpers shared by the detector kernels: rounding to the formats of
// Table I (plus e4m3), the e4m3 per-block scale, error-free transformations
// for the compensated residual, the Gray-QAM slicer, and small reductions.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace fpcg {

// Format codes, identical to the FPCG_* enum of the public header.
enum Fmt : int { F64 = 0, F32 = 1, F16 = 2, BF16 = 3, E4M3 = 4 };

template <typename T>
struct cplx {
  T re, im;
};

// Round-to-nearest-even of an fp32 value to `fmt`, returned as the fp32 value
// of the result (exact).  E4M3 saturates to +-448 (the "satfinite" mode).
__device__ __forceinline__ float round_to(float x, int fmt) {
  switch (fmt) {
    case BF16:
      return __bfloat162float(__float2bfloat16_rn(x));
    case F16:
      return __half2float(__float2half_rn(x));
    case E4M3: {
      __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
      return __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3)));
    }
    default:
      return x;
  }
}

// Smallest power of two s with amax <= 448 s (s = 1 for amax == 0): the
// scale of one e4m3 block, so that amax / s lands in (224, 448] exactly.
__device__ __forceinline__ float e4m3_scale(float amax) {
  if (!(amax > 0.f)) return 1.f;
  int e;
  float m = frexpf(amax, &e);  // amax = m * 2^e, 0.5 <= m < 1
  int k = (m <= 0.875f) ? e - 9 : e - 8;
  return ldexpf(1.f, k);
}

// e4m3_scale(amax) and its reciprocal from the bits of amax (both exact powers
// of two); amax outside [2^-118, 2^127) takes e4m3_scale itself.  amax = 1.f *
// 2^E = m 2^(E+1) with m = 1.f / 2, and m <= 0.875 is 1.f <= 1.75, i.e. a
// fraction field of at most 0x600000.
__device__ __forceinline__ float e4m3_scale_inv(float amax, float& inv) {
  const uint32_t b = __float_as_uint(amax);
  if (b - 0x04800000u < 0x7f000000u - 0x04800000u) {
    const int E = (int)(b >> 23) - 127;
    const int k = (b & 0x7fffffu) <= 0x600000u ? E - 8 : E - 7;
    inv = __uint_as_float((uint32_t)(127 - k) << 23);
    return __uint_as_float((uint32_t)(127 + k) << 23);
  }
  const float s = e4m3_scale(amax);
  inv = 1.f / s;
  return s;
}

// ---- error-free transformations (Knuth TwoSum, FMA-based TwoProd) ---------
// The _rn intrinsics are never contracted into FMAs, which these rely on.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// (hi, lo) += -a*b, keeping the rounding errors of the product and the sum.
__device__ __forceinline__ void df_sub_prod(float& hi, float& lo, float a, float b) {
  float p = __fmul_rn(a, b);
  float pe = __fmaf_rn(a, b, -p);  // a*b = p + pe exactly
  float s, e;
  two_sum(hi, -p, s, e);
  hi = s;
  lo = __fadd_rn(lo, __fsub_rn(e, pe));
}

// (h1, l1) += (h2, l2)
__device__ __forceinline__ void df_add(float& h1, float& l1, float h2, float l2) {
  float s, e;
  two_sum(h1, h2, s, e);
  h1 = s;
  l1 = __fadd_rn(__fadd_rn(l1, l2), e);
}

// ---- Gray-mapped square QAM slicer ----------------------------------------
// t = fl(v * s) with s = fl(sqrt(2(M-1)/3)); the level index is the number of
// integer thresholds 2k - m + 2 (k = 0..m-2) that t reaches, so ties go up
// and values beyond the outer levels clamp.
template <typename T>
__device__ __forceinline__ int axis_level(T v, int m, T s) {
  T t = v * s;
  int j = 0;
  for (int k = 0; k < m - 1; ++k) j += (t >= (T)(2 * k - m + 2)) ? 1 : 0;
  return j;
}

__device__ __forceinline__ int qam_sqrt(int M) {
  return M == 4 ? 2 : M == 16 ? 4 : M == 64 ? 8 : M == 256 ? 16 : 0;
}

__device__ __forceinline__ int qam_bits_axis(int m) {
  return m == 2 ? 1 : m == 4 ? 2 : m == 8 ? 3 : 4;
}

__device__ __forceinline__ int gray(int j) { return j ^ (j >> 1); }

// ---- reductions -----------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace fpcg
