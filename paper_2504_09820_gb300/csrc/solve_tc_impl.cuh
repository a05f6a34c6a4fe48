#pragma once
// Tensor-core solver for given Gram matrices (kernel templates; instantiated
// per K by solve_tc_k{8,16,32,64,128}.cu; K = 8 runs in 16-wide slots holding
// diag(A, I)).  The CG of the fused detector without its Gram pipeline:
// A + sigma^2 I comes from global memory (fpcg_gram's output, or the
// caller's), every warp of a persistent CTA is an independent CG worker with
// its own shared-memory slot (K = 128: four warps per system,
// solve_split_kernel), and systems that share a Gram matrix share the slot's
// 16-bit A and inverted diagonal blocks.
//
// A warp takes a contiguous range of systems.  When the group changes it
// rounds the group's fp32 A to the matvec format into the slot ([Re A; Im A],
// swizzled), copies the diagonal blocks and inverts them (eq. pre_BJ).  The
// right-hand side is either given or the system's matched filter
// b = fl(H_g)^H fl(y_s) (eq. inversion; lanes over antennas, four rows of b at
// a time, warp reductions).  Then CgWarp::detect: Algorithm 2 or 3,
// refinement, slicing, outputs.  With D.resid_gram the refinement residuals
// and rel_res use the group's fp32 A itself, read again from global memory
// (CgWarp RM = 2); else the matvec copy in the slot.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_warp.cuh"
#include "common.cuh"
#include "gram_resid.cuh"
#include "solve_tc.cuh"

namespace fpcg {
namespace {

// Round the group's A (KR x KR, row stride KR) into the slot: 16-bit
// [Re A; Im A] chunks of 8 columns and the fp32 diagonal blocks; rows and
// columns KR..K-1 are those of the identity.  Threads tid, tid + nt, ...;
// each thread issues the loads of UB chunks before it converts any, so UB
// global loads per thread are in flight instead of one round trip per chunk.
template <int K, int KR, bool BF, int LT, int UB = 4>
__device__ __forceinline__ void fill_A(const float2* Ag, const Slot& S, int tid, int nt) {
  constexpr int CPR = K / 8, ITEMS = K * CPR;
  for (int i0 = tid; i0 < ITEMS; i0 += UB * nt) {
    float4 v[UB][4];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int idx = i0 + u * nt, k = idx / CPR, c = idx % CPR;
      if (idx < ITEMS && (KR == K || (k < KR && 8 * c < KR))) {
        const float4* src = reinterpret_cast<const float4*>(Ag + (size_t)k * KR + 8 * c);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[u][q] = __ldg(src + q);
      } else {  // padding: the identity
#pragma unroll
        for (int q = 0; q < 4; ++q)
          v[u][q] = make_float4(k == 8 * c + 2 * q ? 1.f : 0.f, 0.f, k == 8 * c + 2 * q + 1 ? 1.f : 0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int idx = i0 + u * nt, k = idx / CPR, c = idx % CPR;
      if (idx >= ITEMS) break;
      float2 a[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[2 * q] = make_float2(v[u][q].x, v[u][q].y);
        a[2 * q + 1] = make_float2(v[u][q].z, v[u][q].w);
      }
      uint4 re, im;
      re.x = pk2<BF>(a[0].x, a[1].x);
      re.y = pk2<BF>(a[2].x, a[3].x);
      re.z = pk2<BF>(a[4].x, a[5].x);
      re.w = pk2<BF>(a[6].x, a[7].x);
      im.x = pk2<BF>(a[0].y, a[1].y);
      im.y = pk2<BF>(a[2].y, a[3].y);
      im.z = pk2<BF>(a[4].y, a[5].y);
      im.w = pk2<BF>(a[6].y, a[7].y);
      *reinterpret_cast<uint4*>(S.A16 + a16_offset<K>(k, c)) = re;
      *reinterpret_cast<uint4*>(S.A16 + a16_offset<K>(K + k, c)) = im;
      if constexpr (LT > 0) {
        constexpr int MLD = md_row_stride(LT), MBS = md_block_stride(LT);
        const int kb0 = (k / LT) * LT;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int l = 8 * c + m;
          if (l >= kb0 && l < kb0 + LT) S.Md[(k / LT) * MBS + (k % LT) * MLD + (l - kb0)] = a[m];
        }
      }
    }
  }
}

// Ask the bulk-copy engine to pull `bytes` (a multiple of 16, 16-byte aligned)
// into L2 ahead of the loads that will read them.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  for (uint32_t o = 0; o < bytes; o += 32768)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const char*>(p) + o),
                 "r"(bytes - o < 32768u ? bytes - o : 32768u)
                 : "memory");
}

// b of system s (KR entries, given) into the slot, zeros beyond KR.  Plain
// loads: b may share memory with x_hat, which this kernel writes.
template <int K, int KR>
__device__ __forceinline__ void load_b(const float2* bs, const Slot& S, int lane) {
  for (int i = lane; i < K / 2; i += 32)  // two complex entries per float4
    reinterpret_cast<float4*>(S.b)[i] =
        (KR == K || 2 * i < KR) ? reinterpret_cast<const float4*>(bs)[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  __syncwarp();
}

// b = fl(H)^H fl(y) for one system into S.b (rounding of the Gram step); H
// has KR rows, entries KR..K-1 of b are zero.
// Rows k0 = 4 first, 4 (first + step), ... (several warps may split them).
template <int K, int KR>
__device__ void matched_filter(const float2* Hg, const float2* ys, int N, int gram, const Slot& S, int lane,
                               int first = 0, int step = 1) {
  if (first == 0)
    for (int k = KR + lane; k < K; k += 32) S.b[k] = make_float2(0.f, 0.f);
  for (int k0 = 4 * first; k0 < KR; k0 += 4 * step) {
    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
    for (int n = lane; n < N; n += 32) {
      const float2 yy = ys[n];
      const float yr = round_to(yy.x, gram), yi = round_to(yy.y, gram);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 h = Hg[(size_t)(k0 + q) * N + n];
        const float hr = round_to(h.x, gram), hi = round_to(h.y, gram);
        re[q] = fmaf(hr, yr, fmaf(hi, yi, re[q]));  // conj(h_k) y
        im[q] = fmaf(hr, yi, fmaf(-hi, yr, im[q]));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        re[q] += __shfl_xor_sync(0xffffffffu, re[q], o);
        im[q] += __shfl_xor_sync(0xffffffffu, im[q], o);
      }
    if (lane < 4) {
      float r = re[0], i = im[0];
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if (lane == q) {
          r = re[q];
          i = im[q];
        }
      S.b[k0 + lane] = make_float2(r, i);
    }
  }
  __syncwarp();
}

template <int KR, bool BF, int LT>
__global__ void __launch_bounds__(solve_warps(KR) * 32, 1) solve_tc_kernel(const __grid_constant__ SolveTcParams P) {
  constexpr int K = pad_k(KR);
  constexpr int NW = solve_warps(KR);
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* base = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
  const Slot S = slot_carve(base + warp * tc_slot_bytes(K, LT), K, LT);
  CgWarp<K, BF, LT, KR, 1, 1, 2> W(P.D, S, lane);
  const int64_t tw = (int64_t)gridDim.x * NW, gw = (int64_t)blockIdx.x * NW + warp;
  const int64_t chunk = (P.n + tw - 1) / tw;
  const int64_t s0 = gw * chunk, s1 = min(P.n, s0 + chunk);
  if (s0 >= s1) return;
  // group of the first system: binary search in group_start
  int64_t g = s0, g_end = s0 + 1;
  if (P.group_start) {
    int64_t lo = 0, hi = P.n_groups;  // largest g with start[g] <= s0
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (P.group_start[mid] <= s0) lo = mid;
      else hi = mid;
    }
    g = lo;
    g_end = P.group_start[g + 1];
  }
  int64_t cur = -1;
  int st_bj = 0;
  for (int64_t s = s0; s < s1; ++s) {
    if (P.group_start) {
      while (s >= g_end && g + 1 < P.n_groups) {
        ++g;
        g_end = P.group_start[g + 1];
      }
    } else if (P.a_map) {
      const int32_t gi = P.a_map[s];
      if (gi < 0 || gi >= P.n_groups) {  // x_hat = 0, labels 0, status only
        W.bad_index(s);
        continue;
      }
      g = gi;
    } else {
      g = s;
    }
    if (g != cur) {
      fill_A<K, KR, BF, LT>(P.A + (size_t)g * KR * KR, S, lane, 32);
      __syncwarp();
      st_bj = W.bj_setup();
      W.agram = P.D.resid_gram ? P.A + (size_t)g * KR * KR : nullptr;
      cur = g;
    }
    if (P.b) load_b<K, KR>(P.b + (size_t)s * KR, S, lane);
    else matched_filter<K, KR>(P.H + (size_t)g * KR * P.N, P.y + (size_t)s * P.N, P.N, P.gram, S, lane);
    W.detect(s, true, st_bj);
    __syncwarp();
  }
}

// K = 128 independent systems: four warps per system (CgWarp NS = 4), two
// systems per CTA, so an SM works on eight warps where one warp per slot
// would give it two (the 80 KB slots allow two per SM).  A group of four
// warps takes a contiguous range of systems; every step that changes the
// slot is followed by the group's barrier.
template <int KR, bool BF, int LT>
__global__ void __launch_bounds__(kSplitWarps * kSplitGroups * 32, 1)
    solve_split_kernel(const __grid_constant__ SolveTcParams P) {
  constexpr int K = pad_k(KR);
  constexpr int GT = kSplitWarps * 32;  // threads per system
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp / kSplitWarps, sj = warp % kSplitWarps, gtid = sj * 32 + lane;
  uint8_t* base = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
  uint8_t* gbase = base + grp * split_group_bytes(K, LT);
  const Slot S = slot_carve(gbase, K, LT);
  CgWarp<K, BF, LT, KR, 1, kSplitWarps, 2> W(P.D, S, lane);
  W.sj = sj;
  W.bar_id = 1 + grp;
  W.rst = reinterpret_cast<float2*>(gbase + tc_slot_bytes(K, LT) + sj * sizeof(float2) * K);
  const int64_t tg = (int64_t)gridDim.x * kSplitGroups, gg = (int64_t)blockIdx.x * kSplitGroups + grp;
  const int64_t chunk = (P.n + tg - 1) / tg;
  const int64_t s0 = gg * chunk, s1 = min(P.n, s0 + chunk);
  if (s0 >= s1) return;  // the whole group (its barrier is its own)
  int64_t g = s0, g_end = s0 + 1;
  if (P.group_start) {
    int64_t lo = 0, hi = P.n_groups;  // largest g with start[g] <= s0
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (P.group_start[mid] <= s0) lo = mid;
      else hi = mid;
    }
    g = lo;
    g_end = P.group_start[g + 1];
  }
  int64_t cur = -1;
  int st_bj = 0;
  for (int64_t s = s0; s < s1; ++s) {
    if (P.group_start) {
      while (s >= g_end && g + 1 < P.n_groups) {
        ++g;
        g_end = P.group_start[g + 1];
      }
    } else if (P.a_map) {
      const int32_t gi = P.a_map[s];
      if (gi < 0 || gi >= P.n_groups) {
        W.bad_index(s);
        continue;
      }
      g = gi;
    } else {
      g = s;
    }
    W.gsync();  // the previous system is done with b (and A)
    if (g != cur) {
      fill_A<K, KR, BF, LT, 8>(P.A + (size_t)g * KR * KR, S, gtid, GT);
      W.gsync();
      if (gtid == 0 && s + 1 < s1) {  // the next system's A into L2 while this one is solved
        int64_t gn = s + 1;
        if (P.group_start) gn = s + 1 < g_end ? g : g + 1;
        else if (P.a_map) gn = P.a_map[s + 1];
        if (gn != g && gn >= 0 && gn < P.n_groups)
          prefetch_l2(P.A + (size_t)gn * KR * KR, (uint32_t)(sizeof(float2) * KR * KR));
      }
      st_bj = W.bj_setup();
      W.agram = P.D.resid_gram ? P.A + (size_t)g * KR * KR : nullptr;
      cur = g;
    }
    if (P.b) {
      for (int i = gtid; i < K / 2; i += GT)
        reinterpret_cast<float4*>(S.b)[i] = (KR == K || 2 * i < KR) ? reinterpret_cast<const float4*>(
                                                                          P.b + (size_t)s * KR)[i]
                                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      matched_filter<K, KR>(P.H + (size_t)g * KR * P.N, P.y + (size_t)s * P.N, P.N, P.gram, S, lane, sj,
                            kSplitWarps);
    }
    W.gsync();  // b and the slot are complete
    W.detect(s, true, st_bj);
  }
}

// Grouped mode: CTA c takes groups c, c + gridDim.x, ...; for each, all its
// threads round the group's A into the shared slot, warps 0..K/32-1 invert the
// diagonal blocks (one block column per lane), and the eight warps take the
// group's received vectors eight at a time (warp w: vector 8i + w): their b
// (given, or the matched filter formed here), then detect in lockstep, every
// product with A one CTA-wide product for the eight vectors (CgWarp NV = 8).
// A warp without a vector in the last round runs on b = 0 and writes nothing.
// A given b may share memory with x_hat: a vector's b is read before its
// x_hat is written, by the same warp.
template <int KR, bool BF, int LT>
__global__ void __launch_bounds__(kSolveWarps * 32, 2) solve_grouped_kernel(const __grid_constant__ SolveTcParams P) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  constexpr int K = pad_k(KR);
  constexpr int NT = kSolveWarps * 32;
  constexpr int VST = grouped_vec_bytes(K);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* base = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
  Slot S;
  S.A16 = base;
  S.Md = reinterpret_cast<float2*>(base + 4 * K * K);
  uint8_t* vbase = base + 4 * K * K + md_bytes(K, LT);
  S.b = reinterpret_cast<float2*>(vbase + warp * VST);
  S.W = reinterpret_cast<float2*>(vbase + warp * VST + 8 * K);
  S.Pk = reinterpret_cast<uint32_t*>(vbase + kSolveWarps * VST);
  volatile int* flag = reinterpret_cast<volatile int*>(vbase + kSolveWarps * VST + grouped_pk_bytes(K));
  CgWarp<K, BF, LT, KR, kSolveWarps, 1, 2> W(P.D, S, lane);
  W.vw = warp;
  W.vbase = vbase;
  W.vst = VST;
  for (int64_t g = blockIdx.x; g < P.n_groups; g += gridDim.x) {
    const int64_t s0 = P.group_start[g], s1 = P.group_start[g + 1];
    if (s1 <= s0) continue;
    W.agram = P.D.resid_gram ? P.A + (size_t)g * KR * KR : nullptr;
    __syncthreads();  // the previous group's vectors are done with the slot
    fill_A<K, KR, BF, LT>(P.A + (size_t)g * KR * KR, S, threadIdx.x, NT);  // A -> [Re A; Im A], blocks
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    int st0 = 0;
    if constexpr (LT > 0) {  // block-Jacobi setup (eq. pre_BJ), 32 block columns per warp
      constexpr int MLD = md_row_stride(LT), MBS = md_block_stride(LT);
      if (warp * 32 < K && gj_blocks<K, LT, 1>(S.Md, lane, warp * 32)) *flag = 1;
      __syncthreads();
      if (*flag) {  // a failed block: M_d = I for the group
        for (int i = threadIdx.x; i < K * LT; i += NT)
          S.Md[(i / LT / LT) * MBS + ((i / LT) % LT) * MLD + i % LT] =
              make_float2((i / LT) % LT == i % LT ? 1.f : 0.f, 0.f);
        st0 = 8;
      }
      __syncthreads();
    }
    for (int64_t s = s0 + warp; s - warp < s1; s += kSolveWarps) {  // the same rounds on every warp
      const bool valid = s < s1;
      if (!valid) {
        for (int k = lane; k < K; k += 32) S.b[k] = make_float2(0.f, 0.f);
        __syncwarp();
      } else if (P.b) {
        load_b<K, KR>(P.b + (size_t)s * KR, S, lane);  // formed beforehand for the whole group (mf_mma)
      } else {
        matched_filter<K, KR>(P.H + (size_t)g * KR * P.N, P.y + (size_t)s * P.N, P.N, P.gram, S, lane);
      }
      W.detect(s, valid, st0);
      __syncwarp();
    }
  }
}

template <int K, bool BF, int LT>
cudaError_t launch_g(const SolveTcParams& P, int num_sms, cudaStream_t stream) {
  const size_t smem = solve_grouped_smem_bytes(K, LT);
  cudaError_t e =
      cudaFuncSetAttribute(solve_grouped_kernel<K, BF, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_grouped_kernel<K, BF, LT>, kSolveWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > P.n_groups) grid = P.n_groups;
  if (grid <= 0) return cudaSuccess;
  solve_grouped_kernel<K, BF, LT><<<(unsigned)grid, kSolveWarps * 32, smem, stream>>>(P);
  return cudaGetLastError();
}

template <int K, bool BF, int LT>
cudaError_t launch_split(const SolveTcParams& P, int num_sms, cudaStream_t stream) {
  const size_t smem = solve_split_smem_bytes(K, LT);
  cudaError_t e =
      cudaFuncSetAttribute(solve_split_kernel<K, BF, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  constexpr int NT = kSplitWarps * kSplitGroups * 32;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_split_kernel<K, BF, LT>, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)num_sms * per_sm;
  const int64_t need = (P.n + kSplitGroups - 1) / kSplitGroups;
  if (grid > need) grid = need;
  if (grid <= 0) return cudaSuccess;
  solve_split_kernel<K, BF, LT><<<(unsigned)grid, NT, smem, stream>>>(P);
  return cudaGetLastError();
}

template <int K, bool BF, int LT>
cudaError_t launch_s(const SolveTcParams& P, int num_sms, cudaStream_t stream) {
  if constexpr (K == 128) {
    return launch_split<K, BF, LT>(P, num_sms, stream);
  } else {
  const size_t smem = solve_tc_smem_bytes(K, LT);
  cudaError_t e =
      cudaFuncSetAttribute(solve_tc_kernel<K, BF, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  constexpr int W = solve_warps(K);
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_tc_kernel<K, BF, LT>, W * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)num_sms * per_sm;
  const int64_t need = (P.n + W - 1) / W;
  if (grid > need) grid = need;
  if (grid <= 0) return cudaSuccess;
  solve_tc_kernel<K, BF, LT><<<(unsigned)grid, W * 32, smem, stream>>>(P);
  return cudaGetLastError();
  }
}

}  // namespace

template <int K>
cudaError_t launch_solve_grouped_k(const SolveTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream) {
  switch (P.D.L * 2 + (mv_bf16 ? 1 : 0)) {
    case 0: return launch_g<K, false, 0>(P, num_sms, stream);
    case 1: return launch_g<K, true, 0>(P, num_sms, stream);
    case 8: return launch_g<K, false, 4>(P, num_sms, stream);
    case 9: return launch_g<K, true, 4>(P, num_sms, stream);
    case 16: return launch_g<K, false, 8>(P, num_sms, stream);
    case 17: return launch_g<K, true, 8>(P, num_sms, stream);
    case 32: if constexpr (K >= 16) return launch_g<K, false, 16>(P, num_sms, stream); else return cudaErrorInvalidValue;
    case 33: if constexpr (K >= 16) return launch_g<K, true, 16>(P, num_sms, stream); else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <int K>
cudaError_t launch_solve_tc_k(const SolveTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream) {
  switch (P.D.L * 2 + (mv_bf16 ? 1 : 0)) {
    case 0: return launch_s<K, false, 0>(P, num_sms, stream);
    case 1: return launch_s<K, true, 0>(P, num_sms, stream);
    case 8: return launch_s<K, false, 4>(P, num_sms, stream);
    case 9: return launch_s<K, true, 4>(P, num_sms, stream);
    case 16: return launch_s<K, false, 8>(P, num_sms, stream);
    case 17: return launch_s<K, true, 8>(P, num_sms, stream);
    case 32: if constexpr (K >= 16) return launch_s<K, false, 16>(P, num_sms, stream); else return cudaErrorInvalidValue;
    case 33: if constexpr (K >= 16) return launch_s<K, true, 16>(P, num_sms, stream); else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpcg
