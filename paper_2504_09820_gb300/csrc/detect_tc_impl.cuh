#pragma once
// Fused tensor-core detector (kernel templates; instantiated per K by
// detect_tc_k{16,32,64}.cu): the whole path for K in {16, 32, 64} in one
// persistent launch (one CTA per SM, 16 warps).
//
//   warps 0-3    drain warpgroup: TMEM accumulator -> system slots
//   warps 4-9    CG warps: warp 4+c runs every system that lands in slot c
//                (as many slots as shared memory holds, up to six)
//   warps 10-13  converters: FP32 stages -> bf16/fp16 swizzled operand stages
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
//   * refinement: r = b - A x on the tensor cores with the same A and
//     x = x_hi + x_mid + x_lo split over B columns, a correction solve,
//     x += d; rel_res; Gray-QAM decision; bit errors.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "detect_tc.cuh"
#include "tc_pipeline.cuh"

namespace fpcg {

namespace {

constexpr int kThreads = 16 * 32;
constexpr int kMmaWarp = 15;
constexpr int kProdWarp = 14;
constexpr int kCg0 = 4;                     // CG warps 4-9
constexpr int kConv0 = kCg0 + kTcCgWarps;   // converter warps 10-13
constexpr int kConv = kProdWarp - kConv0;

// ---- one system slot in shared memory -----------------------------------------
struct Slot {
  uint8_t* A16;     // [2K][K] 16-bit, row r at r*2K bytes, 16-byte chunk c at (c ^ swz(r))
  float2* Md;       // diagonal blocks of A (fp32), inverted in place (md_*_stride layout)
  float2* b;        // [K]
  float2* W;        // [K] matvec result, redistributed
  uint32_t* Pk;     // [3K] packed B fragments
};

__device__ inline Slot slot_carve(uint8_t* base, int K, int L) {
  Slot s;
  uint8_t* p = base;
  s.A16 = p;
  p += 4 * K * K;
  s.Md = (float2*)p;
  p += sizeof(float2) * (L > 0 ? (K / L) * md_block_stride(L) : 2);
  s.b = (float2*)p;
  p += sizeof(float2) * K;
  s.W = (float2*)p;
  p += sizeof(float2) * K;
  s.Pk = (uint32_t*)p;
  return s;
}

// 16-byte chunk swizzle of row r of a [2K][K] 16-bit matrix (K/8 chunks per
// row): eight consecutive rows at one chunk hit eight different bank groups.
template <int K>
__device__ __forceinline__ uint32_t a16_offset(int r, int chunk) {
  constexpr int CPR = K / 8;                          // chunks per row: 8, 4, 2
  constexpr int SH = CPR == 8 ? 0 : CPR == 4 ? 1 : 2; // rows per swizzle step
  return (uint32_t)(r * (2 * K) + ((chunk ^ ((r >> SH) & (CPR - 1))) << 4));
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
// c = l + 32e (e < NE, c < K) of their blocks.  Per pivot pv, with
// d = 1 / M[pv][pv] and f = column pv of the block:
//   M[pv][j] <- M[pv][j] d,  M[i][j] <- M[i][j] - f_i M[pv][j] d   (j != pv)
//   M[pv][pv] <- d,          M[i][pv] <- -f_i d                    (j == pv)
// (one branch-free update for both cases).  Returns nonzero (on every lane) if
// a pivot was not positive.
template <int K, int LT, int NE>
__device__ __forceinline__ int gj_blocks(float2* Md, int lane) {
  constexpr int LD = md_row_stride(LT), BS = md_block_stride(LT);
  float2* M[NE];
  int j[NE];
  bool on[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int c = lane + 32 * e;
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
template <int K, bool BF, int LT>
struct CgWarp {
  static constexpr int KT = K / 16;          // k-tiles (16 users)
  static constexpr int MT = K / 16;          // m-tiles of Re A (and of Im A)
  static constexpr int E = K == 64 ? 2 : 1;  // vector rows per lane
  static constexpr int NCOL = 6;             // B columns (re, im) x (hi, mid, lo)
  const DetectTcParams& P;
  Slot S;
  int lane, g, t;
  int ipf, alpha_num, iters, refine_steps, refine_iters;  // parameters kept in registers

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
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const float nx = __shfl_down_sync(0xffffffffu, v[e].x, 1);
      const float ny = __shfl_down_sync(0xffffffffu, v[e].y, 1);
      const int rl = lane + 32 * e;
      if (vact() && (rl & 1) == 0) {
        const int kt = rl >> 4, j = rl & 15, tt = (j & 7) >> 1, h = j >> 3;
        uint32_t* w = S.Pk + (kt * NCOL * 4 + tt) * 2 + h;
        float a[4] = {v[e].x, nx, v[e].y, ny};
#pragma unroll
        for (int s3 = 0; s3 < 3; ++s3) {
          float hh[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            hh[u] = round16<BF>(a[u]);
            a[u] = split ? a[u] - hh[u] : 0.f;  // exact remainder of the rounding
          }
          w[(2 * s3) * 8] = pk2<BF>(hh[0], hh[1]);
          w[(2 * s3 + 1) * 8] = pk2<BF>(hh[2], hh[3]);
        }
      }
    }
    __syncwarp();
  }

  // W = A v (res = false) or W = b - A v (res = true: the three column pairs
  // of v are summed), one m-tile (16 rows of Re A and of Im A) at a time; lane
  // (g, t) holds C rows g, g+8 and columns 2t, 2t+1.  Then w = W in the vector
  // layout.
  __device__ __forceinline__ void apply(bool res, float2 (&w)[E]) {
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
    const uint32_t abase = tc::smem_u32(S.A16);
    const int lr = lane & 15, lc = lane >> 4;
#pragma unroll 1  // unrolled runs slower in the full kernel (code size)
    for (int mt = 0; mt < MT; ++mt) {
      float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
      float cr2[4] = {0.f, 0.f, 0.f, 0.f}, ci2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {  // two accumulator chains per part (even / odd kt)
        uint32_t ar[4], ai[4];
        tc::ldmatrix_x4(ar, abase + a16_offset<K>(16 * mt + lr, 2 * kt + lc));
        tc::ldmatrix_x4(ai, abase + a16_offset<K>(K + 16 * mt + lr, 2 * kt + lc));
        if (kt & 1) {
          mma16<BF>(cr2, ar, b0[kt], b1[kt]);
          mma16<BF>(ci2, ai, b0[kt], b1[kt]);
        } else {
          mma16<BF>(cr, ar, b0[kt], b1[kt]);
          mma16<BF>(ci, ai, b0[kt], b1[kt]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        cr[q] += cr2[q];
        ci[q] += ci2[q];
      }
      if (res) {  // add the mid (t = 1) and lo (t = 2) column products into t = 0
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float r1 = __shfl_down_sync(0xffffffffu, cr[q], 1);
          const float r2 = __shfl_down_sync(0xffffffffu, cr[q], 2);
          const float i1 = __shfl_down_sync(0xffffffffu, ci[q], 1);
          const float i2 = __shfl_down_sync(0xffffffffu, ci[q], 2);
          cr[q] += r1 + r2;
          ci[q] += i1 + i2;
        }
      }
      if (t == 0) {
        // rows 16mt+g / +8: (Re A vr - Im A vi) + i (Re A vi + Im A vr)
        float2 w0 = make_float2(cr[0] - ci[1], cr[1] + ci[0]);
        float2 w8 = make_float2(cr[2] - ci[3], cr[3] + ci[2]);
        if (res) {
          const float2 bb0 = S.b[16 * mt + g], bb8 = S.b[16 * mt + g + 8];
          w0 = make_float2(bb0.x - w0.x, bb0.y - w0.y);
          w8 = make_float2(bb8.x - w8.x, bb8.y - w8.y);
        }
        S.W[16 * mt + g] = w0;
        S.W[16 * mt + g + 8] = w8;
      }
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e) w[e] = vact() ? S.W[lane + 32 * e] : make_float2(0.f, 0.f);
    __syncwarp();
  }

  // z = M_d r (z = r without a preconditioner): r is staged in W and each
  // lane reads its block's L entries of it (broadcast) and its row of M_d.
  __device__ __forceinline__ void precond(const float2 (&r)[E], float2 (&z)[E]) {
    if constexpr (LT == 0) {
#pragma unroll
      for (int e = 0; e < E; ++e) z[e] = r[e];
    } else {
      constexpr int MLD = md_row_stride(LT), MBS = md_block_stride(LT);
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (vact()) S.W[lane + 32 * e] = r[e];
      __syncwarp();
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = vact() ? lane + 32 * e : 0;
        const float4* rb = reinterpret_cast<const float4*>(S.W + (k & ~(LT - 1)));
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
  __device__ void detect(int64_t sys, bool valid) {
    int st = 0;
    if constexpr (LT > 0) {  // block-Jacobi setup (eq. pre_BJ); a failed block gives M_d = I
      constexpr int MLD = md_row_stride(LT), MBS = md_block_stride(LT);
      if (gj_blocks<K, LT, E>(S.Md, lane)) {
        st |= 8;
        for (int i = lane; i < K * LT; i += 32)
          S.Md[(i / LT / LT) * MBS + ((i / LT) % LT) * MLD + i % LT] =
              make_float2((i / LT) % LT == i % LT ? 1.f : 0.f, 0.f);
        __syncwarp();
      }
    }
    // per-system inputs of the output stage, loaded now (their latency hides under the solve)
    const int64_t base = sys * (int64_t)K;
    const bool want_sym = valid && (P.sym || P.bit_errors);
    const int M = want_sym ? P.qam[sys] : 0;
    int txv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) txv[e] = (want_sym && P.tx && vact()) ? P.tx[base + lane + 32 * e] : 0;
    float* hist = (P.res_hist && valid) ? P.res_hist + sys * (int64_t)(iters + 1) : nullptr;

    float2 x[E], d[E], r[E], p[E], z[E], w[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      x[e] = d[e] = p[e] = make_float2(0.f, 0.f);
      r[e] = vact() ? S.b[lane + 32 * e] : make_float2(0.f, 0.f);
    }
    int pass = 0, it = 0, iters_p = iters, mask = ~0;
    float rho = 0.f, rho_prev = 1.f, rr = 0.f;
    bool fresh = true;  // r is a new right-hand side: start a pass
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
        pack(w, rt);
        apply(rt, w);
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
        } else {
          float phi, rp;
          dot2(p, w, r, p, phi, rp);
          phi = rip(phi);
          rho_prev = (LT > 0 && alpha_num == 0) ? rip(rp) : rho;
          int bad = 0;
          if (rho_prev == 0.f) bad = 2;
          else if (!(phi > 0.f) || !isfinite(phi) || !isfinite(rho_prev)) bad = 1;
          if (bad) {  // the pass stops here; the history repeats its last value
            st |= bad & mask;
            if (hist && lane == 0)
              for (int k = it + 1; k <= iters_p; ++k) hist[k] = hist[it];
            it = iters_p;
            continue;
          }
          const float alpha = rho_prev / phi;
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
      const float beta = fresh ? 0.f : rho_new / rho_prev;
#pragma unroll
      for (int e = 0; e < E; ++e)
        p[e] = fresh ? z[e] : make_float2(fmaf(beta, p[e].x, z[e].x), fmaf(beta, p[e].y, z[e].y));
      rho = rho_new;
      if (hist && lane == 0) hist[it] = sqrtf(rr);
      fresh = false;
    }

    if (!valid) return;
    float nr = 0.f, nb = 0.f;
    int nonfinite = 0;
    unsigned errs = 0;
    const int m = qam_sqrt(M);
    const float sc = m ? sqrtf((float)(2 * (M - 1) / 3)) : 0.f;  // 2(M-1)/3 is an integer here
    const int nb2 = m ? qam_bits_axis(m) : 0;
    if (vact()) {
#pragma unroll  // x, r, txv stay in registers only with static indices
      for (int e = 0; e < E; ++e) {
        const float2 bv = S.b[lane + 32 * e];
        nr += r[e].x * r[e].x + r[e].y * r[e].y;
        nb += bv.x * bv.x + bv.y * bv.y;
        const int k = lane + 32 * e;
        if (!(isfinite(x[e].x) && isfinite(x[e].y))) nonfinite = 1;
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
    if (lane == 0) {
      if (P.rel_res) P.rel_res[sys] = nb > 0.f ? (double)sqrtf(nr / nb) : 0.0;
      if (nonfinite) st |= 4;
      if (want_sym && m == 0) st |= 16;
      if (P.status) P.status[sys] = st;
    }
  }
};

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
  uint8_t* slots;
};

// Drain warpgroup: tile j of this CTA (TMEM buffer j & 1) holds systems
// seq = j*P + p, p < P, which go to slots seq % nslots.  Thread = TMEM lane =
// row 2k + odd of its system's block.
template <int K, bool BF, int LT>
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
  const size_t slot_bytes = tc_slot_bytes(K, LT);
  int64_t j = 0;
  for (int64_t tile = tile0; tile < pp.ntiles; tile += tstep, ++j) {
    const uint32_t b = (uint32_t)(j & 1), qa = (uint32_t)(j >> 1);
    const int64_t sys = tile * PP + ps;
    const bool valid = sys < pp.batch;
    const float s2 = valid ? (float)P.sigma2[sys] : 1.f;  // issued before the wait
    bool ok = tc::mbar_wait(&S.bars->acc_full[b], qa & 1u, S.abort);
    for (int p = 0; ok && p < PP; ++p) {
      const int64_t seq = j * PP + p;
      const uint32_t sl = (uint32_t)(seq % ns), use = (uint32_t)(seq / ns);
      if (use > 0) ok = tc::mbar_wait(&S.sbars->slot_empty[sl], (use - 1) & 1u, S.abort);
    }
    if (!ok) {
      *S.abort = 1;
      break;
    }
    tc::tc_fence_after();
    const uint32_t tb = lane_base + b * (uint32_t)tcp::kAccCols;
    Slot sl = slot_carve(S.slots + ((j * PP + ps) % ns) * slot_bytes, K, LT);
    const int arow = odd ? K + k : k;           // row of [Re A; Im A]
    const int kb0 = (k / (LT > 0 ? LT : 1)) * LT;  // first column of k's diagonal block
#pragma unroll 1
    for (int cg = blk0; cg < blk0 + twoK; cg += 32) {
      uint32_t v[2][16];
      tc::tmem_ld16_async(tb + (uint32_t)cg, v[0]);
      tc::tmem_ld16_async(tb + (uint32_t)(cg + 16), v[1]);
      tc::tmem_wait_ld();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float a[8];
        const int l0 = (cg + 16 * u - blk0) >> 1;  // first of the 8 columns l of this chunk
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const float vm = __uint_as_float(v[u][2 * m]);
          const float other = __shfl_xor_sync(0xffffffffu, __uint_as_float(v[u][2 * m + 1]), 1);
          float val = odd ? (other - vm) : (vm + other);
          if (!valid) val = 0.f;
          if (l0 + m == k) val = odd ? 0.f : val + s2;
          a[m] = val;
        }
        // 8 columns -> one 16-byte chunk of row arow
        uint4 pkd;
        pkd.x = pk2<BF>(a[0], a[1]);
        pkd.y = pk2<BF>(a[2], a[3]);
        pkd.z = pk2<BF>(a[4], a[5]);
        pkd.w = pk2<BF>(a[6], a[7]);
        *reinterpret_cast<uint4*>(sl.A16 + a16_offset<K>(arow, l0 >> 3)) = pkd;
        if constexpr (LT > 0) {
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const int l = l0 + m;
            if (l >= kb0 && l < kb0 + LT)
              reinterpret_cast<float*>(sl.Md + (k / LT) * MBS + (k % LT) * MLD + (l - kb0))[odd] = a[m];
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
template <int K, bool BF, int LT>
__device__ void cg_role(const DetectTcParams& P, const Smem& S, int c, int64_t tile0, int64_t tstep) {
  const tcp::Pipe& pp = P.pipe;
  const int lane = threadIdx.x & 31;
  constexpr int PP = 64 / K;
  const int ns = P.nslots;
  const int64_t nloc = tile0 < pp.ntiles ? (pp.ntiles - tile0 + tstep - 1) / tstep : 0;
  CgWarp<K, BF, LT> W(P, slot_carve(S.slots + c * tc_slot_bytes(K, LT), K, LT), lane);
  int64_t seq = c;
  for (; seq / PP < nloc; seq += ns) {
    const uint32_t use = (uint32_t)(seq / ns);
    if (!tc::mbar_wait(&S.sbars->slot_full[c], use & 1u, S.abort)) {
      *S.abort = 1;
      break;
    }
    const int64_t tile = tile0 + (seq / PP) * tstep;
    const int64_t sys = tile * PP + seq % PP;
    W.detect(sys, sys < pp.batch);
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

template <int K, bool BF, int LT>
__global__ void __launch_bounds__(kThreads, 1) detect_tc_kernel(const __grid_constant__ DetectTcParams P) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  Smem S;
  {
    const uint32_t a = tc::smem_u32(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (a & 1023u)) & 1023u);
    S.pipe = base;
    S.bars = reinterpret_cast<tcp::Bars*>(base + tcp::pipe_bytes(kTcStages32));
    S.sbars = reinterpret_cast<Bars2*>(S.bars + 1);
    S.tmem_slot = reinterpret_cast<uint32_t*>(S.sbars + 1);
    S.abort = reinterpret_cast<volatile int*>(S.tmem_slot + 1);
    S.slots = base + tc_slots_offset();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const tcp::Pipe& pp = P.pipe;
  for (int i = threadIdx.x; i < tcp::kStages * tcp::kStageBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(tcp::stage16(S.pipe, 0))[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    tcp::init_bars(*S.bars, kConv, kTcStages32);
    for (int i = 0; i < kTcCgWarps; ++i) {
      tc::mbar_init(&S.sbars->slot_full[i], 1);
      tc::mbar_init(&S.sbars->slot_empty[i], 1);
    }
    *S.abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == kMmaWarp) tc::tmem_alloc(S.tmem_slot, 2 * tcp::kAccCols);
  tc::fence_proxy_async();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *S.tmem_slot;
  const int64_t tile0 = blockIdx.x, tstep = gridDim.x;

  if (warp == kMmaWarp) {
    if (lane == 0) tcp::mma_role(pp, S.pipe, *S.bars, S.abort, tmem, tile0, tstep);
    __syncwarp();
  } else if (warp == kProdWarp) {
    if (lane == 0) tcp::producer_role<kTcStages32>(pp, S.pipe, *S.bars, S.abort, tile0, tstep);
    __syncwarp();
  } else if (warp >= kConv0) {
    tcp::converter_role<kConv, kTcStages32>(pp, S.pipe, *S.bars, S.abort, tile0, tstep, warp - kConv0, lane);
  } else if (warp >= kCg0) {
    if (warp - kCg0 < P.nslots) cg_role<K, BF, LT>(P, S, warp - kCg0, tile0, tstep);
  } else {
    drain_role<K, BF, LT>(P, S, tmem, tile0, tstep);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * tcp::kAccCols);
  }
}

template <int K, bool BF, int LT>
cudaError_t launch_k(DetectTcParams P, int num_sms, cudaStream_t stream) {
  const size_t smem = detect_tc_smem_bytes(K, P.L);
  P.nslots = tc_num_slots(K, P.L);
  cudaError_t e =
      cudaFuncSetAttribute(detect_tc_kernel<K, BF, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = P.pipe.ntiles < num_sms ? P.pipe.ntiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  detect_tc_kernel<K, BF, LT><<<(unsigned)grid, kThreads, smem, stream>>>(P);
  return cudaGetLastError();
}

}  // namespace

template <int K>
cudaError_t launch_detect_tc_k(const DetectTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream) {
  switch (P.L * 2 + (mv_bf16 ? 1 : 0)) {
    case 0: return launch_k<K, false, 0>(P, num_sms, stream);
    case 1: return launch_k<K, true, 0>(P, num_sms, stream);
    case 8: return launch_k<K, false, 4>(P, num_sms, stream);
    case 9: return launch_k<K, true, 4>(P, num_sms, stream);
    case 16: return launch_k<K, false, 8>(P, num_sms, stream);
    case 17: return launch_k<K, true, 8>(P, num_sms, stream);
    case 32: return launch_k<K, false, 16>(P, num_sms, stream);
    case 33: return launch_k<K, true, 16>(P, num_sms, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpcg
