// Fused tensor-core detector: the whole path for K in {16, 32, 64} in one
// persistent launch (one CTA per SM).
//
//   warps 0-3    CG warpgroup 0: tiles 0, 2, 4, ... of this CTA (TMEM buffer 0)
//   warps 4-7    CG warpgroup 1: tiles 1, 3, 5, ...             (TMEM buffer 1)
//   warps 8-14   converters: H, y -> bf16/fp16 swizzled stages
//   warp 15      TMEM allocation and the UMMA-issuing thread
//
// Gram + matched filter (Section II, eq. inversion) come out of the tcgen05
// pipeline of tc_pipeline.cuh.  A CG warpgroup then, for its tile of P = 64/K
// systems, copies A and b from TMEM to shared memory and releases the
// accumulator; each system is owned by K/16 warps, each warp by 16 of its rows:
//   * block-Jacobi setup (eq. pre_BJ): the warp inverts its own L x L diagonal
//     blocks (L divides 16) by in-place Gauss-Jordan in shared memory;
//   * A p (u_MV): A rounded to bf16/fp16 lives in registers as mma.sync A
//     fragments, [Re A; Im A] (two 16-row tiles per warp) times the 16x8 B
//     fragment [Re p, Im p, 0...] -- products exact, fp32 sums;
//   * Algorithm 2 / 3: vectors of the warp's rows in registers, inner products
//     reduced over the warp and then over the system's warps (u_IP rounding),
//     updates by FMA at u_W = fp32;
//   * refinement: r = b - A x from the fp32 A in shared memory, a correction
//     solve, x += d; rel_res; Gray-QAM decision; bit errors.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "detect_tc.cuh"
#include "tc_pipeline.cuh"

namespace fpcg {

namespace {

constexpr int kThreads = 16 * 32;
constexpr int kMmaWarp = 15;
constexpr int kConv0 = 8;
constexpr int kConv = 7;  // converter warps 8-14

// Per-warpgroup shared memory (rows are the 64 rows of a tile: row = ps*K + k).
struct CgSmem {
  float2* A;      // [64][K+1]
  float2* b;      // [64]
  float2* v;      // [64] scratch vector (p, then x for residuals)
  float2* r;      // [64] r for the block-Jacobi product
  float2* Md;     // [64][L]
  float* red;     // [3][4][2] partial sums per warp
  double* dred;   // [4][2]
  int* flag;      // [4]
};

__host__ __device__ inline size_t cg_smem_bytes(int K, int L) {
  size_t s = 0;
  s += sizeof(float2) * 64 * (K + 1);
  s += sizeof(float2) * 64 * 3;
  s += sizeof(float2) * 64 * (L > 0 ? L : 1);
  s += sizeof(float) * 3 * 4 * 2;
  s += sizeof(double) * 4 * 2;
  s += sizeof(int) * 4;
  return (s + 127) & ~size_t(127);
}

__device__ inline CgSmem cg_carve(uint8_t* base, int K, int L) {
  CgSmem s;
  uint8_t* p = base;
  s.A = (float2*)p;
  p += sizeof(float2) * 64 * (K + 1);
  s.b = (float2*)p;
  p += sizeof(float2) * 64;
  s.v = (float2*)p;
  p += sizeof(float2) * 64;
  s.r = (float2*)p;
  p += sizeof(float2) * 64;
  s.Md = (float2*)p;
  p += sizeof(float2) * 64 * (L > 0 ? L : 1);
  s.dred = (double*)p;  // 8-byte aligned: everything before is a multiple of 8
  p += sizeof(double) * 4 * 2;
  s.red = (float*)p;
  p += sizeof(float) * 3 * 4 * 2;
  s.flag = (int*)p;
  return s;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <int K, bool BF>
struct CgWarp {
  static constexpr int KT = K / 16;     // k-tiles
  static constexpr int WS = K / 16;     // warps per system
  const DetectTcParams& P;
  CgSmem S;
  int wi, lane, g, t, ps, rb, row0, bar_id;
  int64_t sys;
  bool valid;
  uint32_t afr[2][KT][4];               // [Re A; Im A] fragments of the warp's 16 rows

  __device__ CgWarp(const DetectTcParams& P_, CgSmem S_, int wi_, int lane_, int bar_id_)
      : P(P_), S(S_), wi(wi_), lane(lane_), bar_id(bar_id_) {
    g = lane >> 2;
    t = lane & 3;
    ps = wi / WS;
    rb = wi % WS;
    row0 = ps * K + 16 * rb;
  }

  __device__ __forceinline__ void wg_sync() { tc::bar_sync(bar_id, 128); }

  __device__ __forceinline__ uint32_t pk(float a, float b) { return tcp::pack2(a, b, BF ? 1 : 0); }

  // sum over the warp of a value held by lanes t == 0 (others hold 0)
  __device__ __forceinline__ float wsum8(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
  }

  // Sum of two per-warp partials over the system's warps (one WG barrier).
  __device__ __forceinline__ void sys_sum2(float& a, float& b, int slot) {
    a = wsum8(a);
    b = wsum8(b);
    float* red = S.red + slot * 8;
    if (lane == 0) {
      red[wi * 2] = a;
      red[wi * 2 + 1] = b;
    }
    wg_sync();
    float sa = 0.f, sb = 0.f;
    for (int w = ps * WS; w < ps * WS + WS; ++w) {
      sa += red[w * 2];
      sb += red[w * 2 + 1];
    }
    a = sa;
    b = sb;
  }

  __device__ void build_fragments() {
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      const int c0 = 16 * kt + 2 * t;
      const float2* r0 = S.A + (row0 + g) * (K + 1);
      const float2* r8 = S.A + (row0 + g + 8) * (K + 1);
      afr[0][kt][0] = pk(r0[c0].x, r0[c0 + 1].x);
      afr[0][kt][1] = pk(r8[c0].x, r8[c0 + 1].x);
      afr[0][kt][2] = pk(r0[c0 + 8].x, r0[c0 + 9].x);
      afr[0][kt][3] = pk(r8[c0 + 8].x, r8[c0 + 9].x);
      afr[1][kt][0] = pk(r0[c0].y, r0[c0 + 1].y);
      afr[1][kt][1] = pk(r8[c0].y, r8[c0 + 1].y);
      afr[1][kt][2] = pk(r0[c0 + 8].y, r0[c0 + 9].y);
      afr[1][kt][3] = pk(r8[c0 + 8].y, r8[c0 + 9].y);
    }
  }

  // varpi = A p for the warp's rows g, g+8 (valid in lanes t == 0); p of the
  // whole system is read from S.v.
  __device__ __forceinline__ void matvec(float2& w0, float2& w1) {
    uint32_t b0[KT], b1[KT];
    const float2* pv = S.v + ps * K;
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      b0[kt] = b1[kt] = 0u;
      if (g < 2) {
        const int c0 = 16 * kt + 2 * t;
        const float2 a0 = pv[c0], a1 = pv[c0 + 1], a8 = pv[c0 + 8], a9 = pv[c0 + 9];
        b0[kt] = g == 0 ? pk(a0.x, a1.x) : pk(a0.y, a1.y);
        b1[kt] = g == 0 ? pk(a8.x, a9.x) : pk(a8.y, a9.y);
      }
    }
    float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      if (BF) {
        tc::mma_m16n8k16_bf16(cr, afr[0][kt], b0[kt], b1[kt]);
        tc::mma_m16n8k16_bf16(ci, afr[1][kt], b0[kt], b1[kt]);
      } else {
        tc::mma_m16n8k16_f16(cr, afr[0][kt], b0[kt], b1[kt]);
        tc::mma_m16n8k16_f16(ci, afr[1][kt], b0[kt], b1[kt]);
      }
    }
    // rows g / g+8: (Re A pr - Im A pi) + i (Re A pi + Im A pr)
    w0 = make_float2(cr[0] - ci[1], cr[1] + ci[0]);
    w1 = make_float2(cr[2] - ci[3], cr[3] + ci[2]);
  }

  // z = M_d r for rows g, g+8 (lanes t == 0); r0, r1 already stored in S.r.
  __device__ __forceinline__ void precond(float2 r0, float2 r1, float2& z0, float2& z1) {
    const int L = P.L;
    if (L == 0) {
      z0 = r0;
      z1 = r1;
      return;
    }
    z0 = make_float2(0.f, 0.f);
    z1 = make_float2(0.f, 0.f);
    if (t != 0) return;
    const int i0 = row0 + g, i1 = row0 + g + 8;
    const int s0 = i0 - (i0 - ps * K) % L, s1 = i1 - (i1 - ps * K) % L;
    for (int j = 0; j < L; ++j) {
      const float2 m0 = S.Md[i0 * L + j], q0 = S.r[s0 + j];
      const float2 m1 = S.Md[i1 * L + j], q1 = S.r[s1 + j];
      z0.x = fmaf(m0.x, q0.x, fmaf(-m0.y, q0.y, z0.x));
      z0.y = fmaf(m0.x, q0.y, fmaf(m0.y, q0.x, z0.y));
      z1.x = fmaf(m1.x, q1.x, fmaf(-m1.y, q1.y, z1.x));
      z1.y = fmaf(m1.x, q1.y, fmaf(m1.y, q1.x, z1.y));
    }
  }

  __device__ __forceinline__ float rip(float v) { return round_to(v, P.ip); }

  // Algorithm 2 (L == 0) or 3 (L > 0) from x0 = 0 on rhs (rows g, g+8 in
  // lanes t == 0).  Returns x in x0/x1 and status bits.
  __device__ int solve(float2 q0, float2 q1, int iters, float* hist, float2& x0, float2& x1) {
    const bool act = (t == 0);
    int st = 0;
    float2 r0 = act ? q0 : make_float2(0.f, 0.f), r1 = act ? q1 : make_float2(0.f, 0.f);
    x0 = x1 = make_float2(0.f, 0.f);
    if (act) {
      S.r[row0 + g] = r0;
      S.r[row0 + g + 8] = r1;
    }
    __syncwarp();
    float2 z0, z1;
    precond(r0, r1, z0, z1);
    float2 p0 = z0, p1 = z1;
    float rz = act ? (r0.x * z0.x + r0.y * z0.y + r1.x * z1.x + r1.y * z1.y) : 0.f;
    float rr = act ? (r0.x * r0.x + r0.y * r0.y + r1.x * r1.x + r1.y * r1.y) : 0.f;
    sys_sum2(rz, rr, 0);
    float rho = rip(rz);
    if (hist && lane == 0 && rb == 0) hist[0] = sqrtf(rr);
    bool live = true;
    for (int it = 0; it < iters; ++it) {
      if (act) {
        S.v[row0 + g] = p0;
        S.v[row0 + g + 8] = p1;
      }
      wg_sync();
      float2 w0, w1;
      matvec(w0, w1);
      float phi = act ? (p0.x * w0.x + p0.y * w0.y + p1.x * w1.x + p1.y * w1.y) : 0.f;
      float rp = act ? (r0.x * p0.x + r0.y * p0.y + r1.x * p1.x + r1.y * p1.y) : 0.f;
      sys_sum2(phi, rp, 1);
      phi = rip(phi);
      const float rho_prev = (P.L > 0 && P.alpha_num == 0) ? rip(rp) : rho;
      if (live) {
        if (rho_prev == 0.f) {
          st |= 2;
          live = false;
        } else if (!(phi > 0.f) || !isfinite(phi) || !isfinite(rho_prev)) {
          st |= 1;
          live = false;
        }
      }
      float2 nr0 = r0, nr1 = r1, nx0 = x0, nx1 = x1;
      if (live) {
        const float alpha = rho_prev / phi;
        nx0 = make_float2(fmaf(alpha, p0.x, x0.x), fmaf(alpha, p0.y, x0.y));
        nx1 = make_float2(fmaf(alpha, p1.x, x1.x), fmaf(alpha, p1.y, x1.y));
        nr0 = make_float2(fmaf(-alpha, w0.x, r0.x), fmaf(-alpha, w0.y, r0.y));
        nr1 = make_float2(fmaf(-alpha, w1.x, r1.x), fmaf(-alpha, w1.y, r1.y));
      }
      if (act) {
        S.r[row0 + g] = nr0;
        S.r[row0 + g + 8] = nr1;
      }
      __syncwarp();
      precond(nr0, nr1, z0, z1);
      float rzn = act ? (nr0.x * z0.x + nr0.y * z0.y + nr1.x * z1.x + nr1.y * z1.y) : 0.f;
      float rrn = act ? (nr0.x * nr0.x + nr0.y * nr0.y + nr1.x * nr1.x + nr1.y * nr1.y) : 0.f;
      sys_sum2(rzn, rrn, 2);
      if (live) {
        const float rho_new = rip(rzn);
        const float beta = rho_new / rho_prev;
        p0 = make_float2(fmaf(beta, p0.x, z0.x), fmaf(beta, p0.y, z0.y));
        p1 = make_float2(fmaf(beta, p1.x, z1.x), fmaf(beta, p1.y, z1.y));
        x0 = nx0;
        x1 = nx1;
        r0 = nr0;
        r1 = nr1;
        rho = rho_new;
      }
      if (hist && lane == 0 && rb == 0) hist[it + 1] = live ? sqrtf(rrn) : hist[it];
    }
    return st;
  }

  // out = b - A x for rows g, g+8 (lanes t == 0 get the result); x of the whole
  // system is read from S.v.  Plain fp32 sums, or compensated ones.
  __device__ void residual(float2& o0, float2& o1) {
    const float2* xs = S.v + ps * K;
    const float2* a0 = S.A + (row0 + g) * (K + 1);
    const float2* a1 = S.A + (row0 + g + 8) * (K + 1);
    if (!P.resid_comp) {
      float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
      for (int l = t; l < K; l += 4) {
        const float2 x = xs[l], m0 = a0[l], m1 = a1[l];
        s0.x = fmaf(m0.x, x.x, fmaf(-m0.y, x.y, s0.x));
        s0.y = fmaf(m0.x, x.y, fmaf(m0.y, x.x, s0.y));
        s1.x = fmaf(m1.x, x.x, fmaf(-m1.y, x.y, s1.x));
        s1.y = fmaf(m1.x, x.y, fmaf(m1.y, x.x, s1.y));
      }
#pragma unroll
      for (int o = 1; o < 4; o <<= 1) {
        s0.x += __shfl_xor_sync(0xffffffffu, s0.x, o);
        s0.y += __shfl_xor_sync(0xffffffffu, s0.y, o);
        s1.x += __shfl_xor_sync(0xffffffffu, s1.x, o);
        s1.y += __shfl_xor_sync(0xffffffffu, s1.y, o);
      }
      const float2 b0 = S.b[row0 + g], b1 = S.b[row0 + g + 8];
      o0 = make_float2(b0.x - s0.x, b0.y - s0.y);
      o1 = make_float2(b1.x - s1.x, b1.y - s1.y);
      return;
    }
    float h[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    if (t == 0) {
      h[0] = S.b[row0 + g].x;
      h[1] = S.b[row0 + g].y;
      h[2] = S.b[row0 + g + 8].x;
      h[3] = S.b[row0 + g + 8].y;
    }
    for (int l = t; l < K; l += 4) {
      const float2 x = xs[l], m0 = a0[l], m1 = a1[l];
      df_sub_prod(h[0], lo[0], m0.x, x.x);
      df_sub_prod(h[0], lo[0], -m0.y, x.y);
      df_sub_prod(h[1], lo[1], m0.x, x.y);
      df_sub_prod(h[1], lo[1], m0.y, x.x);
      df_sub_prod(h[2], lo[2], m1.x, x.x);
      df_sub_prod(h[2], lo[2], -m1.y, x.y);
      df_sub_prod(h[3], lo[3], m1.x, x.y);
      df_sub_prod(h[3], lo[3], m1.y, x.x);
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float h2 = __shfl_xor_sync(0xffffffffu, h[c], o), l2 = __shfl_xor_sync(0xffffffffu, lo[c], o);
        df_add(h[c], lo[c], h2, l2);
      }
    o0 = make_float2(__fadd_rn(h[0], lo[0]), __fadd_rn(h[1], lo[1]));
    o1 = make_float2(__fadd_rn(h[2], lo[2]), __fadd_rn(h[3], lo[3]));
  }

  // Gauss-Jordan inversion of the warp's L x L diagonal blocks in S.Md.
  __device__ int bj_setup() {
    const int L = P.L;
    int fail = 0;
    if (L == 0) return 0;
    const int blk = lane / L, j = lane % L;
    const bool on = lane < 16;
    const int R0 = row0 + blk * L;  // first row of the block (tile layout)
    const int kb = R0 - ps * K;     // its first column (system numbering)
    if (on)
      for (int i = 0; i < L; ++i) S.Md[(R0 + i) * L + j] = S.A[(R0 + i) * (K + 1) + kb + j];
    __syncwarp();
    for (int pv = 0; pv < L; ++pv) {
      float2 piv = on ? S.Md[(R0 + pv) * L + pv] : make_float2(1.f, 0.f);
      if (on && !(piv.x > 0.f && isfinite(piv.x))) fail = 1;
      const float den = piv.x * piv.x + piv.y * piv.y;
      const float2 dinv = make_float2(piv.x / den, -piv.y / den);
      __syncwarp();
      if (on && j != pv) S.Md[(R0 + pv) * L + j] = cmul(S.Md[(R0 + pv) * L + j], dinv);
      __syncwarp();
      if (on && j != pv) {
        const float2 prow = S.Md[(R0 + pv) * L + j];
        for (int i = 0; i < L; ++i) {
          if (i == pv) continue;
          const float2 f = S.Md[(R0 + i) * L + pv];
          float2 v = S.Md[(R0 + i) * L + j];
          const float2 fp = cmul(f, prow);
          v.x -= fp.x;
          v.y -= fp.y;
          S.Md[(R0 + i) * L + j] = v;
        }
      }
      __syncwarp();
      if (on) {
        if (j == pv) {
          S.Md[(R0 + pv) * L + pv] = dinv;
        } else {
          const float2 v = cmul(S.Md[(R0 + j) * L + pv], dinv);
          S.Md[(R0 + j) * L + pv] = make_float2(-v.x, -v.y);
        }
      }
      __syncwarp();
    }
    return __any_sync(0xffffffffu, fail);
  }
};

template <int K, bool BF>
__device__ void cg_role(const DetectTcParams& P, tcp::Bars& B, volatile int* abort, uint32_t tmem, uint8_t* cg_base,
                        int wg, int64_t tile0, int64_t tstep) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wi = warp - 4 * wg;  // warp within the warpgroup == TMEM lane quadrant
  CgWarp<K, BF> W(P, cg_carve(cg_base, K, P.L), wi, lane, 1 + wg);
  const tcp::Pipe& pp = P.pipe;
  const int twoK = 2 * K;
  const int trow = 32 * wi + lane;         // TMEM lane of this thread
  const int tps = trow / twoK;             // its system in the tile
  const int tk = (trow % twoK) >> 1;
  const int odd = trow & 1;
  int64_t j = wg;
  int64_t tile = tile0 + wg * tstep;
  for (; tile < pp.ntiles; tile += 2 * tstep, j += 2) {
    const uint32_t qa = (uint32_t)(j >> 1);
    if (!tc::mbar_wait(&B.acc_full[wg], qa & 1u, abort)) {
      *abort = 1;
      break;
    }
    tc::tc_fence_after();
    // ---- TMEM -> shared memory: A (fp32) and b, sigma^2 on the diagonal
    {
      const int64_t tsys = tile * pp.P + tps;
      const bool tvalid = tsys < pp.batch;
      const float s2 = tvalid ? (float)P.sigma2[tsys] : 1.f;
      const int R = tps * K + tk;
      float* Arow = reinterpret_cast<float*>(W.S.A + R * (K + 1));
      float* brow = reinterpret_cast<float*>(W.S.b + R);
      tcp::drain_tile(
          pp, tmem + (uint32_t)wg * tcp::kAccCols, wi, lane,
          [&](int l, float v) {
            if (!tvalid) v = 0.f;
            if (l == tk) v = odd ? 0.f : v + s2;
            Arow[2 * l + odd] = v;
          },
          [&](float v) { brow[odd] = tvalid ? v : 0.f; });
    }
    tc::tc_fence_before();
    W.wg_sync();
    if (wi == 0 && lane == 0) tc::mbar_arrive(&B.acc_empty[wg]);
    W.sys = tile * pp.P + W.ps;
    W.valid = W.sys < pp.batch;
    int st = 0;
    // ---- block-Jacobi setup
    if (lane == 0 && W.rb == 0) W.S.flag[W.ps] = 0;
    W.wg_sync();
    if (W.bj_setup() && lane == 0) atomicOr(&W.S.flag[W.ps], 1);
    W.wg_sync();
    if (P.L > 0 && W.S.flag[W.ps]) {  // fall back to M_d = I for this system
      st |= 8;
      if (lane < 16)
        for (int i = 0; i < P.L; ++i) {
          const int R = W.row0 + lane;
          W.S.Md[R * P.L + i] = make_float2((R - W.ps * K) % P.L == i ? 1.f : 0.f, 0.f);
        }
      __syncwarp();
    }
    W.build_fragments();
    // ---- main solve
    float* hist = (P.res_hist && W.valid) ? P.res_hist + W.sys * (int64_t)(P.iters + 1) : nullptr;
    float2 b0 = W.S.b[W.row0 + W.g], b1 = W.S.b[W.row0 + W.g + 8];
    float2 x0, x1;
    st |= W.solve(b0, b1, P.iters, hist, x0, x1);
    // ---- refinement: x += solve(b - A x)
    for (int rs = 0; rs < P.refine_steps; ++rs) {
      W.wg_sync();  // every warp is done reading S.v (p) of the last iteration
      if (W.t == 0) {
        W.S.v[W.row0 + W.g] = x0;
        W.S.v[W.row0 + W.g + 8] = x1;
      }
      W.wg_sync();
      float2 r0, r1, d0, d1;
      W.residual(r0, r1);
      st |= W.solve(r0, r1, P.refine_iters, nullptr, d0, d1) & 1;
      x0 = make_float2(x0.x + d0.x, x0.y + d0.y);
      x1 = make_float2(x1.x + d1.x, x1.y + d1.y);
    }
    // ---- final residual and outputs
    W.wg_sync();
    if (W.t == 0) {
      W.S.v[W.row0 + W.g] = x0;
      W.S.v[W.row0 + W.g + 8] = x1;
    }
    W.wg_sync();
    float2 r0, r1;
    W.residual(r0, r1);
    double nr = 0.0, nb = 0.0;
    if (W.t == 0) {
      nr = (double)r0.x * r0.x + (double)r0.y * r0.y + (double)r1.x * r1.x + (double)r1.y * r1.y;
      nb = (double)b0.x * b0.x + (double)b0.y * b0.y + (double)b1.x * b1.x + (double)b1.y * b1.y;
    }
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      nr += __shfl_xor_sync(0xffffffffu, nr, o);
      nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    if (lane == 0) {
      W.S.dred[wi * 2] = nr;
      W.S.dred[wi * 2 + 1] = nb;
    }
    int nonfinite = (W.t == 0) && !(isfinite(x0.x) && isfinite(x0.y) && isfinite(x1.x) && isfinite(x1.y));
    nonfinite = __any_sync(0xffffffffu, nonfinite);
    if (nonfinite && lane == 0) atomicOr(&W.S.flag[W.ps], 2);
    W.wg_sync();
    if (W.valid) {
      const int64_t base = W.sys * (int64_t)K;
      const int k0 = W.row0 - W.ps * K + W.g;
      if (W.t == 0) {
        P.x_hat[base + k0] = x0;
        P.x_hat[base + k0 + 8] = x1;
      }
      unsigned errs = 0;
      int bad_qam = 0;
      if (P.sym || P.bit_errors) {
        const int M = P.qam[W.sys];
        const int m = qam_sqrt(M);
        if (m == 0) {
          bad_qam = 1;
          if (P.sym && W.t == 0) {
            P.sym[base + k0] = 0;
            P.sym[base + k0 + 8] = 0;
          }
        } else if (W.t == 0) {
          const int nb2 = qam_bits_axis(m);
          const float s = (float)sqrt(2.0 * (M - 1) / 3.0);
          const int l0 = (gray(axis_level<float>(x0.x, m, s)) << nb2) | gray(axis_level<float>(x0.y, m, s));
          const int l1 = (gray(axis_level<float>(x1.x, m, s)) << nb2) | gray(axis_level<float>(x1.y, m, s));
          if (P.sym) {
            P.sym[base + k0] = (uint8_t)l0;
            P.sym[base + k0 + 8] = (uint8_t)l1;
          }
          if (P.tx) errs = __popc((unsigned)(l0 ^ P.tx[base + k0])) + __popc((unsigned)(l1 ^ P.tx[base + k0 + 8]));
        }
      }
      if (P.bit_errors && P.tx) {
        errs = __reduce_add_sync(0xffffffffu, errs);
        if (lane == 0 && errs) atomicAdd(P.bit_errors, (unsigned long long)errs);
      }
      if (lane == 0 && W.rb == 0) {
        double sr = 0.0, sb = 0.0;
        for (int w = W.ps * CgWarp<K, BF>::WS; w < (W.ps + 1) * CgWarp<K, BF>::WS; ++w) {
          sr += W.S.dred[w * 2];
          sb += W.S.dred[w * 2 + 1];
        }
        if (P.rel_res) P.rel_res[W.sys] = sb > 0.0 ? sqrt(sr / sb) : 0.0;
        if (W.S.flag[W.ps] & 2) st |= 4;
        if (bad_qam) st |= 16;
        if (P.status) P.status[W.sys] = st;
      }
    }
  }
  if (*abort && P.status) {  // systems this warpgroup did not finish
    for (; tile < pp.ntiles; tile += 2 * tstep)
      for (int i = threadIdx.x - 128 * wg; i < pp.P; i += 128)
        if (tile * pp.P + i < pp.batch) P.status[tile * pp.P + i] = 32;
  }
}

struct Smem {
  uint8_t* stages;
  tcp::Bars* bars;
  uint32_t* tmem_slot;
  volatile int* abort;
  uint8_t* cg[2];
};

template <int K, bool BF>
__global__ void __launch_bounds__(kThreads, 1) detect_tc_kernel(DetectTcParams P) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  Smem S;
  {
    const uint32_t a = tc::smem_u32(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (a & 1023u)) & 1023u);
    S.stages = base;
    S.bars = reinterpret_cast<tcp::Bars*>(base + tcp::kStages * tcp::kStageBytes);
    S.tmem_slot = reinterpret_cast<uint32_t*>(S.bars + 1);
    S.abort = reinterpret_cast<volatile int*>(S.tmem_slot + 1);
    uint8_t* cg = base + ((tcp::kStages * tcp::kStageBytes + sizeof(tcp::Bars) + 16 + 127) & ~size_t(127));
    S.cg[0] = cg;
    S.cg[1] = cg + cg_smem_bytes(K, P.L);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const tcp::Pipe& pp = P.pipe;
  for (int i = threadIdx.x; i < tcp::kStages * tcp::kStageBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(S.stages)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < tcp::kStages; ++s) {
      tc::mbar_init(&S.bars->full[s], kConv);
      tc::mbar_init(&S.bars->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&S.bars->acc_full[b], 1);
      tc::mbar_init(&S.bars->acc_empty[b], 1);
    }
    tc::mbar_init(&S.bars->done, 1);
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
    if (lane == 0) tcp::mma_role(pp, S.stages, *S.bars, S.abort, tmem, tile0, tstep);
    __syncwarp();
  } else if (warp >= kConv0) {
    tcp::converter_role<kConv>(pp, S.stages, *S.bars, S.abort, tile0, tstep, warp - kConv0, lane);
  } else {
    const int wg = warp >> 2;
    cg_role<K, BF>(P, *S.bars, S.abort, tmem, S.cg[wg], wg, tile0, tstep);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * tcp::kAccCols);
  }
}

template <int K, bool BF>
cudaError_t launch_k(const DetectTcParams& P, int num_sms, cudaStream_t stream) {
  const size_t smem = detect_tc_smem_bytes(K, P.L);
  cudaError_t e =
      cudaFuncSetAttribute(detect_tc_kernel<K, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = P.pipe.ntiles < num_sms ? P.pipe.ntiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  detect_tc_kernel<K, BF><<<(unsigned)grid, kThreads, smem, stream>>>(P);
  return cudaGetLastError();
}

}  // namespace

bool detect_tc_supported(int K, int L) {
  return (K == 16 || K == 32 || K == 64) && L >= 0 && L <= 16 && (L == 0 || 16 % L == 0);
}

size_t detect_tc_smem_bytes(int K, int L) {
  size_t s = 1024 + ((tcp::kStages * tcp::kStageBytes + sizeof(tcp::Bars) + 16 + 127) & ~size_t(127)) +
             2 * cg_smem_bytes(K, L);
  return s < 120 * 1024 ? 120 * 1024 : s;
}

cudaError_t launch_detect_tc(const DetectTcParams& P, int num_sms, int mv_bf16, cudaStream_t stream) {
  const int K = P.pipe.K;
  if (mv_bf16) {
    if (K == 64) return launch_k<64, true>(P, num_sms, stream);
    if (K == 32) return launch_k<32, true>(P, num_sms, stream);
    if (K == 16) return launch_k<16, true>(P, num_sms, stream);
  } else {
    if (K == 64) return launch_k<64, false>(P, num_sms, stream);
    if (K == 32) return launch_k<32, false>(P, num_sms, stream);
    if (K == 16) return launch_k<16, false>(P, num_sms, stream);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fpcg
