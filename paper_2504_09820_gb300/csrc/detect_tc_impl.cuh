#pragma once
// Fused tensor-core detector (kernel templates; instantiated per K by
// detect_tc_k{16,32,64}.cu): the whole path for K in {16, 32, 64} in one
// persistent launch (one CTA per SM).
//
//   warps 0-3    CG warpgroup 0: tiles 0, 2, 4, ... of this CTA (TMEM buffer 0)
//   warps 4-7    CG warpgroup 1: tiles 1, 3, 5, ...             (TMEM buffer 1)
//   warps 8-13   converters: FP32 stages -> bf16/fp16 swizzled operand stages
//   warp 14      TMA producer of the FP32 stages
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
//   * Algorithm 2 / 3: the first warp of each system holds its vectors (one or
//     two rows per lane): inner products by warp shuffles (u_IP rounding),
//     z = M_d r by shuffles within the block's lanes, updates by FMA at
//     u_W = fp32, p handed to the matvec warps as packed mma B fragments --
//     two warpgroup barriers per iteration;
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
constexpr int kProdWarp = 14;
constexpr int kConv0 = 8;
constexpr int kConv = 6;  // converter warps 8-13

// Per-warpgroup shared memory (rows are the 64 rows of a tile: row = ps*K + k).
struct CgSmem {
  float2* A;      // [64][K+1] fp32 Gram (+ sigma^2)
  float2* b;      // [64]
  float2* W;      // [64] varpi = A p from the mma warps
  float2* X;      // [64] x for the residual
  float2* R;      // [64] residual b - A x
  float2* Md;     // [64][L+1] block-Jacobi inverse rows (padded)
  uint32_t* Pk;   // [64] p packed as the mma B fragments (bf16/fp16 pairs)
  int* flag;      // [4]
};

__device__ inline CgSmem cg_carve(uint8_t* base, int K, int L) {
  CgSmem s;
  uint8_t* p = base;
  s.A = (float2*)p;
  p += sizeof(float2) * 64 * (K + 1);
  s.b = (float2*)p;
  p += sizeof(float2) * 64;
  s.W = (float2*)p;
  p += sizeof(float2) * 64;
  s.X = (float2*)p;
  p += sizeof(float2) * 64;
  s.R = (float2*)p;
  p += sizeof(float2) * 64;
  s.Md = (float2*)p;
  p += sizeof(float2) * 64 * ((L > 0 ? L : 1) + 1);
  s.Pk = (uint32_t*)p;
  p += sizeof(uint32_t) * 64;
  s.flag = (int*)p;
  return s;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CG warpgroup working on a tile of P = 64/K systems.  Every warp owns 16
// rows of one system for the matvec (mma.sync) and the residual; the first
// warp of each system (the "vector warp") owns the system's vectors, one row
// per lane (two for K = 64), and does all of Algorithm 2/3's vector work.
template <int K, bool BF, int LT>
struct CgWarp {
  static constexpr int KT = K / 16;          // k-tiles of the matvec
  static constexpr int WS = K / 16;          // warps per system
  static constexpr int E = K == 64 ? 2 : 1;  // rows per lane in the vector warp
  static constexpr int LD = LT + 1;          // padded row length of M_d

  const DetectTcParams& P;
  CgSmem S;
  int wi, lane, g, t, ps, rb, row0, bar_id;
  bool vec;                                  // this warp is its system's vector warp
  int64_t sys;
  bool valid;
  uint32_t afr[2][KT][4];                    // [Re A; Im A] fragments of the warp's 16 rows

  __device__ CgWarp(const DetectTcParams& P_, CgSmem S_, int wi_, int lane_, int bar_id_)
      : P(P_), S(S_), wi(wi_), lane(lane_), bar_id(bar_id_) {
    g = lane >> 2;
    t = lane & 3;
    ps = wi / WS;
    rb = wi % WS;
    row0 = ps * K + 16 * rb;
    vec = rb == 0;
  }

  __device__ __forceinline__ void wg_sync() { tc::bar_sync(bar_id, 128); }
  __device__ __forceinline__ uint32_t pk(float a, float b) { return tcp::pack2(a, b, BF ? 1 : 0); }
  __device__ __forceinline__ float rip(float v) { return round_to(v, P.ip); }
  // row (tile numbering) of element e of this lane in the vector warp, and whether it exists
  __device__ __forceinline__ int vrow(int e) const { return ps * K + lane + 32 * e; }
  __device__ __forceinline__ bool vact() const { return lane < K; }

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

  // All warps: W[rows of this warp] = A p, p taken from the packed fragments.
  __device__ __forceinline__ void matvec_rows() {
    const uint32_t* pk_sys = S.Pk + ps * 16 * KT;
    float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      uint32_t b0 = 0u, b1 = 0u;
      if (g < 2) {
        const uint2 w = *reinterpret_cast<const uint2*>(pk_sys + ((kt * 2 + g) * 4 + t) * 2);
        b0 = w.x;
        b1 = w.y;
      }
      if (BF) {
        tc::mma_m16n8k16_bf16(cr, afr[0][kt], b0, b1);
        tc::mma_m16n8k16_bf16(ci, afr[1][kt], b0, b1);
      } else {
        tc::mma_m16n8k16_f16(cr, afr[0][kt], b0, b1);
        tc::mma_m16n8k16_f16(ci, afr[1][kt], b0, b1);
      }
    }
    if (t == 0) {  // rows g / g+8: (Re A pr - Im A pi) + i (Re A pi + Im A pr)
      S.W[row0 + g] = make_float2(cr[0] - ci[1], cr[1] + ci[0]);
      S.W[row0 + g + 8] = make_float2(cr[2] - ci[3], cr[3] + ci[2]);
    }
  }

  // Vector warp: store p (one or two rows per lane) as mma B fragments:
  // word ((kt*2 + comp)*4 + tt)*2 + h holds rows 16kt + 8h + 2tt, +1.
  __device__ __forceinline__ void pack_p(const float2 (&p)[E]) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const float nx = __shfl_down_sync(0xffffffffu, p[e].x, 1);
      const float ny = __shfl_down_sync(0xffffffffu, p[e].y, 1);
      const int rl = lane + 32 * e;
      if (vact() && (rl & 1) == 0) {
        const int kt = rl >> 4, j = rl & 15, tt = (j & 7) >> 1, h = j >> 3;
        uint32_t* base = S.Pk + ps * 16 * KT;
        base[((kt * 2 + 0) * 4 + tt) * 2 + h] = pk(p[e].x, nx);
        base[((kt * 2 + 1) * 4 + tt) * 2 + h] = pk(p[e].y, ny);
      }
    }
  }

  // Vector warp: z = M_d r (z = r without a preconditioner); the L rows of a
  // block sit in L consecutive lanes.
  __device__ __forceinline__ void precond(const float2 (&r)[E], float2 (&z)[E]) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if constexpr (LT == 0) {
        z[e] = r[e];
      } else {
        const int first = lane & ~(LT - 1);
        const float2* mrow = S.Md + (vact() ? vrow(e) : 0) * LD;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < LT; ++j) {
          const float qx = __shfl_sync(0xffffffffu, r[e].x, first + j);
          const float qy = __shfl_sync(0xffffffffu, r[e].y, first + j);
          const float2 m = vact() ? mrow[j] : make_float2(0.f, 0.f);
          acc.x = fmaf(m.x, qx, fmaf(-m.y, qy, acc.x));
          acc.y = fmaf(m.x, qy, fmaf(m.y, qx, acc.y));
        }
        z[e] = acc;
      }
    }
  }

  // two sums over the warp at once (interleaved shuffles)
  __device__ __forceinline__ void dot2_re(const float2 (&a)[E], const float2 (&b)[E], const float2 (&c)[E],
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

  __device__ __forceinline__ float dot_re(const float2 (&a)[E], const float2 (&b)[E]) {
    float s = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) s += a[e].x * b[e].x + a[e].y * b[e].y;
    return warp_sum_f(vact() ? s : 0.f);
  }

  // Algorithm 2 (L == 0) / Algorithm 3 (L > 0) from x0 = 0 on the right-hand
  // side rhs[] (shared memory, tile rows).  Every warp of the warpgroup calls it;
  // the vector warps return x in xo and their status bits.
  __device__ int solve(const float2* rhs, int iters, float* hist, float2 (&xo)[E]) {
    int st = 0;
    build_fragments();  // live only inside the solve (the residual between solves needs the registers)
    float2 x[E], r[E], p[E], z[E];
    float rho = 0.f;
    bool live = true;
    if (vec) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        x[e] = make_float2(0.f, 0.f);
        r[e] = vact() ? rhs[vrow(e)] : make_float2(0.f, 0.f);
      }
      precond(r, z);
#pragma unroll
      for (int e = 0; e < E; ++e) p[e] = z[e];
      float rz, rr;
      dot2_re(r, z, r, r, rz, rr);
      rho = rip(rz);
      if (hist && lane == 0) hist[0] = sqrtf(rr);
      pack_p(p);
    }
    for (int it = 0; it < iters; ++it) {
      wg_sync();  // packed p visible
      matvec_rows();
      wg_sync();  // varpi visible
      if (!vec) continue;
      float2 w[E];
#pragma unroll
      for (int e = 0; e < E; ++e) w[e] = vact() ? S.W[vrow(e)] : make_float2(0.f, 0.f);
      float phi, rp;
      dot2_re(p, w, r, p, phi, rp);
      phi = rip(phi);
      const float rho_prev = (LT > 0 && P.alpha_num == 0) ? rip(rp) : rho;
      if (live) {
        if (rho_prev == 0.f) {
          st |= 2;
          live = false;
        } else if (!(phi > 0.f) || !isfinite(phi) || !isfinite(rho_prev)) {
          st |= 1;
          live = false;
        }
      }
      if (live) {
        const float alpha = rho_prev / phi;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          x[e] = make_float2(fmaf(alpha, p[e].x, x[e].x), fmaf(alpha, p[e].y, x[e].y));
          r[e] = make_float2(fmaf(-alpha, w[e].x, r[e].x), fmaf(-alpha, w[e].y, r[e].y));
        }
        precond(r, z);
        float rz, rr;
        dot2_re(r, z, r, r, rz, rr);
        const float rho_new = rip(rz);
        const float beta = rho_new / rho_prev;
#pragma unroll
        for (int e = 0; e < E; ++e) p[e] = make_float2(fmaf(beta, p[e].x, z[e].x), fmaf(beta, p[e].y, z[e].y));
        rho = rho_new;
        if (hist && lane == 0) hist[it + 1] = sqrtf(rr);
        pack_p(p);
      } else if (hist && lane == 0) {
        hist[it + 1] = hist[it];
      }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) xo[e] = x[e];
    return st;
  }

  // All warps: R[rows of this warp] = b - A X (X in shared memory) with fp32
  // sums: lane handles row row0 + (lane & 15) and half of the columns.
  __device__ void residual() {
    const int rl = lane & 15, half = lane >> 4;
    const float2* arow = S.A + (row0 + rl) * (K + 1) + half * (K / 2);
    const float2* xs = S.X + ps * K + half * (K / 2);
    float2 s = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int l = 0; l < K / 2; ++l) {
      const float2 a = arow[l], x = xs[l];
      s.x = fmaf(a.x, x.x, fmaf(-a.y, x.y, s.x));
      s.y = fmaf(a.x, x.y, fmaf(a.y, x.x, s.y));
    }
    s.x += __shfl_xor_sync(0xffffffffu, s.x, 16);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, 16);
    if (half == 0) {
      const float2 bb = S.b[row0 + rl];
      S.R[row0 + rl] = make_float2(bb.x - s.x, bb.y - s.y);
    }
  }

  // All warps: Gauss-Jordan inversion (in place, no pivoting: the blocks are
  // Hermitian positive definite) of the warp's own L x L diagonal blocks in
  // S.Md (rows padded to L+1); lane (block, j) owns column j of its block.
  // Returns nonzero if a pivot was not positive.
  __device__ int bj_setup() {
    if constexpr (LT == 0) {
      return 0;
    } else {
      int fail = 0;
      const int blk = lane / LT, j = lane % LT;
      const bool on = lane < 16;
      const int R0 = row0 + blk * LT;  // first row of the block (tile numbering)
      const int kb = R0 - ps * K;      // its first column (system numbering)
      float2* M = S.Md + R0 * LD;      // M[i*LD + c] = block entry (i, c)
      if (on)
#pragma unroll
        for (int i = 0; i < LT; ++i) M[i * LD + j] = S.A[(R0 + i) * (K + 1) + kb + j];
      __syncwarp();
#pragma unroll
      for (int pv = 0; pv < LT; ++pv) {
        const float2 piv = on ? M[pv * LD + pv] : make_float2(1.f, 0.f);
        if (on && !(piv.x > 0.f && isfinite(piv.x))) fail = 1;
        const float den = piv.x * piv.x + piv.y * piv.y;
        const float2 dinv = make_float2(piv.x / den, -piv.y / den);
        float2 prow = make_float2(0.f, 0.f);
        if (on && j != pv) prow = cmul(M[pv * LD + j], dinv);  // scaled pivot row
        float2 f[LT];
#pragma unroll
        for (int i = 0; i < LT; ++i) f[i] = on ? M[i * LD + pv] : make_float2(0.f, 0.f);  // pivot column
        __syncwarp();
        if (on) {
          if (j != pv) {
#pragma unroll
            for (int i = 0; i < LT; ++i) {
              if (i == pv) continue;
              float2 v = M[i * LD + j];
              const float2 fp = cmul(f[i], prow);
              v.x -= fp.x;
              v.y -= fp.y;
              M[i * LD + j] = v;
            }
            M[pv * LD + j] = prow;
          } else {
#pragma unroll
            for (int i = 0; i < LT; ++i) {
              if (i == pv) continue;
              const float2 v = cmul(f[i], dinv);
              M[i * LD + pv] = make_float2(-v.x, -v.y);
            }
            M[pv * LD + pv] = dinv;
          }
        }
        __syncwarp();
      }
      return __any_sync(0xffffffffu, fail);
    }
  }
};

template <int K, bool BF, int LT>
__device__ void cg_role(const DetectTcParams& P, tcp::Bars& B, volatile int* abort, uint32_t tmem, uint8_t* cg_base,
                        int wg, int64_t tile0, int64_t tstep) {
  using CW = CgWarp<K, BF, LT>;
  constexpr int E = CW::E;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wi = warp - 4 * wg;  // warp within the warpgroup == TMEM lane quadrant
  CW W(P, cg_carve(cg_base, K, P.L), wi, lane, 1 + wg);
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
    if (lane == 0 && W.vec) W.S.flag[W.ps] = 0;
    W.wg_sync();
    if (wi == 0 && lane == 0) tc::mbar_arrive(&B.acc_empty[wg]);
    W.sys = tile * pp.P + W.ps;
    W.valid = W.sys < pp.batch;
    int st = 0;
    // ---- block-Jacobi setup (every warp inverts its own blocks)
    if (W.bj_setup() && lane == 0) atomicOr(&W.S.flag[W.ps], 1);
    W.wg_sync();
    if (LT > 0 && W.S.flag[W.ps]) {  // fall back to M_d = I for this system
      if (W.vec) st |= 8;
      if (lane < 16)
        for (int i = 0; i < LT; ++i) {
          const int R = W.row0 + lane;
          W.S.Md[R * (LT + 1) + i] = make_float2((R - W.ps * K) % LT == i ? 1.f : 0.f, 0.f);
        }
    }
    W.wg_sync();
    // ---- main solve
    float* hist = (P.res_hist && W.valid && W.vec) ? P.res_hist + W.sys * (int64_t)(P.iters + 1) : nullptr;
    float2 x[E];
    st |= W.solve(W.S.b, P.iters, hist, x);
    // ---- refinement: x += solve(b - A x)
    for (int rs = 0; rs < P.refine_steps; ++rs) {
      if (W.vec && W.vact())
#pragma unroll
        for (int e = 0; e < E; ++e) W.S.X[W.vrow(e)] = x[e];
      W.wg_sync();
      W.residual();
      W.wg_sync();
      float2 d[E];
      st |= W.solve(W.S.R, P.refine_iters, nullptr, d) & 1;
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = make_float2(x[e].x + d[e].x, x[e].y + d[e].y);
    }
    // ---- final residual and outputs
    if (W.vec && W.vact())
#pragma unroll
      for (int e = 0; e < E; ++e) W.S.X[W.vrow(e)] = x[e];
    W.wg_sync();
    W.residual();
    W.wg_sync();
    if (W.vec && W.valid) {
      double nr = 0.0, nb = 0.0;
      int nonfinite = 0;
      unsigned errs = 0;
      int bad_qam = 0;
      const int64_t base = W.sys * (int64_t)K;
      const int M = (P.sym || P.bit_errors) ? P.qam[W.sys] : 0;
      const int m = qam_sqrt(M);
      if ((P.sym || P.bit_errors) && m == 0) bad_qam = 1;
      if (W.vact()) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const float2 rr = W.S.R[W.vrow(e)], bb = W.S.b[W.vrow(e)];
          nr += (double)rr.x * rr.x + (double)rr.y * rr.y;
          nb += (double)bb.x * bb.x + (double)bb.y * bb.y;
          const int k = lane + 32 * e;
          if (!(isfinite(x[e].x) && isfinite(x[e].y))) nonfinite = 1;
          P.x_hat[base + k] = x[e];
          if (P.sym || P.bit_errors) {
            int lab = 0;
            if (m) {
              const int nb2 = qam_bits_axis(m);
              const float sc = (float)sqrt(2.0 * (M - 1) / 3.0);
              lab = (gray(axis_level<float>(x[e].x, m, sc)) << nb2) | gray(axis_level<float>(x[e].y, m, sc));
            }
            if (P.sym) P.sym[base + k] = (uint8_t)lab;
            if (P.tx && m) errs += __popc((unsigned)(lab ^ P.tx[base + k]));
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
        if (P.rel_res) P.rel_res[W.sys] = nb > 0.0 ? sqrt(nr / nb) : 0.0;
        if (nonfinite) st |= 4;
        if (bad_qam) st |= 16;
        if (P.status) P.status[W.sys] = st;
      }
    }
    W.wg_sync();  // A, b, R are read until here; the next drain overwrites them
  }
  if (*abort && P.status) {  // systems this warpgroup did not finish
    for (; tile < pp.ntiles; tile += 2 * tstep)
      for (int i = threadIdx.x - 128 * wg; i < pp.P; i += 128)
        if (tile * pp.P + i < pp.batch) P.status[tile * pp.P + i] = 32;
  }
}

struct Smem {
  uint8_t* pipe;
  tcp::Bars* bars;
  uint32_t* tmem_slot;
  volatile int* abort;
  uint8_t* cg[2];
};

template <int K, bool BF, int LT>
__global__ void __launch_bounds__(kThreads, 1) detect_tc_kernel(const __grid_constant__ DetectTcParams P) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  Smem S;
  {
    const uint32_t a = tc::smem_u32(smem_raw);
    uint8_t* base = smem_raw + ((1024u - (a & 1023u)) & 1023u);
    S.pipe = base;
    S.bars = reinterpret_cast<tcp::Bars*>(base + tcp::kPipeBytes);
    S.tmem_slot = reinterpret_cast<uint32_t*>(S.bars + 1);
    S.abort = reinterpret_cast<volatile int*>(S.tmem_slot + 1);
    uint8_t* cg = base + cg_region_offset();
    S.cg[0] = cg;
    S.cg[1] = cg + cg_smem_bytes(K, P.L);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const tcp::Pipe& pp = P.pipe;
  for (int i = threadIdx.x; i < tcp::kStages * tcp::kStageBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(tcp::stage16(S.pipe, 0))[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    tcp::init_bars(*S.bars, kConv);
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
    if (lane == 0) tcp::producer_role(pp, S.pipe, *S.bars, S.abort, tile0, tstep);
    __syncwarp();
  } else if (warp >= kConv0) {
    tcp::converter_role<kConv>(pp, S.pipe, *S.bars, S.abort, tile0, tstep, warp - kConv0, lane);
  } else {
    const int wg = warp >> 2;
    cg_role<K, BF, LT>(P, *S.bars, S.abort, tmem, S.cg[wg], wg, tile0, tstep);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * tcp::kAccCols);
  }
}

template <int K, bool BF, int LT>
cudaError_t launch_k(const DetectTcParams& P, int num_sms, cudaStream_t stream) {
  const size_t smem = detect_tc_smem_bytes(K, P.L);
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
