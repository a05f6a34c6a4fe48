// Generic SIMT detector: one CTA (256 threads) per system, every step of the
// path in one launch.  It covers every size (1 <= K <= 128, any N >= K) and
// every precision mode, and is the plain fp32 CG comparator of the
// tensor-core path.
//
// Per system, in order (each step names the passage it implements):
//   1. Gram + matched filter (Section II, eq. inversion): H and y are staged
//      through shared memory in chunks of antennas, rounded to u_gram on the
//      way in; each thread accumulates one 4x4 tile of the upper triangle of
//      H^H H (fp32 or fp64 FMAs: products of bf16/fp16 values are exact, so
//      this is the tensor-core rounding model), threads k < K accumulate b_k.
//      The lower triangle is mirrored, Im(A_kk) = 0, sigma^2 added once.
//   2. Block-Jacobi inverse (eq. pre_BJ): one warp per L x L diagonal block,
//      in-place Gauss-Jordan without pivoting (the blocks are Hermitian
//      positive definite), lane j owning column j.
//   3. FP-CG / FP-BJ-CG (Algorithms 2 and 3): A p with A and p rounded to
//      u_MV (e4m3: per-block power-of-two scales) and fp32 sums; inner products
//      summed at fp32 and rounded to u_IP; updates by FMA at u_W.
//   4. Refinement: r = b - A x (A rounded to u_MV with fp32 sums, or the Gram
//      matrix with compensated double-fp32 / fp64 sums), a correction solve
//      with step 3, x += d.
//   5. rel_res = ||b - A x|| / ||b||, the Gray-QAM decision, bit errors.
//
// The fp64 mode for K > 64 (IMP = 1): A = H^H H + sigma^2 I in fp64 does not
// fit in shared memory (264 KB at K = 128), so it is never formed.  Every
// product with A is H^H (H v) + sigma^2 v in fp64 straight from H in global
// memory (antennas in chunks of kIC), the block-Jacobi blocks are formed from
// H, and b = H^H y likewise.  The same operator in exact arithmetic; the
// rounding differs at the level of fp64 sums.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "detect_simt.cuh"

namespace fpcg {

namespace {

constexpr int NT = 256;   // threads per CTA
constexpr int TS = 4;     // Gram tile edge
constexpr int kIC = 256;  // antennas per chunk of an implicit (IMP) product with A

template <typename T>
struct Smem {
  cplx<T>* A;     // K x (K+1), row-major, padded
  cplx<T>* Hs;    // CH x (K+1) staging of H (Gram phase)
  cplx<T>* ys;    // CH
  cplx<T>* b;
  cplx<T>* x;
  cplx<T>* r;
  cplx<T>* p;
  cplx<T>* z;
  cplx<T>* w;     // varpi = A p
  cplx<T>* pq;    // p rounded for the matvec
  cplx<T>* Md;    // K x L block inverses (row k holds row k of its block)
  float* sA;      // K x NB e4m3 scales of A
  float* sp;      // NB e4m3 scales of p
  T* red;         // reduction scratch, 4 * 32
  int* flags;     // 4 ints
};

template <typename T>
__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

template <typename T>
__host__ __device__ inline int chunk_rows() { return sizeof(T) == 8 ? 16 : 32; }

// IMP: no A; Hs only as the refinement's scratch (2K), ys as the chunk of H v (kIC).
template <typename T>
__host__ __device__ inline size_t smem_bytes(int K, int L, int mv, bool imp = false) {
  const int CH = chunk_rows<T>();
  const int NB = (2 * K + 31) / 32;
  size_t s = 0;
  s += align16<T>(sizeof(cplx<T>) * (imp ? 0 : (size_t)K * (K + 1)));
  s += align16<T>(sizeof(cplx<T>) * (imp ? (size_t)2 * K : (size_t)CH * (K + 1)));
  s += align16<T>(sizeof(cplx<T>) * (size_t)(imp ? kIC : CH));
  s += 7 * align16<T>(sizeof(cplx<T>) * (size_t)K);
  s += align16<T>(sizeof(cplx<T>) * (size_t)K * (L > 0 ? L : 1));
  s += align16<T>(sizeof(float) * (size_t)K * NB);
  s += align16<T>(sizeof(float) * (size_t)NB);
  s += align16<T>(sizeof(T) * 4 * 32);
  s += align16<T>(sizeof(int) * 4);
  (void)mv;
  return s;
}

template <typename T>
__device__ inline Smem<T> carve(unsigned char* base, int K, int L, bool imp = false) {
  const int CH = chunk_rows<T>();
  const int NB = (2 * K + 31) / 32;
  Smem<T> s;
  size_t o = 0;
  auto take = [&](size_t bytes) { unsigned char* ptr = base + o; o += align16<T>(bytes); return ptr; };
  s.A = (cplx<T>*)take(sizeof(cplx<T>) * (imp ? 0 : (size_t)K * (K + 1)));
  s.Hs = (cplx<T>*)take(sizeof(cplx<T>) * (imp ? (size_t)2 * K : (size_t)CH * (K + 1)));
  s.ys = (cplx<T>*)take(sizeof(cplx<T>) * (size_t)(imp ? kIC : CH));
  s.b = (cplx<T>*)take(sizeof(cplx<T>) * K);
  s.x = (cplx<T>*)take(sizeof(cplx<T>) * K);
  s.r = (cplx<T>*)take(sizeof(cplx<T>) * K);
  s.p = (cplx<T>*)take(sizeof(cplx<T>) * K);
  s.z = (cplx<T>*)take(sizeof(cplx<T>) * K);
  s.w = (cplx<T>*)take(sizeof(cplx<T>) * K);
  s.pq = (cplx<T>*)take(sizeof(cplx<T>) * K);
  s.Md = (cplx<T>*)take(sizeof(cplx<T>) * (size_t)K * (L > 0 ? L : 1));
  s.sA = (float*)take(sizeof(float) * (size_t)K * NB);
  s.sp = (float*)take(sizeof(float) * NB);
  s.red = (T*)take(sizeof(T) * 4 * 32);
  s.flags = (int*)take(sizeof(int) * 4);
  return s;
}

// Round a working-precision value to the Gram input format.
template <typename T>
__device__ inline T round_gram(float v, int gram) {
  if (sizeof(T) == 8) return (T)v;
  return (T)round_to(v, gram);
}

// Sum of `v` over the CTA; every thread gets the result.  Uses red[0..31]
// and one extra slot; two barriers.
template <typename T>
__device__ inline T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();  // red may still be read by a previous call
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = (lane < NT / 32) ? red[lane] : T(0);
  t = warp_sum(t);
  return t;
}

// Two sums at once (fewer barriers).
template <typename T>
__device__ inline void block_sum2(T& a, T& b, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if (lane == 0) {
    red[wid] = a;
    red[32 + wid] = b;
  }
  __syncthreads();
  T ta = (lane < NT / 32) ? red[lane] : T(0);
  T tb = (lane < NT / 32) ? red[32 + lane] : T(0);
  a = warp_sum(ta);
  b = warp_sum(tb);
}

// Round an fp32 inner-product result to u_IP.
template <typename T>
__device__ inline T round_ip(T v, int ip) {
  if (sizeof(T) == 8) return v;
  return (T)round_to((float)v, ip);
}

// ---------------------------------------------------------------------------
// Step 1: Gram matrix and matched filter.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void gram_phase(const SimtParams& P, const Smem<T>& S, int64_t sys) {
  const int K = P.K, N = P.N, CH = chunk_rows<T>();
  const int AS = K + 1, HS = K + 1;
  const int nt = (K + TS - 1) / TS;
  const int ntiles = nt * (nt + 1) / 2;
  const int rounds = (ntiles + NT - 1) / NT;
  const float2* Hg = P.H + (size_t)sys * K * N;
  const float2* yg = P.y + (size_t)sys * N;
  const int tid = threadIdx.x;

  for (int round = 0; round < rounds; ++round) {
    const int t = tid + round * NT;
    int ti = 0, tj = 0;
    const bool has_tile = t < ntiles;
    if (has_tile) {  // column-wise enumeration of the upper triangle: t -> (ti <= tj)
      tj = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
      while ((tj + 1) * (tj + 2) / 2 <= t) ++tj;
      while (tj * (tj + 1) / 2 > t) --tj;
      ti = t - tj * (tj + 1) / 2;
    }
    T accr[TS][TS], acci[TS][TS];
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
      for (int c = 0; c < TS; ++c) accr[a][c] = acci[a][c] = T(0);
    T bre = T(0), bim = T(0);
    const bool do_b = (round == 0) && tid < K;

    for (int n0 = 0; n0 < N; n0 += CH) {
      const int rows = min(CH, N - n0);
      __syncthreads();
      for (int idx = tid; idx < CH * K; idx += NT) {
        const int k = idx / CH, i = idx % CH;
        cplx<T> v;
        if (i < rows) {
          float2 h = Hg[(size_t)k * N + n0 + i];
          v.re = round_gram<T>(h.x, P.gram);
          v.im = round_gram<T>(h.y, P.gram);
        } else {
          v.re = v.im = T(0);
        }
        S.Hs[i * HS + k] = v;
      }
      if (round == 0) {
        for (int i = tid; i < CH; i += NT) {
          cplx<T> v;
          if (i < rows) {
            float2 yy = yg[n0 + i];
            v.re = round_gram<T>(yy.x, P.gram);
            v.im = round_gram<T>(yy.y, P.gram);
          } else {
            v.re = v.im = T(0);
          }
          S.ys[i] = v;
        }
      }
      __syncthreads();
      if (has_tile) {
        const int k0 = ti * TS, l0 = tj * TS;
        for (int i = 0; i < rows; ++i) {
          cplx<T> hk[TS], hl[TS];
#pragma unroll
          for (int a = 0; a < TS; ++a) {
            hk[a] = (k0 + a < K) ? S.Hs[i * HS + k0 + a] : cplx<T>{T(0), T(0)};
            hl[a] = (l0 + a < K) ? S.Hs[i * HS + l0 + a] : cplx<T>{T(0), T(0)};
          }
#pragma unroll
          for (int a = 0; a < TS; ++a)
#pragma unroll
            for (int c = 0; c < TS; ++c) {
              // conj(h_k) * h_l
              accr[a][c] = fma(hk[a].re, hl[c].re, fma(hk[a].im, hl[c].im, accr[a][c]));
              acci[a][c] = fma(hk[a].re, hl[c].im, fma(-hk[a].im, hl[c].re, acci[a][c]));
            }
        }
      }
      if (do_b) {
        for (int i = 0; i < rows; ++i) {
          cplx<T> h = S.Hs[i * HS + tid], yy = S.ys[i];
          bre = fma(h.re, yy.re, fma(h.im, yy.im, bre));
          bim = fma(h.re, yy.im, fma(-h.im, yy.re, bim));
        }
      }
    }
    if (has_tile) {
      const int k0 = ti * TS, l0 = tj * TS;
#pragma unroll
      for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int c = 0; c < TS; ++c) {
          const int k = k0 + a, l = l0 + c;
          if (k < K && l < K && k <= l) {
            S.A[k * AS + l] = cplx<T>{accr[a][c], acci[a][c]};
            S.A[l * AS + k] = cplx<T>{accr[a][c], -acci[a][c]};
          }
        }
    }
    if (do_b) S.b[tid] = cplx<T>{bre, bim};
  }
  __syncthreads();
  const T s2 = (T)P.sigma2[sys];  // fl32(sigma^2) in the fp32 modes
  for (int k = tid; k < K; k += NT) {
    S.A[k * AS + k].re = S.A[k * AS + k].re + s2;
    S.A[k * AS + k].im = T(0);
  }
  __syncthreads();
}

// Load A and b given directly (fpcg_solve_gram).
template <typename T>
__device__ void load_gram(const SimtParams& P, const Smem<T>& S, int64_t sys) {
  const int K = P.K, AS = K + 1;
  const cplx<T>* Ag = (const cplx<T>*)P.Ain + (size_t)sys * K * K;
  const cplx<T>* bg = (const cplx<T>*)P.bin + (size_t)sys * K;
  for (int idx = threadIdx.x; idx < K * K; idx += NT) S.A[(idx / K) * AS + idx % K] = Ag[idx];
  for (int k = threadIdx.x; k < K; k += NT) S.b[k] = bg[k];
  __syncthreads();
}

// Shared-Gram mode: A (with sigma^2 I) of the system's group from Ain, and its
// own matched filter b = fl(H)^H fl(y) (eq. inversion) from the group's H and
// the system's y, rounded like the Gram.  One warp per row k of b, lanes over
// the antennas, shuffle reduction.  Returns false for an index out of range.
template <typename T>
__device__ bool load_shared(const SimtParams& P, const Smem<T>& S, int64_t sys) {
  const int K = P.K, N = P.N, AS = K + 1;
  int64_t g;
  if (P.a_map) {
    g = P.a_map[sys];
  } else {  // largest g with group_start[g] <= sys
    int64_t lo = 0, hi = P.n_shared;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (P.group_start[mid] <= sys) lo = mid;
      else hi = mid;
    }
    g = lo;
  }
  if (g < 0 || g >= P.n_shared) return false;
  const cplx<T>* Ag = (const cplx<T>*)P.Ain + (size_t)g * K * K;
  for (int idx = threadIdx.x; idx < K * K; idx += NT) S.A[(idx / K) * AS + idx % K] = Ag[idx];
  const float2* Hg = P.H + (size_t)g * K * N;
  const float2* yg = P.y + (size_t)sys * N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < K; k += NT / 32) {
    T re = T(0), im = T(0);
    for (int n = lane; n < N; n += 32) {
      const float2 h = Hg[(size_t)k * N + n], yy = yg[n];
      const T hr = round_gram<T>(h.x, P.gram), hi = round_gram<T>(h.y, P.gram);
      const T yr = round_gram<T>(yy.x, P.gram), yi = round_gram<T>(yy.y, P.gram);
      re = fma(hr, yr, fma(hi, yi, re));  // conj(h_k) y
      im = fma(hr, yi, fma(-hi, yr, im));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) S.b[k] = cplx<T>{re, im};
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// Step 2: block-Jacobi inverse, in-place Gauss-Jordan per diagonal block.
// Returns nonzero (in every thread) if some pivot was not positive.
// ---------------------------------------------------------------------------
template <typename T>
__device__ int bj_phase(const SimtParams& P, const Smem<T>& S, bool imp = false) {
  const int K = P.K, L = P.L, AS = K + 1;
  const int d = K / L;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) S.flags[0] = 0;
  if (!imp)  // IMP: the blocks were formed from H (gram_phase_imp)
    for (int idx = threadIdx.x; idx < K * L; idx += NT) {
      const int k = idx / L, j = idx % L;
      const int blk = k / L;
      S.Md[idx] = S.A[k * AS + blk * L + j];
    }
  __syncthreads();
  for (int blk = wid; blk < d; blk += NT / 32) {
    cplx<T>* M = S.Md + (size_t)blk * L * L;  // M[i*L + j]
    int fail = 0;
    for (int pv = 0; pv < L; ++pv) {
      cplx<T> piv = M[pv * L + pv];
      if (!(piv.re > T(0)) || !isfinite((double)piv.re)) fail = 1;
      // 1 / piv (complex)
      T den = piv.re * piv.re + piv.im * piv.im;
      cplx<T> dinv{piv.re / den, -piv.im / den};
      __syncwarp();
      if (lane < L && lane != pv) {  // scale the pivot row
        cplx<T> v = M[pv * L + lane];
        M[pv * L + lane] = cplx<T>{v.re * dinv.re - v.im * dinv.im, v.re * dinv.im + v.im * dinv.re};
      }
      __syncwarp();
      if (lane < L && lane != pv) {  // eliminate column `lane` of every other row
        const cplx<T> pr = M[pv * L + lane];
        for (int i = 0; i < L; ++i) {
          if (i == pv) continue;
          const cplx<T> f = M[i * L + pv];
          cplx<T> v = M[i * L + lane];
          v.re = v.re - (f.re * pr.re - f.im * pr.im);
          v.im = v.im - (f.re * pr.im + f.im * pr.re);
          M[i * L + lane] = v;
        }
      }
      __syncwarp();
      if (lane < L) {  // pivot column
        if (lane == pv) {
          M[pv * L + pv] = dinv;
        } else {
          cplx<T> v = M[lane * L + pv];
          M[lane * L + pv] = cplx<T>{-(v.re * dinv.re - v.im * dinv.im), -(v.re * dinv.im + v.im * dinv.re)};
        }
      }
      __syncwarp();
    }
    if (fail && lane == 0) atomicOr(S.flags, 1);
  }
  __syncthreads();
  const int f = S.flags[0];
  if (f) {  // fall back to M_d = I for this system
    for (int idx = threadIdx.x; idx < K * L; idx += NT) {
      const int k = idx / L, j = idx % L;
      S.Md[idx] = cplx<T>{(k % L) == j ? T(1) : T(0), T(0)};
    }
  }
  __syncthreads();
  return f;
}

// IMP: b = H^H y and (L > 0) the diagonal blocks of A = H^H H + sigma^2 I
// (Im of the diagonal 0), in fp64 from H, y in global memory; thread per
// entry.  Md[k L + j] = A[k][blk L + j] with blk = k / L, as bj_phase expects.
template <typename T>
__device__ void gram_phase_imp(const SimtParams& P, const Smem<T>& S, int64_t sys) {
  const int K = P.K, N = P.N, L = P.L;
  const float2* Hg = P.H + (size_t)sys * K * N;
  const float2* yg = P.y + (size_t)sys * N;
  const T s2 = (T)P.sigma2[sys];
  for (int k = threadIdx.x; k < K; k += NT) {
    const float2* hk = Hg + (size_t)k * N;
    T re = T(0), im = T(0);
    for (int n = 0; n < N; ++n) {  // conj(h) y
      const float2 h = hk[n], v = yg[n];
      re = fma((T)h.x, (T)v.x, fma((T)h.y, (T)v.y, re));
      im = fma((T)h.x, (T)v.y, fma(-(T)h.y, (T)v.x, im));
    }
    S.b[k] = cplx<T>{re, im};
  }
  if (L > 0)
    for (int idx = threadIdx.x; idx < K * L; idx += NT) {
      const int k = idx / L, l = (k / L) * L + idx % L;
      const float2* hk = Hg + (size_t)k * N;
      const float2* hl = Hg + (size_t)l * N;
      T re = T(0), im = T(0);
      for (int n = 0; n < N; ++n) {  // conj(h_k) h_l
        const float2 a = hk[n], c = hl[n];
        re = fma((T)a.x, (T)c.x, fma((T)a.y, (T)c.y, re));
        im = fma((T)a.x, (T)c.y, fma(-(T)a.y, (T)c.x, im));
      }
      if (l == k) {
        re = re + s2;
        im = T(0);
      }
      S.Md[idx] = cplx<T>{re, im};
    }
  __syncthreads();
}

// IMP: w = H^H (H v) + sigma^2 v in fp64, H from global memory in chunks of
// kIC antennas (t = H v of the chunk in S.ys, then w += H^H t).  K <= NT.
template <typename T>
__device__ void matvec_imp(const SimtParams& P, const Smem<T>& S, const cplx<T>* v, cplx<T>* w) {
  const int K = P.K, N = P.N, tid = threadIdx.x;
  const int64_t sys = blockIdx.x;
  const float2* Hg = P.H + (size_t)sys * K * N;
  T wr = T(0), wi = T(0);
  for (int n0 = 0; n0 < N; n0 += kIC) {
    const int cn = min(kIC, N - n0);
    for (int i = tid; i < cn; i += NT) {  // t_i = sum_k H[k][n0 + i] v_k
      T tr = T(0), ti = T(0);
      for (int k = 0; k < K; ++k) {
        const float2 h = Hg[(size_t)k * N + n0 + i];
        const cplx<T> q = v[k];
        tr = fma((T)h.x, q.re, fma(-(T)h.y, q.im, tr));
        ti = fma((T)h.x, q.im, fma((T)h.y, q.re, ti));
      }
      S.ys[i] = cplx<T>{tr, ti};
    }
    __syncthreads();
    if (tid < K) {  // w_k += sum_i conj(H[k][n0 + i]) t_i
      const float2* hk = Hg + (size_t)tid * N + n0;
      for (int i = 0; i < cn; ++i) {
        const float2 h = hk[i];
        const cplx<T> t = S.ys[i];
        wr = fma((T)h.x, t.re, fma((T)h.y, t.im, wr));
        wi = fma((T)h.x, t.im, fma(-(T)h.y, t.re, wi));
      }
    }
    __syncthreads();
  }
  if (tid < K) {
    const T s2 = (T)P.sigma2[sys];
    const cplx<T> q = v[tid];
    w[tid] = cplx<T>{fma(s2, q.re, wr), fma(s2, q.im, wi)};
  }
}

// e4m3 scales of A's rows (blocks of 16 complex = 32 real components).
template <typename T>
__device__ void fp8_scales_A(const SimtParams& P, const Smem<T>& S) {
  const int K = P.K, AS = K + 1, NB = (2 * K + 31) / 32;
  for (int idx = threadIdx.x; idx < K * NB; idx += NT) {
    const int k = idx / NB, bk = idx % NB;
    float amax = 0.f;
    for (int l = bk * 16; l < min(K, bk * 16 + 16); ++l) {
      cplx<T> a = S.A[k * AS + l];
      amax = fmaxf(amax, fmaxf(fabsf((float)a.re), fabsf((float)a.im)));
    }
    S.sA[idx] = e4m3_scale(amax);
  }
}

// z = M_d v (or z = v without a preconditioner), thread per row.
template <typename T>
__device__ inline void apply_precond(const SimtParams& P, const Smem<T>& S, const cplx<T>* v, cplx<T>* z) {
  const int K = P.K, L = P.L;
  for (int k = threadIdx.x; k < K; k += NT) {
    if (L > 0) {
      const int base = (k / L) * L;
      const cplx<T>* row = S.Md + (size_t)k * L;
      T re = T(0), im = T(0);
      for (int j = 0; j < L; ++j) {
        const cplx<T> m = row[j], q = v[base + j];
        re = fma(m.re, q.re, fma(-m.im, q.im, re));
        im = fma(m.re, q.im, fma(m.im, q.re, im));
      }
      z[k] = cplx<T>{re, im};
    } else {
      z[k] = v[k];
    }
  }
}

// ---------------------------------------------------------------------------
// Step 3: Algorithm 2 (L == 0) / Algorithm 3 (L > 0) for `iters` iterations
// on right-hand side S.b (main solve) or S.z-initialised rhs.  The solution
// is left in S.x.  Returns the status bits of this solve.
// ---------------------------------------------------------------------------
template <typename T, int MV, bool IMP = false>
__device__ int cg_phase(const SimtParams& P, const Smem<T>& S, const cplx<T>* rhs, int iters,
                        float* hist, float* coef = nullptr) {
  const int K = P.K, AS = K + 1, L = P.L, NB = (2 * K + 31) / 32;
  const int tid = threadIdx.x;
  int tpr = 32;
  while (tpr > 1 && tpr * K > NT) tpr >>= 1;
  const int row = tid / tpr, part = tid % tpr;
  const bool row_ok = row < K;
  int st = 0;

  // x0 = 0, r0 = rhs, p0 = r0 or M_d r0
  for (int k = tid; k < K; k += NT) {
    S.x[k] = cplx<T>{T(0), T(0)};
    S.r[k] = rhs[k];
  }
  __syncthreads();
  apply_precond(P, S, S.r, S.p);
  __syncthreads();
  T rho;  // carried rho (r^H r for CG, r^H z for BJ)
  {
    T t = T(0), h = T(0);
    for (int k = tid; k < K; k += NT) {
      const cplx<T> r = S.r[k], p = S.p[k];
      t += r.re * p.re + r.im * p.im;
      h += r.re * r.re + r.im * r.im;
    }
    block_sum2(t, h, S.red);
    rho = round_ip(t, P.ip);
    if (hist && tid == 0) hist[0] = (float)sqrt((double)h);
  }
  bool live = true;
  for (int it = 0; it < iters; ++it) {
    // round p for the matvec (e4m3: one scale per 16 complex entries)
    if (MV == E4M3) {
      for (int bk = tid; bk < NB; bk += NT) {
        float amax = 0.f;
        for (int l = bk * 16; l < min(K, bk * 16 + 16); ++l)
          amax = fmaxf(amax, fmaxf(fabsf((float)S.p[l].re), fabsf((float)S.p[l].im)));
        S.sp[bk] = e4m3_scale(amax);
      }
      __syncthreads();
    }
    for (int k = tid; k < K; k += NT) {
      cplx<T> v = S.p[k];
      if (MV == BF16 || MV == F16) {
        v.re = (T)round_to((float)v.re, MV);
        v.im = (T)round_to((float)v.im, MV);
      } else if (MV == E4M3) {
        const float s = S.sp[k / 16];
        v.re = (T)(round_to((float)v.re / s, E4M3) * s);
        v.im = (T)(round_to((float)v.im / s, E4M3) * s);
      }
      S.pq[k] = v;
    }
    __syncthreads();
    // varpi = A p (u_MV); every lane takes part in the shuffles
    if constexpr (IMP) {
      matvec_imp(P, S, S.pq, S.w);
    } else {
      T wr = T(0), wi = T(0);
      const cplx<T>* Arow = S.A + (size_t)(row_ok ? row : 0) * AS;
      for (int l = part; row_ok && l < K; l += tpr) {
        cplx<T> a = Arow[l];
        if (MV == BF16 || MV == F16) {
          a.re = (T)round_to((float)a.re, MV);
          a.im = (T)round_to((float)a.im, MV);
        } else if (MV == E4M3) {
          const float s = S.sA[row * NB + l / 16];
          a.re = (T)(round_to((float)a.re / s, E4M3) * s);
          a.im = (T)(round_to((float)a.im / s, E4M3) * s);
        }
        const cplx<T> q = S.pq[l];
        wr = fma(a.re, q.re, fma(-a.im, q.im, wr));
        wi = fma(a.re, q.im, fma(a.im, q.re, wi));
      }
      for (int o = tpr >> 1; o > 0; o >>= 1) {
        wr += __shfl_xor_sync(0xffffffffu, wr, o);
        wi += __shfl_xor_sync(0xffffffffu, wi, o);
      }
      if (row_ok && part == 0) S.w[row] = cplx<T>{wr, wi};
    }
    __syncthreads();
    // phi = Re(p^H varpi); for BJ with alpha_num = 0 also rho_{i-1} = Re(r^H p)
    T phi = T(0), rp = T(0);
    for (int k = tid; k < K; k += NT) {
      const cplx<T> p = S.p[k], w = S.w[k], r = S.r[k];
      phi += p.re * w.re + p.im * w.im;
      rp += r.re * p.re + r.im * p.im;
    }
    block_sum2(phi, rp, S.red);
    phi = round_ip(phi, P.ip);
    T rho_prev = (L > 0 && P.alpha_num == 0) ? round_ip(rp, P.ip) : rho;
    if (live) {
      if (rho_prev == T(0)) {
        st |= 2;  // FPCG_ST_RHO_ZERO
        live = false;
      } else if (!(phi > T(0)) || !isfinite((double)phi) || !isfinite((double)rho_prev)) {
        st |= 1;  // FPCG_ST_BREAKDOWN
        live = false;
      }
    }
    if (!live) {
      if (hist && tid == 0) hist[it + 1] = hist[it];
      continue;
    }
    const T alpha = rho_prev / phi;
    if (coef && tid == 0) coef[it] = (float)alpha;
    for (int k = tid; k < K; k += NT) {
      cplx<T> x = S.x[k], r = S.r[k];
      const cplx<T> p = S.p[k], w = S.w[k];
      x.re = fma(alpha, p.re, x.re);
      x.im = fma(alpha, p.im, x.im);
      r.re = fma(-alpha, w.re, r.re);
      r.im = fma(-alpha, w.im, r.im);
      S.x[k] = x;
      S.r[k] = r;
    }
    __syncthreads();
    apply_precond(P, S, S.r, S.z);
    __syncthreads();
    T rz = T(0), rr = T(0);
    const cplx<T>* zz = (L > 0) ? S.z : S.r;
    for (int k = tid; k < K; k += NT) {
      const cplx<T> r = S.r[k], z = zz[k];
      rz += r.re * z.re + r.im * z.im;
      rr += r.re * r.re + r.im * r.im;
    }
    block_sum2(rz, rr, S.red);
    const T rho_new = round_ip(rz, P.ip);
    const T beta = rho_new / rho_prev;
    if (coef && tid == 0) coef[iters + it] = (float)beta;
    for (int k = tid; k < K; k += NT) {
      cplx<T> p = S.p[k];
      const cplx<T> z = zz[k];
      p.re = fma(beta, p.re, z.re);
      p.im = fma(beta, p.im, z.im);
      S.p[k] = p;
    }
    rho = rho_new;
    if (hist && tid == 0) hist[it + 1] = (float)sqrt((double)rr);
    __syncthreads();
  }
  __syncthreads();
  return st;
}

// ---------------------------------------------------------------------------
// Step 4/5: residual out = b - A x; returns ||out||^2 and ||b||^2 (fp64) to
// every thread.  resid = FP32: A is the matvec matrix (A rounded to u_MV) and
// the sums are fp32.  resid = FP64 (and the fp64 mode): A is the Gram matrix
// itself and the sums are fp64-accurate -- compensated double-fp32 in the fp32
// modes (FMA TwoProd + TwoSum), plain fp64 in the fp64 mode.
// ---------------------------------------------------------------------------
template <typename T, int MV, bool IMP = false>
__device__ void residual(const SimtParams& P, const Smem<T>& S, cplx<T>* out, double& nr2, double& nb2) {
  const int K = P.K, AS = K + 1, tid = threadIdx.x, NB = (2 * K + 31) / 32;
  int tpr = 32;
  while (tpr > 1 && tpr * K > NT) tpr >>= 1;
  const int row = tid / tpr, part = tid % tpr;
  const bool row_ok = row < K;  // every lane of a warp takes part in the shuffles
  if constexpr (IMP) {  // out = b - (H^H (H x) + sigma^2 x), fp64
    matvec_imp(P, S, S.x, out);
    if (tid < K) {
      const cplx<T> bb = S.b[tid], v = out[tid];
      out[tid] = cplx<T>{bb.re - v.re, bb.im - v.im};
    }
  } else {
    const cplx<T>* Arow = S.A + (size_t)(row_ok ? row : 0) * AS;
    if (sizeof(T) == 8) {
      double sr = 0.0, si = 0.0;
      for (int l = part; row_ok && l < K; l += tpr) {
        const cplx<T> a = Arow[l], x = S.x[l];
        sr = fma((double)a.re, (double)x.re, fma(-(double)a.im, (double)x.im, sr));
        si = fma((double)a.re, (double)x.im, fma((double)a.im, (double)x.re, si));
      }
      for (int o = tpr >> 1; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (row_ok && part == 0) {
        const cplx<T> bb = S.b[row];
        out[row] = cplx<T>{(T)((double)bb.re - sr), (T)((double)bb.im - si)};
      }
    } else if (!P.resid_fp64) {
      float sr = 0.f, si = 0.f;
      for (int l = part; row_ok && l < K; l += tpr) {
        cplx<T> a = Arow[l];
        if (MV == BF16 || MV == F16) {
          a.re = (T)round_to((float)a.re, MV);
          a.im = (T)round_to((float)a.im, MV);
        } else if (MV == E4M3) {
          const float s = S.sA[row * NB + l / 16];
          a.re = (T)(round_to((float)a.re / s, E4M3) * s);
          a.im = (T)(round_to((float)a.im / s, E4M3) * s);
        }
        const cplx<T> x = S.x[l];
        sr = fmaf((float)a.re, (float)x.re, fmaf(-(float)a.im, (float)x.im, sr));
        si = fmaf((float)a.re, (float)x.im, fmaf((float)a.im, (float)x.re, si));
      }
      for (int o = tpr >> 1; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (row_ok && part == 0) {
        const cplx<T> bb = S.b[row];
        out[row] = cplx<T>{(T)((float)bb.re - sr), (T)((float)bb.im - si)};
      }
    } else {
      // (hr, lr) = b_re - sum(a_re x_re - a_im x_im), (hi, li) likewise
      float hr = 0.f, lr = 0.f, hi = 0.f, li = 0.f;
      if (row_ok && part == 0) {
        hr = (float)S.b[row].re;
        hi = (float)S.b[row].im;
      }
      for (int l = part; row_ok && l < K; l += tpr) {
        const cplx<T> a = Arow[l], x = S.x[l];
        df_sub_prod(hr, lr, (float)a.re, (float)x.re);
        df_sub_prod(hr, lr, -(float)a.im, (float)x.im);
        df_sub_prod(hi, li, (float)a.re, (float)x.im);
        df_sub_prod(hi, li, (float)a.im, (float)x.re);
      }
      for (int o = tpr >> 1; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hr, o), l2 = __shfl_xor_sync(0xffffffffu, lr, o);
        const float h3 = __shfl_xor_sync(0xffffffffu, hi, o), l3 = __shfl_xor_sync(0xffffffffu, li, o);
        df_add(hr, lr, h2, l2);
        df_add(hi, li, h3, l3);
      }
      if (row_ok && part == 0) out[row] = cplx<T>{(T)__fadd_rn(hr, lr), (T)__fadd_rn(hi, li)};
    }
  }
  __syncthreads();
  double a = 0.0, c = 0.0;
  for (int k = tid; k < K; k += NT) {
    const cplx<T> v = out[k], bb = S.b[k];
    a += (double)v.re * v.re + (double)v.im * v.im;
    c += (double)bb.re * bb.re + (double)bb.im * bb.im;
  }
  block_sum2(a, c, (double*)S.red);
  nr2 = a;
  nb2 = c;
}

template <typename T, int MV, bool IMP = false>
__global__ void __launch_bounds__(NT) detect_simt_kernel(SimtParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t sys = blockIdx.x;
  if (sys >= P.batch) return;
  Smem<T> S = carve<T>(smem_raw, P.K, P.L, IMP);
  const int K = P.K;
  int st = 0;

  if (P.Ain && (P.a_map || P.group_start)) {
    if (!load_shared(P, S, sys)) {  // index out of range: x = 0, labels 0, status
      cplx<T>* xo = (cplx<T>*)P.x_hat + (size_t)sys * K;
      for (int k = threadIdx.x; k < K; k += NT) {
        xo[k] = cplx<T>{T(0), T(0)};
        if (P.sym) P.sym[(size_t)sys * K + k] = 0;
      }
      if (threadIdx.x == 0) {
        if (P.rel_res) P.rel_res[sys] = 0.0;
        if (P.status) P.status[sys] = 64;  // FPCG_ST_BAD_INDEX
      }
      return;
    }
  } else if (P.Ain) {
    load_gram(P, S, sys);
  } else if constexpr (IMP) {
    gram_phase_imp(P, S, sys);
  } else {
    gram_phase(P, S, sys);
  }
  if (P.A_out) {  // gram-only mode (fpcg_gram)
    cplx<T>* Ao = (cplx<T>*)P.A_out + (size_t)sys * K * K;
    cplx<T>* bo = (cplx<T>*)P.b_out + (size_t)sys * K;
    for (int idx = threadIdx.x; idx < K * K; idx += NT) Ao[idx] = S.A[(idx / K) * (K + 1) + idx % K];
    for (int k = threadIdx.x; k < K; k += NT) bo[k] = S.b[k];
    return;
  }

  if (P.L > 0 && bj_phase(P, S, IMP)) st |= 8;  // FPCG_ST_BJ_FAIL
  if (MV == E4M3) {
    fp8_scales_A(P, S);
    __syncthreads();
  }
  float* hist = P.res_hist ? P.res_hist + (size_t)sys * (P.iters + 1) : nullptr;
  float* coef = P.coeffs ? P.coeffs + (size_t)sys * 2 * P.iters : nullptr;
  if (coef)  // a solve that stops early leaves zeros
    for (int k = threadIdx.x; k < 2 * P.iters; k += NT) coef[k] = 0.f;
  __syncthreads();
  st |= cg_phase<T, MV, IMP>(P, S, S.b, P.iters, hist, coef);

  // refinement: x_hat += solve(A, b - A x_hat)
  for (int rs = 0; rs < P.refine_steps; ++rs) {
    // keep x_hat in w while the correction solve reuses x
    for (int k = threadIdx.x; k < K; k += NT) S.w[k] = S.x[k];
    __syncthreads();
    double nr2, nb2;
    residual<T, MV, IMP>(P, S, S.z, nr2, nb2);  // S.x still holds x_hat
    // the correction solve overwrites x, r, p, z, w, pq: move rhs and x_hat out
    // of the way into the staging buffer (free after the Gram phase)
    cplx<T>* xs = S.Hs;
    cplx<T>* rhs = S.Hs + K;
    for (int k = threadIdx.x; k < K; k += NT) {
      xs[k] = S.w[k];
      rhs[k] = S.z[k];
    }
    __syncthreads();
    st |= cg_phase<T, MV, IMP>(P, S, rhs, P.refine_iters, nullptr) & 1;
    for (int k = threadIdx.x; k < K; k += NT) {
      cplx<T> v = xs[k];
      const cplx<T> d = S.x[k];
      v.re = v.re + d.re;
      v.im = v.im + d.im;
      S.x[k] = v;
    }
    __syncthreads();
  }

  double nr2, nb2;
  residual<T, MV, IMP>(P, S, S.z, nr2, nb2);
  if (threadIdx.x == 0 && P.rel_res) P.rel_res[sys] = nb2 > 0.0 ? sqrt(nr2 / nb2) : 0.0;

  // outputs
  int nonfinite = 0;
  cplx<T>* xo = (cplx<T>*)P.x_hat + (size_t)sys * K;
  for (int k = threadIdx.x; k < K; k += NT) {
    const cplx<T> v = S.x[k];
    xo[k] = v;
    if (!isfinite((double)v.re) || !isfinite((double)v.im)) nonfinite = 1;
  }
  nonfinite = __syncthreads_or(nonfinite);
  if (nonfinite) st |= 4;

  unsigned int errs = 0;
  int bad_qam = 0;
  if (P.sym || P.bit_errors) {
    const int M = P.qam[sys];
    const int m = qam_sqrt(M);
    if (m == 0) {
      bad_qam = 1;
      if (P.sym)
        for (int k = threadIdx.x; k < K; k += NT) P.sym[(size_t)sys * K + k] = 0;
    } else {
      const int nb = qam_bits_axis(m);
      const T s = (T)sqrt(2.0 * (M - 1) / 3.0);
      for (int k = threadIdx.x; k < K; k += NT) {
        const cplx<T> v = S.x[k];
        const int lab = (gray(axis_level<T>(v.re, m, s)) << nb) | gray(axis_level<T>(v.im, m, s));
        if (P.sym) P.sym[(size_t)sys * K + k] = (uint8_t)lab;
        if (P.tx) errs += __popc((unsigned)(lab ^ P.tx[(size_t)sys * K + k]));
      }
    }
  }
  if (bad_qam) st |= 16;
  if (P.bit_errors && P.tx) {
    errs = block_sum<unsigned int>(errs, (unsigned int*)S.red);
    if (threadIdx.x == 0 && errs) atomicAdd(P.bit_errors, (unsigned long long)errs);
  }
  if (threadIdx.x == 0 && P.status) P.status[sys] = st;
}

template <typename T, int MV, bool IMP = false>
cudaError_t launch_one(const SimtParams& P, cudaStream_t stream) {
  const size_t smem = smem_bytes<T>(P.K, P.L, MV, IMP);
  cudaError_t e = cudaFuncSetAttribute(detect_simt_kernel<T, MV, IMP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  detect_simt_kernel<T, MV, IMP><<<(unsigned)P.batch, NT, smem, stream>>>(P);
  return cudaGetLastError();
}

}  // namespace

size_t simt_smem_bytes(int fp64, int K, int L, int mv) {
  return fp64 ? smem_bytes<double>(K, L, mv, K > 64) : smem_bytes<float>(K, L, mv);
}

cudaError_t launch_detect_simt(const SimtParams& P, int fp64, int mv, cudaStream_t stream) {
  if (fp64 && P.K > 64) {  // A too large for shared memory: products from H (not for given A)
    if (P.Ain || P.A_out || !P.H) return cudaErrorInvalidValue;
    return launch_one<double, F64, true>(P, stream);
  }
  if (fp64) return launch_one<double, F64>(P, stream);
  switch (mv) {
    case F32: return launch_one<float, F32>(P, stream);
    case BF16: return launch_one<float, BF16>(P, stream);
    case F16: return launch_one<float, F16>(P, stream);
    case E4M3: return launch_one<float, E4M3>(P, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpcg
