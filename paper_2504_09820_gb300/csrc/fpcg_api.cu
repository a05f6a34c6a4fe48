// C ABI entry points of libfpcg: argument validation and dispatch.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "../../include/fpcg.h"
#include "api_internal.cuh"
#include "detect_simt.cuh"
#include "gram_mma.cuh"
#include "mf_mma.cuh"
#include "gram_tc.cuh"
#include "detect_tc.cuh"
#include "solve_tc.cuh"

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return FPCG_ECUDA;
}

bool is_fmt(int f) { return f >= FPCG_FP64 && f <= FPCG_FP8E4M3; }

// Checks the precision struct; returns FPCG_OK, FPCG_EINVAL or FPCG_ENOTSUP.
int check_prec(const fpcg_precision* p) {
  if (!p) return FPCG_EINVAL;
  if (!is_fmt(p->gram) || !is_fmt(p->mv) || !is_fmt(p->ip) || !is_fmt(p->w) || !is_fmt(p->resid))
    return FPCG_EINVAL;
  if (p->refine_steps < 0 || p->alpha_num < 0 || p->alpha_num > 1) return FPCG_EINVAL;
  if (p->mv == FPCG_FP8E4M3 && p->fp8_block != 32) return FPCG_ENOTSUP;
  if (p->w == FPCG_FP64) {
    if (p->gram != FPCG_FP64 || p->mv != FPCG_FP64 || p->ip != FPCG_FP64) return FPCG_EINVAL;
    return FPCG_OK;
  }
  if (p->w != FPCG_FP32) return FPCG_EINVAL;
  if (p->gram == FPCG_FP64 || p->gram == FPCG_FP8E4M3) return FPCG_EINVAL;
  if (p->mv == FPCG_FP64) return FPCG_EINVAL;
  if (p->ip == FPCG_FP64 || p->ip == FPCG_FP8E4M3) return FPCG_EINVAL;
  if (p->resid != FPCG_FP64 && p->resid != FPCG_FP32) return FPCG_EINVAL;
  return FPCG_OK;
}

int check_device_smem(size_t need) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return cuda_fail(e);
  return need <= (size_t)optin ? FPCG_OK : FPCG_ENOTSUP;
}

bool force_simt() {
  const char* v = getenv("FPCG_FORCE_SIMT");
  return v && v[0] && v[0] != '0';
}


int device_sms(int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e);
  return FPCG_OK;
}

// The CG warp's settings and outputs (shared by the fused detector and the solver).
void cg_params(fpcg::DetectTcParams& T, const int32_t* qam_order, int32_t iters, int32_t block_L,
               const fpcg_precision* prec, int refine_iters, void* x_hat, uint8_t* sym_idx, double* rel_res,
               float* res_hist, const uint8_t* tx_idx, unsigned long long* bit_errors, int32_t* status) {
  T.qam = qam_order;
  T.iters = iters;
  T.L = block_L;
  T.refine_steps = prec->refine_steps;
  T.refine_iters = refine_iters;
  T.alpha_num = prec->alpha_num;
  T.ip = prec->ip;
  T.resid_gram = prec->resid == FPCG_FP64;
  T.x_hat = (float2*)x_hat;
  T.sym = sym_idx;
  T.rel_res = rel_res;
  T.res_hist = res_hist;
  T.tx = tx_idx;
  T.bit_errors = bit_errors;
  T.status = status;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// Precisions the solvers for given Gram matrices run on the tensor cores:
// 16-bit matvec, fp32 vectors, the residual against the matvec matrix (resid
// FP32) or the given fp32 Gram matrix (FP64).
bool tc_prec_ok(const fpcg_precision* p) {
  return p->w == FPCG_FP32 && (p->resid == FPCG_FP32 || p->resid == FPCG_FP64) &&
         (p->mv == FPCG_BF16 || p->mv == FPCG_FP16);
}

}  // namespace

namespace fpcg {

int run_uniform(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
                const void* Ain, const void* bin, int32_t n_rx, int32_t k, int64_t batch, int32_t iters,
                int32_t block_L, const fpcg_precision* prec, void* x_hat, uint8_t* sym_idx,
                double* rel_res, float* res_hist, const uint8_t* tx_idx,
                unsigned long long* bit_errors, int32_t* status, void* stream, int path, bool reset_bits,
                bool status_or, float* coeffs, int cg_warps) {
  int rc = check_prec(prec);
  if (rc) return rc;
  rc = check_detect_args(k, batch, iters, block_L, x_hat, sym_idx, qam_order, tx_idx, bit_errors);
  if (rc) return rc;
  if (!Ain && (n_rx < k || n_rx > 65536)) return FPCG_EINVAL;
  if (Ain ? (!bin) : (!H || !y || !sigma2)) return FPCG_EINVAL;
  const int fp64 = prec->w == FPCG_FP64;
  if (fp64 && k > 64 && Ain) return FPCG_ENOTSUP;  // K > 64 in fp64: products from H only
  const int refine_iters = prec->refine_iters < 0 ? iters : prec->refine_iters;
  cudaStream_t s = (cudaStream_t)stream;
  if (bit_errors && reset_bits) {
    cudaError_t e = cudaMemsetAsync(bit_errors, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (batch == 0) return FPCG_OK;
  const bool tc_possible = Ain ? tc_prec_ok(prec) && fpcg::solve_tc_supported(k, block_L) && aligned16(Ain) &&
                                     aligned16(bin)
                               : tc_capable(k, block_L, prec) && fpcg::tma_pipe_ok(H, y, n_rx);
  if (path == FPCG_PATH_TENSOR_CORE && !tc_possible) return FPCG_ENOTSUP;
  // the step sizes are recorded by the SIMT kernel only (keeping the tensor-core CG loop small)
  const bool tc_ok = tc_possible && !coeffs && (path == FPCG_PATH_TENSOR_CORE || (path < 0 && !force_simt()));
  if (tc_ok && Ain) {  // given Gram matrices: the tensor-core solver
    int sms = 0;
    rc = device_sms(&sms);
    if (rc) return rc;
    rc = check_device_smem(fpcg::solve_tc_smem_bytes(k, block_L));
    if (rc) return rc;
    fpcg::SolveTcParams T;
    memset(&T, 0, sizeof(T));
    cg_params(T.D, qam_order, iters, block_L, prec, refine_iters, x_hat, sym_idx, rel_res, res_hist, tx_idx,
              bit_errors, status);
    T.A = (const float2*)Ain;
    T.b = (const float2*)bin;
    T.n = batch;
    T.n_groups = batch;
    T.N = k;
    T.K = k;
    T.gram = prec->gram;
    T.D.status_or = status_or && status;
    cudaError_t e = fpcg::launch_solve_tc(T, sms, prec->mv == FPCG_BF16, s);
    return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
  }
  int sms_tc = 0;
  if (tc_ok && !Ain) {
    rc = device_sms(&sms_tc);
    if (rc) return rc;
  }
  // the Gram residual's (and the e4m3 matvec's) scratch pool has one region per SM
  const bool f8 = prec->mv == FPCG_FP8E4M3;
  const bool scratch_ok = (prec->resid != FPCG_FP64 && !f8) || sms_tc <= fpcg::kTcScratchRegions;
  if (path == FPCG_PATH_TENSOR_CORE && tc_ok && !Ain && !scratch_ok) return FPCG_ENOTSUP;
  if (tc_ok && scratch_ok) {
    const int sms = sms_tc;
    rc = check_device_smem(fpcg::detect_tc_smem_bytes(k, block_L, f8));
    if (rc) return rc;
    fpcg::DetectTcParams T;
    memset(&T, 0, sizeof(T));
    if (!fpcg::make_pipe(&T.pipe, (const float2*)H, (const float2*)y, n_rx, k, batch, prec->gram == FPCG_BF16))
      return FPCG_ENOTSUP;
    T.sigma2 = sigma2;
    cg_params(T, qam_order, iters, block_L, prec, refine_iters, x_hat, sym_idx, rel_res, res_hist, tx_idx,
              bit_errors, status);
    T.resid_gram = prec->resid == FPCG_FP64;
    T.ncg = cg_warps;
    cudaError_t e = fpcg::launch_detect_tc(T, sms, prec->mv, s);
    return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
  }
  rc = check_device_smem(fpcg::simt_smem_bytes(fp64, k, block_L, prec->mv));
  if (rc) return rc;
  fpcg::SimtParams P;
  memset(&P, 0, sizeof(P));
  P.H = (const float2*)H;
  P.y = (const float2*)y;
  P.sigma2 = sigma2;
  P.qam = qam_order;
  P.Ain = Ain;
  P.bin = bin;
  P.N = Ain ? k : n_rx;
  P.K = k;
  P.iters = iters;
  P.L = block_L;
  P.refine_steps = prec->refine_steps;
  P.refine_iters = refine_iters;
  P.alpha_num = prec->alpha_num;
  P.gram = prec->gram;
  P.ip = prec->ip;
  P.resid_fp64 = prec->resid == FPCG_FP64;
  P.batch = batch;
  P.x_hat = x_hat;
  P.sym = sym_idx;
  P.rel_res = rel_res;
  P.res_hist = res_hist;
  P.tx = tx_idx;
  P.bit_errors = bit_errors;
  P.status = status;
  P.coeffs = coeffs;
  cudaError_t e = fpcg::launch_detect_simt(P, fp64, fp64 ? FPCG_FP64 : prec->mv, s);
  if (e != cudaSuccess) return cuda_fail(e);
  return FPCG_OK;
}

int cuda_error(cudaError_t e) { return cuda_fail(e); }

bool fused_multi_capable(const FusedClass& c, int32_t block_L, const fpcg_precision* prec) {
  return (c.k == 16 || c.k == 32 || c.k == 64) && (prec->mv == FPCG_BF16 || prec->mv == FPCG_FP16) &&
         !force_simt() && tc_capable(c.k, block_L, prec) && c.batch > 0 && c.x_hat &&
         fpcg::tma_pipe_ok(c.H, c.y, c.n) && !check_detect_args(c.k, c.batch, 0, block_L, c.x_hat, c.sym, c.qam,
                                                                c.tx, c.tx ? (const unsigned long long*)1 : nullptr);
}

int fused_cg_warps(int k, int n, int preset) {
  return preset == 6 || (preset == 8 && k <= 32) ? preset : fpcg::tc_cg_warps(k, n);
}

int prepare_fused_pools(void* stream) {
  uint8_t* pool;
  int* busy;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = fpcg::tc_rem_pool<16>(s, &pool, &busy);
  if (e == cudaSuccess) e = fpcg::tc_rem_pool<32>(s, &pool, &busy);
  if (e == cudaSuccess) e = fpcg::tc_rem_pool<64>(s, &pool, &busy);
  return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
}

static_assert(kFusedMultiMax == fpcg::kTcMultiMax, "one limit on the classes of a fused launch");

int run_fused_multi(const FusedClass* cls, int n, int32_t iters, int32_t block_L, const fpcg_precision* prec,
                    unsigned long long* bit_errors, void* stream) {
  if (n < 1 || n > kFusedMultiMax || iters < 0) return FPCG_EINVAL;
  int rc = check_prec(prec);
  if (rc) return rc;
  for (int c = 0; c < n; ++c)
    if (!fused_multi_capable(cls[c], block_L, prec)) return FPCG_ENOTSUP;
  int sms = 0;
  rc = device_sms(&sms);
  if (rc) return rc;
  if (prec->resid == FPCG_FP64 && sms > fpcg::kTcScratchRegions) return FPCG_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  // the parameter block is large (up to ten tensor-map pairs): built on the heap
  fpcg::MultiTcParams* M = new (std::nothrow) fpcg::MultiTcParams;
  if (!M) return FPCG_ENOMEM;
  memset(M, 0, sizeof(*M));
  M->nclass = n;
  cudaError_t e = fpcg::tc_rem_pool<16>(s, &M->pool[0], &M->busy[0]);
  if (e == cudaSuccess) e = fpcg::tc_rem_pool<32>(s, &M->pool[1], &M->busy[1]);
  if (e == cudaSuccess) e = fpcg::tc_rem_pool<64>(s, &M->pool[2], &M->busy[2]);
  if (e != cudaSuccess) {
    delete M;
    return cuda_fail(e);
  }
  const int refine_iters = prec->refine_iters < 0 ? iters : prec->refine_iters;
  size_t smem = 0;
  for (int c = 0; c < n; ++c) {
    const FusedClass& f = cls[c];
    fpcg::DetectTcParams& T = M->cls[c];
    if (!fpcg::make_pipe(&T.pipe, (const float2*)f.H, (const float2*)f.y, f.n, f.k, f.batch,
                         prec->gram == FPCG_BF16)) {
      delete M;
      return FPCG_ENOTSUP;
    }
    T.sigma2 = f.sigma2;
    cg_params(T, f.qam, iters, block_L, prec, refine_iters, f.x_hat, f.sym, f.rel_res, nullptr, f.tx,
              f.tx ? bit_errors : nullptr, f.status);
    T.resid_gram = prec->resid == FPCG_FP64;
    T.ncg = f.cg_warps;
    const size_t sm = fpcg::detect_tc_smem_bytes(f.k, block_L);
    smem = sm > smem ? sm : smem;
  }
  rc = check_device_smem(smem);
  if (!rc) {
    e = fpcg::launch_detect_tc_multi(*M, sms, block_L, prec->mv == FPCG_BF16, prec->resid == FPCG_FP64, s);
    rc = e == cudaSuccess ? FPCG_OK : cuda_fail(e);
  }
  delete M;
  return rc;
}

int check_detect_args(int32_t k, int64_t batch, int32_t iters, int32_t block_L, const void* x_hat,
                      const uint8_t* sym_idx, const int32_t* qam_order, const uint8_t* tx_idx,
                      const unsigned long long* bit_errors) {
  if (k < 1 || k > 128 || batch < 0 || iters < 0) return FPCG_EINVAL;
  if (block_L < 0 || block_L > 32 || (block_L > 0 && k % block_L)) return FPCG_EINVAL;
  if (!x_hat) return FPCG_EINVAL;
  if ((sym_idx || bit_errors) && !qam_order) return FPCG_EINVAL;
  if ((tx_idx != nullptr) != (bit_errors != nullptr)) return FPCG_EINVAL;
  return FPCG_OK;
}

int check_precision(const fpcg_precision* p) { return check_prec(p); }

bool two_pass_capable(int k, int block_L, const fpcg_precision* prec) {
  return tc_prec_ok(prec) && (prec->gram == FPCG_BF16 || prec->gram == FPCG_FP16) && fpcg::gram_mma_supported(k) &&
         fpcg::solve_tc_supported(k, block_L) && !fpcg::detect_tc_supported(k, block_L);
}

bool tc_capable(int k, int block_L, const fpcg_precision* prec) {
  return prec->w == FPCG_FP32 && (prec->gram == FPCG_BF16 || prec->gram == FPCG_FP16) &&
         (prec->mv == FPCG_BF16 || prec->mv == FPCG_FP16 || (prec->mv == FPCG_FP8E4M3 && prec->fp8_block == 32)) &&
         fpcg::detect_tc_supported(k, block_L);
}

}  // namespace fpcg

namespace {
using fpcg::run_uniform;
using fpcg::tc_capable;

int run(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
        const void* Ain, const void* bin, int32_t n_rx, int32_t k, int64_t batch, int32_t iters,
        int32_t block_L, const fpcg_precision* prec, void* x_hat, uint8_t* sym_idx,
        double* rel_res, float* res_hist, const uint8_t* tx_idx,
        unsigned long long* bit_errors, int32_t* status, void* stream) {
  return run_uniform(H, y, sigma2, qam_order, Ain, bin, n_rx, k, batch, iters, block_L, prec, x_hat, sym_idx,
                     rel_res, res_hist, tx_idx, bit_errors, status, stream, -1, true);
}

}  // namespace

extern "C" {

int fpcg_detect(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
                int32_t n_rx, int32_t k, int64_t batch, int32_t iters, const fpcg_precision* prec,
                void* x_hat, uint8_t* sym_idx, double* rel_res, float* res_hist,
                const uint8_t* tx_idx, unsigned long long* bit_errors, int32_t* status,
                void* stream) {
  return run(H, y, sigma2, qam_order, nullptr, nullptr, n_rx, k, batch, iters, 0, prec, x_hat,
             sym_idx, rel_res, res_hist, tx_idx, bit_errors, status, stream);
}

int fpbjcg_detect(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
                  int32_t n_rx, int32_t k, int64_t batch, int32_t iters, int32_t block_L,
                  const fpcg_precision* prec, void* x_hat, uint8_t* sym_idx, double* rel_res,
                  float* res_hist, const uint8_t* tx_idx, unsigned long long* bit_errors,
                  int32_t* status, void* stream) {
  if (block_L < 1) return FPCG_EINVAL;
  return run(H, y, sigma2, qam_order, nullptr, nullptr, n_rx, k, batch, iters, block_L, prec,
             x_hat, sym_idx, rel_res, res_hist, tx_idx, bit_errors, status, stream);
}

int fpcg_detect_shared(const void* A, const void* H, const void* y, const int32_t* rb_index,
                       const int32_t* qam_order, int32_t n_rx, int32_t k, int64_t n_rb, int64_t n_rhs,
                       int32_t iters, int32_t block_L, const fpcg_precision* prec, void* x_hat,
                       uint8_t* sym_idx, double* rel_res, const uint8_t* tx_idx,
                       unsigned long long* bit_errors, int32_t* status, void* stream) {
  int rc = check_prec(prec);
  if (rc) return rc;
  if (!A || !H || !y || !rb_index || !x_hat) return FPCG_EINVAL;
  if (k < 1 || k > 128 || n_rx < k || n_rx > 65536 || n_rb < 0 || n_rhs < 0 || iters < 0) return FPCG_EINVAL;
  if (block_L < 0 || block_L > 32 || (block_L > 0 && k % block_L)) return FPCG_EINVAL;
  if ((sym_idx || bit_errors) && !qam_order) return FPCG_EINVAL;
  if ((tx_idx != nullptr) != (bit_errors != nullptr)) return FPCG_EINVAL;
  const int fp64 = prec->w == FPCG_FP64;
  if (fp64 && k > 64) return FPCG_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  if (bit_errors) {
    cudaError_t e = cudaMemsetAsync(bit_errors, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (n_rhs == 0) return FPCG_OK;
  if (!force_simt() && tc_prec_ok(prec) && fpcg::solve_tc_supported(k, block_L) && aligned16(A)) {
    // the tensor-core solver: a warp refills its slot when the block index changes
    int sms = 0;
    rc = device_sms(&sms);
    if (rc) return rc;
    rc = check_device_smem(fpcg::solve_tc_smem_bytes(k, block_L));
    if (rc) return rc;
    fpcg::SolveTcParams T;
    memset(&T, 0, sizeof(T));
    cg_params(T.D, qam_order, iters, block_L, prec, prec->refine_iters < 0 ? iters : prec->refine_iters, x_hat,
              sym_idx, rel_res, nullptr, tx_idx, bit_errors, status);
    T.A = (const float2*)A;
    T.H = (const float2*)H;
    T.y = (const float2*)y;
    T.a_map = rb_index;
    T.n = n_rhs;
    T.n_groups = n_rb;
    T.N = n_rx;
    T.K = k;
    T.gram = prec->gram;
    cudaError_t e = fpcg::launch_solve_tc(T, sms, prec->mv == FPCG_BF16, s);
    return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
  }
  rc = check_device_smem(fpcg::simt_smem_bytes(fp64, k, block_L, prec->mv));
  if (rc) return rc;
  fpcg::SimtParams P;
  memset(&P, 0, sizeof(P));
  P.H = (const float2*)H;
  P.y = (const float2*)y;
  P.qam = qam_order;
  P.Ain = A;
  P.a_map = rb_index;
  P.n_shared = n_rb;
  P.N = n_rx;
  P.K = k;
  P.iters = iters;
  P.L = block_L;
  P.refine_steps = prec->refine_steps;
  P.refine_iters = prec->refine_iters < 0 ? iters : prec->refine_iters;
  P.alpha_num = prec->alpha_num;
  P.gram = prec->gram;
  P.ip = prec->ip;
  P.resid_fp64 = prec->resid == FPCG_FP64;
  P.batch = n_rhs;
  P.x_hat = x_hat;
  P.sym = sym_idx;
  P.rel_res = rel_res;
  P.tx = tx_idx;
  P.bit_errors = bit_errors;
  P.status = status;
  cudaError_t e = fpcg::launch_detect_simt(P, fp64, fp64 ? FPCG_FP64 : prec->mv, s);
  return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
}

int fpcg_detect_grouped(const void* A, const void* H, const void* y, const int64_t* group_start,
                        const int32_t* qam_order, int32_t n_rx, int32_t k, int64_t n_groups, int64_t n_rhs,
                        int32_t iters, int32_t block_L, const fpcg_precision* prec, void* x_hat,
                        uint8_t* sym_idx, double* rel_res, const uint8_t* tx_idx,
                        unsigned long long* bit_errors, int32_t* status, void* stream) {
  int rc = check_prec(prec);
  if (rc) return rc;
  if (!A || !H || !y || !group_start || !x_hat) return FPCG_EINVAL;
  if (k < 1 || k > 128 || n_rx < k || n_rx > 65536 || n_groups < 1 || n_rhs < 0 || iters < 0) return FPCG_EINVAL;
  if (block_L < 0 || block_L > 32 || (block_L > 0 && k % block_L)) return FPCG_EINVAL;
  if ((sym_idx || bit_errors) && !qam_order) return FPCG_EINVAL;
  if ((tx_idx != nullptr) != (bit_errors != nullptr)) return FPCG_EINVAL;
  const int fp64 = prec->w == FPCG_FP64;
  if (fp64 && k > 64) return FPCG_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  if (bit_errors) {
    cudaError_t e = cudaMemsetAsync(bit_errors, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (n_rhs == 0) return FPCG_OK;
  const int refine_iters = prec->refine_iters < 0 ? iters : prec->refine_iters;
  if (!force_simt() && tc_prec_ok(prec) && fpcg::solve_grouped_supported(k, block_L) && aligned16(A)) {
    int sms = 0;
    rc = device_sms(&sms);
    if (rc) return rc;
    rc = check_device_smem(fpcg::solve_grouped_smem_bytes(k, block_L));
    if (rc) return rc;
    fpcg::SolveTcParams T;
    memset(&T, 0, sizeof(T));
    cg_params(T.D, qam_order, iters, block_L, prec, refine_iters, x_hat, sym_idx, rel_res, nullptr, tx_idx,
              bit_errors, status);
    T.A = (const float2*)A;
    T.H = (const float2*)H;
    T.y = (const float2*)y;
    T.group_start = group_start;
    if ((prec->gram == FPCG_BF16 || prec->gram == FPCG_FP16) && fpcg::mf_mma_supported(k) && aligned16(x_hat)) {
      // every vector's matched filter at once on the tensor cores, into x_hat (same size)
      fpcg::MfMmaParams M{(const float2*)H, (const float2*)y, group_start, (float2*)x_hat, n_rx, k, n_groups};
      cudaError_t e = fpcg::launch_mf_mma(M, prec->gram == FPCG_BF16, s);
      if (e != cudaSuccess) return cuda_fail(e);
      T.b = (const float2*)x_hat;
    }
    T.n = n_rhs;
    T.n_groups = n_groups;
    T.N = n_rx;
    T.K = k;
    T.gram = prec->gram;
    cudaError_t e = fpcg::launch_solve_grouped(T, sms, prec->mv == FPCG_BF16, s);
    return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
  }
  rc = check_device_smem(fpcg::simt_smem_bytes(fp64, k, block_L, prec->mv));
  if (rc) return rc;
  fpcg::SimtParams P;
  memset(&P, 0, sizeof(P));
  P.H = (const float2*)H;
  P.y = (const float2*)y;
  P.qam = qam_order;
  P.Ain = A;
  P.group_start = group_start;
  P.n_shared = n_groups;
  P.N = n_rx;
  P.K = k;
  P.iters = iters;
  P.L = block_L;
  P.refine_steps = prec->refine_steps;
  P.refine_iters = refine_iters;
  P.alpha_num = prec->alpha_num;
  P.gram = prec->gram;
  P.ip = prec->ip;
  P.resid_fp64 = prec->resid == FPCG_FP64;
  P.batch = n_rhs;
  P.x_hat = x_hat;
  P.sym = sym_idx;
  P.rel_res = rel_res;
  P.tx = tx_idx;
  P.bit_errors = bit_errors;
  P.status = status;
  cudaError_t e = fpcg::launch_detect_simt(P, fp64, fp64 ? FPCG_FP64 : prec->mv, s);
  return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
}

int fpcg_detect_coeffs(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
                       int32_t n_rx, int32_t k, int64_t batch, int32_t iters, int32_t block_L,
                       const fpcg_precision* prec, void* x_hat, uint8_t* sym_idx, double* rel_res,
                       const uint8_t* tx_idx, unsigned long long* bit_errors, int32_t* status, float* coeffs,
                       void* stream) {
  if (!coeffs) return FPCG_EINVAL;
  return fpcg::run_uniform(H, y, sigma2, qam_order, nullptr, nullptr, n_rx, k, batch, iters, block_L, prec, x_hat,
                           sym_idx, rel_res, nullptr, tx_idx, bit_errors, status, stream, -1, true, false, coeffs);
}

int fpcg_solve_gram(const void* A, const void* b, int32_t k, int64_t batch, int32_t iters,
                    int32_t block_L, const fpcg_precision* prec, void* x_hat, double* rel_res,
                    float* res_hist, int32_t* status, void* stream) {
  if (!A || !b) return FPCG_EINVAL;
  return run(nullptr, nullptr, nullptr, nullptr, A, b, k, k, batch, iters, block_L, prec, x_hat,
             nullptr, rel_res, res_hist, nullptr, nullptr, status, stream);
}

int fpcg_gram(const void* H, const void* y, const double* sigma2, int32_t n_rx, int32_t k,
              int64_t batch, int32_t gram, void* A, void* b, int32_t* status, void* stream) {
  if (!H || !y || !sigma2 || !A || !b) return FPCG_EINVAL;
  if (k < 1 || k > 128 || n_rx < k || n_rx > 65536 || batch < 0) return FPCG_EINVAL;
  if (gram != FPCG_FP64 && gram != FPCG_FP32 && gram != FPCG_BF16 && gram != FPCG_FP16) return FPCG_EINVAL;
  if (gram == FPCG_FP64 && k > 64) return FPCG_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  if (status) {
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t) * (size_t)batch, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (batch == 0) return FPCG_OK;
  if ((gram == FPCG_BF16 || gram == FPCG_FP16) && fpcg::gram_tc_supported(k) && fpcg::tma_pipe_ok(H, y, n_rx) &&
      !force_simt()) {
    int sms = 0;
    int rc = device_sms(&sms);
    if (rc) return rc;
    rc = check_device_smem(fpcg::gram_tc_smem_bytes());
    if (rc) return rc;
    fpcg::GramTcParams P;
    if (!fpcg::make_pipe(&P.pipe, (const float2*)H, (const float2*)y, n_rx, k, batch, gram == FPCG_BF16))
      return FPCG_ENOTSUP;
    P.sigma2 = sigma2;
    P.A = (float2*)A;
    P.b = (float2*)b;
    P.status = status;
    cudaError_t e = fpcg::launch_gram_tc(P, sms, s);
    return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
  }
  if ((gram == FPCG_BF16 || gram == FPCG_FP16) && k == 128 && fpcg::tma_pipe_ok(H, y, n_rx) &&
      ((uintptr_t)A % 16) == 0 && !force_simt()) {
    int sms = 0;
    int rc = device_sms(&sms);
    if (rc) return rc;
    rc = check_device_smem(fpcg::gram_tc128_smem_bytes());
    if (rc) return rc;
    fpcg::GramTc128Params P;
    memset(&P, 0, sizeof(P));
    if (!fpcg::make_gram_tc128(&P, (const float2*)H, (const float2*)y, (float2*)A, n_rx, batch, gram == FPCG_BF16))
      return FPCG_ENOTSUP;
    P.sigma2 = sigma2;
    P.b = (float2*)b;
    P.status = status;
    cudaError_t e = fpcg::launch_gram_tc128(P, sms, s);
    return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
  }
  if ((gram == FPCG_BF16 || gram == FPCG_FP16) && fpcg::gram_mma_supported(k) && !force_simt()) {
    fpcg::GramMmaParams P{(const float2*)H, (const float2*)y, sigma2, (float2*)A, (float2*)b, n_rx, k, batch};
    cudaError_t e = fpcg::launch_gram_mma(P, gram == FPCG_BF16, s);
    return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
  }
  const int fp64 = gram == FPCG_FP64;
  int rc = check_device_smem(fpcg::simt_smem_bytes(fp64, k, 0, FPCG_FP32));
  if (rc) return rc;
  fpcg::SimtParams P;
  memset(&P, 0, sizeof(P));
  P.H = (const float2*)H;
  P.y = (const float2*)y;
  P.sigma2 = sigma2;
  P.N = n_rx;
  P.K = k;
  P.gram = gram;
  P.ip = FPCG_FP32;
  P.batch = batch;
  P.A_out = A;
  P.b_out = b;
  P.x_hat = A;  // unused in gram-only mode
  cudaError_t e = fpcg::launch_detect_simt(P, fp64, fp64 ? FPCG_FP64 : FPCG_FP32, s);
  return e == cudaSuccess ? FPCG_OK : cuda_fail(e);
}

int fpcg_path(int32_t n_rx, int32_t k, int32_t block_L, const fpcg_precision* prec) {
  if (check_prec(prec)) return -FPCG_EINVAL;
  if (k < 1 || k > 128 || n_rx < k || block_L < 0 || block_L > 32 || (block_L > 0 && k % block_L))
    return -FPCG_EINVAL;
  return !force_simt() && fpcg::tc_capable(k, block_L, prec) && n_rx % 2 == 0 ? FPCG_PATH_TENSOR_CORE
                                                                               : FPCG_PATH_SIMT;
}

const char* fpcg_strerror(int code) {
  switch (code) {
    case FPCG_OK: return "success";
    case FPCG_EINVAL: return "invalid argument";
    case FPCG_ENOTSUP: return "unsupported configuration";
    case FPCG_ECUDA: return "CUDA error";
    case FPCG_ENOMEM: return "out of device memory";
    default: return "unknown error";
  }
}

const char* fpcg_last_cuda_error(void) { return g_cuda_err; }

int fpcg_version(void) { return 100; }

}  // extern "C"
