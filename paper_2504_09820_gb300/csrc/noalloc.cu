// fpcg_detect_noalloc: detection that allocates no device memory at all.
//
// Some callers cannot allocate while they detect: a receiver loop that
// reserved all of its device memory when it started and must not fail or
// block on an allocation in the middle of a slot, or a host framework whose
// own allocator owns the device memory.  fpcg_detect and fpbjcg_detect already
// allocate nothing; the configurations that need scratch memory are the
// two-pass ones (the Gram matrices are formed first, then the systems are
// solved from them: K = 8 and K = 128), for which plans keep workspace of
// their own.
// This entry point gives those callers the two-pass path with its scratch in
// one fixed, file-scope device array instead.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fpcg.h"
#include "api_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB: Gram matrices and matched filters
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_scratch, per device

// Address of the array on the current device.  It is looked up again on every
// call outside a stream capture (a cudaDeviceReset reloads the module and
// moves the array); during a capture, where the lookup might not be allowed,
// the address found by an earlier call on this device is used.
int scratch_address(cudaStream_t stream, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fpcg::cuda_error(e);
  if (dev < 0 || dev >= kMaxDevices) return FPCG_ENOTSUP;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return fpcg::cuda_error(e);
  std::lock_guard<std::mutex> lock(g_mu);
  if (cap == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
    void* a = nullptr;
    e = cudaGetSymbolAddress(&a, g_scratch);
    if (e != cudaSuccess) return fpcg::cuda_error(e);
    g_scratch_addr[dev] = a;
  }
  *out = g_scratch_addr[dev];
  return FPCG_OK;
}

}  // namespace

extern "C" {

int fpcg_detect_noalloc(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
                        int32_t n_rx, int32_t k, int64_t batch, int32_t iters, int32_t block_L,
                        const fpcg_precision* prec, void* x_hat, uint8_t* sym_idx, double* rel_res,
                        float* res_hist, const uint8_t* tx_idx, unsigned long long* bit_errors, int32_t* status,
                        void* stream) {
  if (!prec || fpcg::check_precision(prec)) return FPCG_EINVAL;
  int rc = fpcg::check_detect_args(k, batch, iters, block_L, x_hat, sym_idx, qam_order, tx_idx, bit_errors);
  if (rc) return rc;
  if (!fpcg::two_pass_capable(k, block_L, prec))  // needs no scratch: the ordinary path
    return fpcg::run_uniform(H, y, sigma2, qam_order, nullptr, nullptr, n_rx, k, batch, iters, block_L, prec, x_hat,
                             sym_idx, rel_res, res_hist, tx_idx, bit_errors, status, stream, -1, true);
  if (!H || !y || !sigma2 || n_rx < k || n_rx > 65536) return FPCG_EINVAL;
  // batch * (K*K + K) complex entries must fit; compared by division, so a huge batch cannot wrap
  const size_t per_system = sizeof(float2) * ((size_t)k * k + k);
  if ((uint64_t)batch > kScratchBytes / per_system) return FPCG_ENOTSUP;  // split the batch
  cudaStream_t s = (cudaStream_t)stream;
  void* base = nullptr;
  rc = scratch_address(s, &base);
  if (rc) return rc;
  float2* A = static_cast<float2*>(base);
  float2* b = A + (size_t)batch * k * k;
  // Every argument is checked by now: a bad call has returned before touching
  // the array.  fpcg_gram overwrites A and b entirely and zeroes status;
  // run_uniform zeroes bit_errors and ORs the solve's status bits into the
  // Gram pass's (an FPCG_ST_TIMEOUT there is kept).  Nothing else in the
  // array needs to start at zero.
  rc = fpcg_gram(H, y, sigma2, n_rx, k, batch, prec->gram, A, b, status, s);
  if (rc) return rc;
  return fpcg::run_uniform(nullptr, nullptr, nullptr, qam_order, A, b, k, k, batch, iters, block_L, prec, x_hat,
                           sym_idx, rel_res, res_hist, tx_idx, bit_errors, status, stream, FPCG_PATH_TENSOR_CORE,
                           true, true);
}

}  // extern "C"
