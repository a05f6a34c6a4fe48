// Internal entry points shared by the C ABI files of libfpcg.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fpcg.h"

namespace fpcg {

// One uniform batch (every system with the same N, K): validation and
// dispatch to a kernel.  path: -1 = as fpcg_path chooses, FPCG_PATH_SIMT or
// FPCG_PATH_TENSOR_CORE (FPCG_ENOTSUP if the tensor-core kernel cannot run
// it).  reset_bits: zero *bit_errors first (a plan zeroes it once for all of
// its classes).  status_or (given Gram matrices, tensor-core solver): OR the
// solve's status bits into status[], which the Gram pass filled, instead of
// overwriting them.  cg_warps: the fused kernel's CG warps (fused_cg_warps).
int run_uniform(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
                const void* Ain, const void* bin, int32_t n_rx, int32_t k, int64_t batch, int32_t iters,
                int32_t block_L, const fpcg_precision* prec, void* x_hat, uint8_t* sym_idx,
                double* rel_res, float* res_hist, const uint8_t* tx_idx,
                unsigned long long* bit_errors, int32_t* status, void* stream, int path, bool reset_bits,
                bool status_or = false, float* coeffs = nullptr, int cg_warps = 0);

// CG warps per CTA of the fused kernel for a class: `preset` (6, or 8 for
// K <= 32) if valid, else the default choice for (K, N).
int fused_cg_warps(int k, int n, int preset);

// One class of a fused multi-class launch: its inputs and outputs (device
// pointers at the class's first system), N, K and batch size.
struct FusedClass {
  const void* H;
  const void* y;
  const double* sigma2;
  const int32_t* qam;
  int32_t n, k;
  int64_t batch;
  void* x_hat;
  uint8_t* sym;
  double* rel_res;
  const uint8_t* tx;
  int32_t* status;
  int cg_warps;  // 0: the default choice (fused_cg_warps)
};

// Whether a class can join a fused multi-class launch: the fused kernel's
// K (16, 32, 64), a 16-bit matvec, an even N (the TMA views), aligned data.
bool fused_multi_capable(const FusedClass& c, int32_t block_L, const fpcg_precision* prec);

constexpr int kFusedMultiMax = 10;  // classes per fused multi-class launch

// Detection of n classes (n <= kFusedMultiMax, every one fused_multi_capable, the same
// iterations, block size and precisions) in one launch of the fused kernel;
// bit_errors (nullable) is accumulated into, not zeroed.
int run_fused_multi(const FusedClass* cls, int n, int32_t iters, int32_t block_L, const fpcg_precision* prec,
                    unsigned long long* bit_errors, void* stream);

// Device addresses of the fused kernel's scratch pools on the current device,
// looked up now (call outside a stream capture before capturing a launch
// that needs them).
int prepare_fused_pools(void* stream);

// Checks of the arguments common to every detection entry point (no GPU
// work): FPCG_OK or FPCG_EINVAL.
int check_detect_args(int32_t k, int64_t batch, int32_t iters, int32_t block_L, const void* x_hat,
                      const uint8_t* sym_idx, const int32_t* qam_order, const uint8_t* tx_idx,
                      const unsigned long long* bit_errors);

// Whether the fused tensor-core kernel supports this configuration (alignment
// of the data aside).
bool tc_capable(int k, int block_L, const fpcg_precision* prec);

// Whether a class can run as Gram (mma.sync) + tensor-core solver.
bool two_pass_capable(int k, int block_L, const fpcg_precision* prec);

// FPCG_OK, FPCG_EINVAL or FPCG_ENOTSUP for a precision descriptor.
int check_precision(const fpcg_precision* p);

// Records a CUDA error for fpcg_last_cuda_error and returns FPCG_ECUDA.
int cuda_error(cudaError_t e);

}  // namespace fpcg
