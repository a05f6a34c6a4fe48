/*
 * fpcg.h -- C ABI of libfpcg: batched finite-precision CG detection for
 * massive MIMO on NVIDIA GB300 (sm_103a).
 *
 * The library implements the detectors of "Finite-Precision Conjugate
 * Gradient Method for Massive MIMO Detection" (arXiv 2504.09820):
 *   - LMMSE detection as the linear system A x = b with
 *     A = H^H H + sigma^2 I and b = H^H y (Section II, eq. inversion);
 *   - FP-CG (Algorithm 2): CG with the matrix-vector product A p at precision
 *     u_MV, the inner products at u_IP and every other step at u_W;
 *   - FP-BJ-CG (Algorithm 3): FP-CG left-preconditioned by the block-Jacobi
 *     matrix M_d = diag(A_1^{-1}, ..., A_d^{-1}) of eq. pre_BJ;
 * plus three steps the paper does not have: the Gram matrix and matched
 * filter formed from reduced-precision H and y with fp32 accumulation, an
 * iterative-refinement outer loop (residual b - A x at an accuracy above the
 * working precision, correction solve, x += d), and a Gray-QAM slicer with a
 * bit-error counter.
 *
 * Conventions for every entry point
 *   - All array arguments are DEVICE pointers into memory the caller owns
 *     (e.g. torch tensors' data_ptr()); the library never frees or keeps them.
 *     Inputs are never modified.  Structs passed by pointer are host memory.
 *   - Complex numbers are interleaved (re, im): "c64" is float2, "c128" is
 *     double2.
 *   - Letters follow the build: N = receive antennas (the paper's M),
 *     K = users = Gram dimension (the paper's N), L = block-Jacobi block size.
 *   - H of one system is column-major with leading dimension N: element
 *     (n, k) of system s sits at H[(s*K + k)*N + n].  y is [batch][N].
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream).  The return code reports argument errors and launch
 *     failures only; numerical trouble in a system is reported through that
 *     system's status word and never aborts the batch.
 *   - Entry points are thread-safe.  None calls cudaMalloc or another
 *     allocator, except the batch-plan functions, which own device
 *     workspace for two-pass classes (see the plan section).  Two paths use
 *     fixed device arrays of the library instead (static storage, held by
 *     every process that loads it): the fused tensor-core kernel's residual
 *     against the Gram matrix (resid = FPCG_FP64; a pool of one region per
 *     SM, 30 MiB at K = 64, shared safely by concurrent calls, since at most
 *     one of its CTAs runs per SM), and fpcg_detect_noalloc (below).
 */
#ifndef FPCG_H
#define FPCG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FPCG_API __attribute__((visibility("default")))
#else
#define FPCG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
enum {
  FPCG_OK = 0,
  FPCG_EINVAL = 1,   /* bad argument: null pointer, size out of range, K > N, K % L != 0, ... */
  FPCG_ENOTSUP = 2,  /* valid but not supported here (e.g. the fp64 mode with K > 64 on a given Gram matrix) */
  FPCG_ECUDA = 3,    /* a CUDA call or kernel launch failed; see fpcg_last_cuda_error() */
  FPCG_ENOMEM = 4    /* reserved for entry points that allocate */
};

/* Number formats (Table I of the paper, plus OCP FP8 E4M3). */
enum {
  FPCG_FP64 = 0,
  FPCG_FP32 = 1,
  FPCG_FP16 = 2,
  FPCG_BF16 = 3,
  FPCG_FP8E4M3 = 4
};

/* Per-system status bits (status[s]). */
#define FPCG_ST_BREAKDOWN 1  /* phi <= 0 or a non-finite scalar: the iterate was frozen */
#define FPCG_ST_RHO_ZERO  2  /* rho == 0: the residual vanished (e.g. y = 0); not an error */
#define FPCG_ST_NONFINITE 4  /* the returned x_hat has a non-finite entry */
#define FPCG_ST_BJ_FAIL   8  /* a diagonal block of A is not positive definite */
#define FPCG_ST_BAD_QAM  16  /* qam_order[s] not in {4,16,64,256}: sym_idx left 0 */
#define FPCG_ST_TIMEOUT  32  /* a pipeline wait of the tensor-core kernel gave up: outputs
                                of this system are not valid (never expected; reported
                                instead of hanging the GPU) */
#define FPCG_ST_BAD_INDEX 64 /* fpcg_detect_shared: rb_index[s] outside [0, n_rb): nothing solved,
                                x_hat and labels 0 */

/*
 * Precision of each step (the roles u_MV, u_IP, u_W of Algorithms 2/3).
 *   gram   format H and y are rounded to before the Gram/matched-filter
 *          products (FP64 | FP32 | BF16 | FP16); products and sums are fp32
 *          (fp64 for FP64).
 *   mv     u_MV: A and p are rounded to this format before A p, the products
 *          are summed at fp32 (FP64 | FP32 | BF16 | FP16 | FP8E4M3; e4m3 uses
 *          one power-of-two fp32 scale per `fp8_block` consecutive real
 *          components of a row of A and of p).
 *   ip     u_IP: inner products are summed at fp32 and rounded to this
 *          format (FP32 | BF16 | FP16), or FP64 in the fp64 mode.
 *   w      u_W: vectors x, r, p, z, the block inverses and the scalars
 *          (FP32, or FP64 for the all-fp64 parity mode, which needs
 *          gram = mv = ip = w = FP64 and returns x_hat as c128).
 *   refine_steps  iterative-refinement corrections after the main solve (>= 0).
 *   refine_iters  CG iterations of each correction solve (< 0: same as iters).
 *   alpha_num     FP-BJ-CG only: 0 = alpha's numerator r^H p as Algorithm 3
 *                 writes it, 1 = r^H z (textbook PCG); equal in exact arithmetic.
 *   fp8_block     e4m3 scale block in real components; must be 32.
 *   resid         the residual b - A x of the refinement and of rel_res:
 *                 FPCG_FP64 = A is the Gram matrix as formed (fp32 entries),
 *                 i.e. the refinement converges to the solution of the Gram
 *                 system itself.  On the fused tensor-core kernel A enters as
 *                 its matvec copy A16 plus the 16-bit remainder pieces of
 *                 fl32(A) - A16 (one for fp16: 22 of the 24 significand bits,
 *                 two for bf16: all 24), products exact, fp32 sums, so the
 *                 residual is within about 2^-22 |A||x| of the exact one; the
 *                 tensor-core solvers for given Gram matrices (fpcg_solve_gram,
 *                 fpcg_detect_shared, fpcg_detect_grouped, two-pass plan
 *                 classes, fpcg_detect_noalloc) read the fp32 A again from
 *                 global memory and form b - A x with fp32 products and sums
 *                 (within about (K/32 + 5) u32 |A||x|); the SIMT kernel uses
 *                 compensated double-fp32 products and sums (fp64-accurate;
 *                 GB300's fp64 units are far slower).
 *                 FPCG_FP32 = A is the matvec matrix (A rounded to u_MV) and
 *                 the sums are fp32: refinement then removes the CG iteration
 *                 error only, not the rounding of A (cheaper; every kernel).
 *                 rel_res is always the ratio of the two norms formed in fp64.
 *                 The fp64 mode always uses fp64.
 */
typedef struct fpcg_precision {
  int32_t gram;
  int32_t mv;
  int32_t ip;
  int32_t w;
  int32_t refine_steps;
  int32_t refine_iters;
  int32_t alpha_num;
  int32_t fp8_block;
  int32_t resid;
} fpcg_precision;

/*
 * fpcg_detect -- FP-CG detection (Algorithm 2) of `batch` independent systems.
 *
 * For each system s: A = fl(H)^H fl(H) + sigma2[s] I and b = fl(H)^H fl(y)
 * (Section II, eq. inversion; fl = rounding to prec->gram), `iters`
 * iterations of Algorithm 2 from x0 = 0 with no stopping test (Algorithm 1's
 * fixed iteration count), then prec->refine_steps refinement corrections,
 * then the hard Gray-QAM decision.
 *
 *   H          [batch][K][N] c64 channel matrices (column-major per system)
 *   y          [batch][N] c64 received vectors
 *   sigma2     [batch] double noise variances (>= 0)
 *   qam_order  [batch] int32 constellation sizes in {4,16,64,256};
 *              may be NULL when sym_idx and bit_errors are both NULL
 *   n_rx, k    N and K: 1 <= K <= 128, K <= N <= 65536
 *   batch      number of systems (>= 0; 0 is a no-op apart from zeroing
 *              *bit_errors)
 *   iters      CG iterations of the main solve (>= 0; 0 gives x = 0 before
 *              refinement)
 *   prec       step precisions (host pointer, required)
 *   x_hat      [batch][K] c64 estimates (c128 when prec->w == FPCG_FP64); required
 *   sym_idx    [batch][K] uint8 Gray labels: in-phase bits high, quadrature
 *              bits low; nullable
 *   rel_res    [batch] double ||b - A x_hat||_2 / ||b||_2 (0 when b = 0); nullable
 *   res_hist   [batch][iters+1] float ||r_i||_2 of the main solve's recursive
 *              residual, i = 0..iters; nullable
 *   tx_idx     [batch][K] uint8 transmitted labels; nullable (needs bit_errors)
 *   bit_errors one unsigned 64-bit counter: set to the number of bits in
 *              which sym_idx differs from tx_idx over the batch; nullable
 *   status     [batch] int32 FPCG_ST_* bits; nullable
 *   stream     cudaStream_t
 * Errors: FPCG_EINVAL for a bad argument (nothing is launched), FPCG_ECUDA
 * if a launch fails.  The fp64 mode with K > 64 never forms A (264 KB in
 * fp64 at K = 128, beyond shared memory): each product with A is
 * H^H (H v) + sigma^2 v in fp64 from H itself, the block-Jacobi blocks and b
 * are formed from H; a reference mode, slower than the others.
 */
FPCG_API int fpcg_detect(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
                int32_t n_rx, int32_t k, int64_t batch, int32_t iters,
                const fpcg_precision* prec,
                void* x_hat, uint8_t* sym_idx, double* rel_res, float* res_hist,
                const uint8_t* tx_idx, unsigned long long* bit_errors, int32_t* status,
                void* stream);

/*
 * fpbjcg_detect -- FP-BJ-CG detection (Algorithm 3): as fpcg_detect, with
 * the block-Jacobi preconditioner of eq. pre_BJ built from the L x L
 * diagonal blocks of A (inverted at u_W) and applied as z = M_d r in every
 * iteration.  block_L must divide K and satisfy 1 <= L <= 32 (L = K is a
 * direct block solve).  A block that is not positive definite sets
 * FPCG_ST_BJ_FAIL and that system falls back to M_d = I.
 */
FPCG_API int fpbjcg_detect(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
                  int32_t n_rx, int32_t k, int64_t batch, int32_t iters, int32_t block_L,
                  const fpcg_precision* prec,
                  void* x_hat, uint8_t* sym_idx, double* rel_res, float* res_hist,
                  const uint8_t* tx_idx, unsigned long long* bit_errors, int32_t* status,
                  void* stream);

/*
 * fpcg_solve_gram -- the paper's own interface (Algorithms 1-3 take A and b
 * as inputs): solve A x = b for `batch` Hermitian positive definite K x K
 * systems given directly.
 *   A      [batch][K][K] row-major, c64 (c128 when prec->w == FPCG_FP64)
 *   b      [batch][K] same element type
 *   block_L  0 = FP-CG (Algorithm 2), else FP-BJ-CG (Algorithm 3) with this L
 * prec->gram is ignored; everything else as fpcg_detect.  rel_res, res_hist
 * and status are nullable.  Runs on the tensor-core solver (one warp per
 * system, four for K = 128; A rounded to the matvec format in shared
 * memory) for mv in {BF16,
 * FP16}, w = FP32, resid in {FP32, FP64}, K in {8, 16, 32, 64, 128} (K = 8 in 16-wide slots
 * holding diag(A, I), b padded with zeros: the same iterates), block_L in {0,
 * 4, 8, 16} and 16-byte aligned A, b; else on the SIMT kernel.
 */
FPCG_API int fpcg_solve_gram(const void* A, const void* b, int32_t k, int64_t batch, int32_t iters,
                    int32_t block_L, const fpcg_precision* prec,
                    void* x_hat, double* rel_res, float* res_hist, int32_t* status,
                    void* stream);

/*
 * fpcg_gram -- form the Gram matrix and matched filter only (Section II,
 * eq. inversion): A = fl(H)^H fl(H) + sigma2[s] I and b = fl(H)^H fl(y) for
 * every system, fl = rounding of H and y to `gram` (FPCG_BF16 or FPCG_FP16:
 * exact products and fp32 accumulation on the tensor cores -- the tcgen05
 * pipeline for K in {8,16,32,64,128} with N even and 16-byte aligned H and y
 * (and A at K = 128), mma.sync for K in {8,16,32,64,128} otherwise -- and in
 * fp32 FMAs for other K;
 * FPCG_FP32: fp32; FPCG_FP64: fp64).  The Hermitian A is written in
 * full.  Useful when one A serves many received vectors.
 *   A       [batch][K][K] row-major, c64 (c128 for FPCG_FP64)
 *   b       [batch][K] same element type
 *   status  [batch] int32, nullable: 0, or FPCG_ST_TIMEOUT
 * Other arguments as fpcg_detect.
 */
FPCG_API int fpcg_gram(const void* H, const void* y, const double* sigma2, int32_t n_rx, int32_t k,
                       int64_t batch, int32_t gram, void* A, void* b, int32_t* status, void* stream);

/*
 * fpcg_path -- which kernel fpcg_detect / fpbjcg_detect (block_L = 0 for
 * FP-CG) would use for this configuration: FPCG_PATH_TENSOR_CORE (the fused
 * tcgen05 Gram + mma.sync CG kernel: gram and mv in {BF16, FP16}, w = FP32,
 * resid in {FP32, FP64}, K in {16, 32, 64}, L in {0, 4, 8, 16}, N even; H and y must also be
 * 16-byte aligned, which this query cannot see) or FPCG_PATH_SIMT (one CTA per system, every
 * other configuration); FPCG_EINVAL (negative) for an invalid configuration.
 * Setting the environment variable FPCG_FORCE_SIMT=1 makes every call take
 * the SIMT kernel (same results within rounding; for A/B comparisons).
 * Host only, no GPU needed.
 */
#define FPCG_PATH_SIMT 0
#define FPCG_PATH_TENSOR_CORE 1
/* (plans only) Gram matrices by mma.sync into plan workspace, then the tensor-core
 * solver; for classes the fused kernel does not take (K = 8, K = 128) */
#define FPCG_PATH_TWO_PASS 2
FPCG_API int fpcg_path(int32_t n_rx, int32_t k, int32_t block_L, const fpcg_precision* prec);

/*
 * fpcg_detect_shared -- many right-hand sides per channel (Section II's model
 * with one H for a group of received vectors, e.g. the 12 subcarriers x 14
 * symbols of a resource block).  Each group's Gram matrix is formed once, by
 * fpcg_gram, and kept; every received vector y_s is then detected against the
 * Gram of its group g = rb_index[s]: its own matched filter b_s = fl(H_g)^H
 * fl(y_s) (eq. inversion, rounded to prec->gram like the Gram), then Algorithm
 * 2 (block_L = 0) or Algorithm 3 (block_L > 0), refinement, slicing, as in
 * fpcg_detect.  Tensor-core modes (w = FP32, resid in {FP32, FP64}, mv = BF16 | FP16) with
 * K in {8, 16, 32, 64, 128} and block_L in {0, 4, 8, 16} run on the
 * tensor-core solver: one warp per received vector, the group's 16-bit A and
 * inverted blocks reloaded only when rb_index changes between consecutive
 * vectors (so vectors sorted by group share them); other modes run one CTA
 * per received vector (the SIMT kernel).
 *   A          [n_rb][K][K] complex64 (complex128 in FP64 mode): A_g + sigma_g^2 I,
 *              as fpcg_gram writes it with the same gram format
 *   H          [n_rb][K][N] complex64: the groups' channels (the layout of fpcg_detect)
 *   y          [n_rhs][N] complex64
 *   rb_index   [n_rhs] int32, group of each received vector; one outside [0, n_rb)
 *              gives FPCG_ST_BAD_INDEX for that vector
 *   qam_order, x_hat, sym_idx, rel_res, tx_idx, bit_errors, status: per received
 *              vector, as in fpcg_detect (batch = n_rhs)
 * All device pointers, caller-owned.  Returns FPCG_EINVAL / FPCG_ENOTSUP as
 * fpcg_detect does (K <= 128; K <= 64 in FP64 mode).
 */
FPCG_API int fpcg_detect_shared(const void* A, const void* H, const void* y, const int32_t* rb_index,
                                const int32_t* qam_order, int32_t n_rx, int32_t k, int64_t n_rb,
                                int64_t n_rhs, int32_t iters, int32_t block_L, const fpcg_precision* prec,
                                void* x_hat, uint8_t* sym_idx, double* rel_res, const uint8_t* tx_idx,
                                unsigned long long* bit_errors, int32_t* status, void* stream);

/*
 * fpcg_detect_grouped -- fpcg_detect_shared for received vectors stored grouped
 * by channel: the vectors of group g are y[group_start[g] .. group_start[g+1]).
 * Same computation and arguments otherwise (A from fpcg_gram, H per group,
 * outputs per received vector), with
 *   group_start  device [n_groups + 1] int64, non-decreasing, group_start[0] = 0,
 *                group_start[n_groups] = n_rhs (not checked on the device)
 * Runs on the tensor-core solver when K in {8, 16, 32, 64, 128} (8: padded as
 * in fpcg_solve_gram), block_L in {0, 4, 8, 16}, mv in {BF16, FP16}, w = FP32,
 * resid in {FP32, FP64} and A is 16-byte aligned:
 * the eight warps of a CTA share one group's A (rounded to the matvec format)
 * and inverted diagonal blocks, and each warp detects one received vector at a
 * time.  Otherwise the SIMT kernel (one CTA per received vector).
 */
FPCG_API int fpcg_detect_grouped(const void* A, const void* H, const void* y, const int64_t* group_start,
                                 const int32_t* qam_order, int32_t n_rx, int32_t k, int64_t n_groups,
                                 int64_t n_rhs, int32_t iters, int32_t block_L, const fpcg_precision* prec,
                                 void* x_hat, uint8_t* sym_idx, double* rel_res, const uint8_t* tx_idx,
                                 unsigned long long* bit_errors, int32_t* status, void* stream);

/*
 * ---- Uneven batches: a plan over systems of different (N, K) ----
 *
 * A plan groups the systems of one batch by (N, K) class.  Each class runs as
 * one persistent launch of the kernel that fpcg_path names, or of the other
 * kernel when fpcg_plan_autotune measured it faster on that class.  Both
 * kernels compute the same algorithm (Algorithm 2, or 3 when block_L > 0) at
 * the same precisions, so the choice changes results only within rounding.
 * The class launches can be captured once into a CUDA graph and replayed.
 *
 * Layout ("plan order"): the systems are stored grouped by class, in the
 * caller's order within each class.  fpcg_plan_layout gives, for position i of
 * plan order:
 *   order[i]  the caller's index of the system;
 *   h_off[i]  offset in complex elements of its H (K columns of N, column-major)
 *             in the packed H buffer;
 *   y_off[i]  offset of its y (N) in the packed y buffer;
 *   x_off[i]  offset of its x_hat (K) in the packed x_hat buffer, and of its K
 *             labels in the sym_idx and tx_idx byte buffers;
 *   totals    {elements of H, of y, of x_hat} to allocate.
 * Every class starts on a 256-byte boundary of each buffer.  Per-system arrays
 * (sigma2, qam_order, rel_res, status) are indexed by plan order.
 *
 * Ownership: the plan owns its host tables, the instantiated CUDA graph, a
 * capture stream and, when some class runs in two passes (FPCG_PATH_TWO_PASS:
 * the Gram matrices of the class first, then the solves), device workspace for
 * those Gram matrices (allocated by the first autotune or run);
 * fpcg_plan_destroy frees them.  All data buffers are the caller's device
 * memory.  A plan is not thread-safe; runs of one plan are ordered on the
 * stream they are issued to.
 */
typedef struct fpcg_plan fpcg_plan;

typedef struct fpcg_batch_desc {
  int64_t batch;            /* number of systems, >= 0 */
  const int32_t* n_rx;      /* host [batch]: N of each system, K <= N <= 65536 */
  const int32_t* k;         /* host [batch]: K of each system, 1 <= K <= 128 */
  int32_t iters;            /* CG iterations per system, >= 0 */
  int32_t block_L;          /* 0: FP-CG (Algorithm 2); > 0: FP-BJ-CG (Algorithm 3) with block size
                               min(block_L, K), which must divide K */
  fpcg_precision prec;      /* as for fpcg_detect */
  int32_t flags;            /* FPCG_PLAN_GRAPH: capture the class launches into a CUDA graph on the
                               first run and replay it while the run's pointers stay the same */
} fpcg_batch_desc;

#define FPCG_PLAN_GRAPH 1
#define FPCG_PLAN_PER_CLASS 2 /* one launch per class (by default the fused-kernel classes of the same
                               * block size and precisions share one launch: up to ten per launch) */

typedef struct fpcg_class_info {
  int32_t n_rx, k, block_L; /* the class's N, K and block size (0: FP-CG) */
  int32_t path;             /* FPCG_PATH_SIMT, FPCG_PATH_TENSOR_CORE or FPCG_PATH_TWO_PASS */
  int64_t first, count;     /* its systems: plan positions [first, first + count) */
  int32_t mv;               /* its matvec format (the plan's, or fpcg_plan_autoprec's choice) */
  int32_t launch;           /* index of the launch that detects its systems within one run: classes
                             * that share a fused launch share it (a two-pass class's Gram pass is a
                             * launch of its own before it) */
  double kappa;             /* fpcg_plan_autoprec's condition-number estimate, 0 before */
  int32_t cg_warps;         /* FPCG_PATH_TENSOR_CORE: CG warps per CTA of the fused kernel (6, or 8
                             * for K <= 32: the default choice, or fpcg_plan_autotune's); else 0 */
  int32_t reserved;
} fpcg_class_info;

/* Builds a plan (host only, no GPU work).  FPCG_EINVAL for a bad descriptor,
 * FPCG_ENOMEM if host memory runs out. */
FPCG_API int fpcg_plan_create(const fpcg_batch_desc* desc, fpcg_plan** plan);

/* Plan-order layout (see above); any output pointer may be NULL.  Host only. */
FPCG_API int fpcg_plan_layout(const fpcg_plan* plan, int64_t* order, int64_t* h_off, int64_t* y_off,
                              int64_t* x_off, int64_t totals[3]);

/* Number of classes, and their description when info (n_classes entries) is non-NULL. */
FPCG_API int fpcg_plan_classes(const fpcg_plan* plan, int32_t* n_classes, fpcg_class_info* info);

/* Times, for every class that both kernels can run, each kernel on the given
 * inputs (plan order; outputs are overwritten) and keeps the faster -- on the
 * fused kernel for K <= 32 with six and with eight CG warps per CTA (the
 * results are the same; fpcg_class_info.cg_warps reports the choice).
 * Issues work on `stream` and synchronises it.  Drops a captured graph. */
FPCG_API int fpcg_plan_autotune(fpcg_plan* plan, const void* H, const void* y, const double* sigma2,
                                const int32_t* qam_order, void* x_hat, uint8_t* sym_idx,
                                double* rel_res, int32_t* status, void* stream);

/* Precision selection per class (Sections III-B and IV-B): for every class,
 * fp32 CG (and, with block_L > 0, fp32 FP-BJ-CG) runs min(K, 32) steps on up
 * to 64 of its systems and fpcg_kappa_cg_batch turns the step sizes into
 * condition-number estimates (the median is kept: kappa of A, and kappa_bar
 * of the preconditioned matrix).  The matvec format is then the one eq.
 * heuristic (eq. heuristic_bj for FP-BJ-CG) chooses, capped at fp32, and
 * FP-CG or FP-BJ-CG is chosen by the break-even criterion of Remark 4
 * (fpcg_choose_method with target accuracy tol).  The choices replace the
 * class's mv and block size; its kernel is chosen again (the default, until the
 * next autotune).  Synchronises `stream`; drops a captured graph and the
 * two-pass workspace (allocated again by the next run).  Allocates, and
 * frees, a small device buffer of its own. */
FPCG_API int fpcg_plan_autoprec(fpcg_plan* plan, const void* H, const void* y, const double* sigma2, double tol,
                                void* stream);

/* Detects the whole batch (plan order), asynchronously on `stream`.  Arguments
 * as for fpcg_detect, with the packed buffers of fpcg_plan_layout; bit_errors
 * (with tx_idx) is the total over all classes. */
FPCG_API int fpcg_plan_run(fpcg_plan* plan, const void* H, const void* y, const double* sigma2,
                           const int32_t* qam_order, void* x_hat, uint8_t* sym_idx, double* rel_res,
                           const uint8_t* tx_idx, unsigned long long* bit_errors, int32_t* status,
                           void* stream);

/* Frees the plan (NULL is accepted).  Call it once the plan's work has
 * finished (for instance after synchronising the stream of its last run). */
FPCG_API int fpcg_plan_destroy(fpcg_plan* plan);

/*
 * fpcg_detect_noalloc -- detection that allocates no device memory (the paper
 * has no counterpart: this is about the library's memory, not the method).
 * Same arguments and results as fpbjcg_detect (block_L > 0) or fpcg_detect
 * (block_L = 0).  Configurations that run in two passes (Gram matrices first,
 * then the tensor-core solver: K = 8 and K = 128 with a 16-bit matvec, w =
 * FP32, gram in {BF16, FP16}) keep their Gram matrices and matched filters in one
 * fixed 64 MiB device array of the library; every other configuration takes
 * the ordinary path, which allocates nothing either.
 *   - Limit: batch * K * (K + 1) * 8 bytes <= 64 MiB (K = 128: 508 systems per
 *     call; K = 8: 116508); a larger batch returns FPCG_ENOTSUP (split it).
 *     Every argument is checked before any work is issued, so a refused call
 *     changes nothing (not the array, status or bit_errors).
 *   - The array is shared by all calls on a device: calls must not overlap in
 *     time (issue them on one stream, or wait for one before the next).
 *   - status[] holds the Gram pass's bits (FPCG_ST_TIMEOUT) OR-ed with the
 *     solve's.
 *   - Outside a stream capture every call looks up the array's address
 *     (cudaGetSymbolAddress; the array moves when cudaDeviceReset reloads the
 *     library's module); inside a capture the address found by the previous
 *     call on that device is used, so make one call on each device before any
 *     capture begins, and after a cudaDeviceReset.
 */
FPCG_API int fpcg_detect_noalloc(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
                                 int32_t n_rx, int32_t k, int64_t batch, int32_t iters, int32_t block_L,
                                 const fpcg_precision* prec, void* x_hat, uint8_t* sym_idx, double* rel_res,
                                 float* res_hist, const uint8_t* tx_idx, unsigned long long* bit_errors,
                                 int32_t* status, void* stream);

/*
 * fpcg_detect_coeffs -- fpcg_detect (block_L = 0) or fpbjcg_detect (block_L > 0)
 * that also returns the step sizes of the main solve (Algorithm 2 / 3):
 *   coeffs  [batch][2][iters] float, device, required: coeffs[s][0][j] = alpha_j
 *           and coeffs[s][1][j] = beta_j for j < iters (0 after a breakdown or
 *           rho = 0 stopped the solve).  Refinement passes are not recorded.
 * These are what the exact-arithmetic relation between CG and the Lanczos
 * process turns into Ritz values of A (of the preconditioned matrix for
 * Algorithm 3): fpcg_kappa_cg / fpcg_kappa_cg_batch estimate the condition
 * number that the precision heuristic of Section III-B needs from them.
 * Runs on the SIMT kernel (one CTA per system), which records them; other
 * arguments and errors as fpcg_detect (no res_hist).
 */
FPCG_API int fpcg_detect_coeffs(const void* H, const void* y, const double* sigma2, const int32_t* qam_order,
                                int32_t n_rx, int32_t k, int64_t batch, int32_t iters, int32_t block_L,
                                const fpcg_precision* prec, void* x_hat, uint8_t* sym_idx, double* rel_res,
                                const uint8_t* tx_idx, unsigned long long* bit_errors, int32_t* status,
                                float* coeffs, void* stream);

/*
 * ---- Precision selection (Section IV-B, eq. heuristic and eq. heuristic_bj) ----
 *
 * fpcg_choose_precision -- the lowest-precision Table I format (BF16, FP16,
 * FP32, FP64 in that order) whose unit roundoff u satisfies the paper's
 * heuristic u_MV < 1 / (K^(3/2) sqrt(kappa)).  For FP-CG kappa is that of A;
 * for FP-BJ-CG that of the block-Jacobi preconditioned matrix.  Returns the
 * FPCG_* format code, or -FPCG_EINVAL for k < 1 or kappa < 1 (or not
 * finite).  *u_bound (nullable) receives the bound.  Host only.
 */
FPCG_API int fpcg_choose_precision(int32_t k, double kappa, double* u_bound);

/*
 * fpcg_kappa_cg -- estimate of kappa from the first m CG step sizes alpha_0 ..
 * alpha_{m-1} and beta_0 .. beta_{m-2} of Algorithm 2 or 3 (exact-arithmetic
 * relation between CG and Lanczos): the tridiagonal T_m with diagonal 1/alpha_j
 * + beta_{j-1}/alpha_{j-1} (beta_{-1} = 0) and off-diagonal sqrt(beta_j)/alpha_j
 * has the Ritz values of A (of the preconditioned matrix for Algorithm 3).
 * kappa_hat = largest / smallest eigenvalue of T_m, found by bisection on
 * Sturm sequences; kappa_hat <= kappa, equal after K steps in exact arithmetic.
 * FPCG_EINVAL for m < 1, alpha_j <= 0 or beta_j < 0.  Host only.
 */
FPCG_API int fpcg_kappa_cg(const double* alpha, const double* beta, int32_t m, double* kappa_hat);

/*
 * fpcg_kappa_cg_batch -- fpcg_kappa_cg for every system of a coefficient array
 * as fpcg_detect_coeffs writes it (host memory, [batch][2][iters]), from the
 * first m <= iters step sizes: kappa_hat[s] (host, [batch]) is the estimate,
 * or NaN where the coefficients do not define one (a solve stopped before m
 * steps).  FPCG_EINVAL for m < 1, m > iters or a null pointer.  Host only.
 */
FPCG_API int fpcg_kappa_cg_batch(const float* coeffs, int32_t iters, int32_t m, int64_t batch, double* kappa_hat);

/*
 * fpcg_choose_method -- the break-even criterion of Remark 4 between FP-CG and
 * FP-BJ-CG with block size L: preconditioning pays when the iterations it
 * saves exceed C_BJ / C_CG^it + k_PCG (C_PCG^it / C_CG^it - 1).  Costs are the
 * multiplications of the paper's cost model (Section V-A.1, weights bf16 = fp16
 * = 1, fp32 = 2, fp64 = 4): C_CG^it = K^2 w(mv_cg), C_PCG^it = K^2 w(mv_bj) +
 * K L w(w), C_BJ = (K / L) L^3 w(w).  The iteration counts k are those the CG
 * bound 2 ((sqrt(kappa) - 1) / (sqrt(kappa) + 1))^k <= tol asks for, with
 * kappa for FP-CG and kappa_bar (the preconditioned matrix's) for FP-BJ-CG.
 * Returns L (use FP-BJ-CG) or 0 (use FP-CG); *k_cg and *k_pcg (nullable)
 * receive the counts.  -FPCG_EINVAL for K < 1, L < 1, K % L, kappa or
 * kappa_bar < 1 or not finite, tol outside (0, 1), or an unknown format.
 * Host only.
 */
FPCG_API int fpcg_choose_method(int32_t k, int32_t block_L, double kappa, double kappa_bar, double tol,
                                int32_t mv_cg, int32_t mv_bj, int32_t w, int32_t* k_cg, int32_t* k_pcg);

/*
 * fpcg_fma_probe -- a throughput probe of the CUDA cores, with no counterpart
 * in the paper: it states the fp32 and fp64 FMA rates that bound the SIMT
 * kernels (the fp32 plain-CG comparator's Gram runs on these units).  Launches
 * out_len / 256 blocks of 256 threads on `stream`; every thread runs eight
 * independent FMA chains for `iters` steps in fp64 (fp64 != 0) or fp32 and
 * writes one value to out (device, out_len doubles or floats, caller-owned;
 * its contents mean nothing).  *flops (host, nullable) receives the launch's
 * floating-point operations (2 per FMA); the caller times the launch.
 * Asynchronous.  FPCG_EINVAL for out_len not a positive multiple of 256,
 * iters not a positive multiple of 4, or a null or misaligned out.
 */
FPCG_API int fpcg_fma_probe(int32_t fp64, int64_t iters, void* out, int64_t out_len, double* flops, void* stream);

/* Human-readable text for a return code (static storage). */
FPCG_API const char* fpcg_strerror(int code);

/* Text of the last CUDA error seen by this thread in an entry point, or "". */
FPCG_API const char* fpcg_last_cuda_error(void);

/* Library version as major*10000 + minor*100 + patch. */
FPCG_API int fpcg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FPCG_H */
