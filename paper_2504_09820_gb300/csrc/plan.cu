// Uneven-batch plans (fpcg_plan_*): systems grouped by (N, K) class, the packed
// plan-order layout, the per-class kernel choice (autotuned on request) and the
// CUDA-graph capture of the class launches.  Host code only; the kernels are the
// uniform ones, reached through run_uniform.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fpcg.h"
#include "api_internal.cuh"

struct fpcg_plan {
  struct Class {
    int32_t n, k, L, path;         // path: -1 = default choice, else FPCG_PATH_*
    int32_t ncg = 0;               // fused kernel's CG warps (0: the default choice)
    fpcg_precision prec;           // the plan's, or the one fpcg_plan_autoprec chose for the class
    double kappa = 0.0;            // fpcg_plan_autoprec's estimate (0: none)
    int64_t first, count;          // plan positions
    int64_t h0, y0, x0;            // first element of the class in H, y, x_hat
    int64_t a0, b0;                // two-pass classes: first Gram entry / matched-filter entry in the workspace
  };
  int32_t iters, flags;
  fpcg_precision prec;
  std::vector<Class> cls;
  std::vector<int64_t> order, h_off, y_off, x_off;
  int64_t tot[3] = {0, 0, 0};
  cudaStream_t cap = nullptr;      // capture stream (graphs cannot be captured on the legacy stream)
  float2* ws = nullptr;            // workspace: Gram matrices and matched filters of two-pass classes
  int64_t ws_a = 0;                // complex entries of the Gram part (the matched filters follow)
  cudaGraphExec_t exec = nullptr;  // instantiated graph of the class launches
  const void* key[10] = {};        // the run arguments it was captured with
};

namespace {

constexpr int64_t kAlign = 32;  // elements: 256 bytes of complex64

int64_t align_up(int64_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

void drop_graph(fpcg_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  p->exec = nullptr;
}

int default_path(const fpcg_plan* p, const fpcg_plan::Class& c) {
  (void)p;
  if (fpcg::two_pass_capable(c.k, c.L, &c.prec)) return FPCG_PATH_TWO_PASS;
  return fpcg_path(c.n, c.k, c.L, &c.prec);
}

int path_of(const fpcg_plan* p, const fpcg_plan::Class& c) { return c.path >= 0 ? c.path : default_path(p, c); }

// Device workspace for the two-pass classes (before any capture; grows only).
int ensure_workspace(fpcg_plan* p) {
  if (p->ws) return FPCG_OK;
  int64_t a = 0, b = 0;
  for (auto& c : p->cls) {
    if (!fpcg::two_pass_capable(c.k, c.L, &c.prec)) continue;
    c.a0 = a;
    c.b0 = b;
    a += c.count * (int64_t)c.k * c.k;
    b += c.count * (int64_t)c.k;
  }
  if (a == 0) return FPCG_OK;
  p->ws_a = a;
  const cudaError_t e = cudaMalloc(&p->ws, sizeof(float2) * (size_t)(a + b));
  if (e != cudaSuccess) {
    p->ws = nullptr;
    return e == cudaErrorMemoryAllocation ? FPCG_ENOMEM : fpcg::cuda_error(e);
  }
  return FPCG_OK;
}

// One class on `s` with the given path.
int run_class(fpcg_plan* p, const fpcg_plan::Class& c, int path, const void* H, const void* y, const double* sigma2,
              const int32_t* qam, void* x_hat, uint8_t* sym, double* rel_res, const uint8_t* tx,
              unsigned long long* bits, int32_t* status, cudaStream_t s) {
  const float2* Hc = static_cast<const float2*>(H) + c.h0;
  const float2* yc = static_cast<const float2*>(y) + c.y0;
  float2* xc = static_cast<float2*>(x_hat) + c.x0;
  if (path == FPCG_PATH_TWO_PASS) {
    float2* A = p->ws + c.a0;
    float2* bv = p->ws + p->ws_a + c.b0;
    int rc = fpcg_gram(Hc, yc, sigma2 + c.first, c.n, c.k, c.count, c.prec.gram, A, bv,
                       status ? status + c.first : nullptr, s);
    if (rc) return rc;
    return fpcg::run_uniform(nullptr, nullptr, nullptr, qam ? qam + c.first : nullptr, A, bv, c.k, c.k, c.count,
                             p->iters, c.L, &c.prec, xc, sym ? sym + c.x0 : nullptr,
                             rel_res ? rel_res + c.first : nullptr, nullptr, tx ? tx + c.x0 : nullptr, bits,
                             status ? status + c.first : nullptr, s, FPCG_PATH_TENSOR_CORE, false,
                             true);  // keep a Gram-pass FPCG_ST_TIMEOUT
  }
  return fpcg::run_uniform(Hc, yc, sigma2 + c.first, qam ? qam + c.first : nullptr, nullptr, nullptr, c.n, c.k,
                           c.count, p->iters, c.L, &c.prec, xc, sym ? sym + c.x0 : nullptr,
                           rel_res ? rel_res + c.first : nullptr, nullptr, tx ? tx + c.x0 : nullptr, bits,
                           status ? status + c.first : nullptr, s, path, false, false, nullptr, c.ncg);
}

// A class that may share one launch of the fused kernel with others: the
// fused kernel's path and K, a 16-bit matvec.
bool groupable(const fpcg_plan* p, const fpcg_plan::Class& c) {
  return !(p->flags & FPCG_PLAN_PER_CLASS) && path_of(p, c) == FPCG_PATH_TENSOR_CORE &&
         (c.k == 16 || c.k == 32 || c.k == 64) && (c.prec.mv == FPCG_BF16 || c.prec.mv == FPCG_FP16);
}

bool same_launch(const fpcg_plan::Class& a, const fpcg_plan::Class& b) {
  return a.L == b.L && std::memcmp(&a.prec, &b.prec, sizeof(fpcg_precision)) == 0;
}

fpcg::FusedClass fused_class(const fpcg_plan::Class& c, const void* H, const void* y, const double* sigma2,
                             const int32_t* qam, void* x_hat, uint8_t* sym, double* rel_res, const uint8_t* tx,
                             int32_t* status) {
  fpcg::FusedClass f;
  f.H = static_cast<const float2*>(H) + c.h0;
  f.y = static_cast<const float2*>(y) + c.y0;
  f.sigma2 = sigma2 + c.first;
  f.qam = qam ? qam + c.first : nullptr;
  f.n = c.n;
  f.k = c.k;
  f.batch = c.count;
  f.x_hat = static_cast<float2*>(x_hat) + c.x0;
  f.sym = sym ? sym + c.x0 : nullptr;
  f.rel_res = rel_res ? rel_res + c.first : nullptr;
  f.tx = tx ? tx + c.x0 : nullptr;
  f.status = status ? status + c.first : nullptr;
  f.cg_warps = c.ncg;
  return f;
}

// Launch index of every class within one run: the fused classes of the same
// block size and precisions share one (up to ten per launch), every other
// class has its own.
std::vector<int32_t> launch_ids(const fpcg_plan* p) {
  std::vector<int32_t> id(p->cls.size(), -1);
  int32_t next = 0;
  for (size_t i = 0; i < p->cls.size(); ++i) {
    if (id[i] >= 0) continue;
    id[i] = next;
    if (groupable(p, p->cls[i])) {
      int members = 1;
      for (size_t j = i + 1; j < p->cls.size() && members < fpcg::kFusedMultiMax; ++j)
        if (id[j] < 0 && groupable(p, p->cls[j]) && same_launch(p->cls[i], p->cls[j])) {
          id[j] = next;
          ++members;
        }
    }
    ++next;
  }
  return id;
}

// Issues every class on `s`; bit_errors is zeroed once.  Classes that share a
// launch index run in one launch of the fused kernel (each class on its own if
// the data of one of them does not allow it).
int enqueue(fpcg_plan* p, const void* H, const void* y, const double* sigma2, const int32_t* qam,
            void* x_hat, uint8_t* sym, double* rel_res, const uint8_t* tx, unsigned long long* bits,
            int32_t* status, cudaStream_t s) {
  if (bits) {
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return fpcg::cuda_error(e);
  }
  const std::vector<int32_t> id = launch_ids(p);
  std::vector<bool> done(p->cls.size(), false);
  for (size_t i = 0; i < p->cls.size(); ++i) {
    if (done[i]) continue;
    const auto& c = p->cls[i];
    std::vector<size_t> members;
    for (size_t j = i; j < p->cls.size(); ++j)
      if (id[j] == id[i]) members.push_back(j);
    if (members.size() >= 2) {
      std::vector<fpcg::FusedClass> f;
      bool ok = true;
      for (size_t j : members) {
        f.push_back(fused_class(p->cls[j], H, y, sigma2, qam, x_hat, sym, rel_res, tx, status));
        ok = ok && fpcg::fused_multi_capable(f.back(), c.L, &c.prec);
      }
      if (ok) {
        const int rc = fpcg::run_fused_multi(f.data(), (int)f.size(), p->iters, c.L, &c.prec, bits, s);
        if (rc) return rc;
        for (size_t j : members) done[j] = true;
        continue;
      }
    }
    const int rc = run_class(p, c, path_of(p, c), H, y, sigma2, qam, x_hat, sym, rel_res, tx, bits, status, s);
    if (rc) return rc;
    done[i] = true;
  }
  return FPCG_OK;
}

}  // namespace

extern "C" {

int fpcg_plan_create(const fpcg_batch_desc* d, fpcg_plan** out) {
  if (!d || !out) return FPCG_EINVAL;
  *out = nullptr;
  if (d->batch < 0 || d->iters < 0 || d->block_L < 0 || d->block_L > 32) return FPCG_EINVAL;
  if (d->batch > 0 && (!d->n_rx || !d->k)) return FPCG_EINVAL;
  if (fpcg::check_precision(&d->prec)) return FPCG_EINVAL;
  for (int64_t i = 0; i < d->batch; ++i) {
    const int32_t n = d->n_rx[i], k = d->k[i];
    if (k < 1 || k > 128 || n < k || n > 65536) return FPCG_EINVAL;
    if (d->block_L > 0) {
      const int32_t L = std::min(d->block_L, k);
      if (k % L) return FPCG_EINVAL;
    }
  }
  fpcg_plan* p = new (std::nothrow) fpcg_plan;
  if (!p) return FPCG_ENOMEM;
  try {
    p->iters = d->iters;
    p->flags = d->flags;
    p->prec = d->prec;
    // classes sorted by (K, N); caller order kept inside a class
    std::vector<int64_t> idx((size_t)d->batch);
    for (int64_t i = 0; i < d->batch; ++i) idx[(size_t)i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
      return d->k[a] != d->k[b] ? d->k[a] < d->k[b] : d->n_rx[a] < d->n_rx[b];
    });
    p->order = idx;
    p->h_off.resize((size_t)d->batch);
    p->y_off.resize((size_t)d->batch);
    p->x_off.resize((size_t)d->batch);
    int64_t h = 0, yv = 0, x = 0;
    for (int64_t pos = 0; pos < d->batch; ++pos) {
      const int64_t i = idx[(size_t)pos];
      const int32_t n = d->n_rx[i], k = d->k[i];
      if (p->cls.empty() || p->cls.back().n != n || p->cls.back().k != k) {
        fpcg_plan::Class c;
        c.n = n;
        c.k = k;
        c.L = d->block_L > 0 ? std::min(d->block_L, k) : 0;
        c.prec = d->prec;
        c.path = -1;
        c.first = pos;
        c.count = 0;
        c.a0 = c.b0 = 0;
        c.h0 = h = align_up(h);
        c.y0 = yv = align_up(yv);
        c.x0 = x = align_up(x);
        p->cls.push_back(c);
      }
      p->cls.back().count++;
      p->h_off[(size_t)pos] = h;
      p->y_off[(size_t)pos] = yv;
      p->x_off[(size_t)pos] = x;
      h += (int64_t)n * k;
      yv += n;
      x += k;
    }
    p->tot[0] = align_up(h);
    p->tot[1] = align_up(yv);
    p->tot[2] = align_up(x);
  } catch (const std::bad_alloc&) {
    delete p;
    return FPCG_ENOMEM;
  }
  *out = p;
  return FPCG_OK;
}

int fpcg_plan_layout(const fpcg_plan* p, int64_t* order, int64_t* h_off, int64_t* y_off, int64_t* x_off,
                     int64_t totals[3]) {
  if (!p) return FPCG_EINVAL;
  const size_t n = p->order.size();
  if (order) std::copy(p->order.begin(), p->order.end(), order);
  if (h_off) std::copy(p->h_off.begin(), p->h_off.end(), h_off);
  if (y_off) std::copy(p->y_off.begin(), p->y_off.end(), y_off);
  if (x_off) std::copy(p->x_off.begin(), p->x_off.end(), x_off);
  if (totals) std::copy(p->tot, p->tot + 3, totals);
  (void)n;
  return FPCG_OK;
}

int fpcg_plan_classes(const fpcg_plan* p, int32_t* n_classes, fpcg_class_info* info) {
  if (!p || !n_classes) return FPCG_EINVAL;
  *n_classes = (int32_t)p->cls.size();
  if (info) {
    const std::vector<int32_t> ids = launch_ids(p);
    for (size_t c = 0; c < p->cls.size(); ++c) {
      const auto& k = p->cls[c];
      info[c].n_rx = k.n;
      info[c].k = k.k;
      info[c].block_L = k.L;
      info[c].path = path_of(p, k);
      info[c].first = k.first;
      info[c].count = k.count;
      info[c].mv = k.prec.mv;
      info[c].launch = ids[c];
      info[c].cg_warps = info[c].path == FPCG_PATH_TENSOR_CORE ? fpcg::fused_cg_warps(k.k, k.n, k.ncg) : 0;
      info[c].reserved = 0;
      info[c].kappa = k.kappa;
    }
  }
  return FPCG_OK;
}

int fpcg_plan_autotune(fpcg_plan* p, const void* H, const void* y, const double* sigma2, const int32_t* qam,
                       void* x_hat, uint8_t* sym, double* rel_res, int32_t* status, void* stream) {
  if (!p || !H || !y || !sigma2 || !x_hat) return FPCG_EINVAL;
  if (sym && !qam) return FPCG_EINVAL;
  drop_graph(p);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fpcg::cuda_error(ce);
  }
  int rc = ensure_workspace(p);
  for (auto& c : p->cls) {
    if (rc) break;
    int cand[2] = {-1, FPCG_PATH_SIMT};
    if (fpcg::two_pass_capable(c.k, c.L, &c.prec)) cand[0] = FPCG_PATH_TWO_PASS;
    else if (fpcg::tc_capable(c.k, c.L, &c.prec) && c.n % 2 == 0) cand[0] = FPCG_PATH_TENSOR_CORE;
    if (cand[0] < 0) {
      c.path = FPCG_PATH_SIMT;
      continue;
    }
    // candidates: (path, CG warps of the fused kernel); K <= 32 on the fused
    // kernel tries both six and eight CG warps per CTA
    int cpath[3], cncg[3], nc = 0;
    cpath[nc] = cand[0];
    cncg[nc++] = 0;
    if (cand[0] == FPCG_PATH_TENSOR_CORE && c.k <= 32) {
      cncg[0] = 6;
      cpath[nc] = FPCG_PATH_TENSOR_CORE;
      cncg[nc++] = 8;
    }
    cpath[nc] = FPCG_PATH_SIMT;
    cncg[nc++] = 0;
    float best = -1.f;
    int best_path = cand[0], best_ncg = 0;
    for (int ci = 0; ci < nc; ++ci) {
      const int path = cpath[ci];
      c.ncg = cncg[ci];
      float ms = 0.f;
      for (int rep = 0; rep < 4 && rc == FPCG_OK; ++rep) {  // one warm-up, three timed
        if (rep == 1) cudaEventRecord(e0, s);
        rc = run_class(p, c, path, H, y, sigma2, qam, x_hat, sym, rel_res, nullptr, nullptr, status, s);
      }
      if (rc == FPCG_ENOTSUP && path != FPCG_PATH_SIMT) {  // e.g. unaligned data
        rc = FPCG_OK;
        continue;
      }
      if (rc) break;
      cudaEventRecord(e1, s);
      ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) {
        rc = fpcg::cuda_error(ce);
        break;
      }
      cudaEventElapsedTime(&ms, e0, e1);
      if (best < 0.f || ms < best) {
        best = ms;
        best_path = path;
        best_ncg = cncg[ci];
      }
    }
    if (rc) break;
    c.path = best_path;
    c.ncg = best_ncg;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int fpcg_plan_autoprec(fpcg_plan* p, const void* H, const void* y, const double* sigma2, double tol, void* stream) {
  if (!p || !H || !y || !sigma2 || !(tol > 0.0 && tol < 1.0)) return FPCG_EINVAL;
  constexpr int64_t kSample = 64;
  constexpr int kMaxIters = 32;
  cudaStream_t s = (cudaStream_t)stream;
  drop_graph(p);
  if (p->ws) {  // two-pass eligibility may change with the precisions: the workspace is laid out again
    cudaStreamSynchronize(s);
    cudaFree(p->ws);
    p->ws = nullptr;
  }
  int kmax = 1;
  for (const auto& c : p->cls) kmax = std::max(kmax, c.k);
  float* coeffs = nullptr;
  float2* xs = nullptr;
  cudaError_t e = cudaMalloc(&coeffs, sizeof(float) * 2 * kMaxIters * kSample);
  if (e == cudaSuccess) e = cudaMalloc(&xs, sizeof(float2) * (size_t)kmax * kSample);
  if (e != cudaSuccess) {
    cudaFree(coeffs);
    return e == cudaErrorMemoryAllocation ? FPCG_ENOMEM : fpcg::cuda_error(e);
  }
  std::vector<float> host((size_t)2 * kMaxIters * kSample);
  std::vector<double> kap((size_t)kSample);
  int rc = FPCG_OK;
  // the estimate of kappa (FP-CG) or kappa_bar (FP-BJ-CG, block L): median over
  // the first systems of the class of the Ritz-value estimate from fp32 CG step sizes
  auto estimate = [&](const fpcg_plan::Class& c, int L, double* out) -> int {
    const int64_t n = std::min<int64_t>(c.count, kSample);
    const int m = std::min(c.k, kMaxIters);
    fpcg_precision pe = p->prec;
    pe.gram = pe.mv = pe.ip = pe.w = pe.resid = FPCG_FP32;
    pe.refine_steps = 0;
    int r = fpcg::run_uniform(static_cast<const float2*>(H) + c.h0, static_cast<const float2*>(y) + c.y0,
                              sigma2 + c.first, nullptr, nullptr, nullptr, c.n, c.k, n, m, L, &pe, xs, nullptr,
                              nullptr, nullptr, nullptr, nullptr, nullptr, s, -1, true, false, coeffs);
    if (r) return r;
    cudaError_t ce = cudaMemcpyAsync(host.data(), coeffs, sizeof(float) * 2 * m * n, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return fpcg::cuda_error(ce);
    fpcg_kappa_cg_batch(host.data(), m, m, n, kap.data());
    std::vector<double> v;
    for (int64_t i = 0; i < n; ++i)
      if (kap[(size_t)i] >= 1.0) v.push_back(kap[(size_t)i]);
    if (v.empty()) {
      *out = 1.0;
      return FPCG_OK;
    }
    std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
    *out = v[v.size() / 2];
    return FPCG_OK;
  };
  for (auto& c : p->cls) {
    double kappa = 1.0, kappa_bar = 1.0;
    rc = estimate(c, 0, &kappa);
    if (!rc && c.L > 0) rc = estimate(c, c.L, &kappa_bar);
    if (rc) break;
    // eq. heuristic / eq. heuristic_bj; the matvec never goes above the fp32 working precision
    auto pick = [&](double k) {
      const int f = fpcg_choose_precision(c.k, k, nullptr);
      return f == FPCG_FP64 || f < 0 ? FPCG_FP32 : f;
    };
    const int mv_cg = pick(kappa), mv_bj = pick(kappa_bar);
    int L = 0;
    if (c.L > 0) L = fpcg_choose_method(c.k, c.L, kappa, kappa_bar, tol, mv_cg, mv_bj, FPCG_FP32, nullptr, nullptr);
    if (L < 0) L = c.L;
    c.L = L;
    c.prec.mv = L ? mv_bj : mv_cg;
    c.kappa = L ? kappa_bar : kappa;
    c.path = -1;
  }
  cudaFree(coeffs);
  cudaFree(xs);
  return rc;
}

int fpcg_plan_run(fpcg_plan* p, const void* H, const void* y, const double* sigma2, const int32_t* qam,
                  void* x_hat, uint8_t* sym, double* rel_res, const uint8_t* tx, unsigned long long* bits,
                  int32_t* status, void* stream) {
  if (!p) return FPCG_EINVAL;
  if (!p->cls.empty() && (!H || !y || !sigma2 || !x_hat)) return FPCG_EINVAL;
  if ((sym || bits) && !qam) return FPCG_EINVAL;
  if ((tx != nullptr) != (bits != nullptr)) return FPCG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!(p->flags & FPCG_PLAN_GRAPH)) {
    const int wrc = ensure_workspace(p);
    if (wrc) return wrc;
    return enqueue(p, H, y, sigma2, qam, x_hat, sym, rel_res, tx, bits, status, s);
  }
  const int wrc = ensure_workspace(p);
  if (wrc) return wrc;
  const int prc = fpcg::prepare_fused_pools(s);  // the capture below uses the addresses found now
  if (prc) return prc;
  const void* key[10] = {H, y, sigma2, qam, x_hat, sym, rel_res, tx, bits, status};
  if (p->exec && !std::equal(key, key + 10, p->key)) drop_graph(p);
  if (!p->exec) {
    cudaError_t e = cudaSuccess;
    if (!p->cap) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fpcg::cuda_error(e);
    e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fpcg::cuda_error(e);
    const int rc = enqueue(p, H, y, sigma2, qam, x_hat, sym, rel_res, tx, bits, status, p->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(p->cap, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fpcg::cuda_error(e);
    e = cudaGraphInstantiate(&p->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      p->exec = nullptr;
      return fpcg::cuda_error(e);
    }
    std::copy(key, key + 10, p->key);
  }
  const cudaError_t e = cudaGraphLaunch(p->exec, s);
  return e == cudaSuccess ? FPCG_OK : fpcg::cuda_error(e);
}

int fpcg_plan_destroy(fpcg_plan* p) {
  if (!p) return FPCG_OK;
  drop_graph(p);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->ws) cudaFree(p->ws);
  delete p;
  return FPCG_OK;
}

}  // extern "C"
