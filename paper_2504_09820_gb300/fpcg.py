"""ctypes binding of libfpcg (include/fpcg.h).

The functions named like the C entry points (fpcg_detect, fpbjcg_detect,
fpcg_solve_gram, fpcg_strerror, ...) only marshal arguments: torch CUDA
tensors become device pointers, the current torch stream becomes the
cudaStream_t, and a non-zero return code becomes an exception.  Every step of
the detection runs in the library's kernels; there is no Python or CPU
fallback, and a missing library raises.

``detect`` is a convenience wrapper that allocates the outputs and calls
fpcg_detect or fpbjcg_detect.
"""
import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfpcg.so")

# format codes (FPCG_* in fpcg.h)
FP64, FP32, FP16, BF16, FP8E4M3 = 0, 1, 2, 3, 4
FORMAT = {"fp64": FP64, "fp32": FP32, "fp16": FP16, "bf16": BF16, "e4m3": FP8E4M3, "fp8": FP8E4M3}

# status bits (FPCG_ST_*)
ST_BREAKDOWN, ST_RHO_ZERO, ST_NONFINITE, ST_BJ_FAIL, ST_BAD_QAM, ST_TIMEOUT, ST_BAD_INDEX = 1, 2, 4, 8, 16, 32, 64

# return codes
OK, EINVAL, ENOTSUP, ECUDA, ENOMEM = 0, 1, 2, 3, 4


class FpcgError(RuntimeError):
    def __init__(self, code, where):
        msg = f"{where}: {fpcg_strerror(code)} (code {code})"
        if code == ECUDA:
            msg += ": " + fpcg_last_cuda_error()
        super().__init__(msg)
        self.code = code


class Precision(ctypes.Structure):
    _fields_ = [("gram", ctypes.c_int32), ("mv", ctypes.c_int32), ("ip", ctypes.c_int32),
                ("w", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("refine_iters", ctypes.c_int32), ("alpha_num", ctypes.c_int32),
                ("fp8_block", ctypes.c_int32), ("resid", ctypes.c_int32)]


# resid: "fp64" = refinement residual and rel_res against the fp32 Gram matrix,
# "fp32" = against the matvec-format matrix (see fpcg_precision in fpcg.h)
DEFAULT_RESID = "fp32"


def precision(gram="fp32", mv="fp32", ip="fp32", w="fp32", refine_steps=0, refine_iters=-1,
              alpha_num=0, fp8_block=32, resid=DEFAULT_RESID):
    """Build an fpcg_precision from format names ("fp64", "fp32", "fp16", "bf16", "e4m3")."""
    if w == "fp64":
        gram = mv = ip = resid = "fp64"
    return Precision(FORMAT[gram], FORMAT[mv], FORMAT[ip], FORMAT[w], int(refine_steps),
                     int(refine_iters), int(alpha_num), int(fp8_block), FORMAT[resid])


class BatchDesc(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int64), ("n_rx", ctypes.c_void_p), ("k", ctypes.c_void_p),
                ("iters", ctypes.c_int32), ("block_L", ctypes.c_int32), ("prec", Precision),
                ("flags", ctypes.c_int32)]


class ClassInfo(ctypes.Structure):
    _fields_ = [("n_rx", ctypes.c_int32), ("k", ctypes.c_int32), ("block_L", ctypes.c_int32),
                ("path", ctypes.c_int32), ("first", ctypes.c_int64), ("count", ctypes.c_int64),
                ("mv", ctypes.c_int32), ("launch", ctypes.c_int32), ("kappa", ctypes.c_double),
                ("cg_warps", ctypes.c_int32), ("reserved", ctypes.c_int32)]


PLAN_GRAPH = 1
PLAN_PER_CLASS = 2

_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


def lib():
    """Load libfpcg.so (built in-tree by build.py); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2504_09820_gb300.build.build() (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        det = [_P, _P, _P, _P, _I32, _I32, _I64, _I32]
        outs = [_P, _P, _P, _P, _P, _P, _P, _P]
        L.fpcg_detect.argtypes = det + [ctypes.POINTER(Precision)] + outs
        L.fpcg_detect.restype = ctypes.c_int
        L.fpbjcg_detect.argtypes = det + [_I32, ctypes.POINTER(Precision)] + outs
        L.fpbjcg_detect.restype = ctypes.c_int
        L.fpcg_solve_gram.argtypes = [_P, _P, _I32, _I64, _I32, _I32, ctypes.POINTER(Precision),
                                      _P, _P, _P, _P, _P]
        L.fpcg_solve_gram.restype = ctypes.c_int
        L.fpcg_gram.argtypes = [_P, _P, _P, _I32, _I32, _I64, _I32, _P, _P, _P, _P]
        L.fpcg_gram.restype = ctypes.c_int
        L.fpcg_path.argtypes = [_I32, _I32, _I32, ctypes.POINTER(Precision)]
        L.fpcg_path.restype = ctypes.c_int
        L.fpcg_strerror.argtypes = [ctypes.c_int]
        L.fpcg_strerror.restype = ctypes.c_char_p
        L.fpcg_last_cuda_error.argtypes = []
        L.fpcg_last_cuda_error.restype = ctypes.c_char_p
        L.fpcg_version.argtypes = []
        L.fpcg_version.restype = ctypes.c_int
        L.fpcg_detect_shared.argtypes = [_P, _P, _P, _P, _P, _I32, _I32, _I64, _I64, _I32, _I32,
                                         ctypes.POINTER(Precision), _P, _P, _P, _P, _P, _P, _P]
        L.fpcg_detect_shared.restype = ctypes.c_int
        L.fpcg_detect_grouped.argtypes = [_P, _P, _P, _P, _P, _I32, _I32, _I64, _I64, _I32, _I32,
                                          ctypes.POINTER(Precision), _P, _P, _P, _P, _P, _P, _P]
        L.fpcg_detect_grouped.restype = ctypes.c_int
        L.fpcg_choose_precision.argtypes = [_I32, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
        L.fpcg_choose_precision.restype = ctypes.c_int
        L.fpcg_kappa_cg.argtypes = [_P, _P, _I32, ctypes.POINTER(ctypes.c_double)]
        L.fpcg_kappa_cg.restype = ctypes.c_int
        L.fpcg_detect_noalloc.argtypes = det + [_I32, ctypes.POINTER(Precision)] + outs
        L.fpcg_detect_noalloc.restype = ctypes.c_int
        L.fpcg_plan_create.argtypes = [ctypes.POINTER(BatchDesc), ctypes.POINTER(ctypes.c_void_p)]
        L.fpcg_plan_create.restype = ctypes.c_int
        L.fpcg_plan_layout.argtypes = [_P, _P, _P, _P, _P, _P]
        L.fpcg_plan_layout.restype = ctypes.c_int
        L.fpcg_plan_classes.argtypes = [_P, ctypes.POINTER(_I32), _P]
        L.fpcg_plan_classes.restype = ctypes.c_int
        L.fpcg_plan_autotune.argtypes = [_P] * 10
        L.fpcg_plan_autotune.restype = ctypes.c_int
        L.fpcg_plan_run.argtypes = [_P] * 12
        L.fpcg_plan_run.restype = ctypes.c_int
        L.fpcg_plan_destroy.argtypes = [_P]
        L.fpcg_plan_destroy.restype = ctypes.c_int
        L.fpcg_plan_autoprec.argtypes = [_P, _P, _P, _P, ctypes.c_double, _P]
        L.fpcg_plan_autoprec.restype = ctypes.c_int
        L.fpcg_detect_coeffs.argtypes = det + [_I32, ctypes.POINTER(Precision)] + [_P, _P, _P, _P, _P, _P, _P, _P]
        L.fpcg_detect_coeffs.restype = ctypes.c_int
        L.fpcg_kappa_cg_batch.argtypes = [_P, _I32, _I32, _I64, _P]
        L.fpcg_kappa_cg_batch.restype = ctypes.c_int
        L.fpcg_choose_method.argtypes = [_I32, _I32, ctypes.c_double, ctypes.c_double, ctypes.c_double, _I32, _I32,
                                         _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]
        L.fpcg_choose_method.restype = ctypes.c_int
        L.fpcg_fma_probe.argtypes = [_I32, _I64, _P, _I64, ctypes.POINTER(ctypes.c_double), _P]
        L.fpcg_fma_probe.restype = ctypes.c_int
        _lib = L
    return _lib


PATH_SIMT, PATH_TENSOR_CORE, PATH_TWO_PASS = 0, 1, 2


def fpcg_path(N, K, block_L, prec):
    """Which kernel a detection call with these settings uses (no GPU needed)."""
    rc = lib().fpcg_path(int(N), int(K), int(block_L or 0), ctypes.byref(prec))
    if rc < 0:
        raise FpcgError(-rc, "fpcg_path")
    return rc


FORMAT_NAME = {v: k for k, v in FORMAT.items() if k != "fp8"}


def fpcg_choose_precision(K, kappa):
    """(format name, u bound) of the heuristic of Sections III-B and IV-B (host only)."""
    u = ctypes.c_double()
    rc = lib().fpcg_choose_precision(int(K), float(kappa), ctypes.byref(u))
    if rc < 0:
        raise FpcgError(-rc, "fpcg_choose_precision")
    return FORMAT_NAME[rc], u.value


def fpcg_kappa_cg(alpha, beta):
    """kappa estimate from CG step sizes alpha[0..m-1], beta[0..m-2] (host only)."""
    import numpy as np
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    out = ctypes.c_double()
    _check(lib().fpcg_kappa_cg(a.ctypes.data, b.ctypes.data if b.size else None, int(a.size), ctypes.byref(out)),
           "fpcg_kappa_cg")
    return out.value


def fpcg_kappa_cg_batch(coeffs, m=None):
    """kappa estimates of every system from a host [batch][2][iters] float32
    coefficient array (fpcg_detect_coeffs's layout) using the first m steps."""
    import numpy as np
    c = np.ascontiguousarray(coeffs, dtype=np.float32)
    batch, two, iters = c.shape
    out = np.empty(batch, dtype=np.float64)
    _check(lib().fpcg_kappa_cg_batch(c.ctypes.data, int(iters), int(m or iters), int(batch), out.ctypes.data),
           "fpcg_kappa_cg_batch")
    return out


def fpcg_choose_method(K, L, kappa, kappa_bar, tol, mv_cg="fp16", mv_bj="fp16", w="fp32"):
    """(block size to use: L or 0 for FP-CG, k_cg, k_pcg): Remark 4's break-even (host only)."""
    kc, kp = _I32(), _I32()
    rc = lib().fpcg_choose_method(int(K), int(L), float(kappa), float(kappa_bar), float(tol), FORMAT[mv_cg],
                                  FORMAT[mv_bj], FORMAT[w], ctypes.byref(kc), ctypes.byref(kp))
    if rc < 0:
        raise FpcgError(-rc, "fpcg_choose_method")
    return rc, kc.value, kp.value


def fpcg_detect_coeffs(H, y, sigma2, qam_order, iters, block_L, prec, x_hat, coeffs, sym_idx=None, rel_res=None,
                       tx_idx=None, bit_errors=None, status=None, stream=None):
    """Marshal a call to fpcg_detect_coeffs (coeffs: float32 [batch][2][iters] on the device)."""
    a, b = _detect_args(H, y, sigma2, qam_order, iters, prec, x_hat, sym_idx, rel_res, None,
                        tx_idx, bit_errors, status)
    b = [b[0], b[1], b[2], b[3], b[5], b[6], b[7]]   # no res_hist
    _check(lib().fpcg_detect_coeffs(*a, int(block_L or 0), *b, _ptr(coeffs, torch.float32, "coeffs"),
                                    _stream(stream)), "fpcg_detect_coeffs")


def fpcg_strerror(code):
    return lib().fpcg_strerror(int(code)).decode()


def fpcg_last_cuda_error():
    return lib().fpcg_last_cuda_error().decode()


def fpcg_fma_probe(fp64, iters, out, stream=None):
    """Launch the FMA throughput probe on `out` (a CUDA float32 or float64
    tensor, a multiple of 256 elements); returns the launch's flop count."""
    f = ctypes.c_double(0.0)
    dt = torch.float64 if fp64 else torch.float32
    _check(lib().fpcg_fma_probe(1 if fp64 else 0, int(iters), _ptr(out, dt, "out"), int(out.numel()),
                                ctypes.byref(f), _stream(stream)), "fpcg_fma_probe")
    return f.value


def fpcg_version():
    return lib().fpcg_version()


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _xdtype(prec):
    return torch.complex128 if prec.w == FP64 else torch.complex64


def _check(rc, where):
    if rc != OK:
        raise FpcgError(rc, where)


def _detect_args(H, y, sigma2, qam_order, iters, prec, x_hat, sym_idx, rel_res, res_hist,
                 tx_idx, bit_errors, status):
    if H.dim() != 3:
        raise ValueError("H must be [batch][K][N]")
    batch, K, N = H.shape
    return [_ptr(H, torch.complex64, "H"), _ptr(y, torch.complex64, "y"),
            _ptr(sigma2, torch.float64, "sigma2"), _ptr(qam_order, torch.int32, "qam_order"),
            int(N), int(K), int(batch), int(iters)], \
           [ctypes.byref(prec), _ptr(x_hat, _xdtype(prec), "x_hat"),
            _ptr(sym_idx, torch.uint8, "sym_idx"), _ptr(rel_res, torch.float64, "rel_res"),
            _ptr(res_hist, torch.float32, "res_hist"), _ptr(tx_idx, torch.uint8, "tx_idx"),
            _ptr(bit_errors, torch.int64, "bit_errors"), _ptr(status, torch.int32, "status")]


def fpcg_detect(H, y, sigma2, qam_order, iters, prec, x_hat, sym_idx=None, rel_res=None,
                res_hist=None, tx_idx=None, bit_errors=None, status=None, stream=None):
    """Marshal a call to fpcg_detect (FP-CG, Algorithm 2); tensors on the GPU."""
    a, b = _detect_args(H, y, sigma2, qam_order, iters, prec, x_hat, sym_idx, rel_res, res_hist,
                        tx_idx, bit_errors, status)
    _check(lib().fpcg_detect(*a, *b, _stream(stream)), "fpcg_detect")


def fpbjcg_detect(H, y, sigma2, qam_order, iters, block_L, prec, x_hat, sym_idx=None,
                  rel_res=None, res_hist=None, tx_idx=None, bit_errors=None, status=None,
                  stream=None):
    """Marshal a call to fpbjcg_detect (FP-BJ-CG, Algorithm 3)."""
    a, b = _detect_args(H, y, sigma2, qam_order, iters, prec, x_hat, sym_idx, rel_res, res_hist,
                        tx_idx, bit_errors, status)
    _check(lib().fpbjcg_detect(*a, int(block_L), *b, _stream(stream)), "fpbjcg_detect")


def fpcg_detect_noalloc(H, y, sigma2, qam_order, iters, block_L, prec, x_hat, sym_idx=None, rel_res=None,
                        res_hist=None, tx_idx=None, bit_errors=None, status=None, stream=None):
    """Marshal a call to fpcg_detect_noalloc (no device allocation; block_L 0 = FP-CG)."""
    a, b = _detect_args(H, y, sigma2, qam_order, iters, prec, x_hat, sym_idx, rel_res, res_hist,
                        tx_idx, bit_errors, status)
    _check(lib().fpcg_detect_noalloc(*a, int(block_L or 0), *b, _stream(stream)), "fpcg_detect_noalloc")


def fpcg_solve_gram(A, b, iters, block_L, prec, x_hat, rel_res=None, res_hist=None, status=None,
                    stream=None):
    """Marshal a call to fpcg_solve_gram (A, b given; Algorithms 2/3)."""
    batch, K, _ = A.shape
    dt = _xdtype(prec)
    _check(lib().fpcg_solve_gram(_ptr(A, dt, "A"), _ptr(b, dt, "b"), int(K), int(batch),
                                 int(iters), int(block_L), ctypes.byref(prec),
                                 _ptr(x_hat, dt, "x_hat"), _ptr(rel_res, torch.float64, "rel_res"),
                                 _ptr(res_hist, torch.float32, "res_hist"),
                                 _ptr(status, torch.int32, "status"), _stream(stream)),
           "fpcg_solve_gram")


def fpcg_gram(H, y, sigma2, gram, A, b, status=None, stream=None):
    """Marshal a call to fpcg_gram (A = fl(H)^H fl(H) + sigma^2 I, b = fl(H)^H fl(y))."""
    batch, K, N = H.shape
    dt = torch.complex128 if FORMAT[gram] == FP64 else torch.complex64
    _check(lib().fpcg_gram(_ptr(H, torch.complex64, "H"), _ptr(y, torch.complex64, "y"),
                           _ptr(sigma2, torch.float64, "sigma2"), int(N), int(K), int(batch),
                           FORMAT[gram], _ptr(A, dt, "A"), _ptr(b, dt, "b"),
                           _ptr(status, torch.int32, "status"), _stream(stream)), "fpcg_gram")


def fpcg_detect_shared(A, H, y, rb_index, qam_order, iters, block_L, prec, x_hat, sym_idx=None,
                       rel_res=None, tx_idx=None, bit_errors=None, status=None, stream=None):
    """Marshal a call to fpcg_detect_shared: A [n_rb][K][K] from fpcg_gram, H
    [n_rb][K][N], y [n_rhs][N], rb_index [n_rhs] (group of each y)."""
    n_rb, K, N = H.shape
    n_rhs = y.shape[0]
    dt = _xdtype(prec)
    _check(lib().fpcg_detect_shared(_ptr(A, dt, "A"), _ptr(H, torch.complex64, "H"),
                                    _ptr(y, torch.complex64, "y"), _ptr(rb_index, torch.int32, "rb_index"),
                                    _ptr(qam_order, torch.int32, "qam_order"), int(N), int(K), int(n_rb),
                                    int(n_rhs), int(iters), int(block_L or 0), ctypes.byref(prec),
                                    _ptr(x_hat, dt, "x_hat"), _ptr(sym_idx, torch.uint8, "sym_idx"),
                                    _ptr(rel_res, torch.float64, "rel_res"), _ptr(tx_idx, torch.uint8, "tx_idx"),
                                    _ptr(bit_errors, torch.int64, "bit_errors"), _ptr(status, torch.int32, "status"),
                                    _stream(stream)), "fpcg_detect_shared")


def fpcg_detect_grouped(A, H, y, group_start, qam_order, iters, block_L, prec, x_hat, sym_idx=None,
                        rel_res=None, tx_idx=None, bit_errors=None, status=None, stream=None):
    """Marshal a call to fpcg_detect_grouped: A [n_groups][K][K] from fpcg_gram, H
    [n_groups][K][N], y [n_rhs][N] grouped, group_start [n_groups + 1] int64 (device)."""
    n_groups, K, N = H.shape
    n_rhs = y.shape[0]
    dt = _xdtype(prec)
    _check(lib().fpcg_detect_grouped(_ptr(A, dt, "A"), _ptr(H, torch.complex64, "H"),
                                     _ptr(y, torch.complex64, "y"), _ptr(group_start, torch.int64, "group_start"),
                                     _ptr(qam_order, torch.int32, "qam_order"), int(N), int(K), int(n_groups),
                                     int(n_rhs), int(iters), int(block_L or 0), ctypes.byref(prec),
                                     _ptr(x_hat, dt, "x_hat"), _ptr(sym_idx, torch.uint8, "sym_idx"),
                                     _ptr(rel_res, torch.float64, "rel_res"), _ptr(tx_idx, torch.uint8, "tx_idx"),
                                     _ptr(bit_errors, torch.int64, "bit_errors"), _ptr(status, torch.int32, "status"),
                                     _stream(stream)), "fpcg_detect_grouped")


def detect(H, y, sigma2, qam_order, iters, prec, L=None, tx_idx=None, hist=False, stream=None):
    """Allocate outputs and run fpcg_detect (L None) or fpbjcg_detect (L given).

    Returns a dict of device tensors: x, sym, rel_res, status, and bit_errors
    (when tx_idx is given) and hist (when requested).
    """
    batch, K, N = H.shape
    dev = H.device
    out = {
        "x": torch.empty((batch, K), dtype=_xdtype(prec), device=dev),
        "sym": torch.empty((batch, K), dtype=torch.uint8, device=dev),
        "rel_res": torch.empty(batch, dtype=torch.float64, device=dev),
        "status": torch.empty(batch, dtype=torch.int32, device=dev),
    }
    out["hist"] = torch.empty((batch, iters + 1), dtype=torch.float32, device=dev) if hist else None
    out["bit_errors"] = torch.zeros(1, dtype=torch.int64, device=dev) if tx_idx is not None else None
    kw = dict(sym_idx=out["sym"], rel_res=out["rel_res"], res_hist=out["hist"], tx_idx=tx_idx,
              bit_errors=out["bit_errors"], status=out["status"], stream=stream)
    if L is None:
        fpcg_detect(H, y, sigma2, qam_order, iters, prec, out["x"], **kw)
    else:
        fpbjcg_detect(H, y, sigma2, qam_order, iters, L, prec, out["x"], **kw)
    return out


class Plan:
    """An fpcg_plan over systems of different (N, K) (fpcg_plan_* in fpcg.h).

    ``n_rx`` and ``k`` are per-system sequences in the caller's order.  The
    layout (plan order, offsets, buffer sizes) is read back from the library;
    ``run`` and ``autotune`` take packed device buffers in that layout.
    """

    def __init__(self, n_rx, k, iters, prec, block_L=0, graph=False, per_class=False):
        import numpy as np
        self._n = np.ascontiguousarray(n_rx, dtype=np.int32)
        self._k = np.ascontiguousarray(k, dtype=np.int32)
        if self._n.shape != self._k.shape or self._n.ndim != 1:
            raise ValueError("n_rx and k must be 1-D and of equal length")
        self.batch = int(self._n.size)
        d = BatchDesc(self.batch, self._n.ctypes.data, self._k.ctypes.data, int(iters),
                      int(block_L or 0), prec, (PLAN_GRAPH if graph else 0) | (PLAN_PER_CLASS if per_class else 0))
        h = ctypes.c_void_p()
        _check(lib().fpcg_plan_create(ctypes.byref(d), ctypes.byref(h)), "fpcg_plan_create")
        self._h = h
        self.prec = prec
        self.order = np.empty(self.batch, dtype=np.int64)
        self.h_off = np.empty(self.batch, dtype=np.int64)
        self.y_off = np.empty(self.batch, dtype=np.int64)
        self.x_off = np.empty(self.batch, dtype=np.int64)
        tot = np.empty(3, dtype=np.int64)
        _check(lib().fpcg_plan_layout(self._h, self.order.ctypes.data, self.h_off.ctypes.data,
                                      self.y_off.ctypes.data, self.x_off.ctypes.data, tot.ctypes.data),
               "fpcg_plan_layout")
        self.totals = tuple(int(v) for v in tot)

    def pack(self, H, y, sigma2, qam_order, tx_idx=None, device="cuda"):
        """Copy per-system host arrays (caller order: H[i] (K, N), y[i] (N,),
        sigma2[i], qam_order[i], tx_idx[i] (K,)) into plan-order device buffers."""
        import numpy as np
        Hp = np.zeros(self.totals[0], dtype=np.complex64)
        yp = np.zeros(self.totals[1], dtype=np.complex64)
        txp = np.zeros(self.totals[2], dtype=np.uint8) if tx_idx is not None else None
        s2 = np.empty(self.batch, dtype=np.float64)
        q = np.empty(self.batch, dtype=np.int32)
        for pos, i in enumerate(self.order):
            h = np.asarray(H[i], dtype=np.complex64).ravel()
            Hp[self.h_off[pos]:self.h_off[pos] + h.size] = h
            v = np.asarray(y[i], dtype=np.complex64)
            yp[self.y_off[pos]:self.y_off[pos] + v.size] = v
            if txp is not None:
                t = np.asarray(tx_idx[i], dtype=np.uint8)
                txp[self.x_off[pos]:self.x_off[pos] + t.size] = t
            s2[pos] = sigma2[i]
            q[pos] = qam_order[i]
        out = {"H": torch.from_numpy(Hp).to(device), "y": torch.from_numpy(yp).to(device),
               "sigma2": torch.from_numpy(s2).to(device), "qam": torch.from_numpy(q).to(device)}
        out["tx"] = torch.from_numpy(txp).to(device) if txp is not None else None
        return out

    def unpack(self, packed, k, per_system=None):
        """Split a plan-order buffer into per-system arrays in caller order: x_hat
        or labels (offsets x_off, k[i] entries each) when per_system is None,
        else a per-system array (rel_res, status) indexed by plan position."""
        import numpy as np
        a = packed.cpu().numpy() if isinstance(packed, torch.Tensor) else np.asarray(packed)
        out = [None] * self.batch
        for pos, i in enumerate(self.order):
            out[i] = a[pos] if per_system else a[self.x_off[pos]:self.x_off[pos] + int(k[i])]
        return out

    def classes(self):
        n = _I32()
        _check(lib().fpcg_plan_classes(self._h, ctypes.byref(n), None), "fpcg_plan_classes")
        info = (ClassInfo * n.value)()
        _check(lib().fpcg_plan_classes(self._h, ctypes.byref(n), info), "fpcg_plan_classes")
        return [dict(n_rx=c.n_rx, k=c.k, block_L=c.block_L, path=c.path, first=c.first, count=c.count,
                     mv=FORMAT_NAME[c.mv], kappa=c.kappa, launch=c.launch, cg_warps=c.cg_warps) for c in info]

    def autoprec(self, H, y, sigma2, tol=1e-3, stream=None):
        """Per-class matvec format and FP-CG / FP-BJ-CG choice (fpcg_plan_autoprec)."""
        _check(lib().fpcg_plan_autoprec(self._h, _ptr(H, torch.complex64, "H"), _ptr(y, torch.complex64, "y"),
                                        _ptr(sigma2, torch.float64, "sigma2"), float(tol), _stream(stream)),
               "fpcg_plan_autoprec")

    def _bufs(self, H, y, sigma2, qam_order, x_hat, sym_idx, rel_res, status):
        return [_ptr(H, torch.complex64, "H"), _ptr(y, torch.complex64, "y"),
                _ptr(sigma2, torch.float64, "sigma2"), _ptr(qam_order, torch.int32, "qam_order"),
                _ptr(x_hat, _xdtype(self.prec), "x_hat"), _ptr(sym_idx, torch.uint8, "sym_idx"),
                _ptr(rel_res, torch.float64, "rel_res")], _ptr(status, torch.int32, "status")

    def autotune(self, H, y, sigma2, qam_order, x_hat, sym_idx=None, rel_res=None, status=None,
                 stream=None):
        a, st = self._bufs(H, y, sigma2, qam_order, x_hat, sym_idx, rel_res, status)
        _check(lib().fpcg_plan_autotune(self._h, *a, st, _stream(stream)), "fpcg_plan_autotune")

    def run(self, H, y, sigma2, qam_order, x_hat, sym_idx=None, rel_res=None, tx_idx=None,
            bit_errors=None, status=None, stream=None):
        a, st = self._bufs(H, y, sigma2, qam_order, x_hat, sym_idx, rel_res, status)
        _check(lib().fpcg_plan_run(self._h, *a, _ptr(tx_idx, torch.uint8, "tx_idx"),
                                   _ptr(bit_errors, torch.int64, "bit_errors"), st, _stream(stream)),
               "fpcg_plan_run")

    def close(self):
        if getattr(self, "_h", None):
            lib().fpcg_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
