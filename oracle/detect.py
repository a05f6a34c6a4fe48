"""Detection oracle: Gram/matched filter, direct LMMSE, CG, FP-CG, FP-BJ-CG.

Arrays are batched over independent systems (leading axis); inside one system
every step follows the paper in its order.  H is given in storage layout
(batch, K, N) -- H_arr[s, k, n] = H_s[n, k] -- so that conj(H_arr) @ H_arr^T
is H^H H.

Rounding model for the reduced-precision steps ("tensor-core model"): the
operands of a product are rounded to that step's format, the products and
their sum are formed in float64 (exact or within 2^-53), and the result is
rounded once to the accumulator format (fp32, or fp64 in the fp64 mode).
Vector updates (u_W) are one rounding of the float64 result, which is what a
fused multiply-add gives.

Readings of the paper used here (each is a choice where the text is silent or
self-inconsistent):
* alpha's denominator is p^H A p (Algorithm 2/3), not r^H A p (eq. alpha);
  both are equal in exact arithmetic.  The plain CG of Algorithm 1 keeps the
  eq. alpha form.
* phi and the Algorithm 3 rho are real in exact arithmetic; their real parts
  are used.
* Algorithm 2 recomputes r^H r at its step 5; the value carried from the
  previous iteration's step 9 is identical and is reused.
* Algorithm 3 assigns rho_{i-1} = r^H p before alpha; beta divides by that
  most recent value (alpha_num=0).  alpha_num=1 is textbook PCG (r^H z).
* The paper stores z = M_d r and the block inverses at u_W = fp64; this build
  uses the working precision of the mode (fp32 in the reduced modes).
* Breakdown (phi <= 0, rho_{i-1} == 0 or a non-finite value) freezes that
  system's iterate and sets a status bit; it never aborts the batch.
"""

import numpy as np

from .formats import fl, flc, round_matvec_operand
from . import qam as _qam

# status bits (same meaning as the C ABI's FPCG_ST_* flags)
ST_BREAKDOWN = 1      # phi <= 0 or non-finite scalar: iteration stopped
ST_RHO_ZERO = 2       # rho == 0: exact solution reached (e.g. y = 0)
ST_NONFINITE = 4      # non-finite value in the result
ST_BJ_FAIL = 8        # a diagonal block of A is not positive definite


def _c128(z):
    return np.asarray(z, dtype=np.complex128)


def _hermitian(G):
    """Symmetrise a matrix that is Hermitian in exact arithmetic."""
    return 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))


def _add_diag(G, s):
    out = G.copy()
    k = G.shape[-1]
    idx = np.arange(k)
    out[..., idx, idx] = out[..., idx, idx] + np.asarray(s)[..., None]
    return out


# ---------------------------------------------------------------------------
# Section II, eq. inversion: A_LMMSE = H^H H + sigma^2 I, b = H^H y
# ---------------------------------------------------------------------------

def gram_mf(H, y, sigma2):
    """Exact (float64) Gram matrix and matched filter of Section II."""
    Hs = _c128(H)
    G = _hermitian(np.conj(Hs) @ np.swapaxes(Hs, -1, -2))
    A = _add_diag(G, np.asarray(sigma2, dtype=np.float64))
    b = np.einsum("bkn,bn->bk", np.conj(Hs), _c128(y))
    return A, b


def gram_emul(H, y, sigma2, gram, order_seed=None):
    """Gram step at precision ``gram`` -> (A, b).

    * fp64: A = H^H H + sigma^2 I and b = H^H y exactly in float64.
    * fp32: A = fl32(H^H H), then the diagonal gets fl32(sigma^2) with one
      more rounding; b = fl32(H^H y).
    * bf16/fp16 (the reduced-precision Gram the tensor cores form): H and y
      are rounded to the format (real and imaginary parts separately), the
      products are exact and summed at fp32: A = fl32(fl_g(H)^H fl_g(H)) +
      fl32(sigma^2), b = fl32(fl_g(H)^H fl_g(y)).
    A is exactly Hermitian (only one triangle is formed and mirrored).

    order_seed (not the default model): the sums over the antennas are
    instead accumulated one term at a time in fp32, in an order drawn from
    this seed (the same for every system).  The products and every rounding
    format stay those above; only the order of the fp32 additions, which the
    tensor-core model leaves open, changes.  The spread between the two gives
    the part of a GPU-vs-oracle difference that comes from the order of
    summation alone.
    """
    Hs = _c128(H)
    ys = _c128(y)
    s2 = np.asarray(sigma2, dtype=np.float64)
    if gram == "fp64":
        return gram_mf(Hs, ys, s2)
    if gram in ("bf16", "fp16"):
        Hs = flc(Hs, gram)
        ys = flc(ys, gram)
    elif gram != "fp32":
        raise ValueError(gram)
    s2 = fl(s2, "fp32")
    if order_seed is None:
        G = flc(_hermitian(np.conj(Hs) @ np.swapaxes(Hs, -1, -2)), "fp32")
        b = flc(np.einsum("bkn,bn->bk", np.conj(Hs), ys), "fp32")
    else:
        perm = np.random.default_rng(order_seed).permutation(Hs.shape[-1])
        G = np.zeros(Hs.shape[:-1] + (Hs.shape[-2],), dtype=np.complex128)
        b = np.zeros(Hs.shape[:-1], dtype=np.complex128)
        for n in perm:
            h = Hs[..., n]                                           # (batch, K)
            G = flc(G + np.conj(h)[..., :, None] * h[..., None, :], "fp32")
            b = flc(b + np.conj(h) * ys[..., n, None], "fp32")
        G = _hermitian(G)
    A = flc(_add_diag(G, s2), "fp32")
    return A, b


# ---------------------------------------------------------------------------
# Direct LMMSE solve x = A^{-1} b by Cholesky (the reference the iterative
# detectors approximate).
# ---------------------------------------------------------------------------

def cholesky_solve(A, b):
    A = _c128(A)
    b = _c128(b)
    Lc = np.linalg.cholesky(A)                      # A = Lc Lc^H
    K = A.shape[-1]
    z = np.zeros_like(b)
    for i in range(K):                              # Lc z = b
        z[:, i] = (b[:, i] - np.einsum("bj,bj->b", Lc[:, i, :i], z[:, :i])) / Lc[:, i, i]
    x = np.zeros_like(b)
    LH = np.conj(np.swapaxes(Lc, -1, -2))
    for i in reversed(range(K)):                    # Lc^H x = z
        x[:, i] = (z[:, i] - np.einsum("bj,bj->b", LH[:, i, i + 1:], x[:, i + 1:])) / LH[:, i, i]
    return x


def lmmse(H, y, sigma2):
    A, b = gram_mf(H, y, sigma2)
    return cholesky_solve(A, b)


# ---------------------------------------------------------------------------
# Algorithm 1: CG detection, float64, x0 = 0, fixed iteration count
# ---------------------------------------------------------------------------

def cg(A, b, iters):
    """Algorithm 1 with eq. alpha / update_of_x / update_of_r / beta / update_of_p."""
    A = _c128(A)
    b = _c128(b)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    for _ in range(iters):
        Ap = np.einsum("bkl,bl->bk", A, p)
        rr = np.einsum("bk,bk->b", np.conj(r), r)
        den = np.einsum("bk,bk->b", np.conj(r), Ap)      # r^H A p  (eq. alpha)
        live = rr != 0
        alpha = np.where(live, rr / np.where(live, den, 1), 0)
        x = x + alpha[:, None] * p
        r_new = r - alpha[:, None] * Ap
        rr_new = np.einsum("bk,bk->b", np.conj(r_new), r_new)
        beta = np.where(live, rr_new / np.where(live, rr, 1), 0)
        p = r_new + beta[:, None] * p
        r = r_new
    return x


# ---------------------------------------------------------------------------
# Block-Jacobi preconditioner, eq. pre_BJ: M_d = diag(A_1^{-1}, ..., A_d^{-1})
# ---------------------------------------------------------------------------

def bj_blocks(A, L):
    """The d = K/L diagonal L x L blocks of A, shape (batch, d, L, L)."""
    A = _c128(A)
    K = A.shape[-1]
    if K % L:
        raise ValueError("K must be a multiple of L")
    d = K // L
    return np.stack([A[:, i * L:(i + 1) * L, i * L:(i + 1) * L] for i in range(d)], axis=1)


def bj_inverse(A, L, w="fp32"):
    """M_d blocks: each diagonal block inverted in float64, rounded to u_W.

    Returns (Md (batch, d, L, L), fail (batch,) bool); a block that is not
    positive definite (its Cholesky factorisation fails) marks the system.
    """
    blocks = bj_blocks(A, L)
    B, d = blocks.shape[:2]
    Md = np.zeros_like(blocks)
    fail = np.zeros(B, dtype=bool)
    flat = blocks.reshape(B * d, L, L)
    try:
        np.linalg.cholesky(flat)
        ok = np.ones(B * d, dtype=bool)
    except np.linalg.LinAlgError:
        ok = np.array([_is_pd(m) for m in flat])
    inv = np.zeros_like(flat)
    inv[ok] = np.linalg.inv(flat[ok])
    fail = ~ok.reshape(B, d).all(axis=1)
    Md = flc(inv.reshape(B, d, L, L), w)
    return Md, fail


def _is_pd(m):
    try:
        np.linalg.cholesky(m)
        return True
    except np.linalg.LinAlgError:
        return False


def bj_apply(Md, r):
    """z = M_d r, blockwise (exact in float64; caller rounds)."""
    B, d, L, _ = Md.shape
    return np.einsum("bdij,bdj->bdi", Md, r.reshape(B, d, L)).reshape(B, d * L)


# ---------------------------------------------------------------------------
# Algorithm 2 (FP-CG) and Algorithm 3 (FP-BJ-CG) with explicit rounding
# ---------------------------------------------------------------------------

def _acc_fmt(mv):
    return "fp64" if mv == "fp64" else "fp32"


def _dot_re(u, v, fmt, perm=None):
    """fl_fmt(Re(u^H v)) with the sum formed in float64 (perm: instead
    accumulated term by term in fp32 in that order, then rounded to fmt)."""
    if perm is None:
        return fl(np.real(np.einsum("bk,bk->b", np.conj(u), v)), fmt)
    t = np.real(np.conj(u) * v)
    acc = np.zeros(t.shape[0])
    for k in perm:
        acc = fl(acc + t[:, k], "fp32")
    return fl(acc, fmt)


def _matvec(A_mv, pq, acc, perm=None):
    """fl_acc(A_mv pq) (perm: the sum over columns accumulated in fp32 in that order)."""
    if perm is None:
        return flc(np.einsum("bkl,bl->bk", A_mv, pq), acc)
    out = np.zeros(pq.shape, dtype=np.complex128)
    for j in perm:
        out = flc(out + A_mv[:, :, j] * pq[:, j, None], acc)
    return out


def fp_cg(A_mv, b, iters, mv, ip="fp32", w="fp32", Md=None, alpha_num=0,
          block=32, trace=False, order_seed=None):
    """Algorithm 2 (Md is None) or Algorithm 3 (Md = block inverses).

    A_mv must already hold A rounded for the matvec (``round_matvec_operand``).
    Returns (x, status, hist, tr): hist[:, i] = ||r_i||_2 (recursive residual,
    i = 0..iters) and tr = per-iteration (x_i, r_i) lists when ``trace``.
    order_seed (not the default model): the fp32 sums of the matvec and of the
    inner products accumulate term by term in an order drawn from the seed.
    """
    b = _c128(b)
    B, K = b.shape
    acc = _acc_fmt(mv)
    perm = None if order_seed is None else np.random.default_rng(order_seed).permutation(K)
    if perm is not None and acc != "fp32":
        perm = None                                       # fp64 mode: no fp32 sums to reorder
    _dot = (lambda u, v, f: _dot_re(u, v, f, perm))
    x = np.zeros_like(b)
    r = flc(b, w)
    if Md is None:
        p = r.copy()
        rho = _dot(r, r, ip)                           # r_0^H r_0
    else:
        z = flc(bj_apply(Md, r), w)                       # p_0 = M_d r_0
        p = z
        rho = _dot(r, z, ip)                           # r_0^H z_0 (alpha_num=1)
    status = np.zeros(B, dtype=np.int32)
    active = np.ones(B, dtype=bool)
    hist = np.zeros((B, iters + 1))
    hist[:, 0] = np.sqrt(np.real(np.einsum("bk,bk->b", np.conj(r), r)))
    tr = {"x": [x.copy()], "r": [r.copy()]} if trace else None
    for i in range(iters):
        pq = round_matvec_operand(p, mv, block)
        varpi = _matvec(A_mv, pq, acc, perm)                       # u_MV
        phi = _dot(p, varpi, ip)                                # u_IP
        if Md is not None and alpha_num == 0:
            rho_prev = _dot(r, p, ip)                           # r^H p (Alg. 3)
        else:
            rho_prev = rho
        zero = active & (rho_prev == 0)
        status[zero] |= ST_RHO_ZERO
        bad = active & ~zero & (~np.isfinite(phi) | ~np.isfinite(rho_prev) | (phi <= 0))
        status[bad] |= ST_BREAKDOWN
        active = active & ~zero & ~bad
        safe_phi = np.where(active, phi, 1.0)
        alpha = fl(np.where(active, rho_prev, 0.0) / safe_phi, w)  # u_W
        x_n = flc(x + alpha[:, None] * p, w)
        r_n = flc(r - alpha[:, None] * varpi, w)
        if Md is None:
            z_n = r_n
            rho_n = _dot(r_n, r_n, ip)
        else:
            z_n = flc(bj_apply(Md, r_n), w)
            rho_n = _dot(r_n, z_n, ip)
        safe_rho = np.where(active, rho_prev, 1.0)
        beta = fl(np.where(active, rho_n, 0.0) / safe_rho, w)
        p_n = flc(z_n + beta[:, None] * p, w)
        a = active[:, None]
        x = np.where(a, x_n, x)
        r = np.where(a, r_n, r)
        p = np.where(a, p_n, p)
        rho = np.where(active, rho_n, rho)
        hist[:, i + 1] = np.sqrt(np.real(np.einsum("bk,bk->b", np.conj(r), r)))
        if trace:
            tr["x"].append(x.copy())
            tr["r"].append(r.copy())
    return x, status, hist, tr


# ---------------------------------------------------------------------------
# Full detection pipeline (the operation the C ABI's fpcg_detect/fpbjcg_detect
# perform): Gram -> [BJ] -> CG -> iterative refinement -> residual -> slice.
# ---------------------------------------------------------------------------

DEFAULT_PREC = {"gram": "fp32", "mv": "fp32", "ip": "fp32", "w": "fp32",
                "refine_steps": 0, "refine_iters": None, "alpha_num": 0, "resid": "gram"}

# Matrix of the refinement residual and of rel_res (prec["resid"]); "fp64" and
# "fp32" are the C ABI's names for "gram" and "mv".
RESID_MODES = {"gram": "gram", "fp64": "gram", "mv": "mv", "fp32": "mv", "h": "h"}


def resid(A, x, b):
    """b - A x formed in float64 (the refinement residual and final check)."""
    return _c128(b) - np.einsum("bkl,bl->bk", _c128(A), _c128(x))


def resid_h(H, y, sigma2, x):
    """H^H (y - H x) - sigma^2 x from the stored (complex64) H and y, in float64:
    the residual of the LMMSE system of Section II (eq. inversion) itself, with
    no Gram matrix formed.  H in storage layout (batch, K, N)."""
    Hs = _c128(H)
    x = _c128(x)
    e = _c128(y) - np.einsum("bkn,bk->bn", Hs, x)                 # y - H x
    return np.einsum("bkn,bn->bk", np.conj(Hs), e) - np.asarray(sigma2, dtype=np.float64)[:, None] * x


def detect(H, y, sigma2, qam_order, iters, prec=None, L=None, block=32, order_seed=None):
    """Emulate one detection call; returns a dict of results.

    prec keys: gram, mv, ip, w in {"fp64","fp32","fp16","bf16"} (mv also
    "e4m3"), refine_steps, refine_iters (default: iters), alpha_num, resid.
    L: block-Jacobi block size (None = FP-CG, Algorithm 2).
    order_seed: the fp32 sums of the Gram step, the matvec and the inner
    products in other orders (gram_emul, fp_cg); everything else unchanged.

    Iterative refinement (not in the paper; Theorem 2 of Section III-B is its
    motivation: the attainable accuracy of FP-CG is limited by the gap between
    the true residual b - A x and the recursively updated r, which grows with
    u_MV, so the true residual is recomputed above the working precision and
    a correction is solved for).  resid selects the residual, always formed in
    float64, that drives the corrections and defines rel_res:
      "gram" (default, C ABI FPCG_FP64): b - A x with A, b the Gram matrix and
             matched filter of the gram step (for gram = fp64 the exact ones);
      "mv"   (C ABI FPCG_FP32): b - A_mv x with A rounded to u_MV, the matrix
             the CG products use -- refinement then removes only the CG
             iteration error, not the rounding of A;
      "h":   H^H (y - H x) - sigma^2 x from the stored H and y (resid_h) -- the
             residual of the unrounded LMMSE system; rel_res divides by
             ||H^H y||.
    """
    pr = dict(DEFAULT_PREC)
    pr.update(prec or {})
    w = pr["w"]
    mode = RESID_MODES[pr.get("resid", "gram")]
    A, b = gram_emul(H, y, sigma2, pr["gram"], order_seed)
    B = A.shape[0]
    status = np.zeros(B, dtype=np.int32)
    Md = None
    if L is not None:
        Md, fail = bj_inverse(A, L, w)
        status[fail] |= ST_BJ_FAIL
    A_mv = round_matvec_operand(A, pr["mv"], block)
    if mode == "h":
        _, b_ref = gram_mf(H, y, sigma2)

        def true_res(x):
            return resid_h(H, y, sigma2, x)
    else:
        A_res = A_mv if mode == "mv" else A
        b_ref = b

        def true_res(x):
            return resid(A_res, x, b)
    cg_seed = None if order_seed is None else order_seed + 7919
    x, st, hist, _ = fp_cg(A_mv, b, iters, pr["mv"], pr["ip"], w, Md, pr["alpha_num"], block, order_seed=cg_seed)
    status |= st
    ri = pr["refine_iters"] if pr["refine_iters"] is not None else iters
    for _ in range(int(pr["refine_steps"])):
        rr = flc(true_res(x), w)
        d, st2, _, _ = fp_cg(A_mv, rr, ri, pr["mv"], pr["ip"], w, Md, pr["alpha_num"], block, order_seed=cg_seed)
        status |= st2 & ST_BREAKDOWN
        x = flc(x + d, w)
    nb = np.linalg.norm(_c128(b_ref), axis=1)
    nr = np.linalg.norm(true_res(x), axis=1)
    rel = np.where(nb > 0, nr / np.where(nb > 0, nb, 1.0), 0.0)
    status[~np.all(np.isfinite(x), axis=1)] |= ST_NONFINITE
    qam_order = np.broadcast_to(np.asarray(qam_order), (B,))
    sym = np.zeros(x.shape, dtype=np.uint8)
    sprec = "fp64" if w == "fp64" else "fp32"
    for M in np.unique(qam_order):
        sel = qam_order == M
        sym[sel] = _qam.slice_symbols(x[sel], int(M), sprec)
    return {"x": x, "sym": sym, "rel_res": rel, "status": status, "hist": hist,
            "A": A, "b": b}
