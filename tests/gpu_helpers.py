"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
on a generated batch and the oracle on the same arrays."""
import numpy as np
import torch

from oracle import detect as D
from oracle import qam as Q
from paper_2504_09820_gb300 import fpcg as F


def to_dev(d, dev="cuda:0"):
    return {
        "H": torch.from_numpy(d["H"]).to(dev),
        "y": torch.from_numpy(d["y"]).to(dev),
        "sigma2": torch.from_numpy(d["sigma2"]).to(dev),
        "qam": torch.from_numpy(d["qam"]).to(dev),
        "tx": torch.from_numpy(d["tx"]).to(dev),
    }


def gpu_detect(d, iters, prec_kw, L=None, hist=False, dev="cuda:0", g=None):
    g = g or to_dev(d, dev)
    prec = F.precision(**prec_kw)
    out = F.detect(g["H"], g["y"], g["sigma2"], g["qam"], iters, prec, L=L, tx_idx=g["tx"], hist=hist)
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    return res


ORACLE_KEYS = ("gram", "mv", "ip", "w", "refine_steps", "refine_iters", "alpha_num", "resid")


def oracle_detect(d, iters, prec_kw, L=None, sel=None, order_seed=None):
    pk = {k: v for k, v in prec_kw.items() if k in ORACLE_KEYS}
    pk.setdefault("resid", F.DEFAULT_RESID)   # the binding's default, not the oracle's
    if pk.get("w") == "fp64":
        pk.update(gram="fp64", mv="fp64", ip="fp64")
    if pk.get("refine_iters", -1) is not None and pk.get("refine_iters", -1) < 0:
        pk["refine_iters"] = None
    sl = slice(None) if sel is None else sel
    return D.detect(d["H"][sl], d["y"][sl], d["sigma2"][sl], d["qam"][sl], iters, pk, L=L, order_seed=order_seed)


def rel_err(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def near_threshold(x, M, prec, margin):
    """Mask of entries whose decision statistic t lies within `margin` of a
    threshold on either axis (those may legitimately slice differently)."""
    s = Q.axis_scale(M, prec)
    out = np.zeros(x.shape, dtype=bool)
    m = int(round(np.sqrt(M)))
    for comp in (x.real, x.imag):
        t = comp * s
        for k in range(m - 1):
            out |= np.abs(t - (2 * k - m + 2)) < margin
    return out


def order_spread(d, iters, prec_kw, L=None, sel=None, seeds=(1, 2), key="x"):
    """How far the oracle's own result moves when only the order of its fp32
    sums (Gram step, matvec, inner products; oracle.detect order_seed) changes:
    per system, the largest over the seeds of the relative change of x_hat
    (key "x") or of the absolute change of rel_res (key "rel_res")."""
    ref = oracle_detect(d, iters, prec_kw, L=L, sel=sel)
    spread = None
    for s in seeds:
        alt = oracle_detect(d, iters, prec_kw, L=L, sel=sel, order_seed=s)
        v = rel_err(alt["x"], ref["x"]) if key == "x" else np.abs(alt["rel_res"] - ref["rel_res"])
        spread = v if spread is None else np.maximum(spread, v)
    return spread


def check_reduced_parity(d, x_gpu, x_ref, iters, prec_kw, L=None, sel=None, tol=2e-3):
    """The bar of the reduced-precision modes: x_hat within `tol` relative of
    the oracle's emulated run for every system.  The tensor-core rounding model
    fixes the products and every rounding format but not the order of the fp32
    sums, and an unconverged iterate can move by more than `tol` under that
    order alone (one 16-bit rounding of p or A, or one power-of-two block
    scale, coming out the other way moves it at once: a heavy-tailed effect).
    Where the GPU exceeds `tol`, the regime's own spread is measured -- the
    oracle rerun with its fp32 sums in two other orders on the same systems --
    and the GPU must stay within it: 99th percentile within max(tol, 1.5 x the
    spread's), largest difference within max(tol, 4 x the spread's largest).
    A system beyond that (at most 1% of them) is one where the order decides a
    rounding that moves x_hat at once (an e4m3 step of A_mv: several results
    are correct there); its x_hat must then be one the oracle itself reaches
    under another of its summation orders, within the same bar.
    Returns (errors, spread or None)."""
    e = rel_err(x_gpu, x_ref)
    if e.max() <= tol:
        return e, None
    sp = order_spread(d, iters, prec_kw, L=L, sel=sel)
    q_gpu, q_sp = np.quantile(e, 0.99), np.quantile(sp, 0.99)
    assert q_gpu <= max(tol, 1.5 * q_sp), ("q99", q_gpu, q_sp)
    bar = max(tol, 4 * sp.max())
    out = np.flatnonzero(e > bar)
    if out.size:
        assert out.size <= max(1, e.size // 100), ("max", e.max(), sp.max(), out.size)
        idx = (np.arange(e.size) if sel is None else np.asarray(sel))[out]
        best = np.full(out.size, np.inf)
        for s in range(3, 35):
            alt = oracle_detect(d, iters, prec_kw, L=L, sel=idx, order_seed=s)
            best = np.minimum(best, rel_err(x_gpu[out], alt["x"]))
            if np.all(best <= bar):
                break
        assert np.all(best <= bar), ("max", e[out], best, sp.max(), idx)
    return e, sp


def gram_resid_rel(A, b, x):
    """||b - A x|| / ||b|| in float64 for fp32 A, b and a returned x, and the
    bound on how far the solvers' fp32 residual against a given Gram matrix
    (resid = FP64 on the tensor-core solvers) may move it: per row, 2E fp32
    multiply-adds in a lane (E = max(1, K/32)), five pairwise tree additions
    over the lanes and the subtraction from b, so each of Re and Im of the
    residual is off by at most (2E + 6) u32 times the sum of the magnitudes of
    its terms; in norm, (2E + 6) u32 || (|Re A| + |Im A|)(|Re x| + |Im x|)
    + |Re b| + |Im b| || / ||b||."""
    A, b, x = (np.asarray(v, dtype=np.complex128) for v in (A, b, x))
    K = A.shape[-1]
    E = max(1, K // 32)
    r = b - np.einsum("bkl,bl->bk", A, x)
    nb = np.linalg.norm(b, axis=1)
    aA = np.abs(A.real) + np.abs(A.imag)
    ax = np.abs(x.real) + np.abs(x.imag)
    mag = np.einsum("bkl,bl->bk", aA, ax) + np.abs(b.real) + np.abs(b.imag)
    return np.linalg.norm(r, axis=1) / nb, (2 * E + 6) * 2.0 ** -24 * np.linalg.norm(mag, axis=1) / nb
