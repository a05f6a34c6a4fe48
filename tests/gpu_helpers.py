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


def oracle_detect(d, iters, prec_kw, L=None, sel=None):
    pk = {k: v for k, v in prec_kw.items() if k in ORACLE_KEYS}
    pk.setdefault("resid", F.DEFAULT_RESID)   # the binding's default, not the oracle's
    if pk.get("w") == "fp64":
        pk.update(gram="fp64", mv="fp64", ip="fp64")
    if pk.get("refine_iters", -1) is not None and pk.get("refine_iters", -1) < 0:
        pk["refine_iters"] = None
    sl = slice(None) if sel is None else sel
    return D.detect(d["H"][sl], d["y"][sl], d["sigma2"][sl], d["qam"][sl], iters, pk, L=L)


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
