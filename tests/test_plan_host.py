"""Uneven-batch plans on the host (no GPU): descriptor checks and the packed
plan-order layout of fpcg_plan_layout / fpcg_plan_classes."""
import numpy as np
import pytest

from paper_2504_09820_gb300 import fpcg as F
from paper_2504_09820_gb300 import workload as wl


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_09820_gb300 import build as B
    B.build()
    F.lib()


PREC = dict(gram="bf16", mv="fp16", refine_steps=1)


@pytest.mark.parametrize("resid", ["fp32", "fp64"])
def test_layout_invariants(resid):
    """resid = "fp64" (the residual against the Gram matrix) keeps the same
    paths: the K = 8 and 128 classes run in two passes on the tensor cores."""
    n, k, _, _ = wl.mixed_params(wl.MixedSpec(batch=500, seed=7))
    p = F.Plan(n, k, 6, F.precision(**PREC, resid=resid), block_L=8)
    # order is a permutation that groups by (K, N), caller order kept inside a class
    assert sorted(p.order.tolist()) == list(range(500))
    keys = [(int(k[i]), int(n[i])) for i in p.order]
    assert keys == sorted(keys)
    cls = p.classes()
    assert sum(c["count"] for c in cls) == 500
    for c in cls:
        pos = np.arange(c["first"], c["first"] + c["count"])
        idx = p.order[pos]
        assert np.all(np.diff(idx) > 0)
        assert np.all(n[idx] == c["n_rx"]) and np.all(k[idx] == c["k"])
        assert c["block_L"] == min(8, c["k"])
        # a class starts 256-byte aligned and is contiguous at the uniform strides
        for off, step in ((p.h_off, c["n_rx"] * c["k"]), (p.y_off, c["n_rx"]), (p.x_off, c["k"])):
            assert off[pos[0]] % 32 == 0
            assert np.all(np.diff(off[pos]) == step)
        want = {8: F.PATH_TWO_PASS, 16: F.PATH_TENSOR_CORE, 32: F.PATH_TENSOR_CORE, 64: F.PATH_TENSOR_CORE,
                128: F.PATH_TWO_PASS}.get(c["k"], F.PATH_SIMT)
        assert c["path"] == want
    # classes do not overlap and fit in the totals
    ends = [(p.h_off[c["first"]], p.h_off[c["first"]] + c["count"] * c["n_rx"] * c["k"]) for c in cls]
    for (a0, a1), (b0, b1) in zip(ends, ends[1:]):
        assert a1 <= b0
    assert ends[-1][1] <= p.totals[0]
    p.close()


def test_descriptor_checks():
    pr = F.precision(**PREC)
    with pytest.raises(F.FpcgError):
        F.Plan([64], [0], 6, pr)                  # K < 1
    with pytest.raises(F.FpcgError):
        F.Plan([32], [64], 6, pr)                 # N < K
    with pytest.raises(F.FpcgError):
        F.Plan([64], [24], 6, pr, block_L=16)     # L does not divide K
    with pytest.raises(F.FpcgError):
        F.Plan([64], [16], -1, pr)                # negative iterations
    p = F.Plan([64, 64], [8, 8], 6, pr, block_L=16)  # L = min(16, K) = 8
    assert p.classes()[0]["block_L"] == 8
    p.close()
    e = F.Plan([], [], 4, pr)                     # empty batch
    assert e.totals == (0, 0, 0) and e.classes() == []
    e.close()


def test_launch_indices():
    """The fused-kernel classes (K in {16, 32, 64}) share one launch index,
    up to ten classes per launch; every other class has its own; with
    per_class every class has its own."""
    n, k, _, _ = wl.mixed_params(wl.MixedSpec(batch=500, seed=7))
    p = F.Plan(n, k, 6, F.precision(**PREC), block_L=8)
    cls = p.classes()
    fused = [c for c in cls if c["path"] == F.PATH_TENSOR_CORE]
    rest = [c for c in cls if c["path"] != F.PATH_TENSOR_CORE]
    assert 2 <= len(fused) <= 10 and len({c["launch"] for c in fused}) == 1
    ids = [c["launch"] for c in rest] + [fused[0]["launch"]]
    assert len(set(ids)) == len(ids) and sorted(set(c["launch"] for c in cls)) == list(range(len(ids)))
    q = F.Plan(n, k, 6, F.precision(**PREC), block_L=8, per_class=True)
    assert sorted(c["launch"] for c in q.classes()) == list(range(len(cls)))
    # e4m3 classes and the SIMT path are not grouped
    r = F.Plan(n, k, 6, F.precision(gram="bf16", mv="e4m3", refine_steps=1), block_L=8)
    assert len({c["launch"] for c in r.classes()}) == len(cls)
    for x in (p, q, r):
        x.close()
