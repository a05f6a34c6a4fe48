"""fpcg_detect_noalloc (no device allocation; scratch in a fixed library array):
two calls in a row give exactly what fpcg_gram + fpcg_solve_gram give on the
same systems, oversize batches are refused, and configurations without scratch
give exactly fpbjcg_detect.  Collected last on purpose: it must pass alone and
after every other test."""
import numpy as np
import pytest
import torch

from oracle import qam as Q
from paper_2504_09820_gb300 import fpcg as F
from paper_2504_09820_gb300 import workload as wl

pytestmark = pytest.mark.gpu

PREC = dict(gram="bf16", mv="fp16", refine_steps=1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()


def _data(N, K, B, seed):
    d = wl.generate(wl.Spec(N=N, K=K, batch=B, rho=0.5, qam=64, snr_db=15.0, seed=seed))
    return d, {k: torch.from_numpy(d[k]).cuda() for k in ("H", "y", "sigma2", "qam", "tx")}


def _noalloc(g, K, L, iters=6, pk=PREC):
    B = g["H"].shape[0]
    out = {"x": torch.empty((B, K), dtype=torch.complex64, device="cuda"),
           "sym": torch.empty((B, K), dtype=torch.uint8, device="cuda"),
           "rel": torch.empty(B, dtype=torch.float64, device="cuda"),
           "st": torch.full((B,), 7, dtype=torch.int32, device="cuda"),
           "be": torch.zeros(1, dtype=torch.int64, device="cuda")}
    F.fpcg_detect_noalloc(g["H"], g["y"], g["sigma2"], g["qam"], iters, L, F.precision(**pk), out["x"],
                          sym_idx=out["sym"], rel_res=out["rel"], tx_idx=g["tx"], bit_errors=out["be"],
                          status=out["st"])
    torch.cuda.synchronize()
    return {k: v.cpu() for k, v in out.items()}


def _gram_then_solve(g, K, L, pk=PREC):
    B = g["H"].shape[0]
    A = torch.empty((B, K, K), dtype=torch.complex64, device="cuda")
    b = torch.empty((B, K), dtype=torch.complex64, device="cuda")
    F.fpcg_gram(g["H"], g["y"], g["sigma2"], "bf16", A, b)
    x = torch.empty((B, K), dtype=torch.complex64, device="cuda")
    rel = torch.empty(B, dtype=torch.float64, device="cuda")
    F.fpcg_solve_gram(A, b, 6, L, F.precision(**pk), x, rel_res=rel)
    torch.cuda.synchronize()
    return x.cpu(), rel.cpu()


@pytest.mark.parametrize("resid", ["fp32", "fp64"])
@pytest.mark.parametrize("N,K,L", [(256, 128, 8), (64, 8, 4)])
def test_two_calls_equal_gram_then_solve(N, K, L, resid):
    """resid = "fp64": the solve's residual against the Gram matrix in the
    library's array (read again by the solver)."""
    pk = dict(PREC, resid=resid)
    d, g = _data(N, K, 200, 41)
    first = _noalloc(g, K, L, pk=pk)
    second = _noalloc(g, K, L, pk=pk)
    for k in first:
        assert torch.equal(first[k], second[k]), k
    x, rel = _gram_then_solve(g, K, L, pk=pk)
    assert torch.equal(first["x"], x) and torch.equal(first["rel"], rel)
    assert np.array_equal(Q.slice_symbols(first["x"].numpy(), 64, "fp32"), first["sym"].numpy())
    assert int(first["be"][0]) == Q.bit_errors(first["sym"].numpy(), d["tx"])
    assert torch.all(first["st"] & ~F.ST_RHO_ZERO == 0)   # the Gram pass's status, OR-ed with the solve's


def test_largest_batch_is_accepted_and_one_more_is_refused():
    """The limit batch * K * (K + 1) * 8 bytes <= 64 MiB, at its boundary for
    K = 128: 508 systems fit (and give the two-pass result), 509 do not."""
    limit = (64 << 20) // (128 * 129 * 8)
    assert limit == 508
    _, g = _data(256, 128, limit + 1, 44)
    with pytest.raises(F.FpcgError) as e:
        _noalloc(g, 128, 8)
    assert e.value.code == F.ENOTSUP
    g = {k: v[:limit].contiguous() for k, v in g.items()}
    a = _noalloc(g, 128, 8)
    x, rel = _gram_then_solve(g, 128, 8)
    assert torch.equal(a["x"], x) and torch.equal(a["rel"], rel)


def test_bad_arguments_have_no_side_effects():
    """A refused call returns before any GPU work: the status array it was
    given is not zeroed (the Gram pass would zero it first)."""
    _, g = _data(256, 128, 64, 45)
    with pytest.raises(F.FpcgError) as e:
        _noalloc(g, 128, 8, iters=-1)
    assert e.value.code == F.EINVAL
    st = torch.full((64,), 7, dtype=torch.int32, device="cuda")
    x = torch.empty((64, 128), dtype=torch.complex64, device="cuda")
    with pytest.raises(F.FpcgError):   # bit_errors without tx_idx
        F.fpcg_detect_noalloc(g["H"], g["y"], g["sigma2"], g["qam"], 6, 8, F.precision(**PREC), x,
                              bit_errors=torch.zeros(1, dtype=torch.int64, device="cuda"), status=st)
    torch.cuda.synchronize()
    assert torch.all(st == 7)


def test_oversize_is_refused():
    _, g = _data(256, 128, 520, 42)          # 520 * 128 * 129 * 8 bytes > 64 MiB
    with pytest.raises(F.FpcgError) as e:
        _noalloc(g, 128, 8)
    assert e.value.code == F.ENOTSUP


def test_configurations_without_scratch_take_the_ordinary_path():
    _, g = _data(256, 64, 300, 43)
    a = _noalloc(g, 64, 8)
    ref = F.detect(g["H"], g["y"], g["sigma2"], g["qam"], 6, F.precision(**PREC), L=8, tx_idx=g["tx"])
    torch.cuda.synchronize()
    assert torch.equal(a["x"], ref["x"].cpu()) and torch.equal(a["sym"], ref["sym"].cpu())
