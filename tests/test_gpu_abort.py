"""The bounded waits of the tensor-core pipelines: with the wait budget cut to
one cycle (FPCG_TC_WAIT_CYCLES, read when a call is issued) every wait of the
fused detector and of the Gram kernel gives up at once, the CTAs abort -- after
waiting for the TMA loads and MMAs they had issued -- and every system reports
FPCG_ST_TIMEOUT; the context stays usable and the next call, with the default
budget, gives the usual results."""
import numpy as np
import pytest
import torch

from paper_2504_09820_gb300 import fpcg as F
from paper_2504_09820_gb300 import workload as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()


@pytest.mark.parametrize("resid", ["fp64", "fp32"])
def test_timeout_reported_and_context_usable(monkeypatch, resid):
    d = wl.generate(wl.Spec(N=256, K=64, batch=400, rho=0.5, qam=64, snr_db=15.0, seed=61))
    g = {k: torch.from_numpy(d[k]).cuda() for k in ("H", "y", "sigma2", "qam", "tx")}
    prec = F.precision(gram="bf16", mv="fp16", refine_steps=1, resid=resid)
    assert F.fpcg_path(256, 64, 4, prec) == F.PATH_TENSOR_CORE

    def run():
        out = F.detect(g["H"], g["y"], g["sigma2"], g["qam"], 6, prec, L=4, tx_idx=g["tx"])
        torch.cuda.synchronize()
        return {k: v.cpu() for k, v in out.items() if v is not None}

    ref = run()
    assert torch.all(ref["status"] & F.ST_TIMEOUT == 0)
    monkeypatch.setenv("FPCG_TC_WAIT_CYCLES", "1")
    bad = run()
    assert torch.all(bad["status"] & F.ST_TIMEOUT != 0)
    monkeypatch.delenv("FPCG_TC_WAIT_CYCLES")
    again = run()
    for k in ("x", "sym", "status", "rel_res"):
        assert torch.equal(again[k], ref[k]), k


def test_gram_timeout_reported(monkeypatch):
    d = wl.generate(wl.Spec(N=256, K=64, batch=300, rho=0.5, qam=64, snr_db=15.0, seed=62))
    H, y, s2 = (torch.from_numpy(d[k]).cuda() for k in ("H", "y", "sigma2"))
    A = torch.empty((300, 64, 64), dtype=torch.complex64, device="cuda")
    b = torch.empty((300, 64), dtype=torch.complex64, device="cuda")
    st = torch.empty(300, dtype=torch.int32, device="cuda")
    monkeypatch.setenv("FPCG_TC_WAIT_CYCLES", "1")
    F.fpcg_gram(H, y, s2, "bf16", A, b, status=st)
    torch.cuda.synchronize()
    assert torch.all(st & F.ST_TIMEOUT != 0)
    monkeypatch.delenv("FPCG_TC_WAIT_CYCLES")
    F.fpcg_gram(H, y, s2, "bf16", A, b, status=st)
    torch.cuda.synchronize()
    assert torch.all(st == 0) and torch.isfinite(torch.view_as_real(A)).all()


def test_timeout_in_a_multi_class_launch(monkeypatch):
    """The fused launch over several classes: with the one-cycle budget every
    class's systems report FPCG_ST_TIMEOUT (each class's CTAs abort and the
    next class starts from fresh barriers); with the default budget the
    results are the earlier ones."""
    d = wl.generate_mixed(wl.MixedSpec(batch=300, seed=63))
    prec = F.precision(gram="bf16", mv="fp16", refine_steps=1, resid="fp64")
    p = F.Plan(d["n"], d["k"], 6, prec, block_L=4)
    g = p.pack(d["H"], d["y"], d["sigma2"], d["qam"], d["tx"])
    fused = [c for c in p.classes() if c["path"] == F.PATH_TENSOR_CORE and c["k"] in (16, 32, 64)]
    assert len(fused) >= 2 and len({c["launch"] for c in fused}) == 1

    def run():
        n = p.totals[2]
        x = torch.zeros(n, dtype=torch.complex64, device="cuda")
        st = torch.zeros(p.batch, dtype=torch.int32, device="cuda")
        p.run(g["H"], g["y"], g["sigma2"], g["qam"], x, status=st)
        torch.cuda.synchronize()
        return x.cpu(), st.cpu()

    x0, st0 = run()
    monkeypatch.setenv("FPCG_TC_WAIT_CYCLES", "1")
    _, st1 = run()
    monkeypatch.delenv("FPCG_TC_WAIT_CYCLES")
    for c in fused:
        assert torch.all(st1[c["first"]:c["first"] + c["count"]] & F.ST_TIMEOUT != 0), c
    x2, st2 = run()
    assert torch.equal(x2, x0) and torch.equal(st2, st0)
