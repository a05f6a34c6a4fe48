"""The FMA throughput probe behind the SIMT peaks of the benchmark: it runs,
reports 2 flops per FMA for eight chains per thread, and its chains compute
what a plain loop of fma() computes (so the timed work is the work counted)."""
import numpy as np
import pytest
import torch

from paper_2504_09820_gb300 import fpcg as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()


@pytest.mark.parametrize("fp64", [0, 1])
def test_probe_counts_and_values(fp64):
    n, iters = 512, 64
    out = torch.zeros(n, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
    flops = F.fpcg_fma_probe(fp64, iters, out)
    torch.cuda.synchronize()
    assert flops == 2 * 8 * iters * n
    # thread t, chain c: x <- x * 0.999999 + 1e-7 from x0 = (t + c) 1e-9, iters times; out[t] = sum over c
    t = np.arange(n, dtype=np.float64)[:, None]
    x = (t + np.arange(8)[None, :]) * 1e-9
    for _ in range(iters):
        x = x * 0.999999 + 1e-7
    ref = x.sum(axis=1)
    got = out.cpu().numpy().astype(np.float64)
    assert np.allclose(got, ref, rtol=1e-5 if not fp64 else 1e-12)
