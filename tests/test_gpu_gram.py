"""Gram matrix + matched filter (Section II, eq. inversion) on the tensor cores
through fpcg_gram, against the oracle's reduced-precision Gram (H and y
rounded to bf16/fp16, exact products, one fp32 rounding).  fp32 accumulation
on the tensor cores differs from the exactly-rounded sum by a few fp32 ulps of
the row scale."""
import numpy as np
import pytest
import torch

from oracle import detect as D
from paper_2504_09820_gb300 import fpcg as F
from paper_2504_09820_gb300 import workload as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()


def run_gram(d, gram):
    dev = "cuda:0"
    H = torch.from_numpy(d["H"]).to(dev)
    y = torch.from_numpy(d["y"]).to(dev)
    s2 = torch.from_numpy(d["sigma2"]).to(dev)
    B, K, N = H.shape
    cdt = torch.complex128 if gram == "fp64" else torch.complex64
    A = torch.full((B, K, K), float("nan"), dtype=cdt, device=dev)
    b = torch.full((B, K), float("nan"), dtype=cdt, device=dev)
    st = torch.full((B,), -1, dtype=torch.int32, device=dev)
    F.fpcg_gram(H, y, s2, gram, A, b, status=st)
    torch.cuda.synchronize()
    return A.cpu().numpy(), b.cpu().numpy(), st.cpu().numpy()


def check(d, gram, A, b, st, tol=2e-6):
    Ar, br = D.gram_emul(d["H"], d["y"], d["sigma2"], gram)
    assert np.all(st == 0)
    scale = np.abs(Ar).max(axis=(1, 2))
    errA = np.abs(A - Ar).max(axis=(1, 2)) / scale
    errb = np.abs(b - br).max(axis=1) / np.maximum(np.abs(br).max(axis=1), 1e-30)
    assert np.all(np.isfinite(A)) and np.all(np.isfinite(b))
    assert errA.max() < tol, (errA.max(), int(errA.argmax()))
    assert errb.max() < 10 * tol, (errb.max(), int(errb.argmax()))


@pytest.mark.parametrize("K", [64, 32, 16, 8])
@pytest.mark.parametrize("gram", ["bf16", "fp16"])
def test_tensor_core_gram_packed(K, gram):
    # enough tiles that every CTA reuses its stages and both accumulators,
    # and a ragged last tile when P = 64/K > 1
    batch = 152 * (64 // K) * 3 + (64 // K) // 2 + 1
    d = wl.generate(wl.Spec(N=256, K=K, batch=batch, rho=0.5, qam=16, snr_db=12.0, seed=31 + K))
    A, b, st = run_gram(d, gram)
    check(d, gram, A, b, st)


@pytest.mark.parametrize("N", [64, 70, 33, 512])
def test_tensor_core_gram_ragged_antennas(N):
    d = wl.generate(wl.Spec(N=N, K=16, batch=700, rho=0.3, qam=16, snr_db=10.0, seed=N))
    A, b, st = run_gram(d, "bf16")
    check(d, "bf16", A, b, st)


def test_gram_simt_fallbacks():
    d = wl.generate(wl.Spec(N=100, K=20, batch=300, rho=0.5, qam=16, snr_db=10.0, seed=3))
    for g in ("bf16", "fp32"):
        A, b, st = run_gram(d, g)
        check(d, g, A, b, st)
    A, b, st = run_gram(d, "fp64")
    Ar, br = D.gram_emul(d["H"], d["y"], d["sigma2"], "fp64")
    assert np.abs(A - Ar).max() < 1e-12 and np.abs(b - br).max() < 1e-12


@pytest.mark.parametrize("K,N", [(128, 512), (128, 256), (128, 130), (64, 255), (32, 97), (16, 33), (8, 33), (8, 9)])
@pytest.mark.parametrize("gram", ["bf16", "fp16"])
def test_mma_gram(K, N, gram):
    """The mma.sync Gram (K = 128, or odd N the TMA pipeline cannot address):
    several antenna chunks, a ragged last chunk, against the oracle."""
    d = wl.generate(wl.Spec(N=N, K=K, batch=40, rho=0.5, qam=64, snr_db=15.0, seed=200 + K + N))
    A, b, st = run_gram(d, gram)
    # the mma chain rounds the fp32 accumulator twice per 16 antennas (two MMAs per
    # part); one ulp (2^-23, truncation allowed) of the row scale per rounding
    check(d, gram, A, b, st, tol=max(2e-6, 2 * (-(-N // 16)) * 2.0 ** -23))


@pytest.mark.parametrize("N,batch", [(512, 400), (256, 160), (130, 153), (128, 7)])
@pytest.mark.parametrize("gram", ["bf16", "fp16"])
def test_tcgen05_gram_k128(N, batch, gram, monkeypatch):
    """K = 128 on the tcgen05 pipeline (N even, aligned): Re A and [Im A | b]
    in two TMEM accumulators, the fourth product through the negate-B bit.
    More systems than SMs (the accumulators are reused after each drain) and
    a ragged last antenna chunk, against the oracle."""
    d = wl.generate(wl.Spec(N=N, K=128, batch=batch, rho=0.5, qam=64, snr_db=15.0, seed=300 + N + batch))
    A, b, st = run_gram(d, gram)
    tol = max(2e-6, 2 * (-(-N // 16)) * 2.0 ** -23)
    check(d, gram, A, b, st, tol=tol)
    # the two triangles come from different accumulator entries: Hermitian within the bound
    assert np.abs(A - np.conj(np.swapaxes(A, 1, 2))).max() < 2 * tol * np.abs(A).max()
