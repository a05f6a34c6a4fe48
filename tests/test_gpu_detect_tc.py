"""Fused tensor-core detector (tcgen05 Gram + mma.sync FP-(BJ-)CG) against the
oracle's emulation of the same precisions.  Bar: x_hat within 2e-3 relative for
every system, or within twice the oracle's own spread on that system when only
the fp32 summation order of its Gram step changes (gpu_helpers.
check_reduced_parity); labels equal to the oracle's slicer on the same
estimates, bit-error counter and residual consistent with them."""
import numpy as np
import pytest
import torch

from oracle import detect as D
from oracle import qam as Q
from paper_2504_09820_gb300 import fpcg as F
from paper_2504_09820_gb300 import workload as wl

from gpu_helpers import check_reduced_parity, gpu_detect, oracle_detect, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()


def _check(d, res, ref, iters, pk, L, tol=2e-3):
    check_reduced_parity(d, res["x"], ref["x"], iters, pk, L=L, tol=tol)
    M = int(d["qam"][0])
    assert np.array_equal(Q.slice_symbols(res["x"], M, "fp32"), res["sym"])
    assert int(res["bit_errors"][0]) == Q.bit_errors(res["sym"], d["tx"])
    assert np.all(res["status"] & ~F.ST_RHO_ZERO == 0)


def _own_residual(d, res, gram, mv, resid="fp32"):
    """||b - A x|| / ||b|| of the GPU's own x in float64, with A the GPU's own
    fp32 Gram (fpcg_gram runs the same tensor-core pipeline): as it is for
    resid = "fp64", rounded to the matvec format for resid = "fp32".  The
    oracle's fp32 Gram sums in another order, and an entry next to a rounding
    boundary of the 16-bit format can round the other way there, which moves a
    residual of ~1e-3 noticeably."""
    from oracle.formats import round_matvec_operand
    g = to_dev(d)
    B, K, _ = d["H"].shape
    A = torch.empty((B, K, K), dtype=torch.complex64, device="cuda:0")
    b = torch.empty((B, K), dtype=torch.complex64, device="cuda:0")
    F.fpcg_gram(g["H"], g["y"], g["sigma2"], gram, A, b)
    A = A.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    A_r = A if resid == "fp64" else round_matvec_operand(A, mv, 32)
    return np.linalg.norm(D.resid(A_r, res["x"], b), axis=1) / np.linalg.norm(b, axis=1)


CASES = [
    # K, gram, mv, L, iters, refine, resid ("fp64": against the fp32 Gram; "fp32": the matvec matrix)
    (64, "bf16", "bf16", 8, 6, 1, "fp64"),
    (64, "fp16", "fp16", 8, 6, 1, "fp64"),
    (64, "bf16", "bf16", 0, 10, 1, "fp64"),
    (64, "bf16", "fp16", 16, 5, 2, "fp64"),
    (64, "bf16", "fp16", 4, 7, 1, "fp64"),
    (64, "fp16", "bf16", 4, 6, 0, "fp64"),
    (32, "bf16", "bf16", 8, 8, 1, "fp64"),
    (32, "fp16", "fp16", 16, 6, 1, "fp64"),
    (16, "bf16", "bf16", 4, 8, 1, "fp64"),
    (16, "bf16", "fp16", 0, 12, 1, "fp64"),
    (64, "bf16", "bf16", 16, 4, 1, "fp64"),
    (32, "bf16", "fp16", 4, 6, 2, "fp64"),
    (64, "bf16", "bf16", 8, 6, 1, "fp32"),
    (32, "bf16", "fp16", 4, 6, 2, "fp32"),
    (16, "bf16", "bf16", 0, 12, 1, "fp32"),
]


def test_routing_to_simt():
    """Configurations the fused kernel does not take run on the SIMT kernel."""
    bf = dict(gram="bf16", mv="bf16")
    assert F.fpcg_path(256, 64, 1, F.precision(**bf)) == F.PATH_SIMT          # L not in {0,4,8,16}
    assert F.fpcg_path(256, 64, 2, F.precision(**bf)) == F.PATH_SIMT
    assert F.fpcg_path(256, 128, 8, F.precision(**bf)) == F.PATH_SIMT         # K > 64
    assert F.fpcg_path(64, 8, 4, F.precision(**bf)) == F.PATH_SIMT           # K < 16
    assert F.fpcg_path(256, 64, 8, F.precision(**bf, resid="fp64")) == F.PATH_TENSOR_CORE  # Gram residual
    assert F.fpcg_path(256, 64, 8, F.precision(gram="fp32", mv="bf16")) == F.PATH_SIMT  # fp32 Gram
    assert F.fpcg_path(256, 64, 8, F.precision(gram="bf16", mv="e4m3")) == F.PATH_TENSOR_CORE  # e4m3 A p
    assert F.fpcg_path(256, 128, 8, F.precision(gram="bf16", mv="e4m3")) == F.PATH_SIMT
    assert F.fpcg_path(255, 64, 8, F.precision(**bf)) == F.PATH_SIMT          # odd N (no TMA)
    assert F.fpcg_path(256, 64, 8, F.precision(**bf)) == F.PATH_TENSOR_CORE


@pytest.mark.parametrize("K,gram,mv,L,iters,refine,resid", CASES)
def test_fused_matches_oracle(K, gram, mv, L, iters, refine, resid):
    N = 4 * K
    P = 64 // K
    batch = 152 * P * 2 + P // 2 + 1       # every CTA reuses both accumulators; ragged last tile
    d = wl.generate(wl.Spec(N=N, K=K, batch=batch, rho=0.5, qam=64, snr_db=14.0, seed=500 + K + L))
    pk = dict(gram=gram, mv=mv, refine_steps=refine, resid=resid)
    assert F.fpcg_path(N, K, L, F.precision(**pk)) == F.PATH_TENSOR_CORE
    res = gpu_detect(d, iters, pk, L=(L or None))
    ref = oracle_detect(d, iters, pk, L=(L or None))
    _check(d, res, ref, iters, pk, L or None)
    own = _own_residual(d, res, gram, mv, resid)
    assert np.allclose(res["rel_res"], own, rtol=2e-3, atol=1e-6)


def test_fused_headline_config_full_size_sampled():
    """The benchmark's workload and launch: N=256, K=64, 16384 Kronecker
    channels, the head configuration of bench.py (bf16 Gram, fp16 A p, FP-BJ-CG
    with one refinement pass); oracle on a sample."""
    from bench import HEAD
    spec = wl.c3_kron_256x64()
    d = wl.generate(spec)
    pk = dict(HEAD["prec"])
    assert F.fpcg_path(256, 64, HEAD["L"], F.precision(**pk)) == F.PATH_TENSOR_CORE
    res = gpu_detect(d, HEAD["iters"], pk, L=HEAD["L"])
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(spec.batch, 96, replace=False))
    ref = oracle_detect(d, HEAD["iters"], pk, L=HEAD["L"], sel=sel)
    check_reduced_parity(d, res["x"][sel], ref["x"], HEAD["iters"], pk, L=HEAD["L"], sel=sel)
    assert np.array_equal(Q.slice_symbols(res["x"], 64, "fp32"), res["sym"])
    assert int(res["bit_errors"][0]) == Q.bit_errors(res["sym"], d["tx"])
    # BER of the fused path within 5% of the fp64 direct LMMSE solve (sample)
    xs = D.lmmse(d["H"][:1024], d["y"][:1024], d["sigma2"][:1024])
    e_ref = Q.bit_errors(Q.slice_symbols(xs, 64, "fp64"), d["tx"][:1024])
    e_gpu = Q.bit_errors(res["sym"][:1024], d["tx"][:1024])
    assert abs(e_gpu / e_ref - 1) < 0.05


def test_fused_hist_alpha_and_ip_rounding():
    d = wl.generate(wl.Spec(N=128, K=32, batch=700, rho=0.7, qam=16, snr_db=16.0, seed=77))
    for pk, L in ((dict(gram="bf16", mv="bf16", alpha_num=1, refine_steps=1), 8),
                  (dict(gram="bf16", mv="bf16", ip="bf16", refine_steps=1), 8),
                  (dict(gram="fp16", mv="fp16", refine_steps=2), 4)):
        res = gpu_detect(d, 6, pk, L=L, hist=True)
        ref = oracle_detect(d, 6, pk, L=L)
        _check(d, res, ref, 6, pk, L)
        # ||r_i|| of late iterations is ~1% of ||r_0||; the iterates agree to ~1e-3
        assert np.allclose(res["hist"], ref["hist"], rtol=2e-2, atol=2e-3 * ref["hist"][:, :1])


def test_fused_matches_simt_path(monkeypatch):
    """Same semantics on both kernels: the tensor-core path against the SIMT
    path (forced with FPCG_FORCE_SIMT) on identical inputs."""
    d = wl.generate(wl.Spec(N=256, K=64, batch=600, rho=0.7, qam=64, snr_db=18.0, seed=99))
    pk = dict(gram="bf16", mv="bf16", refine_steps=1)
    assert F.fpcg_path(256, 64, 8, F.precision(**pk)) == F.PATH_TENSOR_CORE
    tc = gpu_detect(d, 6, pk, L=8)
    monkeypatch.setenv("FPCG_FORCE_SIMT", "1")
    assert F.fpcg_path(256, 64, 8, F.precision(**pk)) == F.PATH_SIMT
    simt = gpu_detect(d, 6, pk, L=8)
    monkeypatch.delenv("FPCG_FORCE_SIMT")
    # each path is within 2e-3 of the oracle; they differ by at most the sum
    e = rel_err(tc["x"], simt["x"])
    assert np.quantile(e, 0.99) < 4e-3 and e.max() < 2e-2


def test_fused_edge_cases():
    # y = 0 -> x = 0, RHO_ZERO; iters = 0 -> x = 0 (then refinement) ; determinism
    d = wl.generate(wl.Spec(N=64, K=16, batch=300, qam=16, snr_db=10.0, seed=3))
    d0 = dict(d)
    d0["y"] = np.zeros_like(d["y"])
    res = gpu_detect(d0, 5, dict(gram="bf16", mv="bf16", refine_steps=1), L=4)
    assert np.all(res["x"] == 0) and np.all(res["status"] & F.ST_RHO_ZERO) and np.all(res["rel_res"] == 0)
    res = gpu_detect(d, 0, dict(gram="bf16", mv="bf16"), L=4)
    assert np.all(res["x"] == 0) and np.allclose(res["rel_res"], 1.0)
    a = gpu_detect(d, 6, dict(gram="bf16", mv="bf16", refine_steps=1), L=4)
    b = gpu_detect(d, 6, dict(gram="bf16", mv="bf16", refine_steps=1), L=4)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["sym"], b["sym"])
    # batch smaller than one tile and than the SM count
    d1 = wl.generate(wl.Spec(N=64, K=16, batch=3, qam=16, snr_db=10.0, seed=4))
    res = gpu_detect(d1, 8, dict(gram="bf16", mv="bf16"), L=4)
    ref = oracle_detect(d1, 8, dict(gram="bf16", mv="bf16"), L=4)
    check_reduced_parity(d1, res["x"], ref["x"], 8, dict(gram="bf16", mv="bf16"), L=4)
