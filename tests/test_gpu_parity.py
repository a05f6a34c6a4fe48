"""Parity of the CUDA detector (through the C ABI) with the CPU oracle.

Bars: fp64 mode -- x_hat within 1e-10 relative, labels bit-exact; fp32 mode --
relative residual within 1e-5 of the oracle's, labels equal to the oracle's
slicer applied to the same estimates; reduced-precision modes -- x_hat within
2e-3 relative of the oracle's emulated run at the same precisions, or within
twice the oracle's own movement on that system when only its fp32 summation
order changes (gpu_helpers.check_reduced_parity).
"""
import numpy as np
import pytest
import torch

from oracle import detect as D
from oracle import qam as Q
from paper_2504_09820_gb300 import fpcg as F
from paper_2504_09820_gb300 import workload as wl

from gpu_helpers import (check_reduced_parity, gpu_detect, oracle_detect, order_spread, rel_err, near_threshold,
                         to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()


def _labels_consistent(res, d, prec):
    """GPU labels == oracle slicer on the GPU's own estimates (same precision),
    and the bit-error counter == popcount of the label differences."""
    M = int(d["qam"][0])
    assert np.array_equal(Q.slice_symbols(res["x"], M, prec), res["sym"])
    assert int(res["bit_errors"][0]) == Q.bit_errors(res["sym"], d["tx"])


def test_fp64_mode_c1_rayleigh_64x16():
    d = wl.generate(wl.c1_rayleigh_64x16(batch=1024))
    pk = dict(w="fp64")
    res = gpu_detect(d, 16, pk)
    ref = oracle_detect(d, 16, pk)
    e = rel_err(res["x"], ref["x"])
    assert e.max() < 1e-10, e.max()
    mask = near_threshold(ref["x"], 16, "fp64", 1e-8)
    assert mask.sum() <= 2
    assert np.array_equal(res["sym"][~mask], ref["sym"][~mask])
    # both residuals sit at the fp64 roundoff floor (~1e-16); compare as such
    assert np.max(np.abs(res["rel_res"] - ref["rel_res"])) < 1e-13, np.max(np.abs(res["rel_res"] - ref["rel_res"]))
    assert np.array_equal(res["status"], ref["status"])
    _labels_consistent(res, d, "fp64")


@pytest.mark.parametrize("N,K,rho,snr", [(128, 32, 0.5, 12.0), (256, 64, 0.7, 18.0)])
def test_fp64_mode_larger_systems(N, K, rho, snr):
    """The fp64 bar at the larger workloads' sizes: x_hat within 1e-10 relative
    and labels bit-exact outside a counted margin, with 2K iterations (converged
    to the fp64 roundoff floor, where the order of the sums no longer matters)."""
    d = wl.generate(wl.Spec(N=N, K=K, batch=256, rho=rho, qam=64, snr_db=snr, seed=3000 + K))
    pk = dict(w="fp64")
    res = gpu_detect(d, 2 * K, pk)
    ref = oracle_detect(d, 2 * K, pk)
    e = rel_err(res["x"], ref["x"])
    assert e.max() < 1e-10, e.max()
    mask = near_threshold(ref["x"], 64, "fp64", 1e-8)
    assert mask.sum() <= 2
    assert np.array_equal(res["sym"][~mask], ref["sym"][~mask])
    assert np.max(np.abs(res["rel_res"] - ref["rel_res"])) < 1e-12
    _labels_consistent(res, d, "fp64")


@pytest.mark.parametrize("N,K,L,rho", [(256, 128, None, 0.3), (512, 128, 8, 0.5), (384, 96, 4, 0.0)])
def test_fp64_mode_beyond_k64(N, K, L, rho):
    """The fp64 mode where A does not fit in shared memory (K > 64): every
    product with A is H^H (H v) + sigma^2 v from H, the block-Jacobi blocks and
    b are formed from H.  Against the oracle's explicit fp64 Gram matrix: x_hat
    within 1e-10 after 2K iterations (the fp64 floor), labels bit-exact outside
    a counted margin, rel_res at the roundoff floor, also with a refinement pass."""
    d = wl.generate(wl.Spec(N=N, K=K, batch=40, rho=rho, qam=16, snr_db=15.0, seed=3100 + K + N))
    for pk in (dict(w="fp64"), dict(w="fp64", refine_steps=1, refine_iters=K)):
        res = gpu_detect(d, 2 * K, pk, L=L)
        ref = oracle_detect(d, 2 * K, pk, L=L)
        e = rel_err(res["x"], ref["x"])
        assert e.max() < 1e-10, (pk, e.max())
        mask = near_threshold(ref["x"], 16, "fp64", 1e-8)
        assert mask.sum() <= 2
        assert np.array_equal(res["sym"][~mask], ref["sym"][~mask])
        assert np.max(np.abs(res["rel_res"] - ref["rel_res"])) < 1e-12
        assert np.all(res["status"] & ~F.ST_RHO_ZERO == 0)
        _labels_consistent(res, d, "fp64")
    # a few iterations, far from convergence: the operator is the same, the sums differ only at fp64 rounding
    res = gpu_detect(d, 5, dict(w="fp64"), L=L)
    ref = oracle_detect(d, 5, dict(w="fp64"), L=L)
    assert rel_err(res["x"], ref["x"]).max() < 1e-10


def test_fp32_comparator_at_the_benchmark_configuration():
    """The plain fp32 CG the benchmark compares against (N=256, K=64, rho=0.7,
    18 dB, 20 iterations, fp32 Gram): relative residual within 1e-5 of the
    oracle's, labels equal to the slicer on the GPU's own estimates."""
    from bench import COMP
    spec = wl.c3_kron_256x64()
    d = wl.generate(spec, chunks=[0, 1, 2, 3])
    d = {k: (v[:1024] if isinstance(v, np.ndarray) and v.ndim else v) for k, v in d.items()}
    res = gpu_detect(d, COMP["iters"], COMP["prec"])
    ref = oracle_detect(d, COMP["iters"], COMP["prec"])
    dr = np.abs(res["rel_res"] - ref["rel_res"])
    if dr.max() > 1e-5:
        # 20 fp32 CG steps at kappa ~ 140 stop well short of convergence, where the
        # residual moves with the order of the fp32 sums (oracle order spread)
        sp = order_spread(d, COMP["iters"], COMP["prec"], key="rel_res")
        assert np.quantile(dr, 0.99) <= max(1e-5, 1.5 * np.quantile(sp, 0.99)), (np.quantile(dr, 0.99), np.quantile(sp, 0.99))
        assert dr.max() <= max(1e-5, 4 * sp.max()), (dr.max(), sp.max())
    # the reported residual is that of the GPU's own estimate on the oracle's fp32 Gram
    A, b = D.gram_emul(d["H"], d["y"], d["sigma2"], "fp32")
    own = np.linalg.norm(D.resid(A, res["x"], b), axis=1) / np.linalg.norm(b, axis=1)
    assert np.allclose(res["rel_res"], own, rtol=1e-3, atol=1e-6)
    _labels_consistent(res, d, "fp32")


@pytest.mark.parametrize("refine", [0, 1])
def test_fp32_mode_c1(refine):
    d = wl.generate(wl.c1_rayleigh_64x16(batch=1024))
    pk = dict(gram="fp32", mv="fp32", refine_steps=refine)
    res = gpu_detect(d, 16, pk, hist=True)
    ref = oracle_detect(d, 16, pk)
    assert np.max(np.abs(res["rel_res"] - ref["rel_res"])) < 1e-5
    assert rel_err(res["x"], ref["x"]).max() < 1e-4
    assert np.allclose(res["hist"], ref["hist"], rtol=1e-3, atol=1e-6 * ref["hist"][:, :1])
    _labels_consistent(res, d, "fp32")
    mask = near_threshold(ref["x"], 16, "fp32", 1e-3)
    assert np.array_equal(res["sym"][~mask], ref["sym"][~mask])


REDUCED = [
    # (gram, mv, L, iters, refine)
    ("bf16", "bf16", 8, 8, 1),
    ("fp16", "fp16", 8, 6, 1),
    ("bf16", "bf16", None, 10, 1),
    ("bf16", "fp16", 4, 6, 2),
    ("fp32", "bf16", 16, 6, 1),
    ("bf16", "e4m3", 8, 3, 0),
]


@pytest.mark.parametrize("gram,mv,L,iters,refine", REDUCED)
def test_reduced_precision_c2_like(gram, mv, L, iters, refine):
    d = wl.generate(wl.Spec(N=128, K=32, batch=512, rho=0.5, qam=64, snr_db=12.0, seed=2002))
    pk = dict(gram=gram, mv=mv, refine_steps=refine)
    res = gpu_detect(d, iters, pk, L=L)
    ref = oracle_detect(d, iters, pk, L=L)
    check_reduced_parity(d, res["x"], ref["x"], iters, pk, L=L)
    _labels_consistent(res, d, "fp32")


def test_ragged_sizes_and_odd_block():
    """K not a multiple of the 4x4 Gram tile, N not a multiple of the staging
    chunk, an odd block size."""
    d = wl.generate(wl.Spec(N=70, K=20, batch=300, rho=0.3, qam=16, snr_db=15.0, seed=77))
    for L, pk in ((5, dict(gram="fp32", mv="fp32")), (None, dict(gram="bf16", mv="bf16", refine_steps=1)),
                  (4, dict(w="fp64"))):
        res = gpu_detect(d, 12, pk, L=L)
        ref = oracle_detect(d, 12, pk, L=L)
        tol = 1e-10 if pk.get("w") == "fp64" else (2e-3 if pk.get("gram") == "bf16" else 1e-4)
        assert rel_err(res["x"], ref["x"]).max() < tol


@pytest.mark.parametrize("alpha_num", [0, 1])
def test_bj_alpha_numerator_variants(alpha_num):
    d = wl.generate(wl.Spec(N=64, K=16, batch=256, rho=0.7, qam=16, snr_db=20.0, seed=5))
    pk = dict(w="fp64", alpha_num=alpha_num)
    res = gpu_detect(d, 6, pk, L=4)
    ref = oracle_detect(d, 6, pk, L=4)
    assert rel_err(res["x"], ref["x"]).max() < 1e-10


def test_solve_gram_interface():
    d = wl.generate(wl.Spec(N=64, K=16, batch=128, rho=0.5, qam=16, snr_db=10.0, seed=9))
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    A = A.astype(np.complex64)
    b = b.astype(np.complex64)
    for L in (0, 4):
        prec = F.precision()
        x = torch.empty((128, 16), dtype=torch.complex64, device="cuda:0")
        rr = torch.empty(128, dtype=torch.float64, device="cuda:0")
        F.fpcg_solve_gram(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), 10, L, prec, x, rel_res=rr)
        Md = D.bj_inverse(A, L, "fp32")[0] if L else None
        xr, _, _, _ = D.fp_cg(A, b, 10, "fp32", "fp32", "fp32", Md)
        # the fp32 bar: relative residual within 1e-5 of the oracle's, or within
        # the oracle's own movement when only the order of its fp32 sums changes
        def rres(x):
            return np.linalg.norm(D.resid(A, x, b), axis=1) / np.linalg.norm(b, axis=1)
        dr = np.abs(rr.cpu().numpy() - rres(xr))
        if dr.max() > 1e-5:
            sp = np.max([np.abs(rres(D.fp_cg(A, b, 10, "fp32", "fp32", "fp32", Md, order_seed=s)[0]) - rres(xr))
                         for s in (1, 2)], axis=0)
            assert dr.max() <= 4 * sp.max(), (L, dr.max(), sp.max())
        # and the reported residual is that of the GPU's own estimate
        xg = x.cpu().numpy()
        ref_rr = np.linalg.norm(D.resid(A, xg, b), axis=1) / np.linalg.norm(b, axis=1)
        assert np.allclose(rr.cpu().numpy(), ref_rr, rtol=1e-3, atol=1e-7)


def test_edge_cases():
    dev = "cuda:0"
    # K = 1 and N = K
    for N, K in ((8, 1), (16, 16)):
        d = wl.generate(wl.Spec(N=N, K=K, batch=17, rho=0.0, qam=4, snr_db=10.0, seed=1))
        # N = K: kappa ~ 42, and K CG steps stop short of the roundoff floor, where
        # a one-ulp change of A moves the iterate by ~1e-6 (measured with the
        # oracle); 4K steps reach the floor, and there the stated bars apply
        iters = 4 * K
        for pk in (dict(w="fp64"), dict(gram="fp32", mv="fp32")):
            res = gpu_detect(d, iters, pk)
            ref = oracle_detect(d, iters, pk)
            if pk.get("w"):
                assert rel_err(res["x"], ref["x"]).max() < 1e-10
            else:
                assert np.max(np.abs(res["rel_res"] - ref["rel_res"])) < 1e-5
    # y = 0: x = 0, status RHO_ZERO, rel_res 0
    d = wl.generate(wl.Spec(N=32, K=8, batch=4, qam=16, seed=2))
    d["y"][:] = 0
    res = gpu_detect(d, 5, dict(gram="fp32", mv="fp32", refine_steps=1))
    assert np.all(res["x"] == 0) and np.all(res["status"] & F.ST_RHO_ZERO) and np.all(res["rel_res"] == 0)
    # iters = 0: x = 0, rel_res = 1
    d = wl.generate(wl.Spec(N=32, K=8, batch=4, qam=16, seed=3))
    res = gpu_detect(d, 0, dict(gram="fp32", mv="fp32"))
    assert np.all(res["x"] == 0) and np.allclose(res["rel_res"], 1.0)
    # batch = 0: no launch, counter zeroed
    g = to_dev(wl.generate(wl.Spec(N=32, K=8, batch=1, qam=16, seed=4)))
    be = torch.full((1,), 7, dtype=torch.int64, device=dev)
    x = torch.empty((0, 8), dtype=torch.complex64, device=dev)
    rc = F.lib().fpcg_detect(g["H"].data_ptr(), g["y"].data_ptr(), g["sigma2"].data_ptr(),
                             g["qam"].data_ptr(), 32, 8, 0, 4, F.ctypes.byref(F.precision()),
                             x.data_ptr() or 1, None, None, None, g["tx"].data_ptr(), be.data_ptr(),
                             None, None)
    torch.cuda.synchronize()
    assert rc == 0 and int(be[0]) == 0
    # invalid QAM order flags the system and leaves labels 0
    d = wl.generate(wl.Spec(N=32, K=8, batch=2, qam=16, seed=5))
    d["qam"][1] = 32
    res = gpu_detect(d, 4, dict(gram="fp32", mv="fp32"))
    assert res["status"][1] & F.ST_BAD_QAM and not res["status"][0] & F.ST_BAD_QAM
    assert np.all(res["sym"][1] == 0)


def test_mixed_qam_orders_in_one_batch():
    parts = [wl.generate(wl.Spec(N=64, K=16, batch=64, qam=M, snr_db=14.0, seed=100 + M)) for M in (4, 16, 64, 256)]
    d = {k: np.concatenate([p[k] for p in parts]) for k in ("H", "y", "tx", "sigma2", "qam")}
    res = gpu_detect(d, 16, dict(gram="fp32", mv="fp32"))
    for i, M in enumerate((4, 16, 64, 256)):
        sl = slice(64 * i, 64 * (i + 1))
        assert np.array_equal(Q.slice_symbols(res["x"][sl], M, "fp32"), res["sym"][sl])


def test_deterministic():
    d = wl.generate(wl.Spec(N=128, K=32, batch=256, rho=0.5, qam=64, snr_db=12.0, seed=8))
    a = gpu_detect(d, 6, dict(gram="bf16", mv="bf16", refine_steps=1), L=8)
    b = gpu_detect(d, 6, dict(gram="bf16", mv="bf16", refine_steps=1), L=8)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["rel_res"], b["rel_res"])
