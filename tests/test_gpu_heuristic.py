"""Precision selection from the kernels' own CG step sizes (Sections III-B and
IV-B): kappa estimates from the alpha_j, beta_j that fpcg_detect_coeffs
exports, against the oracle's condition numbers of the same matrices; the
formats eq. heuristic / eq. heuristic_bj choose from them, against the
oracle's choice; and the plan option that applies the choice per class, with
Remark 4's break-even criterion between FP-CG and FP-BJ-CG."""
import numpy as np
import pytest
import torch

from oracle import analysis as An
from oracle import detect as D
from paper_2504_09820_gb300 import fpcg as F
from paper_2504_09820_gb300 import workload as wl

from gpu_helpers import check_reduced_parity, oracle_detect, to_dev

pytestmark = pytest.mark.gpu

FP32 = dict(gram="fp32", mv="fp32", ip="fp32", w="fp32")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()


def _coeffs(d, m, L=0):
    g = to_dev(d)
    B, K, _ = d["H"].shape
    c = torch.empty((B, 2, m), dtype=torch.float32, device="cuda")
    x = torch.empty((B, K), dtype=torch.complex64, device="cuda")
    F.fpcg_detect_coeffs(g["H"], g["y"], g["sigma2"], g["qam"], m, L, F.precision(**FP32), x, c)
    torch.cuda.synchronize()
    return c.cpu().numpy()


def _near_threshold(K, kappa, rel=0.05):
    """kappa within rel of a value where eq. heuristic switches format."""
    out = np.zeros(len(kappa), dtype=bool)
    for name in An.TABLE_I_ORDER:
        from oracle.formats import FORMATS
        k_switch = 1.0 / (FORMATS[name].u * K ** 1.5) ** 2   # u = 1 / (K^1.5 sqrt(kappa))
        out |= np.abs(kappa / k_switch - 1) < rel
    return out


@pytest.mark.parametrize("L", [0, 8])
def test_kappa_from_gpu_step_sizes(L):
    d = wl.generate(wl.Spec(N=128, K=32, batch=256, rho=0.5, qam=16, snr_db=12.0, seed=901))
    K = 32
    c = _coeffs(d, K, L)
    kh = F.fpcg_kappa_cg_batch(c)
    A, _ = D.gram_emul(d["H"], d["y"], d["sigma2"], "fp32")
    if L:
        Md, _ = D.bj_inverse(A, L, "fp64")
        kap = An.kappa(An.bj_preconditioned(A, Md))
    else:
        kap = An.kappa(A)
    ratio = kh / kap
    # Ritz values lie inside the spectrum (up to the fp32 iteration's rounding);
    # after K steps the extreme ones have converged
    assert np.all(ratio < 1.0 + 1e-2), ratio.max()
    assert np.median(ratio) > 0.97 and ratio.min() > 0.7, (np.median(ratio), ratio.min())
    # the formats chosen from the estimates are the oracle's (away from a switch point)
    ok = ~_near_threshold(K, kap)
    got = np.array([F.fpcg_choose_precision(K, k)[0] for k in kh])
    want = np.array([An.choose_precision(K, k) for k in kap])
    assert np.array_equal(got[ok], want[ok]), (got[ok] != want[ok]).sum()


def test_plan_autoprec_per_class():
    """fpcg_plan_autoprec on an uneven batch: every class's matvec format and
    method are what eq. heuristic(_bj) and Remark 4 give for the oracle's
    median condition number of the same sampled systems, and the plan then
    detects at those precisions within the reduced-precision bar."""
    spec = wl.mixed_kron(batch=600, seed=1004)
    spec.ks = (16, 32, 64)
    d = wl.generate_mixed(spec)
    prec = dict(gram="bf16", mv="fp16", refine_steps=1, resid="fp32")
    plan = F.Plan(d["n"], d["k"], 7, F.precision(**prec), block_L=4)
    g = plan.pack(d["H"], d["y"], d["sigma2"], d["qam"], d["tx"])
    plan.autoprec(g["H"], g["y"], g["sigma2"], tol=1e-3)
    x = torch.zeros(plan.totals[2], dtype=torch.complex64, device="cuda")
    sym = torch.zeros(plan.totals[2], dtype=torch.uint8, device="cuda")
    plan.run(g["H"], g["y"], g["sigma2"], g["qam"], x, sym)
    torch.cuda.synchronize()
    xs = plan.unpack(x, d["k"])
    for c in plan.classes():
        idx = plan.order[c["first"]:c["first"] + c["count"]]
        samp = idx[:64]
        K = c["k"]
        H = np.stack([d["H"][i] for i in samp])
        y = np.stack([d["y"][i] for i in samp])
        A, _ = D.gram_emul(H, y, d["sigma2"][samp], "fp32")
        kap = np.median(An.kappa(A))
        Md, _ = D.bj_inverse(A, 4, "fp64")
        kb = np.median(An.kappa(An.bj_preconditioned(A, Md)))
        pick = lambda k: "fp32" if An.choose_precision(K, k) == "fp64" else An.choose_precision(K, k)
        choice, _, _ = An.break_even(K, 4, kap, kb, 1e-3, pick(kap), pick(kb), "fp32")
        if not _near_threshold(K, np.array([kap, kb]), 0.1).any():
            assert c["block_L"] == choice, (c, kap, kb)
            assert c["mv"] == pick(kb if choice else kap), (c, kap, kb)
        assert c["kappa"] == pytest.approx(kb if c["block_L"] else kap, rel=0.15)  # min(K, 32) steps
        # detection at the chosen precisions, against the oracle at the same
        pk = dict(prec, mv=c["mv"])
        cd = {"H": np.stack([d["H"][i] for i in idx]), "y": np.stack([d["y"][i] for i in idx]),
              "sigma2": d["sigma2"][idx], "qam": d["qam"][idx], "tx": np.stack([d["tx"][i] for i in idx])}
        ref = oracle_detect(cd, 7, pk, L=(c["block_L"] or None))
        check_reduced_parity(cd, np.stack([xs[i] for i in idx]), ref["x"], 7, pk, L=(c["block_L"] or None))
