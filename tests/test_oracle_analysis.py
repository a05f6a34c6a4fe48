"""Pins for the paper's closed forms: the cost model of Section V-A.1 against
every percentage printed in Section V-C, Remark 3 and Appendix E; Example 1;
the heuristic of eq. heuristic against its Section V-B.2 worked example; and
the Gram variance of Appendix B against its defining sum and the generator."""
import json
import os

import numpy as np
import pytest

from oracle import analysis as An
from oracle.formats import FORMATS
from paper_2504_09820_gb300 import workload as wl


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def test_cost_model_reproduces_printed_percentages(golden_dir):
    g = _load(golden_dir, "cost_model.json")
    N, L = g["N"], g["L"]
    for c in g["cases"]:
        if c["method"] == "fpcg":
            cost = An.cost_cg(N, c["iters"], c["mv"])
        else:
            cost = An.cost_fpbjcg(N, L, c["iters"], c["mv"], "fp64")
        ref = An.cost_cg(N, c["ref_iters"], "fp64") if c["ref"] == "cg" else An.cost_lmmse(N)
        pct = 100.0 * An.reduction(cost, ref)
        tol = c.get("tolerance_pct", 0.05)
        assert abs(pct - c["reduction_pct"]) <= tol, (c["cite"], pct)


def test_bj_setup_equals_two_cg_iterations(golden_dir):
    g = _load(golden_dir, "cost_model.json")
    ratio = An.cost_bj_setup(g["N"], g["L"], "fp64") / An.cost_cg(g["N"], 1, "fp64")
    assert ratio == g["bj_setup_in_cg_iterations"]["value"]


def test_example1_capacity(golden_dir):
    e = _load(golden_dir, "cost_model.json")["example1"]
    flops = e["iters"] * e["N"] ** 2
    assert flops == e["flops_per_subchannel"]
    tflops = flops * e["subcarriers"] / e["slot_s"] / 1e12
    assert tflops == pytest.approx(e["tflops"], rel=0.05)


def test_heuristic_worked_example(golden_dir):
    g = _load(golden_dir, "heuristic_example.json")
    # the bound 1.33e-3 at N = 32 corresponds to kappa = (1/(1.33e-3 * 32^1.5))^2
    kappa = (1.0 / (g["u_mv_bound"] * g["N"] ** 1.5)) ** 2
    assert An.heuristic_u_mv(g["N"], kappa) == pytest.approx(g["u_mv_bound"], rel=1e-12)
    assert An.choose_precision(g["N"], kappa) == g["selected"]
    # selection walks Table I from the lowest precision
    assert An.choose_precision(g["N"], 1.0) == "bf16"          # bound 5.5e-3 > 3.91e-3
    assert An.choose_precision(g["N"], 1e6) == "fp32"
    assert An.choose_precision(g["N"], 1e30) == "fp64"


def test_heuristic_monte_carlo_lands_on_fp16():
    """The worked example's channel (zeta = 0.5, M = 256, N = 32, 20 dB) has a
    mean condition number whose heuristic bound falls in fp16's slot."""
    from oracle import detect as D
    d = wl.generate(wl.Spec(N=256, K=32, batch=64, rho=0.5, qam=16, snr_db=20.0, seed=11))
    A, _ = D.gram_mf(d["H"], d["y"], d["sigma2"])
    bound = An.heuristic_u_mv(32, np.mean(An.kappa(A)))
    assert FORMATS["fp16"].u < bound < FORMATS["bf16"].u


@pytest.mark.parametrize("M,zeta", [(8, 0.5), (64, 0.5), (256, 0.8), (128, 0.0)])
def test_gram_variance_closed_form(M, zeta):
    assert An.gram_var_closed(M, zeta) == pytest.approx(An.gram_var_sum(M, zeta), rel=1e-12) \
        if zeta > 0 else An.gram_var_sum(M, zeta) == pytest.approx(1.0 / M)


def test_generator_gram_statistics():
    """Theorem 3's proof: E[H^H H] = R_t at any M; Var of an entry = eq. var."""
    M, K, zeta, n = 32, 4, 0.6, 4096
    d = wl.generate(wl.Spec(N=M, K=K, batch=n, rho=zeta, qam=4, snr_db=10.0, seed=3))
    H = d["H"].astype(np.complex128)
    G = np.conj(H) @ np.swapaxes(H, 1, 2)
    mean = G.mean(axis=0)
    Rt = wl.exp_corr(K, zeta)
    assert np.abs(mean - Rt).max() < 5 * np.sqrt(An.gram_var_closed(M, zeta) / n) + 1e-3
    v = G[:, 0, 2].var()
    assert v == pytest.approx(An.gram_var_closed(M, zeta), rel=0.1)


def test_theorem2_bound_scaling_matches_heuristic():
    """The u_MV term of Theorem 2 is O(N^{3/2} u_MV) (eq. or_ph), the power
    eq. heuristic is derived from, and grows as (2i+1) with the iteration."""
    u = 2.0 ** -11
    b1 = An.theorem2_bound(3, 16, 0.0, u, 1.0)
    b4 = An.theorem2_bound(3, 64, 0.0, u, 1.0)
    assert b4 / b1 == pytest.approx(4 ** 1.5, rel=1e-12)
    assert An.heuristic_u_mv(16, 1.0) / An.heuristic_u_mv(64, 1.0) == pytest.approx(4 ** 1.5, rel=1e-12)
    assert An.theorem2_bound(5, 16, 0.0, u, 1.0) / An.theorem2_bound(0, 16, 0.0, u, 1.0) == pytest.approx(11.0)
    # with u_MV = 0 the bound is linear in u_W with slope (1+i) + ((8 sqrt2 + 6) i + 1) Theta
    assert An.theorem2_bound(2, 16, 1.0, 0.0, 1.0) == pytest.approx(3 + (8 * np.sqrt(2) + 6) * 2 + 1)
