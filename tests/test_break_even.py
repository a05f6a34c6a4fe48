"""Remark 4's break-even criterion and the iteration counts it compares, in
the oracle (pinned by the cost model it must agree with) and in the library's
host functions (fpcg_choose_method, fpcg_kappa_cg_batch; no GPU needed)."""
import numpy as np
import pytest

from oracle import analysis as An


@pytest.mark.parametrize("kappa", [1.0, 1.5, 4.0, 40.0, 141.0, 1e4])
@pytest.mark.parametrize("tol", [1e-2, 1e-3, 1e-6])
def test_cg_iterations_is_the_first_count_meeting_the_bound(kappa, tol):
    k = An.cg_iterations(kappa, tol)
    q = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    assert k >= 1
    if kappa > 1:
        assert 2 * q ** k <= tol * (1 + 1e-12) and 2 * q ** (k - 1) > tol


def test_break_even_is_the_cheaper_total_cost():
    """The criterion of Remark 4 is C_PCG < C_CG rearranged: on a grid of
    inputs it picks whichever total cost of the cost model is smaller."""
    for N in (8, 16, 32, 64, 128):
        for L in (1, 2, 4, 8, 16, 32):
            if L > N or N % L:
                continue
            for kappa in (2.0, 20.0, 141.0, 2000.0):
                for kb in (1.0, 1.5, 0.5 * kappa + 0.5, kappa):
                    for mv in ("fp16", "fp32"):
                        choice, kc, kp = An.break_even(N, L, kappa, kb, 1e-3, mv, mv, "fp32")
                        c_cg = An.cost_cg(N, kc, mv)
                        c_pcg = An.cost_fpbjcg(N, L, kp, mv, "fp32")
                        if c_pcg != c_cg:
                            assert (choice == L) == (c_pcg < c_cg), (N, L, kappa, kb, mv)


def test_break_even_trends_of_remark4():
    """For small N and large L the setup outweighs the saving (FP-CG); for
    large N and moderate L it is amortised (FP-BJ-CG)."""
    kappa, kb = 40.0, 8.0
    assert An.break_even(128, 8, kappa, kb, 1e-3)[0] == 8
    assert An.break_even(16, 16, kappa, kb, 1e-3)[0] == 0
    picks = [An.break_even(32, L, kappa, kb, 1e-3)[0] > 0 for L in (2, 4, 8, 16, 32)]
    assert picks[0] and not picks[-1]
    assert picks == sorted(picks, reverse=True)   # once FP-CG wins, larger L does not switch back


def test_library_break_even_matches_oracle():
    from paper_2504_09820_gb300 import fpcg as F
    for N, L in ((16, 4), (32, 8), (64, 4), (64, 16), (128, 8), (32, 32)):
        for kappa in (1.0, 3.0, 40.0, 141.0, 5e3):
            for kb in (1.0, 2.0, kappa):
                for mvs in (("fp16", "fp16"), ("bf16", "fp16"), ("fp32", "fp16"), ("fp32", "fp32")):
                    want = An.break_even(N, L, kappa, kb, 1e-3, mvs[0], mvs[1], "fp32")
                    got = F.fpcg_choose_method(N, L, kappa, kb, 1e-3, mvs[0], mvs[1], "fp32")
                    assert got == want, (N, L, kappa, kb, mvs)
    with pytest.raises(F.FpcgError):
        F.fpcg_choose_method(32, 5, 10.0, 2.0, 1e-3)   # L does not divide K


def test_library_kappa_batch_matches_single():
    from paper_2504_09820_gb300 import fpcg as F
    rng = np.random.default_rng(5)
    iters, batch = 6, 5
    c = np.zeros((batch, 2, iters), dtype=np.float32)
    c[:, 0] = rng.uniform(0.5, 2.0, (batch, iters))
    c[:, 1] = rng.uniform(0.0, 0.9, (batch, iters))
    c[3, 0, 2:] = 0.0                                  # a solve that stopped after 2 steps
    k = F.fpcg_kappa_cg_batch(c, 4)
    for s in range(batch):
        if s == 3:
            assert np.isnan(k[s])
        else:
            want = F.fpcg_kappa_cg(c[s, 0, :4].astype(np.float64), c[s, 1, :3].astype(np.float64))
            assert k[s] == pytest.approx(want, rel=1e-12)
