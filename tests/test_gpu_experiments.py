"""The Section V experiment runner on a small number of trials: the curves
behave as the method says (LMMSE is fp64 CG at 2K iterations, CG converges
to it, block-Jacobi converges faster at zeta = 0.8)."""
import numpy as np
import pytest
import torch

from paper_2504_09820_gb300 import experiments as X
from paper_2504_09820_gb300 import fpcg as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()


def test_convergence_curves_small():
    spec = X._spec(0.8, seed=3)
    r = X.ber_curves(spec, [("cg64", None), ("fp16", X.L_BJ)], [2, 6, 64], 4000)
    cg, bj, lm = r["curves"]["cg64"], r["curves"]["fp16_bj8"], r["lmmse"]
    assert cg[64] == lm                       # the same fp64 algorithm, same iterations
    assert cg[2] > cg[6] > lm * 0.98          # CG approaches LMMSE from above
    assert bj[6] < cg[6]                      # block Jacobi converges faster at zeta = 0.8
    assert abs(bj[64] - lm) < 0.1 * lm


def test_kappa_sample_bj_improves_conditioning():
    k = X.kappa_sample(X._spec(0.8, seed=4, rt_block=True), count=256, bj_L=X.L_BJ)
    assert np.all(k["kappa"] >= 1.0) and np.all(k["kappa_bar"] >= 1.0)
    assert np.mean(k["kappa_bar"]) < np.mean(k["kappa"])   # Theorem 5 on the average


def test_time_varying_runs():
    r = X.exp_time_varying(2000, snrs=(10,), steps=2)
    b = r["ber"]
    assert 0.0 <= b["lmmse"][0] <= b["per_system"][0] * 1.2 + 1e-3
    assert r["format_once"] in ("bf16", "fp16", "fp32", "fp64")
