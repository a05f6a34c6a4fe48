"""Host-side helpers of the Section V experiment runner (no GPU)."""
import numpy as np
import pytest

from paper_2504_09820_gb300 import experiments as X


def test_iterations_to_lmmse():
    curve = {1: 0.2, 2: 0.1, 3: 0.052, 4: 0.0505, 5: 0.05}
    assert X.iterations_to_lmmse(curve, 0.05) == 3          # within 5%
    assert X.iterations_to_lmmse(curve, 0.05, rel=0.01) == 4
    assert X.iterations_to_lmmse({1: 0.3}, 0.05) is None


def test_snr_gap_of_shifted_waterfall():
    """Two BER curves that are the same function of SNR, 1.2 dB apart."""
    snrs = list(range(0, 31, 2))
    f = lambda s: 0.5 * np.exp(-0.5 * 10 ** (s / 10.0) / 4.0)
    ref = [f(s) for s in snrs]
    late = [f(s - 1.2) for s in snrs]
    for lvl in (1e-2, 1e-3):
        assert X.snr_gap(snrs, ref, late, lvl) == pytest.approx(1.2, abs=0.25)
    assert X.snr_gap(snrs, ref, [0.4] * len(snrs), 1e-3) is None


def test_variant_precisions():
    from paper_2504_09820_gb300 import fpcg as F
    p = X.prec_of("mv_bf16")
    assert (p.gram, p.mv, p.ip, p.w, p.refine_steps) == (F.FORMAT["fp32"], F.FORMAT["bf16"], F.FORMAT["fp32"],
                                                         F.FORMAT["fp32"], 0)
    p = X.prec_of("ip_bf16")
    assert (p.mv, p.ip) == (F.FORMAT["fp32"], F.FORMAT["bf16"])
    assert X.prec_of("cg64").w == F.FORMAT["fp64"] and X.prec_of("lmmse").mv == F.FORMAT["fp64"]
