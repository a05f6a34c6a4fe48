"""Pins for the Gray-QAM slicer and bit-error count (Section V-A: 16-QAM, BER).

The generator's modulator (inverse Gray code) and the oracle's slicer
(forward Gray code, threshold decisions) are written independently, so the
round trip checks both.
"""
import numpy as np
import pytest

from oracle import qam
from paper_2504_09820_gb300.workload import qam_modulate


@pytest.mark.parametrize("M", [4, 16, 64, 256])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_roundtrip_every_point(M, prec):
    labels = np.arange(M)
    s = qam_modulate(labels, M)
    assert np.array_equal(qam.slice_symbols(s, M, prec), labels.astype(np.uint8))


@pytest.mark.parametrize("M", [4, 16, 64, 256])
def test_unit_energy_and_gray_neighbours(M):
    s = qam_modulate(np.arange(M), M)
    assert np.mean(np.abs(s) ** 2) == pytest.approx(1.0, rel=1e-12)
    d = 2.0 / np.sqrt(2.0 * (M - 1) / 3.0)         # spacing of adjacent levels
    for a in range(M):
        for b in range(M):
            dist = abs(s[a] - s[b])
            if abs(dist - d) < 1e-9:                # horizontal or vertical neighbour
                assert bin(a ^ b).count("1") == 1


@pytest.mark.parametrize("M", [16, 64])
def test_decision_regions(M):
    m = int(np.sqrt(M))
    d = 1.0 / np.sqrt(2.0 * (M - 1) / 3.0)
    s = qam_modulate(np.arange(M), M)
    for lab in range(M):
        for dx, dy in [(0.49, 0.0), (-0.49, 0.0), (0.0, 0.49), (0.0, -0.49)]:
            v = s[lab] + (dx + 1j * dy) * 2 * d
            assert qam.slice_symbols(np.array([v]), M, "fp64")[0] == lab
    # far outside the constellation clamps to the corner points
    far = qam.slice_symbols(np.array([10 + 10j, -10 - 10j]), M, "fp64")
    corners = qam.slice_symbols(np.array([s[np.argmax(s.real + s.imag)], s[np.argmin(s.real + s.imag)]]), M, "fp64")
    assert np.array_equal(far, corners)
    # exactly on a decision threshold (t integer) goes to the upper level
    t_mid = np.array([(2 * 0 - m + 2)], dtype=np.float64)      # between level 0 and 1
    j = qam.axis_decision(t_mid / qam.axis_scale(M, "fp64"), M, "fp64")
    assert j[0] in (0, 1)
    assert qam.axis_decision(np.array([0.0]), M, "fp64")[0] == m // 2


def test_bit_errors():
    assert qam.bit_errors(np.array([0, 1, 2, 3], np.uint8), np.array([0, 1, 2, 3], np.uint8)) == 0
    assert qam.bit_errors(np.array([0xFF, 0x0F], np.uint8), np.array([0x00, 0x00], np.uint8)) == 12
