"""Gray-mapped square QAM hard slicer and bit-error count.

Section V-A simulates 16-QAM and reports bit error rate; it does not spell out
the constellation.  Reading used here (and by the CUDA slicer):

* Unit average energy square M-QAM, M in {4, 16, 64, 256}, m = sqrt(M) levels
  per axis at (2j - (m-1)) * d, j = 0..m-1, d = 1/sqrt(2(M-1)/3).
* Symbol label: Gray(j_I) in the high log2(m) bits, Gray(j_Q) in the low ones,
  Gray(j) = j xor (j >> 1); j_I from the real part, j_Q from the imaginary part.
* Decision in the precision of the estimate ("fp32" or "fp64"):
  t = fl(v * fl(sqrt(2(M-1)/3))), then j = number of thresholds
  2k - m + 2 (k = 0..m-2) that t reaches.  The thresholds are integers, so the
  comparisons are exact and a tie goes to the upper level; values beyond the
  outer levels clamp to them.
* BER = popcount(label xor transmitted label) / (K * log2 M).
"""

import numpy as np

from .formats import fl

QAM_ORDERS = (4, 16, 64, 256)


def _check(M):
    if M not in QAM_ORDERS:
        raise ValueError(f"unsupported QAM order {M}")
    m = int(round(np.sqrt(M)))
    return m, int(np.log2(m))


def axis_scale(M, prec):
    """fl_prec(sqrt(2(M-1)/3)) = 1/d, the factor that maps the axis to odd integers."""
    return fl(np.sqrt(2.0 * (M - 1) / 3.0), prec)


def axis_decision(v, M, prec):
    """Nearest level index j (0..m-1) of real values ``v`` on one axis."""
    m, _ = _check(M)
    v = fl(np.asarray(v, dtype=np.float64), prec)
    t = fl(v * axis_scale(M, prec), prec)
    j = np.zeros(t.shape, dtype=np.int64)
    for k in range(m - 1):
        j += (t >= 2 * k - m + 2).astype(np.int64)
    return j


def gray(j):
    j = np.asarray(j, dtype=np.int64)
    return j ^ (j >> 1)


def slice_symbols(x, M, prec="fp32"):
    """Hard-decision Gray labels of complex estimates ``x`` (any shape)."""
    _, b = _check(M)
    x = np.asarray(x, dtype=np.complex128)
    gi = gray(axis_decision(x.real, M, prec))
    gq = gray(axis_decision(x.imag, M, prec))
    return ((gi << b) | gq).astype(np.uint8)


def bit_errors(labels, tx):
    """Total number of differing bits between two label arrays."""
    d = np.bitwise_xor(np.asarray(labels, dtype=np.uint8), np.asarray(tx, dtype=np.uint8))
    return int(np.unpackbits(d.reshape(-1, 1), axis=1).sum())


def bits_per_symbol(M):
    return int(np.log2(M))
