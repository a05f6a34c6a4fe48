"""Finite-precision number formats and the rounding operator fl(.).

Definition 1 (Section III-A) defines fl(.) as rounding a real number into a
floating-point system F; Table I lists the formats the paper uses (bfloat16,
fp16, fp32, fp64) by significand bits, exponent bits, unit roundoff u,
smallest normal x_min and largest finite x_max.  The build adds OCP FP8 E4M3
("e4m3fn": 4 significand bits including the implicit one, exponent bias 7,
no infinities, largest finite 448) for the quantised matrix-vector product.

Rounding is round-to-nearest, ties-to-even, with gradual underflow
(subnormals kept).  Overflow goes to +-inf for the IEEE formats; e4m3
saturates to +-448 (the "satfinite" conversion a kernel uses).

Table I prints u = 4.88e-16 for fp64; the unit roundoff of a 53-bit
significand is 2^-53 = 1.11e-16, which is what this module uses.
"""

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Format:
    name: str
    p: int            # significand bits, implicit leading bit included
    emin: int         # exponent of the smallest normal number
    emax: int         # exponent of the largest binade
    xmax: float       # largest finite value
    saturate: bool    # overflow saturates to +-xmax instead of +-inf

    @property
    def u(self) -> float:
        """Unit roundoff 2^-p (Table I, column u)."""
        return 2.0 ** (-self.p)

    @property
    def xmin(self) -> float:
        """Smallest positive normal number 2^emin (Table I, column x_min)."""
        return 2.0 ** self.emin


def _ieee(name, p, ebits):
    bias = 2 ** (ebits - 1) - 1
    emax = bias
    return Format(name, p, 1 - bias, emax, (2.0 - 2.0 ** (1 - p)) * 2.0 ** emax, False)


FORMATS = {
    "bf16": _ieee("bf16", 8, 8),
    "fp16": _ieee("fp16", 11, 5),
    "fp32": _ieee("fp32", 24, 8),
    "fp64": _ieee("fp64", 53, 11),
    # e4m3fn: bias 7, exponent field 1111 is a normal binade except for the
    # all-ones mantissa (NaN), so the largest finite value is 1.75 * 2^8.
    "e4m3": Format("e4m3", 4, -6, 8, 448.0, True),
}


def fl(x, fmt):
    """Round every element of real array ``x`` to format ``fmt`` (Definition 1).

    The value is scaled onto the integer grid of the format's spacing at its
    own binade (clamped at emin for subnormals), rounded half-to-even there,
    and scaled back.  All steps are exact in float64 for the formats here.
    """
    f = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    if fmt == "fp64":
        return x.copy()
    ax = np.abs(x)
    _, e = np.frexp(ax)                      # ax = m * 2^e, 0.5 <= m < 1
    lead = np.maximum(e - 1, f.emin)          # exponent of the leading bit
    q = np.ldexp(1.0, lead - (f.p - 1))       # spacing of F around x
    r = np.rint(x / q) * q                    # np.rint rounds half to even
    big = np.abs(r) > f.xmax
    if np.any(big):
        if f.saturate:
            r = np.where(big, np.copysign(f.xmax, x), r)
        else:
            r = np.where(big, np.copysign(np.inf, x), r)
    return r


def flc(z, fmt):
    """Round a complex array component-wise (real and imaginary part separately)."""
    z = np.asarray(z, dtype=np.complex128)
    return fl(z.real, fmt) + 1j * fl(z.imag, fmt)


# ---------------------------------------------------------------------------
# FP8 e4m3 with per-block power-of-two scales (not in the paper).
#
# A block is a run of ``block`` consecutive real components (real and
# imaginary parts interleaved, as a complex row is stored).  Its scale is the
# smallest power of two s with amax <= 448*s (s = 1 when the block is all
# zero), so dividing by s is exact and the largest element lands in
# (224, 448].  The stored value is q*s with q = fl_e4m3(v/s).
# ---------------------------------------------------------------------------

E4M3_MAX = 448.0


def e4m3_block_scale(amax):
    """Smallest power of two s with amax <= 448*s; 1 where amax == 0."""
    amax = np.asarray(amax, dtype=np.float64)
    m, e = np.frexp(amax)                    # amax = m * 2^e, 0.5 <= m < 1
    # 448 = 0.875 * 2^9: m*2^(e-k) <= 0.875*2^9  <=>  k >= e-9 (m <= .875) else e-8
    k = np.where(m <= 0.875, e - 9, e - 8)
    s = np.ldexp(1.0, k)
    return np.where(amax > 0, s, 1.0)


def quant_e4m3_rows(v, block=32):
    """Quantise real array ``v`` (..., n) along its last axis in blocks.

    Returns (dequantised values, scales of shape (..., ceil(n/block))).  The
    last block of a row may be shorter than ``block``.
    """
    v = np.asarray(v, dtype=np.float64)
    n = v.shape[-1]
    nb = -(-n // block)
    pad = nb * block - n
    vp = np.concatenate([v, np.zeros(v.shape[:-1] + (pad,))], axis=-1) if pad else v
    vb = vp.reshape(v.shape[:-1] + (nb, block))
    s = e4m3_block_scale(np.max(np.abs(vb), axis=-1))
    q = fl(vb / s[..., None], "e4m3")
    out = (q * s[..., None]).reshape(vp.shape)[..., :n]
    return out, s


def complex_to_interleaved(z):
    """(..., n) complex -> (..., 2n) real with re/im interleaved (storage order)."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.empty(z.shape[:-1] + (2 * z.shape[-1],))
    out[..., 0::2] = z.real
    out[..., 1::2] = z.imag
    return out


def interleaved_to_complex(v):
    v = np.asarray(v, dtype=np.float64)
    return v[..., 0::2] + 1j * v[..., 1::2]


def quant_e4m3_complex_rows(z, block=32):
    """Per-block e4m3 quantisation of complex rows stored re/im interleaved."""
    q, s = quant_e4m3_rows(complex_to_interleaved(z), block)
    return interleaved_to_complex(q), s


def round_matvec_operand(z, fmt, block=32):
    """Round a complex matrix/vector operand of A.p to the matvec format.

    For the IEEE formats this is component-wise fl(.); for e4m3 it is the
    per-block scaled quantisation along the last axis (rows of A, or the
    whole vector p).
    """
    if fmt == "e4m3":
        return quant_e4m3_complex_rows(z, block)[0]
    return flc(z, fmt)
