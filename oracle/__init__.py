"""CPU parity oracle for finite-precision CG detection (arXiv 2504.09820).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain, obviously-correct
reference that the CUDA path is checked against.  Only the test suite, the
package's ``smoke()`` self-check and the ``cpu_baseline`` leg of ``bench.py``
(plus ``bench.py --impl reference``) may import it.  The CUDA library never
calls into it and shares no code with it: the only thing both sides share is
the seeded synthetic input generator, which holds none of the detector's
arithmetic.

Everything here computes in float64 (numpy), vectorised over the batch of
independent systems only; within one system every step follows the paper's
definition or algorithm in the paper's order:

* ``formats``  -- the rounding operator fl(.) of Definition 1 for the formats of
  Table I (bf16, fp16, fp32, fp64) plus OCP FP8 e4m3, and the per-block
  power-of-two scaled e4m3 quantiser used for the reduced-precision matvec.
* ``detect``   -- Gram / matched filter (Section II, eq. inversion), the direct
  Cholesky LMMSE solve, plain CG (Algorithm 1), FP-CG (Algorithm 2), the
  block-Jacobi preconditioner (eq. pre_BJ) and FP-BJ-CG (Algorithm 3), the
  iterative-refinement outer loop, and the full detection pipeline.
* ``qam``      -- Gray-mapped square QAM hard slicer and bit-error counting
  (Section V-A uses 16-QAM and reports BER).
* ``analysis`` -- the paper's weighted multiplication-count cost model
  (Section V-A.1), the precision-selection heuristic (eq. heuristic and
  eq. heuristic_bj), the attainable-accuracy bound of Theorem 2, and the
  Gram variance closed form of Appendix B.

Parity status: every function is pinned by a ``-m "not gpu"`` test except the
ones listed as "parity unpinned" in their own docstrings.
"""

from . import formats, qam, detect, analysis  # noqa: F401
