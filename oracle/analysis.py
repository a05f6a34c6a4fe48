"""Closed forms the paper states: cost model, precision heuristic, bounds.

* Cost model (Section V-A.1; used for every percentage in Section V-C,
  Remark 3 and Appendix E): multiplications weighted fp16 : fp32 : fp64 =
  1 : 2 : 4.  CG spends N^2 per iteration on A p (the bottleneck named in
  Section II and Section IV-B), block-Jacobi adds N*L per iteration for
  z = M_d r and d*L^3 once for the block inversion (both at u_W = fp64), and
  direct LMMSE costs N^3 (at fp64).  N is the Gram dimension (K in this
  build's letters).
* Heuristic (eq. heuristic / eq. heuristic_bj): u_MV < 1 / (N^1.5 sqrt(kappa)),
  then take the lowest-precision format of Table I whose u satisfies it.
* Theorem 2: ||b - A x_i - r_i|| / (||A|| ||x||) <= (1+i) u_W + Upsilon_i Theta_i.
* Appendix B, eq. var: Var{h_n^H h_i} = 1/M + (2/M^2)[s(M-1) - s^2(1 - z^(2(M-1)))]
  with s = z^2 / (1 - z^2), z the correlation coefficient, M antennas.
"""

import numpy as np

from .formats import FORMATS

WEIGHT = {"fp16": 1, "bf16": 1, "fp32": 2, "fp64": 4}


def cost_cg(N, iters, mv="fp64"):
    """Weighted multiplications of (FP-)CG: iters * N^2 at the matvec precision."""
    return iters * N * N * WEIGHT[mv]


def cost_bj_setup(N, L, w="fp64"):
    """Inversion of d = N/L diagonal L x L blocks: d * L^3 at u_W."""
    return (N // L) * L ** 3 * WEIGHT[w]


def cost_fpbjcg(N, L, iters, mv="fp16", w="fp64"):
    """FP-BJ-CG: matvecs at u_MV + M_d r (N*L per iteration at u_W) + setup."""
    return cost_cg(N, iters, mv) + iters * N * L * WEIGHT[w] + cost_bj_setup(N, L, w)


def cost_lmmse(N):
    """Direct LMMSE inversion: N^3 multiplications at fp64."""
    return N ** 3 * WEIGHT["fp64"]


def reduction(cost, ref):
    """Fractional cost reduction of ``cost`` relative to ``ref``."""
    return 1.0 - cost / ref


def heuristic_u_mv(N, kappa):
    """Upper bound on u_MV from eq. heuristic (use kappa of the preconditioned
    matrix for eq. heuristic_bj)."""
    return 1.0 / (N ** 1.5 * np.sqrt(kappa))


# Table I formats from the lowest to the highest precision.
TABLE_I_ORDER = ("bf16", "fp16", "fp32", "fp64")


def choose_precision(N, kappa):
    """Lowest-precision Table I format whose unit roundoff meets the heuristic."""
    bound = heuristic_u_mv(N, kappa)
    for name in TABLE_I_ORDER:
        if FORMATS[name].u < bound:
            return name
    return "fp64"


def gamma(n, u):
    """gamma_n = n u / (1 - n u), eq. gamma (Lemma 1)."""
    return n * u / (1.0 - n * u)


def theorem2_bound(i, N, u_w, u_mv, theta):
    """Right-hand side (1+i) u_W + Upsilon_i Theta_i of Theorem 2."""
    ups = ((8 * np.sqrt(2) + 6) * i + 1) * u_w + (2 * i + 1) * 2 * np.sqrt(2) * N ** 1.5 * u_mv
    return (1 + i) * u_w + ups * theta


def gram_var_closed(M, zeta):
    """Appendix B, eq. var."""
    s = zeta ** 2 / (1 - zeta ** 2)
    return 1.0 / M + 2.0 / M ** 2 * (s * (M - 1) - s ** 2 * (1 - zeta ** (2 * (M - 1))))


def gram_var_sum(M, zeta):
    """The same variance from its defining sum 1/M + (2/M^2) sum_{m<o} [R_r]_mo^2."""
    k = np.arange(1, M)
    return 1.0 / M + 2.0 / M ** 2 * np.sum((M - k) * zeta ** (2.0 * k))


def kappa(A):
    """2-norm condition number of each Hermitian positive definite matrix."""
    ev = np.linalg.eigvalsh(np.asarray(A, dtype=np.complex128))
    return ev[..., -1] / ev[..., 0]


def bj_preconditioned(A, Md_blocks):
    """A_bar = M_d^{1/2} A M_d^{1/2} (Theorem 4), from the block inverses."""
    B, d, L, _ = Md_blocks.shape
    K = d * L
    Mh = np.zeros((B, K, K), dtype=np.complex128)
    for i in range(d):
        w, V = np.linalg.eigh(Md_blocks[:, i])
        Mh[:, i * L:(i + 1) * L, i * L:(i + 1) * L] = (V * np.sqrt(w)[:, None, :]) @ np.conj(np.swapaxes(V, -1, -2))
    return Mh @ np.asarray(A, dtype=np.complex128) @ Mh
