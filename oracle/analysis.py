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


def cg_iterations(kappa, tol):
    """Iterations k that the classical CG bound 2 q^k <= tol asks for, with
    q = (sqrt(kappa) - 1) / (sqrt(kappa) + 1) (the A-norm error bound the
    iteration counts of a break-even comparison are read from); 1 for kappa = 1."""
    sk = np.sqrt(float(kappa))
    q = (sk - 1.0) / (sk + 1.0)
    if q <= 0.0:
        return 1
    return int(np.ceil(np.log(tol / 2.0) / np.log(q)))


def break_even(N, L, kappa, kappa_bar, tol, mv_cg="fp16", mv_bj="fp16", w="fp32"):
    """Remark 4's break-even criterion: FP-BJ-CG (block L) is preferable when
    k_CG - k_PCG > C_BJ / C_CG^it + k_PCG (C_PCG^it / C_CG^it - 1), with the
    per-iteration and setup costs of the cost model (Section V-A.1: C_CG^it =
    N^2 w(mv_cg), C_PCG^it = N^2 w(mv_bj) + N L w(w), C_BJ = (N/L) L^3 w(w))
    and the iteration counts of cg_iterations for kappa and kappa_bar.
    Returns (L or 0, k_CG, k_PCG)."""
    k_cg, k_pcg = cg_iterations(kappa, tol), cg_iterations(kappa_bar, tol)
    c_it = N * N * WEIGHT[mv_cg]
    p_it = N * N * WEIGHT[mv_bj] + N * L * WEIGHT[w]
    c_bj = cost_bj_setup(N, L, w)
    use_bj = (k_cg - k_pcg) > c_bj / c_it + k_pcg * (p_it / c_it - 1.0)
    return (L if use_bj else 0), k_cg, k_pcg
