"""Exact-rational pins of where the oracle rounds (Definition 1's fl(.) at the
precision of each role of Algorithms 2 and 3, and of the reduced-precision
Gram step).

A tiny case (K = 2, N = 3) is recomputed here in exact rational arithmetic
(fractions.Fraction) with a rounding function written in this file, so
nothing of the oracle's own format code is reused.  Every role gets a
different precision (u_MV = bf16, u_IP = fp16, u_W = fp32), so a rounding put
at the wrong step, or at the wrong precision, changes the result; each such
misplacement is planted in the rational reference and shown to change it.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import detect as D

BITS = {"bf16": 8, "fp16": 11, "fp32": 24}


def rnd(q, p):
    """q rounded to p significant bits, to nearest, ties to even (normal
    range only: the fixtures below stay far from under- and overflow)."""
    q = Fr(q)
    if q == 0:
        return Fr(0)
    s = 1 if q > 0 else -1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fr(2) ** e > a:
        e -= 1
    while Fr(2) ** (e + 1) <= a:
        e += 1
    ulp = Fr(2) ** (e - p + 1)
    n = a / ulp
    f = n.numerator // n.denominator
    rem = n - f
    if rem > Fr(1, 2) or (rem == Fr(1, 2) and f % 2 == 1):
        f += 1
    return s * f * ulp


def rc(z, p):
    return (rnd(z[0], p), rnd(z[1], p))


def cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def cadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def conj(a):
    return (a[0], -a[1])


def redot(u, v):
    """Re sum conj(u_i) v_i, exactly."""
    return sum(ui[0] * vi[0] + ui[1] * vi[1] for ui, vi in zip(u, v))


def fr(z):
    return (Fr(float(z.real)), Fr(float(z.imag)))


def to_np(v):
    return np.array([float(a) + 1j * float(b) for a, b in v])


# ---------------------------------------------------------------------------
# Algorithm 2 (Md None) / Algorithm 3 (Md = inverted 1 x 1 diagonal blocks),
# x0 = 0, in the paper's step order; `mut` plants one misplaced rounding.
# ---------------------------------------------------------------------------

MUTATIONS = [
    "p_not_rounded_for_matvec",   # A p with p at u_W instead of u_MV
    "matvec_not_rounded",         # varpi = A p kept exact instead of one fp32 rounding
    "phi_with_rounded_p",         # phi = p_q^H varpi instead of p^H varpi
    "alpha_at_u_ip",              # alpha rounded at u_IP instead of u_W
    "x_update_with_rounded_p",    # x += alpha p_q instead of alpha p
    "rho_at_u_w",                 # inner products rounded at u_W instead of u_IP
    "beta_at_u_ip",               # beta rounded at u_IP instead of u_W
    "p_update_at_u_mv",           # next p rounded at u_MV instead of u_W
]


def cg_rational(A_mv, b, iters, mv, ip, w, Md=None, mut=None):
    pm, pi, pw, pa = BITS[mv], BITS[ip], BITS[w], BITS["fp32"]
    K = len(b)
    x = [(Fr(0), Fr(0))] * K
    r = [rc(v, pw) for v in b]

    def zof(rv):
        return list(rv) if Md is None else [rc(cmul(Md[i], rv[i]), pw) for i in range(K)]

    pip = pw if mut == "rho_at_u_w" else pi
    z = zof(r)
    p = list(z)
    rho = rnd(redot(r, z), pip)
    for _ in range(iters):
        pq = list(p) if mut == "p_not_rounded_for_matvec" else [rc(v, pm) for v in p]
        varpi = []
        for i in range(K):
            s = (Fr(0), Fr(0))
            for j in range(K):
                s = cadd(s, cmul(A_mv[i][j], pq[j]))
            varpi.append(s if mut == "matvec_not_rounded" else rc(s, pa))
        phi = rnd(redot(pq if mut == "phi_with_rounded_p" else p, varpi), pi)
        rho_prev = rnd(redot(r, p), pip) if Md is not None else rho   # Algorithm 3: r^H p
        alpha = rnd(rho_prev / phi, pi if mut == "alpha_at_u_ip" else pw)
        xs = pq if mut == "x_update_with_rounded_p" else p
        x = [rc(cadd(x[i], (alpha * xs[i][0], alpha * xs[i][1])), pw) for i in range(K)]
        r = [rc(cadd(r[i], (-alpha * varpi[i][0], -alpha * varpi[i][1])), pw) for i in range(K)]
        z = zof(r)
        rho_n = rnd(redot(r, z), pip)
        beta = rnd(rho_n / rho_prev, pi if mut == "beta_at_u_ip" else pw)
        pp = pm if mut == "p_update_at_u_mv" else pw
        p = [rc(cadd(z[i], (beta * p[i][0], beta * p[i][1])), pp) for i in range(K)]
        rho = rho_n
    return x


def _system(seed):
    """A Hermitian positive definite 2 x 2 with fp32 entries and an fp32 b."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((2, 3)) + 1j * rng.standard_normal((2, 3))
    A = (G.conj() @ G.T + 0.3 * np.eye(2)).astype(np.complex64).astype(np.complex128)
    A = 0.5 * (A + A.conj().T)
    A[0, 0], A[1, 1] = A[0, 0].real, A[1, 1].real
    A = A.astype(np.complex64).astype(np.complex128)
    b = (rng.standard_normal(2) + 1j * rng.standard_normal(2)).astype(np.complex64).astype(np.complex128)
    return A, b


# seeds checked to make every planted mutation visible in x after 2 iterations
@pytest.mark.parametrize("bj,seed", [(False, 136), (True, 35)])
def test_fp_cg_rounding_placement_exact(bj, seed):
    A, b = _system(seed)
    mv, ip, w = "bf16", "fp16", "fp32"
    Af = [[fr(A[i, j]) for j in range(2)] for i in range(2)]
    A_mv = [[rc(Af[i][j], BITS[mv]) for j in range(2)] for i in range(2)]
    bf = [fr(v) for v in b]
    Md = Md_np = None
    if bj:  # L = 1: M_d = diag(fl_w(1 / A_ii))
        Md_np, fail = D.bj_inverse(A[None], 1, w)
        assert not fail.any()
        Md = [(rnd(1 / Af[i][i][0], BITS[w]), Fr(0)) for i in range(2)]
        assert [float(m[0]) for m in Md] == [Md_np[0, i, 0, 0].real for i in range(2)]
    want = cg_rational(A_mv, bf, 2, mv, ip, w, Md)
    x, st, _, _ = D.fp_cg(to_np_matrix(A_mv)[None], b[None], 2, mv, ip, w, Md_np)
    assert not st.any()
    assert np.array_equal(x[0], to_np(want))            # bit for bit
    for m in MUTATIONS:
        assert cg_rational(A_mv, bf, 2, mv, ip, w, Md, mut=m) != want, m


def to_np_matrix(M):
    return np.array([[float(a) + 1j * float(b) for a, b in row] for row in M])


def test_rational_rounding_matches_ieee_casts():
    """The rounding function of this file agrees with numpy's fp16 and fp32
    casts (so the fixture above pins the oracle, not two shared mistakes)."""
    rng = np.random.default_rng(3)
    for v in rng.standard_normal(200) * 10.0 ** rng.integers(-3, 3, 200):
        assert float(rnd(Fr(float(v)), 24)) == float(np.float32(v))
        assert float(rnd(Fr(float(v)), 11)) == float(np.float16(v))


# ---------------------------------------------------------------------------
# The reduced-precision Gram step: A = fl32(fl_g(H)^H fl_g(H)) + fl32(sigma^2)
# (one more rounding on the diagonal), b = fl32(fl_g(H)^H fl_g(y)).
# ---------------------------------------------------------------------------

GRAM_MUTATIONS = ["y_not_rounded", "h_not_rounded", "sigma2_at_u_gram", "diag_rounded_once"]


def gram_rational(H, y, s2, g, mut=None):
    """H: N x K list of complex Fractions (column k = user k), y: N."""
    N, K = len(H), len(H[0])
    pg = BITS[g]
    Hq = [[H[n][k] if mut == "h_not_rounded" else rc(H[n][k], pg) for k in range(K)] for n in range(N)]
    yq = [y[n] if mut == "y_not_rounded" else rc(y[n], pg) for n in range(N)]
    s2q = rnd(s2, pg if mut == "sigma2_at_u_gram" else 24)
    A = [[None] * K for _ in range(K)]
    for k in range(K):
        for l in range(K):
            s = (Fr(0), Fr(0))
            for n in range(N):
                s = cadd(s, cmul(conj(Hq[n][k]), Hq[n][l]))
            if k == l:
                A[k][l] = rc((s[0] + Fr(s2), s[1]), 24) if mut == "diag_rounded_once" else \
                    rc(cadd(rc(s, 24), (s2q, Fr(0))), 24)
            else:
                A[k][l] = rc(s, 24)
    bv = []
    for k in range(K):
        s = (Fr(0), Fr(0))
        for n in range(N):
            s = cadd(s, cmul(conj(Hq[n][k]), yq[n]))
        bv.append(rc(s, 24))
    return A, bv


@pytest.mark.parametrize("g", ["bf16", "fp16"])
def test_gram_emul_rounding_exact(g):
    rng = np.random.default_rng(0)   # checked to make every planted mutation visible
    N, K = 3, 2
    H = (rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))).astype(np.complex64)
    y = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(np.complex64)
    s2 = 0.1234567891234  # not representable in any of the formats
    Hf = [[fr(H[n, k]) for k in range(K)] for n in range(N)]
    yf = [fr(v) for v in y]
    A_want, b_want = gram_rational(Hf, yf, s2, g)
    # oracle input layout: H_arr[s, k, n] = H[n, k]
    A, b = D.gram_emul(H.T[None].astype(np.complex128), y[None].astype(np.complex128), np.array([s2]), g)
    assert np.array_equal(A[0], to_np_matrix(A_want))
    assert np.array_equal(b[0], to_np(b_want))
    for m in GRAM_MUTATIONS:
        Am, bm = gram_rational(Hf, yf, s2, g, mut=m)
        assert (Am, bm) != (A_want, b_want), m
