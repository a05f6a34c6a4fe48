"""Precision selection (eq. heuristic / heuristic_bj) and the kappa estimate from
CG step sizes, in the C library (host only, no GPU)."""
import json
import os

import numpy as np
import pytest

from oracle import analysis as AN
from oracle import detect as D
from paper_2504_09820_gb300 import fpcg as F


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_09820_gb300 import build as B
    B.build()
    F.lib()


def test_worked_example(golden_dir):
    """Section V-B.2: N = 32 users (K here), bound 1.33e-3 -> fp16."""
    g = json.load(open(os.path.join(golden_dir, "heuristic_example.json")))
    K = g["N"]
    kappa = (1.0 / (K ** 1.5 * g["u_mv_bound"])) ** 2
    name, u = F.fpcg_choose_precision(K, kappa)
    assert name == g["selected"] and u == pytest.approx(g["u_mv_bound"], rel=1e-12)


def test_agrees_with_oracle_grid():
    for K in (1, 4, 8, 16, 32, 64, 128):
        for kappa in np.geomspace(1.0, 1e12, 37):
            assert F.fpcg_choose_precision(K, kappa)[0] == AN.choose_precision(K, kappa), (K, kappa)


def test_invalid():
    for K, kappa in ((0, 10.0), (8, 0.5), (8, float("nan")), (8, float("inf"))):
        with pytest.raises(F.FpcgError):
            F.fpcg_choose_precision(K, kappa)
    with pytest.raises(F.FpcgError):
        F.fpcg_kappa_cg([1.0, -0.5], [0.1])
    with pytest.raises(F.FpcgError):
        F.fpcg_kappa_cg([], [])


def _cg_coefficients(A, b, m, M=None):
    """Step sizes of (preconditioned) CG in float64 (Algorithm 1 / PCG)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = r if M is None else M @ r
    p = z.copy()
    rz = np.vdot(r, z).real
    al, be = [], []
    for _ in range(m):
        w = A @ p
        a = rz / np.vdot(p, w).real
        x = x + a * p
        r = r - a * w
        z = r if M is None else M @ r
        rz_new = np.vdot(r, z).real
        al.append(a)
        be.append(rz_new / rz)
        p = z + be[-1] * p
        rz = rz_new
    return np.array(al), np.array(be[:-1])


def _hpd(K, kappa, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((K, K)) + 1j * rng.standard_normal((K, K)))
    ev = np.geomspace(1.0, kappa, K)
    return (Q * ev) @ Q.conj().T


def test_kappa_after_K_steps_is_exact():
    rng = np.random.default_rng(5)
    for K, kappa in ((4, 3.0), (8, 50.0), (16, 20.0)):
        A = _hpd(K, kappa, rng)
        b = rng.standard_normal(K) + 1j * rng.standard_normal(K)
        al, be = _cg_coefficients(A, b, K)
        assert F.fpcg_kappa_cg(al, be) == pytest.approx(kappa, rel=1e-6)
        prev = 1.0
        for m in range(1, K + 1):          # Ritz values interlace: the estimate grows to kappa
            k_m = F.fpcg_kappa_cg(al[:m], be[:m - 1])
            assert prev * (1 - 1e-12) <= k_m <= kappa * (1 + 1e-9)
            prev = k_m


def test_kappa_of_block_jacobi_preconditioned():
    """With M = M_d (block inverses), the estimate is kappa of M_d^(1/2) A M_d^(1/2)."""
    rng = np.random.default_rng(6)
    K, L = 16, 4
    A = _hpd(K, 200.0, rng)[None]
    Md, _ = D.bj_inverse(A, L, "fp64")
    M = np.zeros((K, K), complex)
    for i in range(K // L):
        M[i * L:(i + 1) * L, i * L:(i + 1) * L] = Md[0, i]
    b = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    al, be = _cg_coefficients(A[0], b, K, M)
    want = AN.kappa(AN.bj_preconditioned(A, Md))[0]
    assert F.fpcg_kappa_cg(al, be) == pytest.approx(want, rel=1e-6)
