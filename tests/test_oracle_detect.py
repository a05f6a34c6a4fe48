"""Pins for the detection oracle: Section II (Gram, LMMSE), Algorithms 1-3,
eq. pre_BJ, Theorems 2 and 5, and the refinement loop."""
import numpy as np
import pytest

from oracle import detect as D, qam, analysis as An
from oracle.formats import flc
from paper_2504_09820_gb300 import workload as wl


def _solve(A, b):
    return np.linalg.solve(A, b[..., None])[..., 0]


def _data(N=16, K=4, batch=8, rho=0.0, seed=7, snr=10.0, qamM=16, noiseless=False):
    return wl.generate(wl.Spec(N=N, K=K, batch=batch, rho=rho, qam=qamM, snr_db=snr,
                               seed=seed, noiseless=noiseless))


def test_gram_mf_brute_force():
    d = _data(N=5, K=3, batch=2)
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    for s in range(2):
        H = d["H"][s].T.astype(complex)          # N x K matrix
        y = d["y"][s].astype(complex)
        for k in range(3):
            bb = sum(H[n, k].conjugate() * y[n] for n in range(5))
            assert abs(b[s, k] - bb) < 1e-12
            for l in range(3):
                a = sum(H[n, k].conjugate() * H[n, l] for n in range(5))
                if k == l:
                    a += d["sigma2"][s]
                assert abs(A[s, k, l] - a) < 1e-12


def test_gram_hermitian_pd_and_reduced_modes():
    d = _data(N=64, K=16, batch=32, rho=0.5)
    for g in ("fp64", "fp32", "bf16", "fp16"):
        A, b = D.gram_emul(d["H"], d["y"], d["sigma2"], g)
        assert np.array_equal(A, np.conj(np.swapaxes(A, 1, 2)))
        np.linalg.cholesky(A)                    # positive definite
    A64, b64 = D.gram_mf(d["H"], d["y"], d["sigma2"])
    A, b = D.gram_emul(d["H"], d["y"], d["sigma2"], "fp64")
    assert np.array_equal(A, A64) and np.array_equal(b, b64)
    A16, _ = D.gram_emul(d["H"], d["y"], d["sigma2"], "bf16")
    rel = np.abs(A16 - A64).max() / np.abs(A64).max()
    assert 1e-5 < rel < 2e-2                      # bf16 inputs perturb the Gram


def _gauss_jordan_inverse(M):
    """Textbook Gauss-Jordan with partial pivoting, pure Python."""
    n = len(M)
    a = [[complex(M[i][j]) for j in range(n)] + [1.0 + 0j if i == j else 0j for j in range(n)] for i in range(n)]
    for c in range(n):
        piv = max(range(c, n), key=lambda r: abs(a[r][c]))
        a[c], a[piv] = a[piv], a[c]
        pv = a[c][c]
        a[c] = [v / pv for v in a[c]]
        for r in range(n):
            if r != c:
                f = a[r][c]
                a[r] = [a[r][j] - f * a[c][j] for j in range(2 * n)]
    return [row[n:] for row in a]


@pytest.mark.parametrize("K", [2, 3, 4])
def test_cholesky_lmmse_equals_explicit_inverse(K):
    d = _data(N=8, K=K, batch=3)
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    x = D.cholesky_solve(A, b)
    for s in range(3):
        inv = _gauss_jordan_inverse(A[s].tolist())
        xi = [sum(inv[i][j] * b[s, j] for j in range(K)) for i in range(K)]
        assert np.allclose(x[s], xi, rtol=1e-12, atol=1e-13)


def test_cg_finite_termination_c1():
    """Exact-arithmetic CG terminates in <= K steps; FP64 gets within 1e-10."""
    d = wl.generate(wl.c1_rayleigh_64x16(batch=64))
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    xs = D.cholesky_solve(A, b)
    x = D.cg(A, b, 16)
    assert np.max(np.linalg.norm(x - xs, axis=1) / np.linalg.norm(xs, axis=1)) < 1e-10


def test_cg_iterates_are_krylov_minimisers():
    """x_i minimises the A-norm error over span{b, Ab, ..., A^{i-1} b}."""
    d = _data(N=32, K=8, batch=4, rho=0.3)
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    for i in range(1, 5):
        x = D.cg(A, b, i)
        for s in range(4):
            V = np.stack([np.linalg.matrix_power(A[s], j) @ b[s] for j in range(i)], axis=1)
            c = np.linalg.solve(V.conj().T @ A[s] @ V, V.conj().T @ b[s])
            assert np.allclose(x[s], V @ c, rtol=1e-9, atol=1e-10)


def test_cg_distinct_eigenvalues():
    """CG on a matrix with 3 distinct eigenvalues is exact after 3 iterations."""
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6)))
    A = (Q * np.array([1.0, 1.0, 2.0, 2.0, 5.0, 5.0])) @ Q.conj().T
    A = 0.5 * (A + A.conj().T)
    b = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    x = D.cg(A[None], b[None], 3)[0]
    assert np.allclose(A @ x, b, atol=1e-12)


def test_fpcg_fp64_equals_algorithm1():
    d = _data(N=64, K=16, batch=16, rho=0.5)
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    x1 = D.cg(A, b, 10)
    x2, st, _, _ = D.fp_cg(A, b, 10, "fp64", "fp64", "fp64")
    assert np.allclose(x1, x2, rtol=1e-11, atol=1e-12)
    assert not st.any()


@pytest.mark.parametrize("alpha_num", [0, 1])
@pytest.mark.parametrize("L", [2, 4])
def test_bj_exact_on_block_diagonal(alpha_num, L):
    """Appendix D: A block diagonal with blocks of size L -> A_bar = I and
    FP-BJ-CG returns A^{-1} b after one iteration."""
    d = _data(N=32, K=8, batch=6, rho=0.6)
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    mask = np.kron(np.eye(8 // L), np.ones((L, L)))
    Ab = A * mask
    Md, fail = D.bj_inverse(Ab, L, "fp64")
    assert not fail.any()
    x, st, _, _ = D.fp_cg(Ab, b, 1, "fp64", "fp64", "fp64", Md, alpha_num)
    assert np.allclose(x, _solve(Ab, b), rtol=1e-11, atol=1e-12)
    kbar = An.kappa(An.bj_preconditioned(Ab, Md))
    assert np.allclose(kbar, 1.0, atol=1e-9)
    assert np.all(An.kappa(Ab) > 1.0)           # Theorem 5: kappa(A_bar) < kappa(A)


def test_bj_full_block_is_direct_solve():
    d = _data(N=32, K=8, batch=4, rho=0.8)
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    Md, _ = D.bj_inverse(A, 8, "fp64")
    x, _, _, _ = D.fp_cg(A, b, 1, "fp64", "fp64", "fp64", Md)
    assert np.allclose(x, _solve(A, b), rtol=1e-11, atol=1e-12)


def test_bj_reduces_condition_number_correlated():
    d = _data(N=256, K=32, batch=8, rho=0.8, snr=20.0)
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    Md, _ = D.bj_inverse(A, 8, "fp64")
    assert np.all(An.kappa(An.bj_preconditioned(A, Md)) < An.kappa(A))


@pytest.mark.parametrize("mv", ["bf16", "fp16"])
@pytest.mark.parametrize("rho", [0.0, 0.5, 0.8])
def test_theorem2_attainable_accuracy_bound(mv, rho):
    """||b - A x_i - r_i|| / (||A|| ||x||) <= (1+i) u_W + Upsilon_i Theta_i."""
    d = _data(N=64, K=8, batch=16, rho=rho, snr=20.0)
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    xs = _solve(A, b)
    Amv = D.round_matvec_operand(A, mv)
    _, _, _, tr = D.fp_cg(Amv, b, 8, mv, "fp64", "fp64", trace=True)
    nA = np.linalg.norm(A, 2, axis=(1, 2))
    nx = np.linalg.norm(xs, axis=1)
    from oracle.formats import FORMATS
    theta = np.zeros(16)
    for i, (xi, ri) in enumerate(zip(tr["x"], tr["r"])):
        theta = np.maximum(theta, np.linalg.norm(xi, axis=1) / nx)
        gap = np.linalg.norm(b - np.einsum("bkl,bl->bk", A, xi) - ri, axis=1) / (nA * nx)
        bound = An.theorem2_bound(i, 8, FORMATS["fp64"].u, FORMATS[mv].u, theta)
        assert np.all(gap <= bound)


def test_fpcg_mv_precision_dominates_ip_precision():
    """Remark 1: reduced-precision inner products barely move the attainable
    accuracy, a reduced-precision matvec does (Section V-B.1 trend)."""
    d = _data(N=256, K=32, batch=64, rho=0.5, snr=20.0)
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    xs = _solve(A, b)

    def err(mv, ip):
        x, _, _, _ = D.fp_cg(D.round_matvec_operand(A, mv), b, 30, mv, ip, "fp64")
        return np.median(np.linalg.norm(x - xs, axis=1) / np.linalg.norm(xs, axis=1))

    e_ip = err("fp64", "bf16")
    e_mv = err("bf16", "fp64")
    assert e_ip < e_mv


def test_noiseless_recovers_transmitted_symbols():
    d = _data(N=64, K=16, batch=32, noiseless=True)
    sig = np.full(32, 1e-8)
    r = D.detect(d["H"], d["y"], sig, 16, 16, {"gram": "fp64", "mv": "fp64", "ip": "fp64", "w": "fp64"})
    assert np.array_equal(r["sym"], d["tx"])
    x = D.lmmse(d["H"], d["y"], sig)
    assert np.array_equal(qam.slice_symbols(x, 16, "fp64"), d["tx"])


def test_refinement_with_exact_inner_solve():
    d = wl.generate(wl.c1_rayleigh_64x16(batch=32))
    A, b = D.gram_mf(d["H"], d["y"], d["sigma2"])
    xs = _solve(A, b)
    r = D.detect(d["H"], d["y"], d["sigma2"], 16, 2,
                 {"gram": "fp64", "mv": "fp64", "ip": "fp64", "w": "fp64",
                  "refine_steps": 1, "refine_iters": 16})
    assert np.max(np.linalg.norm(r["x"] - xs, axis=1) / np.linalg.norm(xs, axis=1)) < 1e-10


def test_refinement_recovers_reduced_precision_loss():
    """Each refinement pass brings x closer to the solution of the Gram system
    (the default residual is b - A x on the Gram matrix itself)."""
    d = wl.generate(wl.Spec(N=128, K=32, batch=64, rho=0.5, qam=64, snr_db=20.0, seed=5))
    A, b = D.gram_emul(d["H"], d["y"], d["sigma2"], "bf16")
    xs = _solve(A, b)
    e = []
    for rs in (0, 1, 2):
        r = D.detect(d["H"], d["y"], d["sigma2"], 64, 8, {"gram": "bf16", "mv": "bf16", "refine_steps": rs}, L=8)
        e.append(np.median(np.linalg.norm(r["x"] - xs, axis=1) / np.linalg.norm(xs, axis=1)))
    assert e[0] > 10 * e[1] > 100 * e[2]


def test_refinement_one_step_with_exact_inner_solve_is_exact():
    """Iterative refinement is Newton's method on the linear system: from a
    reduced-precision iterate x0, x0 + A^-1 r(x0) is the solution, to FP64
    accuracy, for the residual of the Gram system and for the residual formed
    from H and y without any Gram matrix (eq. inversion)."""
    d = wl.generate(wl.Spec(N=64, K=16, batch=16, rho=0.5, qam=16, snr_db=15.0, seed=21))
    Aq, bq = D.gram_emul(d["H"], d["y"], d["sigma2"], "bf16")
    x0, _, _, _ = D.fp_cg(D.round_matvec_operand(Aq, "bf16"), bq, 3, "bf16")
    xq = _solve(Aq, bq)
    assert np.median(np.linalg.norm(x0 - xq, axis=1) / np.linalg.norm(xq, axis=1)) > 1e-3
    x1 = x0 + D.cholesky_solve(Aq, D.resid(Aq, x0, bq))
    assert np.max(np.linalg.norm(x1 - xq, axis=1) / np.linalg.norm(xq, axis=1)) < 1e-13
    A64, b64 = D.gram_mf(d["H"], d["y"], d["sigma2"])
    xs = D.cholesky_solve(A64, b64)                        # the unrounded LMMSE solution
    x1h = x0 + D.cholesky_solve(A64, D.resid_h(d["H"], d["y"], d["sigma2"], x0))
    assert np.max(np.linalg.norm(x1h - xs, axis=1) / np.linalg.norm(xs, axis=1)) < 1e-13


@pytest.mark.parametrize("mode", ["gram", "mv", "h"])
def test_refinement_fixed_point_is_the_residual_systems_solution(mode):
    """Repeated refinement with a contracting reduced-precision inner solver
    converges to the solution of the system whose residual drives it: the Gram
    system (A, b) for "gram", the matvec matrix's system (A_mv, b) for "mv",
    the unrounded LMMSE system for "h" -- and not to the other two."""
    d = wl.generate(wl.Spec(N=64, K=16, batch=32, rho=0.3, qam=16, snr_db=20.0, seed=9))
    pk = {"gram": "bf16", "mv": "fp16", "refine_steps": 6, "refine_iters": 8, "resid": mode}
    r = D.detect(d["H"], d["y"], d["sigma2"], 16, 8, pk, L=4)
    Aq, bq = D.gram_emul(d["H"], d["y"], d["sigma2"], "bf16")
    A64, b64 = D.gram_mf(d["H"], d["y"], d["sigma2"])
    sols = {"gram": _solve(Aq, bq), "mv": _solve(D.round_matvec_operand(Aq, "fp16"), bq), "h": _solve(A64, b64)}
    err = {k: np.median(np.linalg.norm(r["x"] - v, axis=1) / np.linalg.norm(v, axis=1)) for k, v in sols.items()}
    assert err[mode] < 2e-6, err                           # fp32 working precision
    for other in sols:
        if other != mode:
            assert err[other] > 20 * err[mode], err
    # rel_res is the residual of that system at the returned x
    if mode == "h":
        want = np.linalg.norm(D.resid_h(d["H"], d["y"], d["sigma2"], r["x"]), axis=1) / np.linalg.norm(b64, axis=1)
    else:
        Ar = Aq if mode == "gram" else D.round_matvec_operand(Aq, "fp16")
        want = np.linalg.norm(D.resid(Ar, r["x"], bq), axis=1) / np.linalg.norm(bq, axis=1)
    assert np.allclose(r["rel_res"], want, rtol=1e-12, atol=0)


def test_zero_rhs_and_zero_iterations():
    d = _data(N=16, K=4, batch=3)
    y0 = np.zeros_like(d["y"])
    r = D.detect(d["H"], y0, d["sigma2"], 16, 5, {})
    assert np.all(r["x"] == 0) and np.all(r["status"] & D.ST_RHO_ZERO) and np.all(r["rel_res"] == 0)
    r = D.detect(d["H"], d["y"], d["sigma2"], 16, 0, {})
    assert np.all(r["x"] == 0) and np.allclose(r["rel_res"], 1.0)


def test_breakdown_flag_on_indefinite_matrix():
    A = np.array([[[1.0, 0.0], [0.0, -1.0]]], dtype=complex)
    b = np.array([[1.0, 1.0]], dtype=complex)
    x, st, _, _ = D.fp_cg(A, b, 3, "fp64", "fp64", "fp64")
    assert st[0] & D.ST_BREAKDOWN


def test_fp32_cg_c1_reaches_working_accuracy():
    d = wl.generate(wl.c1_rayleigh_64x16(batch=128))
    r = D.detect(d["H"], d["y"], d["sigma2"], 16, 16, {"gram": "fp32", "mv": "fp32"})
    assert np.max(r["rel_res"]) < 1e-5
    x = D.lmmse(d["H"], d["y"], d["sigma2"])
    ref = qam.bit_errors(qam.slice_symbols(x, 16, "fp64"), d["tx"])
    assert abs(qam.bit_errors(r["sym"], d["tx"]) - ref) <= 2
