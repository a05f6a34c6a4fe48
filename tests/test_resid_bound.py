"""The error bound that the GPU tests hold the given-Gram solvers' fp32
residual to (gpu_helpers.gram_resid_rel).  b - A x is formed here in the
operation order of those solvers -- per lane 2E fused multiply-adds over its
columns j = lane + 32e, a pairwise tree over the 32 lanes (distance 16, 8, 4,
2, 1), one subtraction from b -- with every operation rounded to fp32
(numpy float32; a fused multiply-add is the float64 result rounded once), and
compared with the same residual in float64.  The systems are Gram systems
near their solution, where b - A x is small against |A||x|: the rounding error
is about 1% of the residual there, and the worst-case bound is about ten times
the largest error seen."""
import numpy as np
import pytest

from gpu_helpers import gram_resid_rel

F32 = np.float32


def _fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def fp32_residual(A, x, b):
    """b - A x in the solvers' fp32 order; A (B, KR, KR), x, b (B, KR) complex64."""
    B, KR, _ = A.shape
    K = max(16, KR)
    E = max(1, K // 32)
    ar, ai = A.real.astype(F32), A.imag.astype(F32)
    xr, xi = x.real.astype(F32), x.imag.astype(F32)
    re = np.zeros((B, KR, 32), F32)
    im = np.zeros((B, KR, 32), F32)
    for e in range(E):
        lanes = np.arange(32)
        j = lanes + 32 * e
        ok = j < KR
        lo, jj = lanes[ok], j[ok]
        a_r, a_i = ar[:, :, jj], ai[:, :, jj]            # (B, KR rows, lanes)
        v_r, v_i = xr[:, None, jj], xi[:, None, jj]
        re[:, :, lo] = _fma(a_r, v_r, _fma(-a_i, v_i, re[:, :, lo]))
        im[:, :, lo] = _fma(a_r, v_i, _fma(a_i, v_r, im[:, :, lo]))
    lanes = np.arange(32)
    for o in (16, 8, 4, 2, 1):
        re = (re + re[:, :, lanes ^ o]).astype(F32)
        im = (im + im[:, :, lanes ^ o]).astype(F32)
    wr = (b.real.astype(F32) - re[:, :, 0]).astype(F32)
    wi = (b.imag.astype(F32) - im[:, :, 0]).astype(F32)
    return wr.astype(np.float64) + 1j * wi.astype(np.float64)


def _gram_system(K, B, seed, kappa_spread=1.0):
    rng = np.random.default_rng(seed)
    N = 4 * K
    H = (rng.standard_normal((B, N, K)) + 1j * rng.standard_normal((B, N, K))) / np.sqrt(2 * N)
    H[:, :, 0] *= kappa_spread                                   # one strong user: larger |A||x|
    A = (np.conj(np.swapaxes(H, 1, 2)) @ H + 0.05 * np.eye(K)).astype(np.complex64)
    x_true = (rng.choice([-3, -1, 1, 3], (B, K)) + 1j * rng.choice([-3, -1, 1, 3], (B, K))) / np.sqrt(10)
    b = np.einsum("bkl,bl->bk", A.astype(np.complex128), x_true).astype(np.complex64)
    # x close to the solution of the fp32 system (the regime of a refined solve)
    x = np.linalg.solve(A.astype(np.complex128), b.astype(np.complex128)[..., None])[..., 0]
    x = (x + 1e-5 * rng.standard_normal(x.shape)).astype(np.complex64)
    return A, x, b


@pytest.mark.parametrize("K", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("spread", [1.0, 30.0])
def test_fp32_residual_within_the_bound(K, spread):
    A, x, b = _gram_system(K, 64, 10 + K, spread)
    w = fp32_residual(A, x, b)
    exact = b.astype(np.complex128) - np.einsum("bkl,bl->bk", A.astype(np.complex128), x.astype(np.complex128))
    nb = np.linalg.norm(b.astype(np.complex128), axis=1)
    err = np.linalg.norm(w - exact, axis=1) / nb
    own, bound = gram_resid_rel(A, b, x)
    assert np.allclose(own, np.linalg.norm(exact, axis=1) / nb, rtol=1e-12)
    assert np.all(err <= bound), np.max(err / bound)
    # the bound is not vacuous here: the rounding error is a visible part of the residual
    assert np.median(err / own) > 1e-3


def test_bound_fails_for_a_coarser_residual():
    """A residual whose products are rounded to bf16 first (the matvec copy of
    A at u_MV = bf16) is far outside the bound: the bound tells the two apart."""
    A, x, b = _gram_system(64, 32, 3)
    Ab = A.real.astype(F32).view(np.uint32)
    Ab = ((Ab + 0x7FFF + ((Ab >> 16) & 1)) & 0xFFFF0000).view(F32)   # round to bf16, ties to even
    Ai = A.imag.astype(F32).view(np.uint32)
    Ai = ((Ai + 0x7FFF + ((Ai >> 16) & 1)) & 0xFFFF0000).view(F32)
    w = fp32_residual((Ab + 1j * Ai).astype(np.complex64), x, b)
    exact = b.astype(np.complex128) - np.einsum("bkl,bl->bk", A.astype(np.complex128), x.astype(np.complex128))
    nb = np.linalg.norm(b.astype(np.complex128), axis=1)
    err = np.linalg.norm(w - exact, axis=1) / nb
    _, bound = gram_resid_rel(A, b, x)
    assert np.all(err > 3 * bound)
