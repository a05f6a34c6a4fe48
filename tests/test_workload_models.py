"""Input models beyond the i.i.d./Kronecker channel (Section IV-B, Section
V-C): multi-antenna users with Assumption 1's block R_t, imperfect CSI, the
first-order Gauss-Markov channel, and the GPU-side generator (run here on the
CPU).  Pinned by their defining statistics, not by the generators' own code."""
import math

import numpy as np
import pytest
import torch

from oracle import analysis as An
from paper_2504_09820_gb300 import workload as wl


def _gram_mean(H):
    H = np.asarray(H, dtype=np.complex128)
    return (np.conj(H) @ np.swapaxes(H, 1, 2)).mean(axis=0)


def test_block_rt_has_no_inter_user_correlation():
    """Assumption 1: E[H^H H] = R_t (Appendix B) with zero blocks between users
    and the exponential matrix inside each user's n_ue antennas."""
    M, K, n_ue, zeta, n = 32, 8, 4, 0.6, 4096
    d = wl.generate(wl.Spec(N=M, K=K, batch=n, rho=zeta, qam=4, snr_db=10.0, seed=21, n_ue=n_ue, rt_block=True))
    mean = _gram_mean(d["H"])
    want = np.zeros((K, K))
    i = np.arange(n_ue)
    for u in range(K // n_ue):
        want[u * n_ue:(u + 1) * n_ue, u * n_ue:(u + 1) * n_ue] = zeta ** np.abs(i[:, None] - i[None, :])
    assert np.abs(mean - want).max() < 5 * np.sqrt(An.gram_var_closed(M, zeta) / n) + 1e-3
    # the full exponential model keeps the inter-user terms
    full = _gram_mean(wl.generate(wl.Spec(N=M, K=K, batch=n, rho=zeta, qam=4, snr_db=10.0, seed=21))["H"])
    assert full[0, n_ue].real == pytest.approx(zeta ** n_ue, abs=0.05)


def test_block_rt_rejects_partial_users():
    with pytest.raises(ValueError):
        wl.Spec(N=32, K=6, batch=1, n_ue=4, rt_block=True)


@pytest.mark.parametrize("eps_db", [20.0, 25.0])
def test_csi_error_power_ratio(eps_db):
    """Channel-to-error power ratio of H_hat = H + dH is eps (entrywise)."""
    d = wl.generate(wl.Spec(N=64, K=8, batch=2000, rho=0.8, qam=16, snr_db=20.0, seed=5))
    Hh = wl.csi_error(d["H"], eps_db, seed=9)
    dH = Hh.astype(np.complex128) - d["H"]
    ratio = np.mean(np.abs(d["H"]) ** 2) / np.mean(np.abs(dH) ** 2)
    assert 10 * np.log10(ratio) == pytest.approx(eps_db, abs=0.05)
    # zero-mean, circular, and independent of H
    assert abs(np.mean(dH)) < 5 * np.sqrt(np.mean(np.abs(dH) ** 2) / dH.size)
    assert abs(np.mean(dH.real * dH.imag)) < 5 * np.mean(np.abs(dH) ** 2) / np.sqrt(dH.size)
    c = np.mean(np.conj(d["H"]) * dH) / np.sqrt(np.mean(np.abs(d["H"]) ** 2) * np.mean(np.abs(dH) ** 2))
    assert abs(c) < 5 / np.sqrt(dH.size)


def _j0_series(x):
    return sum((-1) ** m * (x / 2) ** (2 * m) / math.factorial(m) ** 2 for m in range(40))


def test_doppler_corr_is_bessel_j0():
    assert wl.doppler_corr(0.0, 1e-3) == 1.0
    for fd, tau in ((1000.0, 1e-4), (1000.0, 5e-4), (300.0, 1e-3)):
        assert wl.doppler_corr(fd, tau) == pytest.approx(_j0_series(2 * math.pi * fd * tau), abs=1e-12)
    first_zero = 2.404825557695773  # first root of J0
    assert abs(wl.doppler_corr(first_zero / (2 * math.pi), 1.0)) < 1e-12


def test_gauss_markov_step_correlation_and_stationarity():
    """H_i = a H_{i-1} + sqrt(1-a^2) W_i: one-step correlation a, and the
    spatial statistics E[H^H H] = R_t at every step."""
    a, n = 0.9, 3000
    spec = wl.Spec(N=16, K=4, batch=n, rho=0.5, qam=16, snr_db=15.0, seed=8)
    seq = wl.gauss_markov(spec, 3, a)
    H0, H1, H2 = (np.asarray(s["H"], dtype=np.complex128) for s in seq)
    p = np.mean(np.abs(H0) ** 2)
    assert np.mean(np.conj(H0) * H1).real / p == pytest.approx(a, abs=0.02)
    assert np.mean(np.conj(H0) * H2).real / p == pytest.approx(a * a, abs=0.02)
    Rt = wl.exp_corr(4, 0.5)
    for H in (H1, H2):
        assert np.abs(_gram_mean(H) - Rt).max() < 5 * np.sqrt(An.gram_var_closed(16, 0.5) / n) + 1e-3


def test_gauss_markov_received_vectors_use_the_aged_channel():
    spec = wl.Spec(N=16, K=4, batch=20, rho=0.3, qam=16, snr_db=15.0, seed=2, noiseless=True)
    for s in wl.gauss_markov(spec, 3, 0.7):
        y = np.einsum("bkn,bk->bn", np.asarray(s["H"], dtype=np.complex128), s["x"])
        assert np.abs(y - s["y"]).max() < 1e-5


def test_generate_torch_distributions():
    """The device generator (run on the CPU here): E[H^H H] = R_t, symbols are
    the Gray QAM points of their labels, noise variance sigma^2."""
    spec = wl.Spec(N=32, K=4, batch=0, rho=0.6, qam=64, snr_db=12.0, seed=4)
    d = wl.generate_torch(spec, 0, 4096, device="cpu")
    H = d["H"].numpy()
    assert H.shape == (4096, 4, 32) and H.dtype == np.complex64
    mean = _gram_mean(H)
    assert np.abs(mean - wl.exp_corr(4, 0.6)).max() < 5 * np.sqrt(An.gram_var_closed(32, 0.6) / 4096) + 1e-3
    assert np.abs(d["x"].numpy() - wl.qam_modulate(d["tx"].numpy(), 64)).max() < 1e-12
    n = d["y"].numpy().astype(np.complex128) - np.einsum("bkn,bk->bn", H.astype(np.complex128), d["x"].numpy())
    assert np.mean(np.abs(n) ** 2) == pytest.approx(10 ** -1.2, rel=0.03)
    # reproducible per (seed, chunk), different across chunks
    a = wl.generate_torch(spec, 3, 16, device="cpu")["H"]
    b = wl.generate_torch(spec, 3, 16, device="cpu")["H"]
    c = wl.generate_torch(spec, 4, 16, device="cpu")["H"]
    assert torch.equal(a, b) and not torch.equal(a, c)
