"""Detection on the input models of Section V-C and IV-B against the oracle:
imperfect channel estimates, a Gauss-Markov channel one step later (also with
the Gram matrix of the previous step kept, as a serving loop would keep it),
multi-antenna users (Assumption 1's block R_t), and the LMMSE reference of the
experiment runner against the oracle's Cholesky solve.  Bars as everywhere:
the reduced-precision bar of gpu_helpers.check_reduced_parity, fp64 x_hat
within 1e-10, and BER of the benchmark's schedule within 5% of the oracle's
direct LMMSE solve."""
import numpy as np
import pytest
import torch

from oracle import detect as D
from oracle import qam as Q
from paper_2504_09820_gb300 import fpcg as F
from paper_2504_09820_gb300 import workload as wl

from gpu_helpers import check_reduced_parity, gpu_detect, oracle_detect, rel_err

pytestmark = pytest.mark.gpu

HEAD_LIKE = dict(gram="bf16", mv="fp16", refine_steps=1, resid="fp64")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()


def _ber_vs_lmmse(d, sym, M):
    """Bit errors of the GPU's labels and of the oracle's Cholesky LMMSE on
    the channel the detector was given."""
    x = D.lmmse(d["H"], d["y"], d["sigma2"])
    return Q.bit_errors(sym, d["tx"]), Q.bit_errors(Q.slice_symbols(x, M, "fp64"), d["tx"])


@pytest.mark.parametrize("eps_db", [15.0, 25.0])
def test_imperfect_csi(eps_db):
    """The detector sees H + dH (channel-to-error ratio eps, Section V-C); y
    was made with H.  GPU and oracle detect from the same estimate."""
    d = wl.generate(wl.Spec(N=256, K=64, batch=400, rho=0.5, qam=64, snr_db=18.0, seed=801))
    d = dict(d, H=wl.csi_error(d["H"], eps_db, seed=9))
    res = gpu_detect(d, 7, HEAD_LIKE, L=4)
    ref = oracle_detect(d, 7, HEAD_LIKE, L=4)
    check_reduced_parity(d, res["x"], ref["x"], 7, HEAD_LIKE, L=4)
    e_gpu, e_ref = _ber_vs_lmmse(d, res["sym"], 64)
    assert abs(e_gpu / e_ref - 1) < 0.05, (e_gpu, e_ref)


def test_gauss_markov_step_and_kept_gram():
    """One step of the first-order Gauss-Markov channel (Section V-C): the
    aged channel's detection against the oracle, and detection of the new
    received vectors against the previous step's Gram matrix, kept on the
    device (fpcg_gram once, fpcg_detect_grouped for the next step's vectors)
    against the oracle given the same stale channel."""
    spec = wl.Spec(N=128, K=32, batch=240, rho=0.5, qam=16, snr_db=15.0, seed=802)
    rho_tau = wl.doppler_corr(100.0, 0.5e-3)
    h0, h1 = wl.gauss_markov(spec, 2, rho_tau)
    pk = dict(HEAD_LIKE)
    res = gpu_detect(h1, 7, pk, L=4)
    ref = oracle_detect(h1, 7, pk, L=4)
    check_reduced_parity(h1, res["x"], ref["x"], 7, pk, L=4)
    # the Gram of step 0 kept: one group per system, that system's step-1 vector
    B, K, N = h0["H"].shape
    dev = "cuda:0"
    H0 = torch.from_numpy(h0["H"]).to(dev)
    A = torch.empty((B, K, K), dtype=torch.complex64, device=dev)
    b = torch.empty((B, K), dtype=torch.complex64, device=dev)
    F.fpcg_gram(H0, torch.from_numpy(h0["y"]).to(dev), torch.from_numpy(h0["sigma2"]).to(dev), "bf16", A, b)
    x = torch.empty((B, K), dtype=torch.complex64, device=dev)
    sym = torch.empty((B, K), dtype=torch.uint8, device=dev)
    gs = torch.arange(B + 1, dtype=torch.int64, device=dev)
    pk_tc = dict(pk)   # the grouped solver's residual against the kept Gram matrix
    F.fpcg_detect_grouped(A, H0, torch.from_numpy(h1["y"]).to(dev), gs, torch.from_numpy(h1["qam"]).to(dev),
                          7, 4, F.precision(**pk_tc), x, sym_idx=sym)
    torch.cuda.synchronize()
    stale = dict(h1, H=h0["H"], sigma2=h0["sigma2"])        # the oracle sees the kept channel
    ref_s = oracle_detect(stale, 7, pk_tc, L=4)
    check_reduced_parity(stale, x.cpu().numpy(), ref_s["x"], 7, pk_tc, L=4)
    # the stale Gram costs BER (it is a different channel), the fresh one does not
    e_fresh = Q.bit_errors(res["sym"], h1["tx"])
    e_stale = Q.bit_errors(sym.cpu().numpy(), h1["tx"])
    assert e_stale >= e_fresh


@pytest.mark.parametrize("L", [4, 8])
def test_multi_antenna_users(L):
    """N_UE = 4 antennas per user, Assumption 1's block R_t (no correlation
    between users, exponential within a user); block-Jacobi blocks aligned
    with the users (L = 4) or two users (L = 8), as in Section V-A."""
    spec = wl.Spec(N=256, K=32, batch=384, rho=0.8, qam=16, snr_db=20.0, seed=803, n_ue=4, rt_block=True)
    d = wl.generate(spec)
    pk = dict(HEAD_LIKE)
    res = gpu_detect(d, 6, pk, L=L)
    ref = oracle_detect(d, 6, pk, L=L)
    check_reduced_parity(d, res["x"], ref["x"], 6, pk, L=L)
    e_gpu, e_ref = _ber_vs_lmmse(d, res["sym"], 16)
    assert abs(e_gpu / max(e_ref, 1) - 1) < 0.05 or abs(e_gpu - e_ref) <= 3, (e_gpu, e_ref)


def test_experiment_lmmse_reference_is_the_oracles():
    """The experiment runner's LMMSE (fp64 CG for 2K iterations on the GPU)
    on channels drawn on the device: x_hat within 1e-10 of the oracle's
    Cholesky solve, labels equal outside a counted margin; and its reduced
    variants within the reduced-precision bar of the oracle's emulation."""
    from paper_2504_09820_gb300 import experiments as X
    spec = X._spec(0.8, seed=7)
    g = wl.generate_torch(spec, 0, 256)
    d = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in g.items()}
    r = F.detect(g["H"], g["y"], g["sigma2"], g["qam"], 2 * X.K_STREAMS, X.prec_of("lmmse"), tx_idx=g["tx"])
    torch.cuda.synchronize()
    x_gpu = r["x"].cpu().numpy()
    x_ref = D.lmmse(d["H"], d["y"], d["sigma2"])
    assert rel_err(x_gpu, x_ref).max() < 1e-10
    from gpu_helpers import near_threshold
    mask = near_threshold(x_ref, X.QAM, "fp64", 1e-8)
    assert mask.sum() <= 2
    assert np.array_equal(r["sym"].cpu().numpy()[~mask], Q.slice_symbols(x_ref, X.QAM, "fp64")[~mask])
    pk = dict(gram="fp32", mv="fp16", ip="fp32", w="fp32")
    res = gpu_detect(d, 6, pk, L=X.L_BJ)
    ref = oracle_detect(d, 6, pk, L=X.L_BJ)
    check_reduced_parity(d, res["x"], ref["x"], 6, pk, L=X.L_BJ)
