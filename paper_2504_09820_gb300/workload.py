"""Seeded synthetic MIMO detection workloads.

This module is the ONE piece shared by the CUDA path's tests/bench and the CPU
oracle: it draws inputs and holds none of the detector's arithmetic (no Gram
matrix, no solver, no slicer).  Both sides consume the identical complex64
arrays it returns.

Channel model (Section II, eq. channel_model): H = R_r^{1/2} Omega R_t^{1/2}
with Omega i.i.d. CN(0, 1/N) and exponential correlation r_ij = rho^|i-j|
(real rho, so R is real symmetric Toeplitz); the square roots are the
principal ones (symmetric, as Appendix B uses).  rho = 0 is i.i.d. Rayleigh.
The paper's (M, N) are (N, K) here: N receive antennas, K single-antenna users.

Symbols: square Gray-mapped M-QAM with unit average energy, labels drawn
uniformly.  Noise: CN(0, sigma^2) with sigma^2 = 10^(-SNR/10) (per-stream SNR
with E||h_k||^2 = 1; the paper does not state its convention).

Storage layout (what the C ABI takes): H of one system is column-major with
leading dimension N, complex64 interleaved, i.e. a numpy array of shape
(batch, K, N) with H_arr[s, k, n] = H_s[n, k]; y is (batch, N) complex64.

Randomness: numpy PCG64 streams seeded by SeedSequence([seed, chunk]) for
chunks of CHUNK systems, so a chunk can be regenerated on its own.
"""

from dataclasses import dataclass, field

import numpy as np

CHUNK = 256


def exp_corr(n, rho):
    """Exponential correlation matrix r_ij = rho^|i-j| (eq. 2 with real rho)."""
    i = np.arange(n)
    return float(rho) ** np.abs(i[:, None] - i[None, :])


def sqrt_psd(R):
    """Principal square root of a real symmetric positive semidefinite matrix."""
    w, V = np.linalg.eigh(R)
    return (V * np.sqrt(np.clip(w, 0.0, None))) @ V.T


def gray_decode(g):
    """Inverse of the binary-reflected Gray code, elementwise on integers."""
    j = np.asarray(g, dtype=np.int64).copy()
    shift = 1
    while shift < 16:
        j ^= j >> shift
        shift <<= 1
    return j


def qam_modulate(labels, M):
    """Gray labels (high bits: in-phase, low bits: quadrature) -> unit-energy symbols."""
    m = int(round(np.sqrt(M)))
    b = int(np.log2(m))
    labels = np.asarray(labels, dtype=np.int64)
    ji = gray_decode(labels >> b)
    jq = gray_decode(labels & (m - 1))
    d = 1.0 / np.sqrt(2.0 * (M - 1) / 3.0)
    return ((2 * ji - (m - 1)) + 1j * (2 * jq - (m - 1))) * d


def snr_to_sigma2(snr_db):
    return 10.0 ** (-np.asarray(snr_db, dtype=np.float64) / 10.0)


@dataclass
class Spec:
    """A uniform batch: every system has the same (N, K, rho, QAM order, SNR)."""
    N: int
    K: int
    batch: int
    rho: float = 0.0          # same exponential correlation at both ends
    qam: int = 16
    snr_db: float = 10.0
    seed: int = 1000
    noiseless: bool = False   # y = H x exactly (sigma^2 still reported)
    rho_t: float = field(default=None)  # override for the user side, if given
    n_ue: int = 1             # antennas per user (K = users x n_ue streams)
    rt_block: bool = False    # Assumption 1: no correlation between different users' antennas

    def __post_init__(self):
        if self.rho_t is None:
            self.rho_t = self.rho
        if self.K % self.n_ue:
            raise ValueError("K must be a multiple of the antennas per user")


def _chunk(spec, c, Rr, Rt):
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([spec.seed, c])))
    nb = min(CHUNK, spec.batch - c * CHUNK)
    N, K = spec.N, spec.K
    s = np.sqrt(0.5 / N)
    om_r = rng.standard_normal((nb, N, K)) * s
    om_i = rng.standard_normal((nb, N, K)) * s
    if Rr is not None:   # R_r^{1/2} Omega: one real GEMM per component
        om_r = (Rr @ om_r.transpose(1, 0, 2).reshape(N, nb * K)).reshape(N, nb, K).transpose(1, 0, 2)
        om_i = (Rr @ om_i.transpose(1, 0, 2).reshape(N, nb * K)).reshape(N, nb, K).transpose(1, 0, 2)
    if Rt is not None:   # (.) R_t^{1/2}
        om_r = (om_r.reshape(nb * N, K) @ Rt).reshape(nb, N, K)
        om_i = (om_i.reshape(nb * N, K) @ Rt).reshape(nb, N, K)
    Hm = (om_r + 1j * om_i).astype(np.complex64)            # (nb, N, K)
    tx = rng.integers(0, spec.qam, size=(nb, K)).astype(np.uint8)
    x = qam_modulate(tx, spec.qam)
    sigma2 = float(snr_to_sigma2(spec.snr_db))
    yc = np.einsum("bnk,bk->bn", Hm.astype(np.complex128), x)
    if not spec.noiseless:
        sn = np.sqrt(sigma2 / 2.0)
        yc = yc + (rng.standard_normal((nb, N)) + 1j * rng.standard_normal((nb, N))) * sn
    H_store = np.ascontiguousarray(Hm.transpose(0, 2, 1))   # (nb, K, N): column-major per system
    return H_store, yc.astype(np.complex64), tx, x


def user_corr(spec):
    """R_t of a Spec: the exponential matrix of eq. (2) over all K streams, or,
    with rt_block (Section IV-B, Assumption 1), block-diagonal with one
    n_ue x n_ue exponential block per user and zero blocks between users."""
    if not spec.rt_block:
        return exp_corr(spec.K, spec.rho_t)
    R = np.zeros((spec.K, spec.K))
    for u in range(spec.K // spec.n_ue):
        sl = slice(u * spec.n_ue, (u + 1) * spec.n_ue)
        R[sl, sl] = exp_corr(spec.n_ue, spec.rho_t)
    return R


def generate(spec, chunks=None):
    """Draw the batch (or only the listed chunks, concatenated in order).

    Returns a dict with H (batch, K, N) complex64, y (batch, N) complex64,
    tx (batch, K) uint8 Gray labels, x (batch, K) complex128 transmitted
    symbols, sigma2 (batch,) float64, qam (batch,) int32.
    """
    Rr = None if spec.rho == 0 else sqrt_psd(exp_corr(spec.N, spec.rho))
    Rt = None if spec.rho_t == 0 else sqrt_psd(user_corr(spec))
    nchunks = -(-spec.batch // CHUNK)
    ids = range(nchunks) if chunks is None else chunks
    parts = [_chunk(spec, c, Rr, Rt) for c in ids]
    H = np.concatenate([p[0] for p in parts])
    y = np.concatenate([p[1] for p in parts])
    tx = np.concatenate([p[2] for p in parts])
    x = np.concatenate([p[3] for p in parts])
    n = H.shape[0]
    return {
        "H": H, "y": y, "tx": tx, "x": x,
        "sigma2": np.full(n, float(snr_to_sigma2(spec.snr_db))),
        "qam": np.full(n, spec.qam, dtype=np.int32),
        "N": spec.N, "K": spec.K,
    }


# The five workloads of the detection benchmarks, by what they are.
def c1_rayleigh_64x16(batch=1024, seed=1001):
    """N=64, K=16, i.i.d. Rayleigh, 16-QAM, SNR 10 dB."""
    return Spec(N=64, K=16, batch=batch, rho=0.0, qam=16, snr_db=10.0, seed=seed)


def c2_kron_128x32(batch=8192, snr_db=10.0, seed=1002):
    """N=128, K=32, Kronecker rho=0.5 both ends, 64-QAM, SNR 0..20 dB."""
    return Spec(N=128, K=32, batch=batch, rho=0.5, qam=64, snr_db=snr_db, seed=seed)


def c3_kron_256x64(batch=16384, seed=1003):
    """N=256, K=64, Kronecker rho=0.7 both ends, 64-QAM, SNR 18 dB."""
    return Spec(N=256, K=64, batch=batch, rho=0.7, qam=64, snr_db=18.0, seed=seed)


@dataclass
class MixedSpec:
    """An uneven batch: every system draws its K, the ratio N/K (N capped), rho
    and the QAM order uniformly from the given sets."""
    batch: int
    ks: tuple = (8, 16, 32, 64, 128)
    ratios: tuple = (2, 4, 8)
    n_cap: int = 512
    rhos: tuple = (0.0, 0.3, 0.7)
    qams: tuple = (16, 64, 256)
    snr_db: float = 18.0
    seed: int = 1004


def mixed_params(spec):
    """Per-system (N, K, rho, QAM order) of an uneven batch, in system order."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([spec.seed, 0x6d6978])))
    k = np.asarray(spec.ks, dtype=np.int32)[rng.integers(0, len(spec.ks), spec.batch)]
    r = np.asarray(spec.ratios, dtype=np.int32)[rng.integers(0, len(spec.ratios), spec.batch)]
    n = np.minimum(k * r, spec.n_cap).astype(np.int32)
    rho = np.asarray(spec.rhos, dtype=np.float64)[rng.integers(0, len(spec.rhos), spec.batch)]
    qam = np.asarray(spec.qams, dtype=np.int32)[rng.integers(0, len(spec.qams), spec.batch)]
    return n, k, rho, qam


def generate_mixed(spec):
    """Draw an uneven batch.  Systems with equal (N, K, rho, QAM order) are drawn
    together as one uniform batch (its own seed stream), then put back in
    system order.  Returns per-system lists H[i] (K, N) complex64, y[i] (N,),
    tx[i] (K,) uint8, x[i] (K,) complex128, and arrays n, k, rho, qam, sigma2."""
    n, k, rho, qam = mixed_params(spec)
    H = [None] * spec.batch
    y = [None] * spec.batch
    tx = [None] * spec.batch
    x = [None] * spec.batch
    keys = sorted(set(zip(n.tolist(), k.tolist(), rho.tolist(), qam.tolist())))
    for g, (gn, gk, grho, gq) in enumerate(keys):
        idx = np.nonzero((n == gn) & (k == gk) & (rho == grho) & (qam == gq))[0]
        d = generate(Spec(N=gn, K=gk, batch=len(idx), rho=grho, qam=gq, snr_db=spec.snr_db,
                          seed=spec.seed * 1000 + g))
        for j, i in enumerate(idx):
            H[i], y[i], tx[i], x[i] = d["H"][j], d["y"][j], d["tx"][j], d["x"][j]
    return {"H": H, "y": y, "tx": tx, "x": x, "n": n, "k": k, "rho": rho, "qam": qam,
            "sigma2": np.full(spec.batch, float(snr_to_sigma2(spec.snr_db)))}


def mixed_kron(batch=12000, seed=1004):
    """Uneven batch: K in {8,16,32,64,128}, N = K x {2,4,8} capped at 512, rho in
    {0, 0.3, 0.7}, 16/64/256-QAM, SNR 18 dB."""
    return MixedSpec(batch=batch, seed=seed)


@dataclass
class RBSpec:
    """Resource blocks sharing a channel: n_rb channels H (N x K), each seen by
    res_per_rb received vectors (subcarriers x symbols) with their own symbols
    and noise."""
    N: int
    K: int
    n_rb: int
    res_per_rb: int = 168
    rho: float = 0.5
    qam: int = 64
    snr_db: float = 15.0
    seed: int = 1005


def generate_rb(spec):
    """Draw the channels (one per resource block) and the received vectors.
    Returns H (n_rb, K, N) complex64, y (n_rb*res_per_rb, N) complex64,
    rb_index (n_rb*res_per_rb,) int32 (received vector s belongs to block
    s // res_per_rb), tx (n, K) uint8, x (n, K) complex128, sigma2 (n_rb,)
    float64 (one per block) and qam (n,) int32."""
    ch = generate(Spec(N=spec.N, K=spec.K, batch=spec.n_rb, rho=spec.rho, qam=spec.qam,
                       snr_db=spec.snr_db, seed=spec.seed))
    H = ch["H"]                                      # (n_rb, K, N)
    n = spec.n_rb * spec.res_per_rb
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([spec.seed, 0x7262])))
    tx = rng.integers(0, spec.qam, size=(n, spec.K)).astype(np.uint8)
    x = qam_modulate(tx, spec.qam)
    rb = (np.arange(n) // spec.res_per_rb).astype(np.int32)
    xb = x.reshape(spec.n_rb, spec.res_per_rb, spec.K)
    yc = np.matmul(xb, H.astype(np.complex128)).reshape(n, spec.N)   # y_s = H_rb x_s, block by block
    sigma2 = float(snr_to_sigma2(spec.snr_db))
    sn = np.sqrt(sigma2 / 2.0)
    yc = yc + (rng.standard_normal((n, spec.N)) + 1j * rng.standard_normal((n, spec.N))) * sn
    return {"H": H, "y": yc.astype(np.complex64), "rb_index": rb, "tx": tx, "x": x,
            "sigma2": np.full(spec.n_rb, sigma2), "qam": np.full(n, spec.qam, dtype=np.int32),
            "N": spec.N, "K": spec.K}


# ---- channel-estimate and time-variation input models (Section V-C) ----------

def csi_error(H, eps_db, seed):
    """Imperfect CSI: H_hat = H + dH (Section V-C), dH i.i.d. CN(0, s2) per
    entry with the channel-to-error power ratio eps: s2 = P_h 10^(-eps/10),
    where P_h = 1/N is the average power of an entry of H (Omega's variance,
    unit diagonal of R_r and R_t).  H in the storage layout (batch, K, N);
    returns complex64 of the same shape.  y stays the one made with H."""
    H = np.asarray(H)
    N = H.shape[-1]
    s = np.sqrt(0.5 * 10.0 ** (-float(eps_db) / 10.0) / N)
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0x637369])))
    dH = (rng.standard_normal(H.shape) + 1j * rng.standard_normal(H.shape)) * s
    return (H.astype(np.complex128) + dH).astype(np.complex64)


def doppler_corr(fd_hz, tau_s):
    """rho_tau = J_0(2 pi f_d tau), the one-step correlation of the first-order
    Gauss-Markov channel (Section V-C)."""
    from scipy.special import j0
    return float(j0(2.0 * np.pi * float(fd_hz) * float(tau_s)))


def gauss_markov(spec, steps, rho_tau):
    """A time-varying channel: H_0 drawn from spec, then H_i = rho_tau H_{i-1}
    + sqrt(1 - rho_tau^2) W_i with W_i drawn from the same spatial model
    (Section V-C), and at each step new symbols and noise: y_i = H_i x_i + n_i.
    Returns a list of `steps` dicts shaped like generate()'s (the innovation of
    step i uses seed spec.seed + 7919 i)."""
    out = [generate(spec)]
    a, c = float(rho_tau), float(np.sqrt(max(0.0, 1.0 - rho_tau * rho_tau)))
    for i in range(1, steps):
        w = generate(Spec(**{**spec.__dict__, "seed": spec.seed + 7919 * i}))
        H = (a * out[-1]["H"].astype(np.complex128) + c * w["H"].astype(np.complex128))
        # new symbols and noise from w; y recomputed with the aged channel
        Hc = H.transpose(0, 2, 1)                                    # (b, N, K)
        yc = np.einsum("bnk,bk->bn", Hc, w["x"])
        if not spec.noiseless:
            rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([spec.seed, 0x676d, i])))
            sn = np.sqrt(w["sigma2"][0] / 2.0)
            yc = yc + (rng.standard_normal(yc.shape) + 1j * rng.standard_normal(yc.shape)) * sn
        out.append(dict(w, H=H.astype(np.complex64), y=yc.astype(np.complex64)))
    return out


# ---- the same models drawn on the GPU (large Monte-Carlo runs) ---------------

def generate_torch(spec, chunk, count, device="cuda", h_true=None):
    """`count` systems of spec drawn on `device` with torch's generator
    (Philox) seeded by (spec.seed, chunk): the distributions of generate(),
    another random stream.  For Monte-Carlo runs of 10^5..10^6 systems, where
    drawing on the host would dominate; nothing compares them with the
    oracle.  Returns H (count, K, N) complex64, y (count, N) complex64,
    tx (count, K) uint8, x (count, K) complex128, sigma2 (count,) float64,
    qam (count,) int32.  With
    h_true given (same shape as H), y is formed with h_true instead of a new
    channel (an aged channel, say)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed((int(spec.seed) * 1000003 + int(chunk)) & 0x7FFFFFFFFFFFFFFF)
    N, K = spec.N, spec.K
    if h_true is None:   # complex64 arithmetic: H is stored in complex64 anyway
        s = float(np.sqrt(0.5 / N))
        om = torch.complex(torch.randn((count, N, K), generator=g, device=device, dtype=torch.float32),
                           torch.randn((count, N, K), generator=g, device=device, dtype=torch.float32)) * s
        if spec.rho != 0:
            Rr = torch.as_tensor(sqrt_psd(exp_corr(N, spec.rho)), device=device, dtype=torch.complex64)
            om = Rr @ om
        if spec.rho_t != 0:
            Rt = torch.as_tensor(sqrt_psd(user_corr(spec)), device=device, dtype=torch.complex64)
            om = om @ Rt
        Hm = om                                                       # (count, N, K)
    else:
        Hm = h_true.transpose(1, 2)
    tx = torch.randint(0, spec.qam, (count, K), generator=g, device=device, dtype=torch.int64)
    m = int(round(np.sqrt(spec.qam)))
    b = int(np.log2(m))
    gi, gq = tx >> b, tx & (m - 1)
    ji, jq = gi.clone(), gq.clone()
    sh = 1
    while sh < 16:              # Gray decode per axis
        ji ^= ji >> sh
        jq ^= jq >> sh
        sh <<= 1
    d = 1.0 / np.sqrt(2.0 * (spec.qam - 1) / 3.0)
    x = torch.complex((2 * ji - (m - 1)).double() * d, (2 * jq - (m - 1)).double() * d)
    sigma2 = float(snr_to_sigma2(spec.snr_db))
    y = (Hm.to(torch.complex128) @ x.unsqueeze(-1)).squeeze(-1)
    if not spec.noiseless:
        sn = float(np.sqrt(sigma2 / 2.0))
        y = y + torch.complex(torch.randn((count, N), generator=g, device=device, dtype=torch.float64),
                              torch.randn((count, N), generator=g, device=device, dtype=torch.float64)) * sn
    return {"H": Hm.transpose(1, 2).contiguous(), "y": y.to(torch.complex64), "tx": tx.to(torch.uint8), "x": x,
            "sigma2": torch.full((count,), sigma2, device=device, dtype=torch.float64),
            "qam": torch.full((count,), spec.qam, device=device, dtype=torch.int32)}


def csi_error_torch(H, eps_db, seed, chunk):
    """csi_error on the device (torch generator seeded by (seed, chunk))."""
    import torch
    g = torch.Generator(device=H.device)
    g.manual_seed((int(seed) * 1000033 + int(chunk)) & 0x7FFFFFFFFFFFFFFF)
    N = H.shape[-1]
    s = float(np.sqrt(0.5 * 10.0 ** (-float(eps_db) / 10.0) / N))
    dH = torch.complex(torch.randn(H.shape, generator=g, device=H.device, dtype=torch.float32),
                       torch.randn(H.shape, generator=g, device=H.device, dtype=torch.float32)) * s
    return H + dH
