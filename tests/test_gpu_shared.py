"""fpcg_detect_shared: one Gram per resource block (fpcg_gram), many received
vectors per block, against the oracle run on each vector with its block's H."""
import numpy as np
import pytest
import torch

from oracle import qam as Q
from paper_2504_09820_gb300 import fpcg as F
from paper_2504_09820_gb300 import workload as wl

from gpu_helpers import check_reduced_parity, gram_resid_rel, oracle_detect, rel_err

pytestmark = pytest.mark.gpu

PREC = dict(gram="bf16", mv="fp16", refine_steps=1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()


def _shared(d, iters, L, prec_kw, rb=None):
    n_rb, K, N = d["H"].shape
    dev = "cuda"
    H = torch.from_numpy(d["H"]).to(dev)
    prec = F.precision(**prec_kw)
    xdt = torch.complex128 if prec_kw.get("w") == "fp64" else torch.complex64
    A = torch.empty((n_rb, K, K), dtype=xdt, device=dev)
    b = torch.empty((n_rb, K), dtype=xdt, device=dev)
    F.fpcg_gram(H, torch.zeros((n_rb, N), dtype=torch.complex64, device=dev),
                torch.from_numpy(d["sigma2"]).to(dev), prec_kw["gram"], A, b)
    y = torch.from_numpy(d["y"]).to(dev)
    n = y.shape[0]
    rbi = torch.from_numpy(d["rb_index"] if rb is None else rb).to(dev)
    out = {"x": torch.empty((n, K), dtype=xdt, device=dev), "sym": torch.empty((n, K), dtype=torch.uint8, device=dev),
           "rel": torch.empty(n, dtype=torch.float64, device=dev), "st": torch.empty(n, dtype=torch.int32, device=dev),
           "be": torch.zeros(1, dtype=torch.int64, device=dev)}
    F.fpcg_detect_shared(A, H, y, rbi, torch.from_numpy(d["qam"]).to(dev), iters, L, prec, out["x"],
                         sym_idx=out["sym"], rel_res=out["rel"], tx_idx=torch.from_numpy(d["tx"]).to(dev),
                         bit_errors=out["be"], status=out["st"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _per_vector(d):
    """The same problems as independent systems: each y with its block's H."""
    rb = d["rb_index"]
    return {"H": d["H"][rb], "y": d["y"], "sigma2": d["sigma2"][rb], "qam": d["qam"], "tx": d["tx"]}


@pytest.mark.parametrize("N,K", [(64, 8), (128, 32), (256, 64), (512, 128)])
def test_shared_matches_oracle(N, K):
    d = wl.generate_rb(wl.RBSpec(N=N, K=K, n_rb=5, res_per_rb=24, seed=40 + K))
    L = min(8, K)
    res = _shared(d, 6, L, PREC)
    ref = oracle_detect(_per_vector(d), 6, PREC, L=L)
    check_reduced_parity(_per_vector(d), res["x"], ref["x"], 6, PREC, L=L)
    assert np.array_equal(Q.slice_symbols(res["x"], 64, "fp32"), res["sym"])
    assert int(res["be"][0]) == Q.bit_errors(res["sym"], d["tx"])
    allowed = F.ST_RHO_ZERO | (F.ST_BREAKDOWN if L == K else 0)
    assert np.all(res["st"] & ~allowed == 0)


def test_shared_fp64_equals_exact_solve():
    """fp64 CG, 2K iterations (in fp64 at kappa ~ 20, K steps leave ~1e-6; 2K reach
    rounding level) against the direct solve of each vector's own system."""
    from oracle import detect as D
    d = wl.generate_rb(wl.RBSpec(N=64, K=16, n_rb=3, res_per_rb=12, seed=3))
    res = _shared(d, 32, 0, dict(w="fp64", gram="fp64", mv="fp64", ip="fp64"))
    pv = _per_vector(d)
    A, b = D.gram_mf(pv["H"], pv["y"], pv["sigma2"])
    assert rel_err(res["x"], D.cholesky_solve(A, b)).max() < 1e-10


@pytest.mark.parametrize("force_simt", ["0", "1"])
@pytest.mark.parametrize("K", [8, 16])
def test_shared_bad_index(K, force_simt, monkeypatch):
    """An out-of-range group index on the tensor-core solver and on the SIMT kernel."""
    monkeypatch.setenv("FPCG_FORCE_SIMT", force_simt)
    d = wl.generate_rb(wl.RBSpec(N=64, K=K, n_rb=3, res_per_rb=4, seed=5))
    rb = d["rb_index"].copy()
    rb[2] = 3          # outside [0, n_rb)
    rb[5] = -1
    res = _shared(d, 6, 4, PREC, rb=rb)
    assert res["st"][2] == F.ST_BAD_INDEX and res["st"][5] == F.ST_BAD_INDEX
    assert np.all(res["x"][[2, 5]] == 0)
    ok = np.ones(len(rb), bool)
    ok[[2, 5]] = False
    assert np.all(res["st"][ok] & ~F.ST_RHO_ZERO == 0)
    assert np.all(res["sym"][[2, 5]] == 0) and np.all(res["rel"][[2, 5]] == 0)
    assert int(res["be"][0]) == Q.bit_errors(res["sym"][ok], d["tx"][ok])


@pytest.mark.parametrize("N,K,L", [(64, 8, 4), (32, 8, 8), (64, 8, 0), (128, 32, 8), (512, 128, 16)])
def test_shared_tensor_core_vs_simt(N, K, L, monkeypatch):
    """fpcg_detect_shared on the tensor-core solver (vectors in random block
    order, so the warps refill their slots) against the SIMT kernel on the same
    inputs, and against the oracle."""
    d = wl.generate_rb(wl.RBSpec(N=N, K=K, n_rb=6, res_per_rb=30, seed=70 + N + K + L))
    perm = np.random.default_rng(1).permutation(len(d["rb_index"]))
    d = dict(d, y=d["y"][perm], rb_index=d["rb_index"][perm], qam=d["qam"][perm], tx=d["tx"][perm])
    pk = dict(PREC, mv="bf16") if L == 16 else PREC
    tc = _shared(d, 6, L, pk)
    ref = oracle_detect(_per_vector(d), 6, pk, L=(L or None))
    check_reduced_parity(_per_vector(d), tc["x"], ref["x"], 6, pk, L=(L or None))
    monkeypatch.setenv("FPCG_FORCE_SIMT", "1")
    simt = _shared(d, 6, L, pk)
    e = rel_err(tc["x"], simt["x"])
    assert np.quantile(e, 0.99) < 4e-3 and e.max() < 2e-2, (np.quantile(e, 0.99), e.max())
    assert int(tc["be"][0]) == Q.bit_errors(tc["sym"], d["tx"])
    allowed = F.ST_RHO_ZERO | (F.ST_BREAKDOWN if L == K else 0)
    assert np.all(tc["st"] & ~allowed == 0)


def _grouped(d, iters, L, prec_kw):
    """Same problems through fpcg_detect_grouped (the vectors are block-major)."""
    n_rb, K, N = d["H"].shape
    H = torch.from_numpy(d["H"]).cuda()
    A = torch.empty((n_rb, K, K), dtype=torch.complex64, device="cuda")
    b = torch.empty((n_rb, K), dtype=torch.complex64, device="cuda")
    F.fpcg_gram(H, torch.zeros((n_rb, N), dtype=torch.complex64, device="cuda"),
                torch.from_numpy(d["sigma2"]).cuda(), prec_kw["gram"], A, b)
    rb = d["rb_index"]
    start = np.searchsorted(rb, np.arange(n_rb + 1)).astype(np.int64)
    y = torch.from_numpy(d["y"]).cuda()
    n = y.shape[0]
    out = {"x": torch.empty((n, K), dtype=torch.complex64, device="cuda"),
           "sym": torch.empty((n, K), dtype=torch.uint8, device="cuda"),
           "rel": torch.empty(n, dtype=torch.float64, device="cuda"),
           "st": torch.empty(n, dtype=torch.int32, device="cuda"),
           "be": torch.zeros(1, dtype=torch.int64, device="cuda")}
    F.fpcg_detect_grouped(A, H, y, torch.from_numpy(start).cuda(), torch.from_numpy(d["qam"]).cuda(), iters, L,
                          F.precision(**prec_kw), out["x"], sym_idx=out["sym"], rel_res=out["rel"],
                          tx_idx=torch.from_numpy(d["tx"]).cuda(), bit_errors=out["be"], status=out["st"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("N,K,L", [(64, 16, 4), (128, 32, 8), (256, 64, 8), (256, 64, 0), (256, 64, 16),
                                   (64, 8, 8), (32, 8, 4), (64, 8, 0), (512, 128, 8), (256, 128, 16),
                                   (512, 128, 0)])
def test_grouped_matches_oracle(N, K, L, monkeypatch):
    """Tensor-core grouped solver (K = 8 in 16-wide slots), against the oracle,
    and against the SIMT kernel (forced) on the same inputs."""
    d = wl.generate_rb(wl.RBSpec(N=N, K=K, n_rb=7, res_per_rb=40, seed=90 + K + L))
    pk = dict(PREC, mv="bf16") if L == 16 else PREC
    res = _grouped(d, 6, L, pk)
    ref = oracle_detect(_per_vector(d), 6, pk, L=(L or None))
    check_reduced_parity(_per_vector(d), res["x"], ref["x"], 6, pk, L=(L or None))
    assert np.array_equal(Q.slice_symbols(res["x"], 64, "fp32"), res["sym"])
    assert int(res["be"][0]) == Q.bit_errors(res["sym"], d["tx"])
    allowed = F.ST_RHO_ZERO | (F.ST_BREAKDOWN if L == K else 0)
    assert np.all(res["st"] & ~allowed == 0)
    monkeypatch.setenv("FPCG_FORCE_SIMT", "1")
    simt = _grouped(d, 6, L, pk)
    e2 = rel_err(res["x"], simt["x"])
    assert np.quantile(e2, 0.99) < 4e-3 and e2.max() < 2e-2


# Plain CG (L = 0) runs K iterations: an unconverged plain-CG iterate at
# kappa ~ 40 moves by up to 2e-2 when one fp16 rounding of p comes out the
# other way, which a different fp32 summation order causes now and then (on
# both kernels alike); converged, it is insensitive to that.
@pytest.mark.parametrize("N,K,L,iters", [(256, 64, 8, 6), (512, 128, 8, 6), (64, 8, 4, 6), (32, 8, 8, 6),
                                         (64, 8, 0, 8)])
def test_solve_gram_tensor_core_vs_simt(N, K, L, iters, monkeypatch):
    """fpcg_solve_gram on the tensor-core solver and on the SIMT kernel, each
    against the oracle's emulation of the same precisions (from H and y)."""
    d = wl.generate(wl.Spec(N=N, K=K, batch=300, rho=0.7, qam=64, snr_db=18.0, seed=12))
    H = torch.from_numpy(d["H"]).cuda()
    A = torch.empty((300, K, K), dtype=torch.complex64, device="cuda")
    b = torch.empty((300, K), dtype=torch.complex64, device="cuda")
    F.fpcg_gram(H, torch.from_numpy(d["y"]).cuda(), torch.from_numpy(d["sigma2"]).cuda(), "bf16", A, b)
    prec = F.precision(gram="bf16", mv="fp16", refine_steps=1)
    outs = []
    for force in ("0", "1"):
        monkeypatch.setenv("FPCG_FORCE_SIMT", force)
        x = torch.empty((300, K), dtype=torch.complex64, device="cuda")
        st = torch.empty(300, dtype=torch.int32, device="cuda")
        F.fpcg_solve_gram(A, b, iters, L, prec, x, status=st)
        torch.cuda.synchronize()
        outs.append((x.cpu().numpy(), st.cpu().numpy()))
    pko = dict(gram="bf16", mv="fp16", refine_steps=1)
    ref = oracle_detect(d, iters, pko, L=(L or None))
    for x, _ in outs:
        check_reduced_parity(d, x, ref["x"], iters, pko, L=(L or None))
    allowed = F.ST_RHO_ZERO | (F.ST_BREAKDOWN if L == K else 0)
    assert np.all(outs[0][1] & ~allowed == 0)


def _grouped_subset(d, sizes):
    """Keep the first sizes[g] received vectors of block g (blocks may end up
    empty or with fewer vectors than a CTA has warps)."""
    per = len(d["rb_index"]) // d["H"].shape[0]
    keep = np.concatenate([np.arange(g * per, g * per + m) for g, m in enumerate(sizes)])
    return dict(d, y=d["y"][keep], rb_index=d["rb_index"][keep], qam=d["qam"][keep], tx=d["tx"][keep])


@pytest.mark.parametrize("N,K,L", [(128, 32, 8), (512, 128, 8), (64, 8, 4)])
def test_grouped_ragged_rounds(N, K, L):
    """Groups of 20, 1, 0, 13, 8 and 7 vectors: the last round of a group
    leaves warps without a vector, which run on b = 0 and write nothing."""
    d = wl.generate_rb(wl.RBSpec(N=N, K=K, n_rb=6, res_per_rb=20, seed=300 + K))
    d = _grouped_subset(d, [20, 1, 0, 13, 8, 7])
    res = _grouped(d, 6, L, PREC)
    ref = oracle_detect(_per_vector(d), 6, PREC, L=L)
    check_reduced_parity(_per_vector(d), res["x"], ref["x"], 6, PREC, L=L)
    assert int(res["be"][0]) == Q.bit_errors(res["sym"], d["tx"])
    assert np.all(res["st"] & ~F.ST_RHO_ZERO == 0)


@pytest.mark.parametrize("K", [32, 128])
def test_grouped_lockstep_independence(K):
    """The eight vectors of a round share every product with A, each in its own
    columns: a vector that breaks down at once (y = 0) changes nothing for the
    others, bit for bit, and gets x = 0 with FPCG_ST_RHO_ZERO."""
    d = wl.generate_rb(wl.RBSpec(N=4 * K, K=K, n_rb=3, res_per_rb=24, seed=500 + K))
    a = _grouped(d, 6, 8, PREC)
    z = [3, 30, 41]
    y = d["y"].copy()
    y[z] = 0
    b = _grouped(dict(d, y=y), 6, 8, PREC)
    others = np.setdiff1d(np.arange(len(y)), z)
    assert np.array_equal(a["x"][others], b["x"][others])
    assert np.array_equal(a["rel"][others], b["rel"][others])
    assert np.all(b["x"][z] == 0) and np.all(b["st"][z] == F.ST_RHO_ZERO)


# ---- resid = FP64 on the tensor-core solvers: the residual against the given fp32 A ----

GR = dict(PREC, resid="fp64")


def _solve(A, b, iters, L, pk):
    n, K = b.shape
    x = torch.empty((n, K), dtype=torch.complex64, device="cuda")
    rel = torch.empty(n, dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    F.fpcg_solve_gram(A, b, iters, L, F.precision(**pk), x, rel_res=rel, status=st)
    torch.cuda.synchronize()
    return x.cpu().numpy(), rel.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("N,K,L,iters", [(64, 8, 4, 6), (128, 16, 0, 12), (256, 64, 8, 6), (512, 128, 8, 6),
                                         (512, 128, 16, 5)])
def test_solve_gram_gram_residual(N, K, L, iters, monkeypatch):
    """fpcg_solve_gram with resid = FP64 on the tensor-core solver (the refinement
    residual and rel_res against the given fp32 A, read again from global
    memory): against the oracle with its residual on its own Gram matrix,
    against the SIMT kernel's compensated residual, and rel_res against
    b - A x of the returned x in float64 within the fp32 residual's bound."""
    d = wl.generate(wl.Spec(N=N, K=K, batch=300, rho=0.7, qam=64, snr_db=18.0, seed=13 + K + L))
    H = torch.from_numpy(d["H"]).cuda()
    A = torch.empty((300, K, K), dtype=torch.complex64, device="cuda")
    b = torch.empty((300, K), dtype=torch.complex64, device="cuda")
    F.fpcg_gram(H, torch.from_numpy(d["y"]).cuda(), torch.from_numpy(d["sigma2"]).cuda(), "bf16", A, b)
    pk = dict(GR, mv="bf16") if L == 16 else GR
    x, rel, st = _solve(A, b, iters, L, pk)
    ref = oracle_detect(d, iters, pk, L=(L or None))
    check_reduced_parity(d, x, ref["x"], iters, pk, L=(L or None))
    own, bound = gram_resid_rel(A.cpu().numpy(), b.cpu().numpy(), x)
    assert np.all(np.abs(rel - own) <= 2e-3 * own + bound), np.max(np.abs(rel - own) / (2e-3 * own + bound))
    allowed = F.ST_RHO_ZERO | (F.ST_BREAKDOWN if L == K else 0)
    assert np.all(st & ~allowed == 0)
    monkeypatch.setenv("FPCG_FORCE_SIMT", "1")
    xs, _, _ = _solve(A, b, iters, L, pk)
    e = rel_err(x, xs)
    assert np.quantile(e, 0.99) < 4e-3 and e.max() < 2e-2


@pytest.mark.parametrize("K", [16, 128])
def test_gram_residual_refines_past_the_matvec_matrix(K):
    """Converged solves (2K iterations, plain CG, one refinement pass of 2K more):
    with the residual against the matvec copy of A the refinement stops at the
    rounding of A to fp16, with the residual against A itself it goes on; b - A x
    against the given A (float64) is far smaller with resid = FP64."""
    N = 4 * K
    d = wl.generate(wl.Spec(N=N, K=K, batch=200, rho=0.5, qam=16, snr_db=20.0, seed=31 + K))
    H = torch.from_numpy(d["H"]).cuda()
    A = torch.empty((200, K, K), dtype=torch.complex64, device="cuda")
    b = torch.empty((200, K), dtype=torch.complex64, device="cuda")
    F.fpcg_gram(H, torch.from_numpy(d["y"]).cuda(), torch.from_numpy(d["sigma2"]).cuda(), "bf16", A, b)
    An, bn = A.cpu().numpy(), b.cpu().numpy()
    x64, rel64, _ = _solve(A, b, 2 * K, 0, GR)
    x32, _, _ = _solve(A, b, 2 * K, 0, dict(GR, resid="fp32"))
    own64, bound = gram_resid_rel(An, bn, x64)
    own32, _ = gram_resid_rel(An, bn, x32)
    assert np.median(own32) > 10 * np.median(own64), (np.median(own32), np.median(own64))
    assert np.all(np.abs(rel64 - own64) <= 2e-3 * own64 + bound)


@pytest.mark.parametrize("N,K,L", [(64, 16, 4), (256, 64, 8), (64, 8, 0), (512, 128, 8)])
def test_grouped_gram_residual(N, K, L, monkeypatch):
    """fpcg_detect_grouped with resid = FP64 on the tensor-core solver (eight
    vectors in lockstep; each warp forms its own residual from the group's fp32
    A): against the oracle, the SIMT kernel, and b - A x in float64."""
    d = wl.generate_rb(wl.RBSpec(N=N, K=K, n_rb=7, res_per_rb=40, seed=190 + K + L))
    res = _grouped(d, 6, L, GR)
    pv = _per_vector(d)
    ref = oracle_detect(pv, 6, GR, L=(L or None))
    check_reduced_parity(pv, res["x"], ref["x"], 6, GR, L=(L or None))
    assert int(res["be"][0]) == Q.bit_errors(res["sym"], d["tx"])
    allowed = F.ST_RHO_ZERO | (F.ST_BREAKDOWN if L == K else 0)
    assert np.all(res["st"] & ~allowed == 0)
    # b - A x in float64 with the group's fp32 A as the library forms it and the
    # exact matched filter of the rounded inputs; the kernel's own b (fp32 sums
    # on the tensor cores) is not returned, so the check allows three times the
    # distance of another fp32 summation of b (fpcg_gram per vector) from the exact one
    n_rb = d["H"].shape[0]
    A = torch.empty((n_rb, K, K), dtype=torch.complex64, device="cuda")
    bz = torch.empty((n_rb, K), dtype=torch.complex64, device="cuda")
    F.fpcg_gram(torch.from_numpy(d["H"]).cuda(), torch.zeros((n_rb, N), dtype=torch.complex64, device="cuda"),
                torch.from_numpy(d["sigma2"]).cuda(), "bf16", A, bz)
    A = A.cpu().numpy()[d["rb_index"]]
    from oracle.formats import flc
    b = np.einsum("bkn,bn->bk", np.conj(flc(pv["H"], "bf16")), flc(pv["y"], "bf16"))
    n = len(d["rb_index"])
    Av = torch.empty((n, K, K), dtype=torch.complex64, device="cuda")
    bv = torch.empty((n, K), dtype=torch.complex64, device="cuda")
    F.fpcg_gram(torch.from_numpy(pv["H"]).cuda(), torch.from_numpy(pv["y"]).cuda(),
                torch.from_numpy(pv["sigma2"]).cuda(), "bf16", Av, bv)
    del Av
    db = np.linalg.norm(bv.cpu().numpy() - b, axis=1) / np.linalg.norm(b, axis=1)
    own, bound = gram_resid_rel(A, b, res["x"])
    assert np.all(np.abs(res["rel"] - own) <= 2e-3 * own + bound + 3 * db + 1e-7), \
        np.max(np.abs(res["rel"] - own) - 2e-3 * own - bound - 3 * db)
    monkeypatch.setenv("FPCG_FORCE_SIMT", "1")
    simt = _grouped(d, 6, L, GR)
    e2 = rel_err(res["x"], simt["x"])
    assert np.quantile(e2, 0.99) < 4e-3 and e2.max() < 2e-2


@pytest.mark.parametrize("N,K,L", [(64, 8, 4), (512, 128, 8)])
def test_shared_gram_residual(N, K, L):
    """fpcg_detect_shared with resid = FP64 on the tensor-core solver (vectors in
    random block order: the warps refill their slots and residual matrices)."""
    d = wl.generate_rb(wl.RBSpec(N=N, K=K, n_rb=6, res_per_rb=30, seed=270 + K))
    perm = np.random.default_rng(2).permutation(len(d["rb_index"]))
    d = dict(d, y=d["y"][perm], rb_index=d["rb_index"][perm], qam=d["qam"][perm], tx=d["tx"][perm])
    res = _shared(d, 6, L, GR)
    ref = oracle_detect(_per_vector(d), 6, GR, L=L)
    check_reduced_parity(_per_vector(d), res["x"], ref["x"], 6, GR, L=L)
    assert int(res["be"][0]) == Q.bit_errors(res["sym"], d["tx"])
    assert np.all(res["st"] & ~F.ST_RHO_ZERO == 0)
