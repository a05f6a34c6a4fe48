"""Serving loop on the GPU: requests admitted by memory budget and run
concurrently give, for each request, the same results as that request alone and
as direct fpcg_gram + fpcg_detect_grouped calls on its data."""
import numpy as np
import pytest
import torch

from paper_2504_09820_gb300 import fpcg as F
from paper_2504_09820_gb300 import serve as SV
from paper_2504_09820_gb300 import workload as wl

pytestmark = pytest.mark.gpu

SLOT_SHAPES = [(64, 8), (128, 32), (256, 64), (512, 128)]


@pytest.fixture(scope="module")
def slots():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    F.lib()
    return {(N, K): SV.pin_slot(wl.generate_rb(wl.RBSpec(N=N, K=K, n_rb=10, rho=0.5, qam=64, snr_db=15.0,
                                                          seed=70 + K)))
            for N, K in SLOT_SHAPES}


def _outputs(r):
    return {k: v.clone() for k, v in r.out.items()}


def test_alone_equals_in_mix_and_direct(slots):
    rng = np.random.default_rng(3)
    probe = SV.slot_request(0, slots[(256, 64)], 100, 0.0)
    budget = 3 * SV.request_bytes(probe.n_rb, probe.n_re, 256, 64) + SV.request_bytes(10, 1680, 512, 128)
    srv = SV.Server(budget, n_streams=3)
    srv.run([probe])
    alone = _outputs(probe)
    assert probe.done is not None and probe.latency() > 0

    # the same request among others that arrive while it runs
    mix = [SV.slot_request(0, slots[(256, 64)], 100, 0.002)]
    for i in range(1, 9):
        N, K = SLOT_SHAPES[rng.integers(len(SLOT_SHAPES))]
        mix.append(SV.slot_request(i, slots[(N, K)], int(rng.integers(12, 121)), float(rng.uniform(0, 0.004))))
    srv.run(mix)
    assert all(r.done is not None for r in mix)
    for k, v in alone.items():
        assert torch.equal(v, mix[0].out[k]), k
    # admission kept the budget: the arena is empty again
    assert srv.arena.used == 0 and srv.arena.free_list == [(0, srv.arena.size)]

    # direct library calls on the same data
    d = {k: getattr(probe, k).cuda() for k in ("H", "y", "rb", "start", "sigma2", "qam", "tx")}
    A = torch.empty((probe.n_rb, 64, 64), dtype=torch.complex64, device="cuda")
    b = torch.empty((probe.n_rb, 64), dtype=torch.complex64, device="cuda")
    F.fpcg_gram(d["H"], torch.zeros((probe.n_rb, 256), dtype=torch.complex64, device="cuda"), d["sigma2"],
                "bf16", A, b)
    x = torch.empty((probe.n_re, 64), dtype=torch.complex64, device="cuda")
    sym = torch.empty((probe.n_re, 64), dtype=torch.uint8, device="cuda")
    bits = torch.zeros(1, dtype=torch.int64, device="cuda")
    F.fpcg_detect_grouped(A, d["H"], d["y"], d["start"], d["qam"], 6, 8, F.precision(**srv.prec_kw), x,
                          sym_idx=sym, tx_idx=d["tx"], bit_errors=bits)
    torch.cuda.synchronize()
    assert torch.equal(x.cpu(), alone["x"]) and torch.equal(sym.cpu(), alone["sym"])
    assert int(bits[0]) == int(alone["bits"][0])


def test_budget_limits_concurrency(slots):
    """With room for one large request at a time the requests still all finish,
    in arrival order of admission."""
    reqs = [SV.slot_request(i, slots[(512, 128)], 120, 0.0005 * i) for i in range(4)]
    one = SV.request_bytes(reqs[0].n_rb, reqs[0].n_re, 512, 128)
    srv = SV.Server(int(one * 1.5), n_streams=4)
    srv.run(reqs)
    adm = [r.admitted for r in reqs]
    assert all(r.done is not None for r in reqs) and adm == sorted(adm)
    for a, b in zip(reqs, reqs[1:]):       # never two in flight: each admitted after the previous finished
        assert b.admitted >= a.done


def test_gram_kept_across_aged_slots():
    """gram_max_age = 1: the second slot of a user group (its channel aged by
    one Gauss-Markov step, Section V-C) is detected against the channel
    estimate and Gram matrices kept from the first slot -- exactly what direct
    fpcg_gram + fpcg_detect_grouped calls on the kept channel give -- and a
    slot three steps later forms new ones."""
    import dataclasses
    spec = wl.RBSpec(N=128, K=32, n_rb=6, rho=0.5, qam=64, snr_db=15.0, seed=91)
    s0 = wl.generate_rb(spec)
    w = wl.generate_rb(dataclasses.replace(spec, seed=92))
    a = wl.doppler_corr(100.0, 1e-3)
    c = float(np.sqrt(1.0 - a * a))
    H1 = (a * s0["H"].astype(np.complex128) + c * w["H"].astype(np.complex128)).astype(np.complex64)
    rb = w["rb_index"]
    noise = w["y"].astype(np.complex128) - np.einsum("rkn,rk->rn", w["H"][rb].astype(np.complex128), w["x"])
    y1 = (np.einsum("rkn,rk->rn", H1[rb].astype(np.complex128), w["x"]) + noise).astype(np.complex64)
    s1 = dict(w, H=H1, y=y1)
    p0, p1 = SV.pin_slot(s0), SV.pin_slot(s1)
    S = 60
    probe = SV.slot_request(0, p0, S, 0.0)
    srv = SV.Server(4 * SV.request_bytes(probe.n_rb, probe.n_re, 128, 32), n_streams=2, gram_max_age=1)

    def req(rid, pinned, slot):
        r = SV.slot_request(rid, pinned, S, 0.0)
        r.key, r.slot_index = "group-a", slot
        return r
    r0, r1, r3 = req(0, p0, 0), req(1, p1, 1), req(3, p1, 3)
    srv.run([r0])
    srv.run([r1])
    srv.run([r3])
    assert not r0.reused and r1.reused and not r3.reused

    def direct(Hs, r):
        dev = "cuda"
        H = r.H.clone().to(dev) if Hs is None else torch.from_numpy(Hs[:r.n_rb]).to(dev)
        A = torch.empty((r.n_rb, 32, 32), dtype=torch.complex64, device=dev)
        b = torch.empty((r.n_rb, 32), dtype=torch.complex64, device=dev)
        F.fpcg_gram(H, torch.zeros((r.n_rb, 128), dtype=torch.complex64, device=dev), r.sigma2.to(dev),
                    srv.prec_kw["gram"], A, b)
        x = torch.empty((r.n_re, 32), dtype=torch.complex64, device=dev)
        sym = torch.empty((r.n_re, 32), dtype=torch.uint8, device=dev)
        F.fpcg_detect_grouped(A, H, r.y.to(dev), r.start.to(dev), r.qam.to(dev), srv.iters, min(srv.block_L, 32),
                              srv.prec, x, sym_idx=sym)
        torch.cuda.synchronize()
        return x.cpu(), sym.cpu()
    x1, sym1 = direct(s0["H"], r1)            # the kept (step-0) channel
    assert torch.equal(r1.out["x"], x1) and torch.equal(r1.out["sym"], sym1)
    x3, sym3 = direct(None, r3)               # its own channel: formed anew
    assert torch.equal(r3.out["x"], x3) and torch.equal(r3.out["sym"], sym3)
