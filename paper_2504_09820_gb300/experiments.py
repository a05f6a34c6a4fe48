"""The Monte-Carlo experiments of Section V, run on the library's kernels.

Setup of Section V-A: N = 256 receive antennas, K = 32 streams (8 users with
4 antennas each), 16-QAM, block size L = 8, exponential correlation zeta at
both ends (eq. 2), SNR 20 dB unless swept.  Every detection runs through
fpcg_detect / fpbjcg_detect; the channels and symbols are drawn on the GPU
(workload.generate_torch), and each chunk of trials is drawn once and fed
to every detector variant and iteration count, so all curves of a figure see
the same channels.

Precisions follow the paper's roles: A is formed at fp32 (the paper takes A
as given at full precision), the matrix-vector products at u_MV, the inner
products at u_IP, no refinement steps (Algorithms 2 and 3 as printed).  The
working precision u_W is fp32 (the paper: fp64); "CG fp64" is the all-fp64
mode.  LMMSE is fp64 CG run for 2K iterations, which reaches the exact
LMMSE solution at these condition numbers (finite termination).

  python -m paper_2504_09820_gb300.experiments <name> [--trials T] [--out F]

prints one JSON line per experiment (bit error rates, per variant and point).
Experiments: mv_ip (Fig. ip_mv), heuristic (Fig. Heuristic), convergence
(Fig. pcg, with the iteration counts of Section V-C.3), ber_snr (Fig.
ber_pcg), csi (Fig. ber_pcg_im), time_varying (Fig. ber_time), users
(Assumption 1 against eq. 2's full R_t, with kappa(A) and kappa(A_bar) of
Theorem 5).
"""
import argparse
import json
import math
import sys
import time
from collections import defaultdict

import numpy as np
import torch

from . import fpcg as F
from . import workload as wl

N_RX, K_STREAMS, N_UE, QAM, L_BJ, SNR_DB = 256, 32, 4, 16, 8, 20.0
CHUNK = 32768


def prec_of(name):
    """Precision roles of the named detector variants."""
    if name in ("cg64", "lmmse"):
        return F.precision(w="fp64")
    table = {
        "mv_bf16": dict(mv="bf16", ip="fp32"),
        "ip_bf16": dict(mv="fp32", ip="bf16"),
        "mv_ip_bf16": dict(mv="bf16", ip="bf16"),
        "fp32": dict(mv="fp32", ip="fp32"),
        "fp16": dict(mv="fp16", ip="fp32"),
        "bf16": dict(mv="bf16", ip="fp32"),
    }
    return F.precision(gram="fp32", w="fp32", **table[name])


def _spec(zeta, snr_db=SNR_DB, seed=1, **kw):
    return wl.Spec(N=N_RX, K=K_STREAMS, batch=0, rho=zeta, qam=QAM, snr_db=snr_db, seed=seed, n_ue=N_UE, **kw)


def _bits_per_system():
    return K_STREAMS * int(round(math.log2(QAM)))


def _errors(H, d, iters, prec, L):
    r = F.detect(H, d["y"], d["sigma2"], d["qam"], iters, prec, L=L, tx_idx=d["tx"])
    return r["bit_errors"]


def ber_curves(spec, variants, iters_list, trials, device="cuda", csi_eps=None, lmmse=True):
    """BER of each (name, L) variant at each iteration count, on `trials`
    systems of spec; plus the LMMSE BER.  With csi_eps the detectors see the
    estimate H + dH (channel-to-error ratio csi_eps dB) instead of H."""
    acc = defaultdict(lambda: torch.zeros(1, dtype=torch.int64, device=device))
    done = 0
    c = 0
    while done < trials:
        n = min(CHUNK, trials - done)
        d = wl.generate_torch(spec, c, n, device=device)
        H = wl.csi_error_torch(d["H"], csi_eps, spec.seed, c) if csi_eps is not None else d["H"]
        for name, L in variants:
            prec = prec_of(name)
            for it in iters_list:
                acc[(name, L, it)] += _errors(H, d, it, prec, L)
        if lmmse:
            acc["lmmse"] += _errors(H, d, 2 * K_STREAMS, prec_of("lmmse"), None)
        done += n
        c += 1
    tot = trials * _bits_per_system()
    out = {"trials": trials, "curves": {}, "lmmse": None}
    for name, L in variants:
        key = name if L is None else f"{name}_bj{L}"
        out["curves"][key] = {int(it): int(acc[(name, L, it)].item()) / tot for it in iters_list}
    if lmmse:
        out["lmmse"] = int(acc["lmmse"].item()) / tot
    return out


def iterations_to_lmmse(curve, lmmse, rel=0.05):
    """First iteration count whose BER is within `rel` of the LMMSE BER."""
    for it in sorted(curve):
        if curve[it] <= lmmse * (1.0 + rel):
            return it
    return None


def kappa_sample(spec, count=2048, device="cuda", bj_L=None):
    """Condition numbers of A = H^H H + sigma^2 I (fpcg_gram, fp64) on `count`
    channels; with bj_L also of A_bar = M_d^{1/2} A M_d^{1/2}, M_d the inverse
    of A's L x L diagonal blocks (eq. pre_BJ), via the eigenvalues of M_d A."""
    d = wl.generate_torch(spec, 10 ** 6, count, device=device)
    A = torch.empty((count, K_STREAMS, K_STREAMS), dtype=torch.complex128, device=device)
    b = torch.empty((count, K_STREAMS), dtype=torch.complex128, device=device)
    F.fpcg_gram(d["H"], d["y"], d["sigma2"], "fp64", A, b)
    ev = torch.linalg.eigvalsh(A)
    out = {"kappa": (ev[:, -1] / ev[:, 0]).cpu().numpy()}
    if bj_L:
        D = torch.zeros_like(A)
        for j in range(0, K_STREAMS, bj_L):
            D[:, j:j + bj_L, j:j + bj_L] = torch.linalg.inv(A[:, j:j + bj_L, j:j + bj_L])
        e = torch.linalg.eigvals(D @ A).real
        out["kappa_bar"] = (e.max(dim=1).values / e.min(dim=1).values).cpu().numpy()
    return out


def exp_mv_ip(trials, zetas=(0.0, 0.5, 0.8), iters=range(1, 41)):
    res = {}
    for z in zetas:
        res[str(z)] = ber_curves(_spec(z, seed=11), [("cg64", None), ("mv_bf16", None), ("ip_bf16", None),
                                                     ("mv_ip_bf16", None)], list(iters), trials)
    return {"experiment": "mv_ip", "figure": "Fig. ip_mv", "snr_db": SNR_DB, "results": res}


def exp_heuristic(trials, zetas=(0.0, 0.5, 0.8), iters=range(1, 21)):
    res = {}
    for z in zetas:
        spec = _spec(z, seed=12)
        kap = float(np.mean(kappa_sample(spec)["kappa"]))
        fmt, ub = F.fpcg_choose_precision(K_STREAMS, kap)
        variants = [("cg64", None), ("bf16", None), ("fp16", None)]
        if fmt in ("fp32",):
            variants.append(("fp32", None))
        r = ber_curves(spec, variants, list(iters), trials)
        r.update(mean_kappa=kap, u_bound=ub, chosen=fmt)
        res[str(z)] = r
    return {"experiment": "heuristic", "figure": "Fig. Heuristic", "snr_db": SNR_DB, "results": res}


def exp_convergence(trials, zeta=0.8, iters=range(1, 26)):
    spec = _spec(zeta, seed=13)
    r = ber_curves(spec, [("cg64", None), ("fp32", None), ("fp16", L_BJ)], list(iters), trials)
    lm = r["lmmse"]
    r["iterations_to_lmmse"] = {k: iterations_to_lmmse(v, lm) for k, v in r["curves"].items()}
    r["paper_iterations"] = {"cg64": 15, "fp32": 17, "fp16_bj8": 10}
    return {"experiment": "convergence", "figure": "Fig. pcg", "zeta": zeta, "snr_db": SNR_DB, "results": r}


def snr_gap(snrs, ber_ref, ber, level):
    """SNR (dB) that `ber` needs beyond `ber_ref` to reach BER `level`
    (log-linear interpolation between the sweep points); None if a curve never
    reaches it."""
    def cross(b):
        lb = np.log10(np.maximum(np.asarray(b, dtype=np.float64), 1e-12))
        t = math.log10(level)
        for i in range(len(snrs) - 1):
            if lb[i] >= t >= lb[i + 1] and lb[i] != lb[i + 1]:
                return snrs[i] + (t - lb[i]) / (lb[i + 1] - lb[i]) * (snrs[i + 1] - snrs[i])
        return None
    a, b = cross(ber_ref), cross(ber)
    return None if a is None or b is None else b - a


def _ber_vs_snr(trials, zeta, snrs, iters, csi_eps=None, seed=14):
    curves = defaultdict(list)
    for snr in snrs:
        r = ber_curves(_spec(zeta, snr_db=snr, seed=seed + int(snr * 10)),
                       [("cg64", None), ("fp16", None), ("fp16", L_BJ)], [iters], trials, csi_eps=csi_eps)
        curves["lmmse"].append(r["lmmse"])
        for k, v in r["curves"].items():
            curves[k].append(v[iters])
    gaps = {lvl: snr_gap(list(snrs), curves["lmmse"], curves["fp16_bj8"], lvl) for lvl in (1e-2, 1e-3, 1e-4)}
    return dict(curves), {f"{k:g}": v for k, v in gaps.items()}


def exp_ber_snr(trials, zeta=0.8, snrs=tuple(range(0, 31, 2)), iters=10):
    curves, gaps = _ber_vs_snr(trials, zeta, snrs, iters)
    return {"experiment": "ber_snr", "figure": "Fig. ber_pcg", "zeta": zeta, "iters": iters, "snr_db": list(snrs),
            "ber": curves, "fp16_bj8_gap_db_vs_lmmse": gaps, "paper_gap_db": 1.2}


def exp_csi(trials, zeta=0.8, snrs=tuple(range(0, 31, 2)), iters=10, eps=(20.0, 25.0)):
    res = {}
    for e in eps:
        curves, gaps = _ber_vs_snr(trials, zeta, snrs, iters, csi_eps=e, seed=15)
        res[f"{e:g}"] = {"ber": curves, "fp16_bj8_gap_db_vs_lmmse": gaps}
    return {"experiment": "csi", "figure": "Fig. ber_pcg_im", "zeta": zeta, "iters": iters, "snr_db": list(snrs),
            "results": res}


def _detect_by_format(H, d, iters, fmts, L):
    """Bit errors when system s runs at its own format fmts[s] (one call per format)."""
    errs = torch.zeros(1, dtype=torch.int64, device=H.device)
    for f in sorted(set(fmts.tolist())):
        idx = torch.as_tensor(np.nonzero(fmts == f)[0], device=H.device)
        sub = {k: v[idx] for k, v in d.items() if torch.is_tensor(v) and v.dim() >= 1 and v.shape[0] == H.shape[0]}
        prec = F.precision(w="fp64") if f == "fp64" else F.precision(gram="fp32", mv=f, ip="fp32", w="fp32")
        errs += _errors(H[idx].contiguous(), sub, iters, prec, L)
    return errs


def exp_time_varying(trials, zeta=0.8, snrs=tuple(range(0, 31, 4)), iters=10, fd_hz=1000.0, tau_s=0.5e-3,
                     steps=8, device="cuda"):
    """First-order Gauss-Markov channel over `steps` coherence intervals: the
    heuristic's format chosen once from E{kappa} (footnote of Section III-B)
    against the format chosen per system from its own kappa."""
    a = wl.doppler_corr(fd_hz, tau_s)
    c = math.sqrt(max(0.0, 1.0 - a * a))
    res = {"heuristic_once": [], "per_system": [], "lmmse": []}
    kap0 = float(np.mean(kappa_sample(_spec(zeta, seed=16))["kappa"]))
    fmt_once, _ = F.fpcg_choose_precision(K_STREAMS, kap0)
    per = max(1, trials // steps)
    for snr in snrs:
        spec = _spec(zeta, snr_db=snr, seed=16)
        e_once = torch.zeros(1, dtype=torch.int64, device=device)
        e_per = torch.zeros(1, dtype=torch.int64, device=device)
        e_lm = torch.zeros(1, dtype=torch.int64, device=device)
        H = None
        for i in range(steps):
            w = wl.generate_torch(spec, 1000 + i, per, device=device)
            H = w["H"] if H is None else a * H + c * w["H"]
            d = wl.generate_torch(spec, 2000 + i, per, device=device, h_true=H)
            A = torch.empty((per, K_STREAMS, K_STREAMS), dtype=torch.complex128, device=device)
            b = torch.empty((per, K_STREAMS), dtype=torch.complex128, device=device)
            F.fpcg_gram(H, d["y"], d["sigma2"], "fp64", A, b)
            ev = torch.linalg.eigvalsh(A)
            kap = (ev[:, -1] / ev[:, 0]).cpu().numpy()
            fmts = np.array([F.fpcg_choose_precision(K_STREAMS, float(k))[0] for k in kap])
            e_per += _detect_by_format(H, d, iters, fmts, L_BJ)
            e_once += _errors(H, d, iters, prec_of(fmt_once) if fmt_once != "fp64" else prec_of("cg64"), L_BJ)
            e_lm += _errors(H, d, 2 * K_STREAMS, prec_of("lmmse"), None)
        tot = per * steps * _bits_per_system()
        res["heuristic_once"].append(int(e_once.item()) / tot)
        res["per_system"].append(int(e_per.item()) / tot)
        res["lmmse"].append(int(e_lm.item()) / tot)
    return {"experiment": "time_varying", "figure": "Fig. ber_time", "zeta": zeta, "iters": iters, "fd_hz": fd_hz,
            "tau_s": tau_s, "rho_tau": a, "steps": steps, "format_once": fmt_once, "mean_kappa": kap0,
            "snr_db": list(snrs), "ber": res}


def exp_users(trials, zeta=0.8, iters=range(1, 21)):
    """Multi-antenna users: Assumption 1 (no correlation between users) against
    eq. 2's R_t over all streams; FP-BJ-CG with blocks of two users."""
    res = {}
    for name, blk in (("assumption1", True), ("full_rt", False)):
        spec = _spec(zeta, seed=17, rt_block=blk)
        r = ber_curves(spec, [("cg64", None), ("fp16", None), ("fp16", L_BJ)], list(iters), trials)
        k = kappa_sample(spec, bj_L=L_BJ)
        r.update(mean_kappa=float(np.mean(k["kappa"])), mean_kappa_bar=float(np.mean(k["kappa_bar"])),
                 frac_kappa_bar_below=float(np.mean(k["kappa_bar"] < k["kappa"])))
        r["iterations_to_lmmse"] = {kk: iterations_to_lmmse(v, r["lmmse"]) for kk, v in r["curves"].items()}
        res[name] = r
    return {"experiment": "users", "section": "Section IV-B, Assumption 1, Theorem 5", "zeta": zeta, "results": res}


EXPERIMENTS = {"mv_ip": exp_mv_ip, "heuristic": exp_heuristic, "convergence": exp_convergence,
               "ber_snr": exp_ber_snr, "csi": exp_csi, "time_varying": exp_time_varying, "users": exp_users}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("names", nargs="+", help="experiments to run, or 'all': " + ", ".join(EXPERIMENTS))
    ap.add_argument("--trials", type=int, default=100000, help="systems per point (the paper: 500000)")
    ap.add_argument("--out", default=None, help="append the JSON lines to this file as well")
    a = ap.parse_args(argv)
    F.lib()
    names = list(EXPERIMENTS) if a.names == ["all"] else a.names
    for n in names:
        t0 = time.time()
        r = EXPERIMENTS[n](a.trials)
        torch.cuda.synchronize()
        r["trials_per_point"] = a.trials
        r["seconds"] = round(time.time() - t0, 2)
        line = json.dumps(r)
        print(line, flush=True)
        if a.out:
            with open(a.out, "a") as f:
                f.write(line + "\n")
    return 0


if __name__ == "__main__":
    sys.exit(main())
