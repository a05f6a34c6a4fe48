"""Benchmark: batched FP-BJ-CG MIMO detection on GB300.

One step = one call of the detector over the whole batch (Gram + matched
filter, block-Jacobi setup, CG, refinement, residual check, slicing, bit-error
count) on synthetic inputs already resident in HBM.  The workload is the
N=256 receive-antenna, K=64 user, 16384-channel Kronecker-correlated
(rho=0.7) 64-QAM case at 18 dB.  The same batch is also run through the plain
fp32 CG comparator, and BER is checked against the fp64 direct LMMSE solve on
a sample.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank detects its own batch (weak scaling); rank 0 prints
one JSON line.
"""
import argparse
import math
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_09820_gb300 import workload as wl  # noqa: E402

METRIC = "detections/s at N=256,K=64 vs FP32 CG at equal BER; p99 latency; % roofline"
# arithmetic of the path: bf16 H and y into the Gram (fp32 accumulation), fp16
# A p (fp32 accumulation), fp32 vectors and scalars
DTYPE = "bf16-gram/fp16-matvec/f32-acc"
UNIT = "detections/s"

# Headline configuration (FP-BJ-CG) and the plain fp32 CG comparator.
HEAD = dict(name="FP-BJ-CG", L=4, iters=7,
            prec=dict(gram="bf16", mv="fp16", ip="fp32", w="fp32", refine_steps=1, refine_iters=7, resid="fp64"))
# The uneven-batch and serving workloads use the head's precisions too: the
# solvers for given Gram matrices (two-pass plan classes, the serving loop's
# grouped detection) form their refinement residual against the fp32 Gram
# matrix, read again from global memory.
SOLVER_PREC = dict(HEAD["prec"])
COMP = dict(name="FP32 plain CG", L=None, iters=20,
            prec=dict(gram="fp32", mv="fp32", ip="fp32", w="fp32", refine_steps=0))
# e4m3 A p (per-block power-of-two scales, fp32 accumulation) with the residual
# against the fp32 Gram: the head's path with the matvec in FP8, 6 + 6
# iterations, block-Jacobi L = 4 and 8.
FP8 = [dict(name=f"FP-BJ-CG e4m3 L={L}", L=L, iters=6,
            prec=dict(gram="bf16", mv="e4m3", ip="fp32", w="fp32", refine_steps=1, refine_iters=6, resid="fp64"))
       for L in (4, 8)]


def comparator_flops(N, K, iters):
    """Floating-point operations of one detection by the fp32 comparator
    (8 per complex multiply-add): the Hermitian half of the Gram matrix and
    the matched filter, then per CG iteration the matvec (K^2 complex
    multiply-adds), two inner products and three axpys (about 24 K)."""
    return 8 * N * K * (K + 1) // 2 + 8 * N * K + iters * (8 * K * K + 24 * K)


def gram_half_flops(N, K):
    """The Hermitian half of one Gram matrix: K (K + 1) / 2 entries of N
    complex multiply-adds."""
    return 8 * N * K * (K + 1) // 2


def simt_peaks(dev):
    """fp32 and fp64 FMA rates of the CUDA cores (fpcg_fma_probe, best of
    three launches timed by CUDA events), TFLOP/s."""
    import torch
    from paper_2504_09820_gb300 import fpcg as F
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {}
    for fp64, name, iters in ((0, "fp32_tflops", 65536), (1, "fp64_tflops", 4096)):
        buf = torch.empty(sms * 8 * 256, dtype=torch.float64 if fp64 else torch.float32, device=dev)
        best = 0.0
        for _ in range(4):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fl = F.fpcg_fma_probe(fp64, iters, buf)
            b.record()
            torch.cuda.synchronize(dev)
            best = max(best, fl / (a.elapsed_time(b) / 1e3) / 1e12)
        out[name] = best
    out["method"] = "fpcg_fma_probe: 8 independent FMA chains per thread, 8 CTAs of 256 threads per SM"
    return out


def workload_spec(rank=0):
    s = wl.c3_kron_256x64()
    s.seed = s.seed + 7919 * rank
    return s


def max_over_ranks(x, dist=None, device=None):
    """The largest x over the ranks of the default process group (x itself
    when there is none): the job's time is its slowest rank's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def job_rate(world, per_rank_units, steps, seconds):
    """Whole-job throughput: the units every rank processed per step, over
    the (slowest rank's) time of `steps` steps."""
    return world * per_rank_units * steps / seconds


def bytes_per_detection(N, K):
    """Algorithmic HBM bytes of one detection: read H and y once, write x_hat
    (c64), labels (u8), rel_res (f64) and status (i32)."""
    return N * K * 8 + N * 8 + K * 8 + K + 8 + 4


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per system of the
# head kernel from an ncu capture of a 2048-system case of this workload, keyed
# by the hash of the head kernel's sources (kernel_source_hash) it was taken
# on; a launch moves the same bytes per system, so it scales with the batch.
# None once the kernel changed.
KERNEL_TRAFFIC = {"ccd6513407ee": 135279.0}


def kernel_source_hash(tu="detect_tc_k64.cu"):
    """sha1 (first 12 hex digits) of the head kernel's translation unit and the
    csrc headers it includes, transitively, in name order."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2504_09820_gb300", "csrc")
    seen, todo = set(), [tu]
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(os.path.join(csrc, f)):
            continue
        seen.add(f)
        with open(os.path.join(csrc, f)) as fh:
            todo += re.findall(r'^#include "([^"/]+)"', fh.read(), re.M)
    h = hashlib.sha1()
    for f in sorted(seen):
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"], "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "src": "fallback"}


class Clocks:
    """Sample the SM clock and the clock-event (throttle) reasons during a
    region, through NVML's read-only queries, every ~2 ms from a thread."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device):
        self.dev = torch_device
        self.samples = []
        self.max_mhz = None
        self.err = None

    def _open(self):
        import ctypes
        import torch
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        uuid = "GPU-" + str(torch.cuda.get_device_properties(self.dev).uuid)
        if nv.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) != 0:
            if nv.nvmlDeviceGetHandleByIndex_v2(self.dev.index, ctypes.byref(h)) != 0:
                raise RuntimeError("no NVML handle")
        fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        mx = ctypes.c_uint()
        if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
            self.max_mhz = mx.value
        return nv, h, fn

    def __enter__(self):
        import ctypes
        import threading
        self.stop = threading.Event()
        try:
            nv, h, fn = self._open()
        except Exception as e:  # no NVML: report the region as unsampled
            self.err = str(e)
            self.t = None
            return self

        def poll():
            mhz, rs = ctypes.c_uint(), ctypes.c_ulonglong()
            while not self.stop.is_set():
                if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0 and fn(h, ctypes.byref(rs)) == 0:
                    self.samples.append((mhz.value, rs.value))
                time.sleep(0.002)
        self.nv = nv
        self.t = threading.Thread(target=poll, daemon=True)
        self.t.start()
        time.sleep(0.01)
        return self

    def __exit__(self, *a):
        if self.t is not None:
            self.stop.set()
            self.t.join()
            self.nv.nvmlShutdown()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"],
                    "samples": 0, "note": self.err}
        reasons = sorted({name for _, r in self.samples for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(m for m, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(self.samples)}


def run_reference(args):
    """The oracle (CPU, float64 numpy) on a bounded sample of the workload."""
    from oracle import detect as D
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec = workload_spec()
    sample = 512
    d = wl.generate(spec, chunks=[0, 1])
    sl = slice(0, sample)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        D.detect(d["H"][sl], d["y"][sl], d["sigma2"][sl], d["qam"][sl], HEAD["iters"], HEAD["prec"], L=HEAD["L"])
        t = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(t)
    tot = sum(times)
    v = sample * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(spec),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{sample} systems of the batch per step, float64 numpy emulation "
                                       f"of the {HEAD['name']} path"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def mixed_measure(dev, steps, warmup, batch=None, both=True, autotune=True):
    """Uneven batch through a plan: every system draws K in {8,...,128}, N = K x
    {2, 4, 8} (at most 512), rho and the QAM order; one CUDA graph of the
    plan's launches (one fused launch for the K in {16, 32, 64} classes, the
    Gram pass and the solver of each two-pass class), kernels chosen by the
    autotuner (autotune=False: the plan's default choice, e.g. for profiling,
    where the profiler distorts the autotuner's timings).
    Returns the measurement as a dict (both: also time it without the graph)."""
    import torch
    from paper_2504_09820_gb300 import fpcg as F
    spec = wl.mixed_kron(batch=batch or 12000)
    d = wl.generate_mixed(spec)
    prec = F.precision(**SOLVER_PREC)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for graph in ((True, False) if both else (True,)):
        plan = F.Plan(d["n"], d["k"], HEAD["iters"], prec, block_L=HEAD["L"], graph=graph)
        g = plan.pack(d["H"], d["y"], d["sigma2"], d["qam"], d["tx"], device=dev)
        o = {"x": torch.zeros(plan.totals[2], dtype=torch.complex64, device=dev),
             "sym": torch.zeros(plan.totals[2], dtype=torch.uint8, device=dev),
             "rel": torch.empty(plan.batch, dtype=torch.float64, device=dev),
             "st": torch.empty(plan.batch, dtype=torch.int32, device=dev),
             "be": torch.zeros(1, dtype=torch.int64, device=dev)}
        t0 = time.perf_counter()
        if autotune:
            plan.autotune(g["H"], g["y"], g["sigma2"], g["qam"], o["x"], o["sym"], o["rel"], o["st"],
                          stream=stream)
        t_tune = time.perf_counter() - t0

        def call():
            plan.run(g["H"], g["y"], g["sigma2"], g["qam"], o["x"], o["sym"], o["rel"], g["tx"], o["be"], o["st"],
                     stream=stream)
        for _ in range(warmup):
            call()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(dev) as clk:
            a.record(stream)
            for _ in range(steps):
                call()
            b.record(stream)
            torch.cuda.synchronize(dev)
        res[graph] = {"t": a.elapsed_time(b) / 1e3 / steps, "tune_s": t_tune, "clocks": clk.summary(),
                      "classes": plan.classes(), "bits": int(o["be"][0]), "status_max": int(o["st"].max())}
        del g, o
        plan.close()
    r = res[True]
    B = spec.batch
    algo = float(sum(bytes_per_detection(int(n), int(k)) for n, k in zip(d["n"], d["k"])))
    pk = peaks()
    achieved = algo / r["t"] / 1e9
    nbits = float(sum(int(k) * int(round(math.log2(q))) for k, q in zip(d["k"], d["qam"])))
    paths = {}
    for c in r["classes"]:
        key = {F.PATH_TENSOR_CORE: "tensor_core", F.PATH_TWO_PASS: "two_pass"}.get(c["path"], "simt")
        paths[key] = paths.get(key, 0) + c["count"]
    # one launch per launch index (the fused classes share one), plus the Gram
    # pass of every two-pass class
    launches = len({c["launch"] for c in r["classes"]}) + sum(c["path"] == F.PATH_TWO_PASS for c in r["classes"])
    out = {"value": B / r["t"], "unit": UNIT, "ms_per_step": 1e3 * r["t"], "steps": steps, "warmup": warmup,
           "workload": f"uneven batch of {B}: K in {spec.ks}, N = K x {spec.ratios} capped at {spec.n_cap}, "
                       f"rho in {spec.rhos}, QAM in {spec.qams}, {spec.snr_db} dB",
           "method": HEAD["name"], "block_L": f"min({HEAD['L']}, K)", "iters": HEAD["iters"], "precision": SOLVER_PREC,
           "classes": len(r["classes"]), "launches_per_step": launches, "systems_per_path": paths,
           "graph": True, "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                       "frac": achieved / pk["hbm_gbs"], "algorithmic_bytes_per_launch": algo},
           "autotune_s": r["tune_s"], "ber_total": r["bits"] / nbits, "status_max": r["status_max"],
           "clocks": r["clocks"],
           "class_table": [{k: c[k] for k in ("n_rx", "k", "block_L", "path", "count")} for c in r["classes"]]}
    if both:
        out["without_graph_ms"] = 1e3 * res[False]["t"]
    return out


def run_mixed(args):
    import torch
    from paper_2504_09820_gb300 import fpcg as F
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    F.lib()
    m = mixed_measure(dev, args.steps, args.warmup, args.batch, autotune=not args.no_autotune)
    print(json.dumps({
        "metric": "detections/s, uneven batch (one CUDA graph; one fused launch for the K in {16, 32, 64} classes)",
        "value": m["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": m["ms_per_step"], "higher_is_better": True, "dtype": DTYPE, "data": "synthetic",
        "config": {"workload": m["workload"], "method": m["method"], "block_L": m["block_L"], "iters": m["iters"],
                   "precision": m["precision"], "classes": m["classes"], "systems_per_path": m["systems_per_path"],
                   "l2": "inputs larger than L2; no flush needed"},
        "roofline": dict(m["roofline"], traffic=None, peak_src=peaks()["src"]),
        "without_graph_ms": m.get("without_graph_ms"), "autotune_s": m["autotune_s"],
        "launches_per_step": m["launches_per_step"], "ber_total": m["ber_total"], "status_max": m["status_max"],
        "clocks": m["clocks"], "class_table": m["class_table"],
    }), flush=True)


def serve_measure(dev, n_req=48, fracs=(0.5, 0.8), sat_runs=3):
    """Serving loop: Poisson arrivals of slot requests (14 symbols x S
    subcarriers, S uniform in 48..3300, one channel per 12-subcarrier block,
    (N, K) uniform in {(64,8), (128,32), (256,64), (512,128)}, rho 0.5, 64-QAM,
    15 dB), admitted by a device memory budget onto 4 streams.  First the
    saturation rate (all requests at t = 0), then p50 / p99 latency at loads
    below it.  Returns the measurement as a dict."""
    from paper_2504_09820_gb300 import serve as SV
    slot_shapes = [(64, 8), (128, 32), (256, 64), (512, 128)]
    slots = {(N, K): SV.pin_slot(wl.generate_rb(wl.RBSpec(N=N, K=K, n_rb=275, rho=0.5, qam=64, snr_db=15.0,
                                                          seed=1005 + K)))
             for N, K in slot_shapes}
    rng = np.random.default_rng(1005)
    kinds = [slot_shapes[i] for i in rng.integers(0, len(slot_shapes), n_req)]
    sizes = rng.integers(48, 3301, n_req).tolist()
    budget = 8 << 30
    srv = SV.Server(budget, n_streams=4, iters=HEAD["iters"], block_L=HEAD["L"], prec=SOLVER_PREC, device=dev)

    def requests(arrivals):
        rs = [SV.slot_request(i, slots[kinds[i]], sizes[i], float(arrivals[i])) for i in range(n_req)]
        for r in rs:
            srv.prepare(r)
        return rs
    n_re = sum(SV.SYMBOLS_PER_SLOT * S for S in sizes)
    # warm-up: one full-size slot of every kind (first launches of every kernel), then one pass
    srv.run([SV.slot_request(i, slots[c], 3300, 0.0) for i, c in enumerate(slot_shapes)])
    srv.run(requests(np.zeros(n_req)))
    with Clocks(dev) as clk:
        spans = []
        for _ in range(sat_runs):                       # median of the saturation runs
            sat = srv.run(requests(np.zeros(n_req)))
            spans.append(max(r.done for r in sat))
    makespan = float(np.median(spans))
    sat_rate = n_req / makespan
    loads = []
    for frac in fracs:
        lam = frac * sat_rate
        arr = np.cumsum(rng.exponential(1.0 / lam, n_req))
        rs = srv.run(requests(arr))
        lat = [1e3 * r.latency() for r in rs]
        span = max(r.done for r in rs) - min(r.arrival for r in rs)
        loads.append({"load_frac_of_saturation": frac, "requests_per_s": lam, "p50_ms": SV.percentile(lat, 50),
                      "p99_ms": SV.percentile(lat, 99), "mean_ms": float(np.mean(lat)),
                      "detections_per_s": n_re / span})
    st_max = max(int(r.out["st"].max()) for r in sat)
    return {"workload": f"{n_req} slot requests: 14 symbols x S subcarriers, S uniform 48..3300, (N,K) uniform in "
                        f"{slot_shapes}, rho 0.5, 64-QAM, 15 dB, one Gram per 12-subcarrier block kept across the slot",
            "method": HEAD["name"], "block_L": f"min({HEAD['L']}, K)", "iters": HEAD["iters"], "precision": SOLVER_PREC,
            "budget_bytes": budget, "streams": 4,
            "path": "fpcg_gram per block + fpcg_detect_grouped (tensor-core solver for K in 8..128)",
            "saturation": {"requests_per_s": sat_rate, "detections_per_s": n_re / makespan, "makespan_s": makespan,
                           "makespans_s": spans, "detections": n_re},
            "loads": loads, "status_max": st_max, "clocks": clk.summary(),
            "timing": "host wall clock from arrival to the result on the host (pinned copies included)"}


def run_serve(args):
    import torch
    from paper_2504_09820_gb300 import fpcg as F
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    F.lib()
    m = serve_measure(dev, args.batch or 48)
    print(json.dumps({
        "metric": "p50/p99 latency and detections/s, serving loop (slot requests, Poisson arrivals)",
        "value": m["loads"][-1]["p99_ms"], "unit": "ms (p99 at 0.8 of saturation)", "higher_is_better": False,
        "n_gpus": 1, "data": "synthetic", "dtype": DTYPE,
        "config": {k: m[k] for k in ("workload", "method", "block_L", "iters", "precision", "budget_bytes", "streams",
                                     "path")},
        "saturation": m["saturation"], "loads": m["loads"], "status_max": m["status_max"], "clocks": m["clocks"],
    }), flush=True)


def oracle_single_core(sample):
    """The same oracle emulation timed on one core: a child process with every
    BLAS / OpenMP pool limited to one thread before numpy loads."""
    import subprocess
    code = ("import sys, time, json; sys.path.insert(0, %r)\n"
            "from bench import HEAD, workload_spec\n"
            "from paper_2504_09820_gb300 import workload as wl\n"
            "from oracle import detect as D\n"
            "d = wl.generate(workload_spec(), chunks=[0, 1])\n"
            "n = %d\n"
            "t0 = time.perf_counter()\n"
            "D.detect(d['H'][:n], d['y'][:n], d['sigma2'][:n], d['qam'][:n], HEAD['iters'], HEAD['prec'], L=HEAD['L'])\n"
            "print(json.dumps({'t': time.perf_counter() - t0}))\n") % (ROOT, sample)
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        t = json.loads(out.stdout.strip().splitlines()[-1])["t"]
    except Exception as e:  # report, do not fail the bench
        return {"value": None, "error": str(e)[:200]}
    return {"value": sample / t, "unit": UNIT, "cores": 1, "sample": f"{sample} systems of the batch"}


def config_dict(spec):
    return {"workload": f"kronecker rho={spec.rho} N={spec.N} K={spec.K} batch={spec.batch} "
                        f"{spec.qam}-QAM {spec.snr_db:g} dB",
            "N": spec.N, "K": spec.K, "batch": spec.batch, "rho": spec.rho, "qam": spec.qam,
            "snr_db": spec.snr_db, "method": HEAD["name"], "block_L": HEAD["L"], "iters": HEAD["iters"],
            "precision": HEAD["prec"], "l2": "inputs (2.2 GB/step) larger than L2 (129 MB); no flush needed",
            "parallelism": "replicas: every rank detects its own batch"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--batch", type=int, default=None, help="override the batch (profiling runs)")
    ap.add_argument("--only-head", action="store_true",
                    help="time only the headline detector (profiling runs; no comparator, BER, e2e)")
    ap.add_argument("--workload", default="kron256x64", choices=["kron256x64", "mixed", "serve"],
                    help="mixed: the uneven batch through a plan; serve: the serving loop "
                         "(each prints its own JSON line)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="--workload mixed: keep the plan's default kernel choice (profiling runs)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the serving and uneven-batch sub-measurements of the headline line")
    ap.add_argument("--breakdown", action="store_true",
                    help="also time the Gram alone and the detector without CG iterations")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "mixed":
        run_mixed(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return

    import torch
    from paper_2504_09820_gb300 import fpcg as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    F.lib()

    spec = workload_spec(rank)
    if args.batch:
        spec.batch = args.batch
    d = wl.generate(spec)
    g = {k: torch.from_numpy(d[k]).to(dev) for k in ("H", "y", "sigma2", "qam", "tx")}
    B, K, N = g["H"].shape
    stream = torch.cuda.current_stream(dev)

    def outputs():
        return {"x": torch.empty((B, K), dtype=torch.complex64, device=dev),
                "sym": torch.empty((B, K), dtype=torch.uint8, device=dev),
                "rel": torch.empty(B, dtype=torch.float64, device=dev),
                "st": torch.empty(B, dtype=torch.int32, device=dev),
                "be": torch.zeros(1, dtype=torch.int64, device=dev)}

    def make_call(cfg, o, src):
        prec = F.precision(**cfg["prec"])

        def call():
            if cfg["L"] is None:
                F.fpcg_detect(src["H"], src["y"], src["sigma2"], src["qam"], cfg["iters"], prec, o["x"],
                              sym_idx=o["sym"], rel_res=o["rel"], tx_idx=src["tx"], bit_errors=o["be"],
                              status=o["st"], stream=stream)
            else:
                F.fpbjcg_detect(src["H"], src["y"], src["sigma2"], src["qam"], cfg["iters"], cfg["L"], prec,
                                o["x"], sym_idx=o["sym"], rel_res=o["rel"], tx_idx=src["tx"],
                                bit_errors=o["be"], status=o["st"], stream=stream)
        return call

    def timed(call, steps, warmup):
        for _ in range(warmup):
            call()
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        start.record(stream)
        for a, b in ev:
            a.record(stream)
            call()
            b.record(stream)
        end.record(stream)
        torch.cuda.synchronize(dev)
        total = max_over_ranks(start.elapsed_time(end) / 1e3, dist, dev)
        per = [a.elapsed_time(b) / 1e3 for a, b in ev]
        return total, per

    o_head = outputs()
    head = make_call(HEAD, o_head, g)
    with Clocks(dev) as clk:
        total, per = timed(head, args.steps, args.warmup)
    clocks = clk.summary()
    det_s = job_rate(world, B, args.steps, total)
    ms_step = 1e3 * total / args.steps
    launch_avg = statistics.mean(per)
    if args.only_head:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": det_s, "unit": UNIT, "ms_per_step": ms_step,
                              "batch": B, "steps": args.steps, "clocks": clocks}), flush=True)
        return
    breakdown = None
    if args.breakdown:
        A = torch.empty((B, K, K), dtype=torch.complex64, device=dev)
        bb = torch.empty((B, K), dtype=torch.complex64, device=dev)

        def gram_only():
            F.fpcg_gram(g["H"], g["y"], g["sigma2"], HEAD["prec"]["gram"], A, bb, stream=stream)
        t_gram, _ = timed(gram_only, max(2, args.steps // 2), 1)
        no_cg = dict(HEAD, iters=0, prec=dict(HEAD["prec"], refine_steps=0))
        t_nocg, _ = timed(make_call(no_cg, outputs(), g), max(2, args.steps // 2), 1)
        n2 = max(2, args.steps // 2)
        breakdown = {"gram_only_ms": 1e3 * t_gram / n2, "detect_without_cg_ms": 1e3 * t_nocg / n2,
                     "detect_ms": ms_step,
                     "gram_only_hbm_frac": B * bytes_per_detection(N, K) / (t_gram / n2) / 1e9 / peaks()["hbm_gbs"]}

    # comparator: plain fp32 CG on the same batch
    o_comp = outputs()
    comp = make_call(COMP, o_comp, g)
    c_total, _ = timed(comp, max(2, args.steps // 2), 1)
    comp_det_s = job_rate(world, B, max(2, args.steps // 2), c_total)
    # its Gram phase alone: the same call with no CG iteration
    comp_gram = make_call(dict(COMP, iters=0), outputs(), g)
    cg_total, _ = timed(comp_gram, 2, 1)
    comp_gram_s = cg_total / 2

    # e4m3 A p on the same batch
    o_fp8 = [outputs() for _ in FP8]
    fp8_t = []
    for cfg, o in zip(FP8, o_fp8):
        t8, _ = timed(make_call(cfg, o, g), max(2, args.steps // 2), 1)
        fp8_t.append(t8 / max(2, args.steps // 2))

    # BER of both paths vs fp64 LMMSE on a sample.  The LMMSE estimate is the
    # library's own fp64 path: CG in fp64 for 2K iterations (exact after K in
    # exact arithmetic), sliced by the same slicer; bit errors counted on the GPU.
    ber = None
    if rank == 0:
        # BER of both paths against the direct LMMSE solve (Section II, eq.
        # inversion) of the oracle on a sample, on the host outside the timed
        # regions: float64 Gram matrix of the stored H, Cholesky solve, slicer.
        from oracle import detect as D
        from oracle import qam as Q
        ns = min(1024, B)
        bps = int(round(math.log2(spec.qam)))
        x_lmmse = D.lmmse(d["H"][:ns], d["y"][:ns], d["sigma2"][:ns])
        e_ref = Q.bit_errors(Q.slice_symbols(x_lmmse, spec.qam, "fp64"), d["tx"][:ns])
        # cross-check: the library's own fp64 path (CG in fp64, 2K iterations)
        ref = {k: g[k][:ns].contiguous() for k in g}
        o_ref = {"x": torch.empty((ns, K), dtype=torch.complex128, device=dev),
                 "sym": torch.empty((ns, K), dtype=torch.uint8, device=dev),
                 "be": torch.zeros(1, dtype=torch.int64, device=dev)}
        F.fpcg_detect(ref["H"], ref["y"], ref["sigma2"], ref["qam"], 2 * K, F.precision(w="fp64"), o_ref["x"],
                      sym_idx=o_ref["sym"], tx_idx=ref["tx"], bit_errors=o_ref["be"], stream=stream)
        torch.cuda.synchronize(dev)
        e_cg64 = int(o_ref["be"][0])
        e_head = Q.bit_errors(o_head["sym"][:ns].cpu().numpy(), d["tx"][:ns])
        e_comp = Q.bit_errors(o_comp["sym"][:ns].cpu().numpy(), d["tx"][:ns])
        nbits = ns * K * bps
        fp8_ber = [Q.bit_errors(o["sym"][:ns].cpu().numpy(), d["tx"][:ns]) / e_ref - 1 for o in o_fp8]
        ber = {"sample_systems": ns, "lmmse": e_ref / nbits, "head": e_head / nbits,
               "comparator": e_comp / nbits, "head_rel_to_lmmse": e_head / e_ref - 1,
               "comparator_rel_to_lmmse": e_comp / e_ref - 1,
               "lmmse_reference": "oracle: float64 Gram of the stored H, Cholesky solve (CPU)",
               "gpu_fp64_cg_rel_to_lmmse": e_cg64 / e_ref - 1,
               "head_full_batch": int(o_head["be"][0]) / (B * K * bps),
               "fp8_rel_to_lmmse": fp8_ber}

    # end to end through the public API from pinned host buffers
    hst = {k: g[k].cpu().pin_memory() for k in g}
    o_e2e = outputs()
    dsrc = {k: torch.empty_like(g[k]) for k in g}
    host_out = {"x": torch.empty((B, K), dtype=torch.complex64).pin_memory(),
                "sym": torch.empty((B, K), dtype=torch.uint8).pin_memory(),
                "rel": torch.empty(B, dtype=torch.float64).pin_memory(),
                "st": torch.empty(B, dtype=torch.int32).pin_memory(),
                "be": torch.empty(1, dtype=torch.int64).pin_memory()}
    head_e2e = make_call(HEAD, o_e2e, dsrc)

    def e2e_step():
        for k in dsrc:
            dsrc[k].copy_(hst[k], non_blocking=True)
        head_e2e()
        for k in host_out:
            host_out[k].copy_(o_e2e[k], non_blocking=True)

    e_steps = max(2, args.steps // 2)
    e_total, _ = timed(e2e_step, e_steps, 1)
    h2d = sum(t.numel() * t.element_size() for t in hst.values())
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # the other two parts of the metric, on this GPU after the headline: p50/p99
    # of the serving loop under Poisson load, and the uneven batch in one graph
    serving = mixed = None
    if not args.no_extra:
        sv = serve_measure(dev, 48, fracs=(0.8,), sat_runs=3)
        serving = {"p50_ms": sv["loads"][0]["p50_ms"], "p99_ms": sv["loads"][0]["p99_ms"],
                   "load_frac_of_saturation": 0.8, "requests_per_s": sv["loads"][0]["requests_per_s"],
                   "detections_per_s": sv["loads"][0]["detections_per_s"],
                   "saturation_detections_per_s": sv["saturation"]["detections_per_s"],
                   "workload": sv["workload"], "precision": sv["precision"], "path": sv["path"],
                   "timing": sv["timing"], "status_max": sv["status_max"], "clocks": sv["clocks"]}
        mx = mixed_measure(dev, 5, 3, both=False)
        mixed = {k: mx[k] for k in ("value", "unit", "ms_per_step", "workload", "precision", "classes",
                                    "launches_per_step", "systems_per_path", "graph", "roofline", "ber_total",
                                    "status_max")}

    sp = simt_peaks(dev)
    fp8 = [{"name": cfg["name"], "iters": [cfg["iters"], cfg["prec"]["refine_iters"]], "value": B / t,
            "unit": UNIT, "ms_per_step": 1e3 * t,
            "ber_rel_to_lmmse": (ber["fp8_rel_to_lmmse"][i] if ber else None)} for i, (cfg, t) in
           enumerate(zip(FP8, fp8_t))]
    pk = peaks()
    algo_bytes = B * bytes_per_detection(N, K)
    tpsys = KERNEL_TRAFFIC.get(kernel_source_hash())
    traffic = tpsys * B if tpsys else None
    achieved = algo_bytes / launch_avg / 1e9
    cpu = None
    if not args.no_cpu:
        from oracle import detect as D
        sample = 4096
        t0 = time.perf_counter()
        D.detect(d["H"][:sample], d["y"][:sample], d["sigma2"][:sample], d["qam"][:sample], HEAD["iters"],
                 HEAD["prec"], L=HEAD["L"])
        t = time.perf_counter() - t0
        cpu = {"value": sample / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{sample} systems of the batch, float64 numpy emulation of the {HEAD['name']} path "
                         f"(BLAS threads = cores)",
               "single_core": oracle_single_core(512)}
    line = {
        "metric": METRIC, "value": det_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE, "data": "synthetic", "config": config_dict(spec),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                     "peak_src": pk["src"], "kernel": "detect (whole path, one launch)",
                     "algorithmic_bytes_per_launch": algo_bytes},
        "cpu_baseline": cpu,
        "e2e": {"value": job_rate(world, B, e_steps, e_total), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "comparator": {"name": COMP["name"], "iters": COMP["iters"], "value": comp_det_s, "unit": UNIT,
                       "speedup_of_head": det_s / comp_det_s,
                       "flops_per_detection": comparator_flops(N, K, COMP["iters"]),
                       "tflops": comparator_flops(N, K, COMP["iters"]) * comp_det_s / 1e12,
                       "gram_phase_ms": 1e3 * comp_gram_s,
                       "gram_tflops": B * gram_half_flops(N, K) / comp_gram_s / 1e12,
                       "gram_frac_of_fp32_peak": B * gram_half_flops(N, K) / comp_gram_s / 1e12 / sp["fp32_tflops"],
                       "gram_at_fp32_peak_ms": 1e3 * B * gram_half_flops(N, K) / (sp["fp32_tflops"] * 1e12),
                       "head_speedup_over_gram_at_fp32_peak":
                           B * gram_half_flops(N, K) / (sp["fp32_tflops"] * 1e12) / (ms_step / 1e3)},
        "simt_peaks": sp, "fp8": fp8,
        "ber": ber, "clocks": clocks, "gpu_launches": args.steps, "breakdown": breakdown,
        "serving": serving, "mixed": mixed,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
