"""Serving loop: slot-sized detection requests admitted by device memory, run
concurrently on CUDA streams, with per-request latency.

A request is one slot of one user group: 14 OFDM symbols x S subcarriers seen
through one channel per 12-subcarrier resource block, so the 168 received
vectors of a block share a Gram matrix.  On the device a request runs
  copies in -> fpcg_gram (one A + sigma^2 I per block, kept for the whole slot)
  -> fpcg_detect_grouped (every received vector against its block's A; the
     vectors are stored block by block) -> copies out
on a stream of its own.  Requests that arrive while others run are admitted
as soon as a stream and enough of the memory budget are free (continuous
batching: their work overlaps on the GPU); the rest wait in arrival order.
Latency is measured on the host from a request's arrival to the moment its
results are in host memory (its completion event is polled).

With gram_max_age > 0 the server also keeps Gram matrices across slots:
requests that carry a channel key (one user group's channel, aged by the
Gauss-Markov model of Section V-C from slot to slot) reuse the channel
estimate and the Gram matrices formed for an earlier slot of that key while
it is at most gram_max_age slots old, so such a slot is only copies in,
matched filters and solves; an older (or first) slot forms and keeps new ones.

Everything the detection computes runs in libfpcg's kernels; this module
moves bytes and keeps time.
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import fpcg as F

SYMBOLS_PER_SLOT = 14
SUBCARRIERS_PER_RB = 12


class Arena:
    """First-fit allocator over a fixed byte range (the memory budget).
    Offsets and sizes are multiples of `align` bytes."""

    def __init__(self, size, align=256):
        self.size = int(size) // align * align
        self.align = align
        self.free_list = [(0, self.size)]   # sorted, coalesced (offset, length)
        self.used = 0

    def alloc(self, nbytes):
        n = -(-int(nbytes) // self.align) * self.align
        for i, (off, ln) in enumerate(self.free_list):
            if ln >= n:
                if ln == n:
                    self.free_list.pop(i)
                else:
                    self.free_list[i] = (off + n, ln - n)
                self.used += n
                return off, n
        return None

    def free(self, off, n):
        self.used -= n
        fl = self.free_list
        i = 0
        while i < len(fl) and fl[i][0] < off:
            i += 1
        fl.insert(i, (off, n))
        # coalesce with the neighbours
        if i + 1 < len(fl) and fl[i][0] + fl[i][1] == fl[i + 1][0]:
            fl[i] = (fl[i][0], fl[i][1] + fl[i + 1][1])
            fl.pop(i + 1)
        if i > 0 and fl[i - 1][0] + fl[i - 1][1] == fl[i][0]:
            fl[i - 1] = (fl[i - 1][0], fl[i - 1][1] + fl[i][1])
            fl.pop(i)


@dataclass
class Request:
    """One slot: host (pinned) inputs and outputs, and its timeline."""
    rid: int
    N: int
    K: int
    S: int                      # subcarriers
    arrival: float              # seconds from the start of the run
    H: torch.Tensor             # [n_rb][K][N] complex64
    y: torch.Tensor             # [n_re][N] complex64, resource-block-major
    rb: torch.Tensor            # [n_re] int32
    start: torch.Tensor         # [n_rb + 1] int64: received vectors of block g are [start[g], start[g+1])
    sigma2: torch.Tensor        # [n_rb] float64
    qam: torch.Tensor           # [n_re] int32
    tx: torch.Tensor = None     # [n_re][K] uint8 (optional: bit errors)
    key: object = None          # channel key (Gram reuse across slots); None: not kept
    slot_index: int = 0         # slot number of this request's channel estimate
    out: dict = field(default_factory=dict)
    admitted: float = None
    done: float = None
    reused: bool = False        # detected against a kept Gram of an earlier slot
    keep: list = field(default_factory=list)  # device tensors the in-flight work reads

    @property
    def n_rb(self):
        return self.H.shape[0]

    @property
    def n_re(self):
        return self.y.shape[0]

    def latency(self):
        return None if self.done is None else self.done - self.arrival


def request_layout(n_rb, n_re, N, K):
    """(name, dtype, shape) of every device buffer of a request, in order."""
    return [("H", torch.complex64, (n_rb, K, N)), ("y", torch.complex64, (n_re, N)),
            ("rb", torch.int32, (n_re,)), ("start", torch.int64, (n_rb + 1,)), ("sigma2", torch.float64, (n_rb,)),
            ("qam", torch.int32, (n_re,)), ("tx", torch.uint8, (n_re, K)),
            ("A", torch.complex64, (n_rb, K, K)), ("b", torch.complex64, (n_rb, K)),
            ("x", torch.complex64, (n_re, K)), ("sym", torch.uint8, (n_re, K)),
            ("rel", torch.float64, (n_re,)), ("st", torch.int32, (n_re,)),
            ("bits", torch.int64, (1,))]


def _nbytes(dt, shape):
    return int(np.prod(shape)) * torch.empty((), dtype=dt).element_size()


def request_bytes(n_rb, n_re, N, K, align=256):
    return sum(-(-_nbytes(dt, sh) // align) * align for _, dt, sh in request_layout(n_rb, n_re, N, K))


class Server:
    """Runs requests on `n_streams` streams inside a device memory budget."""

    def __init__(self, budget_bytes, n_streams=4, iters=6, block_L=8, prec=None, device="cuda",
                 max_rb_n=275 * 512, gram_max_age=0):
        F.lib()
        self.dev = torch.device(device)
        self.arena = Arena(budget_bytes)
        self.mem = torch.empty(self.arena.size, dtype=torch.uint8, device=self.dev)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(n_streams)]
        self.iters = iters
        self.block_L = block_L
        self.prec_kw = prec or dict(gram="bf16", mv="fp16", refine_steps=1)
        self.prec = F.precision(**self.prec_kw)
        # fpcg_gram also forms b for one y per system; the Gram is all a slot needs
        self.zero_y = torch.zeros(max_rb_n, dtype=torch.complex64, device=self.dev)
        self.gram_max_age = int(gram_max_age)
        self.kept = {}   # key -> dict(H, A, b, slot, shape, ready event): kept outside the budget

    def _views(self, off, req):
        v, pos = {}, off
        for name, dt, sh in request_layout(req.n_rb, req.n_re, req.N, req.K):
            nb = _nbytes(dt, sh)
            v[name] = self.mem[pos:pos + nb].view(dt).view(sh)
            pos += -(-nb // 256) * 256
        return v

    def _kept_gram(self, req, v, stream):
        """The channel estimate and Gram matrices this request detects with: a
        kept entry of its key while young enough, else new ones formed on
        `stream` (and kept when the request has a key)."""
        shape = (req.n_rb, req.K, req.N)
        ent = self.kept.get(req.key) if (self.gram_max_age > 0 and req.key is not None) else None
        if ent is not None and ent["shape"] == shape and 0 <= req.slot_index - ent["slot"] <= self.gram_max_age:
            stream.wait_event(ent["ready"])   # formed on another stream, maybe
            req.reused = True
            req.keep = [ent["H"], ent["A"]]
            for t in req.keep:
                t.record_stream(stream)
            return ent["H"], ent["A"]
        if self.gram_max_age > 0 and req.key is not None:
            # a new entry (tensors of an older one stay alive while requests still read them)
            H = torch.empty(shape, dtype=torch.complex64, device=self.dev)
            A = torch.empty((req.n_rb, req.K, req.K), dtype=torch.complex64, device=self.dev)
            b = torch.empty((req.n_rb, req.K), dtype=torch.complex64, device=self.dev)
        else:
            H, A, b = v["H"], v["A"], v["b"]
        H.copy_(req.H, non_blocking=True)
        zy = self.zero_y[:req.n_rb * req.N].view(req.n_rb, req.N)
        F.fpcg_gram(H, zy, v["sigma2"], self.prec_kw["gram"], A, b, stream=stream)
        if H is not v["H"]:
            ev = torch.cuda.Event()
            ev.record(stream)
            self.kept[req.key] = {"H": H, "A": A, "b": b, "slot": req.slot_index, "shape": shape, "ready": ev}
            req.keep = [H, A]
        return H, A

    def _issue(self, req, stream, off):
        v = self._views(off, req)
        with torch.cuda.stream(stream):
            for k in ("y", "rb", "start", "sigma2", "qam"):
                v[k].copy_(getattr(req, k), non_blocking=True)
            if req.tx is not None:
                v["tx"].copy_(req.tx, non_blocking=True)
            H, A = self._kept_gram(req, v, stream)
            L = min(self.block_L, req.K) if self.block_L else 0
            F.fpcg_detect_grouped(A, H, v["y"], v["start"], v["qam"], self.iters, L, self.prec, v["x"],
                                  sym_idx=v["sym"], rel_res=v["rel"],
                                  tx_idx=v["tx"] if req.tx is not None else None,
                                  bit_errors=v["bits"] if req.tx is not None else None,
                                  status=v["st"], stream=stream)
            for k in ("x", "sym", "rel", "st", "bits"):
                req.out[k].copy_(v[k], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev

    def prepare(self, req):
        """Pinned host outputs for a request (outside the timed loop)."""
        req.out = {"x": torch.empty((req.n_re, req.K), dtype=torch.complex64).pin_memory(),
                   "sym": torch.empty((req.n_re, req.K), dtype=torch.uint8).pin_memory(),
                   "rel": torch.empty(req.n_re, dtype=torch.float64).pin_memory(),
                   "st": torch.empty(req.n_re, dtype=torch.int32).pin_memory(),
                   "bits": torch.zeros(1, dtype=torch.int64).pin_memory()}

    def run(self, requests, poll_s=20e-6):
        """Serve `requests` (arrival times in seconds from now).  Returns them
        with admitted/done times filled in."""
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            if not r.out:
                self.prepare(r)
            need = request_bytes(r.n_rb, r.n_re, r.N, r.K)
            if need > self.arena.size:
                raise ValueError(f"request {r.rid} needs {need} bytes, more than the budget")
        queue, inflight = [], []          # inflight: (req, stream, event, (off, n))
        free_streams = list(self.streams)
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        i = 0
        while i < len(pending) or queue or inflight:
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i].arrival <= now:
                queue.append(pending[i])
                i += 1
            # admission in arrival order while a stream and memory are free
            while queue and free_streams:
                r = queue[0]
                blk = self.arena.alloc(request_bytes(r.n_rb, r.n_re, r.N, r.K))
                if blk is None:
                    break
                queue.pop(0)
                s = free_streams.pop(0)
                r.admitted = time.perf_counter() - t0
                inflight.append((r, s, self._issue(r, s, blk[0]), blk))
            progressed = False
            for item in list(inflight):
                r, s, ev, blk = item
                if ev.query():
                    r.done = time.perf_counter() - t0
                    self.arena.free(*blk)
                    free_streams.append(s)
                    inflight.remove(item)
                    progressed = True
            if not progressed:
                nxt = pending[i].arrival - (time.perf_counter() - t0) if i < len(pending) else poll_s
                time.sleep(max(0.0, min(poll_s, nxt)))
        return requests


def pin_slot(base):
    """Pinned host tensors of a pre-drawn full-size slot (workload.generate_rb
    output with 168 received vectors per block)."""
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return {"N": base["N"], "K": base["K"], "H": t(base["H"]), "y": t(base["y"]), "rb": t(base["rb_index"]),
            "sigma2": t(base["sigma2"]), "qam": t(base["qam"]), "tx": t(base["tx"])}


def slot_request(rid, pinned, S, arrival):
    """A request of S subcarriers: the first ceil(S/12) blocks and the first
    14 S received vectors of a pinned full-size slot (views, no copies)."""
    n_rb = math.ceil(S / SUBCARRIERS_PER_RB)
    n_re = SYMBOLS_PER_SLOT * S
    per = SYMBOLS_PER_SLOT * SUBCARRIERS_PER_RB
    start = torch.from_numpy(np.minimum(np.arange(n_rb + 1, dtype=np.int64) * per, n_re)).pin_memory()
    return Request(rid=rid, N=pinned["N"], K=pinned["K"], S=S, arrival=arrival, H=pinned["H"][:n_rb],
                   y=pinned["y"][:n_re], rb=pinned["rb"][:n_re], start=start, sigma2=pinned["sigma2"][:n_rb],
                   qam=pinned["qam"][:n_re], tx=pinned["tx"][:n_re])


def percentile(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None
