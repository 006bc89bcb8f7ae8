"""Serving loop for encrypted linear transformations: continuous batching under
an HBM budget, keys and encoded diagonals resident on the device.

A request is one LT: a ciphertext of a given ring degree and level, multiplied
by one of the resident matrices.  The scheduler (one thread) owns a few CUDA
streams.  Whenever a stream is idle it forms the next batch from the queue
(oldest first, up to `max_batch` requests of one context) as long as the
admitted requests' scratch memory fits the HBM budget next to the resident
keys and diagonals, and queues it with lt_eval_batch.  Requests that arrive
while earlier batches are still on the GPU are admitted into the next batch on
another stream, so their work overlaps on the device.  Completion is detected
with CUDA events; latency is completion time minus arrival time.

Every result is what a separate lt_eval of the same request gives (the batched
schedule is bit-identical to the single one).
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    ctx_key: object          # which context (e.g. log N)
    matrix: object           # binding.Diagonals
    ct: object               # binding.Ciphertext (input, device)
    arrival: float           # time.perf_counter() when it arrived
    split: tuple = None      # chosen at admission
    out: object = None       # binding.Ciphertext (output), set at admission
    done: float = None
    scratch_bytes: int = 0


def scratch_bytes(ctx, level: int, split) -> int:
    """Device scratch one TH-BSGS LT takes at `level` with `split`: digit sets of
    the inner and outer layers, the baby pairs, the giant-step accumulators and
    the transform buffers (upper estimate)."""
    n1, n2, n3 = split
    ext = level + ctx.k
    beta = ctx.beta(level)
    limbs = (n1 + max(n3 - 1, 0)) * beta * ext      # digit sets
    limbs += 2 * n1 * ext + 2 * n3 * ext            # pairs and accumulators
    limbs += (max(n1 - 1, n3 - 1, 1) + 2) * level   # moduli-switch buffers
    return limbs * 8 * ctx.N


@dataclass
class Stats:
    latencies: list = field(default_factory=list)
    completed: int = 0
    batches: int = 0
    max_inflight_bytes: int = 0
    admission_waits: int = 0


class LtServer:
    def __init__(self, contexts: dict, hbm_budget: float = 150e9, resident_bytes: int = 0, streams: int = 4,
                 max_batch: int = 16, poll_s: float = 50e-6):
        self.contexts = contexts
        self.budget = float(hbm_budget)
        self.resident = int(resident_bytes)
        self.max_batch = max_batch
        self.poll_s = poll_s
        self.n_streams = streams
        self._streams = None
        self.queue: collections.deque = collections.deque()
        self.lock = threading.Lock()
        self.inflight: dict = {}          # stream index -> (event, [requests], bytes)
        self.inflight_bytes = 0
        self.stats = Stats()
        self.completed: list = []
        self._split_cache: dict = {}

    # --------------------------------------------------------------- public
    def submit(self, req: Request) -> None:
        with self.lock:
            self.queue.append(req)

    def pending(self) -> int:
        with self.lock:
            return len(self.queue) + sum(len(v[1]) for v in self.inflight.values())

    @property
    def streams(self):
        if self._streams is None:
            import torch
            self._streams = [torch.cuda.Stream() for _ in range(self.n_streams)]
        return self._streams

    def step(self) -> int:
        """One scheduler pass: retire finished batches, then fill idle streams.
        Returns the number of requests launched."""
        self._retire()
        launched = 0
        for si in range(self.n_streams):
            if si in self.inflight:
                continue
            batch = self._take_batch()
            if not batch:
                break
            self._launch(si, batch)
            launched += len(batch)
        return launched

    def drain(self, timeout_s: float = 60.0) -> None:
        t_end = time.perf_counter() + timeout_s
        while self.pending():
            if time.perf_counter() > t_end:
                raise TimeoutError("serving loop did not drain")
            if not self.step():
                time.sleep(self.poll_s)

    # --------------------------------------------------------------- internals
    def _split(self, ctx, level: int, n_diag: int):
        key = (id(ctx), level, n_diag)
        sp = self._split_cache.get(key)
        if sp is None:
            sp = ctx.choose_split("th", level, n_diag)
            self._split_cache[key] = sp
        return sp

    def _take_batch(self) -> list:
        with self.lock:
            if not self.queue:
                return []
            head = self.queue[0]
            ctx = self.contexts[head.ctx_key]
            batch, taken = [], []
            budget_left = self.budget - self.resident - self.inflight_bytes
            for idx, r in enumerate(self.queue):
                if len(batch) >= self.max_batch:
                    break
                if r.ctx_key != head.ctx_key:
                    continue
                sp = self._split(ctx, r.ct.level, r.matrix.n_diag)
                need = scratch_bytes(ctx, r.ct.level, sp) + 16 * r.ct.level * ctx.N
                if need > budget_left:
                    if not batch:
                        self.stats.admission_waits += 1
                    break
                r.split, r.scratch_bytes = sp, need
                budget_left -= need
                batch.append(r)
                taken.append(idx)
            for idx in reversed(taken):
                del self.queue[idx]
            return batch

    def _launch(self, si: int, batch: list) -> None:
        import torch
        ctx = self.contexts[batch[0].ctx_key]
        stream = self.streams[si]
        with torch.cuda.stream(stream):
            for r in batch:
                r.out = ctx.ct_empty(r.ct.level - 1)
            ctx.lt_eval_batch([r.ct for r in batch], [r.matrix for r in batch], algos=["th"] * len(batch),
                              splits=[r.split for r in batch], outs=[r.out for r in batch], stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        nbytes = sum(r.scratch_bytes for r in batch)
        with self.lock:  # pending() may read the in-flight table from a submitting thread
            self.inflight[si] = (ev, batch, nbytes)
            self.inflight_bytes += nbytes
            self.stats.max_inflight_bytes = max(self.stats.max_inflight_bytes, self.inflight_bytes)
            self.stats.batches += 1

    def _retire(self) -> None:
        with self.lock:
            items = list(self.inflight.items())
        for si, (ev, batch, nbytes) in items:
            if ev.query():
                now = time.perf_counter()
                for r in batch:
                    r.done = now
                    self.stats.latencies.append(now - r.arrival)
                    self.completed.append(r)
                self.stats.completed += len(batch)
                with self.lock:
                    self.inflight_bytes -= nbytes
                    del self.inflight[si]


def percentile(xs, p: float) -> float:
    s = sorted(xs)
    if not s:
        return float("nan")
    k = min(len(s) - 1, max(0, int(round(p / 100.0 * (len(s) - 1)))))
    return s[k]


def run_open_loop(server: LtServer, arrivals: list, make_request) -> None:
    """Feed requests at their arrival times (seconds from start) and serve them."""
    t0 = time.perf_counter()
    nxt = 0
    while nxt < len(arrivals) or server.pending():
        now = time.perf_counter() - t0
        while nxt < len(arrivals) and arrivals[nxt] <= now:
            server.submit(make_request(nxt, t0 + arrivals[nxt]))
            nxt += 1
        if not server.step():
            time.sleep(server.poll_s)
