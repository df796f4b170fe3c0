"""Serving: continuous batching of pattern queries over one resident text.

Queries (pattern, k) arrive over time.  The server admits queued queries into
a batch whenever a slot (a CUDA stream) is free and the batch's projected
device memory fits the budget; batches are issued without waiting, so those
in different slots run concurrently on the GPU, and queries that arrive
while others run are admitted as soon as a slot and memory free up.  A batch
mixes queries of any m and k in one search call: one scan launch per query,
or one persistent launch for the whole batch (``GpuBackend(batch=...)``).

Memory admission uses a per-query projection of the output size: the
expected number of windows with at most k mismatches, from a Poisson-
binomial model of the per-position mismatch probability (the letter
frequencies the resident text was measured to have when it was coded; a
class position mismatches with the probability of the letters outside it),
padded by a margin.  A query that still overflows its share is re-run alone
with its exact count, which the first run reports.  Latency is completion
minus arrival, where completion is the moment the query's hits are in the
caller's memory (host memory with ``GpuBackend(copy_to_host=True)``, the
device buffers otherwise); results are identical to a search of the query
alone (the kernels are deterministic and queries never interact).

The backend is pluggable: ``GpuBackend`` issues pm_search_ex calls on the
slots' streams; tests may drive the scheduling logic with a CPU stand-in.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np

# letter frequencies (A, C, G, T) assumed when the text's own are not given:
# a genome at 41 % GC
LETTER_P = {"A": 0.295, "C": 0.205, "G": 0.205, "T": 0.295}


def letter_freqs(counts) -> dict:
    """Letter frequencies from a text's letter counts (A, C, G, T order, as
    pm_text_letter_counts gives them)."""
    tot = float(sum(counts))
    if tot <= 0:
        return dict(LETTER_P)
    return {a: c / tot for a, c in zip("ACGT", counts)}
CLASS_LETTERS = {
    "A": "A", "C": "C", "G": "G", "T": "T", "M": "AC", "R": "AG", "W": "AT", "S": "CG",
    "Y": "CT", "K": "GT", "V": "ACG", "H": "ACT", "D": "AGT", "B": "CGT", "N": "ACGT",
}


def _binomial_head(c: int, q: float, k: int) -> list[float]:
    """P[Binomial(c, q) = i] for i = 0..k (log space, so (1-q)^c may underflow
    to 0 without a NaN)."""
    if q <= 0.0:
        return [1.0] + [0.0] * k
    if q >= 1.0:
        return [1.0 if i == c else 0.0 for i in range(k + 1)]
    lq, lp = math.log(q), math.log1p(-q)
    out = []
    for i in range(k + 1):
        if i > c:
            out.append(0.0)
            continue
        lg = math.lgamma(c + 1) - math.lgamma(i + 1) - math.lgamma(c - i + 1)
        out.append(math.exp(lg + i * lq + (c - i) * lp))
    return out


def expected_hits(pattern: str, k: int, n: int, freqs: dict | None = None) -> float:
    """Expected number of windows with at most k mismatches.

    The count of a window is a sum of independent per-position mismatch
    indicators (a Poisson binomial); positions of the same class share one
    probability, so the distribution's head (counts 0..k) is the truncated
    convolution of one binomial per class present.  Costs O(classes * k^2)
    instead of O(m * k): it runs once per submitted query, on the host thread
    that also feeds the GPU."""
    f = freqs or LETTER_P
    m = len(pattern)
    if m > n:
        return 0.0
    if k >= m:
        return float(n - m + 1)
    dist = [1.0] + [0.0] * k
    for ch, c in collections.Counter(pattern.upper()).items():
        q = 1.0 - sum(f[a] for a in CLASS_LETTERS.get(ch, ""))
        b = _binomial_head(c, q, k)
        dist = [sum(dist[j] * b[i - j] for j in range(i + 1)) for i in range(k + 1)]
    return float((n - m + 1) * sum(dist))


def capacity_for(pattern: str, k: int, n: int, freqs: dict | None = None) -> int:
    """Output records to reserve for one query.  The model ignores the
    text's neighbour correlations (CpG depletion, order-2 context), which
    move short patterns' counts by tens of percent, so the margin is wide:
    device memory is cheaper than re-running a batch whose output did not
    fit."""
    e = expected_hits(pattern, k, n, freqs)
    return int(2.0 * e + 16.0 * math.sqrt(e) + 4096)


@dataclass
class Request:
    qid: int
    pattern: str
    k: int
    arrival: float                  # seconds on the server clock
    capacity: int = 0
    start: float | None = None      # issued to the device
    done: float | None = None       # results available
    hits: object = None             # backend-specific (locations, mismatches)
    count: int = -1
    retries: int = 0
    deadline: float | None = None   # server clock; expires if not started by then
    status: str = "queued"          # queued, running, done, cancelled, expired

    @property
    def latency(self) -> float:
        return (self.done - self.arrival) if self.done is not None else float("nan")


@dataclass
class _Flight:
    slot: int
    reqs: list
    handle: object
    nbytes: int


class Server:
    """Continuous-batching scheduler (see the module docstring)."""

    def __init__(self, backend, n: int, slots: int = 3, max_batch: int = 64,
                 mem_budget: int = 8 << 30, clock=time.perf_counter, freqs: dict | None = None,
                 on_result=None, keep_hits: bool = True):
        """freqs: the text's letter frequencies for the admission model
        (default: the backend's ``letter_freqs()`` if it has one, else a
        genome at 41 % GC).  on_result: called with each completed Request
        (hits attached) as soon as it completes.  keep_hits False: the server
        lets go of a request's hits once on_result has seen them and hands the
        batch's buffers back to the backend for reuse (``release``), so the
        hits are valid during on_result only (copy what must outlive it);
        ``done`` then keeps counts and times only."""
        self.backend = backend
        self.n = n
        if freqs is None and hasattr(backend, "letter_freqs"):
            freqs = backend.letter_freqs()
        self.freqs = freqs
        self.max_batch = max_batch
        self.mem_budget = mem_budget
        self.clock = clock
        self.t0 = clock()
        self.queue: collections.deque[Request] = collections.deque()
        self.free_slots = list(range(slots))
        self.flights: list[_Flight] = []
        self.done: list[Request] = []
        self.cancelled: list[Request] = []
        self.expired: list[Request] = []
        self.inflight_bytes = 0
        self._next = 0
        self.batches = 0
        self.max_inflight = 0
        self.on_result = on_result
        self.keep_hits = keep_hits

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, pattern: str, k: int, arrival: float | None = None,
               timeout: float | None = None) -> Request:
        """Queue a query.  timeout: seconds after arrival by which it must
        have started, else it expires unanswered."""
        r = Request(self._next, pattern, int(k), self.now() if arrival is None else arrival)
        r.capacity = capacity_for(pattern, k, self.n, self.freqs)
        if timeout is not None:
            r.deadline = r.arrival + timeout
        self._next += 1
        self.queue.append(r)
        return r

    def cancel(self, r: Request) -> bool:
        """Withdraw a query: a queued one never starts; a running one's
        results are dropped when its batch finishes.  False if it already
        finished (or was withdrawn)."""
        if r.status == "queued":
            self.queue.remove(r)
            r.status = "cancelled"
            self.cancelled.append(r)
            return True
        if r.status == "running":
            r.status = "cancelled"
            return True
        return False

    def _expire(self) -> None:
        now = self.now()
        if not any(r.deadline is not None and r.deadline < now for r in self.queue):
            return
        keep = collections.deque()
        for r in self.queue:
            if r.deadline is not None and r.deadline < now:
                r.status = "expired"
                self.expired.append(r)
            else:
                keep.append(r)
        self.queue = keep

    def _admit(self) -> list[Request]:
        batch, nbytes = [], 0
        while self.queue and len(batch) < self.max_batch:
            r = self.queue[0]
            b = self.backend.bytes_for([r], self.n)
            if batch and self.inflight_bytes + nbytes + b > self.mem_budget:
                break
            if not batch and self.flights and self.inflight_bytes + b > self.mem_budget:
                break  # wait for memory to free up
            batch.append(self.queue.popleft())
            nbytes += b
        return batch

    def step(self) -> int:
        """Harvest finished batches, then issue as many new ones as slots and
        memory allow.  Returns the number of queries completed."""
        finished = 0
        still = []
        for f in self.flights:
            if self.backend.ready(f.handle):
                counts, hits = self.backend.collect(f.handle, f.reqs)
                t = self.now()
                if any(h is None for h in hits):
                    # the batch's output did not fit (nothing was written): run
                    # its queries again, each with at least its exact count
                    for r, c in reversed(list(zip(f.reqs, counts))):
                        if r.status == "cancelled":
                            self.cancelled.append(r)
                            continue
                        r.capacity, r.retries = max(r.capacity, c), r.retries + 1
                        r.status = "queued"
                        self.queue.appendleft(r)
                    if hasattr(self.backend, "release"):
                        self.backend.release(f.handle)  # nothing was handed out
                else:
                    for r, c, h in zip(f.reqs, counts, hits):
                        if r.status == "cancelled":
                            self.cancelled.append(r)
                            continue
                        r.count, r.hits, r.done, r.status = c, h, t, "done"
                        if self.on_result is not None:
                            self.on_result(r)
                        if not self.keep_hits:
                            r.hits = None
                        self.done.append(r)
                        finished += 1
                    if not self.keep_hits and hasattr(self.backend, "release"):
                        self.backend.release(f.handle)
                self.free_slots.append(f.slot)
                self.inflight_bytes -= f.nbytes
            else:
                still.append(f)
        self.flights = still
        self._expire()
        while self.free_slots and self.queue:
            batch = self._admit()
            if not batch:
                break
            slot = self.free_slots.pop()
            t = self.now()
            for r in batch:
                r.start, r.status = t, "running"
            nbytes = self.backend.bytes_for(batch, self.n)
            handle = self.backend.launch(batch, slot)
            self.flights.append(_Flight(slot, batch, handle, nbytes))
            self.inflight_bytes += nbytes
            self.batches += 1
            self.max_inflight = max(self.max_inflight, len(self.flights))
        return finished

    def idle(self) -> bool:
        return not self.queue and not self.flights

    def drain(self, poll: float = 0.0) -> None:
        while not self.idle():
            if self.step() == 0 and poll:
                time.sleep(poll)


def run_trace(server: Server, queries, poll: float = 0.0002) -> dict:
    """Replay a list of (arrival seconds, pattern, k) on the server's clock in
    real time, then drain.  Returns throughput (all queries over the whole
    span, start-up and drain included; and the steady-state completion rate
    over the last nine tenths of the arrival period), latency percentiles and
    the queue depth (queries waiting for a slot), time-weighted over the
    arrival period and at its peak."""
    queries = sorted(queries, key=lambda q: q[0])
    i = 0
    t_start = server.now()
    t_prev, depth_area, depth_max = 0.0, 0.0, 0
    t_arrivals_end = queries[-1][0] if queries else 0.0
    while i < len(queries) or not server.idle():
        now = server.now() - t_start
        while i < len(queries) and queries[i][0] <= now:
            a, p, k = queries[i]
            server.submit(p, k, arrival=t_start + a)
            i += 1
        if now <= t_arrivals_end:
            depth_area += len(server.queue) * (now - t_prev)
            depth_max = max(depth_max, len(server.queue))
            t_prev = now
        if server.step() == 0 and poll:
            time.sleep(poll)
    t_end = server.now()
    lat = np.array([r.latency for r in server.done])
    span = t_end - t_start
    # completion rate in steady state: queries completed between the end of
    # the first tenth of the arrival period and its end, per second of that
    # interval (no start-up, no drain)
    w0, w1 = t_start + 0.1 * t_arrivals_end, t_start + t_arrivals_end
    in_window = sum(1 for r in server.done if r.done is not None and w0 <= r.done < w1)
    return {
        "completed": len(server.done),
        "offered_qps": len(queries) / max(queries[-1][0], 1e-9) if queries else 0.0,
        "throughput_qps": len(server.done) / span if span > 0 else 0.0,
        "steady_qps": in_window / (w1 - w0) if w1 > w0 else 0.0,
        "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
        "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
        "span_s": span,
        "batches": server.batches,
        "max_concurrent_batches": server.max_inflight,
        "retries": sum(r.retries for r in server.done),
        "cancelled": len(server.cancelled),
        "expired": len(server.expired),
        "queue_depth_mean": depth_area / t_prev if t_prev > 0 else 0.0,
        "queue_depth_max": depth_max,
    }


class GpuBackend:
    """Issues each batch as one asynchronous pm_search_ex call on its slot's
    stream (device outputs, scratch from the stream-ordered pool): one scan
    launch per query, or with ``batch`` (batch options, {} for defaults) one
    persistent launch for the whole batch.

    Each batch's offsets follow its search on the slot's stream into pinned
    memory, so the host reads them without waiting on other work.

    copy_to_host: deliver each query's hits in pinned host memory.  Once a
    batch's search has finished, one asynchronous copy of the batch's hits
    into a pinned buffer is queued on the slot's stream; the batch completes
    when that copy has landed, so latency includes the copy to the caller.
    Otherwise the hits stay on the device and a batch completes with its
    search."""

    def __init__(self, text, slots: int = 3, copy_to_host: bool = False, batch: dict | None = None):
        import torch
        from . import api
        self.api = api
        self.torch = torch
        self.text = text
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.copy_to_host = copy_to_host
        self.batch = batch
        self._compiled: dict[str, object] = {}
        self._free: dict[int, list] = {}  # pinned buffers by size (bytes), for reuse

    def letter_freqs(self) -> dict:
        """The resident text's letter frequencies (measured when it was coded)."""
        return letter_freqs(self.text.letter_counts())

    def _pattern(self, p: str):
        c = self._compiled.get(p)
        if c is None:
            c = self.api.pm_compile_pattern(p)
            self._compiled[p] = c
        return c

    def _pinned(self, nbytes: int):
        """A page-locked host buffer (uint8) of at least nbytes: a released one
        of the same power-of-two size when there is one, else a new one
        (pinning pages takes the host thread milliseconds per large buffer)."""
        size = 1 << 16
        while size < nbytes:
            size <<= 1
        free = self._free.get(size)
        if free:
            return free.pop()
        return self.torch.empty(size, dtype=self.torch.uint8, pin_memory=True)

    def release(self, handle) -> None:
        """Take back a finished batch's pinned buffers for later batches.  The
        server calls this once the batch's results were delivered and nobody
        holds them any more (Server keep_hits=False), or when the batch's
        output did not fit (nothing was handed out)."""
        for buf in handle[7]:
            self._free.setdefault(buf.numel(), []).append(buf)
        handle[7] = []

    def bytes_for(self, reqs, n: int) -> int:
        cap = sum(r.capacity for r in reqs)
        if self.batch is not None:  # hits, records, sort and ordering scratch
            return 64 * cap + 4096 * len(reqs) + (1 << 20)
        tiles = sum((max(n - len(r.pattern) + 1, 0) + 4095) // 4096 for r in reqs)
        return 16 * cap + 24 * tiles + 4096 * len(reqs)

    def launch(self, reqs, slot: int):
        torch = self.torch
        st = self.streams[slot]
        cap = sum(r.capacity for r in reqs)
        with torch.cuda.stream(st):
            res = self.api.pm_search_ex(self.text, [self._pattern(r.pattern) for r in reqs],
                                        [r.k for r in reqs], capacity=cap, stream=st, sync=False,
                                        batch=self.batch)
            # the offsets follow the search on its stream into pinned memory, so
            # reading them later waits for nothing else on the device
            nb = res.offsets.numel() * res.offsets.element_size()
            obuf = self._pinned(nb)
            off = obuf[:nb].view(res.offsets.dtype)
            off.copy_(res.offsets, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        # [result, search event, capacity, slot, offsets (pinned host), host hits,
        #  copy event, pinned buffers of the batch]
        return [res, ev, cap, slot, off, None, None, [obuf]]

    def ready(self, handle) -> bool:
        res, ev, cap, slot = handle[0], handle[1], handle[2], handle[3]
        if not self.copy_to_host:
            return ev.query()
        if handle[6] is None:
            if not ev.query():
                return False
            off = handle[4].numpy().astype(np.uint64)  # landed with the search
            handle[4] = off
            total = int(off[-1])
            if total > cap or total == 0:
                return True
            torch = self.torch
            st = self.streams[slot]
            hbuf = self._pinned(8 * total)
            handle[7].append(hbuf)
            host = hbuf[:8 * total].view(torch.int32).view(total, 2)
            with torch.cuda.stream(st):
                host.copy_(res.hits[:total], non_blocking=True)
                cev = torch.cuda.Event()
                cev.record(st)
            handle[5], handle[6] = host, cev
            return False
        return handle[6].query()

    def collect(self, handle, reqs):
        res, cap = handle[0], handle[2]
        off = handle[4]
        if not isinstance(off, np.ndarray):
            off = off.numpy().astype(np.uint64)  # landed with the search
        total = int(off[-1])
        counts = [int(off[i + 1] - off[i]) for i in range(len(reqs))]
        if total > cap:
            return counts, [None] * len(reqs)
        src = handle[5] if self.copy_to_host else res.hits
        out = []
        for i in range(len(reqs)):
            if total == 0:
                out.append(src[0:0] if src is not None else res.hits[0:0].cpu())
            else:
                out.append(src[int(off[i]):int(off[i + 1])])
        return counts, out
