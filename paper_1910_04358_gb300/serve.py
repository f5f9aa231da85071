"""Continuous-batching query server over a resident index.

Requests (2-bit packed sequences) arrive over time.  The engine keeps the
index resident in HBM and a fixed set of slots, each with its own CUDA stream,
page-locked host buffers, device buffers and query workspace.  Whenever a
slot is free it forms the next batch from the requests that have arrived, in
arrival order, bounded by the slot's capacity (queries and bytes) and by an
output-mask memory budget (the answers of all batches in flight must fit it),
copies the batch in, enqueues the query and the copy of the answers back on
the slot's stream, and moves on: batches on different slots overlap on the
device.

Arriving requests are kept in one page-locked arena, each packed at a byte
boundary, in arrival order, so the requests of a batch are one contiguous
span of it: a batch costs one host-to-device copy of its bytes, its
[begin, end) ranges are computed for all of its requests at once, and its
answers are copied from the device straight into their rows of a
page-locked answer array kept in the same order.

`plain_batched` serves the same trace the simple way for comparison: wait
for a fixed number of arrivals, run one batch through the device API, wait
for it, repeat.

Both return per-request answers (bit-identical to querying each request
alone) and latencies (completion time - arrival time).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    packed: np.ndarray     # uint8, bases from bit 0 of byte 0
    n_bases: int
    arrival: float         # seconds from the start of the trace


@dataclass
class ServeResult:
    latency_s: np.ndarray
    answers: np.ndarray    # (requests, W) uint32, by request id
    wall_s: float
    bases: int
    batches: int
    max_in_flight: int
    stats: dict = field(default_factory=dict)

    def summary(self) -> dict:
        lat = self.latency_s * 1e3
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
                "requests": int(lat.size), "batches": self.batches,
                "bp_per_s": self.bases / self.wall_s, "wall_s": self.wall_s,
                "max_in_flight": self.max_in_flight, **self.stats}


class _Trace:
    """A request trace in arrival order, its bytes in one page-locked arena."""

    def __init__(self, requests: list[Request], max_bytes: int):
        import torch
        n = len(requests)
        if sorted(r.rid for r in requests) != list(range(n)):
            raise ValueError("request ids must be 0 .. len(requests) - 1")
        big = [r.rid for r in requests if r.packed.size > max_bytes]
        if big:
            raise ValueError(f"requests {big[:5]} exceed the batch byte limit of {max_bytes}")
        arr = np.array([r.arrival for r in requests], dtype=np.float64)
        self.order = np.argsort(arr, kind="stable")
        self.arrival = arr[self.order]
        self.rid = np.array([requests[i].rid for i in self.order], dtype=np.int64)
        sizes = np.array([requests[i].packed.size for i in self.order], dtype=np.int64)
        self.n_bases = np.array([requests[i].n_bases for i in self.order], dtype=np.int64)
        self.bstart = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(sizes, out=self.bstart[1:])
        self.arena = torch.empty(int(self.bstart[-1]) + 16, dtype=torch.uint8, pin_memory=True)
        if n:
            self.arena.numpy()[: self.bstart[-1]] = np.concatenate([requests[i].packed for i in self.order])
        self.n = n
        self.bases = int(self.n_bases.sum())
        self.answers = None  # page-locked answers in arrival order (set by the server)

    def answer_buffer(self, W: int):
        """Page-locked (n, W) answers in arrival order: each batch's answers
        are copied from the device straight into their rows."""
        import torch
        self.answers = torch.empty((max(self.n, 1), W), dtype=torch.int32, pin_memory=True)
        return self.answers

    def by_request(self) -> np.ndarray:
        """The answers indexed by request id."""
        out = np.empty((self.n, self.answers.shape[1]), dtype=np.uint32)
        out[self.rid] = self.answers.numpy()[: self.n].view(np.uint32)
        return out

    def ranges(self, i0: int, i1: int, begins: np.ndarray, ends: np.ndarray):
        """[begin, end) in bases of requests i0..i1 within their span."""
        b = 4 * (self.bstart[i0:i1] - self.bstart[i0])
        begins[: i1 - i0] = b
        ends[: i1 - i0] = b + self.n_bases[i0:i1]


class _Slot:
    def __init__(self, idx, max_queries: int, max_bytes: int, device):
        import torch
        self.stream = torch.cuda.Stream(device=device)
        self.h_begin = torch.empty(max_queries, dtype=torch.int64, pin_memory=True)
        self.h_end = torch.empty(max_queries, dtype=torch.int64, pin_memory=True)
        self.d_packed = torch.empty(max_bytes + 16, dtype=torch.uint8, device=device)
        self.d_begin = torch.empty(max_queries, dtype=torch.int64, device=device)
        self.d_end = torch.empty(max_queries, dtype=torch.int64, device=device)
        self.d_out = torch.empty((max_queries, idx.W), dtype=torch.int32, device=device)
        ws_bytes = idx.workspace_bytes("seqs", max_queries, max_bytes)
        self.ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        self.ws_ptr = ((base + 255) // 256 * 256, ws_bytes)
        self.event = torch.cuda.Event()
        self.span = (0, 0)     # requests [i0, i1) of the trace in this slot
        self.busy = False

    def launch(self, idx, tr: _Trace, i0: int, i1: int):
        import torch
        n = i1 - i0
        b0, b1 = int(tr.bstart[i0]), int(tr.bstart[i1])
        tr.ranges(i0, i1, self.h_begin.numpy(), self.h_end.numpy())
        with torch.cuda.stream(self.stream):
            self.d_packed[: b1 - b0].copy_(tr.arena[b0:b1], non_blocking=True)
            self.d_begin[:n].copy_(self.h_begin[:n], non_blocking=True)
            self.d_end[:n].copy_(self.h_end[:n], non_blocking=True)
            idx.query_ranges_dev(self.d_packed[: b1 - b0], self.d_begin[:n], self.d_end[:n],
                                 out=self.d_out[:n], stream=self.stream, workspace=self.ws_ptr)
            tr.answers[i0:i1].copy_(self.d_out[:n], non_blocking=True)
            self.event.record(self.stream)
        self.span = (i0, i1)
        self.busy = True


class ServingEngine:
    def __init__(self, idx, slots: int = 4, max_batch_queries: int = 8192,
                 max_batch_bytes: int = 8 << 20, mask_budget_bytes: int = 256 << 20,
                 device: int | None = None):
        import torch
        self.idx = idx
        self.device = torch.device(f"cuda:{idx.device if device is None else device}")
        self.max_q = max_batch_queries
        self.max_bytes = max_batch_bytes
        self.mask_budget = mask_budget_bytes
        self.slots = [_Slot(idx, max_batch_queries, max_batch_bytes, self.device)
                      for _ in range(slots)]

    def _batch_end(self, tr: _Trace, head: int, avail: int, in_flight_mask: int) -> int:
        """Last request (exclusive) of the next batch from the arrived
        requests [head, avail): at least one, then as many as the query and
        byte limits and the output-mask budget allow."""
        row = self.idx.W * 4
        by_mask = (self.mask_budget - in_flight_mask) // row
        cap = max(1, min(self.max_q, by_mask))
        end = min(avail, head + cap)
        by_bytes = int(np.searchsorted(tr.bstart, tr.bstart[head] + self.max_bytes, side="right")) - 1
        return max(head + 1, min(end, by_bytes))

    # -- continuous batching ----------------------------------------------
    def serve(self, requests: list[Request], spin_sleep: float = 20e-6) -> ServeResult:
        tr = _Trace(requests, self.max_bytes)
        tr.answer_buffer(self.idx.W)
        n = tr.n
        done_at = np.zeros(n)
        head = 0            # first request not yet in a batch (arrival order)
        finished = 0
        in_flight_mask = 0
        batches = 0
        max_in_flight = 0
        row = self.idx.W * 4
        t0 = time.perf_counter()
        while finished < n:
            now = time.perf_counter() - t0
            for sl in self.slots:
                if sl.busy and sl.event.query():
                    i0, i1 = sl.span
                    done_at[tr.rid[i0:i1]] = time.perf_counter() - t0
                    finished += i1 - i0
                    in_flight_mask -= (i1 - i0) * row
                    sl.busy = False
            avail = int(np.searchsorted(tr.arrival, now, side="right"))
            launched = False
            for sl in self.slots:
                if head >= avail:
                    break
                if sl.busy:
                    continue
                if in_flight_mask + row > self.mask_budget and any(s.busy for s in self.slots):
                    break
                end = self._batch_end(tr, head, avail, in_flight_mask)
                sl.launch(self.idx, tr, head, end)
                in_flight_mask += (end - head) * row
                head = end
                batches += 1
                launched = True
            max_in_flight = max(max_in_flight, sum(1 for sl in self.slots if sl.busy))
            if not launched:
                if head < n and head >= avail and not any(sl.busy for sl in self.slots):
                    wait = tr.arrival[head] - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 1e-3))
                else:
                    time.sleep(spin_sleep)
        wall = time.perf_counter() - t0
        lat = done_at - np.array([r.arrival for r in sorted(requests, key=lambda r: r.rid)])
        return ServeResult(lat, tr.by_request(), wall, tr.bases, batches, max_in_flight,
                           {"mode": "continuous", "slots": len(self.slots)})


def plain_batched(idx, requests: list[Request], batch_size: int, max_batch_bytes: int = 8 << 20) -> ServeResult:
    """Fixed-size batches, one at a time: wait for batch_size arrivals (or the
    end of the trace), run the batch through the device API with page-locked
    buffers (bytes in, ranges in, query, answers out) and wait for it."""
    import torch
    tr = _Trace(requests, max_batch_bytes)
    tr.answer_buffer(idx.W)
    n = tr.n
    dev = torch.device(f"cuda:{idx.device}")
    sl = _Slot(idx, batch_size, max(max_batch_bytes, 16), dev)
    done_at = np.zeros(n)
    t0 = time.perf_counter()
    batches = 0
    i0 = 0
    while i0 < n:
        i1 = min(n, i0 + batch_size)
        # the batch's bytes must fit the slot
        i1 = max(i0 + 1, min(i1, int(np.searchsorted(tr.bstart, tr.bstart[i0] + max_batch_bytes,
                                                            side="right")) - 1))
        last_arrival = tr.arrival[i1 - 1]
        while time.perf_counter() - t0 < last_arrival:
            time.sleep(min(1e-3, max(0.0, last_arrival - (time.perf_counter() - t0))))
        sl.launch(idx, tr, i0, i1)
        sl.stream.synchronize()
        done_at[tr.rid[i0:i1]] = time.perf_counter() - t0
        batches += 1
        i0 = i1
    wall = time.perf_counter() - t0
    lat = done_at - np.array([r.arrival for r in sorted(requests, key=lambda r: r.rid)])
    return ServeResult(lat, tr.by_request(), wall, tr.bases, batches, 1,
                       {"mode": "plain", "batch_size": batch_size})


def one_batch_rate(idx, requests: list[Request], reps: int = 3) -> dict:
    """The device's batched rate on a trace: every request in one
    query_ranges_dev call, inputs already on the device, timed with CUDA
    events (best of reps) -- the ceiling a server of this trace can approach."""
    import torch
    tr = _Trace(requests, max(r.packed.size for r in requests))
    n = tr.n
    b = torch.empty(n, dtype=torch.int64)
    e = torch.empty(n, dtype=torch.int64)
    tr.ranges(0, n, b.numpy(), e.numpy())
    dev = torch.device(f"cuda:{idx.device}")
    dp, db, de = tr.arena.to(dev), b.to(dev), e.to(dev)
    out = idx.query_ranges_dev(dp, db, de)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        e0.record()
        idx.query_ranges_dev(dp, db, de, out=out)
        e1.record()
        torch.cuda.synchronize(dev)
        best = min(best, e0.elapsed_time(e1))
    return {"ms": best, "bp_per_s": tr.bases / (best / 1e3), "requests_per_s": n / (best / 1e3)}


def make_requests(corpus, arrivals: np.ndarray, lengths: np.ndarray, rng, frac_from_docs=0.7,
                  err_rate=0.001) -> list[Request]:
    """Requests shaped like the serving workload: 70% substrings of documents
    (with read errors), 30% uniform, each packed on its own."""
    from .synth import pack_bases, sample_queries, unpack_bases
    q = sample_queries(rng, corpus, lengths, frac_from_docs, err_rate=err_rate)
    reqs = []
    offs = q.offsets.astype(np.int64)
    for i in range(q.n):
        bases = unpack_bases(q.packed, int(offs[i]), int(offs[i + 1] - offs[i]))
        reqs.append(Request(i, pack_bases(bases), int(bases.size), float(arrivals[i])))
    return reqs
