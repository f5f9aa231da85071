"""Continuous-batching query server over a resident index.

Requests (2-bit packed sequences) arrive over time.  The engine keeps the
index resident in HBM and a fixed set of slots, each with its own CUDA stream,
pinned host buffers, device buffers and query workspace.  Whenever a slot is
free it forms the next batch from the requests that have arrived, in arrival
order, bounded by the slot's capacity and by an output-mask memory budget
(the answers of all batches in flight must fit it), copies the batch in,
enqueues the query and the copy of the answers back on the slot's stream,
and moves on: batches on different slots overlap on the device.  Each
request is packed at a byte boundary of the slot buffer and passed as a
[begin, end) range, so no bases are shifted on the host.

`plain_batched` serves the same trace the simple way for comparison: wait
for a fixed number of arrivals, run one synchronous batch, repeat.

Both return per-request answers (bit-identical to querying each request
alone) and latencies (completion time - arrival time).
"""
from __future__ import annotations

import collections
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
    answers: list
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


class _Slot:
    def __init__(self, idx, max_queries: int, max_bytes: int, device):
        import torch
        self.stream = torch.cuda.Stream(device=device)
        self.h_packed = torch.empty(max_bytes + 16, dtype=torch.uint8, pin_memory=True)
        self.h_begin = torch.empty(max_queries, dtype=torch.int64, pin_memory=True)
        self.h_end = torch.empty(max_queries, dtype=torch.int64, pin_memory=True)
        self.h_out = torch.empty((max_queries, idx.W), dtype=torch.int32, pin_memory=True)
        self.d_packed = torch.empty(max_bytes + 16, dtype=torch.uint8, device=device)
        self.d_begin = torch.empty(max_queries, dtype=torch.int64, device=device)
        self.d_end = torch.empty(max_queries, dtype=torch.int64, device=device)
        self.d_out = torch.empty((max_queries, idx.W), dtype=torch.int32, device=device)
        ws_bytes = idx.workspace_bytes("seqs", max_queries)
        self.ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        self.ws_ptr = ((base + 255) // 256 * 256, ws_bytes)
        self.event = torch.cuda.Event()
        self.batch: list[Request] = []
        self.busy = False
        self.mask_bytes = 0


class ServingEngine:
    def __init__(self, idx, slots: int = 4, max_batch_queries: int = 2048,
                 max_batch_bytes: int = 4 << 20, mask_budget_bytes: int = 64 << 20,
                 device: int | None = None):
        import torch
        self.idx = idx
        self.device = torch.device(f"cuda:{idx.device if device is None else device}")
        self.max_q = max_batch_queries
        self.max_bytes = max_batch_bytes
        self.mask_budget = mask_budget_bytes
        self.slots = [_Slot(idx, max_batch_queries, max_batch_bytes, self.device)
                      for _ in range(slots)]

    # -- one batch ---------------------------------------------------------
    def _launch(self, slot: _Slot, batch: list[Request]):
        import torch
        W = self.idx.W
        pos = 0
        hp = slot.h_packed.numpy()
        hb, he = slot.h_begin.numpy(), slot.h_end.numpy()
        for i, r in enumerate(batch):
            nb = r.packed.size
            hp[pos:pos + nb] = r.packed
            hb[i] = 4 * pos
            he[i] = 4 * pos + r.n_bases
            pos += nb
        n = len(batch)
        with torch.cuda.stream(slot.stream):
            slot.d_packed[:pos].copy_(slot.h_packed[:pos], non_blocking=True)
            slot.d_begin[:n].copy_(slot.h_begin[:n], non_blocking=True)
            slot.d_end[:n].copy_(slot.h_end[:n], non_blocking=True)
            self.idx.query_ranges_dev(slot.d_packed[:pos], slot.d_begin[:n], slot.d_end[:n],
                                      out=slot.d_out[:n], stream=slot.stream,
                                      workspace=slot.ws_ptr)
            slot.h_out[:n].copy_(slot.d_out[:n], non_blocking=True)
            slot.event.record(slot.stream)
        slot.batch = batch
        slot.busy = True
        slot.mask_bytes = n * W * 4

    def _collect(self, slot: _Slot, now: float, answers: list, done_at: np.ndarray):
        out = slot.h_out.numpy()
        for i, r in enumerate(slot.batch):
            answers[r.rid] = out[i].view(np.uint32).copy()
            done_at[r.rid] = now
        slot.busy = False
        slot.batch = []
        released = slot.mask_bytes
        slot.mask_bytes = 0
        return released

    # -- continuous batching ----------------------------------------------
    def serve(self, requests: list[Request], spin_sleep: float = 20e-6) -> ServeResult:
        n = len(requests)
        order = sorted(range(n), key=lambda i: requests[i].arrival)
        answers = [None] * n
        done_at = np.zeros(n)
        pending = collections.deque()
        nxt = 0
        in_flight_mask = 0
        batches = 0
        max_in_flight = 0
        W4 = self.idx.W * 4
        t0 = time.perf_counter()
        finished = 0
        while finished < n:
            now = time.perf_counter() - t0
            while nxt < n and requests[order[nxt]].arrival <= now:
                pending.append(requests[order[nxt]])
                nxt += 1
            for sl in self.slots:
                if sl.busy and sl.event.query():
                    in_flight_mask -= self._collect(sl, time.perf_counter() - t0, answers, done_at)
                    finished += 0  # counted below
            finished = sum(1 for a in answers if a is not None)
            launched = False
            for sl in self.slots:
                if not pending:
                    break
                if sl.busy:
                    continue
                batch, nbytes = [], 0
                while pending and len(batch) < self.max_q:
                    r = pending[0]
                    if nbytes + r.packed.size > self.max_bytes and batch:
                        break
                    if in_flight_mask + (len(batch) + 1) * W4 > self.mask_budget and batch:
                        break
                    batch.append(pending.popleft())
                    nbytes += r.packed.size
                if not batch:
                    break
                self._launch(sl, batch)
                in_flight_mask += len(batch) * W4
                batches += 1
                launched = True
            max_in_flight = max(max_in_flight, sum(1 for sl in self.slots if sl.busy))
            if not launched:
                if nxt < n and not pending and not any(sl.busy for sl in self.slots):
                    wait = requests[order[nxt]].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 1e-3))
                else:
                    time.sleep(spin_sleep)
        wall = time.perf_counter() - t0
        lat = np.array([done_at[i] - requests[i].arrival for i in range(n)])
        bases = sum(r.n_bases for r in requests)
        return ServeResult(lat, answers, wall, bases, batches, max_in_flight,
                           {"mode": "continuous", "slots": len(self.slots)})


def plain_batched(idx, requests: list[Request], batch_size: int) -> ServeResult:
    """Fixed-size batches, one at a time: wait for batch_size arrivals (or the
    end of the trace), query synchronously through the host-buffer ABI."""
    from .synth import PackedStream, unpack_bases
    n = len(requests)
    order = sorted(range(n), key=lambda i: requests[i].arrival)
    answers = [None] * n
    done_at = np.zeros(n)
    t0 = time.perf_counter()
    batches = 0
    for s in range(0, n, batch_size):
        group = [requests[i] for i in order[s:s + batch_size]]
        last_arrival = group[-1].arrival
        while time.perf_counter() - t0 < last_arrival:
            time.sleep(min(1e-3, max(0.0, last_arrival - (time.perf_counter() - t0))))
        ps = PackedStream()
        for r in group:
            ps.append(unpack_bases(r.packed, 0, r.n_bases))
        packed, offs = ps.finish()
        out = idx.query_seqs(packed, offs)
        now = time.perf_counter() - t0
        for i, r in enumerate(group):
            answers[r.rid] = out[i]
            done_at[r.rid] = now
        batches += 1
    wall = time.perf_counter() - t0
    lat = np.array([done_at[i] - requests[i].arrival for i in range(n)])
    return ServeResult(lat, answers, wall, sum(r.n_bases for r in requests), batches, 1,
                       {"mode": "plain", "batch_size": batch_size})


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
