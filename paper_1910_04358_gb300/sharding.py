"""Document-sharded RAMBO (Section 5.3, "Smart parallelism").

The paper indexes the full archive on 100 nodes without any message passing:
a routing hash tau sends each document to one node, the node inserts it into
its own RAMBO of b buckets per repetition with its node-local partition phi,
and the stacked structure is one RAMBO of S*b buckets whose bucket map is
b*tau(D) + phi(D).  Every shard here is an independent index (on one GPU or
spread over several devices); a query is sent to every shard and the global
answer is the shards' answers placed at their documents' global ids -- a
concatenation, with no reduction, because the shards hold disjoint documents.
`composed_partition` gives the equivalent single index's bucket map, which
rambo_set_partition accepts.
"""
from __future__ import annotations

import numpy as np

from . import rambo


def route(K: int, shards: int, seed: int = 0) -> np.ndarray:
    """tau: document -> shard, a seeded splitmix64-style integer hash (host-side
    routing only; it is not part of any index)."""
    x = (np.arange(K, dtype=np.uint64) + np.uint64(seed) * np.uint64(0x9E3779B97F4A7C15))
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    x = x ^ (x >> np.uint64(31))
    return (x % np.uint64(shards)).astype(np.int64)


class ShardedIndex:
    def __init__(self, K: int, b: int, R: int, m: int, eta: int, k: int = 31, seed: int = 0,
                 shards: int = 2, route_seed: int = 0, devices=None):
        self.K, self.b, self.R, self.S = K, b, R, shards
        self.tau = route(K, shards, route_seed)
        self.members = [np.nonzero(self.tau == s)[0] for s in range(shards)]
        self.local = np.zeros(K, dtype=np.int64)
        for s, mem in enumerate(self.members):
            self.local[mem] = np.arange(mem.size)
        devices = devices or [None]
        self.shards = [rambo.Index(max(int(mem.size), 1), b, R, m, eta, k, seed,
                                   device=devices[s % len(devices)])
                       for s, mem in enumerate(self.members)]
        self.W = (K + 31) // 32

    def insert_batch(self, doc_ids, packed, offsets):
        ids = np.asarray(doc_ids, dtype=np.int64)
        offs = np.asarray(offsets, dtype=np.uint64)
        for s in range(self.S):
            sel = np.nonzero(self.tau[ids] == s)[0]
            if sel.size == 0:
                continue
            # each selected document keeps its own [begin, end) in the shared stream
            for i in sel:
                self.shards[s].insert(int(self.local[ids[i]]), _slice_packed(packed, offs[i], offs[i + 1]),
                                      int(offs[i + 1] - offs[i]))

    def query_seqs(self, packed, offsets) -> np.ndarray:
        n = len(offsets) - 1
        bits = np.zeros((n, self.W * 32), dtype=np.uint8)
        for s, idx in enumerate(self.shards):
            mem = self.members[s]
            if mem.size == 0:
                continue
            local = idx.query_seqs(packed, offsets)
            lb = np.unpackbits(local.view(np.uint8), axis=1, bitorder="little")[:, :mem.size]
            bits[:, mem] = lb
        return np.packbits(bits, axis=1, bitorder="little").view(np.uint32).reshape(n, self.W)

    def composed_partition(self) -> np.ndarray:
        """Bucket map of the equivalent single index: b * tau(d) + phi_local(d)."""
        phi = np.zeros((self.K, self.R), dtype=np.uint32)
        for s, idx in enumerate(self.shards):
            mem = self.members[s]
            if mem.size:
                phi[mem] = self.b * s + idx.partition()[: mem.size]
        return phi


def _slice_packed(packed: np.ndarray, b0, b1) -> np.ndarray:
    """The bases [b0, b1) of a packed stream as a packed buffer starting at base 0."""
    from .synth import pack_bases, unpack_bases
    return pack_bases(unpack_bases(packed, int(b0), int(b1 - b0)))
