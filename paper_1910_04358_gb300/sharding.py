"""Document-sharded RAMBO (Section 5.3, "Smart parallelism").

The paper indexes the full archive on 100 nodes without any message passing:
a routing hash tau sends each document to one node, the node inserts it into
its own RAMBO of b buckets per repetition with its node-local partition phi,
and the stacked structure is one RAMBO of S*b buckets whose bucket map is
b*tau(D) + phi(D).  A query is sent to every shard; the global answer is the
shards' answers placed at their documents' global ids -- a concatenation in
global document order, with no reduction, because the shards hold disjoint
documents.

* `ShardedIndex` keeps all shards in one process (on one GPU or spread over
  several devices): each shard inserts its documents straight from the shared
  packed corpus (`rambo_insert_ranges_dev`) and the shards' answers are
  merged on the device (`rambo_merge_shard_answers`).
* `gather_answers` is the multi-process form: every rank answers the same
  batch on its own shard, the local answers are exchanged with one
  all_gather, and each rank merges them into the global answers (on the
  device, or with `merge_answers_host` where the ranks answer on the host).

`composed_partition` gives the equivalent single index's bucket map, which
rambo_set_partition accepts.
"""
from __future__ import annotations

import numpy as np

from . import rambo


def route(K: int, shards: int, seed: int = 0) -> np.ndarray:
    """tau: document -> shard, a seeded splitmix64-style integer hash (host-side
    routing only; it is not part of any index)."""
    x = np.arange(K, dtype=np.uint64) + np.uint64((seed * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF)
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    x = x ^ (x >> np.uint64(31))
    return (x % np.uint64(shards)).astype(np.int64)


def members(tau: np.ndarray, shards: int) -> list[np.ndarray]:
    """Global ids of each shard's documents, increasing: local id j of shard
    s is global document members[s][j]."""
    return [np.nonzero(tau == s)[0] for s in range(shards)]


def merge_answers_host(n: int, K: int, parts) -> np.ndarray:
    """Global answers (n x ceil(K/32) uint32) from shard answers: `parts` is
    a sequence of (local answers n x Ws uint32, global ids of the shard's
    local documents).  Each local bit j is placed at global bit ids[j]."""
    W = (K + 31) // 32
    bits = np.zeros((n, W * 32), dtype=np.uint8)
    for local, ids in parts:
        ids = np.asarray(ids, dtype=np.int64)
        if ids.size == 0:
            continue
        lb = np.unpackbits(np.ascontiguousarray(local, dtype="<u4").view(np.uint8), axis=1,
                           bitorder="little")[:, :ids.size]
        bits[:, ids] |= lb
    return np.packbits(bits, axis=1, bitorder="little").view("<u4").reshape(n, W).astype(np.uint32)


def gather_answers(local, member_lists, K: int, group=None, device_merge: bool = True):
    """All ranks hold answers of the same n queries against their own shard
    (`local`: n x Ws int32 tensor, Ws the widest shard's words, on the
    rank's GPU for NCCL or on the CPU for gloo).  One all_gather exchanges
    them; every rank then merges the world's answers into the global
    answers (n x ceil(K/32)), on the device with the library's merge kernel
    or, for CPU tensors, on the host."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n, ws = local.shape
    flat = torch.empty((world * n, ws), dtype=local.dtype, device=local.device)
    dist.all_gather_into_tensor(flat, local.contiguous(), group=group)
    parts = flat.view(world, n, ws)
    W = (K + 31) // 32
    if device_merge and local.is_cuda:
        out = torch.zeros((n, W), dtype=torch.int32, device=local.device)
        for s in range(world):
            ids = torch.from_numpy(np.asarray(member_lists[s], dtype=np.int32)).to(local.device)
            if ids.numel():
                rambo.merge_shard_answers(parts[s], ids, out)
        return out
    host = parts.cpu().numpy().view(np.uint32)
    return torch.from_numpy(merge_answers_host(n, K, [(host[s], member_lists[s])
                                                      for s in range(world)]).view(np.int32))


class ShardedIndex:
    def __init__(self, K: int, b: int, R: int, m: int, eta: int, k: int = 31, seed: int = 0,
                 shards: int = 2, route_seed: int = 0, devices=None):
        self.K, self.b, self.R, self.S = K, b, R, shards
        self.tau = route(K, shards, route_seed)
        self.members = members(self.tau, shards)
        self.local = np.zeros(K, dtype=np.int64)
        for s, mem in enumerate(self.members):
            self.local[mem] = np.arange(mem.size)
        devices = devices or [0]
        self.devices = [devices[s % len(devices)] for s in range(shards)]
        self.shards = [rambo.Index(max(int(mem.size), 1), b, R, m, eta, k, seed, device=self.devices[s])
                       for s, mem in enumerate(self.members)]
        self.W = (K + 31) // 32

    def insert_batch(self, doc_ids, packed, offsets):
        """Host arrays: documents doc_ids[i] = bases [offsets[i], offsets[i+1])."""
        import torch
        on = {}
        for d in set(self.devices):
            on[d] = torch.from_numpy(np.ascontiguousarray(packed, dtype=np.uint8)).to(f"cuda:{d}")
        self.insert_batch_dev(doc_ids, on, offsets)
        for idx in self.shards:
            idx.sync()

    def insert_batch_dev(self, doc_ids, packed_on, offsets):
        """doc_ids and offsets (n+1) on the host; packed_on maps each shard
        device to the packed corpus there (a CUDA uint8 tensor).  Each shard
        inserts the documents tau sends to it, with one range insert."""
        import torch
        ids = np.asarray(doc_ids, dtype=np.int64)
        offs = np.asarray(offsets, dtype=np.int64)
        for s, idx in enumerate(self.shards):
            sel = np.nonzero(self.tau[ids] == s)[0]
            if sel.size == 0:
                continue
            dev = f"cuda:{self.devices[s]}"
            loc = torch.from_numpy(self.local[ids[sel]].astype(np.int32)).to(dev)
            b = torch.from_numpy(offs[sel]).to(dev)
            e = torch.from_numpy(offs[sel + 1]).to(dev)
            idx.insert_ranges_dev(loc, packed_on[self.devices[s]], b, e)

    def query_seqs_dev(self, packed, offsets, out=None):
        """The batch (CUDA tensors on the first shard's device) against every
        shard; returns the global answers (n x W int32) there."""
        import torch
        n = offsets.numel() - 1
        dev0 = f"cuda:{self.devices[0]}"
        if out is None:
            out = torch.empty((n, self.W), dtype=torch.int32, device=dev0)
        out.zero_()
        for s, idx in enumerate(self.shards):
            mem = self.members[s]
            if mem.size == 0:
                continue
            dev = f"cuda:{self.devices[s]}"
            local = idx.query_seqs_dev(packed.to(dev), offsets.to(dev))
            ids = torch.from_numpy(mem.astype(np.int32)).to(dev0)
            rambo.merge_shard_answers(local.to(dev0), ids, out)
        return out

    def query_seqs(self, packed, offsets) -> np.ndarray:
        import torch
        dev0 = f"cuda:{self.devices[0]}"
        p = torch.from_numpy(np.ascontiguousarray(packed, dtype=np.uint8)).to(dev0)
        o = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.uint64).view(np.int64)).to(dev0)
        out = self.query_seqs_dev(p, o)
        torch.cuda.synchronize(dev0)
        for idx in self.shards:
            idx.sync()
        return rambo.as_u32(out)

    def composed_partition(self) -> np.ndarray:
        """Bucket map of the equivalent single index: b * tau(d) + phi_local(d)."""
        phi = np.zeros((self.K, self.R), dtype=np.uint32)
        for s, idx in enumerate(self.shards):
            mem = self.members[s]
            if mem.size:
                phi[mem] = self.b * s + idx.partition()[: mem.size]
        return phi
