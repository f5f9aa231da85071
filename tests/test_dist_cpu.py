"""The multi-rank plumbing of bench.py on CPU ranks (gloo, world size 2):
max-over-ranks timing, barriers, and the reference arm under torchrun, where
rank 0 alone runs and prints and the other ranks exit 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, local, w = bench.dist_setup("gloo")
    bench.barrier(w)
    m = bench.max_over_ranks(float(10 * (rank + 1)), w)
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((rank, m))


def test_max_over_ranks_and_barrier_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 20.0, 1: 20.0}


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--workload", "tiny", "--steps", "3", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def _shard_worker(rank, world, port, q):
    # one shard per CPU rank, the CPU oracle standing in for the GPU engine:
    # every rank answers the same batch on its shard, the answers are
    # exchanged with one all_gather and merged into global document order
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1910_04358_gb300 import sharding, synth
    dist.init_process_group("gloo")
    K, b, R, m, eta = 130, 6, 3, 1 << 13, 2
    p = synth.Params(K=K, B=world * b, R=R, m=m, eta=eta, k=31, seed=4)
    rng = np.random.default_rng(23)
    corpus = synth.family_corpus(rng, p, n_seeds=10, doc_len=600, sub_rate=0.02)
    qb = synth.sample_queries(rng, corpus, rng.integers(20, 300, size=150), 0.6)
    tau = sharding.route(K, world)
    mem = sharding.members(tau, world)
    offs = corpus.offsets.astype(np.int64)
    # this rank's shard: its documents as local documents 0..K_s-1
    mine = mem[rank]
    shard = oracle.Rambo(max(mine.size, 1), b, R, m, eta, p.k, p.seed)
    for j, d in enumerate(mine.tolist()):
        shard.insert(j, corpus.packed, int(offs[d]), int(offs[d + 1] - offs[d]))
    local = shard.query_seqs(qb.packed, qb.offsets)
    ws = max((x.size + 31) // 32 for x in mem)
    padded = np.zeros((qb.n, ws), dtype=np.uint32)
    padded[:, :local.shape[1]] = local
    got = sharding.gather_answers(torch.from_numpy(padded.view(np.int32)), mem, K).numpy().view(np.uint32)
    # one oracle over all documents with the composed bucket map
    # b * tau(d) + phi_local(d), phi_local from each shard's own local ids
    probe = oracle.Rambo(1, b, R, m, eta, p.k, p.seed)
    phi = np.zeros((K, R), dtype=np.uint32)
    for s in range(world):
        for j, d in enumerate(mem[s].tolist()):
            phi[d] = [b * s + probe.partition(j, r) for r in range(R)]
    one = oracle.Rambo(K, world * b, R, m, eta, p.k, p.seed)
    one.set_partition(phi)
    one.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    want = one.query_seqs(qb.packed, qb.offsets)
    dist.destroy_process_group()
    q.put((rank, bool(np.array_equal(got, want)), int(np.count_nonzero(want))))


def test_document_shards_gathered_equal_one_oracle_with_composed_map():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = dict((r, (ok, nz)) for r, ok, nz in (q.get(timeout=10) for _ in range(2)))
    assert got[0][0] and got[1][0]
    assert got[0][1] > 0  # the answers are not trivially empty
