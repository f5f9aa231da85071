"""Small, self-contained launches of one query stage, for profiling.

  python -m paper_1910_04358_gb300.kernel_case --case kmers|seqs|build|gather
         [--workload medium|large|stream] [--reps N] [--query-path 0|1|2]

Builds the workload's index on cuda:0, then runs the chosen query batch
`reps` times (kmers: the medium workload's 10^6 single 31-mers; seqs: its
sequence batch) so a profiler can capture single launches of the probe,
expansion or fused kernels on a realistic index.  `build` builds the index
`reps` times into fresh handles (the tuning's insert mode) and prints each
build's insert-stage time from the library's CUDA events.  The stream workload
inserts its first `--epochs` epochs of documents (its full document
geometry: 10^5 document bits per answer, R = 6, B = 316) and queries the
last epoch's batch.

`gather` times the random-record gather (rambo_probe_gather: random records of
16..512 bytes from a device buffer, no hashing or bit logic) over record
sizes, loads in flight per lane and buffer sizes, one JSON object per point:
a probe of the index reads one group of G bytes at a random position, so the
row for record = max(G, 16) bounds what the probe kernels can reach.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["kmers", "seqs", "build", "gather"], default="kmers")
    ap.add_argument("--workload", choices=["medium", "large", "stream"], default="medium")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--query-path", type=int, default=0)
    ap.add_argument("--tune", nargs="*", default=[], help="tuning knobs as name=value")
    ap.add_argument("--tuning-from-cache", action="store_true",
                    help="use the tuning bench.py cached for this workload's batch")
    ap.add_argument("--n-docs", type=int, default=None, help="fewer documents (same geometry)")
    ap.add_argument("--m", type=int, default=None, help="bits per filter (smaller index)")
    ap.add_argument("--n-queries", type=int, default=None, help="fewer sequence queries (large)")
    ap.add_argument("--n-seeds", type=int, default=None, help="fewer seed genomes (large)")
    ap.add_argument("--epochs", type=int, default=3, help="insert epochs before the query (stream)")
    ap.add_argument("--buf-gb", type=float, nargs="+", default=[1.0, 64.0], help="gather: buffer sizes")
    ap.add_argument("--records", type=int, nargs="+", default=[16, 32, 64, 128, 256, 512],
                    help="gather: record bytes")
    ap.add_argument("--unroll", type=int, nargs="+", default=[4, 8, 16, 32],
                    help="gather: 16-byte loads in flight per lane")
    a = ap.parse_args(argv)
    if a.case == "gather":
        return gather_case(a)
    import torch

    from . import rambo, synth
    if a.workload == "stream":
        return stream_case(a)
    if a.workload == "medium":
        corpus, kmers, q = synth.medium_workload(n_docs=a.n_docs)
    else:
        kw = {"n_docs": a.n_docs}
        if a.n_queries:
            kw["n_queries"] = a.n_queries
        if a.n_seeds:
            kw["n_seeds"] = a.n_seeds
        corpus, q = synth.large_workload(**kw)
        kmers = np.zeros(0, np.uint64)
    p = corpus.params
    if a.m:
        p = synth.Params(K=p.K, B=p.B, R=p.R, m=a.m, eta=p.eta, k=p.k, seed=p.seed)
    dev = lambda x, dt: torch.from_numpy(np.ascontiguousarray(x).view(dt)).cuda()
    if a.case == "build":
        return build_case(a, corpus, p, dev)
    idx = rambo.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, device=0)
    if a.tuning_from_cache:
        from . import autotune
        n_kmers = q.n_kmers(p.k) + int(kmers.size)
        cached = autotune.load_cached(autotune.CACHE_FILE,
                                      autotune.cache_key(idx, q.n + int(kmers.size), n_kmers))
        if cached:
            idx.set_tuning(**cached)
    else:
        idx.set_tuning(query_path=a.query_path)
    if a.tune:
        idx.set_tuning(**{kv.split("=")[0]: int(kv.split("=")[1]) for kv in a.tune})
    idx.insert_batch_dev(dev(corpus.doc_ids, np.int32), dev(corpus.packed, np.uint8),
                         dev(corpus.offsets, np.int64))
    idx.sync()
    if a.case == "kmers":
        dk = dev(kmers, np.int64)
        out = torch.empty((kmers.size, idx.W), dtype=torch.int32, device="cuda")
        run = lambda: idx.query_kmers_dev(dk, out=out)
    else:
        dp, do = dev(q.packed, np.uint8), dev(q.offsets, np.int64)
        out = torch.empty((q.n, idx.W), dtype=torch.int32, device="cuda")
        run = lambda: idx.query_seqs_dev(dp, do, out=out)
    ms = []
    for _ in range(a.reps):  # each call timed with CUDA events on the launching stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    idx.sync()
    print("ok", a.case, a.workload, int(out.sum().item()),
          "ms per call: best %.3f (of %d; the first includes setup)" % (min(ms[1:] or ms), len(ms)))
    return 0


def build_case(a, corpus, p, dev):
    from . import rambo
    d_ids, d_p, d_o = dev(corpus.doc_ids, np.int32), dev(corpus.packed, np.uint8), dev(corpus.offsets, np.int64)
    kmers = int(np.maximum(np.diff(corpus.offsets.astype(np.int64)) - p.k + 1, 0).sum())
    for _ in range(a.reps):
        idx = rambo.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, device=0)
        if a.tune:
            idx.set_tuning(**{kv.split("=")[0]: int(kv.split("=")[1]) for kv in a.tune})
        idx.profile_reset(timed_stages=("insert",))
        idx.insert_batch_dev(d_ids, d_p, d_o)
        idx.sync()
        ms = idx.profile_read()["insert"]["ms"]
        print(f"build {a.workload} insert_mode {idx.get_tuning()['insert_mode']}: {ms:.2f} ms, "
              f"{kmers / (ms / 1e3):.3e} k-mers/s", flush=True)
        idx.close()
    return 0


def stream_case(a):
    import torch

    from . import rambo, synth
    if a.case != "seqs":
        raise SystemExit("the stream workload has sequence queries only")
    wl = synth.stream_workload(m=a.m)
    p = wl.params
    dev = lambda x, dt: torch.from_numpy(np.ascontiguousarray(x).view(dt)).cuda()
    idx = rambo.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, device=0)
    idx.set_tuning(query_path=a.query_path if a.query_path else 1)
    if a.tuning_from_cache:  # the tuning bench.py keeps for this geometry's epoch batches
        from . import autotune
        key = autotune.cache_key(idx, wl.queries_per_epoch, 0).rsplit("_kpq", 1)[0] + "_stream"
        cached = autotune.load_cached(autotune.CACHE_FILE, key)
        if cached:
            idx.set_tuning(**cached)
    if a.tune:
        idx.set_tuning(**{kv.split("=")[0]: int(kv.split("=")[1]) for kv in a.tune})
    for e in range(max(1, min(a.epochs, wl.n_epochs))):
        (ids, packed, offs), q = wl.epoch(e)
        idx.insert_batch_dev(dev(ids.astype(np.int32), np.int32), dev(packed, np.uint8),
                             dev(offs, np.int64))
    idx.sync()
    dp, do = dev(q.packed, np.uint8), dev(q.offsets, np.int64)
    out = torch.empty((q.n, idx.W), dtype=torch.int32, device="cuda")
    for _ in range(a.reps):
        idx.query_seqs_dev(dp, do, out=out)
    idx.sync()
    print("ok", a.case, a.workload, int(out.sum().item()))
    return 0


def gather_case(a, useful_gb=2.0):
    import json

    import torch

    from . import rambo
    rambo.load()
    for size_gb in a.buf_gb:
        buf = torch.empty(int(size_gb * (1 << 30)), dtype=torch.uint8, device="cuda")
        buf.fill_(3)
        sink = torch.zeros(1, dtype=torch.int64, device="cuda")
        for rb in a.records:
            n = int(useful_gb * (1 << 30)) // rb
            for u in a.unroll:
                rambo.probe_gather(buf, rb, n, 0, 7, sink, unroll=u)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                best = float("inf")
                for r in range(max(1, a.reps)):
                    e0.record()
                    rambo.probe_gather(buf, rb, n, 0, 11 + r, sink, unroll=u)
                    e1.record()
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                print(json.dumps({"buf_gb": size_gb, "record_bytes": rb, "unroll": u, "ms": best,
                                  "probes_per_s": n / best * 1e3, "useful_gb_s": n * rb / best / 1e6,
                                  "line_gb_s": n * max(rb, 128) / best / 1e6}), flush=True)
        del buf
        torch.cuda.empty_cache()
    return 0


if __name__ == "__main__":
    sys.exit(main())
