"""Small, self-contained launches of one query stage, for profiling.

  python -m paper_1910_04358_gb300.kernel_case --case kmers|seqs [--workload medium|large]
         [--reps N] [--query-path 0|1]

Builds the workload's index on cuda:0, then runs the chosen query batch
`reps` times (kmers: the medium workload's 10^6 single 31-mers; seqs: its
sequence batch) so a profiler can capture single launches of the probe,
expansion or fused kernels on a realistic index.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["kmers", "seqs"], default="kmers")
    ap.add_argument("--workload", choices=["medium", "large"], default="medium")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--query-path", type=int, default=0)
    ap.add_argument("--tune", nargs="*", default=[], help="tuning knobs as name=value")
    a = ap.parse_args(argv)
    import torch

    from . import rambo, synth
    if a.workload == "medium":
        corpus, kmers, q = synth.medium_workload()
    else:
        corpus, q = synth.large_workload()
        kmers = np.zeros(0, np.uint64)
    p = corpus.params
    dev = lambda x, dt: torch.from_numpy(np.ascontiguousarray(x).view(dt)).cuda()
    idx = rambo.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, device=0)
    idx.set_tuning(query_path=a.query_path, **{kv.split("=")[0]: int(kv.split("=")[1]) for kv in a.tune})
    idx.insert_batch_dev(dev(corpus.doc_ids, np.int32), dev(corpus.packed, np.uint8),
                         dev(corpus.offsets, np.int64))
    idx.sync()
    if a.case == "kmers":
        dk = dev(kmers, np.int64)
        out = torch.empty((kmers.size, idx.W), dtype=torch.int32, device="cuda")
        for _ in range(a.reps):
            idx.query_kmers_dev(dk, out=out)
    else:
        dp, do = dev(q.packed, np.uint8), dev(q.offsets, np.int64)
        out = torch.empty((q.n, idx.W), dtype=torch.int32, device="cuda")
        for _ in range(a.reps):
            idx.query_seqs_dev(dp, do, out=out)
    idx.sync()
    print("ok", a.case, a.workload, int(out.sum().item()))
    return 0


if __name__ == "__main__":
    sys.exit(main())
