"""Random-record gather sweep: the practical ceiling of index probes.

Times rambo_probe_gather (random records of 16..512 bytes from a device
buffer, no hashing or bit logic) over record sizes, loads in flight per lane
and buffer sizes, and prints one JSON object per point.  A probe of the index
reads one group of G bytes at a random position, so the row for
record = max(G, 16) bounds what the probe kernels can reach.

  python -m paper_1910_04358_gb300.gather_sweep [--buf-gb 1 64] [--records 16 64 256]
                                                 [--unroll 8 32] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import sys


def sweep(buf_gbs, records, unrolls, variants=(0,), reps=4, useful_gb=2.0):
    import torch

    from . import rambo
    rambo.load()
    out = []
    for size_gb in buf_gbs:
        buf = torch.empty(int(size_gb * (1 << 30)), dtype=torch.uint8, device="cuda")
        buf.fill_(3)
        sink = torch.zeros(1, dtype=torch.int64, device="cuda")
        for rb in records:
            n = int(useful_gb * (1 << 30)) // rb
            for u in unrolls:
                for v in variants:
                    rambo.probe_gather(buf, rb, n, v, 7, sink, unroll=u)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    best = float("inf")
                    for r in range(reps):
                        e0.record()
                        rambo.probe_gather(buf, rb, n, v, 11 + r, sink, unroll=u)
                        e1.record()
                        torch.cuda.synchronize()
                        best = min(best, e0.elapsed_time(e1))
                    row = {"buf_gb": size_gb, "record_bytes": rb, "unroll": u, "variant": v,
                           "ms": best, "probes_per_s": n / best * 1e3,
                           "useful_gb_s": n * rb / best / 1e6,
                           "line_gb_s": n * max(rb, 128) / best / 1e6}
                    out.append(row)
                    print(json.dumps(row), flush=True)
        del buf
        torch.cuda.empty_cache()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--buf-gb", type=float, nargs="+", default=[1.0, 64.0])
    ap.add_argument("--records", type=int, nargs="+", default=[16, 32, 64, 128, 256, 512])
    ap.add_argument("--unroll", type=int, nargs="+", default=[4, 8, 16, 32])
    ap.add_argument("--variants", type=int, nargs="+", default=[0])
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    rows = sweep(a.buf_gb, a.records, a.unroll, a.variants)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
