"""Hardware-rate probes behind two design choices.

  l2   64-bit atomicOr at hashed addresses of buffers of several sizes: the
       rate inside L2 (what the region-binned insert's apply pass can reach)
       against the rate over a buffer far larger than L2 (what the direct
       insert meets).
  tmem tensor-memory reads, one CTA per SM, by warps and loads in flight: the
       rate an epilogue can drain accumulators at.

  python -m paper_1910_04358_gb300.hw_probe [--l2-mib 8 32 64 4096] [--tmem]

Prints one JSON object per point.
"""
from __future__ import annotations

import argparse
import json
import sys


def l2_atomics(sizes_mib, ops=256, blocks_per_sm=8, reps=5):
    import torch

    from . import rambo
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = sms * blocks_per_sm
    for mib in sizes_mib:
        words = (mib << 20) // 8
        buf = torch.zeros(words, dtype=torch.int64, device="cuda")
        rambo.probe_l2_atomics(buf, ops, blocks)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            rambo.probe_l2_atomics(buf, ops, blocks)
        e1.record()
        torch.cuda.synchronize()
        n = reps * blocks * 256 * ops
        yield {"probe": "l2_atomics", "buffer_mib": mib,
               "g_atomicor_per_s": n / (e0.elapsed_time(e1) / 1e3) / 1e9}
        del buf
        torch.cuda.empty_cache()


def tmem_read(iters=20000):
    import torch

    from . import rambo
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cycles = torch.zeros(sms, dtype=torch.int64, device="cuda")
    for warps in (4, 8, 16):
        sink = torch.zeros(sms * warps * 32, dtype=torch.int32, device="cuda")
        for lif in (1, 2, 4):
            it = max(1, iters // lif)
            rambo.probe_tmem_read(warps, lif, 10, sink, cycles)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rambo.probe_tmem_read(warps, lif, it, sink, cycles)
            e1.record()
            torch.cuda.synchronize()
            per_cta = warps * it * lif * 4096
            c0 = int(cycles[0].item())
            yield {"probe": "tmem_read", "warps": warps, "loads_in_flight": lif,
                   "bytes_per_cycle_per_sm": per_cta / max(c0, 1),
                   "tb_per_s": sms * per_cta / (e0.elapsed_time(e1) / 1e3) / 1e12}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--l2-mib", type=int, nargs="*", default=[8, 32, 64, 4096])
    ap.add_argument("--tmem", action="store_true", help="also the tensor-memory read probe")
    a = ap.parse_args(argv)
    for row in l2_atomics(a.l2_mib):
        print(json.dumps(row), flush=True)
    if a.tmem:
        for row in tmem_read():
            print(json.dumps(row), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
