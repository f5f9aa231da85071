#!/usr/bin/env python3
"""Benchmark of the batched RAMBO query on one GB300.

One step = one pass of the whole query path (k-mer extraction, hashing,
probing, bucket-space AND, expansion to document masks) over one batch.  The
default workload is the large index: 10,000 documents x 500 kbp (200 seed
genomes, 0.5% substitutions, 0.05% indels), R=5, B=100, m=2^29, eta=2 (a
32 GiB index), and a batch of 10^5 sequences of U[31, 5000] bp, 70% drawn
from documents with 0.1% read errors.  The index is built once before timing
(build throughput is reported beside the query numbers); a sample of the
timed answers is checked against the CPU oracle.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large|medium|tiny|stream]

--impl reference times the CPU oracle (plain single-pass RAMBO in C) on the
host cores, on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1910_04358_gb300.autotune import effective_path  # noqa: E402  (no torch, no library)

METRIC = "k-mer queries/s and query bp/s on 1 GB300 (bit-exact vs oracle); serving p50/p99 ms"
UNIT = "k-mer queries/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
CSRC = os.path.join(ROOT, "paper_1910_04358_gb300", "csrc")
KERNEL_SRC = {"k_fused": "rambo_kernels_fused.cu", "k_probe_seqs": "rambo_kernels_probe.cu",
              "k_binned": "rambo_kernels_binned.cu", "k_segments": "rambo_kernels_segments.cu"}
SECTOR = 32
STAGES_ALL = ("prefix", "register", "insert", "probe_seqs", "probe_kmers", "expand")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
# workloads


def load_workload(name: str):
    from paper_1910_04358_gb300 import synth
    if name == "medium":
        corpus, kmers, q = synth.medium_workload()
        desc = ("1,000 docs x 1 Mbp (20 seed genomes, 1% substitutions); R=4 B=32 m=2^26 eta=2 k=31; "
                "batch = 10^6 single 31-mers (50% present) + 10^4 x 1 kbp sequences (50% from docs)")
    elif name == "large":
        corpus, q = synth.large_workload()
        kmers = np.zeros(0, np.uint64)
        desc = ("10,000 docs x 500 kbp (200 seeds, 0.5% subs, 0.05% indels); R=5 B=100 m=2^29 eta=2 "
                "k=31; batch = 10^5 sequences of U[31,5000] bp, 70% from docs with 0.1% errors")
    elif name == "tiny":
        corpus, q = synth.tiny_workload()
        kmers = np.zeros(0, np.uint64)
        desc = "100 docs x 20 kbp; R=2 B=10 m=2^20 eta=2; batch = 1,000 x 100 bp"
    else:
        raise SystemExit(f"unknown workload {name}")
    return corpus, kmers, q, desc


def batch_stats(p, kmers, q):
    n_seq_kmers = q.n_kmers(p.k)
    total_kmers = int(kmers.size) + n_seq_kmers
    bp = int(kmers.size) * p.k + q.n_bases
    return n_seq_kmers, total_kmers, bp


# ---------------------------------------------------------------------------
# clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []  # (t, sm, max, reasons)
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        threading.Thread(target=self._reader, daemon=True).start()

    def _reader(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = [n for n, v in zip(names, parts[5:9]) if v.lower() == "active"]
            self.samples.append((time.time(), sm, mx, reasons))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        inside = [s for s in self.samples if t0 <= s[0] <= t1]
        window = "timed region"
        if len(inside) < 3:  # short timed region: widen to the surrounding loaded window
            inside = [s for s in self.samples if t0 - 1.0 <= s[0] <= t1 + 0.3]
            window = "timed region +-1 s"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "window": "no samples"}
        reasons = sorted({r for s in inside for r in s[3]})
        return {"sm_mhz": statistics.median(s[1] for s in inside),
                "sm_max_mhz": max(s[2] for s in inside), "reasons": reasons,
                "samples": len(inside), "window": window}


# ---------------------------------------------------------------------------
# roofline helpers


def measured_peak_gbs():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def probe_bytes_per_kmer(info) -> int:
    """eta position groups per k-mer, each rounded up to whole 32-byte sectors."""
    g = info["group_bytes"]
    return info["eta"] * SECTOR * ((g + SECTOR - 1) // SECTOR)


def host_cpu() -> str:
    """Architecture, core count and model name of the host cores."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    arm_parts = {"0xd4f": "Arm Neoverse V2 (Grace)", "0xd40": "Arm Neoverse V1", "0xd4e": "Arm Cortex-X3"}
    model = arm_parts.get(model.lower(), model)
    return f"{platform.machine()}, {os.cpu_count()} cores" + (f", {model}" if model else "")


def probe_algorithmic_bytes(info, n_kmers: int, n_queries: int, n_bases: int) -> int:
    """Bytes the probe kernel must move: the index sectors of every probe, the
    packed input (1/4 byte per base), offsets and k-mer prefix (16 B/query)
    and the per-query bucket-mask write (group bytes per query)."""
    return (n_kmers * probe_bytes_per_kmer(info) + n_bases // 4 + 16 * n_queries
            + n_queries * info["group_bytes"])


def source_digest(path: str) -> str:
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_traffic_per_kmer(workload: str, kernel: str):
    """dram bytes per probed k-mer from a committed ncu capture of one batch
    (for workloads whose batches differ in size), if the sources are
    unchanged since the counters were taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            e = json.load(f)[workload][kernel]
        if e.get("source_sha") != kernel_digest(kernel) or not e.get("kmers_per_launch"):
            return None
        return float(e["dram_bytes_per_launch"]) / float(e["kmers_per_launch"])
    except Exception:
        return None


def measured_traffic(workload: str, kernel: str, n_kmers: int | None = None):
    """dram bytes per launch from a committed ncu capture, if the kernel's
    source (and the shared device headers) has not changed since the counters
    were taken; a capture of a reduced geometry gives bytes per k-mer, scaled
    to the n_kmers of the timed launch."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        e = t[workload][kernel]
        if e.get("source_sha") != kernel_digest(kernel):
            return None
        if e.get("kmers_per_launch"):
            if not n_kmers:
                return None
            return float(e["dram_bytes_per_launch"]) / float(e["kmers_per_launch"]) * n_kmers
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


def kernel_digest(kernel: str) -> str:
    h = hashlib.sha256()
    for f in (KERNEL_SRC[kernel], "rambo_query_common.cuh", "rambo_internal.cuh"):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# distributed plumbing (independent replicas; no data-path collective)


_NCCL_DEVICE = None  # this rank's GPU when the process group is NCCL


def dist_setup(backend: str, always: bool = False):
    """Rank, local rank and world size from the launcher's environment; the
    process group is started for more than one rank, or always when asked
    (a one-rank group needs MASTER_ADDR and MASTER_PORT, as torchrun sets)."""
    global _NCCL_DEVICE
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 or always:
        import torch.distributed as dist
        if backend == "nccl":
            import torch
            # bind the rank to its GPU before NCCL starts, so no collective
            # has to guess the device
            torch.cuda.set_device(local)
            _NCCL_DEVICE = local
            dist.init_process_group(backend=backend, device_id=torch.device(f"cuda:{local}"))
        else:
            dist.init_process_group(backend=backend)
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        if _NCCL_DEVICE is not None:
            dist.barrier(device_ids=[_NCCL_DEVICE])
        else:
            dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# serving (continuous batching vs plain fixed batches, same trace)


def serving_section(idx, corpus, n_req: int, fracs=(0.1, 0.25, 0.5, 0.75, 0.9, 1.1), seed: int = 4):
    """Poisson traces of n_req requests (log-normal lengths, median 300 bp,
    70% from documents with 0.1% errors) at fractions of the plain batched
    server's saturation rate, served by the continuous-batching engine and
    by plain 256-request batches; every answer of the engine is checked
    against the plain server's."""
    from paper_1910_04358_gb300 import serve, synth
    rng = np.random.default_rng([synth.GEN_SEED_BASE + 4, seed])
    _, lengths = synth.serving_trace(rng, n_req, rate_per_s=1.0)
    reqs0 = serve.make_requests(corpus, np.zeros(n_req), lengths, rng)
    eng = serve.ServingEngine(idx, slots=4)
    eng.serve(reqs0[: min(n_req, 2000)])  # warm
    serve.plain_batched(idx, reqs0[: min(n_req, 2000)], batch_size=256)
    # saturation: every request present at t = 0
    plain_sat = serve.plain_batched(idx, reqs0, batch_size=256)
    cont_sat = eng.serve(reqs0)
    same = bool(np.array_equal(plain_sat.answers, cont_sat.answers))
    ps, cs = plain_sat.summary(), cont_sat.summary()
    sat_rps = n_req / ps["wall_s"]
    one = serve.one_batch_rate(idx, reqs0)
    out = {"requests_per_rate": n_req, "length_dist": "log-normal median 300 bp, sigma 1, [31, 10^4]",
           "rates_relative_to": "plain 256-request batches at saturation",
           "saturation": {"plain_batch256": {"requests_per_s": sat_rps, "bp_per_s": ps["bp_per_s"],
                                             "p50_ms": ps["p50_ms"], "p99_ms": ps["p99_ms"]},
                          "continuous": {"requests_per_s": n_req / cs["wall_s"], "bp_per_s": cs["bp_per_s"],
                                         "p50_ms": cs["p50_ms"], "p99_ms": cs["p99_ms"],
                                         "batches": cs["batches"],
                                         "frac_of_one_batch_device_rate": cs["bp_per_s"] / one["bp_per_s"]},
                          "one_batch_device": one},
           "rates": []}
    for f in fracs:
        arrivals = np.cumsum(rng.exponential(1.0 / (f * sat_rps), size=n_req))
        reqs = [serve.Request(r.rid, r.packed, r.n_bases, float(a)) for r, a in zip(reqs0, arrivals)]
        cont = eng.serve(reqs)
        plain = serve.plain_batched(idx, reqs, batch_size=256)
        same = same and bool(np.array_equal(cont.answers, plain.answers))
        c, pl = cont.summary(), plain.summary()
        out["rates"].append({"offered_frac_of_saturation": f, "offered_requests_per_s": f * sat_rps,
                             "continuous": {k: c[k] for k in ("p50_ms", "p99_ms", "bp_per_s", "batches", "max_in_flight")},
                             "plain_batch256": {k: pl[k] for k in ("p50_ms", "p99_ms", "bp_per_s", "batches")}})
    out["answers_identical"] = same
    return out


# ---------------------------------------------------------------------------
# CPU oracle legs


def sample_fracs(workload: str):
    """Every fk-th single k-mer and every fs-th sequence of the batch form
    the oracle's sample (sequences of every length bucket)."""
    return (200, 100) if workload == "medium" else (1, 50)


class OracleSample:
    """Restricted-mode oracle for a sample of the batch: it tracks only the
    probe positions the sample touches, which is exact for those queries."""

    def __init__(self, p, kmers, q, frac_kmers: int, frac_seqs: int):
        import oracle
        from paper_1910_04358_gb300 import synth
        self.p = p
        self.ks = kmers[::frac_kmers] if kmers.size else kmers
        self.k_sel = np.arange(0, kmers.size, frac_kmers)
        self.sel = np.arange(0, q.n, frac_seqs)
        offs = q.offsets.astype(np.int64)
        stream = synth.PackedStream()
        for i in self.sel:
            stream.append(synth.unpack_bases(q.packed, int(offs[i]), int(offs[i + 1] - offs[i])))
        self.s_packed, self.s_offs = stream.finish()
        self.o = oracle.tracking_oracle(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed,
                                        seqs=[(self.s_packed, self.s_offs)], kmers=self.ks)
        self.build_s = None
        self.want_k = self.want_s = None
        self.error = None
        self._thread = None

    def build(self, corpus, threads: int):
        t0 = time.time()
        self.o.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets, threads=threads)
        self.build_s = time.time() - t0

    def answer(self, threads: int):
        self.want_k = self.o.query_kmers(self.ks, threads=threads) if self.ks.size else None
        self.want_s = self.o.query_seqs(self.s_packed, self.s_offs, threads=threads)

    def start(self, corpus, threads: int):
        """Builds and answers on a host thread (the C oracle releases the
        interpreter lock), so the GPU sections run meanwhile."""
        def run():
            try:
                self.build(corpus, threads)
                self.answer(threads)
            except Exception as ex:  # reported by check()
                self.error = repr(ex)
        self._thread = threading.Thread(target=run, daemon=True)
        self._thread.start()

    def join(self):
        if self._thread is not None:
            self._thread.join()
            self._thread = None

    def check(self, out_k, out_s) -> dict:
        """Compares the sampled rows of the GPU outputs with the oracle."""
        from paper_1910_04358_gb300 import rambo
        self.join()
        if self.error:
            return {"ok": False, "error": self.error}
        got_s = rambo.as_u32(out_s)[self.sel]
        bad_s = int(np.sum(np.any(got_s != self.want_s, axis=1)))
        bad_k = 0
        if self.want_k is not None and out_k is not None:
            got_k = rambo.as_u32(out_k)[self.k_sel]
            bad_k = int(np.sum(np.any(got_k != self.want_k, axis=1)))
        L = np.diff(self.s_offs.astype(np.int64))
        return {"ok": bad_s == 0 and bad_k == 0, "sequences_checked": int(self.sel.size),
                "kmers_checked": int(self.ks.size), "mismatched_sequences": bad_s,
                "mismatched_kmers": bad_k,
                "sequence_lengths": [int(L.min()), int(L.max())] if L.size else None,
                "oracle_build_s": self.build_s,
                "what": "the timed step's answers, sampled rows, vs the restricted-mode CPU oracle"}


def time_oracle(o, ks, s_packed, s_offs, threads: int):
    t0 = time.perf_counter()
    if ks.size:
        o.query_kmers(ks, threads=threads)
    if s_offs.size > 1:
        o.query_seqs(s_packed, s_offs, threads=threads)
    return time.perf_counter() - t0


def sample_kmers_count(p, ks, s_offs):
    L = np.diff(s_offs.astype(np.int64))
    return int(ks.size) + int(np.maximum(L - p.k + 1, 0).sum())


def run_reference(args):
    rank, local, world = dist_setup("gloo")
    if rank != 0:
        return 0
    corpus, kmers, q, desc = load_workload(args.workload)
    p = corpus.params
    threads = os.cpu_count() or 1
    fk, fs = sample_fracs(args.workload)
    log(f"[reference] building restricted-mode oracle index on {threads} threads")
    osm = OracleSample(p, kmers, q, fk, fs)
    osm.build(corpus, threads)
    ks, sp, so = osm.ks, osm.s_packed, osm.s_offs
    units = sample_kmers_count(p, ks, so)
    bp = int(ks.size) * p.k + int(so[-1])
    for _ in range(args.warmup):
        time_oracle(osm.o, ks, sp, so, threads)
    times = [time_oracle(osm.o, ks, sp, so, threads) for _ in range(args.steps)]
    total = sum(times)
    value = units * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "desc": desc, "sample": f"1/{fk} of k-mers, 1/{fs} of sequences"},
        "query_bp_per_s": bp * len(times) / total,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{ks.size} k-mers + {so.size - 1} sequences per step "
                                   f"({units} k-mers), restricted-mode index built in {osm.build_s:.1f} s",
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm


def run_stream(args):
    """Streaming update + query: epochs of document inserts, each followed by a
    query batch over everything inserted so far.  All 100 epochs are
    inserted; a step is one epoch's query batch, and the last `steps`
    epochs' batches are timed (the index then holds 9x,000 - 100,000
    documents, 64 GiB); inserts are timed separately."""
    import torch
    rank, local, world = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_1910_04358_gb300 import rambo, synth
    wl = synth.stream_workload()
    p = wl.params
    idx = rambo.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, device=local)
    idx.set_tuning(query_path=args.query_path if args.query_path is not None else 1)
    info = idx.info
    # the epochs' batches differ a little in k-mers per query, so the cached
    # tuning is kept per index geometry and epoch batch size; without one, the
    # autotuner runs on the first epoch's batch, after that epoch
    tuned, cached, tuning_source = None, None, "default (query_path=1)"
    autotuning = not args.no_autotune and args.query_path is None
    if autotuning:
        from paper_1910_04358_gb300 import autotune
        key = autotune.cache_key(idx, wl.queries_per_epoch, 0).rsplit("_kpq", 1)[0] + "_stream"
        cached = None if args.retune else autotune.load_cached(autotune.CACHE_FILE, key)
        if cached:
            idx.set_tuning(**cached)
            tuning_source = f"cached ({os.path.relpath(autotune.CACHE_FILE, ROOT)})"
    to_dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(dev)
    n_epochs = wl.n_epochs
    first_timed = max(0, n_epochs - args.steps)
    stream = torch.cuda.current_stream()
    q_ms, q_kmers, q_bp, ins_ms, ins_kmers, timed = 0.0, 0, 0, 0.0, 0, 0
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.time()
    for e in range(n_epochs):
        (ids, packed, offs), q = wl.epoch(e)
        d_ids, d_p, d_o = to_dev(ids, np.int32), to_dev(packed, np.uint8), to_dev(offs, np.int64)
        d_qp, d_qo = to_dev(q.packed, np.uint8), to_dev(q.offsets, np.int64)
        out = torch.empty((q.n, idx.W), dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        if e == first_timed:
            t_wall0 = time.time()  # the clock record covers the timed epochs
        ev[0].record(stream)
        idx.insert_batch_dev(d_ids, d_p, d_o)
        ev[1].record(stream)
        idx.query_seqs_dev(d_qp, d_qo, out=out)
        ev[2].record(stream)
        torch.cuda.synchronize()
        if e >= first_timed:
            ins_ms += ev[0].elapsed_time(ev[1])
            q_ms += ev[1].elapsed_time(ev[2])
            ins_kmers += int(np.maximum(np.diff(offs.astype(np.int64)) - p.k + 1, 0).sum())
            q_kmers += q.n_kmers(p.k)
            q_bp += q.n_bases
            timed += 1
        if e == 0 and autotuning and not cached:
            tuned = autotune.autotune(idx, lambda: idx.query_seqs_dev(d_qp, d_qo, out=out),
                                      lambda: [out], reps=5)
            log(f"[autotune] best {tuned['best']} {tuned['ms']:.4f} ms/batch")
            autotune.store_cached(autotune.CACHE_FILE, key, tuned["best"])
            tuning_source = "autotuned in this run (first epoch's batch)"
    idx.sync()
    t_wall1 = time.time()
    clocks.stop()
    ms_step = q_ms / max(timed, 1)
    # early exit on the last epoch's batch (the full index; identical answers,
    # k-mers actually probed); reported beside the line, never as `value`
    early = None
    if not args.no_early_exit:
        saved = idx.get_tuning()
        ref = out.clone()
        idx.set_tuning(early_exit=1, query_path=1, fused_short_max=max(saved["fused_short_max"], 1024))
        idx.probed_kmers(reset=True)
        idx.query_seqs_dev(d_qp, d_qo, out=out)
        idx.sync()
        probed = idx.probed_kmers(reset=True)
        same = bool(torch.equal(out, ref))
        ev[0].record(stream)
        for _ in range(3):
            idx.query_seqs_dev(d_qp, d_qo, out=out)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms_ee = ev[0].elapsed_time(ev[1]) / 3
        nk_last = q.n_kmers(p.k)
        early = {"ms_per_batch": ms_ee, "kmer_queries_per_s": nk_last / (ms_ee / 1e3),
                 "seq_kmers_probed": probed, "seq_kmers": nk_last,
                 "probed_frac": probed / max(nk_last, 1), "answers_identical": same,
                 "batch": "the last epoch's query batch"}
        idx.set_tuning(**saved)
    peak, peak_src = measured_peak_gbs()
    kpb = probe_bytes_per_kmer(info)
    # DRAM bytes of the fused launch, scaled from the captured batch by k-mers
    per_kmer = measured_traffic_per_kmer("stream", "k_fused") \
        if effective_path(idx.get_tuning(), info) == 1 else None
    traffic = per_kmer * q_kmers / max(timed, 1) if per_kmer else None
    line = {
        "metric": METRIC, "value": q_kmers / (q_ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": timed, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded)",
        "config": {"workload": "stream", "desc": "100,000 docs x 50 kbp from 2,000 seeds at 1%; "
                   "R=6 B=316 m=2^28 eta=2 k=31 (64 GiB index); all 100 epochs of 1,000 docs "
                   "inserted, the last epochs' query batches timed; each epoch "
                   "followed by 10^4 queries of U[31,2000] bp (70% from inserted docs)",
                   "l2": "inputs larger than L2: index %.1f GB" % (info["index_bytes"] / 1e9)},
        "query_bp_per_s": q_bp / (q_ms / 1e3),
        "insert": {"kmers_per_s": ins_kmers / (ins_ms / 1e3), "ms_per_epoch": ins_ms / max(timed, 1)},
        "roofline": {"bound": "hbm", "kernel": "query step (all query kernels)",
                     "achieved": q_kmers * kpb / (q_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": q_kmers * kpb / (q_ms / 1e3) / 1e9 / peak, "traffic": traffic,
                     "dram_bytes_per_kmer": per_kmer,
                     "dram_gbs": traffic / (ms_step / 1e3) / 1e9 if traffic else None,
                     "dram_frac_of_peak": traffic / (ms_step / 1e3) / 1e9 / peak if traffic else None,
                     "traffic_source": ("profiles/traffic.json (one batch's ncu capture, scaled by "
                                        "k-mers per batch)") if traffic else None,
                     "bytes_per_kmer": kpb, "peak_source": peak_src},
        "clocks": clocks.summary(t_wall0, t_wall1), "tuning": idx.get_tuning(),
        "tuning_source": tuning_source,
        "autotune": ({"trials": len(tuned["trials"]), "best_ms": tuned["ms"]} if tuned else None),
        "early_exit": early,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    idx.close()
    return 0


def run_sharded(args):
    """--gpus N > 1: a document-sharded large index (Section 5.3).  Rank r
    holds shard r, 10,000 documents of the large workload's recipe (shard 0
    is the large corpus itself) as global documents r*10,000 .. r*10,000 +
    9,999, and answers the same batch (the large workload's 10^5 sequences)
    on it; one all_gather exchanges the shards' answers and every rank merges
    them into the global answers (N*10,000 documents).  A step is that whole
    pass.  Per-GPU work is one shard, fixed as N grows (weak scaling); the
    units are k-mer queries against one shard, N per query k-mer."""
    import torch
    import torch.distributed as dist
    rank, local, world = dist_setup("nccl", always=True)
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_1910_04358_gb300 import autotune, rambo, sharding, synth
    t_start = time.time()
    corpus0, q = synth.large_workload()
    corpus = corpus0 if rank == 0 else synth.large_shard_corpus(rank)
    del corpus0
    p = corpus.params
    n_seq_kmers, total_kmers, bp = batch_stats(p, np.zeros(0, np.uint64), q)
    log(f"[bench] rank {rank}: shard generated in {time.time() - t_start:.1f} s")
    osm = None
    if rank == 0 and not args.no_oracle_check:
        fk, fs = sample_fracs("large")
        osm = OracleSample(p, np.zeros(0, np.uint64), q, fk, fs)
        osm.start(corpus, max(1, (os.cpu_count() or 1) - 2))
    to_dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(dev)
    idx = rambo.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, device=local)
    cached = autotune.load_cached(autotune.CACHE_FILE, autotune.cache_key(idx, q.n, total_kmers))
    if cached:
        idx.set_tuning(**cached)
    idx.insert_batch_dev(to_dev(corpus.doc_ids, np.int32), to_dev(corpus.packed, np.uint8),
                         to_dev(corpus.offsets, np.int64))
    idx.sync()
    K_all = world * p.K
    member_lists = [np.arange(s * p.K, (s + 1) * p.K) for s in range(world)]
    d_qp, d_qo = to_dev(q.packed, np.uint8), to_dev(q.offsets, np.int64)
    local_out = torch.empty((q.n, idx.W), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        idx.query_batch_dev(None, d_qp, d_qo, out_seqs=local_out)
        return sharding.gather_answers(local_out, member_lists, K_all)

    for _ in range(args.warmup):
        step()
    idx.sync()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    idx.profile_reset(timed_stages=("probe_seqs",))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    t_wall0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        glob = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier(world)
    idx.sync()
    time.sleep(0.2)
    clocks.stop()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1), world, dev) / args.steps
    prof = idx.profile_read()
    launches = sum(v["launches"] for v in prof.values()) + args.steps * world  # + one merge kernel per shard
    dom_ms = prof["probe_seqs"]["ms"] / max(prof["probe_seqs"]["timed"], 1)
    info = idx.info
    alg_bytes = probe_algorithmic_bytes(info, n_seq_kmers, q.n, q.n_bases)
    if effective_path(idx.get_tuning(), info) == 1:
        alg_bytes += q.n * idx.W * 4
    peak, peak_src = measured_peak_gbs()
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9
    # the oracle check covers shard 0's documents, the first 10,000 global bits
    oracle_check = None
    if osm is not None:
        first = glob[:, : (p.K + 31) // 32].clone()
        if p.K % 32:
            first[:, -1] &= (1 << (p.K % 32)) - 1
        oracle_check = osm.check(None, first)
    # end to end: page-locked inputs in, the global answers out on every rank
    pin_p = torch.from_numpy(q.packed).pin_memory()
    pin_o = torch.from_numpy(q.offsets.view(np.int64)).pin_memory()
    pin_out = torch.empty(glob.shape, dtype=torch.int32).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))

    def step_e2e():
        d_qp.copy_(pin_p, non_blocking=True)
        d_qo.copy_(pin_o, non_blocking=True)
        g = step()
        pin_out.copy_(g, non_blocking=True)
        torch.cuda.synchronize()

    step_e2e()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_e2e()
    t_e2e = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)
    value = world * total_kmers / (ms_step / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded)",
        "config": {"workload": "large", "parallelism": f"document shards x{world}",
                   "desc": (f"document-sharded large index: {world} shards of 10,000 docs x 500 kbp "
                            "(R=5 B=100 m=2^29 eta=2 k=31, 32 GiB each), one per GPU, global documents "
                            f"0..{K_all - 1}; batch = the large workload's 10^5 sequences of U[31,5000] bp "
                            "sent to every shard; answers exchanged with one all_gather and merged"),
                   "units": "k-mer queries against one shard (N per query k-mer)",
                   "l2": "inputs larger than L2: index %.2f GB per GPU probed at random" % (info["index_bytes"] / 1e9)},
        "query_bp_per_s": world * bp / (ms_step / 1e3), "kmers_per_step": world * total_kmers,
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_fused_prep+k_fused (per rank)",
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": dom_ms,
                     "peak_source": peak_src},
        "clocks": clocks.summary(t_wall0, t_wall1),
        "e2e": {"value": world * total_kmers / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": int(q.packed.nbytes + q.offsets.nbytes),
                "d2h_bytes_per_step": int(glob.numel() * 4), "ms_per_step": 1e3 * t_e2e},
        "cpu_baseline": None, "oracle_check": oracle_check,
        "tuning": idx.get_tuning(), "tuning_source": "cached" if cached else "default",
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    idx.close()
    dist.destroy_process_group()
    return 0 if oracle_check is None or oracle_check["ok"] else 1


def run_ours(args):
    import torch
    rank, local, world = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_1910_04358_gb300 import rambo

    t_start = time.time()
    corpus, kmers, q, desc = load_workload(args.workload)
    p = corpus.params
    n_seq_kmers, total_kmers, bp = batch_stats(p, kmers, q)
    log(f"[bench] workload {args.workload} generated in {time.time() - t_start:.1f} s")
    # the oracle's sample of this batch, built on host threads while the GPU
    # sections run (rank 0 only); the timed answers are checked against it
    osm = None
    if rank == 0 and not args.no_oracle_check:
        fk, fs = sample_fracs(args.workload)
        osm = OracleSample(p, kmers, q, fk, fs)
        osm.start(corpus, max(1, (os.cpu_count() or 1) - 2))

    def to_dev(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(dev)

    idx = rambo.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, device=local)
    if args.query_path is not None:
        idx.set_tuning(query_path=args.query_path)
    info = idx.info
    tuned = None
    tuning_source = "default"
    cached = None
    if not args.no_autotune and args.query_path is None:
        from paper_1910_04358_gb300 import autotune
        key = autotune.cache_key(idx, q.n + int(kmers.size), total_kmers)
        cached = None if args.retune else autotune.load_cached(autotune.CACHE_FILE, key)
        if cached:  # applied before the build (its insert mode) and the warm-up steps
            idx.set_tuning(**cached)
            tuning_source = f"cached ({os.path.relpath(autotune.CACHE_FILE, ROOT)})"
    # ---- build (Algorithm 1), timed separately
    d_ids, d_cp, d_co = to_dev(corpus.doc_ids, np.int32), to_dev(corpus.packed, np.uint8), \
        to_dev(corpus.offsets, np.int64)
    torch.cuda.synchronize()
    idx.profile_reset(timed_stages=("insert",))
    t0 = time.perf_counter()
    idx.insert_batch_dev(d_ids, d_cp, d_co)
    idx.sync()
    build_s = time.perf_counter() - t0
    prof_b = idx.profile_read()
    insert_kmers = int(np.maximum(np.diff(corpus.offsets.astype(np.int64)) - p.k + 1, 0).sum())
    del d_cp
    torch.cuda.empty_cache()

    # ---- query batch resident in HBM
    d_k = to_dev(kmers, np.int64) if kmers.size else None
    d_qp, d_qo = to_dev(q.packed, np.uint8), to_dev(q.offsets, np.int64)
    out_k = torch.empty((kmers.size, idx.W), dtype=torch.int32, device=dev) if kmers.size else None
    out_s = torch.empty((q.n, idx.W), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        # one call per batch: the k-mer part runs on the library's side
        # stream next to the sequence part (forked from and joined back to
        # the current stream)
        idx.query_batch_dev(d_k, d_qp, d_qo, out_kmers=out_k, out_seqs=out_s)

    def step_serial():
        # the two parts one after the other on one stream (stage breakdown)
        if d_k is not None:
            idx.query_kmers_dev(d_k, out=out_k)
        idx.query_seqs_dev(d_qp, d_qo, out=out_s)

    for _ in range(args.warmup):
        step()
    idx.sync()
    if not args.no_autotune and args.query_path is None:
        if not cached:
            outs = lambda: [t for t in (out_k, out_s) if t is not None]
            tuned = autotune.autotune(idx, step, outs, reps=7)
            log(f"[autotune] best {tuned['best']} {tuned['ms']:.4f} ms/step")
            autotune.store_cached(autotune.CACHE_FILE, key, tuned["best"])
            tuning_source = "autotuned in this run"
        for _ in range(3):
            step()
        idx.sync()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    idx.profile_reset(timed_stages=("probe_seqs", "probe_kmers"))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    t_wall0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier(world)
    idx.sync()
    time.sleep(0.2)
    clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    # the timed steps' answers, kept for the oracle check
    timed_k = out_k.clone() if out_k is not None else None
    timed_s = out_s.clone()
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_step = ms_total / args.steps
    prof = idx.profile_read()
    launches = sum(v["launches"] for v in prof.values())
    ms_step_eager = ms_step

    # ---- the same steps replayed from a captured CUDA graph (launch overhead gone)
    graph = None
    if not args.no_graph:
        try:
            idx.profile_reset()  # counting only: no event records inside the capture
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step()
            per_step_launches = sum(v["launches"] for v in idx.profile_read().values())
            g.replay()
            torch.cuda.synchronize()
            barrier(world)
            torch.cuda.synchronize()
            gs = torch.cuda.current_stream()
            ev0.record(gs)
            for _ in range(args.steps):
                g.replay()
            ev1.record(gs)
            torch.cuda.synchronize()
            barrier(world)
            ms_g = max_over_ranks(ev0.elapsed_time(ev1), world, dev) / args.steps
            # spread: 10 timed replays of one step each
            singles = []
            for _ in range(10):
                ev0.record(gs)
                g.replay()
                ev1.record(gs)
                torch.cuda.synchronize()
                singles.append(ev0.elapsed_time(ev1))
            graph = {"ms_per_step": ms_g, "launches_per_step": per_step_launches,
                     "single_step_ms": {"best": min(singles),
                                        "median": statistics.median(singles)}}
            if ms_g < ms_step:
                ms_step = ms_g
                launches = per_step_launches * args.steps
            # the graph's answers are the eager answers
            ok_graph = torch.equal(out_s, idx.query_seqs_dev(d_qp, d_qo))
            idx.sync()
            graph["answers_match_eager"] = bool(ok_graph)
        except Exception as ex:
            graph = {"error": repr(ex)}
    # ---- early exit (the paper's "first FALSE is conclusive", Section 3.3.1;
    # RAMBO+ sparse evaluation, Section 5.1): identical answers, fewer k-mers
    # probed.  Reported beside the line, never as `value` (which probes every k-mer).
    early = None
    if not args.no_early_exit and q.n:
        saved = idx.get_tuning()
        ref_s = out_s.clone()
        ref_k = out_k.clone() if out_k is not None else None
        try:
            # early exit is a fused-path option; it is checked inside a query
            # probed whole by one warp, so the batch's 1 kbp queries are kept short
            idx.set_tuning(early_exit=1, query_path=1,
                           fused_short_max=max(saved["fused_short_max"], 1024))
            idx.probed_kmers(reset=True)
            step()
            idx.sync()
            probed = idx.probed_kmers(reset=True)
            same = torch.equal(out_s, ref_s) and (ref_k is None or torch.equal(out_k, ref_k))
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.steps):
                step()
            ev1.record(stream)
            torch.cuda.synchronize()
            ms_ee = ev0.elapsed_time(ev1) / args.steps
            spk = probe_bytes_per_kmer(info) // SECTOR
            early = {"ms_per_step": ms_ee, "kmer_queries_per_s": total_kmers / (ms_ee / 1e3),
                     "seq_kmers_probed": probed, "seq_kmers": n_seq_kmers,
                     "probed_frac": probed / max(n_seq_kmers, 1),
                     "index_sectors_per_step": (probed + int(kmers.size)) * spk,
                     "index_sectors_per_step_without": total_kmers * spk,
                     "answers_identical": bool(same), "segment": saved["early_exit_segment"]}
        except Exception as ex:  # report, do not hide
            early = {"error": repr(ex)}
        finally:
            idx.set_tuning(**saved)
            idx.sync()
    # per-stage breakdown from a separate profiled pass (every stage bracketed)
    idx.profile_reset(timed_stages=STAGES_ALL)
    for _ in range(min(args.steps, 20)):
        step_serial()
    idx.sync()
    prof_all = idx.profile_read()

    value = total_kmers * world / (ms_step / 1e3)
    bp_s = bp * world / (ms_step / 1e3)
    launch_mode = "cuda graph replay" if graph and graph.get("ms_per_step") == ms_step else "eager"

    # ---- roofline of the dominant kernel (sequence probe)
    dom = "probe_seqs" if q.n else "probe_kmers"
    dom_ms = prof[dom]["ms"] / max(prof[dom]["timed"], 1)
    alg_bytes = probe_algorithmic_bytes(info, n_seq_kmers, q.n, q.n_bases)
    path = effective_path(idx.get_tuning(), info)
    if path == 1:  # the fused launch also writes the answer masks
        alg_bytes += q.n * idx.W * 4
    peak, peak_src = measured_peak_gbs()
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9
    src_key = {0: "k_probe_seqs", 1: "k_fused", 2: "k_binned", 3: "k_segments"}[path]
    traffic = measured_traffic(args.workload, src_key, n_seq_kmers)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "frac_of_spec_7900": achieved / 7900.0,
                "dram_bytes_per_kmer": (traffic / n_seq_kmers) if traffic and n_seq_kmers else None,
                # DRAM bytes the kernel really moves (ncu, per launch) over its live launch
                # time: how busy the DRAM system is, 128-byte line fills included
                "dram_gbs": (traffic / (dom_ms / 1e3) / 1e9) if traffic else None,
                "dram_frac_of_peak": (traffic / (dom_ms / 1e3) / 1e9 / peak) if traffic else None,
                "random_line_ceiling": "45-51 G random 128-byte lines/s measured "
                                       "(profiles/k_gather_random_records.md)",
                "traffic_source": ("profiles/traffic.json: ncu DRAM bytes per k-mer on a reduced "
                                   "geometry of this kernel, scaled by the batch's k-mers") if traffic else None,
                "kernel": {0: "k_probe_seqs", 1: "k_fused_prep+k_fused",
                           2: "k_bin_tiles+k_bin_scatter+k_bin_probe",
                           3: "k_seg_cut+k_seg_scan+k_seg_place+segment prefix+k_seg_chunks+k_seg_probe"}[path],
                "algorithmic_bytes_per_launch": alg_bytes,
                "bytes_per_kmer": probe_bytes_per_kmer(info), "avg_launch_ms": dom_ms,
                "peak_source": peak_src}
    kernel_ms = {k: (v["ms"] / (min(args.steps, 20)) if v["timed"] else None)
                 for k, v in prof_all.items()}

    # ---- the timed answers against the CPU oracle (sampled rows; rank 0)
    log(f"[bench] GPU sections done at {time.time() - t_start:.1f} s; waiting for the oracle")
    oracle_check = osm.check(timed_k, timed_s) if osm is not None else None
    log(f"[bench] oracle check {oracle_check} at {time.time() - t_start:.1f} s")
    del timed_k, timed_s
    ok = oracle_check is None or bool(oracle_check["ok"])

    # ---- end to end through the host-buffer C ABI (H2D + D2H inside)
    e2e = None
    if not args.no_e2e:
        pin_k = torch.from_numpy(kmers.view(np.int64)).pin_memory().numpy().view(np.uint64) \
            if kmers.size else kmers
        pin_p = torch.from_numpy(q.packed).pin_memory().numpy()
        pin_o = torch.from_numpy(q.offsets.view(np.int64)).pin_memory().numpy().view(np.uint64)
        pin_ok = torch.empty((kmers.size, idx.W), dtype=torch.int32).pin_memory().numpy() \
            if kmers.size else None
        pin_os = torch.empty((q.n, idx.W), dtype=torch.int32).pin_memory().numpy()
        e2e_steps = max(3, min(args.steps, 30))
        for _ in range(2):
            idx.query_batch(pin_k, pin_p, pin_o, out_kmers=pin_ok, out_seqs=pin_os)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            idx.query_batch(pin_k, pin_p, pin_o, out_kmers=pin_ok, out_seqs=pin_os)
        t_e2e = (time.perf_counter() - t0) / e2e_steps
        t_e2e = max_over_ranks(t_e2e, world, dev)
        h2d = int(kmers.nbytes) + int(q.packed.nbytes) + int(q.offsets.nbytes)
        d2h = (int(kmers.size) + q.n) * idx.W * 4
        e2e = {"value": total_kmers * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * t_e2e, "steps": e2e_steps}

    log(f"[bench] e2e done at {time.time() - t_start:.1f} s")
    # ---- serving: continuous batching on the same resident index
    serving = None
    if not args.no_serving and rank == 0:
        try:
            serving = serving_section(idx, corpus, args.serving_requests)
        except Exception as ex:  # report, do not hide
            serving = {"error": repr(ex)}

    log(f"[bench] serving done at {time.time() - t_start:.1f} s")
    # ---- CPU oracle baseline (rank 0, N = 1 only): the oracle as it stands,
    # timed on the host cores on the checked sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and osm is not None and not osm.error:
        threads = os.cpu_count() or 1
        units = sample_kmers_count(p, osm.ks, osm.s_offs)
        reps, spent = 0, 0.0
        while spent < 10.0 and reps < 200:
            spent += time_oracle(osm.o, osm.ks, osm.s_packed, osm.s_offs, threads)
            reps += 1
        cpu = {"value": units * reps / spent, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{osm.ks.size} single k-mers + {osm.s_offs.size - 1} sequences ({units} k-mers) "
                         f"x {reps} repetitions; restricted-mode oracle index "
                         f"(tracks the sample's probe positions), built in {osm.build_s:.1f} s",
               "host": host_cpu()}

    clk = clocks.summary(t_wall0, t_wall1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "desc": desc,
                   "l2": "inputs larger than L2: index %.2f GB probed at random" % (info["index_bytes"] / 1e9),
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "query_bp_per_s": bp_s, "kmers_per_step": total_kmers, "bp_per_step": bp,
        "gpu_launches": launches, "roofline": roofline, "stage_ms_per_step": kernel_ms,
        "build": {"seconds": build_s, "kmers": insert_kmers, "kmers_per_s": insert_kmers / build_s,
                  "insert_kernel_ms": prof_b["insert"]["ms"] or None,
                  "insert_mode": idx.get_tuning()["insert_mode"]},
        "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "oracle_check": oracle_check,
        "launch_mode": launch_mode, "eager_ms_per_step": ms_step_eager, "graph": graph,
        "tuning": idx.get_tuning(), "tuning_source": tuning_source, "serving": serving,
        "early_exit": early,
        "autotune": ({"trials": len(tuned["trials"]), "best_ms": tuned["ms"]} if tuned else None),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    idx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0 if ok else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["medium", "large", "tiny", "stream"], default="large")
    ap.add_argument("--sharded", action="store_true",
                    help="document-sharded run (the default for more than one rank; one rank needs torchrun)")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the CPU oracle check of the timed answers")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--retune", action="store_true", help="autotune even if a cached tuning exists")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-early-exit", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=20000)
    ap.add_argument("--query-path", type=int, default=None,
                    help="0 = prefix/probe/expand launches, 1 = persistent fused launch")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "stream":
        return run_stream(args)
    if (int(os.environ.get("WORLD_SIZE", "1")) > 1 or args.sharded) and args.workload == "large":
        return run_sharded(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
