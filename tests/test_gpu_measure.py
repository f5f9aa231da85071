"""Measurement support and failure detection on the GPU (no fault, no hang).

* the random-gather probe runs and rejects record sizes it does not serve;
* the host-write probe copies into page-locked memory and refuses pageable
  memory before launching anything;
* a bounded device wait that nothing completes reports RAMBO_ETIMEOUT at the
  next sync, and the handle keeps answering queries correctly afterwards.
"""
import numpy as np
import pytest

import oracle
from paper_1910_04358_gb300 import synth

pytestmark = pytest.mark.gpu


def test_gather_probe_runs_and_checks_record_size(rambo_lib):
    import torch
    buf = torch.ones(1 << 20, dtype=torch.uint8, device="cuda")
    sink = rambo_lib.probe_gather(buf, 16, 1 << 16)
    torch.cuda.synchronize()
    assert sink.numel() == 1
    with pytest.raises(rambo_lib.RamboError):
        rambo_lib.probe_gather(buf, 24, 1 << 10)


def test_host_write_probe_copies_into_pinned_and_refuses_pageable(rambo_lib):
    import torch
    src = torch.arange(1 << 16, dtype=torch.int32, device="cuda").view(torch.uint8)
    dst = torch.zeros(src.numel(), dtype=torch.uint8).pin_memory()
    rambo_lib.probe_host_write(src, dst, 2)
    torch.cuda.synchronize()
    assert torch.equal(dst, src.cpu())
    with pytest.raises(rambo_lib.RamboError):
        rambo_lib.probe_host_write(src, torch.zeros(src.numel(), dtype=torch.uint8), 2)


def test_bounded_wait_expiry_is_reported_and_handle_stays_usable(rambo_lib):
    p = synth.Params(K=50, B=8, R=2, m=1 << 12, eta=2, k=31, seed=2)
    rng = np.random.default_rng(8)
    corpus = synth.family_corpus(rng, p, n_seeds=5, doc_len=400, sub_rate=0.02)
    q = synth.sample_queries(rng, corpus, rng.integers(31, 200, size=40), 0.5)
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    o.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    idx = rambo_lib.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    idx.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    idx.probe_wait_expiry(1000)
    with pytest.raises(rambo_lib.RamboError) as ex:
        idx.sync()
    assert ex.value.code == rambo_lib.RAMBO_ETIMEOUT
    idx.sync()  # the error was reported once and cleared
    assert np.array_equal(idx.query_seqs(q.packed, q.offsets), o.query_seqs(q.packed, q.offsets))
    with pytest.raises(rambo_lib.RamboError):
        idx.probe_wait_expiry(0)


@pytest.mark.gpu
def test_hardware_rate_probes_run():
    # the two probes behind design notes: L2 atomics in and out of L2, and
    # tensor-memory reads; small runs, checked only for sane output
    from paper_1910_04358_gb300 import hw_probe
    rows = list(hw_probe.l2_atomics([8, 256], ops=16, reps=1))
    assert len(rows) == 2 and all(r["g_atomicor_per_s"] > 0 for r in rows)
    rows = list(hw_probe.tmem_read(iters=64))
    assert len(rows) == 9 and all(r["bytes_per_cycle_per_sm"] > 0 for r in rows)
