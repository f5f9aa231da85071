"""Measurement support and failure detection on the GPU (no fault, no hang).

* the random-gather probe runs and rejects record sizes it does not serve;
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
