"""Parity at the workloads' full sizes, in the launch configuration bench.py
times, on sampled outputs the oracle computes one by one (restricted-mode
oracle tracking only the sampled queries' probe positions), plus properties
that hold at any size; and streaming epochs against oracle snapshots."""
import os

import numpy as np
import pytest

import oracle
from paper_1910_04358_gb300 import synth

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


def _dev(a, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()


def _sample_batch(q, idx):
    from paper_1910_04358_gb300.synth import PackedStream, unpack_bases
    offs = q.offsets.astype(np.int64)
    s = PackedStream()
    for i in idx:
        s.append(unpack_bases(q.packed, int(offs[i]), int(offs[i + 1] - offs[i])))
    return s.finish()


def _restricted_oracle(p, corpus, packs, kmers=()):
    """Oracle tracking exactly the probe positions of the given sequences/k-mers."""
    probe = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, tracked=[0])
    pos = set()
    for packed, offs in packs:
        for i in range(offs.size - 1):
            for t in range(int(offs[i]), int(offs[i + 1]) - p.k + 1):
                c = oracle.kmer_canonical(packed, t, p.k)
                pos.update(probe.probe_position(c, j) for j in range(p.eta))
    for x in kmers:
        c = oracle.canonical_of_code(int(x), p.k)
        pos.update(probe.probe_position(c, j) for j in range(p.eta))
    probe.close()
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, tracked=sorted(pos))
    o.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets, threads=THREADS)
    return o


def _check_properties(got, q, p, inserted_mask):
    # every answer is a subset of the inserted documents
    assert not np.any(got & ~inserted_mask[None, :])
    # zero false negatives for exact substrings of a document
    for i in np.nonzero(q.from_doc >= 0)[0][:2000]:
        d = int(q.from_doc[i])
        assert (got[i, d >> 5] >> np.uint32(d & 31)) & 1, f"query {i} misses its source doc {d}"


def test_medium_full_size(rambo_lib):
    from paper_1910_04358_gb300.rambo import as_u32
    corpus, kmers, q = synth.medium_workload()
    p = corpus.params
    idx = rambo_lib.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    idx.insert_batch_dev(_dev(corpus.doc_ids, np.int32), _dev(corpus.packed, np.uint8),
                         _dev(corpus.offsets, np.int64))
    got_s = as_u32(idx.query_seqs_dev(_dev(q.packed, np.uint8), _dev(q.offsets, np.int64)))
    got_k = as_u32(idx.query_kmers_dev(_dev(kmers, np.int64)))
    idx.sync()
    inserted = np.zeros(idx.W, np.uint32)
    for d in range(p.K):
        inserted[d >> 5] |= np.uint32(1) << np.uint32(d & 31)
    _check_properties(got_s, q, p, inserted)
    rng = np.random.default_rng(0)
    si = np.sort(rng.choice(q.n, size=120, replace=False))
    ki = np.sort(rng.choice(kmers.size, size=2000, replace=False))
    sp, so = _sample_batch(q, si)
    o = _restricted_oracle(p, corpus, [(sp, so)], kmers[ki])
    assert np.array_equal(o.query_seqs(sp, so, threads=THREADS), got_s[si])
    assert np.array_equal(o.query_kmers(kmers[ki], threads=THREADS), got_k[ki])


@pytest.mark.slow
def test_large_full_size(rambo_lib):
    from paper_1910_04358_gb300.rambo import as_u32
    corpus, q = synth.large_workload()
    p = corpus.params
    idx = rambo_lib.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    idx.insert_batch_dev(_dev(corpus.doc_ids, np.int32), _dev(corpus.packed, np.uint8),
                         _dev(corpus.offsets, np.int64))
    got = as_u32(idx.query_seqs_dev(_dev(q.packed, np.uint8), _dev(q.offsets, np.int64)))
    idx.sync()
    inserted = np.zeros(idx.W, np.uint32)
    for d in range(p.K):
        inserted[d >> 5] |= np.uint32(1) << np.uint32(d & 31)
    assert not np.any(got & ~inserted[None, :])
    rng = np.random.default_rng(1)
    si = np.sort(rng.choice(q.n, size=60, replace=False))
    sp, so = _sample_batch(q, si)
    o = _restricted_oracle(p, corpus, [(sp, so)])
    assert np.array_equal(o.query_seqs(sp, so, threads=THREADS), got[si])


def test_streaming_epochs_match_oracle_snapshots(rambo_lib):
    # the streaming workload's shape at a size the full oracle handles: every
    # epoch's queries see exactly the documents inserted so far
    wl = synth.stream_workload(n_docs=600, doc_len=5000, n_seeds=60, epoch_docs=150,
                               queries_per_epoch=300, m=1 << 18)
    p = wl.params
    idx = rambo_lib.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    from paper_1910_04358_gb300.rambo import as_u32
    for e in range(wl.n_epochs):
        (ids, packed, offs), q = wl.epoch(e)
        idx.insert_batch_dev(_dev(ids, np.int32), _dev(packed, np.uint8), _dev(offs, np.int64))
        got = as_u32(idx.query_seqs_dev(_dev(q.packed, np.uint8), _dev(q.offsets, np.int64)))
        idx.sync()
        o.insert_batch(ids, packed, offs, threads=THREADS)
        want = o.query_seqs(q.packed, q.offsets, threads=THREADS)
        assert np.array_equal(got, want), f"epoch {e}"
        # nothing from a later epoch can appear
        later = np.zeros(idx.W, np.uint32)
        for d in range(wl.inserted, p.K):
            later[d >> 5] |= np.uint32(1) << np.uint32(d & 31)
        assert not np.any(got & later[None, :])
