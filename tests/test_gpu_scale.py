"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (its cached tuning, the same calls), against the CPU oracle:

* medium (1,000 documents, 1 GiB index): the whole index and every answer
  against a full oracle (R x B separate filters of 2^26 bits);
* large (10^4 documents, 32 GiB index): 1,200 sampled answers (all lengths,
  the longest queries included) and the index bits at 10^5 random positions
  plus every position the sampled queries probe, against a restricted-mode
  oracle that keeps exactly those positions;
* stream (10^5 documents in 100 epochs, 64 GiB index): after epochs 1, 2, 50
  and 100, sampled answers against the restricted oracle built up epoch by
  epoch (snapshot semantics: a query sees exactly the documents inserted
  before it), and no answer naming a later document;

plus the streaming shape at a size the full oracle handles, every answer of
every epoch.
"""
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


def _bench_index(rambo_lib, p, key_fn):
    """An index with the tuning bench.py keeps for this workload's batch."""
    from paper_1910_04358_gb300 import autotune
    idx = rambo_lib.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    cached = autotune.load_cached(autotune.CACHE_FILE, key_fn(idx))
    if cached:
        idx.set_tuning(**cached)
    return idx


def _inserted_mask(W, docs):
    m = np.zeros(W, np.uint32)
    for d in docs:
        m[d >> 5] |= np.uint32(1) << np.uint32(d & 31)
    return m


def _assert_groups_equal(idx, o, p, positions, chunk_groups=1 << 20):
    """GPU position groups vs the oracle's bits at the same positions: bit
    r*B + b of a group is BFU (b, r) (the first ceil(R*B/8) bytes, LSB
    first); the group's padding stays zero."""
    G = idx.info["group_bytes"]
    nbf = p.R * p.B
    row = (nbf + 7) // 8
    positions = np.sort(np.asarray(positions, dtype=np.uint64))
    positions = positions[np.concatenate(([True], positions[1:] != positions[:-1]))]
    want = o.position_bits(positions)
    lastmask = np.uint8((1 << (nbf % 8)) - 1) if nbf % 8 else np.uint8(0xFF)
    starts = np.searchsorted(positions, np.arange(0, p.m + chunk_groups, chunk_groups, dtype=np.uint64))
    for c in range(starts.size - 1):
        a, b = int(starts[c]), int(starts[c + 1])
        if a == b:
            continue
        g0 = c * chunk_groups
        g1 = min(p.m, g0 + chunk_groups)
        blob = idx.copy_index(g0 * G, (g1 - g0) * G).reshape(g1 - g0, G)
        got = blob[positions[a:b].astype(np.int64) - g0]
        body, w = got[:, :row].copy(), want[a:b]
        body[:, row - 1] &= lastmask
        assert np.array_equal(body, w), f"index bits differ in groups {g0}..{g1}"
        if nbf % 8:
            assert not np.any(got[:, row - 1] & ~lastmask)
        assert not np.any(got[:, row:]), "padding bits set"


def test_medium_full_index_and_every_answer(rambo_lib):
    from paper_1910_04358_gb300 import autotune
    from paper_1910_04358_gb300.rambo import as_u32
    corpus, kmers, q = synth.medium_workload()
    p = corpus.params
    total = q.n_kmers(p.k) + int(kmers.size)
    idx = _bench_index(rambo_lib, p, lambda i: autotune.cache_key(i, q.n + int(kmers.size), total))
    idx.insert_batch_dev(_dev(corpus.doc_ids, np.int32), _dev(corpus.packed, np.uint8),
                         _dev(corpus.offsets, np.int64))
    got_k, got_s = idx.query_batch_dev(_dev(kmers, np.int64), _dev(q.packed, np.uint8),
                                       _dev(q.offsets, np.int64))
    idx.sync()
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    o.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets, threads=THREADS)
    # the whole index, position by position (1 GiB of groups)
    _assert_groups_equal(idx, o, p, np.arange(p.m, dtype=np.uint64))
    # every answer of the batch the bench times
    assert np.array_equal(as_u32(got_s), o.query_seqs(q.packed, q.offsets, threads=THREADS))
    assert np.array_equal(as_u32(got_k), o.query_kmers(kmers, threads=THREADS))


def test_large_full_size_sampled_answers_and_index_bits(rambo_lib):
    from paper_1910_04358_gb300 import autotune
    from paper_1910_04358_gb300.rambo import as_u32
    corpus, q = synth.large_workload()
    p = corpus.params
    idx = _bench_index(rambo_lib, p, lambda i: autotune.cache_key(i, q.n, q.n_kmers(p.k)))
    idx.insert_batch_dev(_dev(corpus.doc_ids, np.int32), _dev(corpus.packed, np.uint8),
                         _dev(corpus.offsets, np.int64))
    _, got = idx.query_batch_dev(None, _dev(q.packed, np.uint8), _dev(q.offsets, np.int64))
    got = as_u32(got)
    idx.sync()
    assert not np.any(got & ~_inserted_mask(idx.W, range(p.K))[None, :])
    # 1,200 answers: the 200 longest queries and 1,000 more at random
    L = np.diff(q.offsets.astype(np.int64))
    rng = np.random.default_rng(1)
    longest = np.argsort(L)[-200:]
    rest = rng.choice(np.setdiff1d(np.arange(q.n), longest), size=1000, replace=False)
    si = np.sort(np.concatenate([longest, rest]))
    assert L[si].max() >= 4990 and L[si].min() <= 100
    sp, so = _sample_batch(q, si)
    random_pos = rng.integers(0, p.m, size=100_000).astype(np.uint64)
    probe = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, tracked=[0])
    query_pos = probe.seq_positions(sp, so).ravel()
    probe.close()
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed,
                     tracked=np.concatenate([query_pos, random_pos]))
    o.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets, threads=THREADS)
    assert np.array_equal(o.query_seqs(sp, so, threads=THREADS), got[si])
    _assert_groups_equal(idx, o, p, np.concatenate([query_pos, random_pos]))


def test_stream_full_size_epoch_snapshots(rambo_lib):
    from paper_1910_04358_gb300 import autotune
    from paper_1910_04358_gb300.rambo import as_u32
    wl = synth.stream_workload()
    p = wl.params
    checked = (0, 1, 49, wl.n_epochs - 1)  # after epochs 1, 2, 50 and 100
    epochs, samples = [], {}
    for e in range(wl.n_epochs):
        docs, q = wl.epoch(e)
        epochs.append(docs)
        if e in checked:
            si = np.arange(0, q.n, 40)  # 250 queries
            samples[e] = (q, si, _sample_batch(q, si))
    o = oracle.tracking_oracle(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed,
                               seqs=[s[2] for s in samples.values()])
    key = autotune.cache_key
    idx = _bench_index(rambo_lib, p, lambda i: key(i, wl.queries_per_epoch, 0).rsplit("_kpq", 1)[0] + "_stream")
    for e, (ids, packed, offs) in enumerate(epochs):
        idx.insert_batch_dev(_dev(ids, np.int32), _dev(packed, np.uint8), _dev(offs, np.int64))
        o.insert_batch(ids, packed, offs, threads=THREADS)
        if e not in checked:
            continue
        q, si, (sp, so) = samples[e]
        got = as_u32(idx.query_seqs_dev(_dev(q.packed, np.uint8), _dev(q.offsets, np.int64)))
        idx.sync()
        assert np.array_equal(o.query_seqs(sp, so, threads=THREADS), got[si]), f"epoch {e + 1}"
        later = _inserted_mask(idx.W, range(int(ids[-1]) + 1, p.K))
        assert not np.any(got & later[None, :]), f"epoch {e + 1} names a later document"


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
        later = _inserted_mask(idx.W, range(wl.inserted, p.K))
        assert not np.any(got & later[None, :])
