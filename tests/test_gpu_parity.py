"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Every result here is integer/bit work, so the bar is equality: answer masks,
index bits, bucket->document bitmaps and partitions must match the oracle
exactly on the same seeded inputs.
"""
import numpy as np
import pytest

import oracle
from paper_1910_04358_gb300 import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _dev(a, dtype):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def gpu_index(rambo, p, corpus, via="dev", chunks=1):
    idx = rambo.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    n = corpus.doc_ids.size
    bounds = np.linspace(0, n, chunks + 1).astype(int)
    for a, b in zip(bounds[:-1], bounds[1:]):
        if b <= a:
            continue
        ids = corpus.doc_ids[a:b]
        offs = corpus.offsets[a:b + 1]
        if via == "dev":
            torch = _torch()
            idx.insert_batch_dev(_dev(ids.astype(np.uint32), np.int32),
                                 _dev(corpus.packed, np.uint8),
                                 _dev(offs.astype(np.uint64), np.int64))
            idx.sync()
        else:
            idx.insert_batch(ids, corpus.packed, offs)
    return idx


def oracle_index(p, corpus, threads=4):
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    o.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets, threads=threads)
    return o


def gpu_query_seqs(rambo, idx, q_packed, q_offsets):
    out = idx.query_seqs_dev(_dev(q_packed, np.uint8), _dev(q_offsets.astype(np.uint64), np.int64))
    idx.sync()
    return rambo.as_u32(out)


def assert_index_equal(idx, o, p):
    """GPU bit-sliced groups vs the oracle's separate filters, bit for bit."""
    G = idx.info["group_bytes"]
    words = idx.copy_index().view(np.uint32).reshape(p.m, G // 4)
    for r in range(p.R):
        for b in range(p.B):
            i = r * p.B + b
            gpu_bits = ((words[:, i >> 5] >> np.uint32(i & 31)) & 1).astype(np.uint8)
            fw = o.filter_words(r, b)
            orc_bits = np.unpackbits(fw.view(np.uint8), bitorder="little")[:p.m]
            assert np.array_equal(gpu_bits, orc_bits), f"BFU ({b},{r}) differs"
    # padding bits of every group stay zero
    used = p.R * p.B
    for w in range(G // 4):
        lo = w * 32
        if lo >= used:
            assert not words[:, w].any()
        elif lo + 32 > used:
            assert not (words[:, w] >> np.uint32(used - lo)).any()


def assert_docbits_equal(idx, o, p):
    db = idx.docbits()
    part = idx.partition()
    for d in range(p.K):
        for r in range(p.R):
            assert part[d, r] == o.bucket(d, r)
    for r in range(p.R):
        for b in range(p.B):
            docs = oracle.mask_to_docs(db[r, b])
            want = {d for d in range(p.K) if o.is_inserted(d) and o.bucket(d, r) == b}
            assert docs == want


# ------------------------------------------------------------------ tiny

@pytest.fixture(scope="module")
def tiny():
    corpus, q = synth.tiny_workload()
    p = corpus.params
    return p, corpus, q, oracle_index(p, corpus)


def test_tiny_index_bits_match_oracle(rambo_lib, tiny):
    p, corpus, q, o = tiny
    idx = gpu_index(rambo_lib, p, corpus)
    assert_index_equal(idx, o, p)
    assert_docbits_equal(idx, o, p)


def test_tiny_sequence_queries_match_oracle(rambo_lib, tiny):
    p, corpus, q, o = tiny
    idx = gpu_index(rambo_lib, p, corpus)
    want = o.query_seqs(q.packed, q.offsets)
    got = gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets)
    assert np.array_equal(got, want)
    # the host-buffer entry point gives the same bits
    assert np.array_equal(idx.query_seqs(q.packed, q.offsets), want)


def test_tiny_kmer_queries_match_oracle(rambo_lib, tiny):
    p, corpus, q, o = tiny
    idx = gpu_index(rambo_lib, p, corpus, via="host")
    rng = np.random.default_rng(5)
    kmers = synth.sample_kmers(rng, corpus, 3000, p.k, 0.5)
    want = o.query_kmers(kmers)
    assert np.array_equal(idx.query_kmers(kmers), want)
    got = idx.query_kmers_dev(_dev(kmers, np.int64))
    idx.sync()
    assert np.array_equal(rambo_lib.as_u32(got), want)


# --------------------------------------------------------- parameter sweep

SWEEP = [
    # K,    B,   R,  m,          eta, k   -> group bytes
    (37, 3, 1, 1 << 12, 1, 11),      # 4
    (64, 10, 3, 5003, 2, 15),        # 4, m not a power of two
    (100, 16, 4, 1 << 14, 3, 31),    # 8
    (33, 32, 4, 1 << 13, 2, 31),     # 16
    (200, 30, 2, 1 << 13, 4, 21),    # 8
    (150, 50, 3, 1 << 12, 2, 31),    # 32
    (300, 100, 5, 1 << 13, 2, 31),   # 64
    (500, 64, 6, 12289, 5, 25),      # 64, eta > 4 (probe passes), odd m
    (700, 316, 6, 1 << 12, 2, 31),   # 256
    (90, 700, 3, 1 << 11, 2, 32),    # 512? 2100 bits -> 512 B, k = 32
    (60, 1500, 3, 1 << 10, 3, 31),   # 1024 bytes: two chunks
    (5, 1, 1, 1 << 10, 2, 9),        # B = R = 1
    (1, 4, 2, 1 << 10, 2, 7),        # K = 1
]


@pytest.mark.parametrize("path", [0, 1, 2, 3])
@pytest.mark.parametrize("K,B,R,m,eta,k", SWEEP)
def test_parameter_sweep(rambo_lib, K, B, R, m, eta, k, path):
    p = synth.Params(K=K, B=B, R=R, m=m, eta=eta, k=k, seed=K + B)
    rng = np.random.default_rng(K * 7 + B)
    corpus = synth.family_corpus(rng, p, n_seeds=max(1, K // 8), doc_len=400, sub_rate=0.02)
    q = synth.sample_queries(rng, corpus, rng.integers(max(1, k - 3), 200, size=300), 0.6)
    o = oracle_index(p, corpus)
    idx = gpu_index(rambo_lib, p, corpus, chunks=3)
    # path 1 (persistent fused launch) with small tiles so long queries span tiles
    # path 2 (region-binned) with 1 KiB regions so the batch spans many bins
    # path 3 (content-ordered segments) with segments of about 4 k-mers
    idx.set_tuning(query_path=path, fused_tile_kmers=64, fused_short_max=40, bin_region_kib=1,
                   seg_cut_bits=2)
    assert_index_equal(idx, o, p)
    assert_docbits_equal(idx, o, p)
    assert np.array_equal(gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets),
                          o.query_seqs(q.packed, q.offsets))
    kmers = synth.sample_kmers(rng, corpus, 500, k, 0.5)
    assert np.array_equal(idx.query_kmers(kmers), o.query_kmers(kmers))


@pytest.mark.parametrize("path", [0, 1])
def test_many_documents_several_answer_chunks(rambo_lib, path):
    # more than 4096 documents, so an answer spans several chunks: the fused
    # path decodes each query's passing buckets once for all of them, or scans
    # the mask per chunk when more than 32 buckets pass.  Long queries from
    # documents keep a few buckets, single k-mers dozens, and sequences
    # shorter than k all of them (every inserted document answers).
    p = synth.Params(K=5000, B=316, R=6, m=1 << 15, eta=2, k=31, seed=77)
    rng = np.random.default_rng(77)
    corpus = synth.family_corpus(rng, p, n_seeds=50, doc_len=500, sub_rate=0.01)
    lengths = np.concatenate([rng.integers(31, 400, size=200), np.full(40, 31), np.full(5, 10)])
    q = synth.sample_queries(rng, corpus, lengths, 0.6)
    o = oracle_index(p, corpus)
    idx = gpu_index(rambo_lib, p, corpus)
    idx.set_tuning(query_path=path, fused_tile_kmers=64, fused_short_max=40)
    got = gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets)
    want = o.query_seqs(q.packed, q.offsets)
    assert np.array_equal(got, want)
    # the mix reaches both expansion routes of the fused path
    pops = np.array([len(oracle.mask_to_docs(w)) for w in want])
    assert (pops[-5:] == p.K).all() and (pops[:200] < p.K).all()


@pytest.mark.parametrize("eta", [1, 2, 3])
def test_fused_staged_gathers(rambo_lib, eta):
    # 16-byte groups (one lane per group): the fused launch can gather through
    # shared memory (cp.async) instead of registers; eta 3 keeps the register
    # gathers.  Tiles, short-query thresholds and early exit vary around it.
    p = synth.Params(K=300, B=32, R=4, m=1 << 14, eta=eta, k=31, seed=8)
    rng = np.random.default_rng(eta)
    corpus = synth.family_corpus(rng, p, n_seeds=20, doc_len=600, sub_rate=0.02)
    q = synth.sample_queries(rng, corpus, rng.integers(20, 900, size=300), 0.6)
    o = oracle_index(p, corpus)
    want = o.query_seqs(q.packed, q.offsets)
    idx = gpu_index(rambo_lib, p, corpus)
    for st in (dict(fused_async=1, fused_tile_kmers=1024, fused_short_max=1024),
               dict(fused_async=1, fused_tile_kmers=64, fused_short_max=40),
               dict(fused_async=1, fused_tile_kmers=256, fused_short_max=0, probe_ctas_per_sm=2),
               dict(fused_async=1, fused_tile_kmers=128, fused_short_max=300, early_exit=1,
                    early_exit_segment=128),
               dict(fused_async=0, fused_tile_kmers=64, fused_short_max=40)):
        idx.set_tuning(query_path=1, **st)
        assert np.array_equal(gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets), want), st
    # the single k-mer probe, staged the same way
    kmers = synth.sample_kmers(rng, corpus, 3000, p.k, 0.5)
    want_k = o.query_kmers(kmers)
    for st in (dict(kmer_async=1), dict(kmer_async=1, kmer_probe_ctas_per_sm=1), dict(kmer_async=0)):
        idx.set_tuning(**st)
        assert np.array_equal(idx.query_kmers(kmers), want_k), st


def test_tuning_knobs_do_not_change_results(rambo_lib):
    p = synth.Params(K=300, B=40, R=4, m=1 << 13, eta=2, k=31, seed=4)
    rng = np.random.default_rng(77)
    corpus = synth.family_corpus(rng, p, n_seeds=20, doc_len=500, sub_rate=0.02)
    q = synth.sample_queries(rng, corpus, rng.integers(25, 300, size=400), 0.6)
    kmers = synth.sample_kmers(rng, corpus, 800, p.k, 0.5)
    o = oracle_index(p, corpus)
    want_s, want_k = o.query_seqs(q.packed, q.offsets), o.query_kmers(kmers)
    idx = gpu_index(rambo_lib, p, corpus)
    settings = [dict(use_byte_table=0), dict(use_byte_table=1, byte_table_max_mb=64),
                dict(probe_ctas_per_sm=1, probe_min_kmers_per_warp=4096),
                dict(probe_ctas_per_sm=7, probe_min_kmers_per_warp=0, expand_ctas_per_sm=1),
                dict(expand_ctas_per_sm=64, use_byte_table=0),
                dict(query_path=1, fused_tile_kmers=1024, fused_short_max=1024),
                dict(query_path=1, fused_tile_kmers=32, fused_short_max=0),
                dict(query_path=1, fused_tile_kmers=100, fused_short_max=1 << 20),
                dict(query_path=1, fused_tile_kmers=64, fused_short_max=50, use_byte_table=1,
                     probe_ctas_per_sm=1),
                dict(query_path=0, smem_docbits=0),
                dict(query_path=0, smem_docbits=1, expand_ctas_per_sm=1),
                dict(query_path=1, smem_docbits=0, use_byte_table=0),
                dict(query_path=0, use_nibble_table=1, expand_ctas_per_sm=1),
                dict(query_path=0, use_nibble_table=0),
                dict(query_path=2, bin_region_kib=0),
                dict(query_path=2, bin_region_kib=4)]
    for st in settings:
        idx.set_tuning(**st)
        assert np.array_equal(gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets), want_s), st
        assert np.array_equal(idx.query_kmers(kmers), want_k), st
    # the byte table follows later inserts
    idx.set_tuning(use_byte_table=1)
    extra = synth.family_corpus(np.random.default_rng(5), synth.Params(K=10, B=p.B, R=p.R, m=p.m, eta=2),
                                n_seeds=2, doc_len=300, sub_rate=0.0)
    ids = np.arange(290, 300, dtype=np.uint32)
    idx.insert_batch(ids, extra.packed, extra.offsets)
    o.insert_batch(ids, extra.packed, extra.offsets)
    assert np.array_equal(gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets),
                          o.query_seqs(q.packed, q.offsets))


# ---------------------------------------------------------------- edge cases

def test_edge_cases(rambo_lib):
    p = synth.Params(K=45, B=7, R=3, m=1 << 12, eta=2, k=31, seed=9)
    rng = np.random.default_rng(3)
    lens = [0, 5, 30, 31, 32, 200, 31, 0, 1000]
    docs = [synth.uniform_genome(rng, L) for L in lens]
    packed, offs = synth.pack_many(docs)
    ids = np.array([0, 1, 2, 3, 4, 5, 44, 6, 7], dtype=np.uint32)
    corpus = synth.Corpus(p, ids, packed, offs)
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    o.insert_batch(ids, packed, offs)
    idx = rambo_lib.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    idx.insert_batch(ids, packed, offs)
    # duplicate insert of the whole batch is idempotent
    idx.insert_batch(ids, packed, offs)
    assert_index_equal(idx, o, p)
    assert_docbits_equal(idx, o, p)
    # queries: empty, shorter than k, exactly k, ragged, from the documents
    qs = [np.zeros(0, np.uint8), docs[1][:5], docs[4][:31], docs[5][17:150], docs[8][3:900],
          docs[3], synth.uniform_genome(rng, 31), docs[8]]
    qp, qo = synth.pack_many(qs)
    want = o.query_seqs(qp, qo)
    got = gpu_query_seqs(rambo_lib, idx, qp, qo)
    assert np.array_equal(got, want)
    inserted = {int(d) for d in ids}
    assert oracle.mask_to_docs(got[0]) == inserted  # no term: every inserted document
    assert oracle.mask_to_docs(got[1]) == inserted
    # an empty batch is a no-op
    assert idx.query_seqs(qp[:0], np.zeros(1, np.uint64)).shape == (0, idx.W)
    # misaligned device pointers: the same bytes seen through an odd offset
    torch = _torch()
    qp_pad = np.concatenate([np.zeros(3, np.uint8), qp])
    t = _dev(qp_pad, np.uint8)[3:]
    out = idx.query_seqs_dev(t, _dev(qo.astype(np.uint64), np.int64))
    idx.sync()
    assert np.array_equal(rambo_lib.as_u32(out), want)
    # offsets not starting at zero
    shifted = np.concatenate([np.zeros(1, np.uint64), qo + np.uint64(4)])
    qp2 = np.concatenate([np.zeros(1, np.uint8), qp])
    got2 = idx.query_seqs(qp2, shifted[1:])
    assert np.array_equal(got2, want)


def test_argument_errors(rambo_lib):
    with pytest.raises(rambo_lib.RamboError):
        rambo_lib.Index(0, 1, 1, 64, 1)
    with pytest.raises(rambo_lib.RamboError):
        rambo_lib.Index(4, 2, 1, 64, 0)
    with pytest.raises(rambo_lib.RamboError):
        rambo_lib.Index(4, 2, 1, (1 << 32) + 1, 1)
    idx = rambo_lib.Index(10, 2, 2, 1 << 10, 2, k=31)
    packed, offs = synth.pack_many([np.zeros(40, np.uint8)])
    with pytest.raises(rambo_lib.RamboError) as e:
        idx.insert_batch(np.array([10], np.uint32), packed, offs)
    assert e.value.code == rambo_lib.RAMBO_ERANGE
    with pytest.raises(rambo_lib.RamboError) as e:
        idx.query_kmers(np.array([1 << 62], np.uint64))
    assert e.value.code == rambo_lib.RAMBO_EINVAL
    with pytest.raises(rambo_lib.RamboError) as e:
        idx.query_seqs(packed, np.array([5, 3], np.uint64))
    assert e.value.code == rambo_lib.RAMBO_EINVAL
    # device-side checks latch an error reported by sync, and skip the item
    idx.insert_batch_dev(_dev(np.array([3, 11], np.uint32), np.int32), _dev(packed, np.uint8),
                         _dev(np.array([0, 20, 40], np.uint64), np.int64))
    with pytest.raises(rambo_lib.RamboError) as e:
        idx.sync()
    assert e.value.code == rambo_lib.RAMBO_ERANGE
    idx.sync()  # cleared
    idx.query_kmers_dev(_dev(np.array([1 << 62, 5], np.uint64), np.int64))
    with pytest.raises(rambo_lib.RamboError) as e:
        idx.sync()
    assert e.value.code == rambo_lib.RAMBO_EINVAL
    # mixed batches: host offsets checked before anything runs, device
    # workspace size and alignment checked before anything is enqueued
    good_k = np.array([5, 7], np.uint64)
    with pytest.raises(rambo_lib.RamboError) as e:
        idx.query_batch(good_k, packed, np.array([5, 3], np.uint64))
    assert e.value.code == rambo_lib.RAMBO_EINVAL
    torch = _torch()
    d_k, d_p = _dev(good_k, np.int64), _dev(packed, np.uint8)
    d_o = _dev(np.array([0, 40], np.uint64), np.int64)
    need = idx.workspace_bytes("kmers", 2) + idx.workspace_bytes("seqs", 1)
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    ptr = (buf.data_ptr() + 255) // 256 * 256
    with pytest.raises(rambo_lib.RamboError) as e:  # too small
        idx.query_batch_dev(d_k, d_p, d_o, workspace=(ptr, need - 256))
    assert e.value.code == rambo_lib.RAMBO_EINVAL
    with pytest.raises(rambo_lib.RamboError) as e:  # not 256-byte aligned
        idx.query_batch_dev(d_k, d_p, d_o, workspace=(ptr + 8, need))
    assert e.value.code == rambo_lib.RAMBO_EINVAL
    ok_k, ok_s = idx.query_batch_dev(d_k, d_p, d_o, workspace=(ptr, need))
    idx.sync()
    assert np.array_equal(rambo_lib.as_u32(ok_k), idx.query_kmers(good_k))
    assert np.array_equal(rambo_lib.as_u32(ok_s), idx.query_seqs(packed, np.array([0, 40], np.uint64)))
    # tuning knobs out of range are refused and leave the tuning unchanged
    before = idx.get_tuning()
    for bad in (dict(query_path=4), dict(host_slots=0), dict(host_slots=5), dict(bin_rows=3),
                dict(insert_mode=4), dict(insert_bin_records=100), dict(fused_async=2), dict(kmer_async=2),
                dict(seg_cut_bits=11), dict(early_exit_segment=100)):
        with pytest.raises(rambo_lib.RamboError):
            idx.set_tuning(**bad)
    assert idx.get_tuning() == before


# ------------------------------------------------------------------ folding

@pytest.mark.parametrize("K,B,R,m", [(120, 16, 3, 1 << 12), (300, 100, 5, 1 << 11),
                                     (90, 64, 6, 1 << 10), (40, 2, 2, 1 << 12)])
def test_fold_matches_oracle_and_direct_half_index(rambo_lib, K, B, R, m):
    p = synth.Params(K=K, B=B, R=R, m=m, eta=2, k=31, seed=6)
    rng = np.random.default_rng(K + B)
    corpus = synth.family_corpus(rng, p, n_seeds=max(1, K // 10), doc_len=500, sub_rate=0.02)
    q = synth.sample_queries(rng, corpus, rng.integers(25, 200, size=200), 0.6)
    o = oracle_index(p, corpus)
    idx = gpu_index(rambo_lib, p, corpus)
    before = gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets)
    idx.fold()
    o.fold()
    ph = synth.Params(K=K, B=B // 2, R=R, m=m, eta=2, k=31, seed=6)
    assert_index_equal(idx, o, ph)
    assert_docbits_equal(idx, o, ph)
    after = gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets)
    assert np.array_equal(after, o.query_seqs(q.packed, q.offsets))
    assert np.all((before & ~after) == 0)
    direct = gpu_index(rambo_lib, ph, corpus)
    assert np.array_equal(direct.copy_index(), idx.copy_index())


@pytest.mark.parametrize("K,B,R", [
    (700, 32, 4),    # B % 32 == 0: power-of-two row kernel, W % 4 != 0 (scalar stores)
    (1000, 32, 3),   # ... W % 4 == 0 (16-byte stores)
    (1024, 64, 2),   # two mask words per repetition
    (100, 32, 3),    # one 16-byte slice per row (32 queries per warp)
    (1000, 24, 3),   # B % 32 != 0: generic nibble kernel
])
def test_expansion_variants_on_many_kmer_queries(rambo_lib, K, B, R):
    # enough queries per block that the shared-memory variants engage
    p = synth.Params(K=K, B=B, R=R, m=1 << 14, eta=2, k=31, seed=12)
    rng = np.random.default_rng(31)
    corpus = synth.family_corpus(rng, p, n_seeds=30, doc_len=600, sub_rate=0.02)
    kmers = synth.sample_kmers(rng, corpus, 12_000, p.k, 0.5)
    o = oracle_index(p, corpus)
    want = o.query_kmers(kmers, threads=4)
    idx = gpu_index(rambo_lib, p, corpus)
    for st in (dict(expand_ctas_per_sm=1, use_nibble_table=1, expand_filter=1),
               dict(expand_ctas_per_sm=1, use_nibble_table=1, expand_filter=0),
               dict(expand_ctas_per_sm=8, use_nibble_table=1, expand_filter=0),
               dict(expand_ctas_per_sm=1, use_nibble_table=0, smem_docbits=1),
               dict(expand_ctas_per_sm=1, use_nibble_table=0, smem_docbits=0, use_byte_table=1),
               dict(expand_ctas_per_sm=1, use_nibble_table=0, smem_docbits=0, use_byte_table=0)):
        idx.set_tuning(**st)
        got = idx.query_kmers_dev(_dev(kmers, np.int64))
        idx.sync()
        assert np.array_equal(rambo_lib.as_u32(got), want), st


def test_sequence_batch_past_single_block_scan(rambo_lib):
    # more than 16 * 4096 sequences: the k-mer prefix takes the three-launch
    # multi-block scan instead of the single-block one
    p = synth.Params(K=64, B=8, R=2, m=1 << 13, eta=2, k=31, seed=6)
    rng = np.random.default_rng(44)
    corpus = synth.family_corpus(rng, p, n_seeds=8, doc_len=400, sub_rate=0.02)
    q = synth.sample_queries(rng, corpus, rng.integers(0, 60, size=70_000), 0.5)
    o = oracle_index(p, corpus)
    want = o.query_seqs(q.packed, q.offsets)
    idx = gpu_index(rambo_lib, p, corpus)
    for path in (0, 1, 2):
        idx.set_tuning(query_path=path)
        assert np.array_equal(gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets), want), path


@pytest.mark.parametrize("K,B,R,m", [
    (120, 32, 4, 1 << 13),      # 16-byte groups: repetitions pair up in 64-bit words
    (100, 16, 3, 5003),         # 8-byte groups, m odd: m * Gw odd -> 32-bit atomics
    (64, 10, 3, 4097),          # 4-byte groups, m * Gw odd
    (300, 100, 5, 1 << 12),     # 64-byte groups: repetitions in different words
])
def test_insert_modes_give_identical_index(rambo_lib, K, B, R, m):
    p = synth.Params(K=K, B=B, R=R, m=m, eta=2, k=31, seed=K)
    rng = np.random.default_rng(B * 13 + R)
    corpus = synth.family_corpus(rng, p, n_seeds=max(1, K // 10), doc_len=500, sub_rate=0.02)
    o = oracle_index(p, corpus)
    base = None
    # mode 3 (region-binned) with the default record buffer, and with one of
    # 4096 records: many chunks, and bins that overflow into direct atomics;
    # regions of 64 KiB so that the index spans several, or of 1 KiB so that
    # it spans hundreds
    for mode, recs, kib in ((0, 0, 64), (1, 0, 64), (2, 0, 64), (3, 0, 64), (3, 4096, 64), (3, 0, 1),
                            (3, 8192, 1)):
        idx = rambo_lib.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
        idx.set_tuning(insert_mode=mode, insert_bin_records=recs, bin_region_kib=kib)
        idx.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
        bits = idx.copy_index()
        if base is None:
            base = bits
            assert_index_equal(idx, o, p)
        assert np.array_equal(bits, base), (mode, recs, kib)
        idx.close()


# ------------------------------------------------ region-binned probing (path 2)

@pytest.mark.parametrize("K,B,R,m,eta,region_kib,max_len", [
    (200, 20, 3, 1 << 16, 2, 64, 900),           # 8-byte groups, 8 regions
    (300, 32, 4, 1 << 18, 2, 256, 900),          # 16-byte groups, 16 regions
    (64, 8, 2, (1 << 15) + 123, 2, 16, 900),     # 4-byte groups, m not a power of two, ragged last region
    (300, 32, 4, 1 << 18, 2, 0, 900),            # default region size: one region
    (150, 40, 4, 1 << 16, 2, 64, 900),           # 32-byte groups (two lanes per group)
    (300, 100, 5, 1 << 16, 2, 256, 12000),       # 64-byte groups; queries of up to three scatter tiles
    (300, 100, 5, (1 << 16) + 77, 3, 128, 9000), # 64-byte groups, eta 3 (2730 k-mers a tile), odd m
    (400, 200, 4, 1 << 15, 2, 512, 6000),        # 128-byte groups: path 2 unsupported, path 1 runs
])
def test_binned_path_matches_oracle(rambo_lib, K, B, R, m, eta, region_kib, max_len):
    torch = _torch()
    p = synth.Params(K=K, B=B, R=R, m=m, eta=eta, k=31, seed=9)
    rng = np.random.default_rng(K + B)
    corpus = synth.family_corpus(rng, p, n_seeds=10, doc_len=max(1500, max_len + 100), sub_rate=0.01)
    # lengths from empty to several tiles; whole documents among the sources
    q = synth.sample_queries(rng, corpus, rng.integers(0, max_len, size=300), 0.5)
    o = oracle_index(p, corpus)
    want = o.query_seqs(q.packed, q.offsets)
    idx = gpu_index(rambo_lib, p, corpus)
    idx.set_tuning(query_path=2, bin_region_kib=region_kib)
    # the probe pass at every depth
    for rows in (1, 2, 4):
        idx.set_tuning(bin_rows=rows)
        assert np.array_equal(gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets), want), rows
    idx.set_tuning(bin_rows=2)
    assert np.array_equal(idx.query_seqs(q.packed, q.offsets), want)
    # a workspace without room for the records: the call takes path 1
    d_p, d_o = _dev(q.packed, np.uint8), _dev(q.offsets.astype(np.uint64), np.int64)
    small = idx.workspace_bytes("seqs", q.n)
    buf = torch.empty(small + 256, dtype=torch.uint8, device="cuda")
    ptr = (buf.data_ptr() + 255) // 256 * 256
    out = idx.query_seqs_dev(d_p, d_o, workspace=(ptr, small))
    idx.sync()
    assert np.array_equal(rambo_lib.as_u32(out), want)


@pytest.mark.parametrize("B,R,doc_len", [(16, 3, 1500), (100, 5, 1500), (100, 5, 9000)])
def test_binned_path_overflow_probes_directly(rambo_lib, B, R, doc_len):
    # 2,000 queries over the same document: ten times more probe records than
    # the packed bytes bound the bins for, so most are probed on the spot
    # (16- and 64-byte groups); with 9,000 bases every query has three
    # scatter tiles, more than the tile map holds, so later tiles find their
    # query by search
    p = synth.Params(K=100, B=B, R=R, m=1 << 16, eta=2, k=31, seed=3)
    rng = np.random.default_rng(77)
    corpus = synth.family_corpus(rng, p, n_seeds=10, doc_len=doc_len, sub_rate=0.01)
    o = oracle_index(p, corpus)
    b0, b1 = int(corpus.offsets[7]), int(corpus.offsets[8])
    one = o.query_seqs(corpus.packed, np.array([b0, b1], dtype=np.uint64))
    n = 2000
    idx = gpu_index(rambo_lib, p, corpus)
    idx.set_tuning(query_path=2, bin_region_kib=64)
    begins = _dev(np.full(n, b0, dtype=np.uint64), np.int64)
    ends = _dev(np.full(n, b1, dtype=np.uint64), np.int64)
    out = idx.query_ranges_dev(_dev(corpus.packed, np.uint8), begins, ends)
    idx.sync()
    assert np.array_equal(rambo_lib.as_u32(out), np.repeat(one, n, axis=0))


# ------------------------------------------ content-ordered segments (path 3)

@pytest.mark.parametrize("K,B,R,m,eta", [
    (300, 100, 5, 1 << 16, 2),          # 64-byte groups (four lanes per group)
    (150, 40, 4, (1 << 16) + 77, 3),     # 32-byte groups, eta 3, odd m
    (300, 32, 4, 1 << 18, 2),           # 16-byte groups (one lane)
    (200, 20, 3, 1 << 16, 4),           # 8-byte groups, eta 4
    (64, 8, 2, 1 << 14, 1),             # 4-byte groups, eta 1
    (500, 64, 6, 12289, 5),             # eta 5: path 3 unsupported, path 1 runs
])
def test_segment_path_matches_oracle(rambo_lib, K, B, R, m, eta):
    torch = _torch()
    p = synth.Params(K=K, B=B, R=R, m=m, eta=eta, k=31, seed=5)
    rng = np.random.default_rng(K + B + eta)
    corpus = synth.family_corpus(rng, p, n_seeds=8, doc_len=14000, sub_rate=0.005)
    # lengths from empty to several cut-pass warp ranges (2,048 k-mers each);
    # most queries from documents, so segments repeat across queries
    lengths = np.concatenate([rng.integers(0, 3000, size=250), [0, 5, 30, 31, 32, 13000, 9000]])
    q = synth.sample_queries(rng, corpus, lengths, 0.8, err_rate=0.001)
    # low-complexity queries: every k-mer (or every other) identical, so each
    # position is a cut candidate and only the minimum length spaces them
    extra = [np.zeros(700, np.uint8), np.tile(np.array([0, 1], np.uint8), 600),
             np.tile(np.array([2, 3, 1], np.uint8), 500)]
    qs = [synth.unpack_bases(q.packed, int(q.offsets[i]), int(q.offsets[i + 1] - q.offsets[i]))
          for i in range(q.n)] + extra
    qp, qo = synth.pack_many(qs)
    o = oracle_index(p, corpus)
    want = o.query_seqs(qp, qo)
    idx = gpu_index(rambo_lib, p, corpus)
    for bits in (1, 4, 8):
        idx.set_tuning(query_path=3, seg_cut_bits=bits)
        assert np.array_equal(gpu_query_seqs(rambo_lib, idx, qp, qo), want), bits
    # twice in a row through one workspace (counters and buckets start over)
    idx.set_tuning(seg_cut_bits=4)
    d_p, d_o = _dev(qp, np.uint8), _dev(qo.astype(np.uint64), np.int64)
    need = idx.workspace_bytes("seqs", qo.size - 1, qp.size)
    buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    ptr = (buf.data_ptr() + 255) // 256 * 256
    for _ in range(2):
        out = idx.query_seqs_dev(d_p, d_o, workspace=(ptr, need))
        idx.sync()
        assert np.array_equal(rambo_lib.as_u32(out), want)
    # misaligned packed pointer, and the host-buffer call
    pad = _dev(np.concatenate([np.zeros(5, np.uint8), qp]), np.uint8)[5:]
    out = idx.query_seqs_dev(pad, d_o)
    idx.sync()
    assert np.array_equal(rambo_lib.as_u32(out), want)
    assert np.array_equal(idx.query_seqs(qp, qo), want)
    # separate ranges (not a CSR batch) and a workspace without room for the
    # segments: path 1 answers
    out = idx.query_ranges_dev(d_p, d_o[:-1].contiguous(), d_o[1:].contiguous())
    idx.sync()
    assert np.array_equal(rambo_lib.as_u32(out), want)
    small = idx.workspace_bytes("seqs", qo.size - 1)
    out = idx.query_seqs_dev(d_p, d_o, workspace=(ptr, small))
    idx.sync()
    assert np.array_equal(rambo_lib.as_u32(out), want)


# ------------------------------------------------ mixed batches (both kinds)

def _mixed_case(seed=5):
    p = synth.Params(K=300, B=16, R=3, m=1 << 14, eta=2, k=31, seed=seed)
    rng = np.random.default_rng(seed)
    corpus = synth.family_corpus(rng, p, n_seeds=15, doc_len=800, sub_rate=0.02)
    kmers = synth.sample_kmers(rng, corpus, 7_001, p.k, 0.5)
    q = synth.sample_queries(rng, corpus, rng.integers(0, 400, size=257), 0.5)
    return p, corpus, kmers, q


def test_query_batch_host_pipelined_chunks_match_oracle(rambo_lib):
    p, corpus, kmers, q = _mixed_case()
    o = oracle_index(p, corpus)
    want_k = o.query_kmers(kmers, threads=4)
    want_s = o.query_seqs(q.packed, q.offsets)
    idx = gpu_index(rambo_lib, p, corpus)
    for chunk in (0, 1000, 7_001, 3):  # auto, ragged last chunk, one chunk, many
        for path in (0, 1, 2):
            for prio in (0, 1, 2):
                idx.set_tuning(host_chunk_kmers=chunk, query_path=path, branch_priority=prio)
                got_k, got_s = idx.query_batch(kmers, q.packed, q.offsets)
                assert np.array_equal(got_k, want_k), (chunk, path, prio)
                assert np.array_equal(got_s, want_s), (chunk, path, prio)
    idx.set_tuning(branch_priority=0)
    for cap in (0, 2):  # the fused launch's CTA cap beside the k-mer chunks
        idx.set_tuning(host_fused_ctas_per_sm=cap, query_path=1)
        got_k, got_s = idx.query_batch(kmers, q.packed, q.offsets)
        assert np.array_equal(got_k, want_k) and np.array_equal(got_s, want_s), cap
    idx.set_tuning(host_fused_ctas_per_sm=1)
    for slots in (1, 2, 4):
        idx.set_tuning(host_chunk_kmers=1000, host_slots=slots)
        got_k, got_s = idx.query_batch(kmers, q.packed, q.offsets)
        assert np.array_equal(got_k, want_k), slots
        assert np.array_equal(got_s, want_s), slots
    idx.set_tuning(host_slots=3)
    # answers written straight into page-locked outputs (and pageable ones staged)
    torch = _torch()
    pin_k = torch.zeros((kmers.size, idx.W), dtype=torch.int32).pin_memory().numpy()
    pin_s = torch.zeros((q.n, idx.W), dtype=torch.int32).pin_memory().numpy()
    for direct in (1, 0):
        for chunk in (0, 1000):
            idx.set_tuning(host_direct=direct, host_chunk_kmers=chunk)
            pin_k[:] = 0
            pin_s[:] = 0
            idx.query_batch(kmers, q.packed, q.offsets, out_kmers=pin_k, out_seqs=pin_s)
            assert np.array_equal(pin_k.view(np.uint32), want_k), (direct, chunk)
            assert np.array_equal(pin_s.view(np.uint32), want_s), (direct, chunk)
            got_k, got_s = idx.query_batch(kmers, q.packed, q.offsets)  # pageable outputs
            assert np.array_equal(got_k, want_k) and np.array_equal(got_s, want_s), (direct, chunk)
    idx.set_tuning(host_direct=0, host_chunk_kmers=0)
    # either part may be empty; the single-kind calls go through the same path
    idx.set_tuning(host_chunk_kmers=1000)
    got_k, got_s = idx.query_batch(kmers, q.packed, q.offsets[:1])
    assert np.array_equal(got_k, want_k) and got_s.shape == (0, idx.W)
    got_k, got_s = idx.query_batch(kmers[:0], q.packed, q.offsets)
    assert np.array_equal(got_s, want_s) and got_k.shape == (0, idx.W)
    assert np.array_equal(idx.query_kmers(kmers), want_k)
    assert np.array_equal(idx.query_seqs(q.packed, q.offsets), want_s)


def test_query_batch_host_rejects_bad_kmer_code_after_running(rambo_lib):
    p, corpus, kmers, q = _mixed_case()
    idx = gpu_index(rambo_lib, p, corpus)
    bad = kmers.copy()
    bad[123] |= np.uint64(1) << np.uint64(2 * p.k)
    with pytest.raises(rambo_lib.RamboError):
        idx.query_batch(bad, q.packed, q.offsets)
    # the error is cleared: the next call succeeds
    o = oracle_index(p, corpus)
    assert np.array_equal(idx.query_kmers(kmers), o.query_kmers(kmers, threads=4))


def test_query_batch_dev_and_graph_capture_match_oracle(rambo_lib):
    torch = _torch()
    p, corpus, kmers, q = _mixed_case(seed=8)
    o = oracle_index(p, corpus)
    want_k = o.query_kmers(kmers, threads=4)
    want_s = o.query_seqs(q.packed, q.offsets)
    idx = gpu_index(rambo_lib, p, corpus)
    d_k, d_p = _dev(kmers, np.int64), _dev(q.packed, np.uint8)
    d_o = _dev(q.offsets.astype(np.uint64), np.int64)
    for path in (0, 1, 2):
        for prio in (0, 1, 2):
            idx.set_tuning(query_path=path, branch_priority=prio)
            ok, os_ = idx.query_batch_dev(d_k, d_p, d_o)
            idx.sync()
            assert np.array_equal(rambo_lib.as_u32(ok), want_k), (path, prio)
            assert np.array_equal(rambo_lib.as_u32(os_), want_s), (path, prio)
    # captured once, replayed twice into zeroed outputs
    for path, prio in ((1, 0), (1, 1), (1, 2), (2, 0)):
        idx.set_tuning(query_path=path, branch_priority=prio)
        out_k = torch.zeros((kmers.size, idx.W), dtype=torch.int32, device="cuda")
        out_s = torch.zeros((q.n, idx.W), dtype=torch.int32, device="cuda")
        idx.query_batch_dev(d_k, d_p, d_o, out_kmers=out_k, out_seqs=out_s)
        idx.sync()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            idx.query_batch_dev(d_k, d_p, d_o, out_kmers=out_k, out_seqs=out_s)
        for _ in range(2):
            out_k.zero_()
            out_s.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert np.array_equal(rambo_lib.as_u32(out_k), want_k), prio
            assert np.array_equal(rambo_lib.as_u32(out_s), want_s), prio
        idx.sync()


def test_early_exit_gives_identical_answers_and_probes_fewer_kmers(rambo_lib):
    p = synth.Params(K=200, B=20, R=3, m=1 << 14, eta=2, k=31, seed=21)
    rng = np.random.default_rng(17)
    corpus = synth.family_corpus(rng, p, n_seeds=20, doc_len=3000, sub_rate=0.01)
    # long random queries die after a few k-mers; document substrings do not
    q = synth.sample_queries(rng, corpus, rng.integers(100, 2500, size=300), 0.5)
    o = oracle_index(p, corpus)
    want = o.query_seqs(q.packed, q.offsets)
    idx = gpu_index(rambo_lib, p, corpus)
    idx.set_tuning(query_path=1, fused_tile_kmers=256, fused_short_max=512, early_exit=0)
    assert np.array_equal(gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets), want)
    idx.set_tuning(early_exit=1, early_exit_segment=128)
    idx.probed_kmers(reset=True)
    got = gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets)
    probed = idx.probed_kmers(reset=True)
    assert np.array_equal(got, want)
    assert 0 < probed < q.n_kmers(p.k)


# ------------------------------------------------------ document sharding

def test_sharded_index_equals_composed_single_index_and_oracle(rambo_lib):
    from paper_1910_04358_gb300 import sharding
    K, b, R, S = 150, 8, 3, 3
    p = synth.Params(K=K, B=S * b, R=R, m=1 << 14, eta=2, k=31, seed=4)
    rng = np.random.default_rng(23)
    corpus = synth.family_corpus(rng, p, n_seeds=10, doc_len=600, sub_rate=0.02)
    q = synth.sample_queries(rng, corpus, rng.integers(31, 300, size=200), 0.6)
    sh = sharding.ShardedIndex(K, b, R, p.m, p.eta, p.k, p.seed, shards=S)
    sh.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    got = sh.query_seqs(q.packed, q.offsets)
    phi = sh.composed_partition()
    one = rambo_lib.Index(K, S * b, R, p.m, p.eta, p.k, p.seed)
    one.set_partition(phi)
    one.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    assert np.array_equal(one.query_seqs(q.packed, q.offsets), got)
    o = oracle.Rambo(K, S * b, R, p.m, p.eta, p.k, p.seed)
    o.set_partition(phi)
    o.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    assert np.array_equal(o.query_seqs(q.packed, q.offsets), got)
    with pytest.raises(rambo_lib.RamboError) as e:
        one.set_partition(phi)  # after inserts
    assert e.value.code == rambo_lib.RAMBO_ESTATE


# --------------------------------------------------- documents of words (5.4)

def test_word_documents_match_oracle(rambo_lib):
    rng = np.random.default_rng(101)
    vocab = synth.word_vocabulary(rng, 6000)
    K, B, R, m, eta = 300, 20, 3, 100_003, 2
    docs = synth.word_corpus(rng, K, vocab, 150)
    idx = rambo_lib.Index(K, B, R, m, eta, seed=5)
    o = oracle.Rambo(K, B, R, m, eta, seed=5)
    words_of = [[vocab[i] for i in d] for d in docs]
    # insert in two batches through the device API
    idx.insert_words(np.arange(0, 150, dtype=np.uint32), words_of[:150])
    idx.insert_words(np.arange(150, K, dtype=np.uint32), words_of[150:])
    for d in range(K):
        o.insert_words(d, words_of[d])
    assert_index_equal(idx, o, synth.Params(K=K, B=B, R=R, m=m, eta=eta))
    queries = []
    for i in range(400):
        if i % 3:
            d = int(rng.integers(0, K))
            queries.append([vocab[j] for j in rng.choice(docs[d], size=int(rng.integers(1, 4)), replace=False)])
        else:
            queries.append([vocab[int(j)] for j in rng.integers(0, len(vocab), size=int(rng.integers(1, 3)))])
    got = idx.query_words(queries)
    want = np.stack([o.query_words(q) for q in queries])
    assert np.array_equal(got, want)


# ------------------------------------- document shards: range inserts, merge

@pytest.mark.parametrize("mode", [2, 3])
def test_insert_ranges_subset_and_overlap_match_oracle(rambo_lib, mode):
    # a shard inserts some of a corpus's documents straight from the shared
    # packed stream: out of order, one twice (idempotent), and a range that
    # overlaps another (insert_mode 3 takes the direct insert for ranges)
    torch = _torch()
    p = synth.Params(K=60, B=16, R=3, m=1 << 14, eta=2, k=31, seed=12)
    rng = np.random.default_rng(7)
    corpus = synth.family_corpus(rng, p, n_seeds=8, doc_len=700, sub_rate=0.02)
    offs = corpus.offsets.astype(np.int64)
    pick = np.array([40, 3, 17, 3, 59, 22], dtype=np.int64)
    begins, ends = offs[pick].copy(), offs[pick + 1].copy()
    begins[-1] = offs[17] + 100  # doc 22's slot reads part of doc 17 instead
    ends[-1] = offs[18] + 50
    idx = rambo_lib.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    idx.set_tuning(insert_mode=mode)
    idx.insert_ranges_dev(_dev(pick.astype(np.int32), np.int32), _dev(corpus.packed, np.uint8),
                          _dev(begins, np.int64), _dev(ends, np.int64))
    idx.sync()
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    for d, b0, b1 in zip(pick.tolist(), begins.tolist(), ends.tolist()):
        o.insert(d, corpus.packed, b0, b1 - b0)
    assert_index_equal(idx, o, p)
    assert_docbits_equal(idx, o, p)
    q = synth.sample_queries(rng, corpus, rng.integers(25, 300, size=120), 0.7)
    assert np.array_equal(gpu_query_seqs(rambo_lib, idx, q.packed, q.offsets), o.query_seqs(q.packed, q.offsets))


def test_merge_shard_answers_places_bits_at_global_ids(rambo_lib):
    torch = _torch()
    from paper_1910_04358_gb300 import sharding
    rng = np.random.default_rng(3)
    K, n, S = 1000, 300, 3
    tau = sharding.route(K, S, seed=5)
    mem = sharding.members(tau, S)
    parts, out = [], torch.zeros((n, (K + 31) // 32), dtype=torch.int32, device="cuda")
    for s in range(S):
        ws = (mem[s].size + 31) // 32 + 1  # a padded shard row
        local = rng.integers(0, 1 << 32, size=(n, ws), dtype=np.uint64).astype(np.uint32)
        local[:, (mem[s].size + 31) // 32:] = 0
        if mem[s].size % 32:
            local[:, mem[s].size // 32] &= np.uint32((1 << (mem[s].size % 32)) - 1)
        parts.append((local, mem[s]))
        rambo_lib.merge_shard_answers(_dev(local.view(np.int32), np.int32).view(n, ws),
                                      _dev(mem[s].astype(np.int32), np.int32), out)
    torch.cuda.synchronize()
    assert np.array_equal(rambo_lib.as_u32(out), sharding.merge_answers_host(n, K, parts))
