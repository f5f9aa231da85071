"""Continuous batching returns, for every request, exactly the answer of that
request queried alone -- whatever batch it landed in, whatever else was in
flight -- and the same answers as the plain fixed-batch server."""
import numpy as np
import pytest

from paper_1910_04358_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served(rambo_lib):
    # the large workload's index shape (10,000 documents, R = 5, B = 100,
    # 64-byte groups) with short documents, its query path and tuning
    from paper_1910_04358_gb300 import serve
    p = synth.Params(K=10_000, B=100, R=5, m=1 << 24, eta=2, k=31, seed=0)
    rng = np.random.default_rng(8)
    corpus = synth.family_corpus(rng, p, n_seeds=200, doc_len=2_000, sub_rate=0.005, indel_rate=0.0005)
    idx = rambo_lib.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    idx.set_tuning(query_path=1, fused_tile_kmers=4096, fused_short_max=1024)
    idx.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    arrivals, lengths = synth.serving_trace(rng, 600, rate_per_s=40_000.0, median=300, hi=3000)
    reqs = serve.make_requests(corpus, arrivals, lengths, rng)
    eng = serve.ServingEngine(idx, slots=3, max_batch_queries=24, max_batch_bytes=1 << 16,
                              mask_budget_bytes=40 * idx.W * 4)
    res = eng.serve(reqs)
    return idx, reqs, res


def test_each_answer_equals_the_request_alone(served):
    idx, reqs, res = served
    for r in reqs:
        alone = idx.query_seqs(r.packed, np.array([0, r.n_bases], dtype=np.uint64))[0]
        assert np.array_equal(res.answers[r.rid], alone), f"request {r.rid}"


def test_batches_overlapped_and_budget_respected(served):
    idx, reqs, res = served
    s = res.summary()
    assert s["requests"] == len(reqs)
    assert s["batches"] >= len(reqs) // 24
    assert res.max_in_flight <= 3
    assert res.max_in_flight >= 1
    assert np.all(res.latency_s >= 0)


def test_plain_batched_gives_the_same_answers(served, rambo_lib):
    from paper_1910_04358_gb300 import serve
    idx, reqs, res = served
    plain = serve.plain_batched(idx, reqs, batch_size=64)
    for r in reqs:
        assert np.array_equal(plain.answers[r.rid], res.answers[r.rid])


def test_large_batches_at_saturation_match(served, rambo_lib):
    # every request present at once: the engine forms its largest batches
    from paper_1910_04358_gb300 import serve
    idx, reqs, res = served
    at_once = [serve.Request(r.rid, r.packed, r.n_bases, 0.0) for r in reqs]
    big = serve.ServingEngine(idx, slots=2).serve(at_once)
    assert big.batches <= 2
    assert np.array_equal(big.answers, res.answers)
