"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle against something the paper or the mathematics
fixes: published hash test values, string-level brute force, exact k-mer
sets on tiny inputs, the Lemma 4.1 false-positive bound, the bucket-space
AND identity of Algorithm 2 vs Section 3.3.1, and degenerate cases that
reduce to a plain Bloom filter or to the exact answer.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1910_04358_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

COMP = str.maketrans("ACGT", "TGCA")
DIGIT = {"A": 0, "C": 1, "G": 2, "T": 3}


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.rstrip("\n")
            if not line or line.startswith("#"):
                continue
            key, _, val = line.partition(" ")
            out[key] = val
    return out


def _str(bases):
    return "".join("ACGT"[b] for b in bases)


def _code(s):
    v = 0
    for ch in s:
        v = v * 4 + DIGIT[ch]
    return v


def _canon_str(s):
    rc = s.translate(COMP)[::-1]
    return min(s, rc)  # lexicographic in A<C<G<T


# ---------------------------------------------------------------- hash pins

def test_mmh3_smhasher_verification_code():
    g = _golden("mmh3_x64_128.txt")
    key = bytes(range(256))
    buf = b""
    for i in range(256):
        h1, h2 = oracle.mmh3_x64_128(key[:i], 256 - i)
        buf += h1.to_bytes(8, "little") + h2.to_bytes(8, "little")
    f1, _ = oracle.mmh3_x64_128(buf, 0)
    assert (f1 & 0xFFFFFFFF) == int(g["verification"], 16)


def test_mmh3_published_vector_and_empty_key():
    g = _golden("mmh3_x64_128.txt")
    h1, h2 = oracle.mmh3_x64_128(g["quickbrownfox"].encode(), 0)
    digest = (h1.to_bytes(8, "little") + h2.to_bytes(8, "little")).hex()
    assert digest == g["quickbrownfox_digest"]
    assert oracle.mmh3_x64_128(b"", 0) == (0, 0)


def test_probe_and_partition_use_first_word_of_8_byte_key():
    # The oracle's probe position and partition must be the first word of the
    # (pinned) general hash over the 8-byte little-endian key, reduced mod m / B.
    o = oracle.Rambo(K=50, B=7, R=3, m=1000003, eta=3, k=31, seed=5)
    rng = np.random.default_rng(1)
    for x in rng.integers(0, 1 << 62, size=20, dtype=np.uint64).tolist():
        for j in range(3):
            h1, _ = oracle.mmh3_x64_128(int(x).to_bytes(8, "little"), 5 + j)
            assert o.probe_position(x, j) == h1 % 1000003
    for d in range(50):
        for r in range(3):
            h1, _ = oracle.mmh3_x64_128(d.to_bytes(8, "little"), 5 + 1000 + r)
            assert o.bucket(d, r) == h1 % 7 == o.partition(d, r)


# --------------------------------------------------------- packing / k-mers

def test_packing_hand_values():
    # A C G T -> 0,1,2,3 at bit pairs 0,2,4,6 of byte 0: 0b11100100
    packed = synth.pack_bases(np.array([0, 1, 2, 3, 3, 0], dtype=np.uint8))
    assert packed.tolist() == [0xE4, 0x03]
    assert oracle.unpack(packed, 0, 6).tolist() == [0, 1, 2, 3, 3, 0]
    assert oracle.unpack(packed, 3, 2).tolist() == [3, 3]


def test_kmer_codes_match_string_brute_force():
    rng = np.random.default_rng(7)
    for k in (1, 2, 5, 15, 31, 32):
        bases = rng.integers(0, 4, size=k + 40, dtype=np.uint8)
        packed = synth.pack_bases(bases)
        s = _str(bases)
        for i in range(0, 41):
            w = s[i:i + k]
            assert oracle.kmer_forward(packed, i, k) == _code(w)
            assert oracle.kmer_canonical(packed, i, k) == _code(_canon_str(w))
            assert oracle.canonical_of_code(_code(w), k) == _code(_canon_str(w))


def test_canonical_is_strand_symmetric():
    rng = np.random.default_rng(8)
    for _ in range(200):
        s = _str(rng.integers(0, 4, size=31))
        rc = s.translate(COMP)[::-1]
        assert oracle.canonical_of_code(_code(s), 31) == oracle.canonical_of_code(_code(rc), 31)


# ----------------------------------------------------------- brute force

def _exact_sets(corpus, k):
    sets = []
    for i in range(corpus.params.K):
        s = _str(corpus.doc_bases(i))
        sets.append({_canon_str(s[t:t + k]) for t in range(len(s) - k + 1)})
    return sets


def _build(p, corpus):
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    o.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    return o


def _small_case(K=40, doc_len=600, B=5, R=3, m=1 << 13, eta=2, k=15, n_q=120, qlen=30, seed=0):
    p = synth.Params(K=K, B=B, R=R, m=m, eta=eta, k=k, seed=seed)
    rng = np.random.default_rng(1234 + K + B + R)
    corpus = synth.family_corpus(rng, p, n_seeds=4, doc_len=doc_len, sub_rate=0.03)
    q = synth.sample_queries(rng, corpus, rng.integers(k - 2, qlen + 1, size=n_q), 0.6)
    return p, corpus, q


def _lemma_4_1(o, p, V, d):
    """Lemma 4.1 for document d and a term of multiplicity V: in each
    repetition the merge term 1-(1-1/B)^V plus the Bloom failure term
    p_r (1-1/B)^V, with p_r the measured false-positive rate (fill^eta) of
    the BFU that holds d; repetitions multiply (the lemma's independence)."""
    a = (1 - 1 / p.B) ** V
    f = 1.0
    for r in range(p.R):
        pr = o.fill_fraction(r, o.bucket(d, r)) ** p.eta
        f *= pr * a + 1 - a
    return f


def test_zero_false_negatives_and_fp_bound_lemma_4_1():
    # >= 20 documents per bucket, where a document's own terms are a small
    # share of its BFU (the lemma treats repetitions as independent).
    p, corpus, q = _small_case(K=120, B=5, R=3, m=1 << 16, n_q=150, qlen=30)
    o = _build(p, corpus)
    exact = _exact_sets(corpus, p.k)
    res = o.query_seqs(q.packed, q.offsets)
    fp_obs, fp_exp, var = 0, 0.0, 0.0
    n_single = 0
    for i in range(q.n):
        s = _str(synth.unpack_bases(q.packed, int(q.offsets[i]), int(q.offsets[i + 1] - q.offsets[i])))
        terms = {_canon_str(s[t:t + p.k]) for t in range(len(s) - p.k + 1)}
        truth = {d for d in range(p.K) if terms <= exact[d]}
        got = oracle.mask_to_docs(res[i])
        assert truth <= got, f"false negative on query {i}"
        if len(terms) == 1:
            n_single += 1
            for d in set(range(p.K)) - truth:
                f = _lemma_4_1(o, p, len(truth), d)
                fp_exp += f
                var += f * (1 - f)
            fp_obs += len(got - truth)
    assert n_single >= 5
    assert fp_obs <= fp_exp + 4 * math.sqrt(var) + 3


def test_single_term_fp_rate_within_lemma_4_1_protocol():
    # Section 5.2 evaluation protocol: random unseen terms, each inserted into
    # V documents with V ~ Exp(alpha) (clipped to [1, K]), then queried.
    K, B, R, k, eta = 400, 20, 3, 31, 2
    m = 1 << 16
    rng = np.random.default_rng(99)
    p = synth.Params(K=K, B=B, R=R, m=m, eta=eta, k=k)
    corpus = synth.uniform_corpus(rng, p, 200)
    o = _build(p, corpus)
    present = set()
    for i in range(K):
        s = _str(corpus.doc_bases(i))
        present |= {_canon_str(s[t:t + k]) for t in range(len(s) - k + 1)}
    terms, owners = [], []
    while len(terms) < 200:
        s = _str(rng.integers(0, 4, size=k))
        if _canon_str(s) in present:
            continue
        # alpha = 100 on the paper's 4605-document scale, here scaled to K
        V = int(min(K, max(1, round(rng.exponential(100.0 * K / 4605)))))
        docs = rng.choice(K, size=V, replace=False)
        for d in docs:
            o.insert(int(d), synth.pack_bases(np.array([DIGIT[c] for c in s], np.uint8)), 0, k)
        terms.append(s)
        owners.append(set(int(d) for d in docs))
    fp_obs, fp_exp, var = 0, 0.0, 0.0
    delta_sum = 0.0
    pbar = float(np.mean([o.fill_fraction(r, b) ** eta for r in range(R) for b in range(B)]))
    for s, own in zip(terms, owners):
        got = oracle.mask_to_docs(o.query_kmer(_code(s)))
        assert own <= got
        for d in set(range(K)) - own:
            f = _lemma_4_1(o, p, len(own), d)
            fp_exp += f
            var += f * (1 - f)
        fp_obs += len(got - own)
        # Lemma 4.2: P(any false positive) <= K (1 - (1-p)(1-1/B)^V)^R
        delta_sum += min(1.0, K * (1 - (1 - pbar) * (1 - 1 / B) ** len(own)) ** R)
    assert fp_obs <= fp_exp + 4 * math.sqrt(var) + 3
    n_any = sum(1 for s, own in zip(terms, owners)
                if oracle.mask_to_docs(o.query_kmer(_code(s))) - own)
    assert n_any <= delta_sum + 4 * math.sqrt(delta_sum) + 3


def test_bucket_space_and_identity():
    # Algorithm 2 ("Q in BFU" = every term passes) equals Section 3.3.1
    # (intersection of the per-term answers), because every repetition
    # partitions the documents.
    p, corpus, q = _small_case(K=60, B=6, R=2, m=1 << 12, k=11, n_q=80, qlen=40)
    o = _build(p, corpus)
    res = o.query_seqs(q.packed, q.offsets)
    for i in range(q.n):
        b0, b1 = int(q.offsets[i]), int(q.offsets[i + 1])
        s = _str(synth.unpack_bases(q.packed, b0, b1 - b0))
        if len(s) < p.k:
            continue
        inter = set(range(p.K))
        for t in range(len(s) - p.k + 1):
            inter &= oracle.mask_to_docs(o.query_kmer(_code(s[t:t + p.k])))
        assert inter == oracle.mask_to_docs(res[i])


def test_b1_r1_is_one_bloom_filter_over_the_union():
    K, k, eta, m = 12, 9, 3, 1 << 11
    p = synth.Params(K=K, B=1, R=1, m=m, eta=eta, k=k, seed=3)
    rng = np.random.default_rng(5)
    corpus = synth.uniform_corpus(rng, p, 80)
    o = _build(p, corpus)
    # plain Bloom filter over the union of all documents' terms, Section 2.1
    bf = np.zeros(m, dtype=bool)
    for i in range(K):
        s = _str(corpus.doc_bases(i))
        for t in range(len(s) - k + 1):
            x = _code(_canon_str(s[t:t + k]))
            for j in range(eta):
                bf[oracle.mmh3_x64_128(x.to_bytes(8, "little"), 3 + j)[0] % m] = True
    q = synth.sample_queries(rng, corpus, np.full(200, 12), 0.3)
    res = o.query_seqs(q.packed, q.offsets)
    for i in range(q.n):
        s = _str(synth.unpack_bases(q.packed, int(q.offsets[i]), 12))
        ok = all(bf[oracle.mmh3_x64_128(_code(_canon_str(s[t:t + k])).to_bytes(8, "little"), 3 + j)[0] % m]
                 for t in range(len(s) - k + 1) for j in range(eta))
        assert oracle.mask_to_docs(res[i]) == (set(range(K)) if ok else set())


def test_injective_partition_and_large_filters_give_exact_answer():
    # With B >= K and every phi_r injective there are no merge false positives;
    # with m >> inserted terms no Bloom collisions: the answer is exact.
    K, B, R, k = 6, 16, 2, 13
    seed = next(s for s in range(1000)
                if all(len({oracle.Rambo(K, B, R, 64, 1, k, s).bucket(d, r) for d in range(K)}) == K
                       for r in range(R)))
    p = synth.Params(K=K, B=B, R=R, m=1 << 22, eta=2, k=k, seed=seed)
    rng = np.random.default_rng(11)
    corpus = synth.family_corpus(rng, p, 2, 120, 0.05)
    o = _build(p, corpus)
    exact = _exact_sets(corpus, k)
    q = synth.sample_queries(rng, corpus, rng.integers(k, 30, size=100), 0.8)
    res = o.query_seqs(q.packed, q.offsets)
    for i in range(q.n):
        s = _str(synth.unpack_bases(q.packed, int(q.offsets[i]), int(q.offsets[i + 1] - q.offsets[i])))
        terms = {_canon_str(s[t:t + k]) for t in range(len(s) - k + 1)}
        assert oracle.mask_to_docs(res[i]) == {d for d in range(K) if terms <= exact[d]}


def test_single_document_is_one_bloom_filter():
    p, corpus, q = _small_case(K=1, B=3, R=2, m=1 << 10, k=7, n_q=60, qlen=12)
    o = _build(p, corpus)
    res = o.query_seqs(q.packed, q.offsets)
    s0 = _str(corpus.doc_bases(0))
    for i in range(q.n):
        s = _str(synth.unpack_bases(q.packed, int(q.offsets[i]), int(q.offsets[i + 1] - q.offsets[i])))
        terms = {_code(_canon_str(s[t:t + 7])) for t in range(len(s) - 7 + 1)}
        hits = all(
            all(o.filter_bit(r, o.bucket(0, r), o.probe_position(x, j)) for j in range(p.eta))
            for x in terms for r in range(p.R))
        assert oracle.mask_to_docs(res[i]) == ({0} if hits else set())
        # every true term of the single document passes (no false negatives)
        if all(s[t:t + 7] in s0 or _canon_str(s[t:t + 7]) in
               {_canon_str(s0[u:u + 7]) for u in range(len(s0) - 6)} for t in range(len(s) - 6)):
            assert res[i][0] & 1


# --------------------------------------------------------------- invariants

def test_monotone_in_subsequences():
    p, corpus, q = _small_case(K=30, B=4, R=2, m=1 << 12, k=9, n_q=40, qlen=40)
    o = _build(p, corpus)
    rng = np.random.default_rng(3)
    for i in range(q.n):
        b0, b1 = int(q.offsets[i]), int(q.offsets[i + 1])
        if b1 - b0 < p.k + 2:
            continue
        full = oracle.mask_to_docs(o.query_seq(q.packed, b0, b1 - b0))
        a = int(rng.integers(b0, b1 - p.k))
        e = int(rng.integers(a + p.k, b1 + 1))
        assert full <= oracle.mask_to_docs(o.query_seq(q.packed, a, e - a))


def test_more_documents_never_remove_answers_and_reinsert_is_idempotent():
    p, corpus, q = _small_case(K=40, B=5, R=3, m=1 << 12)
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    half = p.K // 2
    o.insert_batch(corpus.doc_ids[:half], corpus.packed, corpus.offsets[:half + 1])
    r1 = o.query_seqs(q.packed, q.offsets)
    o.insert_batch(corpus.doc_ids[half:], corpus.packed, corpus.offsets[half:])
    r2 = o.query_seqs(q.packed, q.offsets)
    assert np.all((r1 & ~r2) == 0)
    o.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    r3 = o.query_seqs(q.packed, q.offsets)
    assert np.array_equal(r2, r3)
    # threads only spend host cores: same answers
    o2 = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    o2.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets, threads=4)
    assert np.array_equal(o2.query_seqs(q.packed, q.offsets, threads=3), r2)


def test_empty_term_set_returns_inserted_documents():
    p, corpus, _ = _small_case(K=40, B=5, R=3)
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    ids = np.array([1, 5, 33], dtype=np.uint32)
    offs = np.array([0, 100, 200, 300], dtype=np.uint64)
    o.insert_batch(ids, corpus.packed, offs)
    short = o.query_seq(corpus.packed, 0, p.k - 1)
    assert oracle.mask_to_docs(short) == {1, 5, 33}
    assert oracle.mask_to_docs(o.query_seq(corpus.packed, 0, 0)) == {1, 5, 33}


def test_restricted_mode_matches_full_mode():
    p, corpus, q = _small_case(K=40, B=5, R=3, m=1 << 13)
    full = _build(p, corpus)
    want = full.query_seqs(q.packed, q.offsets)
    pos = set()
    for i in range(q.n):
        b0, b1 = int(q.offsets[i]), int(q.offsets[i + 1])
        for t in range(b0, b1 - p.k + 1):
            x = oracle.kmer_canonical(q.packed, t, p.k)
            pos |= {full.probe_position(x, j) for j in range(p.eta)}
    rs = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, tracked=sorted(pos))
    rs.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets, threads=2)
    assert np.array_equal(rs.query_seqs(q.packed, q.offsets), want)


def test_bulk_positions_match_string_brute_force_and_tracking_oracle_is_exact():
    # positions of every window: string-level canonical k-mer, then the pinned
    # byte-string hash of its 8-byte code, first word mod m
    p, corpus, q = _small_case(K=40, B=5, R=3, m=1 << 13)
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    got = o.seq_positions(q.packed, q.offsets)
    want = []
    for i in range(q.n):
        s = _str(oracle.unpack(q.packed, int(q.offsets[i]), int(q.offsets[i + 1] - q.offsets[i])))
        for t in range(len(s) - p.k + 1):
            c = _code(_canon_str(s[t:t + p.k]))
            want.append([oracle.mmh3_x64_128(c.to_bytes(8, "little"), p.seed + j)[0] % p.m
                         for j in range(p.eta)])
    assert got.shape == (len(want), p.eta) and got.tolist() == want
    kmers = synth.sample_kmers(np.random.default_rng(3), corpus, 30, p.k, 0.5)
    kp = o.kmer_positions(kmers)
    for x, row in zip(kmers.tolist(), kp.tolist()):
        s = "".join("ACGT"[(int(x) >> (2 * (p.k - 1 - i))) & 3] for i in range(p.k))
        c = _code(_canon_str(s))
        assert row == [oracle.mmh3_x64_128(c.to_bytes(8, "little"), p.seed + j)[0] % p.m
                       for j in range(p.eta)]
    # the tracking oracle answers those queries exactly as the full one
    full = _build(p, corpus)
    t = oracle.tracking_oracle(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed,
                               seqs=[(q.packed, q.offsets)], kmers=kmers)
    t.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets, threads=2)
    assert np.array_equal(t.query_seqs(q.packed, q.offsets), full.query_seqs(q.packed, q.offsets))
    assert np.array_equal(t.query_kmers(kmers), full.query_kmers(kmers))


def test_position_bits_match_per_filter_bits():
    p, corpus, q = _small_case(K=40, B=5, R=3, m=1 << 13)
    o = _build(p, corpus)
    rng = np.random.default_rng(9)
    pos = rng.integers(0, p.m, size=200).astype(np.uint64)
    got = o.position_bits(pos)
    assert got.shape == (200, (p.R * p.B + 7) // 8)
    for i, x in enumerate(pos.tolist()):
        for r in range(p.R):
            for b in range(p.B):
                f = r * p.B + b
                assert (got[i, f // 8] >> (f % 8)) & 1 == o.filter_bit(r, b, x)
    # restricted mode: tracked positions agree, an untracked one is refused
    t = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed, tracked=pos[:50])
    t.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    assert np.array_equal(t.position_bits(pos[:50]), got[:50])
    untracked = int(np.setdiff1d(np.arange(p.m, dtype=np.uint64), pos[:50])[0])
    with pytest.raises(oracle.OracleError):
        t.position_bits([untracked])


def test_invalid_arguments():
    with pytest.raises(oracle.OracleError):
        oracle.Rambo(0, 1, 1, 8, 1)
    o = oracle.Rambo(4, 2, 1, 64, 1, k=5)
    with pytest.raises(oracle.OracleError):
        o.insert(4, np.zeros(4, np.uint8), 0, 8)
    with pytest.raises(oracle.OracleError):
        o.query_kmer(1 << 10)  # bit at or above 2k


# ------------------------------------------------------------------ folding

def test_fold_equals_index_built_with_half_the_buckets():
    # phi_r(d) = h mod B and B/2 divides B, so folding B -> B/2 must give the
    # index built directly with B/2 buckets, filter for filter and answer for answer
    p, corpus, q = _small_case(K=50, B=8, R=3, m=1 << 12)
    o = _build(p, corpus)
    before = o.query_seqs(q.packed, q.offsets)
    o.fold()
    ph = synth.Params(K=p.K, B=p.B // 2, R=p.R, m=p.m, eta=p.eta, k=p.k, seed=p.seed)
    direct = _build(ph, corpus)
    for r in range(p.R):
        for b in range(ph.B):
            assert np.array_equal(o.filter_words(r, b), direct.filter_words(r, b))
        for d in range(p.K):
            assert o.bucket(d, r) == direct.bucket(d, r)
    after = o.query_seqs(q.packed, q.offsets)
    assert np.array_equal(after, direct.query_seqs(q.packed, q.offsets))
    # folding only adds false positives: the folded answer contains the original one
    assert np.all((before & ~after) == 0)
    with pytest.raises(oracle.OracleError):
        odd = oracle.Rambo(10, 3, 1, 64, 1, k=5)
        odd.fold()


# ---------------------------------------------------- stacked shards (5.3)

def test_stacked_shards_equal_one_rambo_with_composed_bucket_map():
    # Section 5.3: S node-local RAMBOs of b buckets over disjoint documents
    # equal one RAMBO of S*b buckets with bucket map b*tau(D) + phi(D); the
    # global answer is the concatenation of the shards' answers.
    K, b, R, S = 90, 4, 3, 3
    p = synth.Params(K=K, B=b, R=R, m=1 << 12, eta=2, k=15)
    rng = np.random.default_rng(13)
    corpus = synth.family_corpus(rng, p, n_seeds=6, doc_len=400, sub_rate=0.02)
    q = synth.sample_queries(rng, corpus, rng.integers(15, 60, size=80), 0.7)
    tau = np.arange(K) % S
    shards, members = [], []
    for s in range(S):
        mem = np.nonzero(tau == s)[0]
        o = oracle.Rambo(mem.size, b, R, p.m, p.eta, p.k, p.seed)
        for li, d in enumerate(mem):
            o.insert(li, corpus.packed, int(corpus.offsets[d]), int(corpus.offsets[d + 1] - corpus.offsets[d]))
        shards.append(o)
        members.append(mem)
    phi = np.zeros((K, R), dtype=np.uint32)
    for s, (o, mem) in enumerate(zip(shards, members)):
        for li, d in enumerate(mem):
            for r in range(R):
                phi[d, r] = b * s + o.bucket(li, r)
    g = oracle.Rambo(K, S * b, R, p.m, p.eta, p.k, p.seed)
    g.set_partition(phi)
    g.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    want = g.query_seqs(q.packed, q.offsets)
    for i in range(q.n):
        b0, b1 = int(q.offsets[i]), int(q.offsets[i + 1])
        cat = set()
        for o, mem in zip(shards, members):
            cat |= {int(mem[li]) for li in oracle.mask_to_docs(o.query_seq(q.packed, b0, b1 - b0))}
        assert cat == oracle.mask_to_docs(want[i])


# ---------------------------------------------------- documents of words (5.4)

def test_word_documents_zero_fn_and_word_positions():
    # word positions are the general-length hash (pinned above) mod m; a
    # document's own words always pass, a query of several words passes only
    # documents containing all of them (up to Bloom and merge false positives)
    rng = np.random.default_rng(77)
    vocab = [bytes(rng.integers(97, 123, size=int(L)).astype(np.uint8)) for L in rng.integers(2, 14, 400)]
    K = 60
    o = oracle.Rambo(K, 6, 3, 1 << 14, 2, seed=9)
    docs = [set(rng.choice(len(vocab), size=40, replace=False).tolist()) for _ in range(K)]
    for d in range(K):
        o.insert_words(d, [vocab[i] for i in sorted(docs[d])])
    for w in vocab[:20]:
        for j in range(2):
            assert o.word_position(w, j) == oracle.mmh3_x64_128(w, 9 + j)[0] % (1 << 14)
    for _ in range(100):
        qs = rng.choice(len(vocab), size=int(rng.integers(1, 4)), replace=False).tolist()
        got = oracle.mask_to_docs(o.query_words([vocab[i] for i in qs]))
        truth = {d for d in range(K) if set(qs) <= docs[d]}
        assert truth <= got
        # bucket-space identity for word queries
        inter = set(range(K))
        for i in qs:
            inter &= oracle.mask_to_docs(o.query_words([vocab[i]]))
        assert inter == got
