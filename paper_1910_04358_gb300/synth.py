"""Seeded synthetic genomes, documents and queries.

This module holds no part of the method: it draws random DNA, mutates it,
packs it in the library's 2-bit input format and samples queries.  Both the
CUDA path and the CPU oracle consume what it produces; nothing here hashes,
canonicalises or probes.

Inputs stand in for the paper's ENA whole-genome-sequencing files (Section
5.2, "Dataset"), which are not available: documents are families of mutated
copies of uniform random seed genomes, so k-mers are shared within a family
the way they are shared between related microbial samples.

Packed format (the library's input format): base t of a stream sits in byte
t >> 2 at bits 2*(t & 3) .. 2*(t & 3)+1; A=0, C=1, G=2, T=3.  A batch of
sequences is one packed stream plus CSR base offsets (n + 1 values): sequence
i is bases [offsets[i], offsets[i+1]).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GEN_SEED_BASE = 0x52414D42  # "RAMB"


# --------------------------------------------------------------------------
# packing


def pack_bases(bases: np.ndarray) -> np.ndarray:
    """Packs an array of base codes (0..3) four to a byte, first base lowest."""
    b = np.ascontiguousarray(bases, dtype=np.uint8)
    n = b.size
    pad = (-n) % 4
    if pad:
        b = np.concatenate([b, np.zeros(pad, dtype=np.uint8)])
    q = b.reshape(-1, 4)
    return (q[:, 0] | (q[:, 1] << 2) | (q[:, 2] << 4) | (q[:, 3] << 6)).astype(np.uint8)


def unpack_bases(packed: np.ndarray, begin: int, n: int) -> np.ndarray:
    """Inverse of :func:`pack_bases` for bases [begin, begin + n)."""
    t = np.arange(begin, begin + n, dtype=np.int64)
    return ((packed[t >> 2] >> (2 * (t & 3)).astype(np.uint8)) & 3).astype(np.uint8)


class PackedStream:
    """Appends base arrays to one packed stream, tracking CSR base offsets."""

    def __init__(self):
        self._chunks: list[np.ndarray] = []
        self._carry = np.zeros(0, dtype=np.uint8)
        self.offsets = [0]

    def append(self, bases: np.ndarray):
        bases = np.asarray(bases, dtype=np.uint8)
        self.offsets.append(self.offsets[-1] + int(bases.size))
        buf = np.concatenate([self._carry, bases]) if self._carry.size else bases
        whole = (buf.size // 4) * 4
        if whole:
            self._chunks.append(pack_bases(buf[:whole]))
        self._carry = buf[whole:].copy()

    def finish(self) -> tuple[np.ndarray, np.ndarray]:
        chunks = list(self._chunks)
        if self._carry.size:
            chunks.append(pack_bases(self._carry))
        # 16 bytes of zero padding keep any whole-word read of the stream in bounds
        chunks.append(np.zeros(16, dtype=np.uint8))
        packed = np.concatenate(chunks) if chunks else np.zeros(16, dtype=np.uint8)
        return packed, np.asarray(self.offsets, dtype=np.uint64)


def pack_many(seqs: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    s = PackedStream()
    for x in seqs:
        s.append(x)
    return s.finish()


def codes_from_windows(windows: np.ndarray) -> np.ndarray:
    """Library k-mer input format: forward code, first base most significant."""
    w = np.asarray(windows, dtype=np.uint64)
    k = w.shape[1]
    shifts = (2 * (k - 1 - np.arange(k))).astype(np.uint64)
    return np.bitwise_or.reduce(w << shifts[None, :], axis=1).astype(np.uint64)


# --------------------------------------------------------------------------
# random DNA


def uniform_genome(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.integers(0, 4, size=n, dtype=np.uint8)


def substitute(rng: np.random.Generator, seq: np.ndarray, rate: float) -> np.ndarray:
    """i.i.d. point substitutions, each to one of the other three bases."""
    out = seq.copy()
    if rate <= 0 or seq.size == 0:
        return out
    nsub = rng.binomial(seq.size, rate)
    pos = rng.choice(seq.size, size=nsub, replace=False) if nsub else np.zeros(0, np.int64)
    out[pos] = (out[pos] + rng.integers(1, 4, size=nsub, dtype=np.uint8)) & 3
    return out


def indels(rng: np.random.Generator, seq: np.ndarray, rate: float, max_len: int = 10):
    """Short insertions/deletions (50/50) at `rate` events per base, length U[1, max_len]."""
    if rate <= 0 or seq.size == 0:
        return seq
    nev = rng.binomial(seq.size, rate)
    if nev == 0:
        return seq
    pos = np.sort(rng.choice(seq.size, size=nev, replace=False))
    lens = rng.integers(1, max_len + 1, size=nev)
    is_ins = rng.random(nev) < 0.5
    keep = np.ones(seq.size, dtype=bool)
    for p, ln in zip(pos[~is_ins], lens[~is_ins]):
        keep[p:p + ln] = False
    ins_pos, ins_len = pos[is_ins], lens[is_ins]
    out = np.insert(seq, np.repeat(ins_pos, ins_len),
                    rng.integers(0, 4, size=int(ins_len.sum()), dtype=np.uint8))
    # deletions are applied on the original coordinates: map keep-mask through insertion
    keep_full = np.insert(keep, np.repeat(ins_pos, ins_len), True)
    return out[keep_full]


# --------------------------------------------------------------------------
# workloads


@dataclass
class Params:
    K: int
    B: int
    R: int
    m: int
    eta: int
    k: int = 31
    seed: int = 0


@dataclass
class Corpus:
    params: Params
    doc_ids: np.ndarray          # uint32, insertion order
    packed: np.ndarray           # uint8 packed stream
    offsets: np.ndarray          # uint64 (n_docs + 1)
    seeds_of_doc: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))

    @property
    def n_bases(self) -> int:
        return int(self.offsets[-1])

    def doc_bases(self, i: int) -> np.ndarray:
        return unpack_bases(self.packed, int(self.offsets[i]), int(self.offsets[i + 1] - self.offsets[i]))


@dataclass
class QueryBatch:
    packed: np.ndarray
    offsets: np.ndarray
    from_doc: np.ndarray          # source doc index per query, -1 for uniform random

    @property
    def n(self) -> int:
        return self.offsets.size - 1

    @property
    def n_bases(self) -> int:
        return int(self.offsets[-1])

    def n_kmers(self, k: int) -> int:
        L = np.diff(self.offsets.astype(np.int64))
        return int(np.maximum(L - k + 1, 0).sum())


def family_corpus(rng, params: Params, n_seeds: int, doc_len: int, sub_rate: float,
                  indel_rate: float = 0.0) -> Corpus:
    """K documents, each a mutated copy of one of n_seeds uniform seed genomes."""
    seeds = [uniform_genome(rng, doc_len) for _ in range(n_seeds)]
    pick = rng.integers(0, n_seeds, size=params.K)
    s = PackedStream()
    for d in range(params.K):
        doc = substitute(rng, seeds[pick[d]], sub_rate)
        if indel_rate > 0:
            doc = indels(rng, doc, indel_rate)
        s.append(doc)
    packed, offs = s.finish()
    return Corpus(params, np.arange(params.K, dtype=np.uint32), packed, offs, pick)


def uniform_corpus(rng, params: Params, doc_len: int) -> Corpus:
    s = PackedStream()
    for _ in range(params.K):
        s.append(uniform_genome(rng, doc_len))
    packed, offs = s.finish()
    return Corpus(params, np.arange(params.K, dtype=np.uint32), packed, offs)


def sample_queries(rng, corpus: Corpus, lengths: np.ndarray, frac_from_docs: float,
                   err_rate: float = 0.0, alternate: bool = False,
                   docs_pool: np.ndarray | None = None) -> QueryBatch:
    """Queries of the given lengths: a fraction are substrings of random documents
    (with i.i.d. read-error substitutions at err_rate), the rest uniform random.
    ``alternate`` makes even indices doc substrings and odd indices random."""
    n = lengths.size
    s = PackedStream()
    src = np.full(n, -1, dtype=np.int64)
    doc_len = np.diff(corpus.offsets.astype(np.int64))
    pool = np.arange(corpus.params.K) if docs_pool is None else np.asarray(docs_pool)
    for i in range(n):
        L = int(lengths[i])
        from_doc = (i % 2 == 0) if alternate else (rng.random() < frac_from_docs)
        if from_doc:
            d = int(pool[rng.integers(0, pool.size)])
            if doc_len[d] >= L:
                off = int(rng.integers(0, doc_len[d] - L + 1))
                q = unpack_bases(corpus.packed, int(corpus.offsets[d]) + off, L)
                if err_rate > 0:
                    q = substitute(rng, q, err_rate)
                s.append(q)
                src[i] = d
                continue
        s.append(uniform_genome(rng, L))
    packed, offs = s.finish()
    return QueryBatch(packed, offs, src)


def sample_kmers(rng, corpus: Corpus, n: int, k: int, frac_present: float) -> np.ndarray:
    """Single k-mer queries in the library's forward-code format."""
    present = rng.random(n) < frac_present
    windows = rng.integers(0, 4, size=(n, k), dtype=np.uint8)
    doc_len = np.diff(corpus.offsets.astype(np.int64))
    idx = np.nonzero(present)[0]
    if idx.size:
        d = rng.integers(0, corpus.params.K, size=idx.size)
        off = (rng.random(idx.size) * (doc_len[d] - k + 1)).astype(np.int64)
        starts = corpus.offsets[d].astype(np.int64) + off
        t = starts[:, None] + np.arange(k)[None, :]
        windows[idx] = (corpus.packed[t >> 2] >> (2 * (t & 3)).astype(np.uint8)) & 3
    return codes_from_windows(windows)


# --------------------------------------------------------------------------
# the five workloads (shapes of the paper's genomic experiments, Section 5.2)

TINY = "tiny"          # 100 docs x 20 kbp uniform, R=2 B=10 m=2^20
MEDIUM = "medium"      # 1,000 docs x 1 Mbp from 20 seeds, 1% subs, R=4 B=32 m=2^26
LARGE = "large"        # 10,000 docs x 500 kbp from 200 seeds, R=5 B=100 m=2^29
STREAM = "stream"      # 100,000 docs x 50 kbp from 2,000 seeds, R=6 B=316 m=2^28

WORKLOAD_PARAMS = {
    TINY: Params(K=100, B=10, R=2, m=1 << 20, eta=2),
    MEDIUM: Params(K=1000, B=32, R=4, m=1 << 26, eta=2),
    LARGE: Params(K=10000, B=100, R=5, m=1 << 29, eta=2),
    STREAM: Params(K=100000, B=316, R=6, m=1 << 28, eta=2),
}
WORKLOAD_INDEX = {TINY: 1, MEDIUM: 2, LARGE: 3, STREAM: 5}


def rng_for(name: str, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng([GEN_SEED_BASE + WORKLOAD_INDEX[name], salt])


def tiny_workload(scale_docs: int | None = None):
    """100 uniform 20 kbp documents; 1000 x 100 bp queries, even = substrings."""
    p = WORKLOAD_PARAMS[TINY]
    rng = rng_for(TINY)
    corpus = uniform_corpus(rng, p, 20_000)
    q = sample_queries(rng, corpus, np.full(1000, 100), 0.5, alternate=True)
    return corpus, q


def medium_workload(n_docs: int | None = None, doc_len: int = 1_000_000, n_kmers: int = 1_000_000,
                    n_seqs: int = 10_000, seq_len: int = 1000):
    """1,000 x 1 Mbp documents from 20 seeds at 1% substitutions; 10^6 single
    k-mers (50% present) and 10^4 x 1 kbp sequences (50% from documents)."""
    p = WORKLOAD_PARAMS[MEDIUM]
    if n_docs is not None:
        p = Params(K=n_docs, B=p.B, R=p.R, m=p.m, eta=p.eta)
    rng = rng_for(MEDIUM)
    corpus = family_corpus(rng, p, 20, doc_len, 0.01)
    kmers = sample_kmers(rng, corpus, n_kmers, p.k, 0.5)
    q = sample_queries(rng, corpus, np.full(n_seqs, seq_len), 0.5)
    return corpus, kmers, q


def large_workload(n_docs: int | None = None, doc_len: int = 500_000, n_queries: int = 100_000,
                   n_seeds: int = 200):
    """10,000 x 500 kbp documents from 200 seeds, 0.5% substitutions and 0.05%
    indels; 10^5 queries of length U[31, 5000], 70% from documents with 0.1%
    read errors.  A reduced copy that keeps the batch's repetition (k-mers
    shared across queries) scales documents, seeds and queries together."""
    p = WORKLOAD_PARAMS[LARGE]
    if n_docs is not None:
        p = Params(K=n_docs, B=p.B, R=p.R, m=p.m, eta=p.eta)
    rng = rng_for(LARGE)
    corpus = family_corpus(rng, p, n_seeds, doc_len, 0.005, 0.0005)
    lengths = rng.integers(31, 5001, size=n_queries)
    q = sample_queries(rng, corpus, lengths, 0.7, err_rate=0.001)
    return corpus, q


def large_shard_corpus(shard: int, n_docs: int | None = None, doc_len: int = 500_000) -> Corpus:
    """The documents of shard `shard` of a document-sharded large index
    (Section 5.3): shard 0 is the large workload's own corpus; shard s > 0
    draws another 10,000 documents from the same recipe with its own seed."""
    if shard == 0:
        return large_workload(n_docs=n_docs, doc_len=doc_len, n_queries=0)[0]
    p = WORKLOAD_PARAMS[LARGE]
    if n_docs is not None:
        p = Params(K=n_docs, B=p.B, R=p.R, m=p.m, eta=p.eta)
    return family_corpus(rng_for(LARGE, 1000 + shard), p, 200, doc_len, 0.005, 0.0005)


def serving_trace(rng, n: int, rate_per_s: float, median: float = 300.0, sigma: float = 1.0,
                  lo: int = 31, hi: int = 10_000):
    """Poisson arrivals (seconds) and log-normal query lengths clipped to [lo, hi]."""
    arrivals = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    lengths = np.clip(np.round(rng.lognormal(np.log(median), sigma, size=n)), lo, hi).astype(np.int64)
    return arrivals, lengths


class StreamWorkload:
    """Documents arriving in epochs, each followed by a query batch.

    n_seeds uniform seed genomes of doc_len bases; every document is a copy of
    a random seed with i.i.d. substitutions at `divergence`.  After epoch e the
    query batch draws 70% of its sequences from documents inserted so far
    (with 0.1% read errors) and 30% uniform, lengths U[qmin, qmax].
    """

    def __init__(self, params: Params, n_seeds: int, doc_len: int, divergence: float,
                 epoch_docs: int, queries_per_epoch: int, qmin: int = 31, qmax: int = 2000,
                 seed_salt: int = 0):
        self.params = params
        self.doc_len = doc_len
        self.divergence = divergence
        self.epoch_docs = epoch_docs
        self.queries_per_epoch = queries_per_epoch
        self.qmin, self.qmax = qmin, qmax
        self.rng = np.random.default_rng([GEN_SEED_BASE + WORKLOAD_INDEX[STREAM], seed_salt])
        self.seeds = [uniform_genome(self.rng, doc_len) for _ in range(n_seeds)]
        self.n_epochs = (params.K + epoch_docs - 1) // epoch_docs
        self.inserted = 0
        self._docs_so_far: list[np.ndarray] = []

    def epoch(self, e: int):
        """(doc_ids, packed, offsets) of epoch e, then its query batch."""
        lo = e * self.epoch_docs
        hi = min(self.params.K, lo + self.epoch_docs)
        s = PackedStream()
        docs = []
        for _ in range(lo, hi):
            d = substitute(self.rng, self.seeds[int(self.rng.integers(0, len(self.seeds)))],
                           self.divergence)
            s.append(d)
            docs.append(d)
        packed, offs = s.finish()
        self._docs_so_far.extend(docs)
        self.inserted = hi
        ids = np.arange(lo, hi, dtype=np.uint32)
        # queries over everything inserted so far
        n = self.queries_per_epoch
        lengths = self.rng.integers(self.qmin, self.qmax + 1, size=n)
        qs = PackedStream()
        src = np.full(n, -1, dtype=np.int64)
        for i in range(n):
            L = int(lengths[i])
            if self.rng.random() < 0.7:
                d = int(self.rng.integers(0, hi))
                doc = self._docs_so_far[d]
                off = int(self.rng.integers(0, doc.size - L + 1))
                qs.append(substitute(self.rng, doc[off:off + L], 0.001))
                src[i] = d
            else:
                qs.append(uniform_genome(self.rng, L))
        qp, qo = qs.finish()
        return (ids, packed, offs), QueryBatch(qp, qo, src)


def stream_workload(n_docs: int | None = None, doc_len: int = 50_000, n_seeds: int = 2000,
                    epoch_docs: int = 1000, queries_per_epoch: int = 10_000,
                    m: int | None = None) -> StreamWorkload:
    """100,000 x 50 kbp documents from 2,000 seeds at 1% divergence, inserted
    in epochs of 1,000; after each epoch 10^4 queries of 31..2,000 bp."""
    p = WORKLOAD_PARAMS[STREAM]
    p = Params(K=n_docs or p.K, B=p.B, R=p.R, m=m or p.m, eta=p.eta)
    return StreamWorkload(p, n_seeds, doc_len, 0.01, epoch_docs, queries_per_epoch)


# --------------------------------------------------------------------------
# documents of words (the paper's Section 5.4 document-indexing experiment;
# the Wiki-dump and ClueWeb09 samples are not available, so documents draw
# words from a synthetic vocabulary with Zipf-like frequencies)

WORDS = "words"
WORKLOAD_INDEX[WORDS] = 6


def word_vocabulary(rng, n_words: int, mean_len: float = 7.0) -> list[bytes]:
    """Distinct random lowercase words, lengths 1 + Poisson(mean_len - 1)."""
    seen, out = set(), []
    while len(out) < n_words:
        L = 1 + int(rng.poisson(mean_len - 1))
        w = bytes(rng.integers(97, 123, size=L).astype(np.uint8))
        if w not in seen:
            seen.add(w)
            out.append(w)
    return out


def word_corpus(rng, K: int, vocab: list[bytes], terms_per_doc: int, zipf_s: float = 1.07):
    """K documents, each terms_per_doc distinct words drawn with probability
    proportional to 1 / rank^zipf_s.  Returns a list of index arrays."""
    ranks = np.arange(1, len(vocab) + 1, dtype=np.float64)
    p = ranks ** -zipf_s
    p /= p.sum()
    return [np.sort(rng.choice(len(vocab), size=terms_per_doc, replace=False, p=p)) for _ in range(K)]
