"""CPU oracle for RAMBO -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The product path (the CUDA library in
``paper_1910_04358_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``rambo_oracle.c`` (plain C, single-threaded core,
written from the paper: Section 2.1 Bloom filters, Section 3.2 Algorithm 1
insertion, Section 3.3 Algorithm 2 query, Section 3.3.1 sequence queries).
This module only compiles it with gcc and marshals arguments through ctypes.

Parity status: every function is pinned by the ``-m "not gpu"`` tests
(MurmurHash3 verification code, string brute force for canonical k-mers,
brute-force exact k-mer sets, the Lemma 4.1 false-positive bound, the
bucket-space AND identity and the degenerate cases).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rambo_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "librambo_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_EINVAL = -1
ORC_ENOMEM = -2
ORC_ERANGE = -4
ORC_EUNTRACKED = -7


def build(force: bool = False) -> str:
    """Compiles the oracle into ``oracle/_build/librambo_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-Wall", "-Wno-unused-function", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        u32, u64, p = C.c_uint32, C.c_uint64, C.c_void_p
        sig = {
            "orc_mmh3_x64_128": (None, [p, u64, u32, p]),
            "orc_kmer_forward": (u64, [p, u64, u32]),
            "orc_kmer_canonical": (u64, [p, u64, u32]),
            "orc_canonical_of_code": (u64, [u64, u32]),
            "orc_unpack": (None, [p, u64, u64, p]),
            "orc_create": (p, [u32, u32, u32, u64, u32, u32, u64]),
            "orc_create_restricted": (p, [u32, u32, u32, u64, u32, u32, u64, p, u64]),
            "orc_destroy": (None, [p]),
            "orc_partition": (u32, [p, u32, u32]),
            "orc_probe_position": (u64, [p, u64, u32]),
            "orc_insert": (C.c_int, [p, u32, p, u64, u64]),
            "orc_insert_batch": (C.c_int, [p, u32, p, p, p, u32]),
            "orc_query_seq": (C.c_int, [p, p, u64, u64, p]),
            "orc_query_kmer": (C.c_int, [p, u64, p]),
            "orc_query_seqs": (C.c_int, [p, u64, p, p, p, u32]),
            "orc_query_kmers": (C.c_int, [p, u64, p, p, u32]),
            "orc_bucket_of": (u32, [p, u32, u32]),
            "orc_filter_bit": (C.c_int, [p, u32, u32, u64]),
            "orc_filter_words": (None, [p, u32, u32, p]),
            "orc_filter_popcount": (u64, [p, u32, u32]),
            "orc_is_inserted": (C.c_int, [p, u32]),
            "orc_num_filters_bits": (u64, [p]),
            "orc_fold": (C.c_int, [p]),
            "orc_set_partition": (C.c_int, [p, p]),
            "orc_word_position": (u64, [p, p, u64, u32]),
            "orc_insert_words": (C.c_int, [p, u32, p, p, u64]),
            "orc_query_words": (C.c_int, [p, p, p, u64, p]),
            "orc_seq_positions": (C.c_int, [p, u64, p, p, p]),
            "orc_position_bits": (C.c_int, [p, u64, p, p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _sorted_distinct(a) -> np.ndarray:
    """Sorted distinct uint64 values (a sort and a neighbour compare)."""
    a = np.sort(np.asarray(a, dtype=np.uint64).ravel())
    if a.size:
        a = a[np.concatenate(([True], a[1:] != a[:-1]))]
    return np.ascontiguousarray(a)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def mmh3_x64_128(data: bytes, seed: int) -> tuple[int, int]:
    """MurmurHash3_x64_128 of a byte string: (first word, second word)."""
    lib = _load()
    buf = np.frombuffer(bytes(data) + b"\0", dtype=np.uint8)  # non-empty buffer
    out = np.zeros(2, dtype=np.uint64)
    lib.orc_mmh3_x64_128(_ptr(buf), len(data), seed & 0xFFFFFFFF, _ptr(out))
    return int(out[0]), int(out[1])


def kmer_forward(packed: np.ndarray, begin: int, k: int) -> int:
    return int(_load().orc_kmer_forward(_ptr(packed), begin, k))


def kmer_canonical(packed: np.ndarray, begin: int, k: int) -> int:
    return int(_load().orc_kmer_canonical(_ptr(packed), begin, k))


def canonical_of_code(fwd: int, k: int) -> int:
    return int(_load().orc_canonical_of_code(fwd, k))


def unpack(packed: np.ndarray, begin: int, n: int) -> np.ndarray:
    out = np.zeros(max(n, 1), dtype=np.uint8)
    _load().orc_unpack(_ptr(packed), begin, n, _ptr(out))
    return out[:n]


def _pack_words(words):
    buf = np.frombuffer(b"".join(words) + b"\0", dtype=np.uint8)
    offs = np.zeros(len(words) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(w) for w in words]) if words else []
    return buf, offs


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != ORC_OK:
        raise OracleError(f"{what} failed with oracle code {rc}")


class Rambo:
    """Plain RAMBO: R x B separate m-bit Bloom filters plus DocIDs lists.

    ``tracked`` (sorted distinct positions) switches to restricted mode: only
    those positions are kept, which is exact for queries probing nowhere else.
    """

    def __init__(self, K, B, R, m, eta, k=31, seed=0, tracked=None):
        lib = _load()
        self.K, self.B, self.R, self.m, self.eta, self.k, self.seed = K, B, R, m, eta, k, seed
        self.W = (K + 31) // 32
        if tracked is None:
            h = lib.orc_create(K, B, R, m, eta, k, seed)
        else:
            t = _sorted_distinct(tracked)
            self._tracked = t
            h = lib.orc_create_restricted(K, B, R, m, eta, k, seed,
                                          _ptr(t) if t.size else None, t.size)
        if not h:
            raise OracleError("orc_create failed (bad parameters or out of memory)")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _load().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- construction (Algorithm 1) -------------------------------------
    def insert(self, doc_id: int, packed: np.ndarray, begin: int, n_bases: int):
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        _check(_load().orc_insert(self._h, doc_id, _ptr(packed), begin, n_bases), "insert")

    def insert_batch(self, doc_ids, packed, offsets, threads: int = 1):
        ids = np.ascontiguousarray(doc_ids, dtype=np.uint32)
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        offs = np.ascontiguousarray(offsets, dtype=np.uint64)
        assert offs.size == ids.size + 1
        _check(_load().orc_insert_batch(self._h, ids.size, _ptr(ids), _ptr(packed), _ptr(offs),
                                        threads), "insert_batch")

    # -- query (Algorithm 2, Section 3.3.1) ------------------------------
    def query_seq(self, packed, begin, n_bases) -> np.ndarray:
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        out = np.zeros(self.W, dtype=np.uint32)
        _check(_load().orc_query_seq(self._h, _ptr(packed), begin, n_bases, _ptr(out)), "query")
        return out

    def query_seqs(self, packed, offsets, threads: int = 1) -> np.ndarray:
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        offs = np.ascontiguousarray(offsets, dtype=np.uint64)
        n = offs.size - 1
        out = np.zeros((max(n, 0), self.W), dtype=np.uint32)
        if n > 0:
            _check(_load().orc_query_seqs(self._h, n, _ptr(packed), _ptr(offs), _ptr(out),
                                          threads), "query_seqs")
        return out

    def query_kmer(self, fwd: int) -> np.ndarray:
        out = np.zeros(self.W, dtype=np.uint32)
        _check(_load().orc_query_kmer(self._h, fwd, _ptr(out)), "query_kmer")
        return out

    def query_kmers(self, kmers, threads: int = 1) -> np.ndarray:
        km = np.ascontiguousarray(kmers, dtype=np.uint64)
        out = np.zeros((km.size, self.W), dtype=np.uint32)
        if km.size:
            _check(_load().orc_query_kmers(self._h, km.size, _ptr(km), _ptr(out), threads),
                   "query_kmers")
        return out

    # -- documents of words (Section 5.4) ------------------------------------
    def insert_words(self, doc_id: int, words: list[bytes]):
        buf, offs = _pack_words(words)
        _check(_load().orc_insert_words(self._h, doc_id, _ptr(buf), _ptr(offs), len(words)),
               "insert_words")

    def query_words(self, words: list[bytes]) -> np.ndarray:
        buf, offs = _pack_words(words)
        out = np.zeros(self.W, dtype=np.uint32)
        _check(_load().orc_query_words(self._h, _ptr(buf), _ptr(offs), len(words), _ptr(out)),
               "query_words")
        return out

    def word_position(self, word: bytes, j: int) -> int:
        buf, _ = _pack_words([word])
        return int(_load().orc_word_position(self._h, _ptr(buf), len(word), j))

    # -- explicit partition (Section 5.3 routing) ------------------------------
    def set_partition(self, phi):
        """phi[d, r] = bucket of document d in repetition r; before any insert."""
        a = np.ascontiguousarray(phi, dtype=np.uint32)
        assert a.shape == (self.K, self.R)
        _check(_load().orc_set_partition(self._h, _ptr(a)), "set_partition")

    # -- folding over (Section 5.3) -------------------------------------------
    def fold(self):
        """B -> B/2 by ORing bucket b + B/2 onto bucket b in every repetition."""
        _check(_load().orc_fold(self._h), "fold")
        self.B //= 2

    # -- introspection -----------------------------------------------------
    def bucket(self, d: int, r: int) -> int:
        return int(_load().orc_bucket_of(self._h, d, r))

    def partition(self, d: int, r: int) -> int:
        return int(_load().orc_partition(self._h, d, r))

    def probe_position(self, term: int, j: int) -> int:
        return int(_load().orc_probe_position(self._h, term, j))

    def seq_positions(self, packed, offsets) -> np.ndarray:
        """The eta probe positions of every k-mer of every sequence
        [offsets[i], offsets[i+1]), in window order: shape (terms, eta)."""
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        offs = np.ascontiguousarray(offsets, dtype=np.uint64)
        L = np.diff(offs.astype(np.int64))
        terms = int(np.maximum(L - self.k + 1, 0).sum())
        out = np.zeros((max(terms, 1), self.eta), dtype=np.uint64)
        if offs.size > 1:
            _check(_load().orc_seq_positions(self._h, offs.size - 1, _ptr(packed), _ptr(offs),
                                             _ptr(out)), "seq_positions")
        return out[:terms]

    def kmer_positions(self, kmers) -> np.ndarray:
        """The eta probe positions of single k-mers given as forward codes."""
        return np.array([[self.probe_position(canonical_of_code(int(x), self.k), j)
                          for j in range(self.eta)] for x in np.asarray(kmers).tolist()],
                        dtype=np.uint64).reshape(-1, self.eta)

    def filter_bit(self, r: int, b: int, pos: int) -> int:
        return int(_load().orc_filter_bit(self._h, r, b, pos))

    def filter_words(self, r: int, b: int) -> np.ndarray:
        nbits = int(_load().orc_num_filters_bits(self._h))
        out = np.zeros((nbits + 63) // 64, dtype=np.uint64)
        _load().orc_filter_words(self._h, r, b, _ptr(out))
        return out

    def position_bits(self, positions) -> np.ndarray:
        """Bits of all R*B BFUs at each position: row i holds bit r*B + b
        (LSB-first bytes, ceil(R*B/8) of them) = filter (r,b) at positions[i]."""
        pos = np.ascontiguousarray(positions, dtype=np.uint64)
        row = (self.R * self.B + 7) // 8
        out = np.zeros((max(pos.size, 1), row), dtype=np.uint8)
        if pos.size:
            _check(_load().orc_position_bits(self._h, pos.size, _ptr(pos), _ptr(out)), "position_bits")
        return out[:pos.size]

    def fill_fraction(self, r: int, b: int) -> float:
        nbits = int(_load().orc_num_filters_bits(self._h))
        return int(_load().orc_filter_popcount(self._h, r, b)) / nbits

    def is_inserted(self, d: int) -> bool:
        return bool(_load().orc_is_inserted(self._h, d))


def tracking_oracle(K, B, R, m, eta, k, seed, seqs=(), kmers=()) -> "Rambo":
    """An empty restricted-mode oracle that tracks exactly the probe
    positions of the given sequence batches ((packed, offsets) pairs) and
    single k-mers (forward codes): exact for those queries."""
    probe = Rambo(K, B, R, m, eta, k, seed, tracked=[0])
    parts = [probe.seq_positions(pk, of).ravel() for pk, of in seqs]
    km = np.asarray(kmers, dtype=np.uint64)
    if km.size:
        parts.append(probe.kmer_positions(km).ravel())
    probe.close()
    pos = _sorted_distinct(np.concatenate(parts)) if parts else np.zeros(0, np.uint64)
    return Rambo(K, B, R, m, eta, k, seed, tracked=pos)


def mask_to_docs(mask_words: np.ndarray) -> set[int]:
    """Document ids whose bit is set in a K-bit mask (word d>>5, bit d&31)."""
    bits = np.unpackbits(np.ascontiguousarray(mask_words, dtype="<u4").view(np.uint8),
                         bitorder="little")
    return set(np.nonzero(bits)[0].tolist())
