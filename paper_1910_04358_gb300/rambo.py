"""Python binding of librambo_gpu.so (the C ABI in include/rambo.h).

Argument marshalling only: every step of insertion and query runs in the
library's CUDA kernels.  Host-buffer calls take numpy arrays; device calls
take torch CUDA tensors (PyTorch supplies device memory and streams).  There
is no CPU fallback: if the library cannot be built or loaded, importing this
module raises.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import build as _build

RAMBO_OK = 0
RAMBO_EINVAL = -1
RAMBO_ENOMEM = -2
RAMBO_ECUDA = -3
RAMBO_ERANGE = -4
RAMBO_ETIMEOUT = -5
RAMBO_ESTATE = -6

_lock = threading.Lock()
_lib = None


class RamboError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {code} ({_strerror(code)})")


class _Info(C.Structure):
    _fields_ = [("K", C.c_uint32), ("B", C.c_uint32), ("R", C.c_uint32), ("eta", C.c_uint32),
                ("k", C.c_uint32), ("m", C.c_uint64), ("seed", C.c_uint64),
                ("mask_words", C.c_uint32), ("group_bytes", C.c_uint32),
                ("index_bytes", C.c_uint64), ("docbits_bytes", C.c_uint64), ("device", C.c_int)]


def load():
    """Builds (if stale) and loads the CUDA library; raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = C.CDLL(path)
        u32, u64, p, i = C.c_uint32, C.c_uint64, C.c_void_p, C.c_int
        sz = C.c_size_t
        sig = {
            "rambo_create": (i, [u32, u32, u32, u64, u32, u32, u64, i, C.POINTER(p)]),
            "rambo_destroy": (i, [p]),
            "rambo_mask_words": (u32, [p]),
            "rambo_get_info": (i, [p, C.POINTER(_Info)]),
            "rambo_strerror": (C.c_char_p, [i]),
            "rambo_insert": (i, [p, u32, p, u64]),
            "rambo_insert_batch": (i, [p, u32, p, p, p]),
            "rambo_query_kmers": (i, [p, u64, p, p]),
            "rambo_query_seqs": (i, [p, u64, p, p, p]),
            "rambo_insert_workspace": (sz, [p, u64]),
            "rambo_query_kmers_workspace": (sz, [p, u64]),
            "rambo_query_seqs_workspace": (sz, [p, u64]),
            "rambo_insert_batch_dev": (i, [p, u32, p, p, u64, p, p, sz, p]),
            "rambo_query_kmers_dev": (i, [p, u64, p, p, p, sz, p]),
            "rambo_insert_ranges_dev": (i, [p, u32, p, p, u64, p, p, p, sz, p]),
            "rambo_merge_shard_answers": (i, [u64, p, u32, u32, p, p, u32, p]),
            "rambo_query_seqs_dev": (i, [p, u64, p, u64, p, p, p, sz, p]),
            "rambo_sync": (i, [p, p]),
            "rambo_copy_index": (i, [p, u64, u64, p]),
            "rambo_copy_docbits": (i, [p, p]),
            "rambo_copy_partition": (i, [p, p]),
            "rambo_profile_reset": (i, [p, u32]),
            "rambo_profile_read": (i, [p, C.c_void_p]),
            "rambo_get_tuning": (i, [p, C.c_void_p]),
            "rambo_set_tuning": (i, [p, C.c_void_p]),
            "rambo_probe_gather": (i, [p, u64, u32, u64, u32, u32, u64, p, p]),
            "rambo_query_seqs_noalloc": (i, [p, u64, p, u64, p, p, p]),
            "rambo_query_ranges_dev": (i, [p, u64, p, u64, p, p, p, p, sz, p]),
            "rambo_fold": (i, [p]),
            "rambo_set_partition": (i, [p, p]),
            "rambo_probed_kmers": (i, [p, C.POINTER(u64), i]),
            "rambo_insert_words_dev": (i, [p, u32, p, p, u64, p, p, p]),
            "rambo_query_words_workspace": (sz, [p, u64]),
            "rambo_query_words_dev": (i, [p, u64, p, u64, p, p, p, p, sz, p]),
            "rambo_query_batch": (i, [p, u64, p, p, u64, p, p, p]),
            "rambo_probe_wait_expiry": (i, [p, u64, p]),
            "rambo_query_batch_workspace": (sz, [p, u64, u64, u64]),
            "rambo_query_seqs_workspace_for": (sz, [p, u64, u64]),
            "rambo_query_batch_dev": (i, [p, u64, p, p, u64, p, u64, p, p, p, sz, p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def library_path() -> str:
    return _build.LIB


def _strerror(code: int) -> str:
    try:
        return load().rambo_strerror(code).decode()
    except Exception:
        return "?"


def _check(rc: int, what: str):
    if rc != RAMBO_OK:
        raise RamboError(rc, what)


def _check_span(packed: np.ndarray, offs: np.ndarray):
    """The host calls read the bytes holding bases [offs[0], offs[-1])."""
    if offs.size and offs[-1] >= offs[0] and packed.size * 4 < int(offs[-1]):
        raise ValueError("packed buffer is shorter than the bases the offsets address")


def _out_array(out, n: int, W: int) -> np.ndarray:
    if out is None:
        return np.zeros((n, W), dtype=np.uint32)
    if out.dtype not in (np.uint32, np.int32) or out.shape != (n, W) or not out.flags.c_contiguous:
        raise ValueError(f"out must be a C-contiguous ({n}, {W}) 32-bit array")
    return out.view(np.uint32)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data if a.size else None


def _t_ptr(t):
    return t.data_ptr() if t.numel() else None


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Workspace:
    """A 256-byte aligned device buffer owned by torch, grown on demand."""

    def __init__(self, device):
        self.device = device
        self._buf = None
        self.ptr = 0
        self.nbytes = 0

    def get(self, nbytes: int) -> tuple[int, int]:
        import torch
        if nbytes > self.nbytes:
            want = max(nbytes, 256) + nbytes // 4
            self._buf = torch.empty(want + 256, dtype=torch.uint8, device=self.device)
            base = self._buf.data_ptr()
            self.ptr = (base + 255) // 256 * 256
            self.nbytes = want
        return self.ptr, self.nbytes


STAGES = ("prefix", "register", "insert", "probe_seqs", "probe_kmers", "expand")
TUNING_FIELDS = ("probe_ctas_per_sm", "probe_min_kmers_per_warp", "expand_ctas_per_sm",
                 "use_byte_table", "byte_table_max_mb", "query_path", "fused_tile_kmers",
                 "fused_short_max", "smem_docbits", "use_nibble_table",
                 "expand_filter", "early_exit", "early_exit_segment",
                 "kmer_probe_ctas_per_sm", "host_chunk_kmers", "branch_priority",
                 "host_slots", "bin_region_kib", "bin_rows", "host_direct",
                 "host_fused_ctas_per_sm",
                 "insert_mode", "insert_bin_records", "fused_async",
                 "kmer_async", "seg_cut_bits")


class _Tuning(C.Structure):
    _fields_ = [(f, C.c_uint32) for f in TUNING_FIELDS]


def probe_gather(buf, record_bytes: int, n_probes: int, variant: int = 0, seed: int = 1,
                 sink=None, stream=None, unroll: int = 8):
    """Random-record gather over a torch uint8 CUDA tensor (measurement support)."""
    import torch
    if sink is None:
        sink = torch.zeros(1, dtype=torch.int64, device=buf.device)
    _check(load().rambo_probe_gather(buf.data_ptr(), buf.numel(), record_bytes, n_probes, variant,
                                     unroll, seed, sink.data_ptr(), _stream_handle(stream)),
           "rambo_probe_gather")
    return sink


class _Profile(C.Structure):
    _fields_ = [("launches", C.c_uint64 * 6), ("timed", C.c_uint64 * 6), ("ms", C.c_double * 6)]


class Index:
    """One RAMBO index resident on a GPU (Section 3: R x B merged BFUs)."""

    def __init__(self, K: int, B: int, R: int, m: int, eta: int, k: int = 31, seed: int = 0,
                 device: int | None = None):
        lib = load()
        h = C.c_void_p()
        _check(lib.rambo_create(K, B, R, m, eta, k, seed, -1 if device is None else device,
                                C.byref(h)), "rambo_create")
        self._h = h
        info = _Info()
        _check(lib.rambo_get_info(h, C.byref(info)), "rambo_get_info")
        self.info = {f: getattr(info, f) for f, _ in _Info._fields_}
        self.K, self.B, self.R, self.m, self.eta, self.k, self.seed = K, B, R, m, eta, k, seed
        self.W = info.mask_words
        self.device = info.device
        self._ws = {}

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            load().rambo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------- host buffers
    def insert(self, doc_id: int, packed: np.ndarray, n_bases: int):
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        _check_span(packed, np.array([0, n_bases], dtype=np.uint64))
        _check(load().rambo_insert(self._h, doc_id, _np_ptr(packed), n_bases), "rambo_insert")

    def insert_batch(self, doc_ids, packed, offsets):
        ids = np.ascontiguousarray(doc_ids, dtype=np.uint32)
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        offs = np.ascontiguousarray(offsets, dtype=np.uint64)
        if offs.size != ids.size + 1:
            raise ValueError("offsets must have n_docs + 1 entries")
        _check_span(packed, offs)
        _check(load().rambo_insert_batch(self._h, ids.size, _np_ptr(ids), _np_ptr(packed),
                                         _np_ptr(offs)), "rambo_insert_batch")

    def query_kmers(self, kmers, out: np.ndarray | None = None) -> np.ndarray:
        """`out` (optional, e.g. pinned): (n, W) uint32 C-contiguous array."""
        km = np.ascontiguousarray(kmers, dtype=np.uint64)
        out = _out_array(out, km.size, self.W)
        _check(load().rambo_query_kmers(self._h, km.size, _np_ptr(km), _np_ptr(out)),
               "rambo_query_kmers")
        return out

    def query_seqs(self, packed, offsets, out: np.ndarray | None = None) -> np.ndarray:
        """`out` (optional, e.g. pinned): (n, W) uint32 C-contiguous array."""
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        offs = np.ascontiguousarray(offsets, dtype=np.uint64)
        _check_span(packed, offs)
        n = max(offs.size - 1, 0)
        out = _out_array(out, n, self.W)
        _check(load().rambo_query_seqs(self._h, n, _np_ptr(packed), _np_ptr(offs), _np_ptr(out)),
               "rambo_query_seqs")
        return out

    def query_batch(self, kmers, packed, offsets, out_kmers: np.ndarray | None = None,
                    out_seqs: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
        """Single k-mers and sequences in one call (both kinds run concurrently,
        copies pipelined); returns (k-mer answers, sequence answers)."""
        km = np.ascontiguousarray(kmers, dtype=np.uint64)
        packed = np.ascontiguousarray(packed, dtype=np.uint8)
        offs = np.ascontiguousarray(offsets, dtype=np.uint64)
        _check_span(packed, offs)
        ns = max(offs.size - 1, 0)
        out_kmers = _out_array(out_kmers, km.size, self.W)
        out_seqs = _out_array(out_seqs, ns, self.W)
        _check(load().rambo_query_batch(self._h, km.size, _np_ptr(km), _np_ptr(out_kmers), ns,
                                        _np_ptr(packed), _np_ptr(offs) if ns else None,
                                        _np_ptr(out_seqs)), "rambo_query_batch")
        return out_kmers, out_seqs

    # ----------------------------------------------------- device buffers
    def _workspace(self, stream_key, nbytes):
        ws = self._ws.get(stream_key)
        if ws is None:
            ws = self._ws[stream_key] = Workspace(f"cuda:{self.device}")
        return ws.get(nbytes)

    def workspace_bytes(self, kind: str, n: int, packed_bytes: int | None = None) -> int:
        """Device workspace of a call; for "seqs" with packed_bytes, the size
        that lets the tuned query path run (region-binned records included)."""
        if kind == "seqs" and packed_bytes is not None:
            return int(load().rambo_query_seqs_workspace_for(self._h, n, packed_bytes))
        f = {"insert": "rambo_insert_workspace", "kmers": "rambo_query_kmers_workspace",
             "seqs": "rambo_query_seqs_workspace"}[kind]
        return int(getattr(load(), f)(self._h, n))

    def insert_batch_dev(self, doc_ids, packed, offsets, stream=None, workspace=None):
        """doc_ids int32/uint32, packed uint8, offsets int64 (n+1) CUDA tensors."""
        n = doc_ids.numel()
        need = self.workspace_bytes("insert", n)
        s = _stream_handle(stream)
        wp, wn = workspace if workspace is not None else self._workspace(s, need)
        _check(load().rambo_insert_batch_dev(self._h, n, _t_ptr(doc_ids), _t_ptr(packed),
                                             packed.numel(), _t_ptr(offsets), wp, wn, s),
               "rambo_insert_batch_dev")

    def insert_ranges_dev(self, doc_ids, packed, begins, ends, stream=None, workspace=None):
        """Documents doc_ids[i] = bases [begins[i], ends[i]) of `packed` (int32/
        uint32, uint8, int64, int64 CUDA tensors)."""
        n = doc_ids.numel()
        need = self.workspace_bytes("insert", n)
        s = _stream_handle(stream)
        wp, wn = workspace if workspace is not None else self._workspace(s, need)
        _check(load().rambo_insert_ranges_dev(self._h, n, _t_ptr(doc_ids), _t_ptr(packed),
                                              packed.numel(), _t_ptr(begins), _t_ptr(ends), wp, wn, s),
               "rambo_insert_ranges_dev")

    def query_kmers_dev(self, kmers, out=None, stream=None, workspace=None):
        """kmers int64 CUDA tensor of forward codes; returns (n, W) int32 masks."""
        import torch
        n = kmers.numel()
        if out is None:
            out = torch.empty((n, self.W), dtype=torch.int32, device=kmers.device)
        need = self.workspace_bytes("kmers", n)
        s = _stream_handle(stream)
        wp, wn = workspace if workspace is not None else self._workspace(s, need)
        _check(load().rambo_query_kmers_dev(self._h, n, _t_ptr(kmers), _t_ptr(out), wp, wn, s),
               "rambo_query_kmers_dev")
        return out

    def query_seqs_dev(self, packed, offsets, out=None, stream=None, workspace=None):
        """packed uint8 and offsets int64 (n+1) CUDA tensors; returns (n, W) int32."""
        import torch
        n = offsets.numel() - 1
        if out is None:
            out = torch.empty((max(n, 0), self.W), dtype=torch.int32, device=offsets.device)
        need = self.workspace_bytes("seqs", max(n, 0), packed.numel())
        s = _stream_handle(stream)
        wp, wn = workspace if workspace is not None else self._workspace(s, need)
        _check(load().rambo_query_seqs_dev(self._h, max(n, 0), _t_ptr(packed), packed.numel(),
                                           _t_ptr(offsets), _t_ptr(out), wp, wn, s),
               "rambo_query_seqs_dev")
        return out

    def query_batch_dev(self, kmers, packed, offsets, out_kmers=None, out_seqs=None, stream=None,
                        workspace=None):
        """Device form of query_batch: kmers int64, packed uint8, offsets int64
        (n+1) CUDA tensors; the k-mer part runs on a side stream joined back
        to `stream`.  Returns (k-mer answers, sequence answers) (n, W) int32."""
        import torch
        nk = kmers.numel() if kmers is not None else 0
        ns = max(offsets.numel() - 1, 0) if offsets is not None else 0
        dev = (kmers if kmers is not None else offsets).device
        if out_kmers is None:
            out_kmers = torch.empty((nk, self.W), dtype=torch.int32, device=dev)
        if out_seqs is None:
            out_seqs = torch.empty((ns, self.W), dtype=torch.int32, device=dev)
        pb = packed.numel() if ns and packed is not None else 0
        need = int(load().rambo_query_batch_workspace(self._h, nk, ns, pb))
        s = _stream_handle(stream)
        wp, wn = workspace if workspace is not None else self._workspace(s, need)
        _check(load().rambo_query_batch_dev(
            self._h, nk, _t_ptr(kmers) if nk else None, _t_ptr(out_kmers) if nk else None, ns,
            _t_ptr(packed) if ns and packed is not None else None,
            packed.numel() if ns and packed is not None else 0,
            _t_ptr(offsets) if ns else None, _t_ptr(out_seqs) if ns else None, wp, wn, s),
            "rambo_query_batch_dev")
        return out_kmers, out_seqs

    def query_ranges_dev(self, packed, begins, ends, out=None, stream=None, workspace=None):
        """Items [begins[i], ends[i]) of a packed uint8 CUDA tensor (int64 tensors)."""
        import torch
        n = begins.numel()
        if out is None:
            out = torch.empty((n, self.W), dtype=torch.int32, device=begins.device)
        need = self.workspace_bytes("seqs", n, packed.numel())
        s = _stream_handle(stream)
        wp, wn = workspace if workspace is not None else self._workspace(s, need)
        _check(load().rambo_query_ranges_dev(self._h, n, _t_ptr(packed), packed.numel(),
                                             _t_ptr(begins), _t_ptr(ends), _t_ptr(out), wp, wn, s),
               "rambo_query_ranges_dev")
        return out

    def probe_wait_expiry(self, spins: int = 1000, stream=None):
        """Enqueues a bounded wait that runs out (failure-detection check);
        the next sync() raises RamboError with RAMBO_ETIMEOUT."""
        _check(load().rambo_probe_wait_expiry(self._h, spins, _stream_handle(stream)),
               "rambo_probe_wait_expiry")

    def sync(self, stream=None):
        _check(load().rambo_sync(self._h, _stream_handle(stream)), "rambo_sync")

    # -------------------------------------------------- explicit partition
    def set_partition(self, phi):
        """phi[d, r] = bucket of document d in repetition r; before any insert."""
        a = np.ascontiguousarray(phi, dtype=np.uint32)
        if a.shape != (self.K, self.R):
            raise ValueError("phi must be (K, R)")
        _check(load().rambo_set_partition(self._h, _np_ptr(a)), "rambo_set_partition")

    # ------------------------------------------------ documents of words
    @staticmethod
    def _word_batch(items):
        """CSR buffers for a list of items, each a list of byte strings."""
        import torch
        words = [w for it in items for w in it]
        buf = np.frombuffer(b"".join(words) + b"\0" * 8, dtype=np.uint8).copy()
        term_offs = np.zeros(len(words) + 1, dtype=np.int64)
        if words:
            term_offs[1:] = np.cumsum([len(w) for w in words])
        item_terms = np.zeros(len(items) + 1, dtype=np.int64)
        item_terms[1:] = np.cumsum([len(it) for it in items])
        dev = lambda a: torch.from_numpy(a).cuda()
        return dev(buf), int(term_offs[-1]), dev(term_offs), dev(item_terms)

    def insert_words(self, doc_ids, docs, stream=None):
        """docs[i]: list of byte strings (the words of document doc_ids[i])."""
        import torch
        buf, nbytes, toffs, iterms = self._word_batch(docs)
        ids = torch.from_numpy(np.ascontiguousarray(doc_ids, dtype=np.uint32).view(np.int32)).cuda()
        _check(load().rambo_insert_words_dev(self._h, len(docs), _t_ptr(ids), _t_ptr(buf), nbytes,
                                             _t_ptr(toffs), _t_ptr(iterms), _stream_handle(stream)),
               "rambo_insert_words_dev")
        self.sync(stream)

    def query_words(self, queries, stream=None) -> np.ndarray:
        """queries[i]: list of byte strings; returns (n, W) uint32 masks."""
        import torch
        buf, nbytes, toffs, iterms = self._word_batch(queries)
        n = len(queries)
        out = torch.empty((n, self.W), dtype=torch.int32, device="cuda")
        s = _stream_handle(stream)
        need = int(load().rambo_query_words_workspace(self._h, n))
        wp, wn = self._workspace(("words", s), need)
        _check(load().rambo_query_words_dev(self._h, n, _t_ptr(buf), nbytes, _t_ptr(toffs),
                                            _t_ptr(iterms), _t_ptr(out), wp, wn, s),
               "rambo_query_words_dev")
        self.sync(stream)
        return as_u32(out)

    # ------------------------------------------------------------ folding
    def fold(self):
        """Folding over (Section 5.3): B -> B/2, OR of bucket b+B/2 onto b."""
        _check(load().rambo_fold(self._h), "rambo_fold")
        info = _Info()
        _check(load().rambo_get_info(self._h, C.byref(info)), "rambo_get_info")
        self.info = {f: getattr(info, f) for f, _ in _Info._fields_}
        self.B = info.B

    # ------------------------------------------------------------- tuning
    def get_tuning(self) -> dict:
        t = _Tuning()
        _check(load().rambo_get_tuning(self._h, C.addressof(t)), "rambo_get_tuning")
        return {f: getattr(t, f) for f in TUNING_FIELDS}

    def set_tuning(self, **kw):
        cur = self.get_tuning()
        cur.update(kw)
        t = _Tuning(**{f: int(cur[f]) for f in TUNING_FIELDS})
        _check(load().rambo_set_tuning(self._h, C.addressof(t)), "rambo_set_tuning")

    def probed_kmers(self, reset: bool = False) -> int:
        v = C.c_uint64(0)
        _check(load().rambo_probed_kmers(self._h, C.byref(v), 1 if reset else 0),
               "rambo_probed_kmers")
        return v.value

    # ---------------------------------------------------------- profiling
    def profile_reset(self, timed_stages=()):
        mask = 0
        for st in timed_stages:
            mask |= 1 << STAGES.index(st)
        _check(load().rambo_profile_reset(self._h, mask), "rambo_profile_reset")

    def profile_read(self) -> dict:
        pr = _Profile()
        _check(load().rambo_profile_read(self._h, C.addressof(pr)), "rambo_profile_read")
        return {st: {"launches": pr.launches[i], "timed": pr.timed[i], "ms": pr.ms[i]}
                for i, st in enumerate(STAGES)}

    # ------------------------------------------------------ introspection
    def copy_index(self, offset: int = 0, nbytes: int | None = None) -> np.ndarray:
        total = self.info["index_bytes"]
        if nbytes is None:
            nbytes = total - offset
        out = np.zeros(nbytes, dtype=np.uint8)
        _check(load().rambo_copy_index(self._h, offset, nbytes, _np_ptr(out)), "rambo_copy_index")
        return out

    def docbits(self) -> np.ndarray:
        out = np.zeros((self.R, self.B, self.W), dtype=np.uint32)
        _check(load().rambo_copy_docbits(self._h, _np_ptr(out)), "rambo_copy_docbits")
        return out

    def partition(self) -> np.ndarray:
        out = np.zeros((self.K, self.R), dtype=np.uint32)
        _check(load().rambo_copy_partition(self._h, _np_ptr(out)), "rambo_copy_partition")
        return out


def merge_shard_answers(shard_masks, global_ids, out, stream=None):
    """ORs one document shard's answers (n x Ws int32 CUDA tensor, bit j =
    local document j) into the global answers `out` (n x W int32 CUDA
    tensor) at bits global_ids[j] (int32 CUDA tensor of the shard's
    documents' global ids)."""
    n, ws = shard_masks.shape
    _check(load().rambo_merge_shard_answers(n, _t_ptr(shard_masks), ws, global_ids.numel(),
                                            _t_ptr(global_ids), _t_ptr(out), out.shape[1],
                                            _stream_handle(stream)), "rambo_merge_shard_answers")
    return out


def answer_docs(mask_row) -> np.ndarray:
    """Document ids set in one answer mask (W uint32 words; document d is bit
    d & 31 of word d >> 5)."""
    words = np.ascontiguousarray(mask_row).view(np.uint32)
    return np.nonzero(np.unpackbits(words.view(np.uint8), bitorder="little"))[0]


def as_u32(t) -> np.ndarray:
    """A (n, W) int32 torch mask tensor as a host uint32 array."""
    return t.cpu().numpy().view(np.uint32)
