"""The allocation-free sequence query gives the same bits as the workspace one.

rambo_query_seqs_noalloc serves callers that cannot allocate device memory
(hosts that forbid library allocations, threads that must never reach
cudaMalloc): its scratch is a static device array inside the library.  This
file is collected last so a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1910_04358_gb300 import synth

pytestmark = pytest.mark.gpu

STATIC_SCRATCH_BYTES = 8 << 20  # RAMBO_STATIC_SCRATCH_BYTES in include/rambo.h


def _dev(torch, a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()


@pytest.mark.parametrize("tuning", [dict(query_path=0), dict(query_path=1),
                                    dict(query_path=2, bin_region_kib=256), dict(query_path=3)])
def test_noalloc_query_matches_workspace_query_and_oracle_twice(rambo_lib, tuning):
    # each query path the tuning can pick (path 2 with regions large enough
    # that its record bins fit the static scratch), two different batches in
    # a row: the second call must not see what the first left in the array
    import torch
    import oracle
    p = synth.Params(K=150, B=24, R=3, m=1 << 16, eta=2, k=31, seed=3)
    rng = np.random.default_rng(41)
    corpus = synth.family_corpus(rng, p, n_seeds=10, doc_len=2000, sub_rate=0.01)
    idx = rambo_lib.Index(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    idx.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    idx.set_tuning(**tuning)
    o = oracle.Rambo(p.K, p.B, p.R, p.m, p.eta, p.k, p.seed)
    o.insert_batch(corpus.doc_ids, corpus.packed, corpus.offsets)
    lib = rambo_lib.load()
    stream = torch.cuda.current_stream()
    for call, n in enumerate((300, 211)):
        q = synth.sample_queries(rng, corpus, rng.integers(20, 600, size=n), 0.6)
        packed, offs = _dev(torch, q.packed, np.uint8), _dev(torch, q.offsets, np.int64)
        if tuning["query_path"] >= 2:  # the binned / segment layout fits the scratch for this batch
            assert idx.workspace_bytes("seqs", n, packed.numel()) <= STATIC_SCRATCH_BYTES
        want = idx.query_seqs_dev(packed, offs)
        idx.sync()
        got = torch.full((n, idx.W), -1, dtype=torch.int32, device="cuda")
        rc = lib.rambo_query_seqs_noalloc(idx._h, n, packed.data_ptr(), packed.numel(),
                                          offs.data_ptr(), got.data_ptr(), stream.cuda_stream)
        assert rc == rambo_lib.RAMBO_OK, f"call {call}: {rc}"
        idx.sync()
        assert torch.equal(got, want), f"call {call} differs from rambo_query_seqs_dev"
        assert np.array_equal(rambo_lib.as_u32(got), o.query_seqs(q.packed, q.offsets)), \
            f"call {call} differs from the oracle"


def test_noalloc_rejects_batches_beyond_the_scratch(rambo_lib):
    import torch
    idx = rambo_lib.Index(64, 8, 2, 1 << 12, 2, k=31)
    n = 1
    while idx.workspace_bytes("seqs", n) <= STATIC_SCRATCH_BYTES:
        n *= 2
    offs = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    packed = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros((n, idx.W), dtype=torch.int32, device="cuda")
    lib = rambo_lib.load()
    rc = lib.rambo_query_seqs_noalloc(idx._h, n, packed.data_ptr(), packed.numel(), offs.data_ptr(),
                                      out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == rambo_lib.RAMBO_EINVAL
