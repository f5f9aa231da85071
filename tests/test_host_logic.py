"""Host-side helpers (no GPU): answer-mask decoding and the bench's choice of
the query path the library takes."""
import numpy as np

import oracle
from paper_1910_04358_gb300 import rambo


def test_answer_docs_matches_oracle_mask_decoding():
    rng = np.random.default_rng(3)
    for W in (1, 2, 7, 32):
        for _ in range(20):
            m = rng.integers(0, 1 << 32, size=W, dtype=np.uint64).astype(np.uint32)
            m &= rng.integers(0, 1 << 32, size=W, dtype=np.uint64).astype(np.uint32)
            assert set(rambo.answer_docs(m).tolist()) == oracle.mask_to_docs(m)
    assert rambo.answer_docs(np.zeros(4, np.uint32)).size == 0


def test_bench_effective_path():
    import bench
    t = lambda qp: {"query_path": qp}
    assert bench.effective_path(t(2), {"group_bytes": 16}) == 2
    assert bench.effective_path(t(2), {"group_bytes": 64}) == 1
    assert bench.effective_path(t(1), {"group_bytes": 512}) == 1
    assert bench.effective_path(t(1), {"group_bytes": 1024}) == 0
    assert bench.effective_path(t(0), {"group_bytes": 16}) == 0
