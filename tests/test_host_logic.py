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
    assert bench.effective_path(t(2), {"group_bytes": 64}) == 2
    assert bench.effective_path(t(2), {"group_bytes": 128}) == 1
    assert bench.effective_path(t(2), {"group_bytes": 512}) == 1
    assert bench.effective_path(t(1), {"group_bytes": 512}) == 1
    assert bench.effective_path(t(1), {"group_bytes": 1024}) == 0
    assert bench.effective_path(t(0), {"group_bytes": 16}) == 0
    assert bench.effective_path(t(3), {"group_bytes": 64, "eta": 2}) == 3
    assert bench.effective_path(t(3), {"group_bytes": 64, "eta": 5}) == 1
    assert bench.effective_path(t(3), {"group_bytes": 128, "eta": 2}) == 1


class _FakeIndex:
    """Tuning state and geometry of an index, without a device."""

    def __init__(self, group_bytes):
        from paper_1910_04358_gb300 import autotune
        self.info = {"group_bytes": group_bytes}
        self.t = {k: vals[0] for k, vals in autotune.KNOBS}
        self.t.update(query_path=0, fused_tile_kmers=1024, fused_short_max=1024)

    def get_tuning(self):
        return dict(self.t)

    def set_tuning(self, **kw):
        self.t.update(kw)

    def sync(self):
        pass


def _fused_cost(t, info):
    # separate launches beat the fused path at its default tile and threshold,
    # but the fused path with small tiles and a low threshold beats both
    from paper_1910_04358_gb300.autotune import effective_path
    p = effective_path(t, info)
    if p == 0:
        return 1.10
    if p == 2:
        return 1.20 - (0.01 if t["bin_rows"] == 4 else 0.0)
    if p == 3:
        return 1.15 - (0.01 if t["seg_cut_bits"] == 7 else 0.0)
    return 1.105 - 0.03 * (t["fused_tile_kmers"] == 256) - 0.03 * (t["fused_short_max"] == 256)


def test_autotune_descends_from_every_path_the_geometry_runs(monkeypatch):
    import torch
    from paper_1910_04358_gb300 import autotune
    out = torch.zeros(4, dtype=torch.int32)
    # 256-byte groups: a request for the binned or the segment path runs the
    # fused one, so only paths 0 and 1 are searched, and the fused knobs are tuned
    idx = _FakeIndex(256)
    monkeypatch.setattr(autotune, "_time", lambda run, reps: _fused_cost(idx.t, idx.info))
    res = autotune.autotune(idx, lambda: None, lambda: [out], reps=1)
    assert autotune.effective_path(res["best"], idx.info) == 1
    assert res["best"]["fused_tile_kmers"] == 256 and res["best"]["fused_short_max"] == 256
    assert not any(tr["tuning"]["query_path"] in (2, 3) for tr in res["trials"])
    assert not any(tr["tuning"]["bin_rows"] != dict(autotune.KNOBS)["bin_rows"][0] for tr in res["trials"])
    assert idx.get_tuning() == res["best"]
    # 16-byte groups: four distinct paths; the binned and segment knobs vary
    # only on their own paths
    idx = _FakeIndex(16)
    monkeypatch.setattr(autotune, "_time", lambda run, reps: _fused_cost(idx.t, idx.info))
    res = autotune.autotune(idx, lambda: None, lambda: [out], reps=1)
    assert {tr["tuning"]["query_path"] for tr in res["trials"]} == {0, 1, 2, 3}
    assert all(tr["tuning"]["query_path"] == 2 for tr in res["trials"]
               if tr["tuning"]["bin_rows"] == 4)
    assert all(tr["tuning"]["query_path"] == 3 for tr in res["trials"]
               if tr["tuning"]["seg_cut_bits"] == 7)
    assert res["best"]["query_path"] == 1


def test_autotune_rejects_a_candidate_that_changes_the_answers(monkeypatch):
    import pytest
    import torch
    from paper_1910_04358_gb300 import autotune
    idx = _FakeIndex(16)
    start = idx.get_tuning()
    good, bad = torch.zeros(4, dtype=torch.int32), torch.ones(4, dtype=torch.int32)
    monkeypatch.setattr(autotune, "_time", lambda run, reps: 1.0)
    outputs = lambda: [bad if idx.t["fused_short_max"] == 64 else good]
    with pytest.raises(RuntimeError):
        autotune.autotune(idx, lambda: None, outputs, reps=1)
    assert idx.get_tuning() == start


def test_autotune_revisits_a_knob_once_a_later_one_moves(monkeypatch):
    # the expansion grid comes before the staged gathers in the search order;
    # its best value flips once they are on, so one pass would stop short
    import torch
    from paper_1910_04358_gb300 import autotune
    idx = _FakeIndex(16)

    def cost(t):
        if autotune.effective_path(t, idx.info) != 1:
            return 2.0
        e, a = t["expand_ctas_per_sm"], t["fused_async"]
        if a == 0:
            return 1.0 if e == 8 else 1.05
        return {2: 0.90, 8: 0.98}.get(e, 1.0)

    monkeypatch.setattr(autotune, "_time", lambda run, reps: cost(idx.t))
    out = torch.zeros(4, dtype=torch.int32)
    res = autotune.autotune(idx, lambda: None, lambda: [out], reps=1)
    assert res["best"]["fused_async"] == 1 and res["best"]["expand_ctas_per_sm"] == 2
    assert abs(res["ms"] - 0.90) < 1e-9


def test_serving_trace_refuses_requests_beyond_the_batch_bytes():
    import pytest
    from paper_1910_04358_gb300 import serve
    small = serve.Request(0, np.zeros(100, np.uint8), 400, 0.0)
    big = serve.Request(1, np.zeros(5000, np.uint8), 20000, 0.0)
    with pytest.raises(ValueError):
        serve._Trace([small, big], max_bytes=4096)
    with pytest.raises(ValueError):  # ids must be 0 .. n-1
        serve._Trace([serve.Request(3, np.zeros(4, np.uint8), 16, 0.0)], max_bytes=4096)
