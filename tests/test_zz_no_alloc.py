"""The allocation-free entry point gives the same records as the prepared launch.

``dpf_execute_noalloc`` is for callers that cannot allocate device memory
while they run a query (a framework owning all device memory in its own
pool, a serving loop that forbids allocation, code inside another
allocator).  It runs the fused kernel with its scratch in a fixed region of
the library image; the caller owns the output buffers.  This file runs last
so that a failure here leaves every other test already run.  Results are
integers: they must be identical, on two calls in a row (the region keeps
the previous call's contents and each call must clear what it needs).
"""

import numpy as np
import pytest

import paper_2605_10511_gb300 as dpf
import synth

pytestmark = pytest.mark.gpu


def _noalloc(eng, w, cap):
    import torch
    h = eng.plan(w)
    out = torch.zeros(cap * dpf.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    eng.ctx.execute_noalloc(h, out.data_ptr(), cap, cnt.data_ptr(), stream)
    torch.cuda.synchronize()
    n = int(cnt.item())
    raw = out[: n * dpf.RECORD_DTYPE.itemsize].cpu().numpy().tobytes()
    return np.frombuffer(raw, dtype=dpf.RECORD_DTYPE).copy()


def _same(a, b):
    assert a.shape == b.shape, (a, b)
    assert np.array_equal(a["key"], b["key"])
    assert np.array_equal(a["count"], b["count"])
    assert np.array_equal(a["val"], b["val"])


def test_noalloc_matches_prepared_launch_twice():
    eng = dpf.Engine(device=0)
    try:
        workloads = [synth.star_join(rows=(1 << 20) + 333, clustered=True),
                     synth.strings(rows=(1 << 19) + 77, page_rows=32768),
                     synth.scan_filter_aggregate(rows=(1 << 18) + 5),
                     synth.tiny_random_workload(4)]
        for w in workloads:
            eng.load_workload(w)
            want = eng.run(w)
            for _ in range(2):
                _same(_noalloc(eng, w, cap=2048), want)
    finally:
        eng.close()


def test_noalloc_rejects_oversize_plans():
    """200 x 200 groups x 5 int64 accumulators need 1.6 MB > the 1 MiB region:
    rejected with a clear error, while the prepared launch still runs it."""
    rng = np.random.default_rng(9)
    n = 20000
    w = {"name": "noalloc_oversize", "fact": "fact", "tables": {"fact": {
        "rows": n, "page_rows": 4096, "cols": {
            "g1": {"codec": "dict", "values": rng.integers(0, 200, n, dtype=np.int32)},
            "g2": {"codec": "dict", "values": rng.integers(0, 200, n, dtype=np.int32)},
            "m": {"codec": "for", "values": rng.integers(0, 1000, n, dtype=np.int32)}}}},
        "query": {"preds": [], "joins": [], "group": [{"col": "g1"}, {"col": "g2"}],
                  "aggs": [{"op": "sum", "cols": ["m"]}] * 4}}
    eng = dpf.Engine(device=0)
    try:
        eng.load_workload(w)
        assert eng.run(w)["count"].sum() == n
        with pytest.raises(dpf.DpfError) as e:
            _noalloc(eng, w, cap=40000)
        assert e.value.status == -1 and "scratch" in str(e.value)
        small = synth.scan_filter_aggregate(rows=4096, page_rows=4096)
        eng.load_workload(small)
        with pytest.raises(dpf.DpfError) as e:
            _noalloc(eng, small, cap=0)
        assert e.value.status == -1
    finally:
        eng.close()
