"""The allocation-free entry point gives the same records as the prepared launch.

``dpf_execute_noalloc`` is for callers that cannot allocate device memory
while they run a query (a framework owning all device memory in its own
pool, a serving loop that forbids allocation, code inside another
allocator).  It runs the fused kernel with its scratch in a fixed region of
the library image; the caller owns the output buffers.  This file runs last
so that a failure here leaves every other test already run.  Results are
integers: they must be identical, on two calls in a row (the region keeps
the previous call's contents and each call must clear what it needs), and
equal to the oracle's records.  The call refuses a capturing stream, and the
kernel's data checks are read back with ``dpf_noalloc_status``.
"""

import numpy as np
import pytest

import oracle
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
            _same(want, oracle.run_query(w, from_encoded=False, threads=0))
            for _ in range(2):
                _same(_noalloc(eng, w, cap=2048), want)
                assert eng.ctx.noalloc_status() == 0
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


def test_noalloc_refuses_a_capturing_stream():
    """The call copies its plan from memory that lives only for the call, so
    it must not be recorded into a CUDA graph: it fails and enqueues nothing.
    (The capture is ended without replaying anything.)"""
    import torch
    eng = dpf.Engine(device=0)
    try:
        w = synth.scan_filter_aggregate(rows=20000, page_rows=4096)
        eng.load_workload(w)
        want = oracle.run_query(w, from_encoded=False)
        _same(_noalloc(eng, w, cap=4), want)  # the set-up call, outside any capture
        h = eng.plan(w)
        out = torch.zeros(4 * dpf.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            g.capture_begin()
            try:
                with pytest.raises(dpf.DpfError) as e:
                    eng.ctx.execute_noalloc(h, out.data_ptr(), 4, cnt.data_ptr(), s)
            finally:
                g.capture_end()
        assert e.value.status == -1 and "captur" in str(e.value)
        torch.cuda.synchronize()
        _same(_noalloc(eng, w, cap=4), want)  # still usable afterwards
    finally:
        eng.close()


def test_noalloc_status_reports_a_corrupt_dictionary_code():
    """A DICT group-key page that passes load validation (its mini block base
    lies inside the dictionary) but packs a code beyond the dictionary: the
    kernel drops that row and sets its status word, which the status call
    reports as DPF_ECORRUPT (the prepared path reports it from its read)."""
    rng = np.random.default_rng(21)
    n = 3000
    g = np.array([10, 20, 30], np.int32)[rng.integers(0, 3, n)]
    g[0], g[1] = 10, 30  # mini block 0 holds codes 0 and 2: base 0, bit width 2
    m = rng.integers(1, 1000, n, dtype=np.int32)
    enc = dpf.encode_column({"codec": "dict", "values": g}, 1024)
    blob = enc["blob"]
    assert int.from_bytes(blob[16:20].tobytes(), "little") == 0  # base of mini block 0
    assert blob[20] == 2  # its bit width
    nmb = 1024 // 128
    pay = (16 + nmb * 8 + 15) // 16 * 16
    blob[pay] |= 3  # row 0's code becomes 3, beyond the 3-value dictionary
    w = {"name": "noalloc_corrupt", "fact": "fact", "tables": {"fact": {
        "rows": n, "page_rows": 1024, "cols": {"g": {"codec": "dict", "values": g},
                                                "m": {"codec": "for", "values": m}}}},
        "query": {"preds": [], "joins": [], "group": [{"col": "g"}],
                  "aggs": [{"op": "sum", "cols": ["m"]}]}}
    eng = dpf.Engine(device=0)
    try:
        tid = 77
        eng.tables[(w["name"], "fact")] = tid
        eng.cols[(w["name"], "fact", "g")] = eng.ctx.load_encoded(enc, table=tid)
        eng.cols[(w["name"], "fact", "m")] = eng.ctx.load_column(w["tables"]["fact"]["cols"]["m"], table=tid,
                                                                  page_rows=1024)
        clean = synth.scan_filter_aggregate(rows=5000, page_rows=1024)
        eng.load_workload(clean)
        _noalloc(eng, clean, cap=4)
        assert eng.ctx.noalloc_status() == 0
        got = _noalloc(eng, w, cap=8)
        with pytest.raises(dpf.DpfError) as e:
            eng.ctx.noalloc_status()
        assert e.value.status == -9  # DPF_ECORRUPT
        assert int(got["count"].sum()) == n - 1  # the corrupt row was dropped
        with pytest.raises(dpf.DpfError) as e:
            eng.run(w)
        assert e.value.status == -9
        _noalloc(eng, clean, cap=4)  # the next call starts from a clean status word
        assert eng.ctx.noalloc_status() == 0
    finally:
        eng.close()
