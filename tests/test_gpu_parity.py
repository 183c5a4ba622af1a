"""GPU parity: the fused kernel's records equal the oracle's, bit for bit.

Everything is integer (int64 aggregates over int32 inputs), so the
tolerance is zero: keys, counts and every aggregate must be identical.
Cases: random small workloads mixing every operator, codec and ragged tail;
the three workload shapes at sizes spanning many chunks and pages; launch
knobs (chunk rows, threads, hash-table placement); batched launches, CUDA
graph replays and repeated launches (scratch state reset); host-resident
pages; error reporting.
"""

import copy

import numpy as np
import pytest

import oracle
import paper_2605_10511_gb300 as dpf
import synth

pytestmark = pytest.mark.gpu


def assert_same(got, want, what=""):
    assert got.shape == want.shape, (what, got, want)
    assert np.array_equal(got["key"], want["key"]), what
    assert np.array_equal(got["count"], want["count"]), what
    assert np.array_equal(got["val"], want["val"]), what


@pytest.fixture(scope="module")
def eng():
    e = dpf.Engine(device=0)
    yield e
    e.close()


_oracle_cache = {}


def expect(w):
    key = (w["name"], repr(w["query"]))
    if key not in _oracle_cache:
        _oracle_cache[key] = oracle.run_query(w, from_encoded=False)
    return _oracle_cache[key]


@pytest.mark.parametrize("seed", range(40))
def test_random_small_workloads(eng, seed):
    w = synth.tiny_random_workload(seed)
    assert_same(eng.run(w), expect(w), w["name"])


@pytest.fixture(scope="module")
def shapes():
    return {
        "scan": synth.scan_filter_aggregate(rows=1 << 20),
        "star": synth.star_join(rows=(1 << 21) + 777, page_rows=65536, clustered=True),
        "star_unsorted": synth.star_join(rows=(1 << 21) + 777, page_rows=65536, clustered=False),
        "strings": synth.strings(rows=(1 << 20) + 4001, page_rows=32768),
    }


@pytest.mark.parametrize("name", ["scan", "star", "star_unsorted", "strings"])
def test_workload_shapes(eng, shapes, name):
    w = shapes[name]
    assert_same(eng.run(w), expect(w), name)


def _a_step(p):
    """False for a predicate every row passes: the planner compiles it to no step."""
    if p["op"] in ("prefix", "contains") and len(bytes(p["args"][0])) == 0:
        return False
    return not (p["op"] == "like" and all(b == 0x25 for b in bytes(p["args"][0])))


@pytest.mark.parametrize("seed", range(0, 40, 3))
def test_unfused_chain_random_small(eng, seed):
    w = synth.tiny_random_workload(seed)
    q = w["query"]
    preds = [p for p in q["preds"] if _a_step(p)]
    if w["tables"]["fact"]["cols"]["s"]["codec"] == "fsst" and any(p["col"] == "s" for p in preds) \
            or any(p["op"] == "contains" for p in preds) \
            or any("z" in a.get("cols", []) for a in q["aggs"]):
        # the unfused baseline evaluates PREFIX on STR columns only and
        # decodes 32-bit columns only
        with pytest.raises(dpf.DpfError) as ex:
            eng.run_unfused(w)
        assert ex.value.status == -1  # DPF_EINVAL
        return
    assert_same(eng.run_unfused(w), expect(w), w["name"])


@pytest.mark.parametrize("name", ["scan", "star", "strings"])
def test_unfused_chain_shapes(eng, shapes, name):
    w = shapes[name]
    assert_same(eng.run_unfused(w), expect(w), name)
    h = eng.plan(w)
    prep = eng.ctx.prepare_unfused(h)
    try:
        eng.ctx.launch(prep)
        eng.ctx.read_result(prep, 0)
        st = eng.ctx.prep_stats(prep)
        assert st["launches"] >= 4 and st["intermediate_bytes"] > 4 * w["tables"][w["fact"]]["rows"]
    finally:
        eng.ctx.release(prep)


def test_clustered_and_unsorted_star_agree(eng, shapes):
    assert_same(eng.run(shapes["star"]), eng.run(shapes["star_unsorted"]))


@pytest.mark.parametrize("chunk_rows", [512, 2048, 262144])
@pytest.mark.parametrize("threads", [128, 256])
@pytest.mark.parametrize("place", ["smem", "global"])
def test_launch_knobs_do_not_change_results(eng, shapes, chunk_rows, threads, place):
    for name in ("star", "strings"):
        w = shapes[name]
        t = dpf.Tuning(chunk_rows, threads, dpf.HT_PLACE[place], 0)
        assert_same(eng.run(w, tuning=t), expect(w), (name, chunk_rows, threads, place))


def test_batched_launch_equals_each_query(eng, shapes):
    ws = [shapes["scan"], shapes["star"], shapes["strings"]] + [synth.tiny_random_workload(s) for s in (1, 4, 5, 9)]
    for w in ws:
        eng.load_workload(w)
    plans = [eng.plan(w) for w in ws]
    prep = eng.ctx.prepare(plans)
    try:
        eng.ctx.launch(prep)
        for i, w in enumerate(ws):
            assert_same(eng.ctx.read_result(prep, i), expect(w), w["name"])
        # launch again: the kernel left its scratch state zeroed
        eng.ctx.launch(prep)
        for i, w in enumerate(ws):
            assert_same(eng.ctx.read_result(prep, i), expect(w), w["name"])
    finally:
        eng.ctx.release(prep)


def test_graph_replay(eng, shapes):
    import torch
    w = shapes["strings"]
    eng.load_workload(w)
    prep = eng.ctx.prepare([eng.plan(w)])
    s = torch.cuda.Stream()
    try:
        eng.ctx.capture_graph(prep, s)
        for _ in range(3):
            eng.ctx.launch_graph(prep, s)
            assert_same(eng.ctx.read_result(prep, 0), expect(w))
    finally:
        eng.ctx.release(prep)


def test_execute_and_fetch(eng, shapes):
    w = shapes["scan"]
    eng.load_workload(w)
    ids = eng.ctx.execute([eng.plan(w)])
    assert_same(eng.ctx.fetch(ids[0]), expect(w))
    with pytest.raises(dpf.DpfError) as e:
        eng.ctx.fetch(ids[0])
    assert e.value.status == -8


def test_host_resident_fact_table(shapes):
    w = copy.deepcopy(shapes["star"])
    w["name"] += "_host"
    e = dpf.Engine(device=0)
    try:
        e.load_workload(w, fact_placement="host")
        assert_same(e.run(w), expect(shapes["star"]))
        s = copy.deepcopy(shapes["strings"])
        s["name"] += "_host"
        e.load_workload(s, fact_placement="host")
        assert_same(e.run(s), expect(shapes["strings"]))
    finally:
        e.close()


def test_duplicate_build_key_is_reported(eng):
    w = synth.tiny_random_workload(3, rows=1000, page_rows=256)
    w["name"] = "dupkey"
    w["tables"]["dim"]["cols"]["k"]["values"][1] = w["tables"]["dim"]["cols"]["k"]["values"][0]
    w["query"]["joins"] = [{"fk": "fk", "dim": "dim", "key": "k", "preds": [], "payload": []}]
    w["query"]["group"] = []
    eng.load_workload(w)
    with pytest.raises(dpf.DpfError) as e:
        eng.plan(w)
    assert e.value.status == -4


def test_corrupt_pages_are_rejected(eng):
    col = {"codec": "for", "values": np.arange(5000, dtype=np.int32)}
    enc = dpf.encode_column(col, 1024)
    enc["blob"][16 + 4] = 40  # bit width 40 in the first mini block header
    with pytest.raises(dpf.DpfError) as e:
        eng.ctx.load_encoded(enc)
    assert e.value.status == -9


def test_loaded_pages_are_the_encoded_pages(eng):
    w = synth.tiny_random_workload(7)
    eng.load_workload(w)
    for tname, t in w["tables"].items():
        for cname, c in t["cols"].items():
            if c["codec"] == "fsst":
                continue  # independent symbol tables; the CPU tests cross-decode these pages
            got = eng.ctx.column_bytes(eng.col(w, tname, cname))
            want = oracle.encode_column(c, t["page_rows"])["blob"]
            assert np.array_equal(got, want), (tname, cname)


@pytest.mark.parametrize("rows,page_rows", [(1, 128), (127, 128), (129, 128), (5000, 4096),
                                            (1 << 20, 1 << 20), ((1 << 20) + 3, 1 << 20)])
def test_edge_sizes(eng, rows, page_rows):
    """One row, ragged single mini blocks, one row past a page, and the
    largest page (2^20 rows) with a 3-row second page."""
    w = synth.tiny_random_workload(77, rows=rows, page_rows=page_rows)
    w["name"] = f"edge_{rows}_{page_rows}"
    assert_same(eng.run(w), expect(w), w["name"])


def test_largest_ticket(eng, shapes):
    """A ticket of 2^24 rows (the most dpf_prepare accepts) covers many pages."""
    w = shapes["star"]
    t = dpf.Tuning(1 << 24, 256, 0, 0)
    assert_same(eng.run(w, tuning=t), expect(w), "chunk 2^24")


def test_memory_returns_after_release_and_blocks_are_reused(shapes):
    e = dpf.Engine(device=0)
    try:
        w = shapes["scan"]
        e.load_workload(w)
        h = e.plan(w)
        base = e.ctx.memory_used()
        for _ in range(5):
            p = e.ctx.prepare([h])
            e.ctx.launch(p)
            assert_same(e.ctx.read_result(p, 0), expect(w), "reuse")
            e.ctx.release(p)
            assert e.ctx.memory_used() == base
    finally:
        e.close()


def test_budget_is_enforced():
    e = dpf.Engine(device=0, hbm_budget=1 << 20)
    try:
        w = synth.scan_filter_aggregate(rows=1 << 20)  # 4.6 MB of pages
        w["name"] = "budget_scan"
        with pytest.raises(dpf.DpfError) as ex:
            e.load_workload(w)
        assert ex.value.status == -2  # DPF_ENOMEM
    finally:
        e.close()


@pytest.mark.parametrize("clustered", [True, False])
def test_star_with_date_filter_prunes_and_matches(eng, clustered):
    """One year of the date dimension: on the date-clustered fact most mini
    blocks of the date key are skipped from their headers; the unsorted fact
    prunes nothing.  Both equal the oracle and each other."""
    w = synth.star_join(rows=(1 << 21) + 333, page_rows=65536, clustered=clustered, date_year=1994)
    got = eng.run(w)
    assert_same(got, expect(w), ("date filter", clustered))
    assert got.shape[0] >= 1 and int(got["count"].sum()) > 0


@pytest.mark.parametrize("name", ["scan", "star", "strings"])
def test_four_cta_build_matches(eng, shapes, name):
    """The kernel build for four resident CTAs per SM (ctas_per_sm = 4)."""
    w = shapes[name]
    assert_same(eng.run(w, tuning=dpf.Tuning(0, 256, 0, 4)), expect(w), (name, "4 CTAs"))


@pytest.mark.parametrize("text", [False, True])
@pytest.mark.parametrize("op,pat", [("prefix", b"q"), ("contains", b"ab"), ("contains", b"q q"),
                                    ("contains", b""), ("prefix", b""), ("contains", b"x" * 32)])
@pytest.mark.parametrize("codec", ["str", "fsst"])
def test_string_predicates_on_str_and_fsst(eng, codec, op, pat, text):
    """PREFIX and CONTAINS (KMP) on raw and FSST-coded strings, random and
    text-like, with an empty pattern and one longer than every string."""
    w = synth.strings(rows=(1 << 18) + 77, seed=13, page_rows=32768, codec=codec, text=text)
    w["query"]["preds"] = [{"col": "s", "op": op, "args": [pat]}]
    assert_same(eng.run(w), expect(w), (codec, op, pat, text))


def test_fsst_codes_outside_the_table_are_rejected(eng):
    w = synth.strings(rows=5000, seed=3, page_rows=1024, codec="fsst", text=True)
    enc = dpf.encode_column(w["tables"]["fact"]["cols"]["s"], 1024)
    bad = dict(enc, dict=enc["dict"][:6])  # two symbols left: most codes name none
    with pytest.raises(dpf.DpfError) as ex:
        eng.ctx.load_encoded(bad)
    assert ex.value.status == -9  # DPF_ECORRUPT


def test_batch_mixing_lean_and_string_matcher_queries(eng):
    """A batch with one CONTAINS-on-FSST query runs the kernel build with the
    general string matcher for every query in it; the same queries alone run
    the lean build (raw PREFIX, no string step) or the matcher build.  Every
    record equals the oracle's either way."""
    ws = [synth.strings(rows=(1 << 16) + 5, page_rows=8192, seed=61),
          synth.strings(rows=(1 << 16) + 5, page_rows=8192, seed=62, text=True, contains=b"ab", codec="fsst"),
          synth.star_join(rows=(1 << 17) + 3, seed=63)]
    for w in ws:
        eng.load_workload(w)
    plans = [eng.plan(w) for w in ws]
    for i, w in enumerate(ws):
        assert_same(eng.run(w), expect(w), w["name"])
    prep = eng.ctx.prepare(plans)
    try:
        eng.ctx.launch(prep)
        for i, w in enumerate(ws):
            assert_same(eng.ctx.read_result(prep, i), expect(w), ("batch", w["name"]))
    finally:
        eng.ctx.release(prep)
