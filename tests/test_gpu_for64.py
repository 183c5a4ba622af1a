"""GPU parity of 64-bit FOR columns (Sec. 4.1: GPU-FOR extended to BIGINT).

A FOR64 column is read by the fused kernel as an aggregate operand: the
mini block's int64 base plus a field of 0..64 bits taken from its 64-bit
words (through a 128-bit window when the field crosses a word).  Records
must equal the oracle's bit for bit (int64 arithmetic modulo 2^64).
Cases: every bit width 0..64, fields crossing words, the full int64 range,
SUM / SUM_MUL / SUM_SUB mixing FOR64 with FOR and DELTA operands, grouped
and ungrouped, host-resident pages, a BIGINT star join spanning many pages,
pages equal to the oracle's, and the errors for uses other than
aggregation.
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
    for f in ("key", "count", "val"):
        assert np.array_equal(got[f], want[f]), (what, f)


@pytest.fixture(scope="module")
def eng():
    e = dpf.Engine(device=0)
    yield e
    e.close()


def _table_workload(name, cols, rows, page_rows, aggs, group=(), preds=()):
    return {"name": name, "tables": {"fact": {"rows": rows, "page_rows": page_rows, "cols": cols}},
            "fact": "fact", "query": {"preds": list(preds), "joins": [], "group": list(group),
                                      "aggs": aggs}}


def _widths_column(rng, page_rows=256):
    """Mini block k of the column spans exactly 2^(k % 65) - 1 around a
    random base, so every bit width 0..64 occurs; rows are a ragged count."""
    blocks = []
    for k in range(130):
        bw = k % 65
        base = int(rng.integers(-(1 << 62), 1 << 62))
        if bw == 64:
            v = rng.integers(np.iinfo(np.int64).min, np.iinfo(np.int64).max, 128, dtype=np.int64, endpoint=True)
            v[0], v[1] = np.iinfo(np.int64).min, np.iinfo(np.int64).max
        else:
            span = (1 << bw) - 1
            lo = max(np.iinfo(np.int64).min, min(base, np.iinfo(np.int64).max - span))
            off = rng.integers(0, span, 128, dtype=np.uint64, endpoint=True) if bw else np.zeros(128, np.uint64)
            off[0], off[1] = 0, span
            v = (np.uint64(np.int64(lo).view(np.uint64)) + off).view(np.int64)
        blocks.append(v)
    v = np.concatenate(blocks)[:130 * 128 - 37]
    return v


@pytest.mark.parametrize("page_rows", [128, 256, 4096])
def test_every_bit_width(eng, page_rows):
    rng = np.random.default_rng(page_rows)
    z = _widths_column(rng)
    n = z.size
    cols = {"z": {"codec": "for64", "values": z},
            "x": {"codec": "for", "values": rng.integers(-1000, 1000, n, dtype=np.int32)},
            "d": {"codec": "delta", "values": np.sort(rng.integers(0, 1 << 20, n)).astype(np.int32)},
            "g": {"codec": "dict", "values": rng.integers(0, 5, n, dtype=np.int32)}}
    aggs = [{"op": "sum", "cols": ["z"]}, {"op": "sum_mul", "cols": ["z", "x"]},
            {"op": "sum_sub", "cols": ["d", "z"]}, {"op": "sum_mul", "cols": ["z", "z"]}]
    for group in ([], [{"col": "g"}]):
        w = _table_workload(f"widths_{page_rows}_{len(group)}", cols, n, page_rows, aggs, group)
        assert_same(eng.run(w), oracle.run_query(w, from_encoded=False), (page_rows, group))


@pytest.mark.parametrize("seed", range(6))
def test_filtered_rows_read_the_right_fields(eng, seed):
    """Predicates on 32-bit columns leave scattered survivors whose FOR64
    fields are read one by one (ragged tails, empty results)."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 20000))
    cols = {"z": {"codec": "for64", "values": rng.integers(-(1 << 63), (1 << 63) - 1, n, dtype=np.int64,
                                                         endpoint=True) >> int(rng.integers(0, 40))},
            "x": {"codec": "for", "values": rng.integers(0, 100, n, dtype=np.int32)},
            "g": {"codec": "dict", "values": rng.integers(0, 7, n, dtype=np.int32)}}
    cut = int(rng.integers(0, 101))
    w = _table_workload(f"filtered_{seed}", cols, n, int(rng.choice([128, 1024, 8192])),
                        [{"op": "count"}, {"op": "sum", "cols": ["z"]}, {"op": "sum_sub", "cols": ["z", "x"]}],
                        [{"col": "g"}] if seed % 2 else [], [{"col": "x", "op": "lt", "args": [cut]}])
    assert_same(eng.run(w), oracle.run_query(w, from_encoded=False), seed)


def test_bigint_star_join(eng):
    w = synth.star_join(rows=(1 << 21) + 99, bigint_measure=True)
    want = oracle.run_query(w, from_encoded=False)
    assert (np.abs(want["val"][:, 0]) > (1 << 40)).any()
    assert_same(eng.run(w), want)
    for t in (dpf.Tuning(0, 256, 0, 4), dpf.Tuning(1024, 128, dpf.HT_PLACE["global"], 0)):
        assert_same(eng.run(w, tuning=t), want, "tuning")


def test_host_resident_for64_pages():
    w = synth.star_join(rows=(1 << 19) + 3, bigint_measure=True, seed=21)
    want = oracle.run_query(w, from_encoded=False)
    e = dpf.Engine(device=0)
    try:
        e.load_workload(w, fact_placement="host")
        assert_same(e.run(w), want)
    finally:
        e.close()


def test_batched_with_32_bit_queries(eng):
    ws = [synth.star_join(rows=1 << 18, bigint_measure=True, seed=31), synth.star_join(rows=1 << 18, seed=31),
          synth.tiny_random_workload(3)]
    for w in ws:
        eng.load_workload(w)
    plans = [eng.plan(w) for w in ws]
    prep = eng.ctx.prepare(plans)
    try:
        eng.ctx.launch(prep)
        for i, w in enumerate(ws):
            assert_same(eng.ctx.read_result(prep, i), oracle.run_query(w, from_encoded=False), w["name"])
    finally:
        eng.ctx.release(prep)


def test_loaded_pages_equal_the_oracle_pages(eng):
    rng = np.random.default_rng(4)
    z = _widths_column(rng)
    cid = eng.ctx.load_column({"codec": "for64", "values": z}, table=900, page_rows=1024)
    want = oracle.encode_column({"codec": "for64", "values": z}, 1024)["blob"]
    assert np.array_equal(eng.ctx.column_bytes(cid), want)
    info = eng.ctx.column_info(cid)
    assert info["rows"] == z.size and info["raw_bytes"] == 8 * z.size
    eng.ctx.drop_column(cid)


def test_join_keys_and_group_keys_are_rejected(eng):
    """FOR64 columns serve as aggregate operands and in predicates
    (tests/test_gpu_for64_preds.py); as a join's probe column they are
    refused, and the unfused chain refuses FOR64 columns altogether."""
    base = synth.star_join(rows=1 << 14, bigint_measure=True, seed=41)
    eng.load_workload(base)
    cases = []
    w = copy.deepcopy(base)
    w["query"]["joins"][0]["fk"] = "m1"
    cases.append(w)
    for w in cases:
        with pytest.raises(dpf.DpfError) as e:
            eng.run(w)
        assert e.value.status == -1  # DPF_EINVAL
    with pytest.raises(dpf.DpfError) as e:
        eng.run_unfused(base)
    assert e.value.status == -1


def test_corrupt_for64_headers_are_rejected(eng):
    z = np.arange(300, dtype=np.int64) << 33
    enc = dpf.encode_column({"codec": "for64", "values": z}, 256)
    bad = copy.deepcopy(enc)
    bad["blob"][16 + 12] = 65  # bit width 65 in the first mini block header
    with pytest.raises(dpf.DpfError) as e:
        eng.ctx.load_encoded(bad)
    assert e.value.status == -9  # DPF_ECORRUPT
    bad = copy.deepcopy(enc)
    bad["blob"][16 + 8:16 + 12] = np.frombuffer(np.uint32(1 << 20).tobytes(), np.uint8)  # word offset
    with pytest.raises(dpf.DpfError) as e:
        eng.ctx.load_encoded(bad)
    assert e.value.status == -9


def test_wrapping_sums_match_their_closed_forms(eng):
    """The library's int64 sums wrap modulo 2^64 exactly as the closed forms
    of the oracle's pin do (4 * 2^62 -> 0, (2^32)^2 -> 0, INT64_MIN - 1 ->
    INT64_MAX, 3 * 2^40 * -7)."""
    i64 = np.iinfo(np.int64)
    z = np.array([1 << 62] * 4 + [1 << 32, i64.min, 3 << 40], np.int64)
    cols = {"z": {"codec": "for64", "values": z},
            "x": {"codec": "for", "values": np.array([1, 1, 1, 1, 1 << 30, 1, -7], np.int32)},
            "g": {"codec": "dict", "values": np.array([0, 0, 0, 0, 1, 2, 3], np.int32)},
            "one": {"codec": "for", "values": np.ones(7, np.int32)}}
    w = _table_workload("bigint_wrap", cols, 7, 128,
                        [{"op": "sum", "cols": ["z"]}, {"op": "sum_mul", "cols": ["z", "z"]},
                         {"op": "sum_sub", "cols": ["z", "one"]}, {"op": "sum_mul", "cols": ["z", "x"]}],
                        [{"col": "g"}])
    r = eng.run(w)
    assert r["count"].tolist() == [4, 1, 1, 1]
    assert r["val"].tolist() == [[0, 0, -4, 0], [1 << 32, 0, (1 << 32) - 1, 1 << 62],
                                 [int(i64.min), 0, int(i64.max), int(i64.min)],
                                 [3 << 40, 0, (3 << 40) - 1, -21 * (1 << 40)]]
