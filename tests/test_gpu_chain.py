"""GPU parity of join chains: scan, probe and build (Sec. 3.1 Kernel #2).

A chain's inner tables are built by ``dpf_build_hash`` (Kernel #1) and
``dpf_build_hash_probe`` (Kernel #2: the scan probes the earlier tables and
its kept rows, with payload fields carried from them, go into the next
table); the fused kernel then probes the last table (Kernel #3).  Records
must equal the oracle's bit for bit.  Cases: random small chains (dense
and sparse keys, so direct and open-addressing tables at every link,
deeper chains, a table probed by two, payloads from columns and from
earlier tables), the LINEITEM -> ORDERS -> CUSTOMER workload at sizes
spanning many pages, launch knobs, host-resident pages, the entry counts
of the built tables, and error reporting.
"""

import ctypes

import numpy as np
import pytest

import oracle
import paper_2605_10511_gb300 as dpf
import synth
from paper_2605_10511_gb300.engine import PlanHandle
from _hand_worked import hand_worked_chains

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


_want = {}


def expect(w):
    key = (w["name"], repr(w["query"]))
    if key not in _want:
        _want[key] = oracle.run_query(w, from_encoded=False)
    return _want[key]


def test_hand_worked_chain(eng):
    for w, want in hand_worked_chains():
        assert_same(eng.run(w), want, w["name"])


@pytest.mark.parametrize("seed", range(48))
def test_random_small_chains(eng, seed):
    w = synth.tiny_chain_workload(seed)
    assert_same(eng.run(w), expect(w), w["name"])


@pytest.fixture(scope="module")
def chains():
    return {"dense": synth.chain_join(rows=(1 << 21) + 333, page_rows=65536),
            "sparse": synth.chain_join(rows=(1 << 20) + 77, page_rows=32768, sparse_orderkeys=True)}


@pytest.mark.parametrize("name", ["dense", "sparse"])
def test_chain_workload(eng, chains, name):
    w = chains[name]
    got = eng.run(w)
    want = expect(w)
    assert want.shape[0] > 50
    assert_same(got, want, name)


@pytest.mark.parametrize("name", ["dense", "sparse"])
def test_built_tables_hold_the_kept_rows(eng, chains, name):
    """Entries of the CUSTOMER and ORDERS tables equal the rows that pass
    (counted here with numpy from the generated arrays)."""
    w = chains[name]
    eng.load_workload(w)
    j = w["query"]["joins"][0]
    t = w["tables"]
    seg = j["joins"][0]["preds"][0]["args"][0]
    cut = j["preds"][0]["args"][0]
    c_keep = t["customer"]["cols"]["c_segment"]["values"] == seg
    kept_cust = set(t["customer"]["cols"]["c_custkey"]["values"][c_keep].tolist())
    o = t["orders"]["cols"]
    o_keep = (o["o_orderdate"]["values"] < cut) & np.isin(o["o_custkey"]["values"],
                                                          np.array(sorted(kept_cust), np.int32))
    ht_c = eng.build_join(w, j["joins"][0])
    ht_o = eng.build_join(w, j)
    assert eng.ctx.hash_info(ht_c)["entries"] == int(c_keep.sum())
    assert eng.ctx.hash_info(ht_o)["entries"] == int(o_keep.sum())


@pytest.mark.parametrize("place", ["auto", "smem", "global"])
@pytest.mark.parametrize("ctas", [0, 4])
def test_launch_knobs_on_a_chain(eng, chains, place, ctas):
    w = chains["dense"]
    t = dpf.Tuning(0, 256, dpf.HT_PLACE[place], ctas)
    assert_same(eng.run(w, tuning=t), expect(w), (place, ctas))


def test_chain_with_host_resident_pages():
    """Every table's pages in mapped pinned host memory: the build kernels
    and the fused kernel read them over the chip-to-chip link."""
    w = synth.chain_join(rows=(1 << 19) + 5, page_rows=16384, seed=8)
    e = dpf.Engine(device=0)
    try:
        e.load_workload(w, placement="host")
        assert_same(e.run(w), expect(w), "host")
    finally:
        e.close()


def test_chain_groups_by_a_column_of_the_outer_fact(eng):
    for seed in range(3):
        w = synth.tiny_chain_workload(100 + seed, rows=3000, page_rows=256)
        w["query"]["group"] = [{"col": "g"}]
        assert_same(eng.run(w), expect(w), seed)


def _small_chain(eng):
    w = synth.chain_join(rows=1 << 14, page_rows=4096, seed=12)
    eng.load_workload(w)
    col = lambda t, c: eng.col(w, t, c)  # noqa: E731
    ht_c = eng.ctx.build_hash(col("customer", "c_custkey"), [col("customer", "c_nation")])
    return w, col, ht_c


def test_errors_are_reported(eng):
    w, col, ht_c = _small_chain(eng)
    key = col("orders", "o_orderkey")
    fk = [(col("orders", "o_custkey"), ht_c)]
    bad = [
        dict(payload=[("join", 1, 0)], joins=fk),                       # join index out of range
        dict(payload=[("join", 0, 1)], joins=fk),                       # table has one field
        dict(payload=[], joins=[(col("orders", "o_custkey"), 9999)]),   # unknown table
        dict(payload=[], joins=[(col("lineitem", "l_orderkey"), ht_c)]),  # another table's column
        dict(payload=[], joins=[(col("orders", "o_priority"), ht_c)]),  # DICT probe column
        dict(payload=[col("orders", "o_orderdate")], joins=fk),         # FOR payload column
    ]
    for i, b in enumerate(bad):
        with pytest.raises(dpf.DpfError) as e:
            eng.ctx.build_hash_probe(key, **b)
        assert e.value.status == -1, i  # DPF_EINVAL
    with pytest.raises(dpf.DpfError) as e:
        eng.ctx.build_hash_probe(col("orders", "o_priority"), [], [], fk)
    assert e.value.status == -1  # DICT key column


def test_duplicate_key_in_a_probe_build_is_reported(eng):
    w, col, ht_c = _small_chain(eng)
    # o_custkey repeats: as a key of the probe-build it must be reported
    with pytest.raises(dpf.DpfError) as e:
        eng.ctx.build_hash_probe(col("orders", "o_custkey"), [], [],
                                 [(col("orders", "o_custkey"), ht_c)])
    assert e.value.status == -4  # DPF_EDUPKEY


def test_probe_build_matches_a_plain_build_when_nothing_is_dropped(eng):
    """Probing a table that holds every key and carries nothing keeps every
    row: the table equals the one dpf_build_hash makes (same entries, and a
    plan over it gives the same records)."""
    w, col, _ = _small_chain(eng)
    ht_all = eng.ctx.build_hash(col("customer", "c_custkey"))
    a = eng.ctx.build_hash(col("orders", "o_orderkey"), [col("orders", "o_priority")])
    b = eng.ctx.build_hash_probe(col("orders", "o_orderkey"), [col("orders", "o_priority")], [],
                                 [(col("orders", "o_custkey"), ht_all)])
    assert eng.ctx.hash_info(a) == eng.ctx.hash_info(b)
    recs = []
    for ht in (a, b):
        joins = (dpf.Join * 1)(dpf.Join(col("lineitem", "l_orderkey"), ht))
        keys = (dpf.Key * 1)(dpf.Key(1, 0, 0, 0))
        plan = dpf.Plan(0, None, 1, ctypes.cast(joins, ctypes.POINTER(dpf.Join)),
                        1, ctypes.cast(keys, ctypes.POINTER(dpf.Key)), 0, None, 0)
        prep = eng.ctx.prepare([PlanHandle(plan, (joins, keys))])
        try:
            eng.ctx.launch(prep)
            recs.append(eng.ctx.read_result(prep, 0))
        finally:
            eng.ctx.release(prep)
    assert_same(recs[0], recs[1])
    assert recs[0]["count"].sum() == w["tables"]["lineitem"]["rows"]


@pytest.mark.parametrize("rows", [1 << 24, 1 << 26])
def test_chain_with_rank_directory_table(rows):
    """LINEITEM -> ORDERS -> CUSTOMER with ORDERS' kept keys spread over more
    than 2^22 keys: ORDERS' table is a rank directory (presence bits of 64
    keys and a count per 16-byte word, then the kept payloads) instead of one
    word per key of the range.  Its device bytes must be those of the rank
    layout, far below a direct table's 4 bytes per key; the records must
    equal the oracle's; a scan + probe + build probing the rank table (a
    longer chain) is checked the same way in the unfused chain."""
    w = synth.chain_join(rows=rows)
    eng = dpf.Engine(device=0)
    try:
        eng.load_workload(w)
        before = eng.ctx.memory_used()
        j = w["query"]["joins"][0]
        eng.build_joins(w)
        hts = [eng.hts[(w["name"], repr(j))]]
        info = eng.ctx.hash_info(hts[0])
        assert info["capacity"] > 1 << 22, info  # the kept keys' range
        rank_bytes = 16 * ((info["capacity"] + 63) // 64) + 4 * info["entries"]
        grown = eng.ctx.memory_used() - before
        assert grown < 2 * rank_bytes + (64 << 20) and grown < 4 * info["capacity"], (grown, info)
        want = oracle.run_query(w, from_encoded=False, threads=0)
        assert_same(eng.run(w), want, "fused")
        assert_same(eng.run_unfused(w), want, "unfused")
    finally:
        eng.close()
