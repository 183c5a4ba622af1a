"""GPU parity of prepared chains (Sec. 3.1 Kernels #1 -> #2 -> #3 as one unit).

``dpf_build_hash_deferred`` prepares a table without building it;
``dpf_prepare_chain`` makes a batch whose every launch rebuilds its tables
in order and then runs the plan, on one stream, plain or replayed from one
CUDA graph.  Records must equal the oracle's bit for bit on every launch,
the tables' entry counts (read by ``dpf_hash_wait`` after a launch) must
equal the exactly sized builds', a table nothing has run must behave as an
empty table, a referenced table cannot be dropped, and a duplicate key must
come back through the wait.
"""

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


_want = {}


def expect(w):
    key = (w["name"], repr(w["query"]))
    if key not in _want:
        _want[key] = oracle.run_query(w, from_encoded=False, threads=0)
    return _want[key]


@pytest.mark.parametrize("seed", range(12))
def test_random_small_chains(seed):
    w = synth.tiny_chain_workload(seed)
    eng = dpf.Engine(device=0)
    try:
        prep = eng.prepare_chain(w)
        for rep in range(2):  # every launch rebuilds the tables from empty
            eng.ctx.launch(prep)
            assert_same(eng.ctx.read_result(prep, 0), expect(w), (w["name"], rep))
            eng.wait_joins(w, deferred=True)
        eng.ctx.release(prep)
    finally:
        eng.close()


@pytest.mark.parametrize("sparse", [False, True])
def test_chain_plain_and_graph_launches(sparse):
    """Plain launches, then a captured graph replayed three times; entry
    counts equal the exactly sized builds'."""
    import torch
    w = synth.chain_join(rows=(1 << 21) + 333, page_rows=65536, sparse_orderkeys=sparse, seed=3)
    a, b = dpf.Engine(device=0), dpf.Engine(device=0)
    try:
        assert_same(b.run(w), expect(w), "exact")
        prep = a.prepare_chain(w)
        s = torch.cuda.Stream()
        a.ctx.launch(prep, s)
        assert_same(a.ctx.read_result(prep, 0), expect(w), "plain")
        a.wait_joins(w, deferred=True)
        a.ctx.capture_graph(prep, s)
        for rep in range(3):
            a.ctx.launch_graph(prep, s)
            assert_same(a.ctx.read_result(prep, 0), expect(w), ("graph", rep))
            a.wait_joins(w, deferred=True)
        for ta, tb in zip(a.chain_tables(w, deferred=True), b.chain_tables(w)):
            assert a.ctx.hash_info(ta)["entries"] == b.ctx.hash_info(tb)["entries"]
        a.ctx.release(prep)
    finally:
        a.close()
        b.close()


def test_star_join_tables():
    """Four independent deferred tables (no chain between them)."""
    w = synth.star_join(rows=(1 << 22) + 17, page_rows=65536, seed=6)
    eng = dpf.Engine(device=0)
    try:
        prep = eng.prepare_chain(w)
        eng.ctx.launch(prep)
        assert_same(eng.ctx.read_result(prep, 0), expect(w), "star")
        eng.ctx.release(prep)
    finally:
        eng.close()


def test_full_size_chain():
    w = synth.chain_join(rows=1 << 25)
    eng = dpf.Engine(device=0)
    try:
        prep = eng.prepare_chain(w)
        for rep in range(2):
            eng.ctx.launch(prep)
            assert_same(eng.ctx.read_result(prep, 0), expect(w), rep)
        eng.ctx.release(prep)
    finally:
        eng.close()


def test_host_resident_pages():
    w = synth.chain_join(rows=(1 << 19) + 5, page_rows=16384, seed=8)
    eng = dpf.Engine(device=0)
    try:
        eng.load_workload(w, placement="host")
        prep = eng.prepare_chain(w)
        eng.ctx.launch(prep)
        assert_same(eng.ctx.read_result(prep, 0), expect(w), "host")
        eng.ctx.release(prep)
    finally:
        eng.close()


def test_unrun_tables_are_empty_and_referenced_tables_stay():
    """A plan over deferred tables that no chain has run finds no match; a
    table a prepared chain rebuilds cannot be dropped until the chain is
    released."""
    w = synth.chain_join(rows=1 << 16, page_rows=4096, seed=10)
    eng = dpf.Engine(device=0)
    try:
        eng.load_workload(w)
        h = eng.plan(w, deferred=True)
        prep = eng.ctx.prepare([h])
        eng.ctx.launch(prep)
        assert eng.ctx.read_result(prep, 0).shape[0] == 0  # grouped: no group has a row
        eng.ctx.release(prep)
        chain = eng.ctx.prepare_chain(eng.chain_tables(w, deferred=True), [h])
        for ht in eng.chain_tables(w, deferred=True):
            with pytest.raises(dpf.DpfError) as e:
                eng.ctx.drop_hash(ht)
            assert e.value.status == -1
        eng.ctx.launch(chain)
        assert_same(eng.ctx.read_result(chain, 0), expect(w), "after")
        eng.ctx.release(chain)
        for ht in eng.chain_tables(w, deferred=True):
            eng.ctx.drop_hash(ht)
    finally:
        eng.close()


def test_duplicate_key_and_bad_chains():
    w = synth.chain_join(rows=1 << 14, page_rows=4096, seed=12)
    eng = dpf.Engine(device=0)
    try:
        eng.load_workload(w)
        col = lambda t, c: eng.col(w, t, c)  # noqa: E731
        cust = eng.ctx.build_hash_deferred(col("customer", "c_custkey"), [col("customer", "c_nation")])
        bad = eng.ctx.build_hash_deferred(col("orders", "o_custkey"), [], [], [(col("orders", "o_custkey"), cust)])
        plain = eng.ctx.build_hash(col("customer", "c_custkey"))
        h = eng.plan(w, deferred=True)
        for builds in ([plain], [cust, cust], [9999]):  # not deferred, repeated, unknown
            with pytest.raises(dpf.DpfError) as e:
                eng.ctx.prepare_chain(builds, [h])
            assert e.value.status == -1, builds
        prep = eng.ctx.prepare_chain([cust, bad], [h])
        eng.ctx.launch(prep)
        eng.ctx.read_result(prep, 0)
        eng.ctx.hash_wait(cust)
        with pytest.raises(dpf.DpfError) as e:
            eng.ctx.hash_wait(bad)
        assert e.value.status == -4  # DPF_EDUPKEY
        eng.ctx.release(prep)
        with pytest.raises(dpf.DpfError) as e:
            eng.ctx.prepare_chain([cust, bad], [h])  # the failure is sticky
        assert e.value.status == -1
    finally:
        eng.close()
