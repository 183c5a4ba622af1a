"""GPU parity of enqueue-only hash builds (Sec. 3.1 Kernels #1 and #2).

``dpf_build_hash_async`` sizes a table from load-time bounds (the key
column's mini block headers and its row count) and only enqueues the
build, so a chain's builds and the fused plan over the last table run back
to back on one stream.  The records must equal the oracle's bit for bit,
the entry counts must equal those of the exactly sized builds, and errors
that only the kernels find (a duplicate key) must come back through
``dpf_hash_wait`` / ``dpf_hash_info`` and keep the table out of later
plans.  Cases: random small chains, the LINEITEM -> ORDERS -> CUSTOMER
workload (direct, open-addressing and rank-directory tables), the star
join, host-resident pages, a plan enqueued before the wait, a capturing
stream, and errors.
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


def _tables(eng, w):
    """Table ids of w's joins, inner tables first."""
    out = []

    def walk(j):
        for s in j.get("joins", []):
            walk(s)
        out.append(eng.hts[(w["name"], repr(j))])
    for j in w["query"]["joins"]:
        walk(j)
    return out


@pytest.mark.parametrize("seed", range(24))
def test_random_small_chains(seed):
    w = synth.tiny_chain_workload(seed)
    eng = dpf.Engine(device=0)
    try:
        assert_same(eng.run(w, asynchronous=True), expect(w), w["name"])
    finally:
        eng.close()


@pytest.mark.parametrize("sparse", [False, True])
def test_chain_matches_oracle_and_exact_builds(sparse):
    """Records equal the oracle's; every table's entry count (known after
    the wait) equals the exactly sized build's."""
    w = synth.chain_join(rows=(1 << 21) + 333, page_rows=65536, sparse_orderkeys=sparse, seed=3)
    a, b = dpf.Engine(device=0), dpf.Engine(device=0)
    try:
        assert_same(a.run(w, asynchronous=True), expect(w), "async")
        assert_same(b.run(w), expect(w), "exact")
        for ta, tb in zip(_tables(a, w), _tables(b, w)):
            ia, ib = a.ctx.hash_info(ta), b.ctx.hash_info(tb)
            assert ia["entries"] == ib["entries"], (ia, ib)
            assert ia["capacity"] >= ib["capacity"], (ia, ib)  # sized from bounds that hold the kept keys
    finally:
        a.close()
        b.close()


def test_star_join():
    w = synth.star_join(rows=(1 << 22) + 17, page_rows=65536, seed=6)
    eng = dpf.Engine(device=0)
    try:
        assert_same(eng.run(w, asynchronous=True), expect(w), "star")
    finally:
        eng.close()


def test_full_size_chain_with_rank_directory():
    """LINEITEM 2^24 rows: ORDERS' keys span more than 2^22, so its table
    is a rank directory sized for every ORDERS row."""
    w = synth.chain_join(rows=1 << 24)
    eng = dpf.Engine(device=0)
    try:
        assert_same(eng.run(w, asynchronous=True), expect(w), "chain 2^24")
        orders = _tables(eng, w)[-1]
        info = eng.ctx.hash_info(orders)
        assert info["capacity"] > 1 << 22, info
    finally:
        eng.close()


def test_host_resident_pages():
    w = synth.chain_join(rows=(1 << 19) + 5, page_rows=16384, seed=8)
    eng = dpf.Engine(device=0)
    try:
        eng.load_workload(w, placement="host")
        assert_same(eng.run(w, asynchronous=True), expect(w), "host")
    finally:
        eng.close()


def test_plans_enqueued_before_the_wait_on_one_stream():
    """Build both tables, prepare and launch the fused plan on one stream
    without any wait in between, read the records, then wait: the stream
    order alone makes the tables ready for the plan."""
    import torch
    w = synth.chain_join(rows=1 << 20, page_rows=32768, seed=9)
    eng = dpf.Engine(device=0)
    try:
        eng.load_workload(w)
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        for rep in range(3):
            for sig in [k for k in eng.hts if k[0] == w["name"]]:
                eng.ctx.drop_hash(eng.hts.pop(sig))
            h = eng.plan(w, s, asynchronous=True)
            prep = eng.ctx.prepare([h])
            try:
                eng.ctx.launch(prep, s)
                got = eng.ctx.read_result(prep, 0)
            finally:
                eng.ctx.release(prep)
            eng.wait_joins(w)
            assert_same(got, expect(w), rep)
    finally:
        eng.close()


def _small_chain(eng):
    w = synth.chain_join(rows=1 << 14, page_rows=4096, seed=12)
    eng.load_workload(w)
    col = lambda t, c: eng.col(w, t, c)  # noqa: E731
    ht_c = eng.ctx.build_hash_async(col("customer", "c_custkey"), [col("customer", "c_nation")])
    return w, col, ht_c


def test_duplicate_key_is_reported_by_the_wait():
    eng = dpf.Engine(device=0)
    try:
        w, col, ht_c = _small_chain(eng)
        eng.ctx.hash_wait(ht_c)
        # o_custkey repeats: the call enqueues, the kernels find the duplicate
        bad = eng.ctx.build_hash_async(col("orders", "o_custkey"), [], [],
                                       [(col("orders", "o_custkey"), ht_c)])
        for _ in range(2):  # reported by the wait, and again afterwards
            with pytest.raises(dpf.DpfError) as e:
                eng.ctx.hash_wait(bad)
            assert e.value.status == -4  # DPF_EDUPKEY
        with pytest.raises(dpf.DpfError) as e:
            eng.ctx.hash_info(bad)
        assert e.value.status == -4
        # a failed table is refused by later builds and plans
        with pytest.raises(dpf.DpfError) as e:
            eng.ctx.build_hash_async(col("lineitem", "l_orderkey"), [], [],
                                     [(col("lineitem", "l_orderkey"), bad)])
        assert e.value.status == -1
        eng.ctx.drop_hash(bad)
        # the context stays usable
        assert eng.ctx.hash_info(ht_c)["entries"] > 0
    finally:
        eng.close()


def test_errors_at_the_call():
    eng = dpf.Engine(device=0)
    try:
        w, col, ht_c = _small_chain(eng)
        bad = [
            dict(payload=[], joins=[(col("orders", "o_custkey"), 9999)]),   # unknown table
            dict(payload=[("join", 1, 0)], joins=[(col("orders", "o_custkey"), ht_c)]),
            dict(payload=[col("orders", "o_orderdate")], joins=[]),        # FOR payload column
        ]
        for i, b in enumerate(bad):
            with pytest.raises(dpf.DpfError) as e:
                eng.ctx.build_hash_async(col("orders", "o_orderkey"), **b)
            assert e.value.status == -1, i
        with pytest.raises(dpf.DpfError) as e:
            eng.ctx.build_hash_async(col("orders", "o_priority"))  # DICT key column
        assert e.value.status == -1
    finally:
        eng.close()


def test_refuses_a_capturing_stream():
    """The call allocates and copies from host memory, so it cannot be
    recorded into a CUDA graph: it fails and enqueues nothing.  (The
    capture is ended without replaying anything.)"""
    import torch
    eng = dpf.Engine(device=0)
    try:
        w, col, ht_c = _small_chain(eng)
        eng.ctx.hash_wait(ht_c)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            g.capture_begin()
            try:
                with pytest.raises(dpf.DpfError) as e:
                    eng.ctx.build_hash_async(col("orders", "o_orderkey"), [], [],
                                             [(col("orders", "o_custkey"), ht_c)], s)
            finally:
                g.capture_end()
        assert e.value.status == -1 and "captur" in str(e.value)
        torch.cuda.synchronize()
        ok = eng.ctx.build_hash_async(col("orders", "o_orderkey"), [], [],
                                      [(col("orders", "o_custkey"), ht_c)])
        eng.ctx.hash_wait(ok)
    finally:
        eng.close()
