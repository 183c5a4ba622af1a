"""GPU parity with the first step staged in shared memory (cp.async ring).

With staging on, the dense first step reads its mini block headers and
packed words from a per-warp shared-memory ring filled one tile (words) and
two tiles (headers) ahead by asynchronous copies, instead of from global
memory.  Every codec a first step can read (FOR, DICT, DELTA; widths 0..32),
partial tiles at page ends, pages skipped by zone maps, both kernel builds,
ticket sizes that cut pages at every tile, the launch's small tail tickets,
batches (staged whole, or not at all when one query has a string first
step): every record must equal the oracle's.
"""

import numpy as np
import pytest

import oracle
import paper_2605_10511_gb300 as dpf
import synth

pytestmark = pytest.mark.gpu

ON = dpf.STAGING["on"]


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
    k = (w["name"], repr(w["query"]))
    if k not in _want:
        _want[k] = oracle.run_query(w, from_encoded=False, threads=0)
    return _want[k]


def _run(eng, w, tuning):
    eng.load_workload(w)
    h = eng.plan(w)
    prep = eng.ctx.prepare([h], tuning)
    try:
        staged = eng.ctx.prep_tuning(prep)["staging"] == ON
        eng.ctx.launch(prep)
        return eng.ctx.read_result(prep, 0), staged
    finally:
        eng.ctx.release(prep)


@pytest.mark.parametrize("seed", range(40))
def test_random_small_workloads_staged(eng, seed):
    w = synth.tiny_random_workload(seed)
    for t in (dpf.Tuning(512, 256, 0, 0, ON), dpf.Tuning(2048, 128, dpf.HT_PLACE["global"], 4, ON)):
        got, _ = _run(eng, w, t)
        assert_same(got, expect(w), (w["name"], t.chunk_rows))


@pytest.mark.parametrize("name", ["scan", "star", "star_unsorted", "star_year", "star_bigint", "chain"])
@pytest.mark.parametrize("ctas", [0, 4])
def test_shapes_staged(eng, name, ctas):
    rows = (1 << 21) + 777
    w = {"scan": lambda: synth.scan_filter_aggregate(rows=rows, page_rows=16384),
         "star": lambda: synth.star_join(rows=rows, clustered=True),
         "star_unsorted": lambda: synth.star_join(rows=rows, clustered=False, page_rows=32768),
         "star_year": lambda: synth.star_join(rows=rows, clustered=True, date_year=1994),
         "star_bigint": lambda: synth.star_join(rows=rows, clustered=True, bigint_measure=True),
         "chain": lambda: synth.chain_join(rows=1 << 20, page_rows=8192)}[name]()
    for chunk in (1536, 4096, 65536):
        got, staged = _run(eng, w, dpf.Tuning(chunk, 256, 0, ctas, ON))
        assert staged, (name, "the first step was expected to be staged")
        assert_same(got, expect(w), (name, chunk, ctas))


def test_full_size_star_staged(eng):
    """The bench's star join (2^26 rows): big tickets, then the launch's
    small tail tickets, staged."""
    w = synth.star_join(rows=1 << 26, clustered=True)
    got, staged = _run(eng, w, dpf.Tuning(4096, 256, 0, 4, ON))
    assert staged
    assert_same(got, expect(w), "star 2^26 staged")


def test_batches_are_staged_whole_or_not_at_all(eng):
    """A launch stages all of its queries or none: a batch of scan and star
    queries is staged; adding a strings query (a string first step) makes
    the whole batch run unstaged.  Both give the oracle's records."""
    ws = [w for w in synth.batched_workloads(n_queries=16, seed=77, log2_lo=14.0, log2_hi=20.0)
          if not w["name"][4:].startswith("strings")][:8]
    for extra, staged in (([], True), ([synth.strings(rows=200_000, page_rows=8192, seed=9)], False)):
        batch = ws + extra
        for w in batch:
            eng.load_workload(w)
        plans = [eng.plan(w) for w in batch]
        prep = eng.ctx.prepare(plans, dpf.Tuning(2048, 256, 0, 0, ON))
        try:
            assert (eng.ctx.prep_tuning(prep)["staging"] == ON) == staged
            eng.ctx.launch(prep)
            for i, w in enumerate(batch):
                assert_same(eng.ctx.read_result(prep, i), expect(w), w["name"])
        finally:
            eng.ctx.release(prep)


def test_host_resident_pages_are_not_staged(eng):
    w = synth.star_join(rows=(1 << 20) + 5, clustered=True)
    w = dict(w, name=w["name"] + "_host_stage")
    eng.load_workload(w, fact_placement="host")
    got, staged = _run(eng, w, dpf.Tuning(4096, 256, 0, 0, ON))
    assert not staged
    assert_same(got, expect(w), "host")
