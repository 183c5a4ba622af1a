"""Batched launches under the autotuner and the continuous-batching server.

Every result is compared with the oracle (and with the same query run
alone): the launch configuration the tuner picks, the batch a query lands
in, the other queries in flight and admission by memory footprint must not
change any record.
"""

import random
import threading
import time

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


@pytest.fixture(scope="module")
def mix():
    """Small queries of the three shapes over tables of uneven size, plus
    random workloads that touch every operator."""
    ws = synth.batched_workloads(n_queries=12, seed=44, log2_lo=12.0, log2_hi=19.0)
    ws += [synth.tiny_random_workload(s) for s in (2, 3, 7, 11)]
    return ws


@pytest.fixture(scope="module")
def expected(mix):
    return [oracle.run_query(w, from_encoded=False) for w in mix]


def test_autotune_caches_a_grid_point_and_keeps_results(eng, mix, expected):
    for w in mix:
        eng.load_workload(w)
    plans = [eng.plan(w) for w in mix]
    best, ms = eng.ctx.autotune(plans, reps=2)
    assert ms > 0
    assert best["chunk_rows"] in (1024, 2048, 4096, 16384, 65536, 262144)
    assert best["threads"] in (128, 256, 512, 1024)
    assert best["ht_placement"] in (dpf.HT_PLACE["auto"], dpf.HT_PLACE["smem"], dpf.HT_PLACE["global"])
    prep = eng.ctx.prepare(plans)  # tuning fields 0: the cached choice
    try:
        t = eng.ctx.prep_tuning(prep)
        assert (t["chunk_rows"], t["threads"], t["ht_placement"]) == \
            (best["chunk_rows"], best["threads"], best["ht_placement"])
        eng.ctx.launch(prep)
        for i, w in enumerate(mix):
            assert_same(eng.ctx.read_result(prep, i), expected[i], w["name"])
    finally:
        eng.ctx.release(prep)


def test_server_results_equal_alone_and_in_the_mix(eng, mix, expected):
    for w in mix:
        eng.load_workload(w)
    plans = [eng.plan(w) for w in mix]
    alone = [eng.run(w) for w in mix]
    for i, w in enumerate(mix):
        assert_same(alone[i], expected[i], w["name"])
    rng = random.Random(5)
    order = [rng.randrange(len(mix)) for _ in range(120)]
    tickets = [None] * len(order)
    with dpf.Server(eng.ctx, max_batch=8, max_inflight=3) as srv:
        def submitter(part):
            for k in part:
                tickets[k] = srv.submit(plans[order[k]])
                time.sleep(rng.expovariate(4000.0))  # Poisson arrivals, ~4k/s
        idx = list(range(len(order)))
        threads = [threading.Thread(target=submitter, args=(idx[j::2],)) for j in range(2)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        sizes = []
        for k, tk in enumerate(tickets):
            got, times = srv.wait(tk, timeout_ms=60000)
            assert_same(got, alone[order[k]], ("mix", k, mix[order[k]]["name"]))
            assert times["submit_us"] <= times["launch_us"] <= times["done_us"]
            sizes.append(times["batch_size"])
        st = srv.stats()
    assert st["completed"] == len(order) and st["failed"] == 0
    assert max(sizes) > 1, "no two queries shared a launch"


def test_server_admission_by_footprint(eng, mix, expected):
    for w in mix:
        eng.load_workload(w)
    plans = [eng.plan(w) for w in mix]
    foot = [eng.ctx.plan_footprint(p) for p in plans]
    budget = max(foot)  # at most about one query on the device at a time
    with dpf.Server(eng.ctx, max_batch=16, max_inflight=4, mem_budget=budget) as srv:
        tickets = [srv.submit(p) for p in plans]
        for i, tk in enumerate(tickets):
            got, _ = srv.wait(tk, timeout_ms=60000)
            assert_same(got, expected[i], mix[i]["name"])
            assert srv.stats()["in_use_bytes"] <= budget
    with dpf.Server(eng.ctx, mem_budget=min(foot) - 1) as srv:
        with pytest.raises(dpf.DpfError) as e:
            srv.submit(plans[int(np.argmin(foot))])
        assert e.value.status == -5  # DPF_EBUSY


def test_server_wait_errors(eng, mix):
    w = mix[0]
    eng.load_workload(w)
    plan = eng.plan(w)
    with dpf.Server(eng.ctx) as srv:
        with pytest.raises(dpf.DpfError) as e:
            srv.wait(12345, timeout_ms=10)
        assert e.value.status == -8  # DPF_ENOTFOUND
        tk = srv.submit(plan)
        srv.wait(tk, timeout_ms=60000)
        with pytest.raises(dpf.DpfError) as e:
            srv.wait(tk, timeout_ms=10)  # already collected
        assert e.value.status == -8
