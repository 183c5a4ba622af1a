"""The pins catch plausible mistakes in the oracle (CPU only).

Each case copies ``oracle/dpf_oracle.cpp``, plants one mistake (a flipped
comparison, a dropped term, a transposed operand, a wrong index or bit
order), builds the copy into a temporary library and runs the pins of
``test_oracle_format`` / ``test_oracle_query`` against it.  Every mutant
must fail at least one pin; the unmodified oracle must pass them all.
"""

import os
import subprocess
import tempfile

import numpy as np
import pytest

import npeval
import synth
from _hand_worked import HAND_WORKED

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle", "dpf_oracle.cpp")

MUTANTS = {
    "lt_becomes_le": ("case LT: return x < p.args[0];", "case LT: return x <= p.args[0];"),
    "between_open_top": ("return p.args[0] <= x && x <= p.args[1];",
                         "return p.args[0] <= x && x < p.args[1];"),
    "bit_order_msb_first": ("words[bit / 32] |= 1u << (bit % 32);",
                            "words[bit / 32] |= 1u << (31 - bit % 32);"),
    "for_base_subtracted": ("v = int32_t(uint32_t(base) + f);", "v = int32_t(uint32_t(base) - f);"),
    "delta_drops_dmin": ("running += uint32_t(base) + f;", "running += f;"),
    "sum_sub_transposed": ("case SUM_SUB: add = int64_t(uint64_t(x) - uint64_t(y)); break;",
                           "case SUM_SUB: add = int64_t(uint64_t(y) - uint64_t(x)); break;"),
    "sum_mul_wrong_operand": ("case SUM_MUL: add = int64_t(uint64_t(x) * uint64_t(y)); break;",
                              "case SUM_MUL: add = int64_t(uint64_t(x) * uint64_t(x)); break;"),
    "payload_field_ignored": ("(*hit[keys[k].join])[keys[k].field]", "(*hit[keys[k].join])[0]"),
    "bit_width_one_short": ("while (b < 64 && (span >> b) != 0) ++b;",
                            "while (b < 64 && (span >> b) > 1) ++b;"),
    "prefix_needs_longer_string": ("if (len < uint64_t(p.pfx_len)) return false;",
                                   "if (len <= uint64_t(p.pfx_len)) return false;"),
    "rid_index_search_off_by_one": ("if (row_prefix[mid] > r) hi = mid; else lo = mid + 1;",
                                    "if (row_prefix[mid] >= r) hi = mid; else lo = mid + 1;"),
    "count_doubled": ("g.count += 1;", "g.count += 2;"),
    "empty_ungrouped_dropped": ("if (nkeys == 0 && groups.empty()) groups.emplace",
                                "if (false) groups.emplace"),
    "string_start_ignored": ("uint64_t s = start;", "uint64_t s = 0;"),
    "chain_sub_preds_skipped": ("for (int32_t k = 0; k < J.npreds && ok; ++k) ok = eval_pred(*J.dim, J.preds[k], r);",
                                "for (int32_t k = 0; k < J.npreds && ok && depth == 0; ++k) ok = eval_pred(*J.dim, J.preds[k], r);"),
    "chain_sub_field_ignored": ("(*hit[size_t(J.pay_join[f])])[size_t(J.pay_field[f])]",
                                "(*hit[size_t(J.pay_join[f])])[0]"),
    "chain_payload_always_column": ("J.pay_join[f] < 0 ? J.dim->cols[J.pay_cols[f]].v[r]",
                                    "true ? J.dim->cols[J.pay_cols[f]].v[r]"),
    "chain_probes_own_key": ("auto it = subs[size_t(s)].find(J.dim->cols[J.sub[s].fk_col].v[r]);",
                             "auto it = subs[size_t(s)].find(J.dim->cols[J.key_col].v[r]);"),
    "for64_bits_modulo_32": ("words[bit / 64] |= uint64_t(1) << (bit % 64);",
                             "words[bit / 64] |= uint64_t(1) << (bit % 32);"),
    "for64_word_offset_half": ("woff += 2 * bws[m];", "woff += bws[m];"),
    "dict_rank_off_by_one": ("std::lower_bound(dict.begin(), dict.end(), values[r]) - dict.begin();",
                             "std::upper_bound(dict.begin(), dict.end(), values[r]) - dict.begin();"),
    "threads_merge_drops_counts": ("g.count = int64_t(uint64_t(g.count) + uint64_t(kv.second.count));",
                                   "g.count = int64_t(uint64_t(g.count));"),
    "threads_merge_drops_sums": ("g.val[a] = int64_t(uint64_t(g.val[a]) + uint64_t(kv.second.val[a]));",
                                 "g.val[a] = int64_t(uint64_t(kv.second.val[a]));"),
    "threads_range_end_short": ("r1 = std::min(fact->n, r0 + range_rows);",
                                "r1 = std::min(fact->n, r0 + range_rows - 1);"),
    "threads_last_range_skipped": ("for (uint64_t i = uint64_t(t); i < nranges; i += uint64_t(nthreads)) {",
                                   "for (uint64_t i = uint64_t(t); i + 1 < nranges; i += uint64_t(nthreads)) {"),
    "bigint_predicate_in_32_bits": ("  const int64_t x = ival(c, r);", "  const int64_t x = int32_t(ival(c, r));"),
}


def _pins_pass(o):
    """Runs the pins; returns (passed, first failure message)."""
    try:
        for ex in HAND_WORKED:
            if ex["codec"] == "str":
                data = b"".join(ex["strings"])
                offs = np.zeros(len(ex["strings"]) + 1, np.uint64)
                offs[1:] = np.cumsum([len(s) for s in ex["strings"]])
                col = {"codec": "str", "bytes": np.frombuffer(data, np.uint8).copy(), "offsets": offs}
            else:
                col = {"codec": ex["codec"],
                       "values": np.array(ex["values"], np.int64 if ex["codec"] == "for64" else np.int32)}
            enc = o.encode_column(col, ex["page_rows"])
            assert enc["row_prefix"].tolist() == ex["row_prefix"], ex["name"]
            if "page_hex" in ex:
                assert enc["blob"].tobytes().hex() == ex["page_hex"], ex["name"]
            if ex["codec"] != "str":
                assert o.decode_column(enc).tolist() == list(ex["values"]), ex["name"]
                for r in range(len(ex["values"])):
                    assert o.decode_row(enc, r) == ex["values"][r], ex["name"]
            else:
                d, _ = o.decode_column(enc)
                assert d.tobytes() == b"".join(ex["strings"]), ex["name"]
        for seed in range(40):
            w = synth.tiny_random_workload(seed)
            e = npeval.evaluate(w)
            for from_encoded in (False, True):
                g = o.run_query(w, from_encoded=from_encoded)
                assert g.shape == e.shape, seed
                assert np.array_equal(g["key"], e["key"]), seed
                assert np.array_equal(g["count"], e["count"]), seed
                assert np.array_equal(g["val"], e["val"]), seed
        for seed in range(40):  # the threaded walk over page ranges (3 threads)
            w = synth.tiny_random_workload(seed)
            e = npeval.evaluate(w)
            g = o.run_query(w, from_encoded=False, threads=3)
            assert g.shape == e.shape, ("threads", seed)
            for f in ("key", "count", "val"):
                assert np.array_equal(g[f], e[f]), ("threads", seed, f)
        for seed in range(40):
            w = synth.tiny_chain_workload(seed)
            e = npeval.evaluate(w)
            g = o.run_query(w, from_encoded=bool(seed % 2))
            assert g.shape == e.shape, ("chain", seed)
            for f in ("key", "count", "val"):
                assert np.array_equal(g[f], e[f]), ("chain", seed, f)
        w = synth.strings(rows=3000, seed=5, page_rows=1024)
        w["query"]["preds"] = [{"col": "s", "op": "prefix", "args": [b"a" * 45]}]
        w["query"]["group"] = []
        assert o.run_query(w).shape == (1,)
        w = synth.scan_filter_aggregate(rows=20000, seed=1, page_rows=1024)
        e = npeval.evaluate(w)
        g = o.run_query(w)
        assert np.array_equal(g["val"], e["val"]) and np.array_equal(g["count"], e["count"])
        for preds in ([{"col": "m1", "op": "gt", "args": [1 << 40]}],
                      [{"col": "m1", "op": "between", "args": [3 << 30, 1 << 41]}]):  # BIGINT predicates
            w = synth.bigint_filter_star(5000, 7, 1024, preds=preds, joins=False)
            e = npeval.evaluate(w)
            g = o.run_query(w, from_encoded=True)
            for f in ("key", "count", "val"):
                assert np.array_equal(g[f], e[f]), ("bigint", f)
    except Exception as exc:  # noqa: BLE001 - any failure counts as a caught mutant
        return False, f"{type(exc).__name__}: {exc}"
    return True, ""


def _build_variant(src_text, tmpdir, name):
    path = os.path.join(tmpdir, f"{name}.cpp")
    with open(path, "w") as f:
        f.write(src_text)
    so = os.path.join(tmpdir, f"lib{name}.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", so, path])
    return so


def test_unmodified_oracle_passes_pins(oracle_lib):
    ok, msg = _pins_pass(oracle_lib)
    assert ok, msg


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(oracle_lib, name):
    old, new = MUTANTS[name]
    src = open(ORACLE_SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    with tempfile.TemporaryDirectory() as tmp:
        so = _build_variant(src.replace(old, new), tmp, name)
        with oracle_lib.use_library(so):
            ok, _ = _pins_pass(oracle_lib)
    assert not ok, f"mutant {name} survived every pin"
