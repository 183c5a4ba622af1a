"""The launch-configuration JSON of dpf_set_tuning, parsed on the host
(dpf_parse_tuning: no context, no device)."""

import pytest

import paper_2605_10511_gb300 as dpf

ZERO = {"chunk_rows": 0, "threads": 0, "ht_placement": 0, "ctas_per_sm": 0, "staging": 0, "group_agg": 0}


def test_every_key_by_name_and_by_value():
    got = dpf.parse_tuning('{"chunk_rows": 8192, "threads": 1024, "ctas_per_sm": 1,\n'
                           ' "ht_placement": "global", "staging": "on", "group_agg": "warp"}')
    assert got == {"chunk_rows": 8192, "threads": 1024, "ht_placement": 2, "ctas_per_sm": 1, "staging": 1,
                   "group_agg": 1}
    assert dpf.parse_tuning('{"ht_placement": 1, "staging": 2, "group_agg": 2}') == dict(
        ZERO, ht_placement=1, staging=2, group_agg=2)
    assert dpf.parse_tuning(' { } ') == ZERO


def test_empty_and_null_reset():
    assert dpf.parse_tuning("") == ZERO
    assert dpf.parse_tuning(None) == ZERO


@pytest.mark.parametrize("text", [
    '{"chunk_rows": 1000}',          # not a multiple of 512
    '{"chunk_rows": 33554432}',      # above 2^24
    '{"threads": 300}',
    '{"ctas_per_sm": 33}',
    '{"ht_placement": "fast"}',
    '{"staging": 3}',
    '{"group_agg": "sometimes"}',
    '{"threads": -256}',
    '{"threads": 256.0}',
    '{"chunk": 4096}',               # unknown key
    '{"threads": 256,}',             # trailing comma
    '{"threads" 256}',
    '{"threads": 256',
    '"threads": 256}',
    '{"threads": 256} x',
    '{"threads": {"n": 256}}',
    '{"threads": 99999999999}',
])
def test_bad_objects_are_refused(text):
    with pytest.raises(dpf.DpfError) as e:
        dpf.parse_tuning(text)
    assert e.value.status == -1
