"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This package draws random tables and writes down query descriptions.  It
holds none of the method's arithmetic: no encoding, no decoding, no
predicate evaluation, no join and no aggregation.  Both the oracle
(``oracle/``) and the CUDA library's Python binding consume what it returns,
each with its own code.
"""

from .tables import (  # noqa: F401
    ALPHABET,
    batched_workloads,
    bigint_filter_star,
    chain_join,
    date_keys,
    hot_groups,
    scan_filter_aggregate,
    serve_variants,
    star_join,
    strings,
    tiny_chain_workload,
    tiny_random_workload,
)
