"""Rank-coded terms in the wide passes of a synchronous probe, against the oracle.

A column whose terms' key intervals (ranges, single values, one per IN value)
have at most 2047 distinct endpoints over the probe is read by rank: a
pre-pass gives every row its rank among those endpoints (by a search tree, or
by a bucket index and a few halvings), and each pass maps it
to the rank among its own endpoints (a byte map, or 16-bit entries past 255
local endpoints) before one mask lookup per group of 32 terms.  Past that
bound the column's ranges alone may be coded (EQ and IN then by hash table in
a second slot of the column), or the column is not coded at all (interval
trees and compares, in the general wide kernel).  Each case here forces one
of these layouts; every count, sample size and marginal must equal the
oracle's."""
import numpy as np
import pytest

from parity import check_probe
from workloads import BLOCKS, EQ, F32, FULL, I32, I64, IN, RANGE, ROWS, Sample, Term

pytestmark = pytest.mark.gpu

SAMPLES = [Sample(FULL), Sample(ROWS, 0.2, 13), Sample(BLOCKS, 0.3, 4, 256)]


@pytest.fixture(scope="module", params=[0, 1, 2], ids=["search_auto", "search_tree", "search_buckets"])
def rctx(g, request):
    """A context that rank-codes batches over tables of any size (the
    default threshold, 2^20 rows, would leave these small tables uncoded),
    with each way of finding a value's rank: per column, by search tree
    only, by bucket index only."""
    ctx = g.gace_create(0, rank_min_rows=1, rank_search=request.param)
    yield ctx
    g.gace_destroy(ctx)


def _run(g, ctx, orc, cols, dtypes, preds, samples=SAMPLES):
    tid = g.gace_load_columns(ctx, cols)
    try:
        check_probe(g, orc, ctx, tid, cols, dtypes, preds, samples)
    finally:
        g.gace_unload(ctx, tid)


def test_ranges_coded_values_hashed(g, rctx, orc):
    """Column 0 has 1100 distinct EQ values (2200 endpoints, past the bound)
    and 60 ranges: its ranges are rank-coded, its EQ and IN terms hashed in a
    second slot; column 1 (int64) is coded with all its terms."""
    rng = np.random.default_rng(41)
    n = 120_001
    c0 = rng.integers(0, 5000, n).astype(np.int32)
    c1 = rng.integers(-300, 300, n).astype(np.int64) * (2**35 + 7)
    preds = [[Term(0, EQ, int(v))] for v in range(0, 4400, 4)]
    for k in range(60):
        a, b = sorted(int(x) for x in rng.integers(-100, 5100, 2))
        preds.append([Term(0, RANGE, a, b + 1 + k % 5)])
    for k in range(40):
        vals = tuple(int(v) * (2**35 + 7) for v in rng.integers(-320, 320, 1 + k % 7))
        preds.append([Term(1, IN, values=vals)])
        a, b = sorted(int(x) for x in rng.integers(-320, 320, 2))
        preds.append([Term(1, RANGE, a * (2**35 + 7), b * (2**35 + 7) + 1)])
    for k in range(30):
        a, b = sorted(int(x) for x in rng.integers(0, 5000, 2))
        preds.append([Term(0, RANGE, a, b + 1), Term(0, EQ, int(rng.integers(0, 4400)) // 4 * 4),
                      Term(1, EQ, int(rng.integers(-300, 300)) * (2**35 + 7))])
    preds.append([Term(0, IN, values=(0, 4, 8, 5001, -3))])
    _run(g, rctx, orc, [c0, c1], [I32, I64], preds)


def test_uncoded_column_trees_and_compares(g, rctx, orc):
    """Column 0 (float32) has 1100 ranges with distinct endpoints (2200, past
    the bound) and some EQ terms: it keeps interval trees, compares and hash
    tables, so its passes take the general wide kernel; column 1 is coded."""
    rng = np.random.default_rng(43)
    n = 100_003
    c0 = (rng.standard_normal(n) * 50).astype(np.float32)
    c0[::89] = np.nan
    c0[::97] = -0.0
    c1 = rng.integers(-2000, 2000, n).astype(np.int32)
    preds = []
    for k in range(1100):
        a, b = sorted(float(x) for x in rng.standard_normal(2) * 60)
        preds.append([Term(0, RANGE, a, b)])
    for x in (0.0, -0.0, float(c0[5]), float(c0[6]), float("nan")):
        preds.append([Term(0, EQ, x)])
    preds.append([Term(0, IN, values=(0.0, float(c0[7]), float(c0[8])))])
    for k in range(50):
        a, b = sorted(int(x) for x in rng.integers(-2100, 2100, 2))
        preds.append([Term(1, RANGE, a, b + 1)])
        preds.append([Term(1, IN, values=tuple(int(v) for v in rng.integers(-2000, 2000, 1 + k % 9)))])
    for k in range(20):
        a, b = sorted(float(x) for x in rng.standard_normal(2) * 40)
        preds.append([Term(0, RANGE, a, b), Term(1, RANGE, -500 + k, 800)])
    _run(g, rctx, orc, [c0, c1], [F32, I32], preds)


def test_wide_local_rank_maps(g, rctx, orc):
    """800 IN terms on one int32 column over 2046 consecutive values (2047
    endpoints, the bound), each in a two-term predicate so that it is
    evaluated in a pass: more terms than one pass holds, so each pass maps
    the column's ranks to several hundred local endpoints (16-bit entries).
    The two halves of the terms draw from disjoint value ranges, so no pass
    holds every endpoint.  Single-term predicates on the same column are
    counted from the rank histograms."""
    rng = np.random.default_rng(47)
    n = 80_021
    c0 = rng.integers(-20, 2070, n).astype(np.int32)
    c1 = rng.integers(0, 100, n).astype(np.int32)
    preds = []
    for k in range(800):
        lo, hi = (0, 1023) if k < 400 else (1023, 2046)
        vals = tuple(int(v) for v in rng.integers(lo, hi, 1 + k % 4))
        preds.append([Term(0, IN, values=vals), Term(1, RANGE, 0, 60 + k % 7)])
    preds += [[Term(0, IN, values=(0, 2045))], [Term(0, EQ, 1022)], [Term(0, EQ, 1023)]]
    for k in range(40):
        preds.append([Term(0, IN, values=(k, 2045 - k)), Term(1, RANGE, k, k + 30)])
    _run(g, rctx, orc, [c0, c1], [I32, I32], preds, [Sample(FULL), Sample(ROWS, 0.25, 3)])


def test_all_terms_coded_every_dtype(g, rctx, orc):
    """Columns of each type coded with all their terms: ranges that touch and
    nest, EQ at both ends of the domain, IN lists sharing values with ranges
    and with each other, float -0/+0 and NaN rows, conjunctions across
    columns."""
    rng = np.random.default_rng(53)
    n = 150_007
    i32 = rng.integers(-300, 300, n).astype(np.int32)
    i32[::1013] = 2**31 - 1
    i32[::1019] = -2**31
    i64 = rng.integers(-300, 300, n).astype(np.int64) * (2**40 + 1)
    i64[::997] = 2**63 - 1
    f32 = rng.choice(np.array([-1.5, -0.0, 0.0, 0.5, 2.0, np.nan, np.inf, -np.inf], dtype=np.float32), n)
    preds = []
    for k in range(100):
        a, b = sorted(int(x) for x in rng.integers(-320, 320, 2))
        preds.append([Term(0, RANGE, a, b + 1)])
        preds.append([Term(0, IN, values=tuple(int(v) for v in rng.integers(-310, 310, 1 + k % 8)))])
        preds.append([Term(1, RANGE, a * (2**40 + 1), (b + 1) * (2**40 + 1))])
        preds.append([Term(1, EQ, int(rng.integers(-300, 300)) * (2**40 + 1))])
    preds += [[Term(0, EQ, 2**31 - 1)], [Term(0, EQ, -2**31)], [Term(0, RANGE, 100, 2**31 - 1)],
              [Term(0, IN, values=(2**31 - 1, -2**31, 0))], [Term(1, EQ, 2**63 - 1)],
              [Term(1, RANGE, 0, 2**63 - 1)], [Term(1, IN, values=(2**63 - 1, 0, -(2**40 + 1)))]]
    for x in (-0.0, 0.0, 0.5, float("inf"), float("-inf"), float("nan")):
        preds.append([Term(2, EQ, x)])
    preds += [[Term(2, RANGE, -0.0, 1.0)], [Term(2, RANGE, float("-inf"), -0.0)],
              [Term(2, IN, values=(-0.0, 2.0, float("nan")))], [Term(2, RANGE, -1.5, float("inf"))]]
    for k in range(40):
        preds.append([Term(0, RANGE, -k, k + 1), Term(1, IN, values=(k * (2**40 + 1), 0)),
                      Term(2, IN, values=(0.5, -1.5))])
    _run(g, rctx, orc, [i32, i64, f32], [I32, I64, F32], preds)


def test_ranks_per_chunk_of_a_streamed_table(g, rctx, orc):
    """A host table registered with its copy deferred to its first probe
    streams in chunks of 2^20 rows (the last ragged): each chunk gets its own
    row-set masks, ranks and histogram counts before its passes."""
    from parity import host_columns
    from workloads import make_predicates, make_skew_corr

    t = make_skew_corr(n=1_200_007, seed=91, device="cpu", domain=50_000)
    host = host_columns(t)
    preds = make_predicates(t, 400, 1, 3, seed=92, in_len=4)
    tid = g.gace_load_columns(rctx, [c.numpy() for c in t.columns], copy_on_first_probe=True)
    try:
        check_probe(g, orc, rctx, tid, host, t.dtypes, preds, [Sample(FULL), Sample(ROWS, 0.05, 8)])
    finally:
        g.gace_unload(rctx, tid)


def test_rank_search_edge_shapes(g, rctx, orc):
    """Columns whose endpoints stress the bucket index: one endpoint only (an
    EQ on the largest int32), 400 ranges crowded into 64 values next to a few
    far apart (a full bucket needs many halvings), int64 endpoints spanning
    the whole domain, and float endpoints on both sides of zero."""
    rng = np.random.default_rng(67)
    n = 100_003
    c0 = rng.integers(2**31 - 4, 2**31, n, dtype=np.int64).astype(np.int32)
    c1 = np.concatenate([rng.integers(1000, 1064, n - 100), rng.integers(-2**31, 2**31 - 1, 100)]).astype(np.int32)
    c2 = (rng.integers(-2**62, 2**62, n, dtype=np.int64) * 2)
    c2[::7] = rng.integers(-50, 50, c2[::7].shape[0])
    c3 = rng.standard_normal(n).astype(np.float32)
    preds = [[Term(0, EQ, 2**31 - 1)] for _ in range(3)]
    for k in range(400):
        a = 1000 + k % 64
        preds.append([Term(1, RANGE, a, a + 1 + (k // 64))])
    preds += [[Term(1, RANGE, -2**31, -2**30)], [Term(1, RANGE, 2**30, 2**31 - 1)], [Term(1, EQ, -2**31)]]
    for k in range(120):
        a = int(rng.integers(-2**61, 2**61)) * 2
        preds.append([Term(2, RANGE, a, a + int(rng.integers(1, 2**61)))])
        preds.append([Term(2, EQ, int(rng.integers(-50, 50)))])
    for k in range(120):
        a = float(rng.standard_normal())
        preds.append([Term(3, RANGE, a, a + float(rng.uniform(1e-4, 2.0)))])
    for k in range(30):
        preds.append([Term(0, EQ, 2**31 - 1), Term(1, RANGE, 1000 + k, 1010 + k), Term(3, RANGE, -0.5, 0.5)])
    _run(g, rctx, orc, [c0, c1, c2, c3], [I32, I32, I64, F32], preds)
