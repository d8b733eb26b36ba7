"""GPU parity of the fused predicate-batch probe (K1) against the CPU oracle:
bit-exact counts, sample sizes and marginals; selectivities and PCS within
1e-12 relative."""
import itertools

import numpy as np
import pytest
import torch

from golden_io import load_tiny_probe
from parity import check_probe, host_columns
from workloads import (BLOCKS, EQ, F32, FULL, I32, I64, IN, RANGE, ROWS, Sample, Table, Term,
                       make_plain_small, make_predicates, make_skew_corr)

pytestmark = pytest.mark.gpu

SAMPLES = [Sample(FULL), Sample(ROWS, 0.01, 42), Sample(ROWS, 0.1, 42), Sample(BLOCKS, 0.01, 42, 4096),
           Sample(BLOCKS, 0.05, 7, 100)]


def test_hand_counted_fixture(g, gctx, orc):
    arrays, dtypes, preds, expect = load_tiny_probe()
    tid = g.gace_load_columns(gctx, arrays)
    try:
        res, marg = check_probe(g, orc, gctx, tid, arrays, dtypes, preds, [Sample(FULL)])
        assert [int(x) for x in res["match"][0]] == [e["count"] for e in expect]
        for p, e in enumerate(expect):
            if "pcs" in e:
                assert float(res["pcs"][0][p]) == float(e["pcs"])
    finally:
        g.gace_unload(gctx, tid)


@pytest.mark.parametrize("n", [0, 1, 3, 31, 33, 127, 129, 1023, 1025, 4095, 4097, 8193, 65537, 100003])
def test_plain_small_shapes(g, gctx, orc, cuda, n):
    """Plain-probe table at sizes that cover empty, sub-slice, sub-tile,
    several tiles and ragged tails."""
    t = make_plain_small(n=n, seed=100 + n, device=cuda)
    preds = make_predicates(t, 64, 1, 3, seed=n) if n else [[Term(0, RANGE, 0, 10)], [Term(1, EQ, 0)], []]
    tid = g.gace_load_columns(gctx, t.columns)
    try:
        check_probe(g, orc, gctx, tid, host_columns(t), t.dtypes, preds, SAMPLES)
    finally:
        g.gace_unload(gctx, tid)


def test_plain_small_full_size(g, gctx, orc, cuda):
    """1M rows x 4 int32 columns, 64 predicates of 1-3 terms, full scan and a
    1 % row sample with seed 42."""
    t = make_plain_small(n=1_000_000, seed=1001, device=cuda)
    preds = make_predicates(t, 64, 1, 3, seed=2001)
    tid = g.gace_load_columns(gctx, t.columns)
    try:
        check_probe(g, orc, gctx, tid, host_columns(t), t.dtypes, preds,
                    [Sample(FULL), Sample(ROWS, 0.01, 42)])
    finally:
        g.gace_unload(gctx, tid)


def test_mixed_dtypes_wide_batch(g, gctx, orc, cuda):
    """Skew + correlation table shape (int32, int64, float32 columns) with a
    1024-predicate batch of 1-4 terms: several passes, five row sets, PCS."""
    t = make_skew_corr(n=200_003, seed=1002, device=cuda)
    preds = make_predicates(t, 1024, 1, 4, seed=2002)
    tid = g.gace_load_columns(gctx, t.columns)
    try:
        check_probe(g, orc, gctx, tid, host_columns(t), t.dtypes, preds, SAMPLES)
    finally:
        g.gace_unload(gctx, tid)


def test_more_predicates_than_one_pass(g, gctx, orc, cuda):
    t = make_skew_corr(n=50_000, seed=5, device=cuda, domain=50_000)
    preds = make_predicates(t, 1500, 1, 4, seed=6, in_len=16)
    tid = g.gace_load_columns(gctx, t.columns)
    try:
        check_probe(g, orc, gctx, tid, host_columns(t), t.dtypes, preds, [Sample(FULL), Sample(ROWS, 0.3, 1)])
    finally:
        g.gace_unload(gctx, tid)


def test_float_specials(g, gctx, orc):
    specials = [float("-inf"), -1.5, -0.0, 0.0, 1.5, float("nan"), float("inf"), 1e-45, 3.4e38, 2.0, -2.5]
    col = np.array(specials * 37, dtype=np.float32)
    consts = [float("-inf"), -1.5, -0.0, 0.0, 1.5, float("inf"), float("nan"), 1e-46, 1e300, 0.1,
              3.4028235677973366e38, 1.401298464324817e-45]
    terms = []
    for a in consts:
        terms.append(Term(0, EQ, a))
        for b in consts:
            terms.append(Term(0, RANGE, a, b))
    terms += [Term(0, IN, values=(0.0, float("nan"), 1.5, 0.1)), Term(0, IN, values=(-0.0,)),
              Term(0, IN, values=(float("inf"), -2.5, 2.0, 2.0))]
    preds = [[x] for x in terms] + [[terms[3], terms[40]], [terms[-1], terms[-3]]]
    tid = g.gace_load_columns(gctx, [col])
    try:
        check_probe(g, orc, gctx, tid, [col], [F32], preds, [Sample(FULL), Sample(ROWS, 0.5, 3)])
    finally:
        g.gace_unload(gctx, tid)


def test_integer_extremes(g, gctx, orc):
    rng = np.random.default_rng(1)
    i32 = np.array([-2**31, 2**31 - 1, 0, -1, 1, 5, -7] * 300, dtype=np.int32)
    i64 = np.array([-2**63, 2**63 - 1, 0, -1, 1, 2**40, -2**40] * 300, dtype=np.int64)
    rng.shuffle(i32)
    rng.shuffle(i64)
    big = [-2**63, -2**31 - 1, -2**31, -1, 0, 1, 2**31 - 1, 2**31, 2**40, 2**63 - 1]
    terms = []
    for c in (0, 1):
        for a in big:
            terms.append(Term(c, EQ, a))
            for b in big:
                terms.append(Term(c, RANGE, a, b))
        terms.append(Term(c, IN, values=(2**31 - 1, -2**31, 2**40, 7)))
        terms.append(Term(c, IN, values=(2**63 - 1, -2**63, 2**40, -2**40, 5, 5)))
    preds = [[x] for x in terms] + [[terms[1], terms[130]], [terms[5], terms[200], terms[-1]]]
    tid = g.gace_load_columns(gctx, [i32, i64])
    try:
        check_probe(g, orc, gctx, tid, [i32, i64], [I32, I64], preds, [Sample(FULL), Sample(BLOCKS, 0.5, 9, 64)])
    finally:
        g.gace_unload(gctx, tid)


def test_degenerate_predicates(g, gctx, orc, cuda):
    t = make_plain_small(n=70_001, seed=11, device=cuda)
    preds = [
        [], [Term(0, RANGE, 5, 5)], [Term(0, RANGE, 10, 0)], [Term(1, EQ, 2**40)],
        [Term(1, IN, values=(3, 3, 3))], [Term(1, IN, values=(2**40, -2**40))],
        [Term(1, EQ, 0), Term(1, EQ, 0)], [Term(1, EQ, 0), Term(1, EQ, 1)],
        [Term(1, RANGE, 0, 10), Term(1, IN, values=(3, 12, 9))],
        [Term(0, RANGE, -2**63, 2**63 - 1)], [Term(2, RANGE, 0, 100), Term(3, EQ, 5)],
        [Term(3, EQ, 5), Term(2, RANGE, 0, 100)],
    ]
    samples = [Sample(FULL), Sample(ROWS, 0.0, 1), Sample(ROWS, 1.0, 1), Sample(ROWS, -3.0, 1),
               Sample(BLOCKS, 7.0, 1, 5), Sample(BLOCKS, 0.5, 3, 1), Sample(ROWS, 0.5, 3), Sample(BLOCKS, 0.2, 3, 3)]
    tid = g.gace_load_columns(gctx, t.columns)
    try:
        res, _ = check_probe(g, orc, gctx, tid, host_columns(t), t.dtypes, preds, samples)
        # a block of one row is the row sample with the same seed and rate
        assert np.array_equal(res["match"][5], res["match"][6])
    finally:
        g.gace_unload(gctx, tid)


def test_nested_samples(g, gctx, cuda):
    t = make_plain_small(n=300_000, seed=13, device=cuda)
    preds = make_predicates(t, 32, 1, 2, seed=14)
    tid = g.gace_load_columns(gctx, t.columns)
    try:
        rates = [0.001, 0.01, 0.1, 0.5]
        res, _ = g.gace_probe_batch(gctx, tid, preds, [Sample(ROWS, r, 42) for r in rates], t.dtypes)
        for a, b in zip(rates, rates[1:]):
            i, j = rates.index(a), rates.index(b)
            assert (res["match"][i] <= res["match"][j]).all()
            assert res["sample_rows"][i][0] <= res["sample_rows"][j][0]
    finally:
        g.gace_unload(gctx, tid)


def test_misaligned_borrowed_columns(g, gctx, orc, cuda):
    """Columns whose base is not 16-byte aligned take the plain-load path and
    give the same counts; borrowed and copied tables agree."""
    t = make_skew_corr(n=40_001, seed=21, device=cuda, domain=10_000)
    shifted = []
    for c in t.columns:
        buf = torch.empty(c.numel() + 1, dtype=c.dtype, device=cuda)
        buf[1:] = c
        shifted.append(buf[1:])
    assert shifted[0].data_ptr() % 16 != 0
    preds = make_predicates(t, 200, 1, 4, seed=22)
    tid = g.gace_load_columns(gctx, shifted, borrow=True)
    tid2 = g.gace_load_columns(gctx, t.columns, borrow=True)
    try:
        r1, _ = check_probe(g, orc, gctx, tid, host_columns(t), t.dtypes, preds, SAMPLES[:3])
        r2, _ = g.gace_probe_batch(gctx, tid2, preds, SAMPLES[:3], t.dtypes)
        assert np.array_equal(r1["match"], r2["match"])
    finally:
        g.gace_unload(gctx, tid)
        g.gace_unload(gctx, tid2)


def test_host_loaded_table_equals_device_loaded(g, gctx, cuda):
    t = make_plain_small(n=12_345, seed=31, device=cuda)
    preds = make_predicates(t, 16, 1, 3, seed=32)
    a = g.gace_load_columns(gctx, t.columns)
    b = g.gace_load_columns(gctx, [c.cpu().numpy() for c in t.columns])
    try:
        ra, _ = g.gace_probe_batch(gctx, a, preds, SAMPLES, t.dtypes)
        rb, _ = g.gace_probe_batch(gctx, b, preds, SAMPLES, t.dtypes)
        for f in ("match", "sample_rows", "sel"):
            assert np.array_equal(ra[f], rb[f])
        assert np.array_equal(ra["pcs"], rb["pcs"], equal_nan=True)
    finally:
        g.gace_unload(gctx, a)
        g.gace_unload(gctx, b)


def test_errors_are_status_codes(g, gctx, cuda):
    t = make_plain_small(n=1000, seed=1, device=cuda)
    tid = g.gace_load_columns(gctx, t.columns)
    try:
        with pytest.raises(g.GaceError) as e:
            g.gace_probe_batch(gctx, tid, [[Term(9, EQ, 1)]], [Sample(FULL)], t.dtypes)
        assert e.value.status == 1
        with pytest.raises(g.GaceError) as e:
            g.gace_probe_batch(gctx, 999, [[Term(0, EQ, 1)]], [Sample(FULL)], t.dtypes)
        assert e.value.status == 6
        with pytest.raises(g.GaceError) as e:
            g.gace_probe_batch(gctx, tid, [[Term(0, EQ, 1)]], [], t.dtypes)
        assert e.value.status == 1
        with pytest.raises(g.GaceError) as e:
            g.gace_probe_batch(gctx, tid, [[Term(0, EQ, 1)]], [Sample(ROWS, float("nan"), 1)], t.dtypes)
        assert e.value.status == 1
        with pytest.raises(g.GaceError) as e:
            g.gace_probe_batch(gctx, tid, [[Term(0, IN, values=())]], [Sample(FULL)], t.dtypes)
        assert e.value.status == 1
        with pytest.raises(g.GaceError) as e:
            g.gace_unload(gctx, 12345)
        assert e.value.status == 6
    finally:
        g.gace_unload(gctx, tid)


def test_hbm_budget_refuses_table(g, cuda):
    ctx = g.gace_create(0, hbm_budget_bytes=1 << 20)
    try:
        small = torch.zeros(1000, dtype=torch.int32, device=cuda)
        g.gace_load_columns(ctx, [small])
        with pytest.raises(g.GaceError) as e:
            g.gace_load_columns(ctx, [torch.zeros(1 << 20, dtype=torch.int32, device=cuda)])
        assert e.value.status == 2
        # borrowed tables cost the context nothing
        g.gace_load_columns(ctx, [torch.zeros(1 << 20, dtype=torch.int32, device=cuda)], borrow=True)
    finally:
        g.gace_destroy(ctx)


def test_single_predicate_kernel_shapes(g, gctx, orc, cuda):
    """One predicate on one row set (the single-predicate kernel): every
    dtype, IN lists, hashed samples, marginals for PCS, ragged tails, and a
    batch whose marginal-only terms must not join the predicate."""
    for n in (1, 255, 257, 4097, 300_001):
        t = make_skew_corr(n=n, seed=60 + n % 97, device=cuda, domain=1000)
        tid = g.gace_load_columns(gctx, t.columns)
        host = host_columns(t)
        try:
            cases = [
                [Term(0, RANGE, 0, 30)], [Term(4, IN, values=(0, 1, 5, 9))], [Term(6, RANGE, -0.5, 0.5)],
                [Term(0, RANGE, 0, 30), Term(1, EQ, 0)], [Term(2, IN, values=(0, 3)), Term(5, RANGE, 0, 7),
                                                          Term(7, RANGE, 0.0, 2.0)],
            ]
            for pred in cases:
                for smp in (Sample(FULL), Sample(ROWS, 0.05, 42), Sample(BLOCKS, 0.2, 9, 512),
                            Sample(BLOCKS, 0.3, 9, 3)):
                    check_probe(g, orc, gctx, tid, host, t.dtypes, [pred], [smp])
            # an always-false predicate leaves marginal-only terms in the pass
            check_probe(g, orc, gctx, tid, host, t.dtypes,
                        [[Term(0, RANGE, 0, 30)], [Term(1, EQ, 0), Term(3, EQ, 2**40)]], [Sample(FULL)])
        finally:
            g.gace_unload(gctx, tid)


def test_wide_pass_value_tables(g, gctx, orc, cuda):
    """Wide passes look EQ and IN terms up in per-column hash tables: many
    groups of 32 terms on one column, int64 keys, float -0/+0/NaN, values
    shared by several terms, and values absent from the column."""
    rng = np.random.default_rng(3)
    n = 100_003
    i32 = rng.integers(-50, 50, n).astype(np.int32)
    i64 = (rng.integers(-40, 40, n).astype(np.int64) * (2**33 + 1))
    f32 = rng.choice(np.array([0.0, -0.0, 1.5, -2.25, np.nan, np.inf, 3.0], dtype=np.float32), n)
    cols = [i32, i64, f32]
    preds = []
    for v in range(-60, 60):
        preds.append([Term(0, EQ, v)])
    for k in range(40):
        vals = tuple(int(x) for x in rng.integers(-55, 55, 1 + k % 9))
        preds.append([Term(0, IN, values=vals)])
    for v in range(-45, 45, 2):
        preds.append([Term(1, EQ, v * (2**33 + 1))])
        preds.append([Term(1, IN, values=(v * (2**33 + 1), (v + 1) * (2**33 + 1), 7))])
    for x in (0.0, -0.0, 1.5, -2.25, float("nan"), float("inf"), 2.0):
        preds.append([Term(2, EQ, x)])
    preds.append([Term(2, IN, values=(-0.0, 3.0, float("nan")))])
    preds.append([Term(0, EQ, 3), Term(1, IN, values=(0, 2**33 + 1)), Term(2, EQ, 0.0)])
    preds.append([Term(0, RANGE, -10, 10), Term(0, IN, values=(1, 2, 3, 99))])
    tid = g.gace_load_columns(gctx, cols)
    try:
        check_probe(g, orc, gctx, tid, cols, [I32, I64, F32], preds,
                    [Sample(FULL), Sample(ROWS, 0.4, 5), Sample(BLOCKS, 0.5, 5, 128)])
    finally:
        g.gace_unload(gctx, tid)


def test_wide_pass_range_trees(g, gctx, orc, cuda):
    """Wide passes evaluate range terms by per-column interval trees of 32
    terms: more than 32 overlapping ranges per column (several trees), nested,
    shared and touching endpoints, unbounded ones, on int32, int64 and float32
    columns, alone and in conjunctions."""
    rng = np.random.default_rng(17)
    n = 100_003
    i32 = rng.integers(-1000, 1000, n).astype(np.int32)
    i64 = rng.integers(-1000, 1000, n).astype(np.int64) * (2**34 + 3)
    f32 = (rng.standard_normal(n) * 10).astype(np.float32)
    f32[::97] = np.nan
    f32[::101] = -0.0
    cols = [i32, i64, f32]
    preds = []
    for k in range(80):
        a, b = sorted(int(x) for x in rng.integers(-1100, 1100, 2))
        preds.append([Term(0, RANGE, a, b + (k % 3))])
    preds += [[Term(0, RANGE, -2**31, 0)], [Term(0, RANGE, 0, 2**31 - 1)], [Term(0, RANGE, -5, 5)],
              [Term(0, RANGE, 5, 15)], [Term(0, RANGE, -5, 15)], [Term(0, RANGE, 10, 3)]]
    for k in range(40):
        a, b = sorted(int(x) for x in rng.integers(-1100, 1100, 2))
        preds.append([Term(1, RANGE, a * (2**34 + 3), b * (2**34 + 3) + k)])
    preds += [[Term(1, RANGE, -2**63, 0)], [Term(1, RANGE, 1, 2**63 - 1)]]
    for k in range(40):
        a, b = sorted(float(x) for x in rng.standard_normal(2) * 12)
        preds.append([Term(2, RANGE, a, b)])
    preds += [[Term(2, RANGE, float("-inf"), 0.0)], [Term(2, RANGE, -0.0, float("inf"))],
              [Term(2, RANGE, 0.0, 1e-30)], [Term(2, RANGE, float("-inf"), float("inf"))]]
    for k in range(30):
        a, b = sorted(int(x) for x in rng.integers(-1000, 1000, 2))
        c, d = sorted(float(x) for x in rng.standard_normal(2) * 10)
        preds.append([Term(0, RANGE, a, b), Term(2, RANGE, c, d)])
    tid = g.gace_load_columns(gctx, cols)
    try:
        check_probe(g, orc, gctx, tid, cols, [I32, I64, F32], preds,
                    [Sample(FULL), Sample(ROWS, 0.3, 11), Sample(BLOCKS, 0.5, 2, 1000)])
    finally:
        g.gace_unload(gctx, tid)


@pytest.mark.parametrize("samples", [
    [Sample(BLOCKS, 0.01, 42, 4096)],
    [Sample(BLOCKS, 0.05, 7, 3000)],
    [Sample(BLOCKS, 0.02, 1, 65536), Sample(BLOCKS, 0.3, 9, 8192)],
    [Sample(BLOCKS, 0.01, 5, 1000)],
    [Sample(BLOCKS, 0.001, 3, 2048), Sample(BLOCKS, 0.0, 3, 2048)],
])
@pytest.mark.parametrize("npreds", [1, 3])
def test_block_samples_skip_tiles(g, gctx, orc, cuda, samples, npreds):
    """Probes whose row sets are all block samples read only the tiles that
    hold a sampled block: counts, sample sizes and marginals still equal the
    oracle's over int32 and int64 columns, several thousand tiles and a ragged
    tail (block sizes that are and are not powers of two, several sets, a
    block size too small for skipping, an empty sample)."""
    t = make_skew_corr(n=3_000_777, seed=77, device=cuda)
    for cols in ([0, 2], [4, 5]):
        sub = Table(t.name, [t.columns[c] for c in cols], [t.dtypes[c] for c in cols], [t.domains[c] for c in cols])
        preds = make_predicates(sub, npreds, 1, 2, seed=npreds)
        preds = [[Term(cols[x.col], x.op, x.a, x.b, x.values) for x in p] for p in preds]
        tid = g.gace_load_columns(gctx, t.columns, borrow=True)
        try:
            check_probe(g, orc, gctx, tid, host_columns(t), t.dtypes, preds, samples)
        finally:
            g.gace_unload(gctx, tid)


@pytest.mark.parametrize("n", [1000, 65537, 1_000_003])
def test_single_predicate_sparse_row_samples(g, gctx, orc, cuda, n):
    """One predicate of 1-4 terms over int32, int64 and float32 columns on one
    sparse row sample (the single-predicate evaluation with per-row hashing):
    counts, sample sizes and marginals equal the oracle's at every rate, on
    ragged tails."""
    rng = np.random.default_rng(n)
    c0 = rng.integers(-1000, 1000, n).astype(np.int32)
    c1 = rng.integers(-2**40, 2**40, n).astype(np.int64)
    c2 = rng.standard_normal(n).astype(np.float32)
    c3 = rng.integers(0, 50, n).astype(np.int32)
    cols, dtypes = [c0, c1, c2, c3], [I32, I64, F32, I32]
    terms = [Term(0, RANGE, -300, 400), Term(1, RANGE, -2**39, 2**39), Term(2, RANGE, -1.0, 0.5),
             Term(3, IN, values=(1, 3, 5, 7, 11, 13)), Term(0, EQ, 17)]
    tid = g.gace_load_columns(gctx, [torch.as_tensor(c, device=cuda) for c in cols])
    try:
        for k, pred in enumerate([terms[:1], terms[1:2], terms[2:3], terms[:4], [terms[4]], [terms[1], terms[3]]]):
            for rate in (0.001, 0.01, 1 / 32, 0.05):
                check_probe(g, orc, gctx, tid, cols, dtypes, [pred], [Sample(ROWS, rate, 7 + k)])
    finally:
        g.gace_unload(gctx, tid)
