"""Pins of the CPU oracle against facts that do not come from the oracle itself:
published hash outputs, hand counts, brute force over every tiny table, closed
forms, set-algebra identities, and the HyperLogLog error bound."""
import itertools
import math

import numpy as np
import pytest

from golden_io import load_splitmix_vectors, load_tiny_probe
from workloads import (BLOCKS, EQ, F32, FULL, I32, I64, IN, RANGE, ROWS, JoinSide, Sample,
                       Table, Term, make_plain_small, make_predicates)

M64 = (1 << 64) - 1


# ----------------------------------------------------------------- hashing

def test_splitmix64_published_outputs(orc):
    for state, out in load_splitmix_vectors():
        # the generator adds the increment before mixing; the oracle's
        # splitmix64(x) takes the state before that increment
        assert orc.splitmix64(state) == out


def test_seeded_hash_composition(orc):
    for x, s in [(0, 0), (1, 42), (123456789, 7), (M64, M64), (1 << 40, 3)]:
        assert orc.hash64(x, s) == orc.splitmix64(x ^ orc.splitmix64(s))


# ----------------------------------------------------------------- sampling

def test_threshold_closed_forms(orc):
    assert orc.threshold(0.0) == (0, 0)
    assert orc.threshold(-1.0) == (0, 0)
    assert orc.threshold(float("nan"))[0] == 0
    assert orc.threshold(1.0)[0] == 1
    assert orc.threshold(2.5)[0] == 1
    assert orc.threshold(0.5) == (2, 1 << 63)
    assert orc.threshold(0.25) == (2, 1 << 62)
    assert orc.threshold(2.0 ** -64) == (2, 1)
    assert orc.threshold(math.nextafter(1.0, 0.0)) == (2, (1 << 64) - (1 << 11))
    assert orc.threshold(0.01) == (2, int(0.01 * 2.0 ** 64))


def _small_table(n=20000, seed=5):
    return make_plain_small(n=n, seed=seed, device="cpu")


def test_rate_one_equals_full_and_rate_zero_is_empty(orc):
    t = _small_table()
    preds = make_predicates(t, 24, 1, 3, seed=11)
    full = orc.probe(t.columns, t.dtypes, preds, Sample(FULL))
    for kind in (ROWS, BLOCKS):
        one = orc.probe(t.columns, t.dtypes, preds, Sample(kind, 1.0, 42, 64))
        assert one.n_sample == t.nrows
        assert np.array_equal(one.counts, full.counts)
        zero = orc.probe(t.columns, t.dtypes, preds, Sample(kind, 0.0, 42, 64))
        assert zero.n_sample == 0 and not zero.counts.any()


def test_samples_are_nested_in_rate(orc):
    s1, s2 = Sample(ROWS, 0.01, 42), Sample(ROWS, 0.1, 42)
    for row in range(0, 50000, 7):
        if orc.row_in_sample(s1, row):
            assert orc.row_in_sample(s2, row)
    b1, b2 = Sample(BLOCKS, 0.05, 9, 100), Sample(BLOCKS, 0.3, 9, 100)
    for row in range(0, 100000, 37):
        if orc.row_in_sample(b1, row):
            assert orc.row_in_sample(b2, row)


def test_row_sample_size_is_binomial(orc):
    n = 200000
    t = Table("u", [np.zeros(n, dtype=np.int32)], [I32], [1])
    for rate in (0.001, 0.01, 0.1, 0.5):
        for seed in range(4):
            r = orc.probe(t.columns, t.dtypes, [[]], Sample(ROWS, rate, seed))
            z = (r.n_sample - n * rate) / math.sqrt(n * rate * (1 - rate))
            assert abs(z) < 5.0, (rate, seed, r.n_sample)


def test_block_sample_keeps_whole_blocks(orc):
    n, b = 10007, 64  # ragged last block
    s = Sample(BLOCKS, 0.3, 17, b)
    kept_blocks = set()
    for row in range(n):
        k = orc.row_in_sample(s, row)
        blk = row // b
        if row % b == 0:
            first = k
            if k:
                kept_blocks.add(blk)
        assert k == first
    t = Table("u", [np.zeros(n, dtype=np.int32)], [I32], [1])
    r = orc.probe(t.columns, t.dtypes, [[]], s)
    expect = sum(min(n, (blk + 1) * b) - blk * b for blk in kept_blocks)
    assert r.n_sample == expect
    assert 0 < len(kept_blocks) < (n + b - 1) // b


def test_block_of_one_row_equals_row_sample(orc):
    t = _small_table(5000, 3)
    preds = make_predicates(t, 16, 1, 3, seed=4)
    a = orc.probe(t.columns, t.dtypes, preds, Sample(ROWS, 0.2, 99))
    b = orc.probe(t.columns, t.dtypes, preds, Sample(BLOCKS, 0.2, 99, 1))
    assert a.n_sample == b.n_sample and np.array_equal(a.counts, b.counts)


def test_seed_changes_sample(orc):
    s1, s2 = Sample(ROWS, 0.5, 1), Sample(ROWS, 0.5, 2)
    diff = sum(orc.row_in_sample(s1, r) != orc.row_in_sample(s2, r) for r in range(2000))
    assert 800 < diff < 1200


# ----------------------------------------------------------------- term evaluation

def test_hand_counted_golden_probe(orc):
    arrays, dtypes, preds, expect = load_tiny_probe()
    r = orc.probe(arrays, dtypes, preds, Sample(FULL))
    assert r.n_sample == 8
    off = 0
    for k, (p, e) in enumerate(zip(preds, expect)):
        assert int(r.counts[k]) == e["count"], e
        if "marginals" in e:
            assert [int(x) for x in r.marginals[off:off + len(p)]] == e["marginals"]
            c_a, c_b = e["marginals"]
            assert orc.pcs(int(r.counts[k]), c_a, c_b, 8) == float(e["pcs"])
        off += len(p)


def _naive_rows(rows, term, isf):
    """Second formulation: the set of row ids where a term holds."""
    out = set()
    for i, row in enumerate(rows):
        x = row[term.col]
        if term.op == EQ:
            ok = x == term.a
        elif term.op == RANGE:
            ok = term.a <= x < term.b
        else:
            ok = any(x == v for v in term.values)
        if ok:
            out.add(i)
    return out


def _all_terms_int(ncols, vals):
    terms = []
    for c in range(ncols):
        for v in vals + [max(vals) + 1, -1]:
            terms.append(Term(c, EQ, v))
        lim = [min(vals) - 1] + vals + [max(vals) + 1]
        for lo, hi in itertools.product(lim, lim):
            terms.append(Term(c, RANGE, lo, hi))
        for k in (1, 2, 3):
            for sub in itertools.combinations(vals, k):
                terms.append(Term(c, IN, values=sub))
        terms.append(Term(c, IN, values=(vals[0], vals[0])))
    return terms


def test_brute_force_every_tiny_int_table(orc):
    """Every table of up to 3 rows over an int32 and an int64 column with
    values in {0,1,2}: each single term and each two-column conjunction
    against a set-intersection count."""
    vals = [0, 1, 2]
    terms = _all_terms_int(2, vals)
    t0 = [t for t in terms if t.col == 0]
    t1 = [t for t in terms if t.col == 1]
    rng = np.random.default_rng(0)
    pairs = [[t0[i], t1[j]] for i, j in zip(rng.integers(0, len(t0), 60), rng.integers(0, len(t1), 60))]
    preds = [[t] for t in terms] + pairs + [[]]
    checked = 0
    for n in range(0, 4):
        for cells in itertools.product(vals, repeat=2 * n):
            rows = [(cells[2 * i], cells[2 * i + 1]) for i in range(n)]
            cols = [np.array([r[0] for r in rows], dtype=np.int32),
                    np.array([r[1] for r in rows], dtype=np.int64)]
            r = orc.probe(cols, [I32, I64], preds, Sample(FULL), nrows=n)
            for k, p in enumerate(preds):
                s = set(range(n))
                for t in p:
                    s &= _naive_rows(rows, t, False)
                assert int(r.counts[k]) == len(s), (rows, p)
            checked += 1
    assert checked == 1 + 9 + 81 + 729


def test_brute_force_float_specials(orc):
    specials = [float("-inf"), -1.5, -0.0, 0.0, 1.5, float("nan"), float("inf"), 1e-45, 3.4e38]
    consts = [float("-inf"), -1.5, -0.0, 0.0, 1.5, float("inf"), float("nan"), 1e-46, 1e300, 0.1]
    terms = []
    for a in consts:
        terms.append(Term(0, EQ, a))
        for b in consts:
            terms.append(Term(0, RANGE, a, b))
    terms.append(Term(0, IN, values=(0.0, float("nan"), 1.5, 0.1)))
    terms.append(Term(0, IN, values=(-0.0,)))
    col = np.array(specials, dtype=np.float32)
    rows = [(float(x),) for x in col]
    preds = [[t] for t in terms]
    r = orc.probe([col], [F32], preds, Sample(FULL))
    for k, p in enumerate(preds):
        assert int(r.counts[k]) == len(_naive_rows(rows, p[0], True)), p


def test_count_identities(orc):
    t = _small_table(30000, 8)
    n = t.nrows
    preds = [
        [Term(0, RANGE, 1000, 400000)], [Term(0, RANGE, 1000, 123456)], [Term(0, RANGE, 123456, 400000)],
        [Term(1, IN, values=(0, 1, 5, 5, 17))], [Term(1, EQ, 0)], [Term(1, EQ, 1)], [Term(1, EQ, 5)],
        [Term(1, EQ, 17)], [], [Term(3, RANGE, 0, 100)],
        [Term(1, RANGE, 0, 50), Term(3, RANGE, 10, 60), Term(0, RANGE, 0, 900000)],
    ]
    r = orc.probe(t.columns, t.dtypes, preds, Sample(FULL))
    c = [int(x) for x in r.counts]
    assert c[0] == c[1] + c[2]                     # RANGE split at an interior point
    assert c[3] == c[4] + c[5] + c[6] + c[7]       # IN is the sum of EQ over distinct values
    assert c[8] == n                               # empty conjunction matches every row
    assert c[9] == n                               # c3 lies in [0, 100)
    m = [int(x) for x in r.marginals]
    assert c[10] <= min(m[-3:])                    # conjunction <= each marginal
    for k in range(8):                             # single-term predicate equals its marginal
        if len(preds[k]) == 1:
            idx = sum(len(p) for p in preds[:k])
            assert m[idx] == c[k]


# ----------------------------------------------------------------- PCS

def test_pcs_closed_form_for_nested_conditions(orc):
    t = _small_table(50000, 2)
    n = t.nrows
    a, b = Term(1, RANGE, 100, 200), Term(2, RANGE, 700, 1450)  # c2 = 7 c1 + [0, 50): A implies B
    r = orc.probe(t.columns, t.dtypes, [[a, b]], Sample(FULL))
    c_ab = int(r.counts[0])
    c_a, c_b = (int(x) for x in r.marginals)
    assert c_ab == c_a > 0
    assert orc.pcs(c_ab, c_a, c_b, n) == n / c_b
    assert orc.pcs(c_ab, c_a, c_b, n) > 1.6


def test_pcs_near_one_for_independent_columns(orc):
    n = 400000
    t = make_plain_small(n=n, seed=12)
    a, b = Term(0, RANGE, 0, 500000), Term(3, RANGE, 0, 50)
    r = orc.probe(t.columns, t.dtypes, [[a, b]], Sample(FULL))
    pcs = orc.pcs(int(r.counts[0]), int(r.marginals[0]), int(r.marginals[1]), n)
    assert abs(pcs - 1.0) < 0.012  # about 6 binomial standard deviations
    assert math.isnan(orc.pcs(0, 0, 5, 10))


# ----------------------------------------------------------------- HyperLogLog

def _distinct(n, seed):
    rng = np.random.default_rng(seed)
    return rng.choice(1 << 40, size=n, replace=False).astype(np.int64)


def test_ndv_exact_matches_numpy_unique(orc):
    t = _small_table(20000, 1)
    for c in range(4):
        assert orc.ndv_exact(t.columns[c], I32) == len(np.unique(t.columns[c].numpy()))
    f = np.array([0.0, -0.0, np.nan, np.nan, 1.0, 1.0, -1.0], dtype=np.float32)
    assert orc.ndv_exact(f, F32) == 4


def test_hll_estimate_closed_forms(orc):
    assert orc.hll_estimate(np.zeros(1024, np.uint8), 10) == 0.0
    e = orc.hll_estimate(np.ones(16, np.uint8), 4)
    assert e == pytest.approx(0.673 * 256 / 8, rel=1e-15)
    m = 1024
    regs = np.array([0] * 512 + [1] * 512, dtype=np.uint8)
    assert orc.hll_estimate(regs, 10) == pytest.approx(m * math.log(2.0), rel=1e-15)
    k = 12
    regs = np.full(4096, k, dtype=np.uint8)
    alpha = 0.7213 / (1 + 1.079 / 4096)
    assert orc.hll_estimate(regs, 12) == pytest.approx(alpha * 4096 * 2.0 ** k, rel=1e-14)


def test_hll_single_value_register(orc):
    for p, x in [(4, 0), (12, -5), (14, 123456789), (18, 1 << 33)]:
        col = np.full(10, x, dtype=np.int64)
        regs = orc.hll_registers(col, I64, p, 42)
        nz = np.nonzero(regs)[0]
        assert len(nz) == 1
        h = orc.hash64(x & M64, 42)
        j = h >> (64 - p)
        w = (h << p) & M64
        rho = (64 - p + 1) if w == 0 else 64 - w.bit_length() + 1
        assert nz[0] == j and regs[j] == rho


def test_hll_order_and_duplicate_invariance(orc):
    x = _distinct(5000, 1)
    dup = np.concatenate([x, x[::3], x[::7]])
    perm = np.random.default_rng(2).permutation(dup)
    r1 = orc.hll_registers(x, I64, 12, 7)
    assert np.array_equal(r1, orc.hll_registers(dup, I64, 12, 7))
    assert np.array_equal(r1, orc.hll_registers(perm, I64, 12, 7))
    # int32 values hash as their sign-extended 64-bit value
    y = (x % 1000000 - 500000).astype(np.int32)
    assert np.array_equal(orc.hll_registers(y, I32, 12, 7),
                          orc.hll_registers(y.astype(np.int64), I64, 12, 7))


@pytest.mark.parametrize("p", [10, 12])
def test_hll_error_within_published_bound(orc, p):
    """Large range: RMS relative error over 64 hash seeds within 1.3 x the
    standard error 1.04/sqrt(m), each seed within 4 x (Flajolet et al.)."""
    m = 1 << p
    x = _distinct(50 * m, p)
    se = 1.04 / math.sqrt(m)
    errs = []
    for seed in range(64):
        e = orc.hll_estimate(orc.hll_registers(x, I64, p, seed), p)
        errs.append(e / len(x) - 1.0)
    errs = np.array(errs)
    assert np.sqrt(np.mean(errs ** 2)) <= 1.3 * se
    assert np.max(np.abs(errs)) <= 4 * se
    assert abs(np.mean(errs)) <= 3 * se / 8  # no systematic bias (mean of 64)


def test_hll_small_range_linear_counting(orc):
    p = 12
    m = 1 << p
    n = m // 20
    t = n / m
    sd = math.sqrt(m * (math.exp(t) - t - 1)) / n  # linear counting standard error
    errs = []
    for seed in range(64):
        x = _distinct(n, 100 + seed)
        errs.append(orc.hll_estimate(orc.hll_registers(x, I64, p, seed), p) / n - 1.0)
    errs = np.array(errs)
    assert np.max(np.abs(errs)) <= 4.5 * sd
    assert np.sqrt(np.mean(errs ** 2)) <= 1.3 * sd


# ----------------------------------------------------------------- joins

def _side(cols, dtypes, key_col, terms):
    return JoinSide(Table("s", cols, dtypes, []), key_col, terms)


def _nested_loop(fk, fpass, key, dpass):
    a = fk[fpass]
    b = key[dpass]
    return int((a[:, None] == b[None, :]).sum())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_join_card_equals_nested_loop(orc, seed):
    rng = np.random.default_rng(seed)
    nf, nd, K = 2000, 1500, 800
    fk = rng.zipf(1.3, nf).astype(np.int64) % (K + 40) - 20     # some keys outside [0, K)
    f1 = rng.integers(0, 100, nf).astype(np.int32)
    key = rng.integers(0, K, nd).astype(np.int32)                # duplicates allowed
    g1 = rng.integers(0, 100, nd).astype(np.int32)
    ft = [Term(1, RANGE, 0, 40)]
    dt = [Term(1, RANGE, 20, 90)]
    F = _side([fk.astype(np.int32), f1], [I32, I32], 0, ft)
    D = _side([key, g1], [I32, I32], 0, dt)
    rc, card, fp, dp = orc.join_card(F, D, K)
    assert rc == 0
    fpass, dpass = (f1 >= 0) & (f1 < 40), (g1 >= 20) & (g1 < 90)
    assert card == _nested_loop(fk, fpass, key.astype(np.int64), dpass)
    assert fp == int(fpass.sum()) and dp == int(dpass.sum())


def test_join_unique_keys_and_full_filters(orc):
    rng = np.random.default_rng(4)
    K = 500
    key = rng.permutation(K).astype(np.int32)
    fk = rng.integers(-10, K + 10, 3000).astype(np.int32)
    F = _side([fk], [I32], 0, [])
    D = _side([key], [I32], 0, [])
    rc, card, fp, dp = orc.join_card(F, D, K)
    assert rc == 0 and fp == 3000 and dp == K
    assert card == int(((fk >= 0) & (fk < K)).sum())
    rc, card2, _, _ = orc.join_card(F, _side([key], [I32], 0, [Term(0, RANGE, 0, 100)]), K)
    assert card2 <= fp and card2 == int(((fk >= 0) & (fk < 100)).sum())


def test_join_rejects_dim_key_outside_domain(orc):
    F = _side([np.array([1, 2], np.int32)], [I32], 0, [])
    D = _side([np.array([1, 5], np.int32)], [I32], 0, [])
    assert orc.join_card(F, D, 5)[0] == 1
    # the out-of-domain row is filtered away: accepted
    D2 = _side([np.array([1, 5], np.int32)], [I32], 0, [Term(0, RANGE, 0, 5)])
    rc, card, _, _ = orc.join_card(F, D2, 5)
    assert rc == 0 and card == 1


def test_chain_card_equals_triple_nested_loop(orc):
    rng = np.random.default_rng(7)
    K1, K2 = 60, 25
    nf, n1, n2 = 300, 80, 40
    fk = rng.integers(0, K1 + 5, nf).astype(np.int32)
    f1 = rng.integers(0, 10, nf).astype(np.int32)
    d1key = rng.integers(0, K1, n1).astype(np.int32)
    d1g = rng.integers(0, 10, n1).astype(np.int32)
    d1fk2 = rng.integers(-2, K2 + 3, n1).astype(np.int32)
    d2key = rng.integers(0, K2, n2).astype(np.int32)
    d2h = rng.integers(0, 10, n2).astype(np.int32)
    F = _side([fk, f1], [I32, I32], 0, [Term(1, RANGE, 0, 7)])
    D1 = _side([d1key, d1g, d1fk2], [I32, I32, I32], 0, [Term(1, IN, values=(1, 2, 3, 5, 8))])
    D2 = _side([d2key, d2h], [I32, I32], 0, [Term(1, RANGE, 2, 10)])
    rc, card, fp, p1, p2 = orc.chain_card(F, D1, 2, D2, K1, K2)
    assert rc == 0
    brute = 0
    for r in range(nf):
        if not (0 <= f1[r] < 7):
            continue
        for d in range(n1):
            if d1g[d] not in (1, 2, 3, 5, 8) or d1key[d] != fk[r]:
                continue
            for e in range(n2):
                if 2 <= d2h[e] < 10 and d2key[e] == d1fk2[d]:
                    brute += 1
    assert card == brute and brute > 0
    assert (fp, p1, p2) == (int(((f1 >= 0) & (f1 < 7)).sum()),
                            int(np.isin(d1g, [1, 2, 3, 5, 8]).sum()),
                            int(((d2h >= 2) & (d2h < 10)).sum()))


def test_chain_reduces_to_two_table_join(orc):
    rng = np.random.default_rng(9)
    K1, K2 = 200, 50
    fk = rng.integers(0, K1, 4000).astype(np.int32)
    d1key = rng.permutation(K1).astype(np.int32)
    d1fk2 = (np.arange(K1) % K2).astype(np.int32)
    d2key = rng.permutation(K2).astype(np.int32)
    F = _side([fk], [I32], 0, [])
    D1 = _side([d1key, d1fk2], [I32, I32], 0, [Term(0, RANGE, 0, 150)])
    D2 = _side([d2key], [I32], 0, [])
    rc, card3, *_ = orc.chain_card(F, D1, 1, D2, K1, K2)
    rc2, card2, *_ = orc.join_card(F, D1, K1)
    assert rc == rc2 == 0 and card3 == card2


# ----------------------------------------------------------------- Risky Gate

def test_gate_hand_worked_cases(orc):
    """Section III-C, Eq. 1-3 with the paper's thresholds: the cases of
    tests/golden/gate_cases.json, worked by hand."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "gate_cases.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        args = {k: float(c[k]) for k in ("ndv_hist", "ndv_est", "sel_est", "sel_probe", "pcs") if k in c}
        flags, drift, sel_err = orc.gate(**args)
        assert flags == c["flags"], c["note"]
        if "drift" in c:
            assert (math.isnan(drift) if c["drift"] is None else math.isclose(drift, c["drift"], rel_tol=1e-12)), c
        if "sel_err" in c:
            assert math.isclose(sel_err, c["sel_err"], rel_tol=1e-12), c


def test_gate_thresholds_are_the_papers(orc):
    assert (orc.GATE_DRIFT_MIN, orc.GATE_SEL_ERR_MAX, orc.GATE_PCS_HIGH, orc.GATE_PCS_LOW) == (0.25, 0.01, 1.6, 0.7)
    # each flag is monotone in its signal's distance from the trusted value
    prev = 0
    for est in (1000, 900, 800, 760, 750, 700, 0):
        f = orc.gate(ndv_hist=1000.0, ndv_est=float(est))[0]
        assert f >= prev
        prev = f
    assert [orc.gate(pcs=x)[0] for x in (0.5, 0.69, 0.7, 1.0, 1.6, 1.61, 3.0)] == [4, 4, 0, 0, 0, 4, 4]
    # a missing signal never flags
    assert orc.gate() == (0, orc.gate()[1], orc.gate()[2]) and orc.gate()[0] == 0


def test_probe_cost_closed_forms(orc):
    """The break-even model (Section V, item 2): call cost alone at N = 0;
    linear in N; a narrow batch costs its bytes, a wide one its compare
    operations; the break-even N solves total = alt."""
    r = dict(hbm_rate=4e12, ops_rate=1e13, h2d_rate=5e10, hash_ns=2e-3, call_ms=0.05)
    assert orc.probe_cost(0, 1, 1, 4, 0, True, 0.0, 1.0, r) == (0.05, True, True)
    t1 = orc.probe_cost(10**8, 1, 1, 4, 0, True, 0.0, 0.0, r)[0] - 0.05
    t2 = orc.probe_cost(2 * 10**8, 1, 1, 4, 0, True, 0.0, 0.0, r)[0] - 0.05
    assert math.isclose(t1, 0.1, rel_tol=1e-12) and math.isclose(t2, 2 * t1, rel_tol=1e-12)  # 400 MB at 4 TB/s
    # one hashed set adds N x 2 ps: 0.2 ms for 1e8 rows
    assert math.isclose(orc.probe_cost(10**8, 1, 2, 4, 1, True, 0.0, 0.0, r)[0] - 0.05, 0.3, rel_tol=1e-12)
    # 33 predicates take the wide model: 1e8 rows x 100 ops at 1e13/s = 1 ms
    total, narrow, _ = orc.probe_cost(10**8, 33, 33, 4, 0, True, 100.0, 0.0, r)
    assert not narrow and math.isclose(total - 0.05, 1.0, rel_tol=1e-12)
    # non-resident columns add their copy: 400 MB at 50 GB/s = 8 ms
    assert math.isclose(orc.probe_cost(10**8, 1, 1, 4, 0, False, 0.0, 0.0, r)[0] - 0.05, 8.1, rel_tol=1e-12)
    # break-even: offload exactly when total < alt
    n_star = (1.0 - 0.05) / (4 / 4e12 * 1e3)
    assert orc.probe_cost(int(n_star) - 1, 1, 1, 4, 0, True, 0.0, 1.0, r)[2]
    assert not orc.probe_cost(int(n_star) + 1, 1, 1, 4, 0, True, 0.0, 1.0, r)[2]
