"""Break-even model (Section V, item 2) on a live context: default rates
before any timing, the context's own measured rates after timed probes, its
predictions within a factor of two of the measured kernel time, and every
answer equal to the oracle's formula at the answer's rates."""
import math

import pytest

from workloads import FULL, RANGE, ROWS, Sample, Term, make_predicates, make_skew_corr

pytestmark = pytest.mark.gpu


def _same_as_oracle(orc, a, q):
    rates = {k: a[k] for k in ("hbm_rate", "ops_rate", "h2d_rate", "hash_ns", "call_ms")}
    total, narrow, offload = orc.probe_cost(q["nrows"], q["npreds"], q.get("nterms", q["npreds"]), q["row_bytes"],
                                            q.get("hashed_sets", 0), q.get("resident", True), q.get("ops_per_row", 0.0),
                                            q["alt_ms"], rates)
    assert math.isclose(a["total_ms"], total, rel_tol=1e-12, abs_tol=1e-15)
    assert bool(a["narrow"]) == narrow and bool(a["offload"]) == offload


def test_break_even_rates_and_predictions(g, orc, cuda):
    ctx = g.gace_create(0)
    t = make_skew_corr(n=50_000_000, seed=33, device=cuda)
    tid = g.gace_load_columns(ctx, t.columns, borrow=True)
    try:
        q = dict(nrows=t.nrows, npreds=1, nsets=1, row_bytes=4, alt_ms=1.0)
        a = g.gace_break_even(ctx, **q)
        assert a["measured"] == 0 and a["narrow"] == 1
        _same_as_oracle(orc, a, q)
        # timed narrow probes: one int32 range, full scan
        g.gace_stats_reset(ctx, time_kernels=True)
        pred = [[Term(0, RANGE, 0, 1000)]]
        for _ in range(6):
            g.gace_probe_batch(ctx, tid, pred, [Sample(FULL)], t.dtypes)
        st = g.gace_stats_read(ctx)["probe_narrow"]
        a = g.gace_break_even(ctx, **q)
        assert a["measured"] & 1
        measured_ms = st["total_ms"] / st["launches"]
        assert 0.5 < a["kernel_ms"] / measured_ms < 2.0, (a, measured_ms)
        _same_as_oracle(orc, a, q)
        # the measurements survive a statistics reset
        g.gace_stats_reset(ctx, time_kernels=False)
        assert g.gace_break_even(ctx, **q)["hbm_rate"] == a["hbm_rate"]
        # timed wide passes: 200 predicates over all columns
        preds = make_predicates(t, 200, 1, 3, seed=9)
        g.gace_stats_reset(ctx, time_kernels=True)
        for _ in range(3):
            g.gace_probe_batch(ctx, tid, preds, [Sample(FULL), Sample(ROWS, 0.01, 42)], t.dtypes)
        st = g.gace_stats_read(ctx)["probe_wide"]
        ops_per_row = st["ops"] / st["rows"]
        nterms = len({x for p in preds for x in p})
        qw = dict(nrows=t.nrows, npreds=len(preds), nsets=2, hashed_sets=1, nterms=nterms, row_bytes=40,
                  ops_per_row=ops_per_row * st["rows"] / (3 * t.nrows), alt_ms=5.0)
        aw = g.gace_break_even(ctx, **qw)
        assert aw["measured"] & 2 and aw["narrow"] == 0
        measured_call = st["total_ms"] / 3
        assert 0.5 < aw["kernel_ms"] / measured_call < 2.0, (aw, measured_call)
        _same_as_oracle(orc, aw, qw)
        # non-resident columns add a key-only copy; a generous alternative makes offload pay
        for resident in (False, True):
            for alt in (0.0, 1e9):
                qq = dict(q, resident=resident, alt_ms=alt)
                _same_as_oracle(orc, g.gace_break_even(ctx, **qq), qq)
        with pytest.raises(g.GaceError):
            g.gace_break_even(ctx, nrows=10, npreds=1, nsets=0)
        with pytest.raises(g.GaceError):
            g.gace_break_even(ctx, nrows=10, npreds=1, nsets=1, hashed_sets=2)
    finally:
        g.gace_unload(ctx, tid)
        g.gace_destroy(ctx)
