"""Materialised samples and the resident store of samples and sketches.

A materialised sample is a table of its own: a full scan of it must return
exactly the oracle's counts, sample sizes, selectivities, PCS and marginals of
the sampled scan of the base table, and its columns must hold exactly the
sample's rows (checked through HyperLogLog registers of its columns against
the oracle's over the kept rows, which the oracle's membership test lists).
The store must give every form of the calls the same results with and
without it, admit after the configured number of uses, evict the least
recently used entries under a small budget, refuse what cannot fit, and
forget what it drew from an unloaded table."""
import numpy as np
import pytest
import torch

from batch_util import to_requests
from parity import check_probe, close, host_columns
from workloads import (BLOCKS, F32, FULL, I32, I64, RANGE, ROWS, Sample, Term, make_batched, make_predicates,
                       make_skew_corr)

pytestmark = pytest.mark.gpu

SAMPLED = [Sample(ROWS, 0.01, 42), Sample(ROWS, 0.1, 42), Sample(BLOCKS, 0.01, 42, 4096),
           Sample(BLOCKS, 0.05, 7, 3000)]


@pytest.fixture(scope="module")
def table(cuda):
    # 3M rows: 733 sample tiles with a ragged last one; every column type
    return make_skew_corr(n=3_000_017, seed=77, device=cuda, domain=50_000)


@pytest.fixture(scope="module")
def host(table):
    return host_columns(table)


def _probe_full(g, ctx, sid, preds, dtypes):
    return g.gace_probe_batch(ctx, sid, preds, [Sample(FULL)], dtypes, marginals=True)


@pytest.mark.parametrize("npreds", [12, 48])  # narrow and wide passes
def test_materialized_sample_equals_oracle(g, gctx, orc, table, host, npreds):
    preds = make_predicates(table, npreds, 1, 3, seed=900 + npreds)
    tid = g.gace_load_columns(gctx, table.columns, borrow=True)
    try:
        for smp in SAMPLED:
            sid, rows = g.gace_sample_materialize(gctx, tid, smp)
            try:
                res, marg = _probe_full(g, gctx, sid, preds, table.dtypes)
                ref = orc.probe(host, table.dtypes, preds, smp, marginals=True)
                assert rows == ref.n_sample, (smp, rows, ref.n_sample)
                assert np.array_equal(res["match"][0], ref.counts), smp
                assert (res["sample_rows"][0] == ref.n_sample).all()
                assert np.array_equal(marg[0], ref.marginals), smp
                # the unmaterialised call: the same results, element by element
                base, bmarg = g.gace_probe_batch(gctx, tid, preds, [smp], table.dtypes, marginals=True)
                for f in ("match", "sample_rows", "sel"):
                    assert np.array_equal(res[f], base[f]), (smp, f)
                assert np.array_equal(res["pcs"], base["pcs"], equal_nan=True)
                assert np.array_equal(marg, bmarg)
            finally:
                g.gace_unload(gctx, sid)
    finally:
        g.gace_unload(gctx, tid)


def test_sample_holds_the_kept_rows(g, gctx, orc, cuda):
    """HLL registers of every column of the sample table equal the oracle's
    registers over exactly the rows the oracle's membership test keeps."""
    t = make_skew_corr(n=200_003, seed=78, device=cuda, domain=20_000)
    hst = host_columns(t)
    tid = g.gace_load_columns(gctx, t.columns, borrow=True)
    try:
        for smp in (Sample(ROWS, 0.1, 42), Sample(BLOCKS, 0.2, 5, 1000)):
            kept = np.array([orc.row_in_sample(smp, i) for i in range(t.nrows)], dtype=bool)
            sid, rows = g.gace_sample_materialize(gctx, tid, smp)
            try:
                assert rows == int(kept.sum())
                for c in range(len(t.columns)):
                    col = np.asarray(hst[c])[kept]
                    regs, est = g.gace_ndv(gctx, sid, c, 12, 9)
                    ref = orc.hll_registers(col, t.dtypes[c], 12, 9)
                    assert np.array_equal(regs, ref), (smp, c)
                    assert close(est, orc.hll_estimate(ref, 12))
            finally:
                g.gace_unload(gctx, sid)
    finally:
        g.gace_unload(gctx, tid)


def test_materialize_rejects_full_and_degenerate(g, gctx, cuda):
    t = make_skew_corr(n=10_000, seed=79, device=cuda)
    tid = g.gace_load_columns(gctx, t.columns, borrow=True)
    try:
        for smp in (Sample(FULL), Sample(ROWS, 0.0, 1), Sample(ROWS, 1.0, 1)):
            with pytest.raises(g.GaceError) as e:
                g.gace_sample_materialize(gctx, tid, smp)
            assert e.value.status == g.GACE_EINVAL
        sid, rows = g.gace_sample_materialize(gctx, tid, Sample(ROWS, 1e-9, 3))  # an empty sample
        res, _ = _probe_full(g, gctx, sid, [[Term(0, RANGE, 0, 10**6)], []], t.dtypes)
        assert rows == 0 and (res["sample_rows"] == 0).all() and (res["match"] == 0).all()
        g.gace_unload(gctx, sid)
    finally:
        g.gace_unload(gctx, tid)


def test_store_sync_calls(g, orc, table, host, cuda):
    """The synchronous calls with the store on: the first sampled probe admits
    its sample, the next ones hit it; a probe that mixes the full table, two
    resident samples and a sample that is not resident yet is split and
    equals the oracle on every row set; NDV answers from a resident sketch."""
    ctx = g.gace_create(0)
    try:
        tid = g.gace_load_columns(ctx, table.columns, borrow=True)
        preds = make_predicates(table, 40, 1, 4, seed=901)
        g.gace_resident_configure(ctx, 8 << 30)
        for k in range(2):
            check_probe(g, orc, ctx, tid, host, table.dtypes, preds, [SAMPLED[0]])
            st = g.gace_resident_stats_read(ctx)
            assert st["admitted"] == 1 and st["sample_hits"] == k and st["samples"] == 1
        mix = [Sample(FULL), SAMPLED[0], SAMPLED[2], SAMPLED[1], SAMPLED[0]]
        check_probe(g, orc, ctx, tid, host, table.dtypes, preds, mix)
        st = g.gace_resident_stats_read(ctx)
        assert st["samples"] == 3 and st["admitted"] == 3
        for k in range(2):
            regs, est = g.gace_ndv(ctx, tid, 4, 14, 42)
            ref = orc.hll_registers(host[4], I64, 14, 42)
            assert np.array_equal(regs, ref) and close(est, orc.hll_estimate(ref, 14))
        st = g.gace_resident_stats_read(ctx)
        assert st["sketch_hits"] == 1 and st["sketches"] == 1
        assert st["used_bytes"] <= st["budget_bytes"]
        g.gace_unload(ctx, tid)
        st = g.gace_resident_stats_read(ctx)
        assert st["samples"] == 0 and st["sketches"] == 0 and st["used_bytes"] == 0
    finally:
        g.gace_destroy(ctx)


def test_store_admit_after(g, orc, table, host):
    ctx = g.gace_create(0)
    try:
        tid = g.gace_load_columns(ctx, table.columns, borrow=True)
        g.gace_resident_configure(ctx, 8 << 30, admit_after=3)
        preds = [[Term(0, RANGE, 0, 100)], [Term(6, RANGE, -0.5, 0.5), Term(2, RANGE, 0, 1000)]]
        for k in range(4):
            check_probe(g, orc, ctx, tid, host, table.dtypes, preds, [SAMPLED[1]])
            st = g.gace_resident_stats_read(ctx)
            assert st["admitted"] == (1 if k >= 2 else 0), (k, st)
        assert st["sample_hits"] == 1 and st["sample_misses"] == 3
    finally:
        g.gace_destroy(ctx)


def test_store_small_budget_evicts_and_refuses(g, orc, cuda):
    """A budget that holds one 10 % sample of a 2M-row table: the second
    table's sample evicts the first's; a sample larger than the budget is
    refused and the probe scans the base table; every answer equals the
    oracle's.  Prefetch of what cannot fit fails with GACE_ENOMEM."""
    ctx = g.gace_create(0)
    try:
        tabs = [make_skew_corr(n=2_000_000, seed=80 + k, device=cuda, domain=10_000) for k in range(2)]
        hosts = [host_columns(t) for t in tabs]
        tids = [g.gace_load_columns(ctx, t.columns, borrow=True) for t in tabs]
        one = 2_000_000 * 40 // 10  # bytes of one 10 % sample of 40-byte rows
        g.gace_resident_configure(ctx, int(one * 1.5))
        preds = [[Term(0, RANGE, 0, 50), Term(1, RANGE, 0, 50)], [Term(7, RANGE, -1.0, 0.0)]]
        smp = Sample(ROWS, 0.1, 42)
        check_probe(g, orc, ctx, tids[0], hosts[0], tabs[0].dtypes, preds, [smp])
        check_probe(g, orc, ctx, tids[1], hosts[1], tabs[1].dtypes, preds, [smp])
        st = g.gace_resident_stats_read(ctx)
        assert st["admitted"] == 2 and st["evicted"] == 1 and st["samples"] == 1, st
        assert st["used_bytes"] <= st["budget_bytes"]
        big = Sample(ROWS, 0.5, 42)
        check_probe(g, orc, ctx, tids[0], hosts[0], tabs[0].dtypes, preds, [big])
        st = g.gace_resident_stats_read(ctx)
        assert st["refused"] == 1, st
        with pytest.raises(g.GaceError) as e:
            g.gace_resident_prefetch(ctx, tids[0], big)
        assert e.value.status == g.GACE_ENOMEM
        g.gace_resident_prefetch(ctx, tids[0], Sample(ROWS, 0.01, 42))
        assert g.gace_resident_stats_read(ctx)["samples"] == 2
    finally:
        g.gace_destroy(ctx)


def test_hbm_budget_limits_materialisation(g, cuda):
    t = make_skew_corr(n=1_000_000, seed=81, device=cuda)
    ctx = g.gace_create(0, hbm_budget_bytes=3 << 20)  # the workspace fits, a 10 % sample (4 MB) does not
    try:
        tid = g.gace_load_columns(ctx, t.columns, borrow=True)
        with pytest.raises(g.GaceError) as e:
            g.gace_sample_materialize(ctx, tid, Sample(ROWS, 0.1, 42))
        assert e.value.status == g.GACE_ENOMEM
    finally:
        g.gace_destroy(ctx)


def _mixed(g, cuda, seed):
    tables, reqs = make_batched(ntables=8, min_rows=50_000, max_rows=3_000_000, nprobes=160, seed=seed, device=cuda)
    return tables, reqs


def _compare(reqs, got, want):
    for r, a, b in zip(reqs, got, want):
        if r["kind"] == "probe":
            for f in ("match", "sample_rows", "sel"):
                assert np.array_equal(a.results[f], b.results[f]), (r, f)
            assert np.array_equal(a.results["pcs"], b.results["pcs"], equal_nan=True)
            assert np.array_equal(a.marginals, b.marginals)
        elif r["kind"] == "ndv":
            assert np.array_equal(a.registers, b.registers) and a.estimate == b.estimate
        else:
            assert a.result == b.result


def test_store_batched_and_served(g, cuda):
    """A mixed batch and the same requests served: with the store on (after a
    first run admits the samples and sketches) every result equals the run
    without it; the second run hits the store."""
    tables, reqs = _mixed(g, cuda, 1007)
    ctx = g.gace_create(0)
    try:
        tids = [g.gace_load_columns(ctx, t.columns, borrow=True) for t in tables]
        plain = to_requests(g, tids, tables, reqs)
        g.gace_run_batch(ctx, plain)
        g.gace_resident_configure(ctx, 4 << 30)
        for run in range(2):
            batch = to_requests(g, tids, tables, reqs)
            g.gace_run_batch(ctx, batch)
            _compare(reqs, batch, plain)
        st = g.gace_resident_stats_read(ctx)
        assert st["sample_hits"] > 0 and st["sketch_hits"] > 0, st
        g.gace_serve_start(ctx, always_step=True, sketch_cache=-1, probe_cache=-1)
        served = to_requests(g, tids, tables, reqs)
        tickets = [g.gace_submit(ctx, q) for q in served]
        for t in tickets:
            assert g.gace_poll(ctx, t, 10_000_000)
        _compare(reqs, served, plain)
        # a base table whose resident samples are idle may be unloaded
        g.gace_serve_stop(ctx)
        before = g.gace_resident_stats_read(ctx)["samples"]
        g.gace_unload(ctx, tids[0])
        assert g.gace_resident_stats_read(ctx)["samples"] <= before
    finally:
        g.gace_destroy(ctx)
