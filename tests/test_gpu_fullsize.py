"""GPU parity at the benchmark's full sizes, in the calls bench.py times:
outputs the oracle can compute one by one (sampled predicates of the
1024-predicate batch on 100M rows, every HLL sketch, the 500M-row joins, a
sample of the batched and served requests) against the oracle, and every
batched and served request against its synchronous call."""
import numpy as np
import pytest
import torch

from batch_util import check_against_sync, to_requests
from parity import close, host_columns
from workloads import (BLOCKS, FULL, RANGE, ROWS, JoinSide, Sample, Table, Term, make_batched, make_join,
                       make_plain_small, make_predicates, make_skew_corr)

pytestmark = pytest.mark.gpu

SAMPLES = [Sample(FULL), Sample(ROWS, 0.001, 42), Sample(ROWS, 0.01, 42), Sample(ROWS, 0.1, 42),
           Sample(BLOCKS, 0.01, 42, 4096)]


def _free():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_config1_hll_full_size(g, gctx, orc, cuda):
    """Config 1: HLL p = 12 of each of the 4 columns of the 1M-row table."""
    t = make_plain_small(n=1_000_000, seed=1001, device=cuda)
    tid = g.gace_load_columns(gctx, t.columns, borrow=True)
    try:
        for c in range(4):
            regs, est = g.gace_ndv(gctx, tid, c, 12, 42)
            ref = orc.hll_registers(t.columns[c].cpu(), t.dtypes[c], 12, 42)
            assert np.array_equal(regs, ref) and close(est, orc.hll_estimate(ref, 12))
    finally:
        g.gace_unload(gctx, tid)


def test_config2_sampled_predicates_and_sketches(g, gctx, orc, cuda):
    """Config 2 (100M rows x 8 columns): the bench's 1024-predicate batch on
    its five row sets in one call; eight sampled predicates (counts, sample
    sizes, selectivities, PCS, term marginals) and all eight HLL p = 14
    sketches against the oracle over every row."""
    t = make_skew_corr(n=100_000_000, seed=1002, device=cuda)
    preds = make_predicates(t, 1024, 1, 4, seed=2002)
    tid = g.gace_load_columns(gctx, t.columns, borrow=True)
    try:
        batch = g.TermBatch(preds, t.dtypes)
        res, marg = g.gace_probe_batch(gctx, tid, preds, SAMPLES, t.dtypes, marginals=True, batch=batch)
        regs = [g.gace_ndv(gctx, tid, c, 14, 42) for c in range(len(t.columns))]
        host = host_columns(t)
        rng = np.random.default_rng(20251203)
        pick = sorted(rng.choice(len(preds), 8, replace=False).tolist())
        two = [p for p in range(len(preds)) if len(preds[p]) == 2]
        if not any(len(preds[p]) == 2 for p in pick):
            pick[0] = two[0]  # at least one PCS
        offs = np.cumsum([0] + [len(p) for p in preds])
        sub = [preds[p] for p in pick]
        for s, smp in enumerate(SAMPLES):
            ref = orc.probe(host, t.dtypes, sub, smp, marginals=True)
            assert int(res["sample_rows"][s][0]) == ref.n_sample
            k = 0
            for j, p in enumerate(pick):
                assert int(res["match"][s][p]) == int(ref.counts[j]), (s, p)
                assert close(float(res["sel"][s][p]), orc.selectivity(int(ref.counts[j]), ref.n_sample))
                for q in range(len(preds[p])):
                    assert int(marg[s][offs[p] + q]) == int(ref.marginals[k + q]), (s, p, q)
                if len(preds[p]) == 2:
                    pcs = orc.pcs(int(ref.counts[j]), int(ref.marginals[k]), int(ref.marginals[k + 1]), ref.n_sample)
                    assert close(float(res["pcs"][s][p]), pcs), (s, p)
                k += len(preds[p])
        for c in range(len(t.columns)):
            ref = orc.hll_registers(host[c], t.dtypes[c], 14, 42)
            assert np.array_equal(regs[c][0], ref), c
            assert close(regs[c][1], orc.hll_estimate(ref, 14))
    finally:
        g.gace_unload(gctx, tid)
        del t
        _free()


def test_config3_joins_full_size(g, gctx, orc, cuda):
    """Config 3: the bench's joins of the 500M-row fact table and 10M-row
    dimension at 1 % and 10 % filters, and the 3-table chain, against the
    oracle's histograms over every row."""
    f, dm, d2 = make_join(seed=1003, device=cuda)
    fid = g.gace_load_columns(gctx, f.columns, borrow=True)
    did = g.gace_load_columns(gctx, dm.columns, borrow=True)
    d2id = g.gace_load_columns(gctx, d2.columns, borrow=True)
    try:
        fh, dh, d2h = (Table(x.name, host_columns(x), x.dtypes) for x in (f, dm, d2))
        for w in (10, 100):
            ft, dt = [Term(1, RANGE, 0, w)], [Term(1, RANGE, 0, w)]
            out = g.gace_join_card(gctx, g.JoinSideSpec(fid, 0, ft, f.dtypes), g.JoinSideSpec(did, 0, dt, dm.dtypes),
                                   10_000_000)
            rc, card, fp, dp = orc.join_card(JoinSide(fh, 0, ft), JoinSide(dh, 0, dt), 10_000_000)
            assert rc == 0 and (out["card"], out["fact_rows"], out["dim_rows"]) == (card, fp, dp), w
        ft, dt, d2t = [Term(1, RANGE, 0, 100)], [Term(1, RANGE, 0, 500)], [Term(1, RANGE, 0, 500)]
        out = g.gace_join_card(gctx, g.JoinSideSpec(fid, 0, ft, f.dtypes), g.JoinSideSpec(did, 0, dt, dm.dtypes),
                               10_000_000, g.JoinSideSpec(d2id, 0, d2t, d2.dtypes), 1_000_000, 3)
        rc, card, fp, p1, p2 = orc.chain_card(JoinSide(fh, 0, ft), JoinSide(dh, 0, dt), 3, JoinSide(d2h, 0, d2t),
                                              10_000_000, 1_000_000)
        assert rc == 0 and (out["card"], out["fact_rows"], out["dim_rows"], out["dim2_rows"]) == (card, fp, p1, p2)
    finally:
        for t in (fid, did, d2id):
            g.gace_unload(gctx, t)
        del f, dm, d2
        _free()


def _oracle_request(orc, tables, r):
    """The oracle's answer for one generated request, as (kind, values)."""
    if r["kind"] == "probe":
        t = tables[r["table"]]
        return orc.probe(host_columns(t), t.dtypes, r["preds"], r["samples"][0])
    if r["kind"] == "ndv":
        t = tables[r["table"]]
        return orc.hll_registers(t.columns[r["col"]].cpu(), t.dtypes[r["col"]], r["p"], r["seed"])
    f, d = tables[r["fact"]], tables[r["dim"]]
    fh, dh = Table("f", host_columns(f), f.dtypes), Table("d", host_columns(d), d.dtypes)
    return orc.join_card(JoinSide(fh, 0, r["fact_terms"]), JoinSide(dh, 0, r["dim_terms"]), r["key_domain"])


def _check_oracle_sample(g, orc, tables, reqs, breqs, n, max_rows, seed):
    rows = [max(tables[r["table"]].nrows if r["kind"] != "join" else
                max(tables[r["fact"]].nrows, tables[r["dim"]].nrows), 0) for r in reqs]
    cand = [i for i, nr in enumerate(rows) if nr <= max_rows]
    rng = np.random.default_rng(seed)
    for i in rng.choice(cand, min(n, len(cand)), replace=False):
        r, q = reqs[i], breqs[i]
        ref = _oracle_request(orc, tables, r)
        if r["kind"] == "probe":
            assert np.array_equal(q.results["match"][0], ref.counts), i
            assert int(q.results["sample_rows"][0][0]) == ref.n_sample
            assert np.array_equal(q.marginals[0], ref.marginals), i
        elif r["kind"] == "ndv":
            assert np.array_equal(q.registers, ref), i
        else:
            rc, card, fp, dp = ref
            assert rc == 0 and (q.result["card"], q.result["fact_rows"], q.result["dim_rows"]) == (card, fp, dp), i


def test_config4_batched_full_size(g, gctx, orc, cuda):
    """Config 4: 4096 requests over 256 tables (1e4..5e7 rows) in one tuned
    batch, as the bench runs it; every request equals its synchronous call and
    a sample of 16 equals the oracle."""
    tables, reqs = make_batched(ntables=256, min_rows=10_000, max_rows=50_000_000, nprobes=4096, seed=1004,
                                device=cuda)
    tids = [g.gace_load_columns(gctx, t.columns, borrow=True) for t in tables]
    try:
        g.gace_tune_batch(gctx, to_requests(g, tids, tables, reqs))
        breqs = to_requests(g, tids, tables, reqs)
        assert g.gace_run_batch(gctx, breqs) == [0] * len(reqs)
        check_against_sync(g, gctx, tids, tables, reqs, breqs)
        _check_oracle_sample(g, orc, tables, reqs, breqs, 16, 20_000_000, 4)
    finally:
        for t in tids:
            g.gace_unload(gctx, t)
        del tables
        _free()


def test_config5_served_full_size(g, orc, cuda):
    """Config 5: the request mix over 64 tables (1e6..2e8 rows) arriving at
    10k requests/s through the served form (saturated: requests queue, fuse and
    share steps); every request equals its synchronous call and a sample of 8
    equals the oracle."""
    ctx = g.gace_create(0)
    tables, reqs = make_batched(ntables=64, min_rows=1_000_000, max_rows=200_000_000, nprobes=4000, seed=1005,
                                device=cuda)
    tids = [g.gace_load_columns(ctx, t.columns, borrow=True) for t in tables]
    try:
        arrival = np.cumsum(np.random.default_rng(7).exponential(1e5, len(reqs))).astype(np.uint64)
        breqs = to_requests(g, tids, tables, reqs)
        done, st = g.gace_serve_replay(ctx, breqs, arrival, 0)
        assert (st == 0).all() and (done >= arrival).all()
        g.gace_serve_stop(ctx)
        check_against_sync(g, ctx, tids, tables, reqs, breqs)
        _check_oracle_sample(g, orc, tables, reqs, breqs, 8, 30_000_000, 5)
    finally:
        g.gace_destroy(ctx)
        del tables
        _free()
