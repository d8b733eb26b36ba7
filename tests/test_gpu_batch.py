"""GPU tests of the batched form (gace_run_batch): every request of a mixed
batch gives exactly what its synchronous call gives (which the other GPU tests
pin to the oracle), a sample of them is checked against the oracle directly,
a replayed graph with new contents stays exact, a bad request fails alone,
and tuning changes nothing but speed."""
import os

import numpy as np
import pytest

from batch_util import check_against_sync as _check_against_sync
from batch_util import to_requests as _to_requests
from parity import close, host_columns
from workloads import (BLOCKS, FULL, I32, RANGE, ROWS, JoinSide, Sample, Table, Term, make_batched,
                       make_join, make_predicates)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batched(g, gctx, cuda):
    tables, reqs = make_batched(ntables=12, min_rows=1000, max_rows=400_000, nprobes=150, seed=11, device=cuda)
    tids = [g.gace_load_columns(gctx, t.columns) for t in tables]
    yield tables, reqs, tids
    for t in tids:
        g.gace_unload(gctx, t)


def test_mixed_batch_equals_synchronous_calls(g, gctx, batched):
    tables, reqs, tids = batched
    breqs = _to_requests(g, tids, tables, reqs)
    st = g.gace_run_batch(gctx, breqs)
    assert st == [0] * len(reqs)
    _check_against_sync(g, gctx, tids, tables, reqs, breqs)
    # replay: same shape, so the captured graph runs again with the same result
    breqs2 = _to_requests(g, tids, tables, reqs)
    g.gace_run_batch(gctx, breqs2)
    for a, b in zip(breqs, breqs2):
        if isinstance(a, g.ProbeRequest):
            assert np.array_equal(a.results["match"], b.results["match"])
        elif isinstance(a, g.NdvRequest):
            assert np.array_equal(a.registers, b.registers)
        else:
            assert a.result == b.result


def test_batch_against_oracle(g, gctx, orc, batched):
    tables, reqs, tids = batched
    pick = [r for r in reqs if r["kind"] != "join"][:25] + [r for r in reqs if r["kind"] == "join"][:4]
    breqs = _to_requests(g, tids, tables, pick)
    g.gace_run_batch(gctx, breqs)
    for r, q in zip(pick, breqs):
        if r["kind"] == "probe":
            t = tables[r["table"]]
            ref = orc.probe(host_columns(t), t.dtypes, r["preds"], r["samples"][0])
            assert np.array_equal(q.results["match"][0], ref.counts)
            assert int(q.results["sample_rows"][0][0]) == ref.n_sample
            assert np.array_equal(q.marginals[0], ref.marginals)
        elif r["kind"] == "ndv":
            t = tables[r["table"]]
            regs = orc.hll_registers(t.columns[r["col"]].cpu(), t.dtypes[r["col"]], r["p"], r["seed"])
            assert np.array_equal(q.registers, regs)
            assert close(q.estimate, orc.hll_estimate(regs, r["p"]))
        else:
            f, d = tables[r["fact"]], tables[r["dim"]]
            fh = Table("f", host_columns(f), f.dtypes)
            dh = Table("d", host_columns(d), d.dtypes)
            rc, card, fp, dp = orc.join_card(JoinSide(fh, 0, r["fact_terms"]), JoinSide(dh, 0, r["dim_terms"]),
                                             r["key_domain"])
            assert rc == 0 and q.result["card"] == card and q.result["fact_rows"] == fp


def test_graph_replay_with_new_contents(g, gctx, batched):
    """Two batches of the same shape but different constants: the second
    replays the first's graph with new staging contents."""
    tables, reqs, tids = batched
    probes = [r for r in reqs if r["kind"] == "probe"][:40]
    moved = []
    for r in probes:
        t = tables[r["table"]]
        preds = make_predicates(t, 1, len(r["preds"][0]), len(r["preds"][0]), seed=hash(str(r)) % 10000)
        moved.append(dict(r, preds=preds))
    for batch in (probes, moved, probes):
        breqs = _to_requests(g, tids, tables, batch)
        g.gace_run_batch(gctx, breqs)
        _check_against_sync(g, gctx, tids, tables, batch, breqs)


@pytest.mark.parametrize("fact_filters", [1, 2])
def test_joins_every_method_and_chain(g, gctx, orc, cuda, fact_filters):
    """Every join method and the chain in one batch, equal to the synchronous
    calls and the oracle; with two fact filters the fact side reads three
    columns (12-byte rows: half-size tiles in the staged side kernel)."""
    f, d, d2 = make_join(n_fact=700_001, n_dim=50_000, n_dim2=5000, seed=5, device=cuda)
    fid, did, d2id = (g.gace_load_columns(gctx, t.columns) for t in (f, d, d2))
    try:
        ft = [Term(1, RANGE, 0, 300)] + ([Term(2, RANGE, 50, 950)] if fact_filters == 2 else [])
        dt, d2t = [Term(2, RANGE, 100, 900)], [Term(1, RANGE, 0, 500)]
        F = g.JoinSideSpec(fid, 0, ft, f.dtypes)
        D = g.JoinSideSpec(did, 0, dt, d.dtypes)
        D2 = g.JoinSideSpec(d2id, 0, d2t, d2.dtypes)
        breqs = []
        for method in (0, 1, 2):
            breqs.append(g.JoinRequest(F, D, 50_000, method=method))
            breqs.append(g.JoinRequest(F, D, 50_000, D2, 5000, 3, method=method))
        assert g.gace_run_batch(gctx, breqs) == [0] * len(breqs)
        for k, q in enumerate(breqs):
            if k % 2 == 0:
                ref = g.gace_join_card(gctx, F, D, 50_000)
            else:
                ref = g.gace_join_card(gctx, F, D, 50_000, D2, 5000, 3)
            assert q.result == ref
        fh, dh, d2h = (Table(t.name, host_columns(t), t.dtypes) for t in (f, d, d2))
        rc, card, *_ = orc.chain_card(JoinSide(fh, 0, ft), JoinSide(dh, 0, dt), 3, JoinSide(d2h, 0, d2t), 50_000, 5000)
        assert rc == 0 and breqs[1].result["card"] == card
    finally:
        for t in (fid, did, d2id):
            g.gace_unload(gctx, t)


def test_bad_request_fails_alone(g, gctx, batched):
    tables, reqs, tids = batched
    good = [r for r in reqs if r["kind"] == "probe"][:3]
    breqs = _to_requests(g, tids, tables, good)
    bad = g.ProbeRequest(tids[0], [[Term(99, RANGE, 0, 1)]], [Sample(FULL)], tables[0].dtypes)
    missing = g.NdvRequest(12345, 0, 12, 1)
    st = g.gace_run_batch(gctx, [breqs[0], bad, breqs[1], missing, breqs[2]], raise_on_error=False)
    assert st[0] == st[2] == st[4] == 0 and st[1] == 1 and st[3] == 6
    _check_against_sync(g, gctx, tids, tables, good, breqs)


def test_tuning_changes_only_speed(g, gctx, batched, tmp_path):
    tables, reqs, tids = batched
    sub = reqs[:60]
    g.gace_tune_batch(gctx, _to_requests(g, tids, tables, sub))
    path = str(tmp_path / "tune.jsonl")
    g.gace_tune_save(gctx, path)
    assert os.path.getsize(path) > 0
    ctx2 = g.gace_create(0)
    try:
        g.gace_tune_load(ctx2, path)
        tids2 = [g.gace_load_columns(ctx2, t.columns, borrow=True) for t in tables]
        breqs = _to_requests(g, tids2, tables, sub)
        g.gace_run_batch(ctx2, breqs)
        _check_against_sync(g, ctx2, tids2, tables, sub, breqs)
    finally:
        g.gace_destroy(ctx2)


def test_empty_batch_and_empty_tables(g, gctx, cuda):
    assert g.gace_run_batch(gctx, []) == []
    import torch
    tid = g.gace_load_columns(gctx, [torch.zeros(0, dtype=torch.int32, device=cuda)])
    try:
        q = [g.ProbeRequest(tid, [[Term(0, RANGE, 0, 5)]], [Sample(FULL), Sample(ROWS, 0.5, 1)], [I32]),
             g.NdvRequest(tid, 0, 10, 3)]
        assert g.gace_run_batch(gctx, q) == [0, 0]
        assert not q[0].results["match"].any() and not q[1].registers.any() and q[1].estimate == 0.0
    finally:
        g.gace_unload(gctx, tid)


def test_fused_probes_on_one_table(g, gctx, batched):
    """Probes on one table run as fused requests (shared scans): more distinct
    row sets than one request holds, marginals wanted by some members only,
    and one member with a bad column, which fails alone."""
    tables, reqs, tids = batched
    t, tid = tables[3], tids[3]
    pool = [Sample(FULL), Sample(ROWS, 0.01, 42), Sample(ROWS, 0.1, 7), Sample(BLOCKS, 0.05, 9, 4096),
            Sample(ROWS, 0.5, 1), Sample(BLOCKS, 0.2, 3, 512), Sample(ROWS, 0.3, 11), Sample(ROWS, 0.7, 12),
            Sample(BLOCKS, 0.5, 5, 100), Sample(ROWS, 1.0, 2)]
    rng = np.random.default_rng(17)
    specs = []
    for i in range(40):
        preds = make_predicates(t, int(rng.integers(1, 4)), 1, 3, seed=500 + i)
        smp = [pool[k] for k in rng.choice(len(pool), int(rng.integers(1, 4)), replace=False)]
        specs.append((preds, smp, bool(rng.random() < 0.5)))
    # members that share row sets and read a subset of one member's columns: fused
    def rng_term(c, k):
        if t.dtypes[c] == I32:
            return Term(c, RANGE, 10 * k, 10 * k + 50_000)
        return Term(c, RANGE, -1.0 + 0.1 * k, 0.5 + 0.1 * k)
    shared = [Sample(ROWS, 0.1, 7), Sample(FULL)]
    specs.append(([[rng_term(1, 0), rng_term(2, 0), rng_term(3, 0)]], shared, True))
    for k in range(1, 12):
        cols = [1 + (k % 3)] if k % 2 else [1, 2 + (k % 2)]
        specs.append(([[rng_term(c, k) for c in cols], [rng_term(cols[0], k + 1)]], shared, bool(k % 3)))
    breqs = [g.ProbeRequest(tid, p, s, t.dtypes, marginals=m) for p, s, m in specs]
    bad = g.ProbeRequest(tid, [[Term(99, RANGE, 0, 1)]], [Sample(FULL)], t.dtypes)
    st = g.gace_run_batch(gctx, breqs[:20] + [bad] + breqs[20:], raise_on_error=False)
    assert st[20] == g.GACE_EINVAL and st[:20] + st[21:] == [0] * len(specs)
    for (preds, smp, m), q in zip(specs, breqs):
        res, marg = g.gace_probe_batch(gctx, tid, preds, smp, t.dtypes, marginals=m)
        for f in ("match", "sample_rows", "sel"):
            assert np.array_equal(q.results[f], res[f])
        assert np.array_equal(q.results["pcs"], res["pcs"], equal_nan=True)
        if m:
            assert np.array_equal(q.marginals, marg)


def _set_fusion_rule(g, ctx, tables, reqs, n, mode, tmp_path):
    """Loads a tuning line that makes batches of this request shape (n
    requests reading these tables' rows) use fusion rule `mode`."""
    import json

    rows = 0
    for r in reqs:
        if r["kind"] == "join":
            rows += tables[r["fact"]].nrows + tables[r["dim"]].nrows
        else:
            rows += tables[r["table"]].nrows
    log2 = lambda x: max(0, int(x).bit_length() - 1)  # noqa: E731
    path = tmp_path / f"fuse{mode}.jsonl"
    path.write_text(json.dumps({"requests_log2": log2(n), "rows_log2": log2(rows), "fuse": mode}) + "\n")
    g.gace_tune_load(ctx, str(path))


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_every_fusion_rule_gives_the_same_results(g, batched, tmp_path, mode):
    """Under each fusion rule (one-predicate probes alone; fused too; groups
    with the union of their members' row sets and columns; fused only on a
    shared row sample, with the union of their columns) every request of
    the mixed batch (planned on the host workers: more than 64 requests)
    gives what its synchronous call gives."""
    tables, reqs, _ = batched
    ctx = g.gace_create(0)
    try:
        tids = [g.gace_load_columns(ctx, t.columns, borrow=True) for t in tables]
        _set_fusion_rule(g, ctx, tables, reqs, len(reqs), mode, tmp_path)
        breqs = _to_requests(g, tids, tables, reqs)
        assert g.gace_run_batch(ctx, breqs) == [0] * len(reqs)
        _check_against_sync(g, ctx, tids, tables, reqs, breqs)
    finally:
        g.gace_destroy(ctx)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_fusion_rules_on_one_table(g, batched, tmp_path, mode):
    """One-predicate probes on one row set, and probes on different row sets
    and columns, fused on one table under rules 1, 2 and 3: each member's counts,
    selectivities, PCS and marginals equal its synchronous call's."""
    tables, _, _ = batched
    t = tables[3]
    pool = [Sample(FULL), Sample(ROWS, 0.01, 42), Sample(BLOCKS, 0.01, 42, 4096), Sample(ROWS, 0.1, 7),
            Sample(BLOCKS, 0.05, 9, 512)]
    rng = np.random.default_rng(23 + mode)
    specs = []
    for i in range(48):
        npred = 1 if i % 3 else int(rng.integers(2, 4))
        preds = make_predicates(t, npred, 1, 4, seed=900 + i)
        smp = [pool[int(rng.integers(0, len(pool)))]] if i % 4 else \
            [pool[k] for k in rng.choice(len(pool), 2, replace=False)]
        specs.append((preds, smp, bool(i % 5 == 0)))
    ctx = g.gace_create(0)
    try:
        tid = g.gace_load_columns(ctx, t.columns, borrow=True)
        pseudo = [{"kind": "probe", "table": 0}] * len(specs)
        _set_fusion_rule(g, ctx, [t], pseudo, len(specs), mode, tmp_path)
        breqs = [g.ProbeRequest(tid, p, s, t.dtypes, marginals=m) for p, s, m in specs]
        assert g.gace_run_batch(ctx, breqs) == [0] * len(specs)
        for (preds, smp, m), q in zip(specs, breqs):
            res, marg = g.gace_probe_batch(ctx, tid, preds, smp, t.dtypes, marginals=m)
            for f in ("match", "sample_rows", "sel"):
                assert np.array_equal(q.results[f], res[f])
            assert np.array_equal(q.results["pcs"], res["pcs"], equal_nan=True)
            if m:
                assert np.array_equal(q.marginals, marg)
    finally:
        g.gace_destroy(ctx)


def test_plain_async_equals_synchronous_calls(g, gctx, batched):
    """The plain path with its calls spread over three contexts (one host
    thread and stream each, request i on context i % 3, each context holding
    the same borrowed columns): every request gives what its synchronous call
    gives, and a bad request fails alone."""
    tables, reqs, tids = batched
    ctxs = [g.gace_create(0) for _ in range(3)]
    try:
        ctids = [[g.gace_load_columns(c, t.columns, borrow=True) for t in tables] for c in ctxs]
        sub = reqs[:90]
        per = [_to_requests(g, ctids[i % 3], tables, [r])[0] for i, r in enumerate(sub)]
        assert g.gace_run_plain_async(ctxs, per) == [0] * len(sub)
        _check_against_sync(g, gctx, tids, tables, sub, per)
        bad = g.NdvRequest(12345, 0, 12, 1)
        st = g.gace_run_plain_async(ctxs, per[:4] + [bad] + per[4:8])
        assert st[4] == g.GACE_ENOTFOUND and st[:4] + st[5:] == [0] * 8
    finally:
        for c in ctxs:
            g.gace_destroy(c)


def test_plain_async_concurrent_sketches_of_different_sizes(g, batched):
    """Sketches of p = 12 and p = 14 (16 KB and 64 KB of shared registers)
    launched at once from four contexts on four host threads: every call
    succeeds (each kernel's shared-memory limit is set once, to the device's
    maximum, not per launch to the launch's own size, which another thread's
    launch could undercut) and gives its synchronous call's registers."""
    tables, _, _ = batched
    ctxs = [g.gace_create(0) for _ in range(4)]
    try:
        ctids = [[g.gace_load_columns(c, t.columns, borrow=True) for t in tables] for c in ctxs]
        for _ in range(3):
            reqs = [g.NdvRequest(ctids[i % 4][i % len(tables)], 0, 12 if (i // 4) % 2 else 14, 5)
                    for i in range(160)]
            assert g.gace_run_plain_async(ctxs, reqs) == [0] * len(reqs)
            for i in range(0, len(reqs), 37):
                regs, est = g.gace_ndv(ctxs[0], ctids[0][i % len(tables)], 0, 12 if (i // 4) % 2 else 14, 5)
                assert np.array_equal(reqs[i].registers, regs) and reqs[i].estimate == est
    finally:
        for c in ctxs:
            g.gace_destroy(c)
