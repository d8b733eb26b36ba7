"""GPU tests of the served form (gace_submit / gace_poll / gace_serve_replay):
every request answered in the mix of a continuous batch gives exactly what its
synchronous call gives, also when admission by memory makes requests wait,
when chunks and steps are tiny (many phases spread over many steps), through
the sketch cache, and through both replay modes; the ticket, unload and stop
rules hold."""
import numpy as np
import pytest

from batch_util import check_against_sync, to_requests
from workloads import FULL, I32, RANGE, Sample, Term, make_batched, make_join

pytestmark = pytest.mark.gpu

POLL_US = 60_000_000


@pytest.fixture(scope="module")
def sctx(g, cuda):
    ctx = g.gace_create(0)
    yield ctx
    g.gace_destroy(ctx)


@pytest.fixture(scope="module")
def served(g, sctx, cuda):
    tables, reqs = make_batched(ntables=10, min_rows=1000, max_rows=300_000, nprobes=120, seed=21, device=cuda)
    tids = [g.gace_load_columns(sctx, t.columns, borrow=True) for t in tables]
    yield tables, reqs, tids
    g.gace_serve_stop(sctx)
    for t in tids:
        g.gace_unload(sctx, t)


def _submit_all(g, ctx, breqs):
    tickets = [g.gace_submit(ctx, q) for q in breqs]
    for t in tickets:
        assert g.gace_poll(ctx, t, POLL_US)
    return tickets


@pytest.mark.parametrize("step_rows,chunk_rows", [(0, 0), (1 << 16, 1 << 12), (300, 128)])
def test_served_equals_synchronous_calls(g, sctx, served, step_rows, chunk_rows):
    tables, reqs, tids = served
    g.gace_serve_start(sctx, step_rows=step_rows, chunk_rows=chunk_rows, sketch_cache=-1, always_step=True,
                        probe_cache=-1)
    try:
        breqs = to_requests(g, tids, tables, reqs)
        _submit_all(g, sctx, breqs)
        check_against_sync(g, sctx, tids, tables, reqs, breqs)
    finally:
        g.gace_serve_stop(sctx)


def test_admission_by_memory(g, sctx, served):
    """A 1 MiB arena and two slots: most requests wait for admission and all
    still come back exact."""
    tables, reqs, tids = served
    g.gace_serve_start(sctx, arena_bytes=1 << 20, max_inflight=2, sketch_cache=-1, always_step=True, probe_cache=-1)
    try:
        pick = reqs[:60]
        breqs = to_requests(g, tids, tables, pick)
        _submit_all(g, sctx, breqs)
        check_against_sync(g, sctx, tids, tables, pick, breqs)
        # a join whose histogram alone exceeds the arena is refused at submission
        f = tables[0]
        big = g.JoinRequest(g.JoinSideSpec(tids[0], 0, [], f.dtypes), g.JoinSideSpec(tids[1], 0, [], tables[1].dtypes),
                            1 << 22)
        with pytest.raises(g.GaceError) as e:
            g.gace_submit(sctx, big)
        assert e.value.status == g.GACE_ENOMEM
    finally:
        g.gace_serve_stop(sctx)


def test_tickets_cache_and_unload(g, sctx, served, cuda):
    tables, reqs, tids = served
    g.gace_serve_start(sctx, step_rows=128, chunk_rows=128, always_step=True)
    try:
        with pytest.raises(g.GaceError) as e:
            g.gace_poll(sctx, 987654321, 0)
        assert e.value.status == g.GACE_ENOTFOUND
        # sketch cache: the second identical NDV request completes at submission
        q1 = g.NdvRequest(tids[2], 1, 12, 77)
        t1 = g.gace_submit(sctx, q1)
        assert g.gace_poll(sctx, t1, POLL_US)
        q2 = g.NdvRequest(tids[2], 1, 12, 77)
        t2 = g.gace_submit(sctx, q2)
        assert g.gace_poll(sctx, t2, 0)
        assert np.array_equal(q1.registers, q2.registers) and q1.estimate == q2.estimate
        regs, est = g.gace_ndv(sctx, tids[2], 1, 12, 77)
        assert np.array_equal(regs, q2.registers) and est == q2.estimate
        # polled tickets are forgotten
        with pytest.raises(g.GaceError):
            g.gace_poll(sctx, t1, 0)
        # a table with a request in flight cannot be unloaded; 128-row steps
        # keep a 1M-row probe on the GPU for thousands of steps
        import torch
        col = torch.arange(1_000_000, dtype=torch.int32, device=cuda)
        tid = g.gace_load_columns(sctx, [col], borrow=True)
        q = g.ProbeRequest(tid, [[Term(0, RANGE, 10, 500_010)]], [Sample(FULL)], [I32])
        t = g.gace_submit(sctx, q)
        with pytest.raises(g.GaceError) as e:
            g.gace_unload(sctx, tid)
        assert e.value.status == g.GACE_EBUSY
        assert g.gace_poll(sctx, t, POLL_US)
        assert int(q.results["match"][0, 0]) == 500_000
        g.gace_unload(sctx, tid)
        # argument errors come back from submission, without a ticket
        with pytest.raises(g.GaceError) as e:
            g.gace_submit(sctx, g.NdvRequest(tids[0], 0, 30, 1))
        assert e.value.status == g.GACE_EINVAL
        with pytest.raises(g.GaceError) as e:
            g.gace_submit(sctx, g.NdvRequest(99999, 0, 12, 1))
        assert e.value.status == g.GACE_ENOTFOUND
    finally:
        g.gace_serve_stop(sctx)


def test_replay_modes(g, sctx, served):
    tables, reqs, tids = served
    pick = reqs[:80]
    rng = np.random.default_rng(5)
    arrival = np.cumsum(rng.exponential(20_000.0, len(pick))).astype(np.uint64)  # 50k requests/s
    for mode in (0, 1):
        breqs = to_requests(g, tids, tables, pick)
        done, st = g.gace_serve_replay(sctx, breqs, arrival, mode)
        assert (st == 0).all()
        assert (done >= arrival).all()
        check_against_sync(g, sctx, tids, tables, pick, breqs)
    g.gace_serve_stop(sctx)


def test_join_chain_served(g, sctx, orc, cuda):
    f, d, d2 = make_join(n_fact=300_001, n_dim=20_000, n_dim2=3000, seed=8, device=cuda)
    fid, did, d2id = (g.gace_load_columns(sctx, t.columns, borrow=True) for t in (f, d, d2))
    try:
        g.gace_serve_start(sctx, step_rows=1 << 15, chunk_rows=1 << 13, always_step=True)
        F = g.JoinSideSpec(fid, 0, [Term(1, RANGE, 0, 300)], f.dtypes)
        D = g.JoinSideSpec(did, 0, [Term(2, RANGE, 100, 900)], d.dtypes)
        D2 = g.JoinSideSpec(d2id, 0, [Term(1, RANGE, 0, 500)], d2.dtypes)
        breqs = []
        for method in (0, 1, 2):
            breqs.append(g.JoinRequest(F, D, 20_000, method=method))
            breqs.append(g.JoinRequest(F, D, 20_000, D2, 3000, 3, method=method))
        _submit_all(g, sctx, breqs)
        one = g.gace_join_card(sctx, F, D, 20_000)
        two = g.gace_join_card(sctx, F, D, 20_000, D2, 3000, 3)
        for k, q in enumerate(breqs):
            assert q.result == (one if k % 2 == 0 else two)
    finally:
        g.gace_serve_stop(sctx)
        for t in (fid, did, d2id):
            g.gace_unload(sctx, t)


def test_destroy_drains_a_running_server(g, served, cuda):
    tables, reqs, _ = served
    ctx = g.gace_create(0)
    tids = [g.gace_load_columns(ctx, t.columns, borrow=True) for t in tables]
    breqs = to_requests(g, tids, tables, reqs[:20])
    tickets = [g.gace_submit(ctx, q) for q in breqs]
    assert tickets == sorted(tickets)
    g.gace_destroy(ctx)  # waits for the queued requests, then frees the arena


@pytest.mark.parametrize("fuse_samples", [False, True])
def test_fused_admission(g, sctx, served, cuda, fuse_samples):
    """Probes on one table that queue up while the GPU is busy are admitted
    together and run as fused requests (shared scans); each member's results
    equal its own synchronous call's.  With fuse_samples, one-predicate probes
    on a shared row sample fuse too."""
    import torch

    from workloads import BLOCKS, ROWS, make_predicates

    tables, reqs, tids = served
    t, tid = tables[4], tids[4]
    col = torch.arange(2_000_000, dtype=torch.int32, device=cuda)
    slow = g.gace_load_columns(sctx, [col], borrow=True)
    pool = [Sample(FULL), Sample(ROWS, 0.01, 42), Sample(ROWS, 0.1, 7), Sample(BLOCKS, 0.05, 9, 4096),
            Sample(ROWS, 0.5, 1), Sample(BLOCKS, 0.2, 3, 512), Sample(ROWS, 0.3, 11), Sample(ROWS, 0.7, 12),
            Sample(BLOCKS, 0.5, 5, 100), Sample(ROWS, 1.0, 2)]
    rng = np.random.default_rng(23)
    specs = []
    for i in range(40):
        preds = make_predicates(t, int(rng.integers(1, 4)), 1, 3, seed=900 + i)
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
    # one-predicate probes on a row sample (fused under fuse_samples)
    for k in range(12):
        preds = make_predicates(t, 1, 1, 4, seed=700 + k)
        specs.append((preds, [Sample(ROWS, 0.01, 42) if k % 3 else Sample(ROWS, 0.1, 7)], bool(k % 2)))
    g.gace_serve_start(sctx, step_rows=4096, chunk_rows=4096, always_step=True, probe_cache=-1,
                       fuse_samples=fuse_samples)
    try:
        hold = g.ProbeRequest(slow, [[Term(0, RANGE, 0, 1000)]], [Sample(FULL)], [I32])
        th = g.gace_submit(sctx, hold)
        breqs = [g.ProbeRequest(tid, p, s, t.dtypes, marginals=m) for p, s, m in specs]
        tickets = [g.gace_submit(sctx, q) for q in breqs]
        g.gace_stats_reset(sctx)
        for tk in tickets + [th]:
            assert g.gace_poll(sctx, tk, POLL_US)
        assert int(hold.results["match"][0, 0]) == 1000
        for (preds, smp, m), q in zip(specs, breqs):
            res, marg = g.gace_probe_batch(sctx, tid, preds, smp, t.dtypes, marginals=m)
            for f in ("match", "sample_rows", "sel"):
                assert np.array_equal(q.results[f], res[f])
            assert np.array_equal(q.results["pcs"], res["pcs"], equal_nan=True)
            if m:
                assert np.array_equal(q.marginals, marg)
    finally:
        g.gace_serve_stop(sctx)
        g.gace_unload(sctx, slow)


def test_request_alone_on_idle_server(g, sctx, served):
    """An idle server runs a lone request through its synchronous call; the
    results are the same, and requests that overlap still take the steps."""
    tables, reqs, tids = served
    g.gace_serve_start(sctx, sketch_cache=-1, probe_cache=-1)
    try:
        g.gace_stats_reset(sctx)
        pick = reqs[:12]
        breqs = to_requests(g, tids, tables, pick)
        for q in breqs:  # one at a time: each finds the server idle
            assert g.gace_poll(sctx, g.gace_submit(sctx, q), POLL_US)
        st = g.gace_stats_read(sctx)
        assert st["serve_alone"]["launches"] == len(pick)
        check_against_sync(g, sctx, tids, tables, pick, breqs)
    finally:
        g.gace_serve_stop(sctx)


def test_probe_result_cache(g, sctx, cuda):
    """A probe whose every count an earlier probe returned (the same
    predicates in another order, spelling and batch) is answered at
    submission with the synchronous call's results; unloading the table
    forgets its counts."""
    import torch

    from workloads import EQ, IN, ROWS

    gen = torch.Generator(device=cuda).manual_seed(5)
    cols = [torch.randint(0, 1000, (2_000_003,), generator=gen, device=cuda, dtype=torch.int32) for _ in range(3)]
    tid = g.gace_load_columns(sctx, cols, borrow=True)
    dt = [I32] * 3
    smp = [Sample(FULL), Sample(ROWS, 0.1, 3)]
    a, b, c, d = (Term(0, RANGE, 10, 400), Term(1, EQ, 7), Term(2, IN, values=(1, 5, 9, 5)),
                  Term(1, RANGE, 0, 500))
    first = [[a, b], [c], [a, d, c]]
    again = [[b, a], [Term(2, IN, values=(9, 1, 5))], [c, d, a], [a, a, b]]  # same conjunctions, other spellings
    g.gace_serve_start(sctx)
    try:
        g.gace_stats_reset(sctx)
        q1 = g.ProbeRequest(tid, first, smp, dt, marginals=True)
        assert g.gace_poll(sctx, g.gace_submit(sctx, q1), POLL_US)
        q2 = g.ProbeRequest(tid, again, smp, dt, marginals=True)
        assert g.gace_poll(sctx, g.gace_submit(sctx, q2), 0)  # complete at submission
        assert g.gace_stats_read(sctx)["serve_probe_cache"]["launches"] == 1
        res, marg = g.gace_probe_batch(sctx, tid, again, smp, dt, marginals=True)
        for f in ("match", "sample_rows", "sel"):
            assert np.array_equal(q2.results[f], res[f])
        assert np.array_equal(q2.results["pcs"], res["pcs"], equal_nan=True)
        assert np.array_equal(q2.marginals, marg)
        # a predicate never measured is not answered from the cache
        q3 = g.ProbeRequest(tid, [[a, c]], smp, dt)
        t3 = g.gace_submit(sctx, q3)
        assert g.gace_poll(sctx, t3, POLL_US)
        assert g.gace_stats_read(sctx)["serve_probe_cache"]["launches"] == 1
        # unloading forgets the table's counts: other data under the same probe
        g.gace_unload(sctx, tid)
        cols2 = [torch.randint(0, 1000, (2_000_003,), generator=gen, device=cuda, dtype=torch.int32) for _ in range(3)]
        tid = g.gace_load_columns(sctx, cols2, borrow=True)
        q4 = g.ProbeRequest(tid, again, smp, dt, marginals=True)
        assert g.gace_poll(sctx, g.gace_submit(sctx, q4), POLL_US)
        res, marg = g.gace_probe_batch(sctx, tid, again, smp, dt, marginals=True)
        assert np.array_equal(q4.results["match"], res["match"]) and np.array_equal(q4.marginals, marg)
    finally:
        g.gace_serve_stop(sctx)
        g.gace_unload(sctx, tid)
