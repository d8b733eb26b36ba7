"""GPU parity of join cardinality (K5/K6): exact int64 against the oracle for
both methods, one and two hops, filters, key types and domain errors."""
import numpy as np
import pytest
import torch

from workloads import EQ, I32, I64, IN, RANGE, JoinSide, Table, Term, make_join

pytestmark = pytest.mark.gpu

METHODS = [0, 1, 2]


def _host(t):
    return Table(t.name, [c.cpu() if hasattr(c, "cpu") else c for c in t.columns], t.dtypes)


def _run(g, ctx, tabs, fact, dim, K, dim2=None, K2=0, fk2=0, method=0):
    fid, fk, ft = fact
    did, dk, dt = dim
    F = g.JoinSideSpec(tabs[fid][0], fk, ft, tabs[fid][1].dtypes)
    D = g.JoinSideSpec(tabs[did][0], dk, dt, tabs[did][1].dtypes)
    D2 = None
    if dim2 is not None:
        d2id, d2k, d2t = dim2
        D2 = g.JoinSideSpec(tabs[d2id][0], d2k, d2t, tabs[d2id][1].dtypes)
    return g.gace_join_card(ctx, F, D, K, D2, K2, fk2, method)


@pytest.fixture(scope="module")
def joined(g, gctx, cuda):
    f, d, d2 = make_join(n_fact=3_000_001, n_dim=100_000, n_dim2=10_000, seed=77, device=cuda)
    tabs = {}
    for name, t in (("f", f), ("d", d), ("d2", d2)):
        tabs[name] = (g.gace_load_columns(gctx, t.columns), t, _host(t))
    yield tabs
    for tid, _, _ in tabs.values():
        g.gace_unload(gctx, tid)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("wf,wd", [(1, 1000), (5, 500), (50, 100), (500, 10), (1000, 1000)])
def test_two_table_join(g, gctx, orc, joined, method, wf, wd):
    ft, dt = [Term(1, RANGE, 0, wf)], [Term(2, RANGE, 0, wd)]
    out = _run(g, gctx, joined, ("f", 0, ft), ("d", 0, dt), 100_000, method=method)
    rc, card, fp, dp = orc.join_card(JoinSide(joined["f"][2], 0, ft), JoinSide(joined["d"][2], 0, dt), 100_000)
    assert rc == 0
    assert (out["card"], out["fact_rows"], out["dim_rows"]) == (card, fp, dp)


@pytest.mark.parametrize("method", METHODS)
def test_chain_join(g, gctx, orc, joined, method):
    ft = [Term(1, RANGE, 0, 300), Term(2, IN, values=tuple(range(0, 1000, 3)))]
    dt = [Term(1, RANGE, 100, 900)]
    d2t = [Term(1, RANGE, 0, 500)]
    out = _run(g, gctx, joined, ("f", 0, ft), ("d", 0, dt), 100_000, dim2=("d2", 0, d2t), K2=10_000,
               fk2=3, method=method)
    rc, card, fp, p1, p2 = orc.chain_card(JoinSide(joined["f"][2], 0, ft), JoinSide(joined["d"][2], 0, dt), 3,
                                          JoinSide(joined["d2"][2], 0, d2t), 100_000, 10_000)
    assert rc == 0
    assert (out["card"], out["fact_rows"], out["dim_rows"], out["dim2_rows"]) == (card, fp, p1, p2)


@pytest.mark.parametrize("method", METHODS)
def test_random_small_joins(g, gctx, orc, method):
    rng = np.random.default_rng(5)
    for trial in range(6):
        nf, nd, K = int(rng.integers(0, 5000)), int(rng.integers(1, 3000)), int(rng.integers(1, 2000))
        kdt = np.int64 if trial % 2 else np.int32
        fk = (rng.zipf(1.2, nf) % (K + 30) - 10).astype(kdt)
        f1 = rng.integers(0, 50, nf).astype(np.int32)
        key = rng.integers(0, K, nd).astype(kdt)
        g1 = rng.integers(0, 50, nd).astype(np.int32)
        fdt = [I64 if kdt == np.int64 else I32, I32]
        F = Table("f", [fk, f1], fdt)
        D = Table("d", [key, g1], fdt)
        fid, did = g.gace_load_columns(gctx, [fk, f1]), g.gace_load_columns(gctx, [key, g1])
        tabs = {"f": (fid, F, F), "d": (did, D, D)}
        try:
            ft = [Term(1, IN, values=tuple(int(x) for x in rng.integers(0, 50, 9)))]
            dt = [Term(1, RANGE, 5, 45), Term(0, RANGE, 0, K)]
            out = _run(g, gctx, tabs, ("f", 0, ft), ("d", 0, dt), K, method=method)
            rc, card, fp, dp = orc.join_card(JoinSide(F, 0, ft), JoinSide(D, 0, dt), K)
            assert rc == 0 and (out["card"], out["fact_rows"], out["dim_rows"]) == (card, fp, dp)
        finally:
            g.gace_unload(gctx, fid)
            g.gace_unload(gctx, did)


def test_dim_key_outside_domain_is_einval(g, gctx, orc, cuda):
    fk = torch.tensor([1, 2, 3], dtype=torch.int32, device=cuda)
    key = torch.tensor([1, 7], dtype=torch.int32, device=cuda)
    fid, did = g.gace_load_columns(gctx, [fk]), g.gace_load_columns(gctx, [key])
    try:
        for method in METHODS:
            with pytest.raises(g.GaceError) as e:
                g.gace_join_card(gctx, g.JoinSideSpec(fid, 0, [], [I32]), g.JoinSideSpec(did, 0, [], [I32]), 5,
                                 method=method)
            assert e.value.status == 1
        # filtered away: accepted and equal to the oracle
        dt = [Term(0, RANGE, 0, 5)]
        out = g.gace_join_card(gctx, g.JoinSideSpec(fid, 0, [], [I32]), g.JoinSideSpec(did, 0, dt, [I32]), 5)
        F = Table("f", [fk.cpu()], [I32])
        D = Table("d", [key.cpu()], [I32])
        rc, card, _, _ = orc.join_card(JoinSide(F, 0, []), JoinSide(D, 0, dt), 5)
        assert rc == 0 and out["card"] == card == 1
    finally:
        g.gace_unload(gctx, fid)
        g.gace_unload(gctx, did)


def test_always_false_filter(g, gctx, cuda):
    fk = torch.arange(100, dtype=torch.int32, device=cuda)
    fid = g.gace_load_columns(gctx, [fk])
    try:
        for method in METHODS:
            out = g.gace_join_card(gctx, g.JoinSideSpec(fid, 0, [Term(0, EQ, 2**40)], [I32]),
                                   g.JoinSideSpec(fid, 0, [], [I32]), 100, method=method)
            assert out == {"card": 0, "fact_rows": 0, "dim_rows": 100, "dim2_rows": 0}
    finally:
        g.gace_unload(gctx, fid)


@pytest.mark.parametrize("method", METHODS)
def test_skewed_keys_small_domain(g, gctx, orc, cuda, method):
    """A dimension of 4M rows whose keys are Zipf-skewed over a 4096-key
    domain (a quarter of the rows on key 0), and a fact of 6M rows over the
    same domain: the dimension (and, for the dot product, the fact) histogram
    runs per CTA in shared memory; counts equal the oracle's."""
    from workloads import I32, zipf_column, uniform_int_column
    from workloads.gen import _gen

    gen = _gen(4242, cuda)
    K = 4096
    dk = zipf_column(4_000_000, 1.3, K, gen, cuda)
    d1 = uniform_int_column(4_000_000, 0, 100, gen, cuda)
    fk = zipf_column(6_000_000, 1.1, K, gen, cuda)
    f1 = uniform_int_column(6_000_000, 0, 100, gen, cuda)
    assert float((dk == 0).float().mean()) > 0.2
    d = Table("d", [dk, d1], [I32, I32])
    f = Table("f", [fk, f1], [I32, I32])
    did, fid = g.gace_load_columns(gctx, d.columns), g.gace_load_columns(gctx, f.columns)
    try:
        for wd, wf in ((100, 100), (30, 70)):
            dt, ft = [Term(1, RANGE, 0, wd)], [Term(1, RANGE, 0, wf)]
            out = g.gace_join_card(gctx, g.JoinSideSpec(fid, 0, ft, f.dtypes), g.JoinSideSpec(did, 0, dt, d.dtypes),
                                   K, None, 0, 0, method)
            rc, card, fp, dp = orc.join_card(JoinSide(_host(f), 0, ft), JoinSide(_host(d), 0, dt), K)
            assert rc == 0
            assert (out["card"], out["fact_rows"], out["dim_rows"]) == (card, fp, dp)
    finally:
        g.gace_unload(gctx, did)
        g.gace_unload(gctx, fid)


@pytest.mark.parametrize("method", METHODS)
def test_staged_and_direct_sides(g, gctx, orc, cuda, method):
    """The same join over 16-byte aligned columns (staged scans) and over
    columns borrowed one element off alignment (direct loads), with int64
    keys and float32, int64 and IN filters on several columns: both equal the
    oracle, row counts included, over ragged tile tails."""
    from workloads import F32

    gen = torch.Generator(device=cuda).manual_seed(31)
    nf, nd, K = 1_000_003, 50_001, 50_000
    fk = torch.randint(-3, K + 3, (nf + 1,), generator=gen, device=cuda, dtype=torch.int64)
    f1 = torch.rand(nf + 1, generator=gen, device=cuda, dtype=torch.float32)
    f2 = torch.randint(0, 1000, (nf + 1,), generator=gen, device=cuda, dtype=torch.int64)
    dk = torch.randint(0, K, (nd + 1,), generator=gen, device=cuda, dtype=torch.int64)
    d1 = torch.randint(0, 100, (nd + 1,), generator=gen, device=cuda, dtype=torch.int32)
    fdt, ddt = [I64, F32, I64], [I64, I32]
    ft = [Term(1, RANGE, 0.25, 0.75), Term(2, RANGE, 100, 899), Term(2, IN, values=tuple(range(0, 1000, 2)))]
    dt = [Term(1, RANGE, 10, 60)]
    results = []
    for aligned in (True, False):  # the same values: copies, then views one element in
        fcols = [fk[1:], f1[1:], f2[1:]]
        dcols = [dk[1:], d1[1:]]
        if aligned:
            fcols, dcols = [c.clone() for c in fcols], [c.clone() for c in dcols]
        fid, did = g.gace_load_columns(gctx, fcols, borrow=True), g.gace_load_columns(gctx, dcols, borrow=True)
        try:
            out = g.gace_join_card(gctx, g.JoinSideSpec(fid, 0, ft, fdt), g.JoinSideSpec(did, 0, dt, ddt), K,
                                   None, 0, 0, method)
            F = Table("f", [c.cpu() for c in fcols], fdt)
            D = Table("d", [c.cpu() for c in dcols], ddt)
            rc, card, fp, dp = orc.join_card(JoinSide(F, 0, ft), JoinSide(D, 0, dt), K)
            assert rc == 0
            assert (out["card"], out["fact_rows"], out["dim_rows"]) == (card, fp, dp), aligned
            results.append(out)
        finally:
            g.gace_unload(gctx, fid)
            g.gace_unload(gctx, did)
    assert results[0] == results[1]


@pytest.mark.parametrize("method", METHODS)
def test_skewed_keys_large_domain(g, gctx, orc, cuda, method):
    """Zipf(1.3) keys over a 200 000-key domain (above the shared-memory
    histogram's): the global histograms keep their hot keys in each CTA's
    shared-memory cache; counts equal the oracle's, plain and batched."""
    from workloads import I32, uniform_int_column, zipf_column
    from workloads.gen import _gen

    gen = _gen(5151, cuda)
    K = 200_000
    d = Table("d", [zipf_column(3_000_000, 1.3, K, gen, cuda), uniform_int_column(3_000_000, 0, 100, gen, cuda)],
              [I32, I32])
    f = Table("f", [zipf_column(5_000_000, 1.1, K, gen, cuda), uniform_int_column(5_000_000, 0, 100, gen, cuda)],
              [I32, I32])
    did, fid = g.gace_load_columns(gctx, d.columns), g.gace_load_columns(gctx, f.columns)
    try:
        dt, ft = [Term(1, RANGE, 0, 70)], [Term(1, RANGE, 10, 90)]
        F, D = g.JoinSideSpec(fid, 0, ft, f.dtypes), g.JoinSideSpec(did, 0, dt, d.dtypes)
        out = g.gace_join_card(gctx, F, D, K, None, 0, 0, method)
        rc, card, fp, dp = orc.join_card(JoinSide(_host(f), 0, ft), JoinSide(_host(d), 0, dt), K)
        assert rc == 0
        assert (out["card"], out["fact_rows"], out["dim_rows"]) == (card, fp, dp)
        q = g.JoinRequest(F, D, K, method=method)
        assert g.gace_run_batch(gctx, [q]) == [0]
        assert q.result == out
    finally:
        g.gace_unload(gctx, did)
        g.gace_unload(gctx, fid)
