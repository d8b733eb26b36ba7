"""Tables whose copy is deferred to their first probe (GACE_COPY_ON_FIRST_PROBE).

The first probe of such a table streams it in row chunks on a second stream
while every pass runs on the chunks already copied; row ids stay table-global,
so row and block samples (and the tile skipping of block samples) are the
ones of the whole table.  Every result must equal the oracle's, for wide,
narrow and single-predicate passes, whichever call reads the table first."""
import numpy as np
import pytest

from parity import check_probe, close, host_columns
from workloads import BLOCKS, FULL, I64, RANGE, ROWS, Sample, Term, make_predicates, make_skew_corr

pytestmark = pytest.mark.gpu

SAMPLES = [Sample(FULL), Sample(ROWS, 0.01, 42), Sample(BLOCKS, 0.01, 42, 4096), Sample(BLOCKS, 0.05, 9, 3000)]


@pytest.fixture(scope="module")
def table():
    # 3M rows on the host: three chunks of 2^20 rows, the last one ragged
    t = make_skew_corr(n=3_000_017, seed=88, device="cpu", domain=50_000)
    return t, host_columns(t)


@pytest.mark.parametrize("npreds", [48, 12])  # wide, narrow
def test_first_probe_streams_the_table(g, gctx, orc, table, npreds):
    t, host = table
    preds = make_predicates(t, npreds, 1, 3, seed=700 + npreds)
    tid = g.gace_load_columns(gctx, [c.numpy() for c in t.columns], copy_on_first_probe=True)
    try:
        check_probe(g, orc, gctx, tid, host, t.dtypes, preds, SAMPLES)  # the streamed first probe
        check_probe(g, orc, gctx, tid, host, t.dtypes, preds, SAMPLES)  # the table is resident now
        regs, est = g.gace_ndv(gctx, tid, 4, 12, 3)
        ref = orc.hll_registers(host[4], I64, 12, 3)
        assert np.array_equal(regs, ref) and close(est, orc.hll_estimate(ref, 12))
    finally:
        g.gace_unload(gctx, tid)


@pytest.mark.parametrize("smp", [Sample(FULL), Sample(ROWS, 0.1, 5), Sample(BLOCKS, 0.02, 5, 8192)])
def test_single_predicate_first(g, gctx, orc, table, smp):
    t, host = table
    preds = [[Term(0, RANGE, 0, 300), Term(6, RANGE, -0.5, 1.0)]]
    tid = g.gace_load_columns(gctx, [c.numpy() for c in t.columns], copy_on_first_probe=True)
    try:
        check_probe(g, orc, gctx, tid, host, t.dtypes, preds, [smp])
    finally:
        g.gace_unload(gctx, tid)


def test_other_calls_complete_the_copy_first(g, gctx, orc, table):
    t, host = table
    tid = g.gace_load_columns(gctx, [c.numpy() for c in t.columns], copy_on_first_probe=True)
    try:
        regs, _ = g.gace_ndv(gctx, tid, 0, 14, 42)  # not a probe: the whole copy, then the sketch
        assert np.array_equal(regs, orc.hll_registers(host[0], t.dtypes[0], 14, 42))
        check_probe(g, orc, gctx, tid, host, t.dtypes, make_predicates(t, 40, 1, 4, seed=77), SAMPLES)
    finally:
        g.gace_unload(gctx, tid)
    # unloading a table that was never read
    tid = g.gace_load_columns(gctx, [c.numpy() for c in t.columns], copy_on_first_probe=True)
    g.gace_unload(gctx, tid)


def test_first_probe_with_the_resident_store(g, orc, table):
    """With the store on, a sampled probe completes the copy, then reads the
    resident sample."""
    t, host = table
    ctx = g.gace_create(0)
    try:
        g.gace_resident_configure(ctx, 1 << 30)
        tid = g.gace_load_columns(ctx, [c.numpy() for c in t.columns], copy_on_first_probe=True)
        check_probe(g, orc, ctx, tid, host, t.dtypes, make_predicates(t, 20, 1, 3, seed=78), SAMPLES)
        assert g.gace_resident_stats_read(ctx)["admitted"] == 3
    finally:
        g.gace_destroy(ctx)


def test_device_columns_are_refused(g, gctx, cuda):
    import torch

    col = torch.arange(1000, dtype=torch.int32, device=cuda)
    with pytest.raises(g.GaceError) as e:
        g.gace_load_columns(gctx, [col], copy_on_first_probe=True)
    assert e.value.status == g.GACE_EINVAL
