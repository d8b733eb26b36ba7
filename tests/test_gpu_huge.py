"""A table just over 2^31 rows: global row ids beyond int32, and CTAs whose
32-bit counters must not overflow.

One int32 column of 2^31 + 4097 rows (8.6 GB), uniform on [0, 1000).  Three
distinct predicates (a RANGE, an EQ, and a two-term conjunction on the same
column, for PCS) are counted on the full table, a 1 % row sample and a 1 %
sample of 4096-row blocks (seed 42), with marginals, and compared with the
oracle element by element:
  * through a context whose probe launches are capped at one CTA, so that the
    grid-doubling guard must raise the grid until no CTA counts 2^31 rows in
    its 32-bit counters (one call with all three row sets, the narrow
    evaluation; and one single-predicate call per row set);
  * through a context with the full grid, 33 predicates (the three, with the
    RANGE repeated) so that the pass takes the wide evaluation.
The oracle runs once per row set over every row (about a minute in all)."""
import numpy as np
import pytest
import torch

from parity import close
from workloads import BLOCKS, EQ, FULL, I32, RANGE, ROWS, Sample, Term

pytestmark = pytest.mark.gpu

N = 2**31 + 4097
SAMPLES = [Sample(FULL), Sample(ROWS, 0.01, 42), Sample(BLOCKS, 0.01, 42, 4096)]
DISTINCT = [[Term(0, RANGE, 0, 100)], [Term(0, EQ, 7)], [Term(0, RANGE, 0, 500), Term(0, RANGE, 250, 750)]]


@pytest.fixture(scope="module")
def huge(cuda):
    free, _ = torch.cuda.mem_get_info(cuda)
    if free < 12 * 2**30:
        pytest.skip("needs 12 GB of free device memory")
    g = torch.Generator(device=cuda)
    g.manual_seed(2031)
    col = torch.randint(0, 1000, (N,), generator=g, device=cuda, dtype=torch.int32)
    host = col.cpu().numpy()
    yield col, host
    del col
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def oracle_results(orc, huge):
    _, host = huge
    return [orc.probe([host], [I32], DISTINCT, s, marginals=True) for s in SAMPLES]


def _compare(res, marg, ref, pred_map, s):
    """res[s][p] against oracle predicate pred_map[p]; marginals per input term."""
    got = res["match"][s]
    want = np.array([ref.counts[k] for k in pred_map], dtype=np.uint64)
    assert np.array_equal(got, want), (s, got[:5], want[:5])
    assert (res["sample_rows"][s] == ref.n_sample).all()
    for p, k in enumerate(pred_map):
        assert close(float(res["sel"][s][p]), float(ref.counts[k]) / ref.n_sample if ref.n_sample else 0.0)
    return got


def _term_offsets(preds):
    off, out = 0, []
    for p in preds:
        out.append(off)
        off += len(p)
    return out


def test_capped_grid_narrow_and_single(g, orc, huge, oracle_results):
    col, _ = huge
    ctx = g.gace_create(0, max_ctas=1)
    try:
        tid = g.gace_load_columns(ctx, [col], borrow=True)
        # all three row sets in one call: the narrow evaluation
        res, marg = g.gace_probe_batch(ctx, tid, DISTINCT, SAMPLES, [I32], marginals=True)
        offs = _term_offsets(DISTINCT)
        for s, ref in enumerate(oracle_results):
            _compare(res, marg, ref, [0, 1, 2], s)
            assert np.array_equal(marg[s], ref.marginals), s
            pcs = orc.pcs(int(ref.counts[2]), int(ref.marginals[offs[2]]), int(ref.marginals[offs[2] + 1]),
                          ref.n_sample)
            assert close(float(res["pcs"][s][2]), pcs)
        # one predicate on one row set per call: the single-predicate evaluation
        for s, smp in enumerate(SAMPLES):
            r1, m1 = g.gace_probe_batch(ctx, tid, DISTINCT[:1], [smp], [I32], marginals=True)
            ref = oracle_results[s]
            assert int(r1["match"][0][0]) == int(ref.counts[0]), s
            assert int(r1["sample_rows"][0][0]) == ref.n_sample, s
            assert int(m1[0][0]) == int(ref.marginals[0]), s
        g.gace_unload(ctx, tid)
    finally:
        g.gace_destroy(ctx)


def test_full_grid_wide_pass(g, gctx, huge, oracle_results):
    col, _ = huge
    preds = [DISTINCT[0]] * 31 + [DISTINCT[1], DISTINCT[2]]
    pred_map = [0] * 31 + [1, 2]
    tid = g.gace_load_columns(gctx, [col], borrow=True)
    try:
        res, _ = g.gace_probe_batch(gctx, tid, preds, SAMPLES, [I32], marginals=True)
        for s, ref in enumerate(oracle_results):
            _compare(res, None, ref, pred_map, s)
        st = g.gace_stats_read(gctx)
        assert "probe_wide" in st
    finally:
        g.gace_unload(gctx, tid)
