"""Estimation stability vs budget (the paper's Experiment B analogue): over
40 seeds per sample rate, the GPU's sampled sel(A and B) and PCS equal the
oracle's (the samples are the same rows), so their coefficients of variation
agree; and the variation shrinks as the budget grows."""
import math

import numpy as np
import pytest

from parity import host_columns
from workloads import BLOCKS, RANGE, ROWS, Sample, Term, make_plain_small

pytestmark = pytest.mark.gpu


def _cv(x):
    m = x.mean(axis=0)
    return x.std(axis=0) / m


def test_cv_of_sel_and_pcs_equals_oracle(g, gctx, orc, cuda):
    t = make_plain_small(n=300_007, seed=4242, device=cuda)
    host = host_columns(t)
    # a correlated pair (c2 = 7 c1 + noise) and an independent one
    preds = [[Term(1, RANGE, 0, 20), Term(2, RANGE, 0, 140)], [Term(0, RANGE, 0, 300_000), Term(3, RANGE, 0, 30)]]
    seeds = list(range(1, 41))
    tid = g.gace_load_columns(gctx, t.columns)
    try:
        cvs = {}
        for rate, block in ((0.01, 0), (0.1, 0), (0.5, 0), (0.05, 1000)):
            sel_g, pcs_g, sel_o, pcs_o = [], [], [], []
            for b in range(0, len(seeds), 8):
                smp = [Sample(BLOCKS, rate, s, block) if block else Sample(ROWS, rate, s) for s in seeds[b:b + 8]]
                res, marg = g.gace_probe_batch(gctx, tid, preds, smp, t.dtypes, marginals=True)
                for k, sm in enumerate(smp):
                    ref = orc.probe(host, t.dtypes, preds, sm, marginals=True)
                    assert np.array_equal(res["match"][k], ref.counts) and int(res["sample_rows"][k][0]) == ref.n_sample
                    assert np.array_equal(marg[k], ref.marginals)
                    sel_g.append(res["sel"][k].tolist())
                    pcs_g.append(res["pcs"][k].tolist())
                    sel_o.append([orc.selectivity(int(c), ref.n_sample) for c in ref.counts])
                    pcs_o.append([orc.pcs(int(ref.counts[p]), int(ref.marginals[2 * p]), int(ref.marginals[2 * p + 1]),
                                          ref.n_sample) for p in range(len(preds))])
            cg, co = _cv(np.array(sel_g)), _cv(np.array(sel_o))
            pg, po = _cv(np.array(pcs_g)), _cv(np.array(pcs_o))
            for a, b in zip(np.concatenate([cg, pg]), np.concatenate([co, po])):
                assert math.isclose(a, b, rel_tol=1e-12), (rate, a, b)
            cvs[(rate, block)] = cg
        # more budget, less variation (row samples of 1 % vs 50 %)
        assert (cvs[(0.01, 0)] > cvs[(0.5, 0)]).all()
    finally:
        g.gace_unload(gctx, tid)
