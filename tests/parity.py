"""Helpers that run the same probe through the library (C ABI) and the CPU
oracle and compare them element by element."""
import math

import numpy as np

# Selectivities and PCS are one IEEE double expression of identical integers
# on both sides, so they must agree to 1e-12 relative (in practice exactly).
REL_TOL = 1e-12


def close(a: float, b: float) -> bool:
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return a == b or abs(a - b) <= REL_TOL * max(abs(a), abs(b))


def host_columns(table):
    return [c.detach().cpu() if hasattr(c, "detach") else c for c in table.columns]


def check_probe(g, orc, ctx, tid, columns_host, dtypes, preds, samples, marginals=True):
    """Runs one batch on the GPU and checks every count, sample size,
    selectivity, PCS and marginal against the oracle."""
    res, marg = g.gace_probe_batch(ctx, tid, preds, samples, dtypes, marginals=marginals)
    for s, smp in enumerate(samples):
        ref = orc.probe(columns_host, dtypes, preds, smp, marginals=True)
        got = res["match"][s]
        bad = np.nonzero(got != ref.counts)[0]
        assert len(bad) == 0, (f"sample {s} ({smp}): {len(bad)} predicates differ, first {bad[:5]}: "
                               f"gpu {got[bad[:5]]} oracle {ref.counts[bad[:5]]}")
        assert (res["sample_rows"][s] == ref.n_sample).all(), (s, res["sample_rows"][s][:3], ref.n_sample)
        if marginals:
            assert np.array_equal(marg[s], ref.marginals), f"sample {s}: marginals differ"
        off = 0
        for p, pred in enumerate(preds):
            sel = orc.selectivity(int(ref.counts[p]), ref.n_sample)
            assert close(float(res["sel"][s][p]), sel)
            if len(pred) == 2:
                pcs = orc.pcs(int(ref.counts[p]), int(ref.marginals[off]), int(ref.marginals[off + 1]),
                              ref.n_sample)
                assert close(float(res["pcs"][s][p]), pcs), (s, p, res["pcs"][s][p], pcs)
            else:
                assert math.isnan(float(res["pcs"][s][p]))
            off += len(pred)
    return res, marg
