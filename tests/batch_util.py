"""Shared by the batched and served GPU tests: request objects from the
generated workload, and the check that each request's outputs equal its
synchronous call's (which the other GPU tests pin to the oracle)."""
import numpy as np


def to_requests(g, tids, tables, reqs):
    out = []
    for r in reqs:
        if r["kind"] == "probe":
            t = tables[r["table"]]
            out.append(g.ProbeRequest(tids[r["table"]], r["preds"], r["samples"], t.dtypes, marginals=True))
        elif r["kind"] == "ndv":
            out.append(g.NdvRequest(tids[r["table"]], r["col"], r["p"], r["seed"]))
        else:
            f, d = tables[r["fact"]], tables[r["dim"]]
            out.append(g.JoinRequest(g.JoinSideSpec(tids[r["fact"]], 0, r["fact_terms"], f.dtypes),
                                     g.JoinSideSpec(tids[r["dim"]], 0, r["dim_terms"], d.dtypes),
                                     r["key_domain"]))
    return out


def check_against_sync(g, gctx, tids, tables, reqs, breqs):
    for r, q in zip(reqs, breqs):
        if r["kind"] == "probe":
            t = tables[r["table"]]
            res, marg = g.gace_probe_batch(gctx, tids[r["table"]], r["preds"], r["samples"], t.dtypes, marginals=True)
            for f in ("match", "sample_rows", "sel"):
                assert np.array_equal(q.results[f], res[f]), (r, f)
            assert np.array_equal(q.results["pcs"], res["pcs"], equal_nan=True)
            assert np.array_equal(q.marginals, marg)
        elif r["kind"] == "ndv":
            regs, est = g.gace_ndv(gctx, tids[r["table"]], r["col"], r["p"], r["seed"])
            assert np.array_equal(q.registers, regs) and q.estimate == est
        else:
            f, d = tables[r["fact"]], tables[r["dim"]]
            ref = g.gace_join_card(gctx, g.JoinSideSpec(tids[r["fact"]], 0, r["fact_terms"], f.dtypes),
                                   g.JoinSideSpec(tids[r["dim"]], 0, r["dim_terms"], d.dtypes), r["key_domain"])
            assert q.result == ref, (r, q.result, ref)
