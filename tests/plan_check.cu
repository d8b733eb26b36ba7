// Host-only check of the probe planner (plan_probe, no GPU) on a seeded
// predicate batch of the benchmark's shape written by the calling test
// (terms, predicates, IN values, samples as the C structs): for a table of
// 100M rows (so that the batch is rank-coded) and of 1000 rows (not coded),
// every predicate is settled exactly once (a pass counts it, or the rank
// histograms do, or it is never or always true), every pass holds the terms
// of its predicates and keeps the kernel's limits, and every rank code's
// keys are sorted and distinct.  Prints each case, then "ok", or the first
// broken rule.
#include <algorithm>
#include <cstdio>
#include <fstream>
#include <iterator>
#include <set>
#include <string>
#include <vector>

#include "gace_host.h"

namespace {

template <class T>
std::vector<T> load(const std::string& path) {
    std::ifstream f(path, std::ios::binary);
    std::vector<char> b((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
    std::vector<T> v(b.size() / sizeof(T));
    if (!v.empty()) memcpy(v.data(), b.data(), v.size() * sizeof(T));
    return v;
}

int fail_msg(const char* what, uint64_t a, uint64_t b) {
    printf("%s (%llu, %llu)\n", what, (unsigned long long)a, (unsigned long long)b);
    return 1;
}

}  // namespace

int main(int argc, char** argv) {
    if (argc < 2) return fail_msg("usage: plan_check <dir>", 0, 0);
    const std::string d = std::string(argv[1]) + "/";
    auto terms = load<gace_term>(d + "terms.bin");
    auto preds = load<gace_pred>(d + "preds.bin");
    auto ins = load<gace_scalar>(d + "ins.bin");
    auto samples = load<gace_sample>(d + "samples.bin");
    auto dtypes = load<int32_t>(d + "dtypes.bin");
    gace_ctx* ctx = new gace_ctx();
    ctx->sms = 152;
    ctx->smem_optin = 232448;
    ctx->smem_per_sm = 233472;
    for (uint64_t nrows : {100000000ull, 1000ull}) {
        TableRec tab;
        tab.nrows = nrows;
        for (size_t c = 0; c < dtypes.size(); ++c) {
            ColumnRec cr;
            cr.dtype = dtypes[c];
            cr.dptr = reinterpret_cast<void*>(0x100000000ull * (c + 1));
            tab.cols.push_back(cr);
        }
        std::vector<gace_pred_result> results(samples.size() * preds.size());
        std::vector<uint64_t> marg(samples.size() * terms.size());
        ProbeRequest r;
        r.samples = samples.data();
        r.nsamples = static_cast<uint32_t>(samples.size());
        r.terms = terms.data();
        r.nterms = static_cast<uint32_t>(terms.size());
        r.in_values = ins.data();
        r.nin = static_cast<uint32_t>(ins.size());
        r.preds = preds.data();
        r.npreds = static_cast<uint32_t>(preds.size());
        r.results = results.data();
        r.term_marginals = marg.data();
        ProbePlan plan;
        if (plan_probe(ctx, tab, r, false, plan, kWideWarps, true) != GACE_OK) {
            printf("plan failed: %s\n", gace_last_error());
            return 1;
        }
        if (nrows > 1000 && plan.codes.empty()) return fail_msg("a 100M-row batch was not rank-coded", nrows, 0);
        if (nrows == 1000 && !plan.codes.empty()) return fail_msg("a 1000-row batch was rank-coded", nrows, 0);
        // every device predicate in exactly one pass, with its terms
        std::vector<int> seen(preds.size(), 0);
        for (size_t k = 0; k < plan.passes.size(); ++k) {
            const Pass& ps = plan.passes[k];
            if (ps.preds.size() > kPassPreds) return fail_msg("pass predicates over the limit", k, ps.preds.size());
            if (ps.uterms.size() > kPassTerms) return fail_msg("pass terms over the limit", k, ps.uterms.size());
            if (ps.args.smem_bytes > static_cast<uint32_t>(ctx->smem_optin))
                return fail_msg("pass shared memory over the opt-in limit", k, ps.args.smem_bytes);
            const std::set<uint32_t> in_pass(ps.uterms.begin(), ps.uterms.end());
            for (uint32_t p : ps.preds) {
                ++seen[p];
                for (uint32_t u : plan.pred_u[p])
                    if (!in_pass.count(u)) return fail_msg("a predicate's term is missing from its pass", p, u);
            }
        }
        for (size_t p = 0; p < preds.size(); ++p) {
            const int st = plan.pstate[p];
            if (st == 0 && seen[p] != 1) return fail_msg("a device predicate is not in exactly one pass", p, seen[p]);
            if (st != 0 && seen[p] != 0) return fail_msg("a settled predicate is also in a pass", p, st);
            if (st == 3 && (plan.pred_u[p].size() != 1 || !plan.hist_term(plan.pred_u[p][0])))
                return fail_msg("a histogram-counted predicate has no histogram term", p, plan.pred_u[p].size());
            if (st > 3) return fail_msg("a predicate state out of range", p, st);
        }
        // every input term maps to a unique term (or is never true)
        for (size_t t = 0; t < terms.size(); ++t)
            if (plan.t2u[t] != UINT32_MAX && plan.t2u[t] >= plan.uterms.size())
                return fail_msg("a term maps outside the unique terms", t, plan.t2u[t]);
        for (const RankCode& rc : plan.codes) {
            for (size_t i = 1; i < rc.keys.size(); ++i)
                if (rc.keys[i - 1] >= rc.keys[i]) return fail_msg("rank keys not sorted and distinct", rc.col, i);
            if (rc.keys.size() > kRankPlanMax) return fail_msg("too many rank keys", rc.col, rc.keys.size());
        }
        printf("rows %llu: %zu passes, %zu codes\n", (unsigned long long)nrows, plan.passes.size(), plan.codes.size());
    }
    printf("ok\n");
    return 0;
}
