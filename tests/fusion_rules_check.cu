// Host-only check of the batched form's fusion rules (fusable_probe and
// FusedProbe::fits, no GPU) on one table of four int32 and two int64
// columns: which probe requests may fuse, and with which group, under rules
// 0 (one-predicate probes on one row set alone; members share row sets and
// read a subset of the group's columns), 1 (one-predicate probes too), 2
// (the union of row sets and columns) and 3 (one-predicate probes only on a
// shared hashed row sample; the same row sets, the union of columns), and
// the limits every rule keeps (16 bytes per row, 32 predicates, 32 terms, 8
// row sets).  Prints "ok" or the first failed expectation.
#include <cstdio>
#include <vector>

#include "gace_host.h"

namespace {

int failures = 0;

void expect(bool got, bool want, const char* what, int mode) {
    if (got != want) {
        printf("rule %d: %s: got %d, expected %d\n", mode, what, got, want);
        ++failures;
    }
}

// A probe request of npreds one-term RANGE predicates on the given columns
// (cycled) over the given row sets; the arrays live in the returned holder.
struct Probe {
    std::vector<gace_term> terms;
    std::vector<gace_pred> preds;
    std::vector<gace_sample> samples;
    std::vector<gace_pred_result> results;
    gace_request q{};
    Probe(std::vector<uint32_t> cols, uint32_t npreds, std::vector<gace_sample> smp) : samples(std::move(smp)) {
        for (uint32_t p = 0; p < npreds; ++p) {
            gace_term t{};
            t.col = cols[p % cols.size()];
            t.op = GACE_RANGE;
            t.a.i = 10 * p;
            t.b.i = 10 * p + 5;
            terms.push_back(t);
            preds.push_back({p, 1});
        }
        results.resize(samples.size() * npreds);
        q.kind = GACE_REQ_PROBE;
        q.table_id = 1;
        q.samples = samples.data();
        q.nsamples = static_cast<uint32_t>(samples.size());
        q.terms = terms.data();
        q.nterms = static_cast<uint32_t>(terms.size());
        q.preds = preds.data();
        q.npreds = npreds;
        q.results = results.data();
    }
};

gace_sample full() { return gace_sample{GACE_FULL, 0, 1.0, 0}; }
gace_sample rows(double r, uint64_t seed) { return gace_sample{GACE_ROWS, 0, r, seed}; }
gace_sample blocks(double r) { return gace_sample{GACE_BLOCKS, 4096, r, 9}; }

}  // namespace

int main() {
    TableRec tab;
    tab.nrows = 1000000;
    for (int c = 0; c < 6; ++c) {
        ColumnRec cr;
        cr.dtype = c < 4 ? GACE_I32 : GACE_I64;
        tab.cols.push_back(cr);
    }
    for (int mode = 0; mode <= 3; ++mode) {
        // which requests are candidates at all
        Probe single_full({0}, 1, {full()}), single_rows({0}, 1, {rows(0.01, 42)}), single_blocks({0}, 1, {blocks(0.01)});
        Probe multi({0, 1}, 3, {full()}), many_sets({0}, 2, {full(), rows(0.1, 1)});
        expect(fusable_probe(single_full.q, mode), mode == 1 || mode == 2, "one predicate, full scan", mode);
        expect(fusable_probe(single_rows.q, mode), mode != 0, "one predicate, row sample", mode);
        expect(fusable_probe(single_blocks.q, mode), mode == 1 || mode == 2, "one predicate, block sample", mode);
        expect(fusable_probe(multi.q, mode), true, "three predicates", mode);
        expect(fusable_probe(many_sets.q, mode), true, "two row sets", mode);

        // joining a group seeded by a request on columns 0 and 1, all rows
        FusedProbe grp;
        grp.mode = mode;
        Probe seed({0, 1}, 2, {full()});
        expect(grp.fits(seed.q, tab), true, "an empty group", mode);
        grp.add(0, seed.q, tab);
        Probe subset({1}, 2, {full()}), newcol({2}, 2, {full()}), othersets({0}, 2, {rows(0.1, 1)});
        expect(grp.fits(subset.q, tab), true, "a subset of the group's columns", mode);
        expect(grp.fits(newcol.q, tab), mode >= 2, "a column the group does not read", mode);
        expect(grp.fits(othersets.q, tab), mode == 2, "other row sets", mode);
        // 16 bytes per row at most: columns 0..3 (16 B), then an int64 column
        Probe wide4({0, 1, 2, 3}, 4, {full()}), wide64({4}, 1, {full()});
        FusedProbe g16;
        g16.mode = mode;
        g16.add(0, wide4.q, tab);
        expect(g16.fits(wide64.q, tab), false, "past 16 bytes per row", mode);
        // 32 predicates and 32 terms at most
        Probe p20({0}, 20, {full()}), p13({0}, 13, {full()}), p12({0}, 12, {full()});
        FusedProbe g32;
        g32.mode = mode;
        g32.add(0, p20.q, tab);
        expect(g32.fits(p13.q, tab), false, "past 32 predicates", mode);
        expect(g32.fits(p12.q, tab), true, "32 predicates", mode);
        // 8 row sets at most (rule 2 takes their union)
        if (mode == 2) {
            FusedProbe g8;
            g8.mode = mode;
            std::vector<Probe> ps;
            ps.reserve(9);
            for (int k = 0; k < 9; ++k) ps.emplace_back(std::vector<uint32_t>{0}, 1, std::vector<gace_sample>{rows(0.1, 100 + k)});
            for (int k = 0; k < 8; ++k) {
                expect(g8.fits(ps[k].q, tab), true, "up to 8 row sets", mode);
                g8.add(k, ps[k].q, tab);
            }
            expect(g8.fits(ps[8].q, tab), false, "a ninth row set", mode);
        }
    }
    if (failures) return 1;
    printf("ok\n");
    return 0;
}
