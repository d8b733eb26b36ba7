// gace_batch_host.cpp -- host side of the batched form (gace_run_batch) and
// its autotuner.
//
// A batch of requests is compiled into jobs: a probe into its passes (in the
// wide layout, so one kernel evaluates any of them), an NDV request into one
// HLL job, a join into histogram jobs and, in later phases, the jobs that read
// those histograms (the largest entry for the overflow check, then the gather
// or dot product; a chain adds the weight update between).  Each job is cut
// into items of `chunk` rows.  Everything the kernels read lives in one
// workspace arena:
//
//   [jobs][items][probe arguments, pass inputs, join sides, IN pools]   uploaded
//   [status, queue heads, counters, registers, join scalars]  cleared, read back
//   [join histograms and weights]                                     cleared
//
// The upload, the clearing, one persistent launch per phase and the read-back
// are captured as one CUDA graph and replayed while later batches have the
// same shape (same sizes and addresses); only the pinned staging contents
// change.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <fstream>
#include <limits>
#include <map>
#include <memory>
#include <sstream>
#include <string>
#include <vector>

#include "gace_host.h"
#include "gace_hot.h"

namespace gace {
namespace host {

HostPool::~HostPool() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        stop_ = true;
    }
    wake_.notify_all();
    for (std::thread& t : threads_) t.join();
}

void HostPool::work() {
    uint64_t seen = 0;
    for (;;) {
        const std::function<void(uint32_t)>* fn;
        uint32_t n;
        {
            std::unique_lock<std::mutex> lk(mu_);
            wake_.wait(lk, [&] { return stop_ || gen_ != seen; });
            if (stop_) return;
            seen = gen_;
            fn = fn_;
            n = n_;
        }
        for (uint32_t i = next_.fetch_add(1); i < n; i = next_.fetch_add(1)) (*fn)(i);
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (--busy_ == 0) done_.notify_all();
        }
    }
}

void HostPool::run(uint32_t n, const std::function<void(uint32_t)>& fn) {
    if (threads_.empty()) {
        const unsigned hw = std::thread::hardware_concurrency();
        const unsigned nt = hw > 1 ? std::min(hw - 1, 7u) : 0u;
        for (unsigned t = 0; t < nt; ++t) threads_.emplace_back([this] { work(); });
    }
    if (threads_.empty() || n < 2) {
        for (uint32_t i = 0; i < n; ++i) fn(i);
        return;
    }
    {
        std::lock_guard<std::mutex> lk(mu_);
        fn_ = &fn;
        n_ = n;
        next_.store(0);
        busy_ = static_cast<uint32_t>(threads_.size());
        ++gen_;
    }
    wake_.notify_all();
    for (uint32_t i = next_.fetch_add(1); i < n; i = next_.fetch_add(1)) fn(i);
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return busy_ == 0; });
    fn_ = nullptr;
}

namespace {




int log2_bucket(uint64_t x) {
    int b = 0;
    while (x > 1) {
        x >>= 1;
        ++b;
    }
    return b;
}

}  // namespace

bool fusable_probe(const gace_request& r, int mode) {
    if (r.kind != GACE_REQ_PROBE || !r.samples || r.nsamples == 0 || r.nsamples > kMaxSets) return false;
    // one predicate on one row set runs the register-only single-predicate
    // evaluation, cheaper per row than the narrow evaluation a fused group
    // needs: fusing it trades its bytes for more instructions per row, which
    // pays only where many such requests read one table (modes 1 and 2), or
    // where each of them would hash every row for the same row sample (mode 3)
    if (r.npreds <= 1 && r.nsamples <= 1) {
        if (mode == 0) return false;
        if (mode == 3 && !(r.nsamples == 1 && r.samples[0].kind == GACE_ROWS && r.samples[0].rate > 0.0 &&
                           r.samples[0].rate < 1.0))
            return false;
    }
    if (r.npreds > static_cast<uint32_t>(kNarrowMax) || r.nterms > static_cast<uint32_t>(kNarrowMax)) return false;
    if (r.nin > FusedProbe::kMaxIn) return false;
    if (r.npreds && (!r.preds || !r.results)) return false;
    if (r.nterms && !r.terms) return false;
    // every index must stay inside the member's own arrays once they are concatenated
    for (uint32_t p = 0; p < r.npreds; ++p)
        if (static_cast<uint64_t>(r.preds[p].term_off) + r.preds[p].term_cnt > r.nterms) return false;
    for (uint32_t t = 0; t < r.nterms; ++t)
        if (r.terms[t].op == GACE_IN &&
            (!r.in_values || static_cast<uint64_t>(r.terms[t].in_off) + r.terms[t].in_len > r.nin))
            return false;
    return true;
}

namespace {

bool same_sample(const gace_sample& a, const gace_sample& b) {
    return a.kind == b.kind && a.block_rows == b.block_rows && a.seed == b.seed &&
           memcmp(&a.rate, &b.rate, sizeof(double)) == 0;
}

}  // namespace

uint64_t probe_colmask(const gace_request& r) {
    uint64_t m = 0;
    for (uint32_t t = 0; t < r.nterms; ++t) {
        if (r.terms[t].col >= 64) return ~0ull;
        m |= 1ull << r.terms[t].col;
    }
    return m;
}

namespace {

uint32_t mask_rowbytes(uint64_t m, const TableRec& t) {
    uint32_t b = 0;
    for (uint32_t c = 0; c < 64; ++c)
        if (m >> c & 1) b += c < t.cols.size() ? dtype_width(t.cols[c].dtype) : 1000;
    return b;
}

}  // namespace

bool FusedProbe::fits(const gace_request& r, const TableRec& t) const {
    if (!GACE_FUSE) return false;
    const uint64_t m = probe_colmask(r);
    if (m == ~0ull || mask_rowbytes(colmask | m, t) > kMaxRowBytes) return false;
    if (!members.empty()) {
        if (mode < 2 && (m | colmask) != colmask) return false;  // a new column: no saving on it
        if (mode != 2) {  // the same row sets (rule 2 takes their union)
            if (r.nsamples != members[0].q->nsamples) return false;
            for (uint32_t k = 0; k < r.nsamples; ++k)
                if (!same_sample(r.samples[k], members[0].q->samples[k])) return false;
        }
    }
    if (preds.size() + r.npreds > static_cast<size_t>(kNarrowMax)) return false;
    if (terms.size() + r.nterms > static_cast<size_t>(kNarrowMax)) return false;
    if (in_values.size() + r.nin > kMaxIn) return false;
    size_t nsets = samples.size();
    for (uint32_t s = 0; s < r.nsamples; ++s) {
        bool found = false;
        for (const gace_sample& x : samples) found = found || same_sample(x, r.samples[s]);
        for (uint32_t u = 0; u < s && !found; ++u) found = same_sample(r.samples[u], r.samples[s]);
        if (!found) ++nsets;
    }
    return nsets <= static_cast<size_t>(kMaxSets);
}

void FusedProbe::add(uint32_t index, const gace_request& r, const TableRec& t) {
    tab = &t;
    colmask |= probe_colmask(r);
    Member m;
    m.index = index;
    m.q = &r;
    m.term_off = static_cast<uint32_t>(terms.size());
    m.pred_off = static_cast<uint32_t>(preds.size());
    const uint32_t in_base = static_cast<uint32_t>(in_values.size());
    for (uint32_t t = 0; t < r.nterms; ++t) {
        gace_term x = r.terms[t];
        if (x.op == GACE_IN) x.in_off += in_base;
        terms.push_back(x);
    }
    if (r.nin) in_values.insert(in_values.end(), r.in_values, r.in_values + r.nin);
    for (uint32_t p = 0; p < r.npreds; ++p) {
        gace_pred x = r.preds[p];
        x.term_off += m.term_off;
        preds.push_back(x);
    }
    for (uint32_t s = 0; s < r.nsamples; ++s) {
        uint32_t k = 0;
        while (k < samples.size() && !same_sample(samples[k], r.samples[s])) ++k;
        if (k == samples.size()) samples.push_back(r.samples[s]);
        m.set_map[s] = k;
    }
    table_id = r.table_id;
    members.push_back(m);
}

void FusedProbe::seal() {
    bool want_marg = false;
    for (const Member& m : members) want_marg = want_marg || m.q->term_marginals;
    results.assign(samples.size() * preds.size(), gace_pred_result{});
    marg.assign(want_marg ? samples.size() * terms.size() : 0, 0);
    q = gace_request{};
    q.kind = GACE_REQ_PROBE;
    q.table_id = table_id;
    q.samples = samples.data();
    q.nsamples = static_cast<uint32_t>(samples.size());
    q.terms = terms.data();
    q.nterms = static_cast<uint32_t>(terms.size());
    q.in_values = in_values.data();
    q.nin = static_cast<uint32_t>(in_values.size());
    q.preds = preds.data();
    q.npreds = static_cast<uint32_t>(preds.size());
    q.results = results.data();
    q.term_marginals = want_marg ? marg.data() : nullptr;
}

void FusedProbe::scatter() const {
    const size_t np = preds.size(), nt = terms.size();
    for (const Member& m : members) {
        const gace_request& r = *m.q;
        for (uint32_t s = 0; s < r.nsamples; ++s) {
            for (uint32_t p = 0; p < r.npreds; ++p) r.results[s * r.npreds + p] = results[m.set_map[s] * np + m.pred_off + p];
            if (r.term_marginals)
                for (uint32_t t = 0; t < r.nterms; ++t)
                    r.term_marginals[s * r.nterms + t] = marg[m.set_map[s] * nt + m.term_off + t];
        }
    }
}

gace_status compile_probe(gace_ctx* ctx, const TableRec* tab, const gace_request& q, ReqPlan& rp) {
    rp.q = &q;
    rp.kind = GACE_REQ_PROBE;
    ProbeRequest& r = rp.pr;
    r.samples = q.samples;
    r.nsamples = q.nsamples;
    r.terms = q.terms;
    r.nterms = q.nterms;
    r.in_values = q.in_values;
    r.nin = q.nin;
    r.preds = q.preds;
    r.npreds = q.npreds;
    r.results = q.results;
    r.term_marginals = q.term_marginals;
    if (gace_status s = check_probe_request(r)) return s;
    if (!tab) tab = find_table(ctx, q.table_id);
    if (!tab) return fail(GACE_ENOTFOUND, "table %u is not loaded", q.table_id);
    return plan_probe(ctx, *tab, r, false, rp.plan, kProbeWarps);
}

// Compiles one request (argument checks, plans, join sides).
gace_status compile_request(gace_ctx* ctx, const gace_request& q, ReqPlan& rp) {
    rp.q = &q;
    rp.kind = q.kind;
    if (q.kind == GACE_REQ_PROBE) return compile_probe(ctx, nullptr, q, rp);
    if (q.kind == GACE_REQ_NDV) {
        if (q.p < 4 || q.p > 18) return fail(GACE_EINVAL, "p = %u outside 4..18", q.p);
        TableRec* tab = find_table(ctx, q.table_id);
        if (!tab) return fail(GACE_ENOTFOUND, "table %u is not loaded", q.table_id);
        if (q.col >= tab->cols.size())
            return fail(GACE_EINVAL, "column %u of a %zu-column table", q.col, tab->cols.size());
        rp.tab = tab;
        HllArgs& a = rp.hll;
        a.col = tab->cols[q.col].dptr;
        a.nrows = tab->nrows;
        a.dtype = static_cast<uint32_t>(tab->cols[q.col].dtype);
        a.p = q.p;
        a.seedhash = splitmix64_host(q.hash_seed);
        a.aligned = (reinterpret_cast<uintptr_t>(a.col) & 15u) == 0;
        return GACE_OK;
    }
    if (q.kind != GACE_REQ_JOIN) return fail(GACE_EINVAL, "request kind %u invalid", q.kind);
    if (!q.join || !q.join_out) return fail(GACE_EINVAL, "join or join_out is NULL");
    const gace_join& spec = *q.join;
    rp.spec = spec;
    if (spec.hops != 1 && spec.hops != 2) return fail(GACE_EINVAL, "hops = %u (1 or 2)", spec.hops);
    if (spec.method > GACE_JOIN_GATHER) return fail(GACE_EINVAL, "method %u invalid", spec.method);
    if (spec.key_domain == 0 || spec.key_domain > (1ull << 32))
        return fail(GACE_EINVAL, "key_domain %llu outside 1..2^32", (unsigned long long)spec.key_domain);
    if (spec.hops == 2 && (spec.key_domain2 == 0 || spec.key_domain2 > (1ull << 32)))
        return fail(GACE_EINVAL, "key_domain2 %llu outside 1..2^32", (unsigned long long)spec.key_domain2);
    if (gace_status st = build_side(ctx, spec.fact, "fact", -1, rp.side[0], rp.pool, &rp.tabs[0], nullptr, rp.work[0]))
        return st;
    if (gace_status st = build_side(ctx, spec.dim, "dim", spec.hops == 2 ? static_cast<int>(spec.dim_fk2_col) : -1,
                                    rp.side[1], rp.pool, &rp.tabs[1], &rp.fk2_slot, rp.work[1]))
        return st;
    if (spec.hops == 2)
        if (gace_status st = build_side(ctx, spec.dim2, "dim2", -1, rp.side[2], rp.pool, &rp.tabs[2], nullptr,
                                        rp.work[2]))
            return st;
    rp.hist_dot = spec.method == GACE_JOIN_HIST_DOT;
    if (rp.tabs[1]->nrows >= (1ull << 32) || (rp.tabs[2] && rp.tabs[2]->nrows >= (1ull << 32)))
        return fail(GACE_EINVAL, "a histogrammed dimension has 2^32 or more rows");
    if (rp.hist_dot && rp.tabs[0]->nrows >= (1ull << 32))
        return fail(GACE_EINVAL, "GACE_JOIN_HIST_DOT needs a fact table below 2^32 rows");
    rp.K = spec.key_domain;
    rp.K2 = spec.hops == 2 ? spec.key_domain2 : 0;
    return GACE_OK;
}


// Offsets of a request's data inside the input, small-output and big-output
// regions (relative to each region).
void place_request(ReqPlan& rp, Ws& win, Ws& wsmall, Ws& wbig) {
    if (rp.status != GACE_OK || rp.fused >= 0) return;
    if (rp.kind == GACE_REQ_PROBE) {
        rp.args_off.clear();
        for (Pass& ps : rp.plan.passes) {
            rp.args_off.push_back(win.take(sizeof(ProbeArgs)));
            ps.in_off = win.take(ps.in_bytes);
            ps.out_off = wsmall.take(ps.out_bytes);
        }
    } else if (rp.kind == GACE_REQ_NDV) {
        rp.regs_off = wsmall.take((1ull << rp.hll.p) * 4);
    } else {
        const int nsides = rp.spec.hops == 2 ? 3 : 2;
        for (int i = 0; i < nsides; ++i) rp.side_off[i] = win.take(sizeof(SideArgs));
        rp.pool_off = win.take(rp.pool.size() * 4 + 16);
        rp.sc_off = wsmall.take(64 + 16);  // fact_pass dim_pass dim2_pass sum max_h max_w | status
        rp.hd_off = wbig.take((rp.spec.hops == 2 ? rp.K2 : rp.K) * 4);
        if (rp.spec.hops == 2) rp.w_off = wbig.take(rp.K * 8);
        if (rp.hist_dot) rp.hf_off = wbig.take(rp.K * 4);
    }
}

void shift_request(ReqPlan& rp, uint64_t in_base, uint64_t small_base, uint64_t big_base) {
    if (rp.status != GACE_OK || rp.fused >= 0) return;
    if (rp.kind == GACE_REQ_PROBE) {
        for (uint64_t& o : rp.args_off) o += in_base;
        for (Pass& ps : rp.plan.passes) {
            ps.in_off += in_base;
            ps.out_off += small_base;
        }
    } else if (rp.kind == GACE_REQ_NDV) {
        rp.regs_off += small_base;
    } else {
        for (uint64_t& o : rp.side_off) o += in_base;
        rp.pool_off += in_base;
        rp.sc_off += small_base;
        rp.hd_off += big_base;
        rp.w_off += big_base;
        rp.hf_off += big_base;
    }
}

// The jobs of a request, with device pointers into the arena at dws (dws may
// be null when only the count, units and phases are wanted).
void emit_jobs(ReqPlan& rp, unsigned char* dws, unsigned int* batch_status, std::vector<JobRec>& jobs) {
    if (rp.status != GACE_OK || rp.fused >= 0) return;
    if (rp.kind == GACE_REQ_PROBE) {
        for (size_t k = 0; k < rp.plan.passes.size(); ++k) {
            const Pass& ps = rp.plan.passes[k];
            JobRec jr;
            jr.job.kind = kJobProbe;
            jr.job.probe = reinterpret_cast<const ProbeArgs*>(dws + rp.args_off[k]);
            jr.units = rp.plan.tab->nrows;
            jr.smem = ps.args.smem_bytes;
            if (ps.args.narrow) {
                jr.granule = ps.args.tile_rows;
                jr.cls = kClassProbe;
            }
            jr.family = "batch_probe";
            jr.rows = jr.units;
            jr.bytes = jr.units * ps.rowbytes;
            jr.ops = jr.units * ps.ops_per_row;
            jobs.push_back(jr);
        }
        return;
    }
    if (rp.kind == GACE_REQ_NDV) {
        JobRec jr;
        jr.job.kind = kJobHll;
        jr.job.hll = rp.hll;
        jr.job.hll.regs = reinterpret_cast<uint32_t*>(dws + rp.regs_off);
        jr.job.hll.status = batch_status;
        jr.units = rp.hll.nrows;
        // shared-memory registers: 32-bit up to p = 14, one byte for p = 15, 16
        jr.smem = rp.hll.p <= 14 ? (4u << rp.hll.p) : rp.hll.p <= 16 ? (1u << rp.hll.p) : 0u;
        jr.cost = 2;  // a 64-bit hash and a register check per row
        jr.family = "batch_hll";
        jr.rows = jr.units;
        jr.bytes = jr.units * dtype_width(static_cast<int>(rp.hll.dtype));
        jr.ops = jr.units;
        jobs.push_back(jr);
        return;
    }
    // join: sides point at the pool, the per-request status word and the pass counters
    unsigned long long* sc = reinterpret_cast<unsigned long long*>(dws + rp.sc_off);
    unsigned int* jstatus = reinterpret_cast<unsigned int*>(dws + rp.sc_off + 64);
    const bool two = rp.spec.hops == 2;
    const int nsides = two ? 3 : 2;
    for (int i = 0; i < nsides; ++i) {
        rp.side[i].pool = reinterpret_cast<const uint32_t*>(dws + rp.pool_off);
        rp.side[i].status = jstatus;
        rp.side[i].pass_count = sc + i;
    }
    rp.side[0].domain = rp.K;
    rp.side[1].domain = rp.K;
    if (two) rp.side[2].domain = rp.K2;
    auto side_dev = [&](int i) { return reinterpret_cast<const SideArgs*>(dws + rp.side_off[i]); };
    uint32_t* hd = reinterpret_cast<uint32_t*>(dws + rp.hd_off);
    unsigned long long* w = reinterpret_cast<unsigned long long*>(dws + rp.w_off);
    uint32_t* hf = reinterpret_cast<uint32_t*>(dws + rp.hf_off);
    auto side_job = [&](uint32_t kind, int i, uint32_t phase, uint32_t strict) {
        JobRec jr;
        jr.cost = 2;  // latency-bound: a key's filter, then its weight or histogram update
        if (rp.side[i].stage_bytes) {  // aligned, narrow rows: the staged side kernel, by whole tiles
            jr.cls = kClassSide;
            // global histograms keep a hot-key cache (8 bytes per slot) after the stages
            const bool hot =
                kHotCache && (kind == kJobHist || kind == kJobHistAgg) && rp.side[i].domain <= 0xFFFFFFFFull;
            jr.smem = rp.side[i].smem_bytes + (hot ? 8u << kHotLog : 0u);
            jr.granule = rp.side[i].tile_rows;
        }
        jr.job.kind = kind;
        jr.job.side = side_dev(i);
        jr.job.strict = strict;
        jr.phase = phase;
        jr.units = rp.work[i].rows;
        jr.family = "batch_join";
        jr.rows = rp.work[i].rows;
        jr.bytes = rp.work[i].rows * rp.work[i].rowbytes;
        jr.ops = rp.work[i].rows * rp.work[i].ops_per_row;
        return jr;
    };
    auto vec_job = [&](uint32_t kind, uint64_t n, uint32_t phase, uint64_t bytes_per) {
        JobRec jr;
        jr.job.kind = kind;
        jr.phase = phase;
        jr.units = n;
        jr.family = "batch_join";
        jr.rows = n;
        jr.bytes = n * bytes_per;
        jr.ops = n;
        return jr;
    };
    // small key domains are histogrammed per CTA in shared memory (after the
    // staging buffers when the side's columns stream through the pipeline)
    auto smem_hist = [&](JobRec& jr, int i, uint64_t domain) {
        if (domain > kSmemHistMax) return;
        const SideArgs& sa = rp.side[i];
        const bool staged = sa.stage_bytes && sa.tile_rows % (128u * (kHistThreads / 32)) == 0;
        jr.cls = kClassHist;
        jr.smem = (staged ? sa.smem_bytes : 0u) + static_cast<uint32_t>(domain) * 4u;
        jr.granule = round_up(4 * domain, 128);  // at least 4 rows per bin and item
        if (staged) jr.granule = round_up(jr.granule, sa.tile_rows);
    };
    // phase 0: the dimension histogram the others read (and the fact histogram)
    JobRec h = side_job(kJobHist, two ? 2 : 1, 0, 1);
    h.job.hist = hd;
    smem_hist(h, two ? 2 : 1, two ? rp.K2 : rp.K);
    jobs.push_back(h);
    if (rp.hist_dot) {
        JobRec hfj = side_job(kJobHistAgg, 0, 0, 0);
        hfj.job.hist = hf;
        smem_hist(hfj, 0, rp.K);
        jobs.push_back(hfj);
    }
    // its largest entry for the overflow check
    JobRec mx = vec_job(kJobMax32, two ? rp.K2 : rp.K, 1, 4);
    mx.job.weight = hd;
    mx.job.out = sc + 4;
    jobs.push_back(mx);
    uint32_t last = 1;
    const void* weight = hd;
    if (two) {  // chain weights w[k1] += h_D2[fk2] over the filtered first dimension
        JobRec ch = side_job(kJobChain, 1, 1, 1);
        ch.job.weight = hd;
        ch.job.fk2_slot = rp.fk2_slot;
        ch.job.domain2 = rp.K2;
        ch.job.w64 = w;
        jobs.push_back(ch);
        JobRec mw = vec_job(kJobMax64, rp.K, 2, 8);
        mw.job.weight = w;
        mw.job.out = sc + 5;
        jobs.push_back(mw);
        last = 2;
        weight = w;
    }
    if (rp.hist_dot) {
        JobRec d = vec_job(two ? kJobDot64 : kJobDot32, rp.K, last, two ? 12 : 8);
        d.job.hist = hf;
        d.job.weight = weight;
        d.job.out = sc + 3;
        jobs.push_back(d);
    } else {
        JobRec gj = side_job(two ? kJobGather64 : kJobGather32, 0, last, 0);
        gj.job.weight = weight;
        gj.job.out = sc + 3;
        jobs.push_back(gj);
    }
}

gace_status batch_setup(gace_ctx* ctx) {
    if (ctx->batch_ready) return GACE_OK;
    cudaError_t e = batch_configure(ctx->smem_optin);
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel attributes");
    for (cudaStream_t& a : ctx->batch_aux)
        if (!a && (e = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "batch streams");
    for (int ph = 0; ph < kPhases; ++ph) {
        if (!ctx->batch_fork[ph] &&
            (e = cudaEventCreateWithFlags(&ctx->batch_fork[ph], cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "batch events");
        for (cudaEvent_t& j : ctx->batch_join[ph])
            if (!j && (e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "batch events");
    }
    ctx->batch_ready = true;
    return GACE_OK;
}

uint64_t item_units(const JobRec& jr, uint64_t chunk) {
    uint64_t piece = std::max<uint64_t>(128, chunk / jr.cost);
    if (jr.cls == kClassProbe || jr.cls == kClassSide)
        piece = std::max<uint64_t>(piece, 4 * jr.granule);  // bulk copies overlap
    return round_up(piece, jr.granule);
}

// Items of `chunk` units per job, ordered by phase, then class; the range of
// each (phase, class).
void make_items(const std::vector<JobRec>& jobs, uint64_t chunk, std::vector<BatchItem>& items,
                uint32_t (&pbeg)[kPhases][kClasses], uint32_t (&pcnt)[kPhases][kClasses]) {
    items.clear();
    for (int ph = 0; ph < kPhases; ++ph) {
        for (int c = 0; c < kClasses; ++c) {
            pbeg[ph][c] = static_cast<uint32_t>(items.size());
            for (uint32_t j = 0; j < jobs.size(); ++j) {
                if (jobs[j].phase != static_cast<uint32_t>(ph) || jobs[j].cls != c) continue;
                const uint64_t step = item_units(jobs[j], chunk);
                for (uint64_t b = 0; b < jobs[j].units; b += step) {
                    BatchItem it{};
                    it.job = j;
                    it.begin = b;
                    it.end = std::min(jobs[j].units, b + step);
                    items.push_back(it);
                }
            }
            pcnt[ph][c] = static_cast<uint32_t>(items.size()) - pbeg[ph][c];
        }
    }
}


namespace {

struct BatchRun {
    std::vector<JobRec> jobs;
    std::vector<BatchItem> items;
    uint32_t pbeg[kPhases][kClasses] = {}, pcnt[kPhases][kClasses] = {};
    uint64_t jobs_off = 0, items_off = 0, in_end = 0, small_base = 0, small_end = 0, end = 0;
    uint32_t smem[kClasses] = {};
    int grid[kClasses] = {1, 1, 1, 1};
    uint64_t rows = 0, bytes = 0, ops = 0;
    int launches = 0;
};

// Lays out the arena for `chunk`-unit items and a grid of ctas_per_sm CTAs per
// SM (0 = as many as fit), and writes every input into pinned staging.
gace_status build_batch(gace_ctx* ctx, std::vector<ReqPlan>& rps, uint64_t chunk, int ctas_per_sm, BatchRun& br) {
    br = BatchRun();
    Ws win, wsmall, wbig;
    wsmall.take(512);  // batch status word, queue heads
    for (ReqPlan& rp : rps) place_request(rp, win, wsmall, wbig);
    for (ReqPlan& rp : rps) emit_jobs(rp, nullptr, nullptr, br.jobs);
    // a light batch is cut finer so that it still spreads over every SM:
    // about two items per resident CTA
    uint64_t work = 0;
    for (const JobRec& jr : br.jobs) work += jr.units;
    const uint64_t want = static_cast<uint64_t>(ctx->sms) * 3 * 2;
    chunk = std::max<uint64_t>(128, std::min(chunk, round_up(work / want, 128)));
    make_items(br.jobs, chunk, br.items, br.pbeg, br.pcnt);
    Ws main;
    br.jobs_off = main.take(std::max<size_t>(1, br.jobs.size()) * sizeof(BatchJob));
    br.items_off = main.take(std::max<size_t>(1, br.items.size()) * sizeof(BatchItem));
    const uint64_t in_base = main.take(win.off);
    br.in_end = main.off;
    br.small_base = main.take(wsmall.off);
    br.small_end = main.off;
    const uint64_t big_base = main.take(wbig.off);
    br.end = main.off;
    for (ReqPlan& rp : rps) shift_request(rp, in_base, br.small_base, big_base);
    if (gace_status st = ctx->ensure_ws(br.end)) return st;
    if (gace_status st = ctx->ensure_pin(br.small_end)) return st;
    unsigned char* pin = ctx->pin;
    unsigned char* dws = ctx->ws;
    unsigned int* bstatus = reinterpret_cast<unsigned int*>(dws + br.small_base);
    // inputs: pass tables and argument copies, join sides and pools (each
    // request's into its own staging bytes: a large batch on the workers)
    auto stage_one = [&](uint32_t i) {
        ReqPlan& rp = rps[i];
        if (rp.status != GACE_OK || rp.fused >= 0 || rp.kind != GACE_REQ_PROBE) return;
        for (size_t k = 0; k < rp.plan.passes.size(); ++k) {
            Pass& ps = rp.plan.passes[k];
            stage_pass(ps, pin, dws, bstatus);
            memcpy(pin + rp.args_off[k], &ps.args, sizeof(ProbeArgs));
        }
    };
    const uint32_t nrp = static_cast<uint32_t>(rps.size());
    if (nrp >= kParallelRequests)
        ctx->workers.run(nrp, stage_one);
    else
        for (uint32_t i = 0; i < nrp; ++i) stage_one(i);
    for (const JobRec& jr : br.jobs) br.smem[jr.cls] = std::max(br.smem[jr.cls], jr.smem);
    br.jobs.clear();
    for (ReqPlan& rp : rps) emit_jobs(rp, dws, bstatus, br.jobs);
    for (ReqPlan& rp : rps) {
        if (rp.status != GACE_OK || rp.kind != GACE_REQ_JOIN) continue;
        const int nsides = rp.spec.hops == 2 ? 3 : 2;
        for (int i = 0; i < nsides; ++i) memcpy(pin + rp.side_off[i], &rp.side[i], sizeof(SideArgs));
        if (!rp.pool.empty()) memcpy(pin + rp.pool_off, rp.pool.data(), rp.pool.size() * 4);
    }
    std::vector<BatchJob> jobs(br.jobs.size());
    for (size_t j = 0; j < br.jobs.size(); ++j) {
        jobs[j] = br.jobs[j].job;
        br.rows += br.jobs[j].rows;
        br.bytes += br.jobs[j].bytes;
        br.ops += br.jobs[j].ops;
    }
    if (!jobs.empty()) memcpy(pin + br.jobs_off, jobs.data(), jobs.size() * sizeof(BatchJob));
    if (!br.items.empty()) memcpy(pin + br.items_off, br.items.data(), br.items.size() * sizeof(BatchItem));
    for (int c = 0; c < kClasses; ++c) {
        uint32_t items = 0;
        for (int ph = 0; ph < kPhases; ++ph) {
            items = std::max(items, br.pcnt[ph][c]);
            br.launches += br.pcnt[ph][c] > 0;
        }
        if (!items) continue;
        const int occ = batch_occupancy(br.smem[c], c);
        if (occ < 1)
            return fail(GACE_ECUDA, "batch kernel cannot be resident with %u bytes of shared memory", br.smem[c]);
        const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
        br.grid[c] = std::max(1, ctx->sms * per_sm);
    }
    return GACE_OK;
}

// Upload, clear, one launch per phase, read-back: on stream s.
cudaError_t enqueue_batch(gace_ctx* ctx, const BatchRun& br, cudaStream_t s) {
    unsigned char* dws = ctx->ws;
    unsigned char* pin = ctx->pin;
    cudaError_t e = cudaMemcpyAsync(dws, pin, br.in_end, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(dws + br.small_base, 0, br.end - br.small_base, s)) != cudaSuccess) return e;
    const BatchItem* items = reinterpret_cast<const BatchItem*>(dws + br.items_off);
    const BatchJob* jobs = reinterpret_cast<const BatchJob*>(dws + br.jobs_off);
    unsigned int* heads = reinterpret_cast<unsigned int*>(dws + br.small_base + 256);
    for (int ph = 0; ph < kPhases; ++ph) {
        // a phase's classes on parallel streams (graph branches), joined before the next phase
        if ((e = cudaEventRecord(ctx->batch_fork[ph], s)) != cudaSuccess) return e;
        int branch = 0;
        for (int c = 0; c < kClasses; ++c) {
            if (!br.pcnt[ph][c]) continue;
            cudaStream_t on = branch == 0 ? s : ctx->batch_aux[branch - 1];
            if (branch > 0 && (e = cudaStreamWaitEvent(on, ctx->batch_fork[ph], 0)) != cudaSuccess) return e;
            if ((e = batch_launch(items + br.pbeg[ph][c], br.pcnt[ph][c], jobs, heads + ph * kClasses + c,
                                  br.grid[c], br.smem[c], c, on)) != cudaSuccess)
                return e;
            if (branch > 0) {
                if ((e = cudaEventRecord(ctx->batch_join[ph][branch - 1], on)) != cudaSuccess) return e;
                if ((e = cudaStreamWaitEvent(s, ctx->batch_join[ph][branch - 1], 0)) != cudaSuccess) return e;
            }
            ++branch;
        }
    }
    return cudaMemcpyAsync(pin + br.small_base, dws + br.small_base, br.small_end - br.small_base,
                           cudaMemcpyDeviceToHost, s);
}

// Runs a built batch: through the cached graph when the shape repeats (or a
// new capture), or eagerly; waits for it.
gace_status exec_batch(gace_ctx* ctx, const BatchRun& br, bool use_graph) {
    std::vector<uint64_t> key = {reinterpret_cast<uint64_t>(ctx->ws), reinterpret_cast<uint64_t>(ctx->pin),
                                 br.jobs_off, br.items_off, br.in_end, br.small_base, br.small_end, br.end};
    for (int c = 0; c < kClasses; ++c) {
        key.push_back(br.smem[c]);
        key.push_back(static_cast<uint64_t>(br.grid[c]));
        for (int ph = 0; ph < kPhases; ++ph) {
            key.push_back(br.pbeg[ph][c]);
            key.push_back(br.pcnt[ph][c]);
        }
    }
    auto launch = [&]() -> cudaError_t {
        if (!use_graph) return enqueue_batch(ctx, br, ctx->stream);
        if (!ctx->graph_exec || ctx->graph_key != key) {
            if (ctx->graph_exec) {
                cudaGraphExecDestroy(ctx->graph_exec);
                ctx->graph_exec = nullptr;
            }
            if (!ctx->capture_stream) {
                cudaError_t e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
                if (e != cudaSuccess) return e;
            }
            cudaError_t e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return e;
            cudaError_t ee = enqueue_batch(ctx, br, ctx->capture_stream);
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(ctx->capture_stream, &graph);
            if (ee != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return ee;
            }
            if (e != cudaSuccess) return e;
            e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                ctx->graph_exec = nullptr;
                return e;
            }
            ctx->graph_key = key;
        }
        return cudaGraphLaunch(ctx->graph_exec, ctx->stream);
    };
    CK(ctx->traced("batch", br.rows, br.bytes, br.ops, launch));
    ctx->stats["batch_kernel"].launches += br.launches;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->collect();
    return GACE_OK;
}

}  // namespace

// Outputs of one request from its read-back counters: host_base + offset
// addresses what the request's small-output region held; status is the word
// its probe and HLL jobs reported to.
void finish_request(gace_ctx* ctx, ReqPlan& rp, const unsigned char* host_base, unsigned int status) {
    const unsigned __int128 lim = static_cast<unsigned __int128>(1) << 63;
    if (rp.status != GACE_OK || rp.fused >= 0) return;
    if (rp.kind != GACE_REQ_JOIN && status) {
        rp.status = read_status(ctx, status);
        rp.error = gace_last_error();
        return;
    }
    if (rp.kind == GACE_REQ_PROBE) {
        std::vector<const unsigned long long*> outs;
        for (const Pass& ps : rp.plan.passes)
            outs.push_back(reinterpret_cast<const unsigned long long*>(host_base + ps.out_off));
        assemble_probe(rp.plan, rp.pr, outs);
    } else if (rp.kind == GACE_REQ_NDV) {
        const uint64_t m = 1ull << rp.hll.p;
        const uint32_t* r32 = reinterpret_cast<const uint32_t*>(host_base + rp.regs_off);
        std::vector<uint8_t> regs(m);
        for (uint64_t j = 0; j < m; ++j) regs[j] = static_cast<uint8_t>(r32[j]);
        if (rp.q->registers_out) memcpy(rp.q->registers_out, regs.data(), m);
        if (rp.q->estimate_out) *rp.q->estimate_out = hll_estimate_host(regs.data(), rp.hll.p);
    } else {
        const unsigned long long* h = reinterpret_cast<const unsigned long long*>(host_base + rp.sc_off);
        const unsigned int st = *reinterpret_cast<const unsigned int*>(host_base + rp.sc_off + 64);
        gace_status err = GACE_OK;
        if (st & kStatusKeyDomain)
            err = fail(GACE_EINVAL, "a filtered dimension row has a key outside its domain");
        else if (rp.spec.hops == 1 && static_cast<unsigned __int128>(h[0]) * h[4] >= lim)
            err = fail(GACE_EOVERFLOW, "fact_rows * max h_D >= 2^63");
        else if (rp.spec.hops == 2 && static_cast<unsigned __int128>(h[1]) * h[4] >= lim)
            err = fail(GACE_EOVERFLOW, "dim_rows * max h_D2 >= 2^63");
        else if (rp.spec.hops == 2 && static_cast<unsigned __int128>(h[0]) * h[5] >= lim)
            err = fail(GACE_EOVERFLOW, "fact_rows * max w >= 2^63");
        if (err != GACE_OK) {
            rp.status = err;
            rp.error = gace_last_error();
            return;
        }
        gace_join_result& out = *rp.q->join_out;
        out.card = static_cast<int64_t>(h[3]);
        out.fact_rows = h[0];
        out.dim_rows = h[1];
        out.dim2_rows = rp.spec.hops == 2 ? h[2] : 0;
    }
}

namespace {

// Outputs of every request from the read-back counters.
void finish_batch(gace_ctx* ctx, std::vector<ReqPlan>& rps, const BatchRun& br) {
    const unsigned int bst = *reinterpret_cast<const unsigned int*>(ctx->pin + br.small_base);
    const uint32_t n = static_cast<uint32_t>(rps.size());
    if (n >= kParallelRequests)  // each request's outputs are its own
        ctx->workers.run(n, [&](uint32_t i) { finish_request(ctx, rps[i], ctx->pin, bst); });
    else
        for (ReqPlan& rp : rps) finish_request(ctx, rp, ctx->pin, bst);
}

// Plans of a batch: probes on one table are fused greedily in request order
// (the fused plans follow the n requests' own entries in rps); a fused
// request that does not compile is undone and its members compiled alone,
// so each reports its own error.
gace_status compile_all(gace_ctx* ctx, const gace_request* reqs, uint32_t n, std::vector<ReqPlan>& rps,
                        std::vector<std::unique_ptr<FusedProbe>>& fused, int mode) {
    // one plan per request, then one per fused group (at most one per
    // request): reserved at once, so that appending groups moves no plan
    rps.clear();
    rps.reserve(2 * static_cast<size_t>(n));
    rps.resize(n);
    fused.clear();
    std::vector<bool> alone(n, true);
    // candidates by table, the requests reading the most columns first (they seed the groups)
    std::vector<std::pair<uint32_t, const TableRec*>> cand;
    for (uint32_t i = 0; i < n; ++i) {
        if (!fusable_probe(reqs[i], mode)) continue;
        const TableRec* tab = find_table(ctx, reqs[i].table_id);
        if (tab) cand.emplace_back(i, tab);  // else compiled alone, which reports it
    }
    std::stable_sort(cand.begin(), cand.end(), [&](const auto& a, const auto& b) {
        if (reqs[a.first].table_id != reqs[b.first].table_id) return reqs[a.first].table_id < reqs[b.first].table_id;
        return __builtin_popcountll(probe_colmask(reqs[a.first])) > __builtin_popcountll(probe_colmask(reqs[b.first]));
    });
    size_t table_begin = 0;  // groups of the current table start here in `fused`
    for (size_t c = 0; c < cand.size(); ++c) {
        const uint32_t i = cand[c].first;
        if (c > 0 && reqs[cand[c - 1].first].table_id != reqs[i].table_id) table_begin = fused.size();
        size_t gi = table_begin;
        while (gi < fused.size() && !fused[gi]->fits(reqs[i], *cand[c].second)) ++gi;
        if (gi == fused.size()) {
            fused.push_back(std::make_unique<FusedProbe>());
            fused.back()->mode = mode;
        }
        fused[gi]->add(i, reqs[i], *cand[c].second);
        alone[i] = false;
    }
    std::vector<uint32_t> groups;  // fused groups of two or more members
    for (size_t f = 0; f < fused.size(); ++f) {
        FusedProbe& fp = *fused[f];
        if (fp.members.size() == 1) {  // nothing shared: the request runs as itself
            alone[fp.members[0].index] = true;
            continue;
        }
        fp.seal();
        groups.push_back(static_cast<uint32_t>(f));
    }
    std::vector<uint32_t> lone;
    for (uint32_t i = 0; i < n; ++i)
        if (alone[i]) lone.push_back(i);
    // plans of the groups and of the lone requests: each writes only its own
    // ReqPlan, so a large batch plans them on the host workers
    std::vector<ReqPlan> gplans(groups.size());
    auto plan_one = [&](uint32_t k) {
        if (k < groups.size()) {
            gplans[k].status = compile_request(ctx, fused[groups[k]]->q, gplans[k]);
            return;
        }
        const uint32_t i = lone[k - groups.size()];
        rps[i].status = compile_request(ctx, reqs[i], rps[i]);
        if (rps[i].status != GACE_OK) rps[i].error = gace_last_error();
    };
    const uint32_t ntasks = static_cast<uint32_t>(groups.size() + lone.size());
    bool parallel = ntasks >= kParallelRequests;
    if (parallel) {
        // a table copied at its first use completes its copy here, once, on
        // this thread; the workers then only read the table records
        auto ready = [&](uint32_t id) {
            const TableRec* t = find_table(ctx, id);
            return !t || t->pending.empty();
        };
        for (uint32_t i = 0; i < n && parallel; ++i) {
            const gace_request& q = reqs[i];
            if (q.kind != GACE_REQ_JOIN) {
                parallel = ready(q.table_id);
            } else if (q.join) {
                parallel = ready(q.join->fact.table_id) && ready(q.join->dim.table_id) &&
                           (q.join->hops != 2 || ready(q.join->dim2.table_id));
            }
        }
    }
    if (parallel) {
        const int device = ctx->device;
        ctx->workers.run(ntasks, [&](uint32_t k) {
            cudaSetDevice(device);
            plan_one(k);
        });
    } else {
        for (uint32_t k = 0; k < ntasks; ++k) plan_one(k);
    }
    std::vector<uint32_t> undone;  // members of groups that did not compile
    for (size_t k = 0; k < groups.size(); ++k) {
        const FusedProbe& fp = *fused[groups[k]];
        if (gplans[k].status != GACE_OK) {
            for (const FusedProbe::Member& m : fp.members) undone.push_back(m.index);
            continue;
        }
        for (const FusedProbe::Member& m : fp.members) {
            rps[m.index].kind = GACE_REQ_PROBE;
            rps[m.index].q = &reqs[m.index];
            rps[m.index].fused = static_cast<int>(rps.size());
        }
        rps.push_back(std::move(gplans[k]));
    }
    std::sort(undone.begin(), undone.end());
    for (uint32_t i : undone) {
        rps[i].status = compile_request(ctx, reqs[i], rps[i]);
        if (rps[i].status != GACE_OK) rps[i].error = gace_last_error();
    }
    return GACE_OK;
}

// Members of fused probes take the fused request's status and results.
void finish_fused(std::vector<ReqPlan>& rps, const std::vector<std::unique_ptr<FusedProbe>>& fused, uint32_t n) {
    for (uint32_t i = 0; i < n; ++i) {
        ReqPlan& rp = rps[i];
        if (rp.fused < 0) continue;
        const ReqPlan& fp = rps[rp.fused];
        rp.status = fp.status;
        rp.error = fp.error;
    }
    for (const auto& f : fused)
        if (f->members.size() > 1 && rps[f->members[0].index].fused >= 0 &&
            rps[rps[f->members[0].index].fused].status == GACE_OK)
            f->scatter();
}

// Shape of a batch before it is planned: (log2 requests, log2 rows of the
// tables its requests read), the key of its fusion rules.
std::pair<int, int> request_key(gace_ctx* ctx, const gace_request* reqs, uint32_t n) {
    uint64_t rows = 0;
    auto add = [&](uint32_t id) {
        if (const TableRec* t = find_table_raw(ctx, id)) rows += t->nrows;
    };
    for (uint32_t i = 0; i < n; ++i) {
        const gace_request& q = reqs[i];
        if (q.kind != GACE_REQ_JOIN) {
            add(q.table_id);
        } else if (q.join) {
            add(q.join->fact.table_id);
            add(q.join->dim.table_id);
            if (q.join->hops == 2) add(q.join->dim2.table_id);
        }
    }
    return {log2_bucket(n), log2_bucket(rows)};
}

std::pair<int, int> shape_key(const std::vector<ReqPlan>& rps) {
    uint64_t njobs = 0, units = 0;
    for (const ReqPlan& rp : rps) {
        if (rp.status != GACE_OK || rp.fused >= 0) continue;
        if (rp.kind == GACE_REQ_PROBE) {
            njobs += rp.plan.passes.size();
            units += rp.plan.passes.size() * rp.plan.tab->nrows;
        } else if (rp.kind == GACE_REQ_NDV) {
            njobs += 1;
            units += rp.hll.nrows;
        } else {
            njobs += 4;
            units += rp.work[0].rows + rp.work[1].rows + rp.work[2].rows;
        }
    }
    return {log2_bucket(njobs), log2_bucket(units)};
}


// Statuses of the caller's requests (answered ones succeeded), the sketches
// the batch computed kept; the first failure's status and message.
gace_status report_resident(gace_ctx* ctx, const ResidentBatch& rb, const std::vector<ReqPlan>& rps, uint32_t n_in,
                            gace_status* statuses) {
    const uint32_t n = static_cast<uint32_t>(rb.reqs.size());
    std::vector<gace_status> st(n);
    for (uint32_t k = 0; k < n; ++k) st[k] = rps[k].status;
    rb.keep_sketches(ctx, st);
    if (statuses)
        for (uint32_t i = 0; i < n_in; ++i) statuses[i] = GACE_OK;
    gace_status first = GACE_OK;
    std::string msg;
    for (uint32_t k = 0; k < n; ++k) {
        if (statuses) statuses[rb.index[k]] = st[k];
        if (first == GACE_OK && st[k] != GACE_OK) {
            first = st[k];
            msg = "request " + std::to_string(rb.index[k]) + ": " + rps[k].error;
        }
    }
    if (first != GACE_OK) set_last_error_message(msg.c_str());
    return first;
}

}  // namespace
}  // namespace host
}  // namespace gace

using namespace gace::host;

namespace {

gace_status batch_prologue(gace_ctx* ctx, const gace_request* reqs, uint32_t n) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (n && !reqs) return fail(GACE_EINVAL, "reqs is NULL");
    return batch_setup(ctx);
}

}  // namespace

extern "C" {

gace_status gace_run_batch(gace_ctx* ctx, const gace_request* in, uint32_t n_in, gace_status* statuses) {
    if (!ctx) return fail(GACE_EINVAL, "context is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (gace_status s = batch_prologue(ctx, in, n_in)) return s;
    // host phases into the statistics when kernels are timed (launches =
    // calls, total_ms = wall time of the phase)
    auto t_prev = std::chrono::steady_clock::now();
    auto phase = [&](const char* name) {
        if (!ctx->timing) return;
        const auto t = std::chrono::steady_clock::now();
        gace_ctx::KStat& k = ctx->stats[name];
        k.launches++;
        k.ms += std::chrono::duration<double, std::milli>(t - t_prev).count();
        t_prev = t;
    };
    ResidentBatch rb;
    rb.build(ctx, in, n_in);
    phase("host_batch_resident");
    const gace_request* reqs = rb.reqs.data();
    const uint32_t n = static_cast<uint32_t>(rb.reqs.size());
    std::vector<ReqPlan> rps;
    std::vector<std::unique_ptr<FusedProbe>> fused;
    const auto ft = ctx->fuse_tune.find(request_key(ctx, reqs, n));
    compile_all(ctx, reqs, n, rps, fused, ft == ctx->fuse_tune.end() ? 0 : ft->second);
    phase("host_batch_compile");
    uint64_t chunk = kDefaultChunk;
    int per_sm = 0;
    const auto it = ctx->tune.find(shape_key(rps));
    if (it != ctx->tune.end()) {
        chunk = it->second.chunk;
        per_sm = it->second.ctas_per_sm;
    }
    BatchRun br;
    if (gace_status st = build_batch(ctx, rps, chunk, per_sm, br)) return st;
    phase("host_batch_build");
    if (gace_status st = exec_batch(ctx, br, true)) return st;
    phase("host_batch_run");
    finish_batch(ctx, rps, br);
    finish_fused(rps, fused, n);
    const gace_status rs = report_resident(ctx, rb, rps, n_in, statuses);
    phase("host_batch_finish");
    return rs;
}

gace_status gace_tune_batch(gace_ctx* ctx, const gace_request* in, uint32_t n_in) {
    if (!ctx) return fail(GACE_EINVAL, "context is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (gace_status s = batch_prologue(ctx, in, n_in)) return s;
    ResidentBatch rb;
    rb.build(ctx, in, n_in);
    const gace_request* reqs = rb.reqs.data();
    const uint32_t n = static_cast<uint32_t>(rb.reqs.size());
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    // every fusion rule, each over the grid of chunk sizes and CTAs per SM
    gace_ctx::TuneEntry best;
    best.ms = std::numeric_limits<double>::infinity();
    double best_total = std::numeric_limits<double>::infinity();
    std::pair<int, int> best_key{0, 0};
    int best_mode = 0;
    gace_status rc = GACE_OK;
    for (int mode = 0; mode <= 3 && rc == GACE_OK; ++mode) {
        std::vector<ReqPlan> rps;
        std::vector<std::unique_ptr<FusedProbe>> fused;
        // a rule is ranked by the batch's planning time plus its device time
        const auto t_plan = std::chrono::steady_clock::now();
        compile_all(ctx, reqs, n, rps, fused, mode);
        const double plan_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_plan).count();
        double mode_ms = std::numeric_limits<double>::infinity();
        for (uint64_t chunk = 1ull << 17; chunk <= (1ull << 23) && rc == GACE_OK; chunk <<= 2) {
            for (int per_sm : {1, 2, 0}) {
                BatchRun br;
                if ((rc = build_batch(ctx, rps, chunk, per_sm, br)) != GACE_OK) break;
                double ms = std::numeric_limits<double>::infinity();
                for (int rep = 0; rep < 2 && rc == GACE_OK; ++rep) {
                    cudaEventRecord(a, ctx->stream);
                    cudaError_t e = enqueue_batch(ctx, br, ctx->stream);
                    cudaEventRecord(b, ctx->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(b);
                    float t = 0.f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
                    if (e != cudaSuccess) rc = cuda_fail(e, "tuning run");
                    ms = std::min(ms, static_cast<double>(t));
                }
                mode_ms = std::min(mode_ms, ms);
                if (rc == GACE_OK && plan_ms + ms < best_total) {
                    best_total = plan_ms + ms;
                    best.ms = ms;
                    best.chunk = chunk;
                    best.ctas_per_sm = per_sm;
                    best_key = shape_key(rps);
                    best_mode = mode;
                }
            }
        }
        // each rule's best device time and its planning time, for the caller's record
        static const char* const kNames[4] = {"tune_batch_fuse0", "tune_batch_fuse1", "tune_batch_fuse2",
                                              "tune_batch_fuse3"};
        static const char* const kPlan[4] = {"tune_batch_plan0", "tune_batch_plan1", "tune_batch_plan2",
                                             "tune_batch_plan3"};
        gace_ctx::KStat& k = ctx->stats[kNames[mode]];
        k.launches++;
        k.ms += mode_ms;
        gace_ctx::KStat& kp = ctx->stats[kPlan[mode]];
        kp.launches++;
        kp.ms += plan_ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != GACE_OK) return rc;
    ctx->tune[best_key] = best;
    ctx->fuse_tune[request_key(ctx, reqs, n)] = best_mode;
    // leave the requests' outputs from a run with the chosen configuration
    std::vector<ReqPlan> rps;
    std::vector<std::unique_ptr<FusedProbe>> fused;
    compile_all(ctx, reqs, n, rps, fused, best_mode);
    BatchRun br;
    if (gace_status st = build_batch(ctx, rps, best.chunk, best.ctas_per_sm, br)) return st;
    if (gace_status st = exec_batch(ctx, br, false)) return st;
    finish_batch(ctx, rps, br);
    finish_fused(rps, fused, n);
    return report_resident(ctx, rb, rps, n_in, nullptr);
}

gace_status gace_tune_save(gace_ctx* ctx, const char* path) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (!path) return fail(GACE_EINVAL, "path is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::ofstream f(path);
    if (!f) return fail(GACE_EINVAL, "cannot write %s", path);
    for (const auto& kv : ctx->tune)
        f << "{\"jobs_log2\": " << kv.first.first << ", \"units_log2\": " << kv.first.second
          << ", \"chunk\": " << kv.second.chunk << ", \"ctas_per_sm\": " << kv.second.ctas_per_sm
          << ", \"ms\": " << kv.second.ms << "}\n";
    for (const auto& kv : ctx->fuse_tune)
        f << "{\"requests_log2\": " << kv.first.first << ", \"rows_log2\": " << kv.first.second
          << ", \"fuse\": " << kv.second << "}\n";
    return f ? GACE_OK : fail(GACE_EINVAL, "cannot write %s", path);
}

gace_status gace_tune_load(gace_ctx* ctx, const char* path) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (!path) return fail(GACE_EINVAL, "path is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::ifstream f(path);
    if (!f) return fail(GACE_ENOTFOUND, "cannot read %s", path);
    std::string line;
    while (std::getline(f, line)) {
        int jl = 0, ul = 0, per_sm = 0, mode = 0;
        unsigned long long chunk = 0;
        double ms = 0;
        if (sscanf(line.c_str(), " {\"requests_log2\": %d, \"rows_log2\": %d, \"fuse\": %d", &jl, &ul, &mode) == 3) {
            if (mode >= 0 && mode <= 3) ctx->fuse_tune[{jl, ul}] = mode;
            continue;
        }
        if (sscanf(line.c_str(), " {\"jobs_log2\": %d, \"units_log2\": %d, \"chunk\": %llu, \"ctas_per_sm\": %d, \"ms\": %lf",
                   &jl, &ul, &chunk, &per_sm, &ms) != 5)
            continue;
        if (chunk < 128 || (chunk & (chunk - 1))) continue;  // chunks are powers of two >= 128
        gace_ctx::TuneEntry e;
        e.chunk = chunk;
        e.ctas_per_sm = per_sm;
        e.ms = ms;
        ctx->tune[{jl, ul}] = e;
    }
    return GACE_OK;
}

}  // extern "C"
