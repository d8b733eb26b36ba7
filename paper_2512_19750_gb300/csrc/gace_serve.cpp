// gace_serve.cpp -- the served form: continuous batching of requests that
// arrive one at a time (gace_submit / gace_poll) and an open-loop load driver
// (gace_serve_replay).
//
// A request is copied, checked and compiled at submission (the same plans,
// jobs and phases as the batched form) and laid out as one block:
//
//   [inputs: probe arguments, pass tables, join sides, IN pools]  uploaded once
//   [small outputs: status word, counters, HLL registers, join scalars]  cleared, gathered at the end
//   [big state: join histograms and chain weights]                cleared
//
// The scheduler thread admits queued requests in arrival order while their
// blocks fit in the arena (first fit) and fewer than max_inflight are in
// flight.  Each step takes chunks round-robin from every admitted request's
// current phase until step_rows units are taken; a request's next phase
// starts in a later step than the one that issued its previous phase's last
// chunk, which stream order then guarantees has finished.  One step is, on
// the server's stream:
//
//   upload [queue head | new inputs | items | jobs | scatter | gather]
//   k_copy   scatter: new inputs into their blocks, zero their outputs
//   k_batch  the step's items over the persistent work queue
//   k_copy   gather: the small outputs of requests whose last chunk ran
//   read-back of the gathered outputs, then an event
//
// Two steps are in flight at once (double-buffered staging); a finished
// step's requests are assembled on the host, their blocks freed, and their
// tickets completed.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "gace_host.h"

namespace gace {
namespace host {

namespace {

constexpr uint64_t kDefaultArena = 1ull << 30;
constexpr uint32_t kDefaultInflight = 4096;
constexpr int32_t kDefaultSketches = 1024;
constexpr int32_t kDefaultProbeCounts = 1 << 16;
// Only probes of at most this many (predicate, sample) counts go through the
// count cache (the gate's small probes): keying a large batch's every count
// would cost the scheduler more than the cache saves.
constexpr uint64_t kCachedProbeMaxCounts = 256;
constexpr uint64_t kDefaultStepRows = 1ull << 29;
constexpr uint64_t kDefaultServeChunk = 1ull << 18;
constexpr uint64_t kCopyPiece = 1ull << 16;    // bytes per scatter / gather descriptor
constexpr size_t kMaxStepItems = 1u << 16;     // items per step
constexpr uint64_t kCtasPerSmGuess = 3;         // resident batch CTAs per SM, for sizing light steps
constexpr uint64_t kItemsPerCta = 2;
constexpr size_t kDirectCopies = 2;             // at most this many blocks moved by plain copies per step
constexpr uint64_t kDirectBlockMax = 256u << 10;
constexpr uint64_t kSpinNs = 500000;            // busy-wait on a step's completion before sleeping
constexpr uint64_t kIdleSpinUs = 10000;         // an idle scheduler watches the queue this long before sleeping
                                                // (gace_serve_config.idle_spin_us = 0)

uint64_t now_ns() {
    return static_cast<uint64_t>(std::chrono::duration_cast<std::chrono::nanoseconds>(
                                     std::chrono::steady_clock::now().time_since_epoch())
                                     .count());
}

// A request with its own copies of every input array.
struct OwnedRequest {
    gace_request q{};
    std::vector<gace_sample> samples;
    std::vector<gace_term> terms;
    std::vector<gace_scalar> in_values;
    std::vector<gace_pred> preds;
    gace_join join{};
    std::vector<gace_term> side_terms[3];
    std::vector<gace_scalar> side_in[3];

    template <typename T>
    static const T* own(std::vector<T>& v, const T* src, uint64_t n) {
        if (!src) return nullptr;  // the request's checks report a NULL array with n > 0
        v.assign(src, src + n);
        return v.data();
    }

    void copy_from(const gace_request& r) {
        q = r;
        if (r.kind == GACE_REQ_PROBE) {
            q.samples = own(samples, r.samples, r.nsamples);
            q.terms = own(terms, r.terms, r.nterms);
            q.in_values = own(in_values, r.in_values, r.nin);
            q.preds = own(preds, r.preds, r.npreds);
        } else if (r.kind == GACE_REQ_JOIN && r.join) {
            join = *r.join;
            gace_join_side* sides[3] = {&join.fact, &join.dim, &join.dim2};
            for (int i = 0; i < 3; ++i) {
                sides[i]->terms = own(side_terms[i], sides[i]->terms, sides[i]->nterms);
                sides[i]->in_values = own(side_in[i], sides[i]->in_values, sides[i]->nin);
            }
            q.join = &join;
        }
    }
};

// Where a replayed request's completion goes.
struct ReplaySink {
    uint64_t t0 = 0;
    uint64_t* done_ns = nullptr;
    gace_status* statuses = nullptr;
    uint32_t remaining = 0;  // guarded by ServeState::mu
};

struct SketchKey {
    uint32_t table, col, p;
    uint64_t seed;
    bool operator<(const SketchKey& o) const {
        return std::tie(table, col, p, seed) < std::tie(o.table, o.col, o.p, o.seed);
    }
};

// A count a finished probe returned (a predicate's match, a term's marginal,
// a sample's size), kept for reuse (Section V, item 3: probe results cached
// by bind value); keyed by count_key.
struct CountEntry {
    uint64_t value;
    uint32_t table;
    std::list<std::string>::iterator lru;
};

struct Sketch {
    std::vector<uint8_t> regs;
    double estimate = 0.0;
    std::list<SketchKey>::iterator lru;
};

// One request from submission to completion.
struct Live {
    uint64_t ticket = 0;
    OwnedRequest req;
    ReqPlan rp;
    // tracing: submission, admission, the enqueue of the step with its last chunk
    uint64_t t_submit = 0, t_admit = 0, t_last = 0;
    uint32_t tables[3] = {0, 0, 0};
    int ntables = 0;
    // block layout (offsets from the block's start)
    uint64_t in_bytes = 0, small_rel = 0, small_bytes = 0, block_bytes = 0;
    uint64_t block = ~0ull;  // arena offset once admitted
    // device form, after admission
    std::vector<JobRec> jobs;
    uint32_t phase_list[kPhases] = {0, 0, 0};
    int nphases = 0;
    // issue state
    int pi = -1;                     // index into phase_list
    std::vector<uint32_t> pjobs;     // jobs of the current phase with units
    size_t jk = 0;                   // next job of pjobs
    uint64_t unit = 0;               // next unit of that job
    int64_t last_step = -1;          // step that issued the current phase's last chunk
    bool issued_all = false;
    int64_t step_stamp = -1;         // step whose job table holds this request's jobs
    uint32_t step_job_base = 0;
    // completion
    ReplaySink* sink = nullptr;
    uint32_t sink_index = 0;
    bool cacheable = false;
    bool keep_resident = false;  // an NDV request whose sketch the resident store keeps
    bool finished = false;
    bool fusable = false;  // a probe that may share its table's scan with others
    // a fused group: the members' predicates run as one request (fp); the
    // members keep their tickets and table references
    std::unique_ptr<FusedProbe> fp;
    std::vector<std::unique_ptr<Live>> members;
};

struct Done {
    gace_status status = GACE_OK;
    std::string error;
};

// First-fit allocator over the arena's offsets.
struct Arena {
    std::map<uint64_t, uint64_t> free_;  // offset -> bytes
    void reset(uint64_t bytes) {
        free_.clear();
        if (bytes) free_[0] = bytes;
        free_bytes = bytes;
    }
    uint64_t free_bytes = 0;
    uint64_t alloc(uint64_t bytes) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const uint64_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            free_bytes -= bytes;
            return off;
        }
        return ~0ull;
    }
    void release(uint64_t off, uint64_t bytes) {
        free_bytes += bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
};

// Staging of one step (two of them alternate).
struct StepSet {
    unsigned char* host = nullptr;  // pinned upload
    unsigned char* dev = nullptr;   // its device copy
    uint64_t cap = 0;
    unsigned char* rb_host = nullptr;  // pinned read-back
    unsigned char* rb_dev = nullptr;   // gathered small outputs
    uint64_t rb_cap = 0;
    cudaEvent_t done = nullptr, k0 = nullptr, k1 = nullptr;
    cudaEvent_t fork = nullptr, join[kClasses - 1] = {};
    bool busy = false, timed = false;
    std::vector<std::pair<Live*, uint64_t>> finishing;  // request, read-back offset
    uint64_t rows = 0, bytes = 0, ops = 0;
    uint32_t copies = 0, launches = 0;
    uint64_t t_enqueued = 0;
};

// Where a served request's time goes (sums over completed requests, ns).
struct Phases {
    uint64_t n = 0, queue = 0, run = 0, gpu = 0, finish = 0;
};

}  // namespace

struct ServeState {
    gace_ctx* ctx = nullptr;
    gace_serve_config cfg{};
    uint64_t chunk = 0;
    unsigned char* arena = nullptr;
    Arena alloc;
    cudaStream_t stream = nullptr;
    cudaStream_t aux[kClasses - 1] = {};  // a step's other classes run beside the first
    std::thread thr;

    // guarded by mu
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<std::unique_ptr<Live>> pending;
    std::atomic<uint32_t> npending{0};  // pending.size(), readable without mu
    std::unordered_map<uint64_t, Done> done;
    std::unordered_map<uint64_t, bool> open;  // submitted, not yet completed
    std::unordered_map<uint32_t, int> table_refs;
    uint64_t next_ticket = 1;
    std::map<SketchKey, Sketch> cache;
    std::list<SketchKey> lru;
    std::unordered_map<std::string, CountEntry> counts;
    std::list<std::string> counts_lru;
    gace_status sticky = GACE_OK;  // a CUDA failure of the scheduler
    std::string sticky_msg;

    // scheduler thread only
    uint32_t nlive = 0;  // admitted requests (members of fused groups counted one by one)
    std::vector<std::unique_ptr<Live>> live;
    StepSet sets[2];
    int64_t step = 0;
    uint64_t rr = 0;
    std::map<uint64_t, int> occ;  // (class, dynamic shared memory) -> CTAs per SM
    Phases phases;                // published with the kernel statistics

    void run();
    void run_alone(Live& lv);
    void publish_phases();
    void take(std::vector<std::unique_ptr<Live>>& cands);
    void admit(std::vector<std::unique_ptr<Live>>& cands, std::vector<std::unique_ptr<Live>>& admitted,
               bool& blocked);
    gace_status build_step(StepSet& S, std::vector<std::unique_ptr<Live>>& admitted);
    void complete(StepSet& S);
    void finish(Live& lv, gace_status st, const std::string& err);
    void fail_all(gace_status st, const std::string& msg);
    int occupancy(uint32_t smem, int cls);  // CTAs of a batch kernel per SM
    // the fusion rule of admitted probes (FusedProbe::mode)
    int fuse_rule() const { return (cfg.flags & GACE_SERVE_FUSE_SAMPLES) ? 3 : 0; }
};

namespace {

// Block layout of a compiled request; its plan's offsets become offsets from
// the block's start.
void layout_request(Live& lv) {
    Ws win, wsmall, wbig;
    wsmall.take(256);  // the status word of the request's probe and HLL jobs
    place_request(lv.rp, win, wsmall, wbig);
    lv.in_bytes = round_up(win.off, 16);
    lv.small_rel = round_up(win.off, 256);
    lv.small_bytes = round_up(wsmall.off, 16);
    const uint64_t big_rel = lv.small_rel + round_up(wsmall.off, 256);
    lv.block_bytes = std::max<uint64_t>(256, big_rel + round_up(wbig.off, 256));
    shift_request(lv.rp, 0, lv.small_rel, big_rel);
    if (lv.fp) return;  // a fused group: its members hold the table references
    const gace_request& q = lv.req.q;
    if (q.kind == GACE_REQ_JOIN) {
        lv.tables[lv.ntables++] = q.join->fact.table_id;
        lv.tables[lv.ntables++] = q.join->dim.table_id;
        if (q.join->hops == 2) lv.tables[lv.ntables++] = q.join->dim2.table_id;
    } else {
        lv.tables[lv.ntables++] = q.table_id;
    }
}

// Inputs of an admitted request into host staging at pin (offsets as in its
// block), device pointers into its block at dws; its jobs and phases.
void stage_request(Live& lv, unsigned char* pin, unsigned char* dws) {
    ReqPlan& rp = lv.rp;
    unsigned int* status = reinterpret_cast<unsigned int*>(dws + lv.small_rel);
    if (rp.kind == GACE_REQ_PROBE) {
        for (size_t k = 0; k < rp.plan.passes.size(); ++k) {
            Pass& ps = rp.plan.passes[k];
            stage_pass(ps, pin, dws, status);
            memcpy(pin + rp.args_off[k], &ps.args, sizeof(ProbeArgs));
        }
    }
    lv.jobs.clear();
    emit_jobs(rp, dws, status, lv.jobs);
    if (rp.kind == GACE_REQ_JOIN) {
        const int nsides = rp.spec.hops == 2 ? 3 : 2;
        for (int i = 0; i < nsides; ++i) memcpy(pin + rp.side_off[i], &rp.side[i], sizeof(SideArgs));
        if (!rp.pool.empty()) memcpy(pin + rp.pool_off, rp.pool.data(), rp.pool.size() * 4);
    }
    lv.nphases = 0;
    for (uint32_t ph = 0; ph < static_cast<uint32_t>(kPhases); ++ph)
        for (const JobRec& jr : lv.jobs)
            if (jr.phase == ph && jr.units) {
                lv.phase_list[lv.nphases++] = ph;
                break;
            }
}

void enter_phase(Live& lv) {
    lv.pjobs.clear();
    const uint32_t ph = lv.phase_list[lv.pi];
    for (uint32_t j = 0; j < lv.jobs.size(); ++j)
        if (lv.jobs[j].phase == ph && lv.jobs[j].units) lv.pjobs.push_back(j);
    lv.jk = 0;
    lv.unit = 0;
}

void add_copies(std::vector<CopyDesc>& v, unsigned char* dst, const unsigned char* src, uint64_t bytes) {
    for (uint64_t o = 0; o < bytes; o += kCopyPiece) {
        CopyDesc d{};
        d.dst = dst + o;
        d.src = src ? src + o : nullptr;
        d.bytes = std::min(kCopyPiece, bytes - o);
        v.push_back(d);
    }
}

// Completion of a ticket (the caller holds srv.mu).
void deliver(ServeState& srv, uint64_t ticket, ReplaySink* sink, uint32_t idx, gace_status st,
             const std::string& err) {
    if (sink) {
        sink->done_ns[idx] = now_ns() - sink->t0;
        sink->statuses[idx] = st;
        --sink->remaining;
    } else {
        Done& d = srv.done[ticket];
        d.status = st;
        d.error = err;
        srv.open.erase(ticket);
    }
    srv.cv_done.notify_all();
}

void cache_put(ServeState& srv, const SketchKey& key, std::vector<uint8_t>&& regs, double est) {
    const size_t cap = static_cast<size_t>(srv.cfg.sketch_cache);
    auto it = srv.cache.find(key);
    if (it != srv.cache.end()) {
        srv.lru.erase(it->second.lru);
        srv.cache.erase(it);
    }
    srv.lru.push_front(key);
    Sketch& s = srv.cache[key];
    s.regs = std::move(regs);
    s.estimate = est;
    s.lru = srv.lru.begin();
    while (srv.cache.size() > cap) {
        srv.cache.erase(srv.lru.back());
        srv.lru.pop_back();
    }
}

SketchKey sketch_key(const gace_request& q) { return SketchKey{q.table_id, q.col, q.p, q.hash_seed}; }

// Key of a count: the table, the row set (kind, keep rule, threshold, seed
// hash, block size) and the conjunction's normalised terms in canonical
// order (none: the set's sample size).  Equal keys are equal counts, whatever
// the request that measured them.
std::string count_key(uint32_t table, const SetDesc& d, std::vector<const NTerm*> terms) {
    std::sort(terms.begin(), terms.end(), [](const NTerm* a, const NTerm* b) { return *a < *b; });
    std::string k;
    auto put = [&](const void* p, size_t n) { k.append(static_cast<const char*>(p), n); };
    put(&table, 4);
    put(&d.kind, 4);
    put(&d.mode, 4);
    put(&d.thresh, 8);
    put(&d.seedhash, 8);
    put(&d.block_rows, 8);
    for (const NTerm* t : terms) {
        const uint32_t nin = static_cast<uint32_t>(t->in.size());
        put(&t->col, 4);
        put(&t->kind, 4);
        put(&t->a, 8);
        put(&t->b, 8);
        put(&nin, 4);
        if (nin) put(t->in.data(), 4ull * nin);
    }
    return k;
}

std::vector<const NTerm*> pred_terms(const ProbePlan& plan, uint32_t p) {
    std::vector<const NTerm*> v;
    for (uint32_t u : plan.pred_u[p]) v.push_back(&plan.uterms[u]);
    return v;
}

// Keeps the counts of a finished probe (caller holds srv.mu).
void counts_put(ServeState& srv, uint32_t table, const ReqPlan& rp) {
    const size_t cap = static_cast<size_t>(srv.cfg.probe_cache);
    if (!cap) return;
    const ProbePlan& plan = rp.plan;
    const ProbeRequest& r = rp.pr;
    if (static_cast<uint64_t>(r.npreds + r.nterms) * r.nsamples > kCachedProbeMaxCounts) return;
    auto put = [&](std::string&& key, uint64_t v) {
        auto it = srv.counts.find(key);
        if (it != srv.counts.end()) {
            srv.counts_lru.splice(srv.counts_lru.begin(), srv.counts_lru, it->second.lru);
            return;
        }
        srv.counts_lru.push_front(key);
        srv.counts.emplace(std::move(key), CountEntry{v, table, srv.counts_lru.begin()});
        while (srv.counts.size() > cap) {
            srv.counts.erase(srv.counts_lru.back());
            srv.counts_lru.pop_back();
        }
    };
    for (uint32_t s = 0; s < r.nsamples; ++s) {
        if (plan.set_dev[s] < 0) continue;
        const SetDesc& d = plan.sets[plan.set_dev[s]].d;
        if (r.npreds) put(count_key(table, d, {}), r.results[static_cast<uint64_t>(s) * r.npreds].sample_rows);
        for (uint32_t p = 0; p < r.npreds; ++p)
            if (plan.pstate[p] == 0)
                put(count_key(table, d, pred_terms(plan, p)), r.results[static_cast<uint64_t>(s) * r.npreds + p].match);
        if (r.term_marginals)
            for (uint32_t t = 0; t < r.nterms; ++t)
                if (plan.t2u[t] != UINT32_MAX)
                    put(count_key(table, d, {&plan.uterms[plan.t2u[t]]}),
                        r.term_marginals[static_cast<uint64_t>(s) * r.nterms + t]);
    }
}

// Answers a compiled probe from kept counts when every count it needs is
// known (caller holds srv.mu): the outputs are assembled exactly as the
// synchronous call assembles them.
bool counts_answer(ServeState& srv, uint32_t table, const ReqPlan& rp) {
    if (!srv.cfg.probe_cache) return false;
    const ProbePlan& plan = rp.plan;
    const ProbeRequest& r = rp.pr;
    if (static_cast<uint64_t>(r.npreds + r.nterms) * r.nsamples > kCachedProbeMaxCounts) return false;
    const uint32_t ns = r.nsamples, np = r.npreds, nt = r.nterms;
    bool want_marg = r.term_marginals != nullptr;
    for (uint32_t p = 0; p < np; ++p) want_marg = want_marg || r.preds[p].term_cnt == 2;
    std::vector<uint64_t> nsv(ns, 0), match(static_cast<size_t>(ns) * np, 0), marg;
    if (want_marg) marg.assign(static_cast<size_t>(ns) * nt, 0);
    std::vector<std::list<std::string>::iterator> touched;
    auto get = [&](const std::string& key, uint64_t& v) {
        auto it = srv.counts.find(key);
        if (it == srv.counts.end()) return false;
        v = it->second.value;
        touched.push_back(it->second.lru);
        return true;
    };
    for (uint32_t s = 0; s < ns; ++s) {
        if (plan.set_dev[s] < 0) continue;
        const SetDesc& d = plan.sets[plan.set_dev[s]].d;
        if (d.mode == 1) {
            nsv[s] = plan.tab->nrows;
        } else if (!get(count_key(table, d, {}), nsv[s])) {
            return false;
        }
        for (uint32_t p = 0; p < np; ++p)
            if (plan.pstate[p] == 0 && !get(count_key(table, d, pred_terms(plan, p)), match[static_cast<size_t>(s) * np + p]))
                return false;
        if (want_marg)
            for (uint32_t t = 0; t < nt; ++t)
                if (plan.t2u[t] != UINT32_MAX &&
                    !get(count_key(table, d, {&plan.uterms[plan.t2u[t]]}), marg[static_cast<size_t>(s) * nt + t]))
                    return false;
    }
    for (auto& it : touched) srv.counts_lru.splice(srv.counts_lru.begin(), srv.counts_lru, it);
    assemble_probe_counts(
        plan, r, [&](uint32_t s) { return nsv[s]; },
        [&](uint32_t p, uint32_t s) { return match[static_cast<size_t>(s) * np + p]; },
        [&](uint32_t t, uint32_t s) -> uint64_t { return want_marg ? marg[static_cast<size_t>(s) * nt + t] : 0; });
    return true;
}

gace_status alloc_step(StepSet& S, uint64_t up, uint64_t rb) {
    if (up > S.cap) {
        if (S.host) cudaFreeHost(S.host);
        if (S.dev) cudaFree(S.dev);
        S.host = nullptr;
        S.dev = nullptr;
        S.cap = 0;
        const uint64_t cap = round_up(std::max<uint64_t>(up + up / 2, 1ull << 20), 1ull << 16);
        CK(cudaHostAlloc(reinterpret_cast<void**>(&S.host), cap, cudaHostAllocDefault));
        CK(cudaMalloc(&S.dev, cap));
        S.cap = cap;
    }
    if (rb > S.rb_cap) {
        if (S.rb_host) cudaFreeHost(S.rb_host);
        if (S.rb_dev) cudaFree(S.rb_dev);
        S.rb_host = nullptr;
        S.rb_dev = nullptr;
        S.rb_cap = 0;
        const uint64_t cap = round_up(std::max<uint64_t>(rb + rb / 2, 1ull << 20), 1ull << 16);
        CK(cudaHostAlloc(reinterpret_cast<void**>(&S.rb_host), cap, cudaHostAllocDefault));
        CK(cudaMalloc(&S.rb_dev, cap));
        S.rb_cap = cap;
    }
    return GACE_OK;
}

// One request through its synchronous call (the plain path).
gace_status run_plain(gace_ctx* ctx, const gace_request& q) {
    switch (q.kind) {
        case GACE_REQ_PROBE:
            return gace_probe_batch(ctx, q.table_id, q.samples, q.nsamples, q.terms, q.nterms, q.in_values, q.nin,
                                    q.preds, q.npreds, q.results, q.term_marginals);
        case GACE_REQ_NDV:
            return gace_ndv(ctx, q.table_id, q.col, q.p, q.hash_seed, q.registers_out, q.estimate_out);
        case GACE_REQ_JOIN:
            return gace_join_card(ctx, q.join, q.join_out);
        default:
            return fail(GACE_EINVAL, "request kind %u invalid", q.kind);
    }
}

}  // namespace

int ServeState::occupancy(uint32_t smem, int cls) {
    const uint64_t key = (static_cast<uint64_t>(cls) << 32) | smem;
    auto it = occ.find(key);
    return it == occ.end() ? (occ[key] = batch_occupancy(smem, cls)) : it->second;
}

constexpr size_t kAdmitWindow = 1024;  // queued requests considered per admission round

// Moves queued requests, in arrival order, out of the queue while slots and
// the arena's free bytes allow (the caller holds mu).
void ServeState::take(std::vector<std::unique_ptr<Live>>& cands) {
    uint64_t room = alloc.free_bytes;
    while (!pending.empty() && cands.size() < kAdmitWindow && nlive + cands.size() < cfg.max_inflight) {
        if (pending.front()->block_bytes > room) break;
        room -= pending.front()->block_bytes;
        cands.push_back(std::move(pending.front()));
        pending.pop_front();
    }
    npending.store(static_cast<uint32_t>(pending.size()), std::memory_order_relaxed);
}

// Admission of the requests taken from the queue: probes on one table are
// fused (shared scans) and compiled as one request; then blocks are
// allocated in order, first fit.  What does not fit goes back to the head of
// the queue.
void ServeState::admit(std::vector<std::unique_ptr<Live>>& cands, std::vector<std::unique_ptr<Live>>& admitted,
                       bool& blocked) {
    std::vector<std::unique_ptr<Live>> units;
    std::map<uint32_t, std::vector<Live*>> open;  // table -> its groups
    // fusable probes that read the most columns seed the groups
    std::stable_sort(cands.begin(), cands.end(), [](const std::unique_ptr<Live>& a, const std::unique_ptr<Live>& b) {
        const int ca = a->fusable ? __builtin_popcountll(probe_colmask(a->req.q)) : 99;
        const int cb = b->fusable ? __builtin_popcountll(probe_colmask(b->req.q)) : 99;
        return ca > cb;
    });
    for (auto& c : cands) {
        if (!c->fusable) {
            units.push_back(std::move(c));
            continue;
        }
        const TableRec& tab = *c->rp.plan.tab;
        std::vector<Live*>& groups = open[c->req.q.table_id];
        Live* grp = nullptr;
        for (Live* g2 : groups)
            if (g2->fp->fits(c->req.q, tab)) {
                grp = g2;
                break;
            }
        if (!grp) {
            auto fresh = std::make_unique<Live>();
            fresh->fp = std::make_unique<FusedProbe>();
            fresh->fp->mode = fuse_rule();
            grp = fresh.get();
            groups.push_back(grp);
            units.push_back(std::move(fresh));
        }
        grp->fp->add(static_cast<uint32_t>(grp->members.size()), c->req.q, tab);
        grp->members.push_back(std::move(c));
    }
    cands.clear();
    std::vector<std::unique_ptr<Live>> ready;
    for (auto& u : units) {
        if (!u->fp) {
            ready.push_back(std::move(u));
            continue;
        }
        if (u->members.size() == 1) {  // nothing shared: the request runs with its own plan
            ready.push_back(std::move(u->members[0]));
            continue;
        }
        u->fp->seal();
        if (compile_probe(ctx, u->fp->tab, u->fp->q, u->rp) != GACE_OK) {
            for (auto& m : u->members) ready.push_back(std::move(m));  // each runs alone
            continue;
        }
        layout_request(*u);
        ready.push_back(std::move(u));
    }
    size_t i = 0;
    while (i < ready.size()) {
        Live& u = *ready[i];
        const uint64_t off = alloc.alloc(u.block_bytes);
        if (off == ~0ull) {
            if (!u.fp) break;
            // a group that does not fit runs as its members, each of which fits the arena alone
            std::vector<std::unique_ptr<Live>> ms = std::move(u.members);
            ready.erase(ready.begin() + static_cast<std::ptrdiff_t>(i));
            ready.insert(ready.begin() + static_cast<std::ptrdiff_t>(i), std::make_move_iterator(ms.begin()),
                         std::make_move_iterator(ms.end()));
            continue;
        }
        u.block = off;
        nlive += u.fp ? static_cast<uint32_t>(u.members.size()) : 1u;
        admitted.push_back(std::move(ready[i]));
        ++i;
    }
    if (i < ready.size()) {
        blocked = true;
        std::vector<std::unique_ptr<Live>> back;
        for (; i < ready.size(); ++i) {
            if (ready[i]->fp)
                for (auto& m : ready[i]->members) back.push_back(std::move(m));
            else
                back.push_back(std::move(ready[i]));
        }
        std::lock_guard<std::mutex> lk(mu);
        for (auto it = back.rbegin(); it != back.rend(); ++it) pending.push_front(std::move(*it));
        npending.store(static_cast<uint32_t>(pending.size()), std::memory_order_relaxed);
    }
}

// A request is done: free its block, drop its table references, complete its ticket.
void ServeState::finish(Live& lv, gace_status st, const std::string& err) {
    if (lv.block != ~0ull) alloc.release(lv.block, lv.block_bytes);
    lv.block = ~0ull;
    lv.issued_all = true;
    if (lv.fp) {  // a fused group: every member completes with the group's status
        if (st == GACE_OK) lv.fp->scatter();
        for (auto& m : lv.members) finish(*m, st, err);
        lv.finished = true;
        return;
    }
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < lv.ntables; ++i)
        if (--table_refs[lv.tables[i]] == 0) table_refs.erase(lv.tables[i]);
    --nlive;
    if (st == GACE_OK && lv.cacheable && lv.rp.kind == GACE_REQ_NDV) {
        std::vector<uint8_t> regs(lv.req.q.registers_out, lv.req.q.registers_out + (1ull << lv.rp.hll.p));
        cache_put(*this, sketch_key(lv.req.q), std::move(regs), *lv.req.q.estimate_out);
    }
    if (st == GACE_OK && lv.req.q.kind == GACE_REQ_PROBE && lv.rp.plan.tab) counts_put(*this, lv.req.q.table_id, lv.rp);
    deliver(*this, lv.ticket, lv.sink, lv.sink_index, st, err);
    lv.finished = true;
}

void ServeState::fail_all(gace_status st, const std::string& msg) {
    {
        std::lock_guard<std::mutex> lk(mu);
        if (sticky == GACE_OK) {
            sticky = st;
            sticky_msg = msg;
        }
    }
    cudaStreamSynchronize(stream);
    for (cudaStream_t a : aux) cudaStreamSynchronize(a);
    for (StepSet& S : sets) {
        S.busy = false;
        S.finishing.clear();
    }
    for (auto& p : live)
        if (!p->finished) finish(*p, st, msg);
    live.clear();
}

gace_status ServeState::build_step(StepSet& S, std::vector<std::unique_ptr<Live>>& admitted) {
    S.finishing.clear();
    S.rows = S.bytes = S.ops = 0;
    S.copies = 0;
    // newly admitted requests: stage their inputs
    std::vector<unsigned char> inbuf;
    std::vector<std::pair<Live*, uint64_t>> scat;  // request, offset in inbuf
    uint64_t in_total = 0;
    for (auto& p : admitted) in_total += round_up(p->in_bytes, 256);
    inbuf.resize(in_total);
    uint64_t pos = 0;
    const uint64_t t_build = now_ns();
    for (auto& p : admitted) {
        p->t_admit = t_build;
        for (auto& m : p->members) m->t_admit = t_build;
        stage_request(*p, inbuf.data() + pos, arena + p->block);
        scat.emplace_back(p.get(), pos);
        pos += round_up(p->in_bytes, 256);
        live.push_back(std::move(p));
    }
    admitted.clear();
    // phases and the round-robin ring
    std::vector<Live*> ring;
    uint64_t rb_total = 0;
    auto finishing = [&](Live* lv) {
        lv->issued_all = true;
        S.finishing.emplace_back(lv, rb_total);
        rb_total += round_up(lv->small_bytes, 256);
    };
    for (auto& p : live) {
        Live& lv = *p;
        if (lv.issued_all) continue;
        if (lv.nphases == 0) {
            finishing(&lv);
            continue;
        }
        if (lv.pi < 0 || (lv.jk >= lv.pjobs.size() && lv.last_step < step)) {
            ++lv.pi;
            enter_phase(lv);
        }
        if (lv.jk < lv.pjobs.size()) ring.push_back(&lv);
    }
    std::vector<BatchItem> citems[kClasses];
    std::vector<BatchJob> jobs;
    uint32_t smem[kClasses] = {};
    size_t nitems = 0;
    if (!ring.empty()) {
        const size_t n = ring.size();
        const size_t start = static_cast<size_t>(rr++ % n);
        uint64_t budget = cfg.step_rows;
        // A light step (a few small requests) is cut finer, down to one tile,
        // so that it still spreads over every SM: about kItemsPerCta items per
        // resident CTA, never more than the configured chunk.
        uint64_t work = 0;
        for (Live* lv : ring)
            for (size_t k = lv->jk; k < lv->pjobs.size() && work < budget; ++k)
                work += lv->jobs[lv->pjobs[k]].units - (k == lv->jk ? lv->unit : 0);
        work = std::min(work, budget);
        const uint64_t want = static_cast<uint64_t>(ctx->sms) * kCtasPerSmGuess * kItemsPerCta;
        const uint64_t step_chunk = std::max<uint64_t>(128, std::min(chunk, round_up(work / want, 128)));
        bool progress = true;
        while (budget > 0 && progress && nitems < kMaxStepItems) {
            progress = false;
            for (size_t i = 0; i < n && budget > 0 && nitems < kMaxStepItems; ++i) {
                Live& lv = *ring[(start + i) % n];
                if (lv.jk >= lv.pjobs.size()) continue;
                if (lv.step_stamp != step) {
                    lv.step_stamp = step;
                    lv.step_job_base = static_cast<uint32_t>(jobs.size());
                    for (size_t j = 0; j < lv.jobs.size(); ++j) {
                        jobs.push_back(lv.jobs[j].job);
                        uint32_t& sm = smem[lv.jobs[j].cls];
                        sm = std::max(sm, lv.jobs[j].smem);
                    }
                }
                const uint32_t j = lv.pjobs[lv.jk];
                const JobRec& jr = lv.jobs[j];
                const uint64_t b = lv.unit, e = std::min(jr.units, b + item_units(jr, step_chunk));
                BatchItem it{};
                it.job = lv.step_job_base + j;
                it.begin = b;
                it.end = e;
                citems[jr.cls].push_back(it);
                ++nitems;
                S.rows += (e - b) * (jr.rows / jr.units);
                S.bytes += (e - b) * (jr.bytes / jr.units);
                S.ops += (e - b) * (jr.ops / jr.units);
                budget -= std::min(budget, e - b);
                progress = true;
                lv.unit = e;
                if (lv.unit >= jr.units) {
                    ++lv.jk;
                    lv.unit = 0;
                }
                if (lv.jk >= lv.pjobs.size()) {
                    lv.last_step = step;
                    if (lv.pi == lv.nphases - 1) finishing(&lv);
                }
            }
        }
    }
    if (scat.empty() && nitems == 0 && S.finishing.empty()) return GACE_OK;
    // A light step (a couple of small requests admitted or finishing) copies
    // their blocks with plain async copies; otherwise one scatter and one
    // gather launch move every request's data.
    bool direct_in = scat.size() <= kDirectCopies;
    for (auto& sp : scat) direct_in = direct_in && sp.first->block_bytes <= kDirectBlockMax;
    const bool direct_out = S.finishing.size() <= kDirectCopies;
    // upload layout: [queue heads | inputs | items by class | jobs | scatter | gather]
    // (direct: the inputs are whole block images, zeroed outputs included)
    Ws u;
    u.take(256);
    uint64_t in_bytes_up = in_total;
    if (direct_in) {
        in_bytes_up = 0;
        for (auto& sp : scat) in_bytes_up += round_up(sp.first->block_bytes, 256);
    }
    const uint64_t in_off = u.take(in_bytes_up);
    std::vector<BatchItem> items;
    items.reserve(nitems);
    for (int c = 0; c < kClasses; ++c) items.insert(items.end(), citems[c].begin(), citems[c].end());
    const uint64_t items_off = u.take(items.size() * sizeof(BatchItem));
    const uint64_t jobs_off = u.take(jobs.size() * sizeof(BatchJob));
    size_t nscat = 0, ngath = 0;
    if (!direct_in)
        for (auto& sp : scat)
            nscat += (sp.first->in_bytes + kCopyPiece - 1) / kCopyPiece +
                     (sp.first->block_bytes - sp.first->small_rel + kCopyPiece - 1) / kCopyPiece;
    if (!direct_out)
        for (auto& f : S.finishing) ngath += (f.first->small_bytes + kCopyPiece - 1) / kCopyPiece;
    const uint64_t scat_off = u.take(nscat * sizeof(CopyDesc));
    const uint64_t gath_off = u.take(ngath * sizeof(CopyDesc));
    if (gace_status st = alloc_step(S, u.off, rb_total)) return st;
    std::vector<CopyDesc> sdesc, gdesc;
    if (!direct_in)
        for (auto& sp : scat) {
            Live& lv = *sp.first;
            unsigned char* blk = arena + lv.block;
            add_copies(sdesc, blk, S.dev + in_off + sp.second, lv.in_bytes);
            add_copies(sdesc, blk + lv.small_rel, nullptr, lv.block_bytes - lv.small_rel);
        }
    if (!direct_out)
        for (auto& f : S.finishing)
            add_copies(gdesc, S.rb_dev + f.second, arena + f.first->block + f.first->small_rel, f.first->small_bytes);
    if (sdesc.size() != nscat || gdesc.size() != ngath)
        return fail(GACE_ECUDA, "serving step: %zu / %zu copy descriptors, %zu / %zu expected", sdesc.size(),
                    gdesc.size(), nscat, ngath);
    memset(S.host, 0, 256);
    std::vector<std::pair<Live*, uint64_t>> images;  // direct: request, offset of its block image
    if (direct_in) {
        uint64_t at = in_off;
        for (auto& sp : scat) {
            Live& lv = *sp.first;
            if (lv.in_bytes) memcpy(S.host + at, inbuf.data() + sp.second, lv.in_bytes);
            memset(S.host + at + lv.in_bytes, 0, lv.block_bytes - lv.in_bytes);
            images.emplace_back(&lv, at);
            at += round_up(lv.block_bytes, 256);
        }
    } else if (in_total) {
        memcpy(S.host + in_off, inbuf.data(), in_total);
    }
    if (!items.empty()) memcpy(S.host + items_off, items.data(), items.size() * sizeof(BatchItem));
    if (!jobs.empty()) memcpy(S.host + jobs_off, jobs.data(), jobs.size() * sizeof(BatchJob));
    if (nscat) memcpy(S.host + scat_off, sdesc.data(), nscat * sizeof(CopyDesc));
    if (ngath) memcpy(S.host + gath_off, gdesc.data(), ngath * sizeof(CopyDesc));
    const int copy_grid = std::max(1, ctx->sms * 4);
    CK(cudaMemcpyAsync(S.dev, S.host, u.off, cudaMemcpyHostToDevice, stream));
    for (auto& im : images)
        CK(cudaMemcpyAsync(arena + im.first->block, S.host + im.second, im.first->block_bytes, cudaMemcpyHostToDevice,
                           stream));
    if (nscat) {
        CK(copy_launch(reinterpret_cast<const CopyDesc*>(S.dev + scat_off), static_cast<uint32_t>(nscat),
                       std::min<int>(copy_grid, static_cast<int>(nscat)), stream));
        ++S.copies;
    }
    S.timed = !items.empty();
    S.launches = 0;
    if (!items.empty()) {
        CK(cudaEventRecord(S.k0, stream));
        // the classes' persistent kernels on parallel streams: one kernel's
        // draining CTAs leave their slots to the next kernel's instead of idling
        CK(cudaEventRecord(S.fork, stream));
        size_t first = 0;
        int branch = 0;
        for (int c = 0; c < kClasses; ++c) {
            const size_t cnt = citems[c].size();
            if (!cnt) continue;
            const int per_sm = occupancy(smem[c], c);
            if (per_sm < 1)
                return fail(GACE_ECUDA, "batch kernel cannot be resident with %u bytes of shared memory", smem[c]);
            const int grid = static_cast<int>(std::min<size_t>(static_cast<size_t>(per_sm) * ctx->sms, cnt));
            cudaStream_t on = branch == 0 ? stream : aux[branch - 1];
            if (branch > 0) CK(cudaStreamWaitEvent(on, S.fork, 0));
            CK(batch_launch(reinterpret_cast<const BatchItem*>(S.dev + items_off) + first, static_cast<uint32_t>(cnt),
                            reinterpret_cast<const BatchJob*>(S.dev + jobs_off),
                            reinterpret_cast<unsigned int*>(S.dev) + c, grid, smem[c], c, on));
            if (branch > 0) {
                CK(cudaEventRecord(S.join[branch - 1], on));
                CK(cudaStreamWaitEvent(stream, S.join[branch - 1], 0));
            }
            first += cnt;
            ++branch;
            ++S.launches;
        }
        CK(cudaEventRecord(S.k1, stream));
    }
    if (ngath) {
        CK(copy_launch(reinterpret_cast<const CopyDesc*>(S.dev + gath_off), static_cast<uint32_t>(ngath),
                       std::min<int>(copy_grid, static_cast<int>(ngath)), stream));
        ++S.copies;
        if (rb_total) CK(cudaMemcpyAsync(S.rb_host, S.rb_dev, rb_total, cudaMemcpyDeviceToHost, stream));
    } else {
        for (auto& f : S.finishing)
            CK(cudaMemcpyAsync(S.rb_host + f.second, arena + f.first->block + f.first->small_rel,
                               f.first->small_bytes, cudaMemcpyDeviceToHost, stream));
    }
    CK(cudaEventRecord(S.done, stream));
    S.busy = true;
    S.t_enqueued = now_ns();
    for (auto& f : S.finishing) {
        f.first->t_last = S.t_enqueued;
        for (auto& m : f.first->members) m->t_last = S.t_enqueued;
    }
    ++step;
    return GACE_OK;
}

// Waits for a step and completes the requests whose last chunk it ran.
void ServeState::complete(StepSet& S) {
    if (!S.busy) return;
    cudaError_t e = cudaEventSynchronize(S.done);
    if (e != cudaSuccess) {
        fail_all(cuda_fail(e, "a serving step"), gace_last_error());
        return;
    }
    S.busy = false;
    const uint64_t t_detect = now_ns();
    float ms = 0.f;
    if (S.timed) cudaEventElapsedTime(&ms, S.k0, S.k1);
    for (auto& f : S.finishing) {
        Live& lv = *f.first;
        const unsigned char* rb = S.rb_host + f.second;
        const unsigned int status = *reinterpret_cast<const unsigned int*>(rb);
        // host_base + (an offset in the small region) addresses its read-back copy
        const unsigned char* host_base =
            reinterpret_cast<const unsigned char*>(reinterpret_cast<uintptr_t>(rb) - lv.small_rel);
        lv.rp.status = GACE_OK;
        std::vector<uint8_t> regs;
        const bool keeps = lv.rp.kind == GACE_REQ_NDV && (lv.cacheable || lv.keep_resident);
        if (keeps && !lv.req.q.registers_out) {
            // the caches keep the registers even when the caller does not want them
            regs.resize(1ull << lv.rp.hll.p);
            lv.req.q.registers_out = regs.data();
        }
        double est = 0.0;
        if (keeps && !lv.req.q.estimate_out) lv.req.q.estimate_out = &est;
        finish_request(ctx, lv.rp, host_base, status);
        if (lv.keep_resident && lv.rp.status == GACE_OK) {
            const gace_request& q = lv.req.q;
            std::lock_guard<std::mutex> lk(ctx->mu);
            resident_sketch_put(ctx, q.table_id, q.col, q.p, q.hash_seed, q.registers_out);
        }
        finish(lv, lv.rp.status, lv.rp.error);
        const uint64_t t_done = now_ns();
        auto account = [&](const Live& r) {
            phases.n += 1;
            phases.queue += r.t_admit - r.t_submit;
            phases.run += r.t_last - r.t_admit;
            phases.gpu += t_detect - r.t_last;
            phases.finish += t_done - t_detect;
        };
        if (lv.fp)
            for (auto& m : lv.members) account(*m);
        else
            account(lv);
    }
    S.finishing.clear();
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        gace_ctx::KStat& k = ctx->stats["serve_step"];
        k.launches += S.timed ? 1 : 0;
        k.rows += S.rows;
        k.bytes += S.bytes;
        k.ops += S.ops;
        if (ctx->timing) k.ms += ms;
        if (S.launches) ctx->stats["batch_kernel"].launches += S.launches;
        if (S.copies) ctx->stats["serve_copy"].launches += S.copies;
        publish_phases();
    }
    live.erase(std::remove_if(live.begin(), live.end(),
                              [](const std::unique_ptr<Live>& p) { return p->finished; }),
               live.end());
}

// A request alone on an idle server runs through its synchronous call on the
// scheduler thread: with nothing to batch it with, a step's upload, launches
// and read-back would only add latency (a lone request fills one step anyway,
// so requests arriving meanwhile wait no longer than they would behind it).
void ServeState::run_alone(Live& lv) {
    ++nlive;
    lv.t_admit = now_ns();
    std::vector<uint8_t> regs;
    double est = 0.0;
    if (lv.req.q.kind == GACE_REQ_NDV && lv.cacheable) {  // the cache keeps what the caller may not want
        if (!lv.req.q.registers_out) {
            regs.resize(1ull << lv.req.q.p);
            lv.req.q.registers_out = regs.data();
        }
        if (!lv.req.q.estimate_out) lv.req.q.estimate_out = &est;
    }
    const gace_status st = run_plain(ctx, lv.req.q);
    const std::string err = st != GACE_OK ? std::string(gace_last_error()) : std::string();
    lv.t_last = now_ns();
    lv.rp.kind = lv.req.q.kind;
    if (lv.req.q.kind == GACE_REQ_NDV) lv.rp.hll.p = lv.req.q.p;
    finish(lv, st, err);
    const uint64_t t_done = now_ns();
    phases.n += 1;
    phases.queue += lv.t_admit - lv.t_submit;
    phases.gpu += lv.t_last - lv.t_admit;
    phases.finish += t_done - lv.t_last;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->stats["serve_alone"].launches += 1;
    publish_phases();
}

// The request phases into the kernel statistics: launches = requests,
// total_ms = summed time (the caller holds ctx->mu).
void ServeState::publish_phases() {
    const char* names[4] = {"serve_req_queue", "serve_req_run", "serve_req_gpu", "serve_req_finish"};
    const uint64_t vals[4] = {phases.queue, phases.run, phases.gpu, phases.finish};
    for (int i = 0; i < 4; ++i) {
        gace_ctx::KStat& q = ctx->stats[names[i]];
        q.launches += phases.n;
        q.ms += vals[i] / 1e6;
    }
    phases = Phases();
}

void ServeState::run() {
    cudaSetDevice(ctx->device);
    for (;;) {
        std::vector<std::unique_ptr<Live>> cands, admitted;
        std::unique_ptr<Live> fast;
        bool blocked = false, quit = false;
        auto issuable = [&]() {
            for (auto& p : live)
                if (!p->issued_all) return true;
            return false;
        };
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (!pending.empty() || issuable() || sets[0].busy || sets[1].busy) break;
                if (stop) {
                    quit = true;
                    break;
                }
                // Idle: watch the queue for a while before sleeping, so that a
                // request arriving soon does not wait out a thread wake-up
                // (tens of microseconds, most of a small probe's latency).
                lk.unlock();
                const uint64_t t0 = now_ns();
                const uint64_t spin_ns = (cfg.idle_spin_us ? cfg.idle_spin_us : kIdleSpinUs) * 1000ull;
                while (npending.load(std::memory_order_relaxed) == 0 && now_ns() - t0 < spin_ns)
                    std::this_thread::yield();
                lk.lock();
                if (!pending.empty() || stop) continue;
                cv_work.wait(lk);
            }
            if (!quit && sticky != GACE_OK) {
                // after a CUDA failure every request fails with it
                while (!pending.empty()) {
                    Live& lv = *pending.front();
                    for (int i = 0; i < lv.ntables; ++i)
                        if (--table_refs[lv.tables[i]] == 0) table_refs.erase(lv.tables[i]);
                    deliver(*this, lv.ticket, lv.sink, lv.sink_index, sticky, sticky_msg);
                    pending.pop_front();
                }
                npending.store(0, std::memory_order_relaxed);
            } else if (!quit) {
                if (!(cfg.flags & GACE_SERVE_ALWAYS_STEP) && live.empty() && !sets[0].busy && !sets[1].busy &&
                    pending.size() == 1) {
                    fast = std::move(pending.front());  // an idle server: nothing to batch with
                    pending.pop_front();
                    npending.store(0, std::memory_order_relaxed);
                } else {
                    take(cands);
                    if (cands.empty() && !pending.empty()) blocked = true;
                }
            }
        }
        if (quit) break;
        if (fast) {
            run_alone(*fast);
            continue;
        }
        if (!cands.empty()) admit(cands, admitted, blocked);
        if (!admitted.empty() || issuable()) {
            StepSet& S = sets[step & 1];
            if (S.busy) complete(S);
            if (gace_status st = build_step(S, admitted)) fail_all(st, gace_last_error());
            continue;
        }
        StepSet* oldest = sets[step & 1].busy ? &sets[step & 1] : (sets[(step + 1) & 1].busy ? &sets[(step + 1) & 1] : nullptr);
        if (!oldest) continue;
        if (blocked) {
            complete(*oldest);
            continue;
        }
        // Nothing to issue: spin on the step for a while (a sleep costs tens of
        // microseconds of wake-up), leaving as soon as a request arrives.
        const uint64_t t0 = now_ns();
        cudaError_t q = cudaEventQuery(oldest->done);
        while (q == cudaErrorNotReady && npending.load(std::memory_order_relaxed) == 0 && now_ns() - t0 < kSpinNs) {
            std::this_thread::yield();
            q = cudaEventQuery(oldest->done);
        }
        if (q != cudaErrorNotReady) {
            complete(*oldest);
        } else if (npending.load(std::memory_order_relaxed) == 0) {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait_for(lk, std::chrono::microseconds(50), [&]() { return !pending.empty() || stop; });
        }
    }
}

namespace {

std::shared_ptr<ServeState> get_server(gace_ctx* ctx) {
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    return ctx->serve;
}

void free_server(ServeState& s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    for (StepSet& S : s.sets) {
        if (S.host) cudaFreeHost(S.host);
        if (S.dev) cudaFree(S.dev);
        if (S.rb_host) cudaFreeHost(S.rb_host);
        if (S.rb_dev) cudaFree(S.rb_dev);
        for (cudaEvent_t e : {S.done, S.k0, S.k1, S.fork})
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : S.join)
            if (e) cudaEventDestroy(e);
        S = StepSet();
    }
    if (s.arena) cudaFree(s.arena);
    s.arena = nullptr;
    if (s.stream) cudaStreamDestroy(s.stream);
    s.stream = nullptr;
    for (cudaStream_t& a : s.aux) {
        if (a) cudaStreamDestroy(a);
        a = nullptr;
    }
}

// Starts the scheduler; the caller holds ctx->mu and ctx->serve is empty.
gace_status start_locked(gace_ctx* ctx, const gace_serve_config* cfg, std::shared_ptr<ServeState>& out) {
    auto s = std::make_shared<ServeState>();
    s->ctx = ctx;
    if (cfg) s->cfg = *cfg;
    gace_serve_config& c = s->cfg;
    if (!c.arena_bytes) c.arena_bytes = kDefaultArena;
    if (!c.max_inflight) c.max_inflight = kDefaultInflight;
    if (!c.sketch_cache) c.sketch_cache = kDefaultSketches;
    if (c.sketch_cache < 0) c.sketch_cache = 0;
    if (!c.probe_cache) c.probe_cache = kDefaultProbeCounts;
    if (c.probe_cache < 0) c.probe_cache = 0;
    if (!c.step_rows) c.step_rows = kDefaultStepRows;
    if (!c.chunk_rows) c.chunk_rows = kDefaultServeChunk;
    // the kernels count an item's rows in 32-bit shared counters
    if (c.chunk_rows > (1ull << 30))
        return fail(GACE_EINVAL, "chunk_rows %llu above 2^30", (unsigned long long)c.chunk_rows);
    s->chunk = round_up(c.chunk_rows, 128);
    c.arena_bytes = round_up(c.arena_bytes, 1 << 20);
    if (!ctx->fits(c.arena_bytes))
        return fail(GACE_ENOMEM, "serving arena of %llu bytes exceeds the HBM budget",
                    (unsigned long long)c.arena_bytes);
    DeviceGuard g(ctx->device);
    if (gace_status st = batch_setup(ctx)) return st;
    auto undo = [&](gace_status st) {
        free_server(*s);
        return st;
    };
    cudaError_t e = cudaMalloc(&s->arena, c.arena_bytes);
    if (e != cudaSuccess) {
        s->arena = nullptr;
        return fail(GACE_ENOMEM, "cudaMalloc(%llu) for the serving arena: %s", (unsigned long long)c.arena_bytes,
                    cudaGetErrorString(e));
    }
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess)
        return undo(cuda_fail(e, "serving stream"));
    for (cudaStream_t& a : s->aux)
        if ((e = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking)) != cudaSuccess)
            return undo(cuda_fail(e, "serving stream"));
    for (StepSet& S : s->sets) {
        if ((e = cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&S.fork, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreate(&S.k0)) != cudaSuccess || (e = cudaEventCreate(&S.k1)) != cudaSuccess)
            return undo(cuda_fail(e, "serving events"));
        for (cudaEvent_t& j : S.join)
            if ((e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming)) != cudaSuccess)
                return undo(cuda_fail(e, "serving events"));
    }
    s->alloc.reset(c.arena_bytes);
    ctx->used += c.arena_bytes;
    ServeState* raw = s.get();
    s->thr = std::thread([raw]() { raw->run(); });
    {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        ctx->serve = s;
    }
    out = s;
    return GACE_OK;
}

// The running scheduler, started with defaults when there is none (the
// caller holds ctx->mu).
gace_status ensure_server(gace_ctx* ctx, std::shared_ptr<ServeState>& out) {
    out = get_server(ctx);
    if (out) return GACE_OK;
    return start_locked(ctx, nullptr, out);
}

gace_status stop_server(gace_ctx* ctx) {
    std::shared_ptr<ServeState> s = get_server(ctx);
    if (!s) return GACE_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return GACE_OK;  // another caller is stopping it
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->thr.joinable()) s->thr.join();
    {
        DeviceGuard g(ctx->device);
        free_server(*s);
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->used -= s->cfg.arena_bytes;
    }
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    if (ctx->serve == s) ctx->serve.reset();
    return GACE_OK;
}

// Copies, checks and queues one request; completion goes to the ticket table,
// or to sink[idx] when sink is set.
gace_status submit_request(gace_ctx* ctx, const gace_request& req, uint64_t* ticket_out, ReplaySink* sink,
                           uint32_t idx) {
    auto lv = std::make_unique<Live>();
    lv->req.copy_from(req);
    lv->sink = sink;
    lv->sink_index = idx;
    lv->t_submit = now_ns();
    const gace_request& q = lv->req.q;
    std::shared_ptr<ServeState> srv;
    std::lock_guard<std::mutex> ck(ctx->mu);
    if (gace_status s = ensure_server(ctx, srv)) return s;
    if (q.kind == GACE_REQ_NDV && srv->cfg.sketch_cache > 0) {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->cache.find(sketch_key(q));
        if (it != srv->cache.end()) {
            Sketch& sk = it->second;
            if (q.registers_out) memcpy(q.registers_out, sk.regs.data(), sk.regs.size());
            if (q.estimate_out) *q.estimate_out = sk.estimate;
            srv->lru.splice(srv->lru.begin(), srv->lru, sk.lru);
            const uint64_t t = srv->next_ticket++;
            if (ticket_out) *ticket_out = t;
            if (!sink) srv->open[t] = true;
            deliver(*srv, t, sink, idx, GACE_OK, std::string());
            return GACE_OK;
        }
        lv->cacheable = true;
    }
    if (q.kind == GACE_REQ_NDV && ctx->resident.sketches_on() && q.p >= 4 && q.p <= 18) {
        const TableRec* tab = find_table(ctx, q.table_id);
        if (tab && q.col < tab->cols.size()) {
            std::vector<uint8_t> r(1ull << q.p);
            if (resident_sketch_get(ctx, q.table_id, q.col, q.p, q.hash_seed, r.data())) {
                if (q.registers_out) memcpy(q.registers_out, r.data(), r.size());
                if (q.estimate_out) *q.estimate_out = hll_estimate_host(r.data(), q.p);
                std::lock_guard<std::mutex> lk(srv->mu);
                const uint64_t t = srv->next_ticket++;
                if (ticket_out) *ticket_out = t;
                if (!sink) srv->open[t] = true;
                deliver(*srv, t, sink, idx, GACE_OK, std::string());
                return GACE_OK;
            }
            lv->keep_resident = true;
        }
    }
    if (q.kind == GACE_REQ_PROBE) {  // one resident sample: a full scan of it
        static const gace_sample kFull{GACE_FULL, 0, 1.0, 0};
        std::vector<uint32_t> pinned;
        resident_rewrite(ctx, lv->req.q, &kFull, pinned, true);
    }
    if (gace_status s = compile_request(ctx, q, lv->rp)) return s;
    if (q.kind == GACE_REQ_PROBE && srv->cfg.probe_cache > 0) {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (counts_answer(*srv, q.table_id, lv->rp)) {
            const uint64_t t = srv->next_ticket++;
            if (ticket_out) *ticket_out = t;
            if (!sink) srv->open[t] = true;
            deliver(*srv, t, sink, idx, GACE_OK, std::string());
            ctx->stats["serve_probe_cache"].launches += 1;
            return GACE_OK;
        }
    }
    layout_request(*lv);
    lv->fusable = fusable_probe(q, srv->fuse_rule()) && lv->rp.plan.passes.size() <= 1;
    if (lv->block_bytes > srv->cfg.arena_bytes)
        return fail(GACE_ENOMEM, "the request needs %llu bytes of the %llu-byte serving arena",
                    (unsigned long long)lv->block_bytes, (unsigned long long)srv->cfg.arena_bytes);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return fail(GACE_EBUSY, "the scheduler is stopping");
        if (srv->sticky != GACE_OK) return fail(srv->sticky, "%s", srv->sticky_msg.c_str());
        lv->ticket = srv->next_ticket++;
        if (ticket_out) *ticket_out = lv->ticket;
        if (!sink) srv->open[lv->ticket] = true;
        for (int i = 0; i < lv->ntables; ++i) ++srv->table_refs[lv->tables[i]];
        srv->pending.push_back(std::move(lv));
        srv->npending.store(static_cast<uint32_t>(srv->pending.size()), std::memory_order_relaxed);
    }
    srv->cv_work.notify_one();
    return GACE_OK;
}

void wait_until(uint64_t t) {
    for (;;) {
        const uint64_t n = now_ns();
        if (n >= t) return;
        const uint64_t d = t - n;
        if (d > 200000)
            std::this_thread::sleep_for(std::chrono::nanoseconds(d - 100000));
        else if (d > 20000)
            std::this_thread::yield();
    }
}

}  // namespace

void serve_shutdown(gace_ctx* ctx) { stop_server(ctx); }

bool serve_table_busy(gace_ctx* ctx, uint32_t table_id) {
    std::shared_ptr<ServeState> s = get_server(ctx);
    if (!s) return false;
    std::lock_guard<std::mutex> lk(s->mu);
    return s->table_refs.count(table_id) != 0;
}

gace_status serve_forget_table(gace_ctx* ctx, uint32_t table_id) {
    std::shared_ptr<ServeState> s = get_server(ctx);
    if (!s) return GACE_OK;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->table_refs.count(table_id))
        return fail(GACE_EBUSY, "requests on table %u are queued or in flight", table_id);
    for (auto it = s->cache.begin(); it != s->cache.end();) {
        if (it->first.table == table_id) {
            s->lru.erase(it->second.lru);
            it = s->cache.erase(it);
        } else {
            ++it;
        }
    }
    for (auto it = s->counts.begin(); it != s->counts.end();) {
        if (it->second.table == table_id) {
            s->counts_lru.erase(it->second.lru);
            it = s->counts.erase(it);
        } else {
            ++it;
        }
    }
    return GACE_OK;
}

}  // namespace host
}  // namespace gace

extern "C" {

gace_status gace_serve_start(gace_ctx* ctx, const gace_serve_config* cfg) {
    if (gace_status s = check_ctx(ctx)) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (get_server(ctx)) return fail(GACE_EBUSY, "the scheduler is already running");
    std::shared_ptr<ServeState> s;
    return start_locked(ctx, cfg, s);
}

gace_status gace_serve_stop(gace_ctx* ctx) {
    if (gace_status s = check_ctx(ctx)) return s;
    return stop_server(ctx);
}

gace_status gace_submit(gace_ctx* ctx, const gace_request* req, uint64_t* ticket_out) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (!req || !ticket_out) return fail(GACE_EINVAL, "req or ticket_out is NULL");
    return submit_request(ctx, *req, ticket_out, nullptr, 0);
}

gace_status gace_poll(gace_ctx* ctx, uint64_t ticket, uint64_t timeout_us) {
    if (gace_status s = check_ctx(ctx)) return s;
    std::shared_ptr<ServeState> s = get_server(ctx);
    if (!s) return fail(GACE_ENOTFOUND, "ticket %llu unknown: the scheduler is not running", (unsigned long long)ticket);
    Done d;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto ready = [&]() { return s->done.count(ticket) != 0; };
        if (!ready()) {
            if (!s->open.count(ticket)) return fail(GACE_ENOTFOUND, "ticket %llu unknown", (unsigned long long)ticket);
            if (timeout_us)
                s->cv_done.wait_for(lk, std::chrono::microseconds(std::min<uint64_t>(timeout_us, 1ull << 40)), ready);
            if (!ready()) return GACE_EPENDING;
        }
        auto it = s->done.find(ticket);
        d = std::move(it->second);
        s->done.erase(it);
    }
    if (d.status != GACE_OK) set_last_error_message(d.error.c_str());
    return d.status;
}

gace_status gace_serve_replay(gace_ctx* ctx, const gace_request* reqs, uint32_t n, const uint64_t* arrival_ns,
                              uint32_t mode, uint64_t* done_ns, gace_status* statuses) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (n && (!reqs || !arrival_ns || !done_ns)) return fail(GACE_EINVAL, "reqs, arrival_ns or done_ns is NULL");
    if (mode > 1) return fail(GACE_EINVAL, "mode %u (0 served, 1 plain)", mode);
    for (uint32_t i = 1; i < n; ++i)
        if (arrival_ns[i] < arrival_ns[i - 1]) return fail(GACE_EINVAL, "arrival_ns decreases at %u", i);
    std::vector<gace_status> local(statuses ? 0 : n);
    gace_status* st = statuses ? statuses : local.data();
    if (mode == 1) {
        const uint64_t t0 = now_ns();
        for (uint32_t i = 0; i < n; ++i) {
            wait_until(t0 + arrival_ns[i]);
            st[i] = run_plain(ctx, reqs[i]);
            done_ns[i] = now_ns() - t0;
        }
    } else {
        std::shared_ptr<ServeState> srv;
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            if (gace_status s = ensure_server(ctx, srv)) return s;
        }
        ReplaySink sink;
        sink.done_ns = done_ns;
        sink.statuses = st;
        sink.remaining = n;
        sink.t0 = now_ns();
        for (uint32_t i = 0; i < n; ++i) {
            wait_until(sink.t0 + arrival_ns[i]);
            const gace_status rc = submit_request(ctx, reqs[i], nullptr, &sink, i);
            if (rc != GACE_OK) {  // rejected at submission: complete it here
                std::lock_guard<std::mutex> lk(srv->mu);
                deliver(*srv, 0, &sink, i, rc, std::string());
            }
        }
        std::unique_lock<std::mutex> lk(srv->mu);
        srv->cv_done.wait(lk, [&]() { return sink.remaining == 0; });
    }
    for (uint32_t i = 0; i < n; ++i)
        if (st[i] != GACE_OK) return st[i];
    return GACE_OK;
}

gace_status gace_run_plain_async(gace_ctx* const* ctxs, uint32_t nctx, const gace_request* reqs, uint32_t n,
                                 gace_status* statuses) {
    if (nctx == 0 || !ctxs) return fail(GACE_EINVAL, "ctxs is NULL or nctx is 0");
    if (n && !reqs) return fail(GACE_EINVAL, "reqs is NULL");
    for (uint32_t k = 0; k < nctx; ++k)
        if (gace_status s = check_ctx(ctxs[k])) return s;
    std::vector<gace_status> local(statuses ? 0 : n);
    gace_status* st = statuses ? statuses : local.data();
    // context k's requests k, k + nctx, ... in order, on a thread of its own;
    // each call waits for its own stream only, so calls on different
    // contexts overlap on the GPU
    std::vector<std::string> first_error(nctx);
    auto lane = [&](uint32_t k) {
        for (uint32_t i = k; i < n; i += nctx) {
            st[i] = run_plain(ctxs[k], reqs[i]);
            if (st[i] != GACE_OK && first_error[k].empty()) first_error[k] = gace_last_error();
        }
    };
    std::vector<std::thread> threads;
    for (uint32_t k = 1; k < nctx; ++k) threads.emplace_back(lane, k);
    lane(0);
    for (std::thread& t : threads) t.join();
    for (uint32_t i = 0; i < n; ++i)
        if (st[i] != GACE_OK) {
            set_last_error_message(("request " + std::to_string(i) + ": " + first_error[i % nctx]).c_str());
            return st[i];
        }
    return GACE_OK;
}

}  // extern "C"
