// gace_host.h -- host-runtime types and helpers shared by the translation
// units of libgace (context, tables, term normalisation, probe planning).
// Internal: not part of the public ABI (include/gace.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/gace.h"
#include "gace_internal.h"

struct gace_ctx;

namespace gace {
namespace host {

struct ServeState;  // the served form's scheduler (gace_serve.cpp)

// Sets the thread-local error message and returns s.
gace_status fail(gace_status s, const char* fmt, ...);
gace_status cuda_fail(cudaError_t e, const char* what);

#define CK(call)                                           \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return ::gace::host::cuda_fail(e_, #call); \
    } while (0)

// splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014), host side.
inline uint64_t splitmix64_host(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

inline uint32_t dtype_width(int dt) { return dt == GACE_I64 ? 8u : 4u; }

inline uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct ColumnRec {
    int dtype = 0;
    void* dptr = nullptr;
    bool owned = false;  // allocated by the context (stream-ordered, freed with cudaFreeAsync)
    uint64_t bytes = 0;
};

struct TableRec {
    uint64_t nrows = 0;
    std::vector<ColumnRec> cols;
    uint64_t owned_bytes = 0;
    uint32_t sample_of = 0;  // a materialised sample: the table it was drawn from (0: none)
    std::vector<const void*> pending;  // GACE_COPY_ON_FIRST_PROBE: host sources not yet copied
    bool in_store = false;   // owned by the resident store (evictable)
};

// ---------------------------------------------------------------- resident store
// Samples and HyperLogLog sketches kept in device memory under a byte budget
// (gace_resident_configure); the caller of every function below holds ctx->mu.
struct ResidentKey {
    uint32_t table = 0, kind = 0;
    uint64_t thresh = 0, seedhash = 0, block_rows = 0;
    bool operator<(const ResidentKey& o) const {
        return std::tie(table, kind, thresh, seedhash, block_rows) <
               std::tie(o.table, o.kind, o.thresh, o.seedhash, o.block_rows);
    }
};
struct ResidentSample {
    uint32_t sample_table = 0;
    uint64_t bytes = 0;
    uint64_t last_use = 0;
};
struct ResidentSketchKey {
    uint32_t table = 0, col = 0, p = 0;
    uint64_t seed = 0;
    bool operator<(const ResidentSketchKey& o) const {
        return std::tie(table, col, p, seed) < std::tie(o.table, o.col, o.p, o.seed);
    }
};
struct ResidentSketch {
    unsigned char* dregs = nullptr;  // 2^p one-byte registers (device)
    uint64_t bytes = 0;
    uint64_t last_use = 0;
};
struct ResidentStore {
    uint64_t budget = 0;      // 0: the store is off
    uint32_t admit_after = 1;
    uint32_t flags = 0;
    uint64_t used = 0, tick = 0;
    std::map<ResidentKey, ResidentSample> samples;
    std::map<ResidentKey, uint32_t> seen;  // uses of samples that are not resident
    std::map<ResidentSketchKey, ResidentSketch> sketches;
    gace_resident_stats st{};
    bool samples_on() const { return budget && (flags & GACE_RESIDENT_SAMPLES); }
    bool sketches_on() const { return budget && (flags & GACE_RESIDENT_SKETCHES); }
};

// ---------------------------------------------------------------- host workers

// A few host threads that plan a large batch's requests and assemble their
// results in parallel (each request's plan and outputs are its own).  Started
// at the first parallel call, joined when the context is destroyed.
class HostPool {
public:
    ~HostPool();
    // fn(i) for every i in [0, n), on the workers and the calling thread;
    // returns when every call has returned.  Calls of run() do not overlap
    // (the context's mutex is held).
    void run(uint32_t n, const std::function<void(uint32_t)>& fn);

private:
    void work();
    std::vector<std::thread> threads_;
    std::mutex mu_;
    std::condition_variable wake_, done_;
    const std::function<void(uint32_t)>* fn_ = nullptr;
    uint32_t n_ = 0;
    std::atomic<uint32_t> next_{0};
    uint32_t busy_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};
// Requests at which a batch plans and assembles them on the workers.
constexpr uint32_t kParallelRequests = 64;

}  // namespace host
}  // namespace gace

using namespace gace;
using namespace gace::host;

struct gace_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 0;
    int smem_optin = 0;
    int smem_per_sm = 0;     // shared memory of one SM (bytes)
    uint64_t budget = 0;       // 0 = unlimited
    uint64_t used = 0;         // owned tables + workspace + pinned
    uint64_t timeout_ns = 2000ull * 1000000ull;
    uint32_t max_ctas = 0;     // cap on the CTAs of a probe launch (0 = none)
    uint64_t rank_min_rows = 0;  // smallest table a batch probe rank-codes (0: kRankMinRows)
    uint32_t rank_search = 0;    // gace_config.rank_search
    std::mutex mu;
    std::unordered_map<uint32_t, TableRec> tables;
    uint32_t next_id = 1;
    unsigned char* ws = nullptr;  // device workspace
    uint64_t ws_cap = 0;
    unsigned char* pin = nullptr;  // pinned host staging
    uint64_t pin_cap = 0;
    unsigned int* d_status = nullptr;
    // Stream-ordered allocations of the columns, samples and sketches the
    // context owns come from its own pool, which keeps freed memory for reuse
    // (a table loaded and unloaded step after step does not map its pages
    // again each time) and returns it to the device when the context ends.
    cudaMemPool_t pool = nullptr;
    // copies of tables loaded with GACE_COPY_ON_FIRST_PROBE, in chunks, and
    // the events the probe's passes wait for
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> chunk_events;

    cudaError_t alloc_async(void** p, uint64_t bytes) {
        return pool ? cudaMallocFromPoolAsync(p, bytes, pool, stream) : cudaMallocAsync(p, bytes, stream);
    }

    // kernel statistics (tracing)
    struct KStat {
        uint64_t launches = 0, rows = 0, bytes = 0, ops = 0;
        double ms = 0.0;
    };
    struct Timed {
        std::string name;
        cudaEvent_t a, b;
        uint64_t bytes, ops;
    };
    std::map<std::string, KStat> stats;
    // measured probe costs for the break-even model (kept across stats resets):
    // the timed narrow and wide probe launches' work and device time
    struct CostRec {
        uint64_t launches = 0;
        double bytes = 0.0, ops = 0.0, ms = 0.0;
    };
    CostRec cost_narrow, cost_wide;
    bool timing = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<Timed> pending;

    cudaEvent_t take_event() {
        if (!ev_free.empty()) {
            cudaEvent_t e = ev_free.back();
            ev_free.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }

    // Counts one launch with its algorithmic work and, when timing, brackets
    // it with events on the context stream.
    template <typename F>
    cudaError_t traced(const char* name, uint64_t rows, uint64_t bytes, uint64_t ops, F&& launch) {
        KStat& k = stats[name];
        k.launches++;
        k.rows += rows;
        k.bytes += bytes;
        k.ops += ops;
        if (!timing) return launch();
        cudaEvent_t a = take_event(), b = take_event();
        if (a) cudaEventRecord(a, stream);
        cudaError_t e = launch();
        if (b) cudaEventRecord(b, stream);
        if (a && b) pending.push_back({name, a, b, bytes, ops});
        return e;
    }

    // Host phases of a call (when timing): the wall time since phase_t into
    // stats[name] (launches = phases recorded), then phase_t restarts.
    std::chrono::steady_clock::time_point phase_t;
    void host_phase(const char* name) {
        if (!timing) return;
        const auto now = std::chrono::steady_clock::now();
        KStat& k = stats[name];
        k.launches++;
        k.ms += std::chrono::duration<double, std::milli>(now - phase_t).count();
        phase_t = now;
    }

    // After a stream synchronisation: fold event pairs into the statistics.
    void collect() {
        for (auto& t : pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
                stats[t.name].ms += ms;
                CostRec* c = t.name == "probe_narrow" ? &cost_narrow : t.name == "probe_wide" ? &cost_wide : nullptr;
                if (c) {
                    c->launches++;
                    c->bytes += static_cast<double>(t.bytes);
                    c->ops += static_cast<double>(t.ops);
                    c->ms += ms;
                }
            }
            ev_free.push_back(t.a);
            ev_free.push_back(t.b);
        }
        pending.clear();
    }

    // batched form: tuning table, capture stream and the last batch's graph
    struct TuneEntry {
        uint64_t chunk = 0;
        int ctas_per_sm = 0;
        double ms = 0.0;
    };
    std::map<std::pair<int, int>, TuneEntry> tune;  // (log2 jobs, log2 rows) -> best
    // fusion rules (FusedProbe::mode) per request shape: (log2 requests,
    // log2 rows of the tables they read) -> mode
    std::map<std::pair<int, int>, int> fuse_tune;
    cudaStream_t capture_stream = nullptr;
    cudaStream_t batch_aux[kClasses - 1] = {};  // a phase's other classes run beside the first
    cudaEvent_t batch_fork[kPhases] = {};
    cudaEvent_t batch_join[kPhases][kClasses - 1] = {};
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<uint64_t> graph_key;
    bool batch_ready = false;

    // served form: the scheduler, when running
    std::mutex serve_mu;
    std::shared_ptr<ServeState> serve;

    // resident samples and sketches
    ResidentStore resident;

    // host workers of large batches
    HostPool workers;

    bool fits(uint64_t extra) const { return budget == 0 || used + extra <= budget; }

    gace_status ensure_ws(uint64_t bytes) {
        bytes = round_up(bytes ? bytes : 256, 1 << 20);
        if (bytes <= ws_cap) return GACE_OK;
        if (!fits(bytes - ws_cap))
            return fail(GACE_ENOMEM, "workspace of %llu bytes exceeds the HBM budget",
                        (unsigned long long)bytes);
        CK(cudaStreamSynchronize(stream));
        if (ws) {
            cudaFree(ws);
            used -= ws_cap;
            ws = nullptr;
            ws_cap = 0;
        }
        cudaError_t e = cudaMalloc(&ws, bytes);
        if (e != cudaSuccess) {
            ws = nullptr;
            return fail(GACE_ENOMEM, "cudaMalloc(%llu) for the workspace: %s",
                        (unsigned long long)bytes, cudaGetErrorString(e));
        }
        ws_cap = bytes;
        used += bytes;
        return GACE_OK;
    }

    gace_status ensure_pin(uint64_t bytes) {
        bytes = round_up(bytes ? bytes : 256, 1 << 16);
        if (bytes <= pin_cap) return GACE_OK;
        CK(cudaStreamSynchronize(stream));
        if (pin) {
            cudaFreeHost(pin);
            pin = nullptr;
            pin_cap = 0;
        }
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&pin), bytes, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            pin = nullptr;
            return fail(GACE_ENOMEM, "cudaHostAlloc(%llu): %s", (unsigned long long)bytes,
                        cudaGetErrorString(e));
        }
        pin_cap = bytes;
        return GACE_OK;
    }
};


namespace gace {
namespace host {

// ---------------------------------------------------------------- terms

struct NTerm {
    uint32_t col = 0;
    uint32_t kind = kFalse;
    uint64_t a = 0, b = 0;
    std::vector<uint32_t> in;  // pool words
    bool operator<(const NTerm& o) const {
        return std::tie(col, kind, a, b, in) < std::tie(o.col, o.kind, o.a, o.b, o.in);
    }
    bool operator==(const NTerm& o) const {
        return col == o.col && kind == o.kind && a == o.a && b == o.b && in == o.in;
    }
};
// Hash of a normalised term (deduplication of a request's terms).
struct NTermHash {
    size_t operator()(const NTerm& t) const {
        auto mix = [](uint64_t h, uint64_t v) {
            h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
            return h * 0xBF58476D1CE4E5B9ull;
        };
        uint64_t h = mix(mix(mix(t.col, t.kind), t.a), t.b);
        for (uint32_t w : t.in) h = mix(h, w);
        return static_cast<size_t>(h ^ (h >> 31));
    }
};

gace_status normalize_term(const gace_term& t, int dtype, const gace_scalar* in_values, uint32_t nin, NTerm& out);
bool is_in_kind(uint32_t k);
uint32_t in_count(const NTerm& t);

// Slots per entry of a wide pass's EQ/IN hash tables (the inverse of their
// load factor): a two-choice table fills reliably below half its slots.
#ifndef GACE_VS_SLOTS
#define GACE_VS_SLOTS 2
#endif
constexpr uint64_t kVsSlotsPerEntry = GACE_VS_SLOTS;

#ifndef GACE_TREE_MIN
#define GACE_TREE_MIN 24
#endif
// A column's range terms beyond its full groups of 32 use an interval tree only
// when at least this many (a tree costs about as much as this many compares).
constexpr uint32_t kTreeMin = GACE_TREE_MIN;

// The tables one column's terms need in a wide pass (pass packing).
// Terms fill groups of 32 in order, so the open group is always the last one:
// a few counters give the tables' size in constant time per term.
struct ColPool {
    uint32_t nvs = 0;    // EQ / IN terms (groups of 32, in order)
    uint64_t last = 0;   // entries of the last group
    uint64_t most = 0;   // entries of the fullest group
    uint32_t nr = 0;     // multi-value range terms (a column coded with all its terms: every term)
    uint64_t niv = 0;    // key intervals of the rank-coded terms (one per IN value)
    uint32_t rstride = 0;  // rank-coded column: its endpoints + 1 (0: trees)
    bool rank_all = false;  // rank-coded with all its terms (no hash tables)
    bool is64 = false;   // 64-bit keys
    void add(const NTerm& t);
    uint32_t words() const;
};
uint64_t term_cost(const NTerm& t);
// One distinct value of a wide pass's EQ/IN group and the group's terms that hold it.
struct VsEntry {
    uint32_t lo, hi, mask;
};
DevTerm make_devterm(const NTerm& t, uint32_t pool_off);

// ---------------------------------------------------------------- sets

struct SetPlan {
    SetDesc d;
    uint32_t orig;
};

gace_status make_set(const gace_sample& s, SetDesc& d);

// ---------------------------------------------------------------- probe plan

// A pass holds at most kPassTerms terms and kPassPreds predicates, and no
// more than keeps kWideCtas CTAs of the wide kernel resident per SM (its
// register budget allows three): the larger the pass, the fewer full scans of
// the referenced columns, until the pass's shared memory costs a CTA.
#ifndef GACE_PASS_TERMS
#define GACE_PASS_TERMS 512
#endif
#ifndef GACE_PASS_PREDS
#define GACE_PASS_PREDS 512
#endif
#ifndef GACE_WIDE_CTAS
#define GACE_WIDE_CTAS 3
#endif
constexpr uint32_t kPassTerms = GACE_PASS_TERMS;
constexpr uint32_t kPassPreds = GACE_PASS_PREDS;
constexpr int kWideCtas = GACE_WIDE_CTAS;
constexpr uint32_t kPassPool = 16384;  // pool words: IN lists (narrow) or EQ/IN tables (wide)

struct Pass {
    std::vector<uint32_t> preds;   // device predicate indices (input numbering)
    std::vector<uint32_t> uterms;  // unique terms placed in this pass
    // built:
    std::vector<DevTerm> dterms;
    std::vector<uint32_t> pool, poff, pterm;
    std::vector<uint32_t> u_local;  // unique term -> local index (parallel to uterms order)
    std::vector<std::pair<uint32_t, uint32_t>> slots;  // (col, first local term)
    ProbeArgs args{};
    uint64_t in_off = 0, out_off = 0;  // workspace offsets
    uint64_t ops_per_row = 0;          // compares per row (statistics)
    uint32_t rowbytes = 0;             // bytes per row of the referenced columns
    uint64_t in_bytes = 0, out_bytes = 0;
    // the marginals of every term come from the rank histograms of their
    // columns (all terms rank-coded), not from the pass's counters
    bool hist_marg = false;
};

struct Ws {
    uint64_t off = 0;
    uint64_t take(uint64_t bytes, uint64_t align = 256) {
        off = round_up(off, align);
        const uint64_t r = off;
        off += bytes;
        return r;
    }
};

gace_status check_ctx(gace_ctx* ctx);
// A loaded table (its pending copy completed first), or nullptr.
TableRec* find_table(gace_ctx* ctx, uint32_t id);
// The same without completing a pending copy.
TableRec* find_table_raw(gace_ctx* ctx, uint32_t id);
// Copies a table's pending host sources (GACE_COPY_ON_FIRST_PROBE) and waits.
gace_status complete_load(gace_ctx* ctx, TableRec& t);
gace_status read_status(gace_ctx* ctx, unsigned int st);

// The arguments of one probe (gace_probe_batch, or a probe request of a batch).
struct ProbeRequest {
    const gace_sample* samples = nullptr;
    uint32_t nsamples = 0;
    const gace_term* terms = nullptr;
    uint32_t nterms = 0;
    const gace_scalar* in_values = nullptr;
    uint32_t nin = 0;
    const gace_pred* preds = nullptr;
    uint32_t npreds = 0;
    gace_pred_result* results = nullptr;
    uint64_t* term_marginals = nullptr;
};

// A probe compiled into device passes: row sets, deduplicated terms, the
// predicates' states and the passes that evaluate them.
// A column whose range terms (or all terms) the wide passes of a synchronous
// probe read by rank: the sorted distinct endpoints of the key intervals of
// those terms over the whole plan (each interval's start and the key just past
// its end) and their search tree for k_probe_rank (level order, padded with the
// largest key).
struct RankCode {
    uint32_t col = 0;
    uint32_t dtype = 0;
    std::vector<uint64_t> keys;
    std::vector<uint32_t> tree;  // search tree words: keys, or (lo, hi) pairs for int64; or the bucket index
    uint32_t levels = 0;         // search tree levels (0: the bucket index below)
    uint64_t bbase = 0;          // bucket index (RankArgs): base key, buckets, shifts, halvings
    uint32_t bnb = 0, bsmin = 0, bmbits = 0, bsteps = 0;
    bool all_terms = false;      // EQ and IN terms too (each value a one-key interval)
    bool used = false;           // some wide pass of the plan reads the column's ranks
    bool hist_fits = false;      // its histograms fit the rank pass's shared memory
    bool hist = false;           // the rank pass counts each row set's ranks (marginals)
    const unsigned long long* hist_host = nullptr;  // after a run: [set][rank] counts
};
// Most endpoints a column may have to be rank-coded: each group of 32 of its
// range terms then holds endpoints + 1 mask words of the pass's shared pool.
#ifndef GACE_RANK_PLAN_MAX
#define GACE_RANK_PLAN_MAX 2047
#endif
constexpr uint32_t kRankPlanMax = GACE_RANK_PLAN_MAX;
// A coded column's search structures from its sorted keys: the level-order
// search tree (rc.tree, rc.levels), then, per rank_search (gace_config), the
// bucket index in its place (rc.levels = 0, rc.b*; RankArgs).
void build_rank_tree(RankCode& rc);
void build_rank_buckets(RankCode& rc, uint32_t search);
// A synchronous probe rank-codes its columns when it has more than
// kNarrowMax predicates, at least kRankMinTerms distinct terms (more than one
// wide pass holds) and at least kRankMinRows rows (the context's
// rank_min_rows when set).
#ifndef GACE_RANK_MIN_TERMS
#define GACE_RANK_MIN_TERMS 384
#endif
constexpr size_t kRankMinTerms = GACE_RANK_MIN_TERMS;
constexpr uint64_t kRankMinRows = 1ull << 20;
// Most shared memory of a rank pass that also counts its row sets' ranks.
constexpr uint64_t kRankHistSmem = 96u << 10;

struct ProbePlan {
    const TableRec* tab = nullptr;
    std::vector<SetPlan> sets;     // device row sets
    std::vector<int32_t> set_dev;  // sample -> device set, -1 if empty
    std::vector<NTerm> uterms;
    std::vector<uint32_t> t2u;     // input term -> unique term (UINT32_MAX: never true)
    std::vector<uint8_t> pstate;   // 0 device, 1 never true, 2 always true, 3 from rank histograms
    std::vector<std::vector<uint32_t>> pred_u;
    bool want_marg = false;
    std::vector<Pass> passes;
    std::vector<RankCode> codes;       // rank-coded columns
    std::vector<int32_t> code_of_col;  // column -> codes index, -1 if not coded
    // per unique term read by rank, its key intervals as column endpoint
    // indices [r0, r1): span[span_off[u] .. span_off[u + 1])
    std::vector<uint32_t> span_off;
    std::vector<std::pair<uint32_t, uint32_t>> span;
    // unique term u's marginals (and, for a single-term predicate, its count)
    // come from its column's rank histograms
    bool hist_term(uint32_t u) const {
        if (u + 1 >= span_off.size() || span_off[u + 1] == span_off[u]) return false;
        return codes[code_of_col[uterms[u].col]].hist;
    }
};

// Argument checks that need no table.
gace_status check_probe_request(const ProbeRequest& r);
// Compiles a probe; force_wide builds every pass in the wide-kernel layout.
// wide_warps: warps of the CTA that runs the plan's wide passes (kWideWarps
// for the synchronous kernel, kProbeWarps for the batched form's).
// rank_code: the wide passes read the range terms of columns with at most
// kRankPlanMax endpoints by the rows' ranks (run_planned computes them).
// trace: the planner's phases go to the context's statistics when it times
// (host_plan_sets, _terms, _rank, _pack, _build; only from a caller that
// holds the context's mutex and plans on one thread).
gace_status plan_probe(gace_ctx* ctx, const TableRec& tab, const ProbeRequest& r, bool force_wide,
                       ProbePlan& plan, uint32_t wide_warps, bool rank_code = false, bool trace = false);
// Bytes of a pass's inputs (terms, pool, predicate CSR) and outputs (counters).
void pass_sizes(Pass& ps);
// Copies a pass's inputs into pinned staging at ps.in_off and points its
// arguments at their device copies (workspace base dws) and at its outputs.
void stage_pass(Pass& ps, unsigned char* pin, unsigned char* dws, unsigned int* status);
// A probe (or one part of a probe whose row sets span several tables) with its plan.
struct PlannedProbe {
    const TableRec* tab = nullptr;
    ProbeRequest r;
    ProbePlan plan;
};
// Runs planned probes with one upload, their passes' launches, one read-back
// and a wait on the context stream, then assembles each part's results.
// lazy: the one part's table, whose pending copy (GACE_COPY_ON_FIRST_PROBE)
// then streams in kLoadChunks row chunks overlapped with the passes.
// A table whose rank-coded columns' ranks would take more than kRankScratch
// bytes runs its passes in row chunks, the ranks of one chunk at a time.
gace_status run_planned(gace_ctx* ctx, std::vector<PlannedProbe>& parts, TableRec* lazy = nullptr);
constexpr uint64_t kLoadChunks = 12;
#ifndef GACE_RANK_SCRATCH_MB
#define GACE_RANK_SCRATCH_MB 2048
#endif
constexpr uint64_t kRankScratch = static_cast<uint64_t>(GACE_RANK_SCRATCH_MB) << 20;
// Results from the passes' counters (host copies, one pointer per pass).
void assemble_probe(const ProbePlan& plan, const ProbeRequest& r,
                    const std::vector<const unsigned long long*>& pass_out);

// The request's outputs from its counts: ns_of(s) = rows of sample s (0 for
// an empty sample), match_of(p, s) = count of device predicate p on the
// sample, marg_of(t, s) = marginal of input term t (0 when never true or the
// sample is empty).  The one place where selectivities and PCS are computed,
// so that counts from passes and counts from the served form's result cache
// give the same doubles.
template <class NsOf, class MatchOf, class MargOf>
void assemble_probe_counts(const ProbePlan& plan, const ProbeRequest& r, NsOf&& ns_of, MatchOf&& match_of,
                           MargOf&& marg_of) {
    const uint32_t nsamples = r.nsamples, nterms = r.nterms, npreds = r.npreds;
    for (uint32_t s = 0; s < nsamples; ++s) {
        const uint64_t ns = ns_of(s);
        for (uint32_t p = 0; p < npreds; ++p) {
            uint64_t m = 0;
            if (plan.pstate[p] == 2)
                m = ns;
            else if ((plan.pstate[p] == 0 || plan.pstate[p] == 3) && plan.set_dev[s] >= 0)
                m = match_of(p, s);
            gace_pred_result& res = r.results[static_cast<uint64_t>(s) * npreds + p];
            res.match = m;
            res.sample_rows = ns;
            res.sel = ns ? static_cast<double>(m) / static_cast<double>(ns) : 0.0;
            res.pcs = std::numeric_limits<double>::quiet_NaN();
            if (r.preds[p].term_cnt == 2) {
                const uint64_t ca = marg_of(r.preds[p].term_off, s), cb = marg_of(r.preds[p].term_off + 1, s);
                if (ca != 0 && cb != 0)
                    res.pcs = (static_cast<double>(m) * static_cast<double>(ns)) /
                              (static_cast<double>(ca) * static_cast<double>(cb));
            }
        }
        if (r.term_marginals)
            for (uint32_t t = 0; t < nterms; ++t) r.term_marginals[static_cast<uint64_t>(s) * nterms + t] = marg_of(t, s);
    }
}

// ---------------------------------------------------------------- HLL, joins

double hll_estimate_host(const uint8_t* regs, uint32_t p);

struct SideWork {
    uint64_t rows = 0, rowbytes = 0, ops_per_row = 1;
};
// A pass skips tiles only when each spans at most this many sample blocks.
constexpr uint64_t kSkipBlocksPerTile = 8;
// A kernel whose one wait (on an mbarrier phase nothing completes) gives up
// after timeout_ns and sets kStatusTimeout in *status.
cudaError_t wait_check_launch(unsigned int* status, uint64_t timeout_ns, cudaStream_t s);
void plan_side_stages(SideArgs& a);
gace_status build_side(gace_ctx* ctx, const gace_join_side& js, const char* name, int extra_col, SideArgs& a,
                       std::vector<uint32_t>& pool, TableRec** tab_out, uint32_t* extra_slot, SideWork& work);


// ---------------------------------------------------------------- batched and served forms

constexpr uint64_t kDefaultChunk = 1ull << 20;
constexpr uint32_t kHllSmem = 1u << 16;  // 32-bit registers for p <= 14, one-byte for p = 15, 16

struct JobRec {
    BatchJob job{};
    uint32_t phase = 0;
    uint64_t units = 0;  // rows, or histogram entries
    uint64_t granule = 128;  // items start on multiples of this (a narrow pass's tile)
    int cls = kClassGeneral;  // the persistent kernel that drains its items
    uint32_t smem = 0;        // dynamic shared memory its items need
    uint32_t cost = 1;        // time per unit relative to a narrow probe row: items get chunk / cost
                              // units, so that items of every kind take about as long
                              // (long items of one kind leave the other CTAs idle at a
                              // launch's end)
    const char* family = "";
    uint64_t rows = 0, bytes = 0, ops = 0;  // statistics
};

// A compiled request: its plan and where its data sits in the arena
// (offsets relative to the input, small-output and big-output regions).
// The sides of a join request, allocated at their first use: a batch builds
// one plan per request and most requests are not joins (three sides take
// 5.5 KB, most of a plan).
struct JoinSides {
    std::unique_ptr<SideArgs[]> p;
    SideArgs& operator[](int i) {
        if (!p) p.reset(new SideArgs[3]());
        return p[i];
    }
    const SideArgs& operator[](int i) const { return p[i]; }
    JoinSides() = default;
    JoinSides(JoinSides&&) = default;
    JoinSides& operator=(JoinSides&&) = default;
    JoinSides(const JoinSides& o) { *this = o; }
    JoinSides& operator=(const JoinSides& o) {
        if (this != &o) {
            p.reset();
            if (o.p) {
                p.reset(new SideArgs[3]());
                for (int i = 0; i < 3; ++i) p[i] = o.p[i];
            }
        }
        return *this;
    }
};

struct ReqPlan {
    gace_status status = GACE_OK;
    std::string error;
    uint32_t kind = 0;
    const gace_request* q = nullptr;
    // probe
    ProbeRequest pr;
    ProbePlan plan;
    std::vector<uint64_t> args_off;  // input region: ProbeArgs copy per pass
    // ndv
    uint64_t regs_off = 0;  // small region
    HllArgs hll{};
    TableRec* tab = nullptr;
    // join
    gace_join spec{};
    JoinSides side;
    SideWork work[3]{};
    TableRec* tabs[3]{};
    uint32_t fk2_slot = 0;
    bool hist_dot = false;
    uint64_t K = 0, K2 = 0;
    std::vector<uint32_t> pool;
    uint64_t pool_off = 0, side_off[3] = {0, 0, 0};  // input region
    uint64_t sc_off = 0;                              // small region: scalars and status
    uint64_t hd_off = 0, w_off = 0, hf_off = 0;       // big region
    int fused = -1;  // >= 0: absorbed into that fused probe, which runs instead
};

// Shared scans: probe requests on one table fused into one request whose
// passes evaluate every member's predicates on their common row sets (limits
// of a narrow pass), so the table's columns are read once.  Counts are exact
// integers, so each member's results equal its own call's.
struct FusedProbe {
    struct Member {
        uint32_t index = 0;  // the member's position in its batch (or queue)
        const gace_request* q = nullptr;
        uint32_t pred_off = 0, term_off = 0;
        uint32_t set_map[kMaxSets] = {0};
    };
    uint32_t table_id = 0;
    const TableRec* tab = nullptr;
    uint64_t colmask = 0;  // columns referenced by the members' terms
    std::vector<gace_sample> samples;
    std::vector<gace_term> terms;
    std::vector<gace_scalar> in_values;
    std::vector<gace_pred> preds;
    std::vector<gace_pred_result> results;
    std::vector<uint64_t> marg;
    std::vector<Member> members;
    gace_request q{};
    // Fusion rules: 0, the rules of fits() below (a one-predicate request on
    // one row set runs alone); 1, such requests fuse too; 2, as 1, and a group
    // takes the union of its members' row sets (at most kMaxSets) and of their
    // columns (at most kMaxRowBytes per row); 3, only such requests on a
    // hashed row sample fuse (then one hash per row serves the group), with
    // the same row sets and the union of their columns.  The batch autotuner
    // picks one per batch shape.
    int mode = 0;

    static constexpr uint32_t kMaxIn = 1024;     // IN values of all members
#ifndef GACE_FUSE
#define GACE_FUSE 1
#endif
    static constexpr uint32_t kMaxRowBytes = 16;  // bytes per row of the referenced columns: the
                                                  // pass's tiles still stage
    // Whether r (a fusable probe on table t) can join: the same row sets as the
    // group's and no column the group does not read already, so that joining
    // removes r's whole scan and adds no hashing or counting per row beyond
    // r's own predicates (the probe kernels are issue-bound, not HBM-bound,
    // once a pass evaluates many predicates on many row sets).
    bool fits(const gace_request& r, const TableRec& t) const;
    void add(uint32_t index, const gace_request& r, const TableRec& t);
    // Points q at the merged arrays and sizes the result buffers.
    void seal();
    // Each member's results and marginals from the fused ones.
    void scatter() const;
};

// Whether a probe request is a candidate for fusion under the rules of `mode`
// (FusedProbe::mode).
bool fusable_probe(const gace_request& r, int mode = 0);
// The columns a probe's terms reference as a bit mask (~0 when one is >= 64);
// fused groups are seeded with the requests that read the most columns.
uint64_t probe_colmask(const gace_request& r);

// Argument checks and plans of one request.
gace_status compile_request(gace_ctx* ctx, const gace_request& q, ReqPlan& rp);
// The same for a probe; with tab set, on that table without a look-up in the
// context's table map.
gace_status compile_probe(gace_ctx* ctx, const TableRec* tab, const gace_request& q, ReqPlan& rp);
// Offsets of a request's data in the input, small-output and big-output regions.
void place_request(ReqPlan& rp, Ws& win, Ws& wsmall, Ws& wbig);
// Adds the regions' bases to those offsets.
void shift_request(ReqPlan& rp, uint64_t in_base, uint64_t small_base, uint64_t big_base);
// Jobs of a request, with device pointers into the workspace at dws.
void emit_jobs(ReqPlan& rp, unsigned char* dws, unsigned int* status, std::vector<JobRec>& jobs);
// One-time setup of the batch kernels' attributes, streams and events.
gace_status batch_setup(gace_ctx* ctx);
// Units per item of a job for a chunk size: chunk / cost, on the job's
// granule, probe items at least four tiles.
uint64_t item_units(const JobRec& jr, uint64_t chunk);
// Items of `chunk` units per job, ordered by phase, then class.
void make_items(const std::vector<JobRec>& jobs, uint64_t chunk, std::vector<BatchItem>& items,
                uint32_t (&pbeg)[kPhases][kClasses], uint32_t (&pcnt)[kPhases][kClasses]);
// A request's outputs from what its small-output region held.
void finish_request(gace_ctx* ctx, ReqPlan& rp, const unsigned char* host_base, unsigned int status);

// ---------------------------------------------------------------- resident store

// The materialised sample of table `tab` under set d (kind 1 or 2, mode 2): a
// new table with every column, the kept rows in row order.  room(bytes) is
// asked, once the sample's size is known, whether that many bytes may be
// allocated (it may evict); false refuses with GACE_ENOMEM.
gace_status materialize_sample(gace_ctx* ctx, const TableRec& tab, const SetDesc& d,
                               const std::function<bool(uint64_t)>& room, TableRec& out);
// The resident sample table for (table_id, d), or 0: a hit refreshes its
// recency; a miss counts the use and, when `admit` is set and the sample has
// been asked for admit_after times, materialises it into the store (evicting
// least recently used entries outside `pinned`).  Sample tables in `pinned`
// are not evicted; the returned one is added to it.
uint32_t resident_sample(gace_ctx* ctx, uint32_t table_id, const SetDesc& d, bool admit,
                         std::vector<uint32_t>& pinned);
// The resident sketch's registers into regs (host, 2^p bytes): true on a hit.
bool resident_sketch_get(gace_ctx* ctx, uint32_t table, uint32_t col, uint32_t p, uint64_t seed, uint8_t* regs);
// Keeps a computed sketch (when sketches are on and it fits after eviction).
void resident_sketch_put(gace_ctx* ctx, uint32_t table, uint32_t col, uint32_t p, uint64_t seed,
                         const uint8_t* regs);
// Drops every resident entry drawn from table_id (its unload).
void resident_forget_table(gace_ctx* ctx, uint32_t table_id);
// Whether served requests read a resident sample drawn from table_id (any, for 0).
bool resident_samples_busy(gace_ctx* ctx, uint32_t table_id);
// Drops every entry (the store turned off, or the context destroyed).
void resident_clear(gace_ctx* ctx);
// Frees a table's owned columns on the context stream and its bytes from the
// context's accounting (the caller erases it from ctx->tables).
void free_table_columns(gace_ctx* ctx, TableRec& t);
// A probe request whose row sets are all one sample (0 < rate < 1) that the
// store holds (or admits) becomes a full scan of the sample table: q's
// table_id and samples are replaced (full points at a GACE_FULL sample).
bool resident_rewrite(gace_ctx* ctx, gace_request& q, const gace_sample* full, std::vector<uint32_t>& pinned,
                      bool admit);

// A batch's requests as the resident store sees them: probes whose one row
// set is a resident sample rewritten to full scans of it, NDV requests
// answered from resident sketches taken out; what runs is reqs, whose entry k
// is the caller's request index[k].
struct ResidentBatch {
    std::vector<gace_request> reqs;
    std::vector<uint32_t> index;
    std::vector<std::vector<uint8_t>> regs;  // registers of NDV requests that did not ask for them
    std::vector<uint32_t> pinned;
    void build(gace_ctx* ctx, const gace_request* in, uint32_t n);
    // After the run: keeps the sketches the batch computed.
    void keep_sketches(gace_ctx* ctx, const std::vector<gace_status>& st) const;
};

// Served form: stops the scheduler of a context (after its requests have
// finished); forgets a table's cached sketches, GACE_EBUSY while requests on
// the table are in flight.  The caller holds ctx->mu for serve_forget_table.
void serve_shutdown(gace_ctx* ctx);
gace_status serve_forget_table(gace_ctx* ctx, uint32_t table_id);
// Whether served requests on the table are queued or in flight.
bool serve_table_busy(gace_ctx* ctx, uint32_t table_id);

}  // namespace host
}  // namespace gace
