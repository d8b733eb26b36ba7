// gace_resident.cpp -- materialised samples (K3b) and the resident store of
// samples and HyperLogLog sketches.
//
// The gate probes the same row or block samples, and asks for the same NDV
// sketches, again and again while queries are planned (Section III-A); the
// Measurement Engine's sampling and summaries (Section III-B) are worth
// keeping in device memory between its invocations.  A materialised sample is
// a table of its own (the kept rows of every column, in row order): a full
// scan of it gives exactly the integers of the sampled scan of the base
// table, at r N rows instead of N rows and N hashes.  The store keeps such
// samples and sketches under a byte budget, admits a sample after a number
// of uses, and evicts the least recently used entries that no request in
// flight reads.  Every function here runs with ctx->mu held.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <mutex>
#include <vector>

#include "gace_host.h"

namespace gace {
namespace host {

namespace {

ResidentKey key_of(uint32_t table, const SetDesc& d) {
    ResidentKey k;
    k.table = table;
    k.kind = d.kind;
    k.thresh = d.thresh;
    k.seedhash = d.seedhash;
    k.block_rows = d.kind == 2 ? d.block_rows : 0;
    return k;
}

bool is_pinned(const std::vector<uint32_t>& pinned, uint32_t id) {
    return std::find(pinned.begin(), pinned.end(), id) != pinned.end();
}

void drop_sample(gace_ctx* ctx, std::map<ResidentKey, ResidentSample>::iterator it) {
    ResidentStore& R = ctx->resident;
    auto t = ctx->tables.find(it->second.sample_table);
    if (t != ctx->tables.end()) {
        free_table_columns(ctx, t->second);
        ctx->tables.erase(t);
    }
    R.used -= it->second.bytes;
    R.samples.erase(it);
}

void drop_sketch(gace_ctx* ctx, std::map<ResidentSketchKey, ResidentSketch>::iterator it) {
    ResidentStore& R = ctx->resident;
    if (it->second.dregs) cudaFreeAsync(it->second.dregs, ctx->stream);
    R.used -= it->second.bytes;
    ctx->used -= it->second.bytes;
    R.sketches.erase(it);
}

// Evicts least recently used entries (samples outside `pinned` and not read by
// a served request in flight; sketches) until `bytes` more fit both the
// store's budget and the context's.  False when they cannot.
bool make_room(gace_ctx* ctx, uint64_t bytes, const std::vector<uint32_t>& pinned) {
    ResidentStore& R = ctx->resident;
    if (bytes > R.budget) return false;
    while (R.used + bytes > R.budget || !ctx->fits(bytes)) {
        auto best_s = R.samples.end();
        auto best_k = R.sketches.end();
        uint64_t best = ~0ull;
        for (auto it = R.samples.begin(); it != R.samples.end(); ++it) {
            if (it->second.last_use >= best || is_pinned(pinned, it->second.sample_table)) continue;
            if (serve_table_busy(ctx, it->second.sample_table)) continue;
            best = it->second.last_use;
            best_s = it;
        }
        for (auto it = R.sketches.begin(); it != R.sketches.end(); ++it) {
            if (it->second.last_use >= best) continue;
            best = it->second.last_use;
            best_k = it;
            best_s = R.samples.end();
        }
        if (best_k != R.sketches.end()) {
            drop_sketch(ctx, best_k);
            R.st.sketch_evicted++;
        } else if (best_s != R.samples.end()) {
            drop_sample(ctx, best_s);
            R.st.evicted++;
        } else {
            return false;
        }
    }
    return true;
}

// Materialises (table_id, d) into the store; 0 when it does not fit.
uint32_t admit_sample(gace_ctx* ctx, uint32_t table_id, const SetDesc& d, std::vector<uint32_t>& pinned) {
    ResidentStore& R = ctx->resident;
    const TableRec* tab = find_table(ctx, table_id);
    if (!tab) return 0;
    TableRec t;
    auto room = [&](uint64_t b) { return make_room(ctx, b, pinned); };
    if (materialize_sample(ctx, *tab, d, room, t) != GACE_OK) {
        R.st.refused++;
        return 0;
    }
    const uint32_t id = ctx->next_id++;
    t.sample_of = table_id;
    t.in_store = true;
    const ResidentKey k = key_of(table_id, d);
    R.used += t.owned_bytes;
    ResidentSample rs;
    rs.sample_table = id;
    rs.bytes = t.owned_bytes;
    rs.last_use = ++R.tick;
    R.samples[k] = rs;
    R.seen.erase(k);
    R.st.admitted++;
    ctx->tables.emplace(id, std::move(t));
    pinned.push_back(id);
    return id;
}

}  // namespace

void free_table_columns(gace_ctx* ctx, TableRec& t) {
    for (auto& c : t.cols)
        if (c.owned && c.dptr) {
            cudaFreeAsync(c.dptr, ctx->stream);
            c.dptr = nullptr;
        }
    ctx->used -= t.owned_bytes;
    t.owned_bytes = 0;
}

gace_status materialize_sample(gace_ctx* ctx, const TableRec& tab, const SetDesc& d,
                               const std::function<bool(uint64_t)>& room, TableRec& out) {
    if (tab.cols.size() > static_cast<size_t>(kMaxSampleCols))
        return fail(GACE_EINVAL, "a table of %zu columns (at most %d are sampled)", tab.cols.size(), kMaxSampleCols);
    if ((d.kind != 1 && d.kind != 2) || d.mode != 2)
        return fail(GACE_EINVAL, "only row or block samples with 0 < rate < 1 are materialised");
    SampleArgs a{};
    a.nrows = tab.nrows;
    a.ntiles = (tab.nrows + kSampleTileRows - 1) / kSampleTileRows;
    a.set = d;
    a.ncols = static_cast<uint32_t>(tab.cols.size());
    uint64_t rowbytes = 0;
    for (uint32_t c = 0; c < a.ncols; ++c) {
        a.src[c] = tab.cols[c].dptr;
        a.width[c] = dtype_width(tab.cols[c].dtype);
        rowbytes += a.width[c];
    }
    Ws ws;
    const uint64_t cnt_off = ws.take(a.ntiles * 4);
    const uint64_t off_off = ws.take(a.ntiles * 8);
    if (gace_status st = ctx->ensure_ws(ws.off)) return st;
    if (gace_status st = ctx->ensure_pin(ws.off)) return st;
    a.tile_count = reinterpret_cast<uint32_t*>(ctx->ws + cnt_off);
    a.tile_off = reinterpret_cast<const uint64_t*>(ctx->ws + off_off);
    const int grid = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(a.ntiles, static_cast<uint64_t>(ctx->sms) * 8)));
    uint64_t total = 0;
    if (a.ntiles) {
        CK(ctx->traced("sample_count", a.nrows, 0, a.nrows, [&] { return sample_count_launch(a, grid, ctx->stream); }));
        CK(cudaMemcpyAsync(ctx->pin + cnt_off, ctx->ws + cnt_off, a.ntiles * 4, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->collect();
        const uint32_t* cnt = reinterpret_cast<const uint32_t*>(ctx->pin + cnt_off);
        uint64_t* off = reinterpret_cast<uint64_t*>(ctx->pin + off_off);
        for (uint64_t t = 0; t < a.ntiles; ++t) {
            off[t] = total;
            total += cnt[t];
        }
    }
    uint64_t bytes = 0;
    for (uint32_t c = 0; c < a.ncols; ++c) bytes += round_up(total * a.width[c] + 16, 256);
    if (!room(bytes))
        return fail(GACE_ENOMEM, "a sample of %llu bytes does not fit the resident store", (unsigned long long)bytes);
    if (!ctx->fits(bytes))
        return fail(GACE_ENOMEM, "a sample of %llu bytes exceeds the HBM budget", (unsigned long long)bytes);
    out = TableRec();
    out.nrows = total;
    for (uint32_t c = 0; c < a.ncols; ++c) {
        ColumnRec r;
        r.dtype = tab.cols[c].dtype;
        r.bytes = total * a.width[c];
        const uint64_t alloc = round_up(r.bytes + 16, 256);
        cudaError_t e = ctx->alloc_async(&r.dptr, alloc);
        if (e != cudaSuccess) {
            for (auto& x : out.cols) cudaFreeAsync(x.dptr, ctx->stream);
            out.cols.clear();
            return fail(GACE_ENOMEM, "cudaMallocAsync(%llu) for a sample column: %s", (unsigned long long)alloc,
                        cudaGetErrorString(e));
        }
        r.owned = true;
        out.owned_bytes += alloc;
        a.dst[c] = r.dptr;
        out.cols.push_back(r);
    }
    ctx->used += out.owned_bytes;
    if (total) {
        CK(cudaMemcpyAsync(ctx->ws + off_off, ctx->pin + off_off, a.ntiles * 8, cudaMemcpyHostToDevice, ctx->stream));
        // algorithmic bytes: the kept rows read and written once
        CK(ctx->traced("sample_scatter", a.nrows, 2 * total * rowbytes, a.nrows,
                       [&] { return sample_scatter_launch(a, grid, ctx->stream); }));
    }
    // requests of the served form read the sample on the scheduler's stream
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->collect();
    return GACE_OK;
}

uint32_t resident_sample(gace_ctx* ctx, uint32_t table_id, const SetDesc& d, bool admit,
                         std::vector<uint32_t>& pinned) {
    ResidentStore& R = ctx->resident;
    if (!R.samples_on() || d.mode != 2 || (d.kind != 1 && d.kind != 2)) return 0;
    const TableRec* tab = find_table(ctx, table_id);
    if (!tab || tab->sample_of) return 0;  // samples are drawn from base tables only
    const ResidentKey k = key_of(table_id, d);
    auto it = R.samples.find(k);
    if (it != R.samples.end()) {
        it->second.last_use = ++R.tick;
        R.st.sample_hits++;
        pinned.push_back(it->second.sample_table);
        return it->second.sample_table;
    }
    R.st.sample_misses++;
    if (!admit) return 0;
    uint32_t& seen = R.seen[k];
    ++seen;
    if (seen < std::max<uint32_t>(1, R.admit_after)) return 0;
    return admit_sample(ctx, table_id, d, pinned);
}

bool resident_rewrite(gace_ctx* ctx, gace_request& q, const gace_sample* full, std::vector<uint32_t>& pinned,
                      bool admit) {
    if (q.kind != GACE_REQ_PROBE || q.nsamples != 1 || !q.samples || !ctx->resident.samples_on()) return false;
    SetDesc d;
    if (make_set(q.samples[0], d) != GACE_OK) return false;  // the request's own checks report it
    const uint32_t id = resident_sample(ctx, q.table_id, d, admit, pinned);
    if (!id) return false;
    q.table_id = id;
    q.samples = full;
    return true;
}

bool resident_sketch_get(gace_ctx* ctx, uint32_t table, uint32_t col, uint32_t p, uint64_t seed, uint8_t* regs) {
    ResidentStore& R = ctx->resident;
    if (!R.sketches_on()) return false;
    auto it = R.sketches.find(ResidentSketchKey{table, col, p, seed});
    if (it == R.sketches.end()) {
        R.st.sketch_misses++;
        return false;
    }
    const uint64_t m = 1ull << p;
    if (ctx->ensure_pin(m) != GACE_OK) return false;
    if (cudaMemcpyAsync(ctx->pin, it->second.dregs, m, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return false;
    memcpy(regs, ctx->pin, m);
    it->second.last_use = ++R.tick;
    R.st.sketch_hits++;
    return true;
}

void resident_sketch_put(gace_ctx* ctx, uint32_t table, uint32_t col, uint32_t p, uint64_t seed,
                         const uint8_t* regs) {
    ResidentStore& R = ctx->resident;
    if (!R.sketches_on() || !find_table(ctx, table)) return;
    const ResidentSketchKey k{table, col, p, seed};
    if (R.sketches.count(k)) return;
    const uint64_t m = 1ull << p, bytes = round_up(m, 256);
    const std::vector<uint32_t> none;
    if (!make_room(ctx, bytes, none)) return;
    if (ctx->ensure_pin(m) != GACE_OK) return;
    ResidentSketch sk;
    if (ctx->alloc_async(reinterpret_cast<void**>(&sk.dregs), bytes) != cudaSuccess) return;
    memcpy(ctx->pin, regs, m);
    if (cudaMemcpyAsync(sk.dregs, ctx->pin, m, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaFreeAsync(sk.dregs, ctx->stream);
        return;
    }
    sk.bytes = bytes;
    sk.last_use = ++R.tick;
    R.used += bytes;
    ctx->used += bytes;
    R.sketches[k] = sk;
}

void resident_forget_table(gace_ctx* ctx, uint32_t table_id) {
    ResidentStore& R = ctx->resident;
    for (auto it = R.samples.begin(); it != R.samples.end();) {
        auto cur = it++;
        if (cur->first.table == table_id) drop_sample(ctx, cur);
    }
    for (auto it = R.sketches.begin(); it != R.sketches.end();) {
        auto cur = it++;
        if (cur->first.table == table_id) drop_sketch(ctx, cur);
    }
    for (auto it = R.seen.begin(); it != R.seen.end();) {
        if (it->first.table == table_id)
            it = R.seen.erase(it);
        else
            ++it;
    }
}

void resident_clear(gace_ctx* ctx) {
    ResidentStore& R = ctx->resident;
    while (!R.samples.empty()) drop_sample(ctx, R.samples.begin());
    while (!R.sketches.empty()) drop_sketch(ctx, R.sketches.begin());
    R.seen.clear();
}

// Whether a resident sample drawn from table_id is read by served requests.
bool resident_samples_busy(gace_ctx* ctx, uint32_t table_id) {
    for (const auto& kv : ctx->resident.samples)
        if ((table_id == 0 || kv.first.table == table_id) && serve_table_busy(ctx, kv.second.sample_table))
            return true;
    return false;
}

void ResidentBatch::build(gace_ctx* ctx, const gace_request* in, uint32_t n) {
    static const gace_sample kFull{GACE_FULL, 0, 1.0, 0};
    reqs.clear();
    index.clear();
    regs.clear();
    pinned.clear();
    const ResidentStore& R = ctx->resident;
    for (uint32_t i = 0; i < n; ++i) {
        gace_request q = in[i];
        if (q.kind == GACE_REQ_NDV && R.sketches_on() && q.p >= 4 && q.p <= 18) {
            const TableRec* tab = find_table(ctx, q.table_id);
            if (tab && q.col < tab->cols.size()) {
                std::vector<uint8_t> r(1ull << q.p);
                if (resident_sketch_get(ctx, q.table_id, q.col, q.p, q.hash_seed, r.data())) {
                    if (q.registers_out) memcpy(q.registers_out, r.data(), r.size());
                    if (q.estimate_out) *q.estimate_out = hll_estimate_host(r.data(), q.p);
                    continue;  // answered: no job
                }
                if (!q.registers_out) {  // the store keeps what the caller may not want
                    regs.emplace_back(1ull << q.p);
                    q.registers_out = regs.back().data();
                }
            }
        }
        resident_rewrite(ctx, q, &kFull, pinned, true);
        reqs.push_back(q);
        index.push_back(i);
    }
}

void ResidentBatch::keep_sketches(gace_ctx* ctx, const std::vector<gace_status>& st) const {
    if (!ctx->resident.sketches_on()) return;
    for (size_t k = 0; k < reqs.size(); ++k) {
        const gace_request& q = reqs[k];
        if (q.kind == GACE_REQ_NDV && st[k] == GACE_OK && q.registers_out)
            resident_sketch_put(ctx, q.table_id, q.col, q.p, q.hash_seed, q.registers_out);
    }
}

}  // namespace host
}  // namespace gace

using namespace gace::host;

extern "C" {

gace_status gace_sample_materialize(gace_ctx* ctx, uint32_t table_id, const gace_sample* sample,
                                    uint32_t* sample_table_out, uint64_t* rows_out) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (!sample || !sample_table_out) return fail(GACE_EINVAL, "sample or sample_table_out is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    TableRec* tab = find_table(ctx, table_id);
    if (!tab) return fail(GACE_ENOTFOUND, "table %u is not loaded", table_id);
    SetDesc d;
    if (gace_status st = make_set(*sample, d)) return st;
    TableRec t;
    if (gace_status st = materialize_sample(ctx, *tab, d, [](uint64_t) { return true; }, t)) return st;
    const uint32_t id = ctx->next_id++;
    t.sample_of = table_id;
    const uint64_t rows = t.nrows;
    ctx->tables.emplace(id, std::move(t));
    *sample_table_out = id;
    if (rows_out) *rows_out = rows;
    return GACE_OK;
}

gace_status gace_resident_configure(gace_ctx* ctx, const gace_resident_config* cfg) {
    if (gace_status s = check_ctx(ctx)) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    ResidentStore& R = ctx->resident;
    gace_resident_config c{};
    if (cfg) c = *cfg;
    if (c.flags & ~(GACE_RESIDENT_SAMPLES | GACE_RESIDENT_SKETCHES))
        return fail(GACE_EINVAL, "resident flags 0x%x invalid", c.flags);
    if (!c.flags) c.flags = GACE_RESIDENT_SAMPLES | GACE_RESIDENT_SKETCHES;
    if (resident_samples_busy(ctx, 0)) return fail(GACE_EBUSY, "served requests read resident samples");
    if (c.budget_bytes != R.budget || c.flags != R.flags || c.admit_after != R.admit_after) {
        resident_clear(ctx);
        R.st = gace_resident_stats{};  // a new configuration counts afresh
    }
    R.budget = c.budget_bytes;
    R.flags = c.flags;
    R.admit_after = c.admit_after;
    CK(cudaStreamSynchronize(ctx->stream));
    return GACE_OK;
}

gace_status gace_resident_prefetch(gace_ctx* ctx, uint32_t table_id, const gace_sample* sample) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (!sample) return fail(GACE_EINVAL, "sample is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    ResidentStore& R = ctx->resident;
    if (!R.samples_on()) return fail(GACE_EINVAL, "the resident store does not keep samples");
    const TableRec* tab = find_table(ctx, table_id);
    if (!tab) return fail(GACE_ENOTFOUND, "table %u is not loaded", table_id);
    if (tab->sample_of) return fail(GACE_EINVAL, "table %u is itself a sample", table_id);
    SetDesc d;
    if (gace_status st = make_set(*sample, d)) return st;
    if (d.mode != 2 || (d.kind != 1 && d.kind != 2))
        return fail(GACE_EINVAL, "only row or block samples with 0 < rate < 1 are kept");
    std::vector<uint32_t> pinned;
    auto it = R.samples.find(key_of(table_id, d));
    if (it != R.samples.end()) {
        it->second.last_use = ++R.tick;
        return GACE_OK;
    }
    if (!admit_sample(ctx, table_id, d, pinned))
        return fail(GACE_ENOMEM, "the sample does not fit the resident store (%llu of %llu bytes used)",
                    (unsigned long long)R.used, (unsigned long long)R.budget);
    return GACE_OK;
}

gace_status gace_resident_stats_read(gace_ctx* ctx, gace_resident_stats* out) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (!out) return fail(GACE_EINVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    const ResidentStore& R = ctx->resident;
    *out = R.st;
    out->budget_bytes = R.budget;
    out->used_bytes = R.used;
    out->samples = R.samples.size();
    out->sketches = R.sketches.size();
    return GACE_OK;
}

}  // extern "C"
