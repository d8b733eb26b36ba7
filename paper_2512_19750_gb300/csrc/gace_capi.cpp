// gace_capi.cpp -- host runtime behind the C ABI of include/gace.h.
//
// A context owns one CUDA stream, the tables registered on it, a device
// workspace and a pinned host staging buffer, all accounted against an HBM
// budget.  Every entry point validates its arguments, compiles its request
// into the kernels' compact forms (normalised terms, deduplicated, grouped by
// column), launches on the context stream, reads back the integer results and
// derives the doubles on the host.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "gace_host.h"

namespace {

thread_local std::string g_last_error;

}  // namespace

void gace::set_last_error_message(const char* msg) { g_last_error = msg; }

namespace gace {
namespace host {

gace_status fail(gace_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

gace_status cuda_fail(cudaError_t e, const char* what) {
    return fail(GACE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}









// ---------------------------------------------------------------- terms


uint32_t fbits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

// Smallest float >= x, and largest float < x (x a finite or infinite double).
float float_at_or_above(double x) {
    float f = static_cast<float>(x);
    if (static_cast<double>(f) < x) f = std::nextafter(f, std::numeric_limits<float>::infinity());
    return f;
}
float float_below(double x) {
    float f = static_cast<float>(x);
    if (static_cast<double>(f) >= x) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
    return f;
}

// Normalises a term on a column of dtype into an inclusive interval or a
// deduplicated IN list in the column's own domain (or kFalse).
gace_status normalize_term(const gace_term& t, int dtype, const gace_scalar* in_values,
                           uint32_t nin, NTerm& out) {
    out = NTerm();
    out.col = t.col;
    if (t.op > GACE_IN) return fail(GACE_EINVAL, "term op %u is not EQ/RANGE/IN", t.op);
    if (t.op == GACE_IN) {
        if (t.in_len == 0 || t.in_len > 4096)
            return fail(GACE_EINVAL, "IN list length %u outside 1..4096", t.in_len);
        if ((uint64_t)t.in_off + t.in_len > nin || in_values == nullptr)
            return fail(GACE_EINVAL, "IN list [%u, %u) outside in_values[%u]", t.in_off,
                        t.in_off + t.in_len, nin);
    }
    if (dtype == GACE_I32 || dtype == GACE_I64) {
        const int64_t lo_lim = dtype == GACE_I32 ? INT32_MIN : INT64_MIN;
        const int64_t hi_lim = dtype == GACE_I32 ? INT32_MAX : INT64_MAX;
        const uint32_t rk = dtype == GACE_I32 ? kRangeI32 : kRangeI64;
        auto set_range = [&](int64_t lo, int64_t hi) {  // inclusive, lo <= hi
            out.kind = rk;
            out.a = static_cast<uint64_t>(lo);
            out.b = static_cast<uint64_t>(hi) - static_cast<uint64_t>(lo);
            if (dtype == GACE_I32) {
                out.a &= 0xFFFFFFFFull;
                out.b &= 0xFFFFFFFFull;
            }
        };
        if (t.op == GACE_EQ) {
            const int64_t v = t.a.i;
            if (v < lo_lim || v > hi_lim) return GACE_OK;  // kFalse
            set_range(v, v);
        } else if (t.op == GACE_RANGE) {
            const int64_t lo = t.a.i, hi = t.b.i;
            if (lo >= hi) return GACE_OK;
            const int64_t l = std::max(lo, lo_lim);
            const int64_t h = std::min(hi - 1, hi_lim);
            if (l > h) return GACE_OK;
            set_range(l, h);
        } else {
            std::vector<int64_t> v;
            for (uint32_t k = 0; k < t.in_len; ++k) {
                const int64_t x = in_values[t.in_off + k].i;
                if (x >= lo_lim && x <= hi_lim) v.push_back(x);
            }
            std::sort(v.begin(), v.end());
            v.erase(std::unique(v.begin(), v.end()), v.end());
            if (v.empty()) return GACE_OK;
            if (v.size() == 1) {
                set_range(v[0], v[0]);
            } else {
                out.kind = dtype == GACE_I32 ? kInI32 : kInI64;
                for (int64_t x : v) {
                    out.in.push_back(static_cast<uint32_t>(static_cast<uint64_t>(x)));
                    if (dtype == GACE_I64)
                        out.in.push_back(static_cast<uint32_t>(static_cast<uint64_t>(x) >> 32));
                }
            }
        }
        return GACE_OK;
    }
    // float32 column, double constants compared exactly
    if (t.op == GACE_EQ) {
        const double v = t.a.f;
        if (std::isnan(v)) return GACE_OK;
        const float f = static_cast<float>(v);
        if (static_cast<double>(f) != v) return GACE_OK;
        out.kind = kRangeF32;
        out.a = out.b = fbits(f);
    } else if (t.op == GACE_RANGE) {
        const double lo = t.a.f, hi = t.b.f;
        if (std::isnan(lo) || std::isnan(hi) || !(lo < hi)) return GACE_OK;
        const float fl = float_at_or_above(lo), fh = float_below(hi);
        if (!(fl <= fh)) return GACE_OK;
        out.kind = kRangeF32;
        out.a = fbits(fl);
        out.b = fbits(fh);
    } else {
        std::vector<uint32_t> v;
        for (uint32_t k = 0; k < t.in_len; ++k) {
            const double x = in_values[t.in_off + k].f;
            if (std::isnan(x)) continue;
            float f = static_cast<float>(x);
            if (static_cast<double>(f) != x) continue;
            if (f == 0.0f) f = 0.0f;  // -0 and +0 compare equal: keep one
            v.push_back(fbits(f));
        }
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        if (v.empty()) return GACE_OK;
        out.kind = kRangeF32;
        if (v.size() == 1) {
            out.a = out.b = v[0];
        } else {
            out.kind = kInF32;
            out.in = v;
        }
    }
    return GACE_OK;
}

bool is_in_kind(uint32_t k) { return k == kInI32 || k == kInI64 || k == kInF32; }

uint32_t in_count(const NTerm& t) {
    return t.kind == kInI64 ? static_cast<uint32_t>(t.in.size() / 2) : static_cast<uint32_t>(t.in.size());
}

// Pool words of one column's tables in a wide pass (an upper bound for a
// narrow pass, whose pool holds only the IN values): one hash table per group
// of 32 EQ/IN terms in order, all of one capacity (the next power of two >=
// kVsSlotsPerEntry times the largest group's entries, at least 64), one interval tree per full
// group of 32 range terms (or last group of at least kTreeMin), and one word
// of alignment.
uint32_t ColPool::words() const {
    const uint32_t trees = nr / 32 + (nr % 32 >= kTreeMin ? 1 : 0);
    uint64_t w = 1;
    if (nvs) {
        uint32_t tlog = 6;
        while ((1ull << tlog) < kVsSlotsPerEntry * most) ++tlog;
        w += static_cast<uint64_t>((nvs + 31) / 32) * (1ull << tlog) * (is64 ? 4u : 2u);
    }
    if (rstride) {  // rank-coded: the smaller of the column-rank tables and a rank map + local tables
        const uint64_t g = (nr + 31) / 32, ml = std::min<uint64_t>(2ull * (rank_all ? niv : nr), rstride - 1);
        const uint64_t direct = g * rstride;
        const uint64_t mapped = (rstride * (ml <= 255 ? 1 : 2) + 3) / 4 + g * (ml + 1);
        w += std::min(direct, mapped);
    } else {
        w += static_cast<uint64_t>(trees) * (is64 ? kTreeWords64 : kTreeWords32);
    }
    return w > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(w);
}

void ColPool::add(const NTerm& t) {
    if (rank_all) {
        ++nr;
        niv += is_in_kind(t.kind) ? in_count(t) : 1;
        return;
    }
    uint64_t entries = 0;
    if (is_in_kind(t.kind))
        entries = in_count(t);
    else if (term_cost(t) == 1)
        entries = 1;  // a single value: looked up like an EQ term
    if (!entries) {
        ++nr;
        ++niv;
        return;
    }
    if (nvs % 32 == 0) last = 0;  // a new group
    last += entries;
    most = std::max(most, last);
    ++nvs;
}

// Minimum compares a row needs for a term: one for a single value, two for a
// range, k for an IN list of k values.
uint64_t term_cost(const NTerm& t) {
    if (is_in_kind(t.kind)) return in_count(t);
    const bool single = t.kind == kRangeF32 ? t.a == t.b : t.b == 0;
    return single ? 1 : 2;
}

DevTerm make_devterm(const NTerm& t, uint32_t pool_off) {
    DevTerm d{};
    if (is_in_kind(t.kind)) {
        d.a_lo = pool_off;
        d.b_lo = in_count(t);
    } else {
        d.a_lo = static_cast<uint32_t>(t.a);
        d.a_hi = static_cast<uint32_t>(t.a >> 32);
        d.b_lo = static_cast<uint32_t>(t.b);
        d.b_hi = static_cast<uint32_t>(t.b >> 32);
    }
    return d;
}

// ---------------------------------------------------------------- sets


gace_status make_set(const gace_sample& s, SetDesc& d) {
    d = SetDesc{};
    if (s.kind > GACE_BLOCKS) return fail(GACE_EINVAL, "sample kind %u invalid", s.kind);
    d.kind = s.kind;
    d.mode = 1;
    if (s.kind == GACE_FULL) return GACE_OK;
    if (std::isnan(s.rate)) return fail(GACE_EINVAL, "sample rate is NaN");
    if (s.kind == GACE_BLOCKS && s.block_rows == 0)
        return fail(GACE_EINVAL, "block_rows must be >= 1");
    if (!(s.rate > 0.0)) {
        d.mode = 0;
    } else if (s.rate >= 1.0) {
        d.mode = 1;
    } else {
        d.mode = 2;
        d.thresh = static_cast<uint64_t>(std::ldexp(s.rate, 64));
    }
    d.seedhash = splitmix64_host(s.seed);
    d.block_rows = s.kind == GACE_BLOCKS ? s.block_rows : 1;
    d.block_shift = -1;
    if (s.kind == GACE_BLOCKS && (s.block_rows & (s.block_rows - 1)) == 0) {
        int sh = 0;
        while ((1ull << sh) < s.block_rows) ++sh;
        d.block_shift = sh;
    }
    return GACE_OK;
}

// ---------------------------------------------------------------- probe plan


gace_status check_ctx(gace_ctx* ctx) {
    if (!ctx) return fail(GACE_EINVAL, "context is NULL");
    return GACE_OK;
}

TableRec* find_table_raw(gace_ctx* ctx, uint32_t id) {
    auto it = ctx->tables.find(id);
    return it == ctx->tables.end() ? nullptr : &it->second;
}

gace_status complete_load(gace_ctx* ctx, TableRec& t) {
    if (t.pending.empty()) return GACE_OK;
    for (size_t c = 0; c < t.cols.size(); ++c)
        if (t.cols[c].bytes)
            CK(cudaMemcpyAsync(t.cols[c].dptr, t.pending[c], t.cols[c].bytes, cudaMemcpyHostToDevice, ctx->stream));
    // the served form's stream reads tables too: the copy is complete on return
    CK(cudaStreamSynchronize(ctx->stream));
    t.pending.clear();
    return GACE_OK;
}

TableRec* find_table(gace_ctx* ctx, uint32_t id) {
    TableRec* t = find_table_raw(ctx, id);
    if (t && !t->pending.empty() && complete_load(ctx, *t) != GACE_OK) return nullptr;
    return t;
}

gace_status read_status(gace_ctx* ctx, unsigned int st) {
    if (st & kStatusTimeout)
        return fail(GACE_ETIMEDOUT, "a device-side wait gave up after %llu ms",
                    (unsigned long long)(ctx->timeout_ns / 1000000ull));
    if (st & kStatusCasLimit) return fail(GACE_ETIMEDOUT, "a bounded device CAS loop gave up");
    return GACE_OK;
}

// Order-preserving unsigned key of a column value: the sign bit flipped for
// integers; for float32 bits, -0 taken as +0, negatives complemented, positives
// with the sign bit set, and NaN below every key (it is in no range).
uint64_t value_key(uint64_t bits, uint32_t dtype) {
    if (dtype == GACE_I32) return static_cast<uint32_t>(bits) ^ 0x80000000u;
    if (dtype == GACE_I64) return bits ^ 0x8000000000000000ull;
    uint32_t f = static_cast<uint32_t>(bits);
    if ((f << 1) == 0) f = 0;
    if ((f & 0x7FFFFFFFu) > 0x7F800000u) return 0;
    return (f & 0x80000000u) ? ~f : (f | 0x80000000u);
}

// Inclusive key interval of a normalised range term.
std::pair<uint64_t, uint64_t> range_keys(const NTerm& t, uint32_t dtype) {
    if (dtype == GACE_I32) {
        const uint32_t lo = static_cast<uint32_t>(t.a), hi = lo + static_cast<uint32_t>(t.b);
        return {value_key(lo, dtype), value_key(hi, dtype)};
    }
    if (dtype == GACE_I64) return {value_key(t.a, dtype), value_key(t.a + t.b, dtype)};
    return {value_key(t.a, dtype), value_key(t.b, dtype)};
}

// Inclusive key intervals of a normalised term: its range, or one one-key
// interval per IN value (NaN values were dropped, -0 keys as +0).
void term_intervals(const NTerm& t, uint32_t dtype, std::vector<std::pair<uint64_t, uint64_t>>& out) {
    out.clear();
    if (!is_in_kind(t.kind)) {
        out.push_back(range_keys(t, dtype));
        return;
    }
    const bool is64 = dtype == GACE_I64;
    for (size_t w = 0; w < t.in.size(); w += is64 ? 2 : 1) {
        const uint64_t bits = is64 ? (t.in[w] | (static_cast<uint64_t>(t.in[w + 1]) << 32)) : t.in[w];
        const uint64_t k = value_key(bits, dtype);
        out.push_back({k, k});
    }
}

// One group's interval tree (layout in gace_internal.h): endpoints are the
// intervals' starts and the keys just past their ends; the mask of rank r (r
// endpoints <= the key) holds the terms whose interval contains endpoint r-1.
void build_range_tree(const std::vector<std::pair<uint64_t, uint64_t>>& iv, bool is64, uint32_t* out) {
    const uint64_t kmax = is64 ? ~0ull : 0xFFFFFFFFull;
    std::vector<uint64_t> e;
    for (const auto& x : iv) {
        e.push_back(x.first);
        if (x.second < kmax) e.push_back(x.second + 1);
    }
    std::sort(e.begin(), e.end());
    e.erase(std::unique(e.begin(), e.end()), e.end());
    const size_t m = e.size();  // <= 64 for 32 intervals
    std::vector<uint64_t> sorted(e);
    sorted.resize(kTreeNodes, kmax);
    // level-order (1-based) layout of the perfect tree whose in-order is
    // `sorted`: node i on level L (2^L <= i < 2^(L+1)) is in-order element
    // ((2 (i - 2^L) + 1) << (levels - 1 - L)) - 1
    std::vector<uint64_t> node(kTreeNodes + 1);
    for (uint32_t L = 0; L < static_cast<uint32_t>(kTreeLevels); ++L)
        for (uint32_t i = 1u << L; i < (2u << L); ++i)
            node[i] = sorted[((2 * (i - (1u << L)) + 1) << (kTreeLevels - 1 - L)) - 1];
    uint32_t* masks = out + (is64 ? 2 * kTreeNodes + 2 : kTreeNodes + 1);
    for (size_t i = 1; i <= kTreeNodes; ++i) {
        if (is64) {
            out[2 * (i - 1)] = static_cast<uint32_t>(node[i]);
            out[2 * (i - 1) + 1] = static_cast<uint32_t>(node[i] >> 32);
        } else {
            out[i - 1] = static_cast<uint32_t>(node[i]);
        }
    }
    uint32_t last = 0;
    for (size_t r = 0; r <= kTreeNodes; ++r) {
        uint32_t mask = 0;
        if (r == 0) {
            mask = 0;
        } else if (r <= m) {
            for (size_t k = 0; k < iv.size(); ++k)
                if (iv[k].first <= e[r - 1] && e[r - 1] <= iv[k].second) mask |= 1u << k;
            last = mask;
        } else {
            mask = last;  // only the largest key reaches past the real endpoints
        }
        masks[r] = mask;
    }
}

// Two-choice (cuckoo) hash tables of a column's EQ/IN groups (layout in
// gace_internal.h): every group's keys are placed at one of their two slots,
// vs_slot(key, m1) or vs_slot(key, m2), moving a resident key to its other
// slot when both are taken (at most kCuckooKicks moves per insertion).  When
// a group cannot be placed, new multipliers are drawn (a fixed seeded
// sequence, so a batch always gets the same tables) and, every eighth try, the
// tables double.  All groups of a column share one capacity and the
// multipliers.
constexpr int kCuckooKicks = 96;

bool build_cuckoo(const std::vector<std::vector<VsEntry>>& keys, bool is64, uint32_t slot, uint32_t& tlog,
                  uint32_t& m1, uint32_t& m2, std::vector<uint32_t>& tabs) {
    const uint32_t ew = is64 ? 4u : 2u;
    for (uint32_t attempt = 0; attempt < 64; ++attempt) {
        if (attempt > 0 && attempt % 8 == 0) ++tlog;
        if (tlog > 20) return false;
        m1 = static_cast<uint32_t>(splitmix64_host(0xC0C0ull * (slot + 1) + 2 * attempt)) | 1u;
        m2 = static_cast<uint32_t>(splitmix64_host(0xC0C0ull * (slot + 1) + 2 * attempt + 1)) | 1u;
        if (m1 == m2) continue;
        const uint32_t cap = 1u << tlog;
        tabs.assign(static_cast<size_t>(keys.size()) * cap * ew, 0u);
        bool ok = true;
        for (size_t g = 0; g < keys.size() && ok; ++g) {
            uint32_t* tab = tabs.data() + g * cap * ew;
            for (const VsEntry& e0 : keys[g]) {
                VsEntry cur = e0;
                uint32_t at = vs_slot(cur.lo, cur.hi, m1, tlog);
                bool placed = false;
                for (int kick = 0; kick <= kCuckooKicks; ++kick) {
                    uint32_t* x = tab + static_cast<size_t>(at) * ew;
                    uint32_t& mask = is64 ? x[2] : x[1];
                    if (mask == 0) {
                        x[0] = cur.lo;
                        if (is64) x[1] = cur.hi;
                        mask = cur.mask;
                        placed = true;
                        break;
                    }
                    const VsEntry out{x[0], is64 ? x[1] : 0u, mask};  // evicted: goes to its other slot
                    x[0] = cur.lo;
                    if (is64) x[1] = cur.hi;
                    mask = cur.mask;
                    cur = out;
                    const uint32_t a1 = vs_slot(cur.lo, cur.hi, m1, tlog);
                    at = a1 == at ? vs_slot(cur.lo, cur.hi, m2, tlog) : a1;
                }
                if (!placed) {
                    ok = false;
                    break;
                }
            }
        }
        if (ok) return true;
    }
    return false;
}

// Builds the device form of a pass and the probe arguments (without pointers).
gace_status build_pass(gace_ctx* ctx, const TableRec& tab, Pass& ps, const std::vector<NTerm>& uterms,
                       const std::vector<std::vector<uint32_t>>& pred_u,
                       const std::vector<SetPlan>& sets, bool want_marg, bool force_wide, uint32_t wide_warps,
                       ProbePlan& plan) {
    std::vector<RankCode>& codes = plan.codes;
    const std::vector<int32_t>& code_of_col = plan.code_of_col;
    // Narrow passes (at most 32 predicates and terms) evaluate IN lists by
    // compare; wide passes look up every EQ and IN term of a column in that
    // column's hash tables.  Order: by column, ranges (or, wide, multi-value
    // ranges) first, then IN lists (or, wide, single values and IN lists).
    const bool narrow = !force_wide && ps.preds.size() <= static_cast<size_t>(kNarrowMax) &&
                        ps.uterms.size() <= static_cast<size_t>(kNarrowMax);
    // a wide pass reads every term of a column coded with all its terms by rank
    auto rank_all = [&](uint32_t col) {
        return !narrow && !code_of_col.empty() && code_of_col[col] >= 0 && codes[code_of_col[col]].all_terms;
    };
    auto valueset = [&](const NTerm& t) {
        return !rank_all(t.col) && (is_in_kind(t.kind) || (!narrow && term_cost(t) == 1));
    };
    std::vector<uint32_t> order = ps.uterms;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        const NTerm &a = uterms[x], &b = uterms[y];
        const int ia = valueset(a), ib = valueset(b);
        return std::tie(a.col, ia) < std::tie(b.col, ib);
    });
    std::vector<uint32_t> local(uterms.size(), 0);  // unique term -> index in the pass
    ps.uterms = order;
    ps.slots.clear();
    ps.dterms.clear();
    ps.pool.clear();
    ProbeArgs& A = ps.args;
    A = ProbeArgs{};
    uint32_t nslots = 0;
    for (uint32_t i = 0; i < order.size(); ++i) {
        const NTerm& t = uterms[order[i]];
        local[order[i]] = i;
        uint32_t poff = 0;
        if (narrow && is_in_kind(t.kind)) {
            poff = static_cast<uint32_t>(ps.pool.size());
            ps.pool.insert(ps.pool.end(), t.in.begin(), t.in.end());
        }
        ps.dterms.push_back(make_devterm(t, poff));
        ps.ops_per_row += term_cost(t);
        // a rank-coded column's EQ/IN terms take a slot of their own in a wide
        // pass (its ranges' slot reads ranks, not values)
        const bool coded = !narrow && !code_of_col.empty() && code_of_col[t.col] >= 0;
        const bool split = coded && nslots > 0 && ps.slots.back().first == t.col && valueset(t) &&
                           A.slots[nslots - 1].iend == A.slots[nslots - 1].rend &&
                           A.slots[nslots - 1].rend > A.slots[nslots - 1].rbeg;
        if (nslots == 0 || ps.slots.back().first != t.col || split) {
            if (nslots == kMaxSlots) return fail(GACE_EINVAL, "a pass references more than %d columns", kMaxSlots);
            ps.slots.push_back({t.col, i});
            SlotDesc& sd = A.slots[nslots++];
            const ColumnRec& c = tab.cols[t.col];
            sd.ptr = c.dptr;
            sd.dtype = static_cast<uint32_t>(c.dtype);
            sd.width = dtype_width(c.dtype);
            sd.rbeg = i;
            sd.rend = i;
            sd.iend = i;
        }
        SlotDesc& sd = A.slots[nslots - 1];
        if (valueset(t)) {
            sd.iend = i + 1;
        } else {
            sd.rend = i + 1;
            sd.iend = i + 1;
        }
    }
    if (!narrow) {
        // one two-choice hash table per group of 32 EQ/IN terms of a column:
        // key -> mask of the group's terms that contain it
        for (uint32_t s = 0; s < nslots; ++s) {
            SlotDesc& sd = A.slots[s];
            const uint32_t nvs = sd.iend - sd.rend;
            if (nvs == 0) continue;
            const bool is64 = sd.dtype == GACE_I64;
            sd.ngroups = (nvs + 31) / 32;
            // values of each term as (lo, hi) keys, floats with -0 -> +0
            std::vector<std::vector<std::pair<uint32_t, uint32_t>>> vals(nvs);
            size_t most = 0;
            for (uint32_t k = 0; k < nvs; ++k) {
                const NTerm& t = uterms[order[sd.rend + k]];
                if (is_in_kind(t.kind)) {
                    for (size_t w = 0; w < t.in.size(); w += is64 ? 2 : 1)
                        vals[k].push_back({t.in[w], is64 ? t.in[w + 1] : 0u});
                } else {
                    vals[k].push_back({static_cast<uint32_t>(t.a), is64 ? static_cast<uint32_t>(t.a >> 32) : 0u});
                }
                if (sd.dtype == GACE_F32)
                    for (auto& kv : vals[k])
                        if ((kv.first << 1) == 0) kv.first = 0;
            }
            // distinct keys of each group with the mask of the group's terms that hold them
            std::vector<std::vector<VsEntry>> keys(sd.ngroups);
            for (uint32_t g = 0; g < sd.ngroups; ++g) {
                std::vector<VsEntry>& out = keys[g];
                for (uint32_t k = 32 * g; k < std::min(nvs, 32 * g + 32); ++k)
                    for (const auto& kv : vals[k]) out.push_back({kv.first, kv.second, 1u << (k - 32 * g)});
                std::sort(out.begin(), out.end(), [](const VsEntry& x, const VsEntry& y) {
                    return x.hi != y.hi ? x.hi < y.hi : x.lo < y.lo;
                });
                size_t n = 0;  // equal keys merged: one entry with the OR of their terms
                for (size_t i = 0; i < out.size(); ++i) {
                    if (n && out[n - 1].lo == out[i].lo && out[n - 1].hi == out[i].hi)
                        out[n - 1].mask |= out[i].mask;
                    else
                        out[n++] = out[i];
                }
                out.resize(n);
                most = std::max(most, out.size());
            }
            uint32_t tlog = 6;
            while ((1ull << tlog) < kVsSlotsPerEntry * most) ++tlog;
            std::vector<uint32_t> tabs;
            uint32_t m1 = 0, m2 = 0;
            if (!build_cuckoo(keys, is64, s, tlog, m1, m2, tabs))
                return fail(GACE_EINVAL, "no two-choice table holds the EQ/IN values of a column");
            sd.tlog = tlog;
            sd.vm1 = m1;
            sd.vm2 = m2;
            sd.toff = static_cast<uint32_t>(ps.pool.size());
            ps.pool.insert(ps.pool.end(), tabs.begin(), tabs.end());
        }
    }
    if (!narrow) {
        // rank-coded columns: per group of 32 range terms, the mask of the
        // group's terms that hold each rank's keys (rank r: the keys from
        // endpoint r-1 up to endpoint r; rank 0 lies below every interval)
        for (uint32_t s = 0; s < nslots; ++s) {
            SlotDesc& sd = A.slots[s];
            const uint32_t nr = sd.rend - sd.rbeg;
            const uint32_t col = ps.slots[s].first;
            if (nr == 0 || code_of_col.empty() || code_of_col[col] < 0) continue;
            if (sd.iend != sd.rend) return fail(GACE_EINVAL, "rank-coded slot of column %u holds EQ/IN terms", col);
            RankCode& rc = codes[code_of_col[col]];
            rc.used = true;
            const uint32_t m = static_cast<uint32_t>(rc.keys.size());
            // the slot's own endpoints (local) marked among the column's, and
            // pre[r] = the local endpoints below column endpoint r: a row of
            // column rank r has local rank pre[r]
            std::vector<uint32_t> pre(m + 1, 0u);
            for (uint32_t k = 0; k < nr; ++k) {
                const uint32_t u = order[sd.rbeg + k];
                for (uint32_t i = plan.span_off[u]; i < plan.span_off[u + 1]; ++i) {
                    pre[plan.span[i].first] = 1;
                    if (plan.span[i].second < m) pre[plan.span[i].second] = 1;
                }
            }
            uint32_t ml = 0;
            for (uint32_t r = 0; r <= m; ++r) {
                const uint32_t mark = pre[r];
                pre[r] = ml;
                ml += r < m ? mark : 0u;
            }
            sd.rtree = nr;
            sd.rgroups = (nr + 31) / 32;
            // a map from column rank to local rank (bytes, or 16-bit entries
            // past 255 local endpoints) when it takes less room
            const uint32_t mapw = ml <= 255 ? 1 : 2;
            const uint64_t direct = static_cast<uint64_t>(sd.rgroups) * (m + 1);
            const uint64_t mapped = ((m + 1) * mapw + 3) / 4 + static_cast<uint64_t>(sd.rgroups) * (ml + 1);
            const bool use_map = mapped < direct;
            if (use_map) {
                const uint32_t off = static_cast<uint32_t>(ps.pool.size());
                sd.rmap = (off + 1) | (mapw == 2 ? kRankMap16 : 0u);
                ps.pool.resize(ps.pool.size() + ((m + 1) * mapw + 3) / 4, 0u);
                unsigned char* map8 = reinterpret_cast<unsigned char*>(ps.pool.data() + off);
                uint16_t* map16 = reinterpret_cast<uint16_t*>(ps.pool.data() + off);
                for (uint32_t r = 0; r <= m; ++r) {
                    if (mapw == 1)
                        map8[r] = static_cast<unsigned char>(pre[r]);
                    else
                        map16[r] = static_cast<uint16_t>(pre[r]);
                }
            }
            sd.rstride = use_map ? ml + 1 : m + 1;
            sd.roff = static_cast<uint32_t>(ps.pool.size());
            ps.pool.resize(ps.pool.size() + static_cast<size_t>(sd.rgroups) * sd.rstride, 0u);
            // mask of rank s >= 1: the terms holding the (s-1)-th endpoint
            // (local or column); a term's intervals do not overlap, so each
            // toggles its bit on at its first endpoint and off past its last
            std::vector<uint32_t> flip(sd.rstride + 1);
            for (uint32_t g = 0; g < sd.rgroups; ++g) {
                std::fill(flip.begin(), flip.end(), 0u);
                for (uint32_t k = 32 * g; k < std::min(nr, 32 * g + 32); ++k) {
                    const uint32_t u = order[sd.rbeg + k], bit = 1u << (k % 32);
                    for (uint32_t i = plan.span_off[u]; i < plan.span_off[u + 1]; ++i) {
                        const uint32_t a = use_map ? pre[plan.span[i].first] : plan.span[i].first;
                        const uint32_t b = use_map ? pre[plan.span[i].second] : plan.span[i].second;
                        flip[a] ^= bit;
                        flip[b] ^= bit;
                    }
                }
                uint32_t* masks = ps.pool.data() + sd.roff + static_cast<size_t>(g) * sd.rstride;
                uint32_t run = 0;
                for (uint32_t r = 0; r + 1 < sd.rstride; ++r) {
                    run ^= flip[r];
                    masks[r + 1] = run;
                }
            }
        }
        A.ranks_only = 1;
        bool all_ranked = nslots > 0;  // every term of the pass read by rank
        for (uint32_t s = 0; s < nslots; ++s) {
            if (A.slots[s].rend > A.slots[s].rbeg && !A.slots[s].rstride) A.ranks_only = 0;
            if (!A.slots[s].rstride || A.slots[s].iend != A.slots[s].rend) all_ranked = false;
        }
        for (uint32_t s = 0; s < nslots && all_ranked; ++s)
            all_ranked = codes[code_of_col[ps.slots[s].first]].hist;
        ps.hist_marg = want_marg && all_ranked;
        // one interval tree per full group of 32 range terms of a column (and
        // per last group of at least kTreeMin); fewer terms are cheaper by compare
        for (uint32_t s = 0; s < nslots; ++s) {
            SlotDesc& sd = A.slots[s];
            if (sd.rstride) continue;
            const uint32_t all = sd.rend - sd.rbeg, rem = all % 32;
            const uint32_t nr = all - (rem >= kTreeMin ? 0 : rem);
            sd.rtree = nr;
            if (nr == 0) continue;
            const bool is64 = sd.dtype == GACE_I64;
            const uint32_t gw = is64 ? kTreeWords64 : kTreeWords32;
            if (ps.pool.size() & 1) ps.pool.push_back(0);  // 8-byte aligned key pairs
            sd.rgroups = (nr + 31) / 32;
            sd.roff = static_cast<uint32_t>(ps.pool.size());
            ps.pool.resize(ps.pool.size() + static_cast<size_t>(sd.rgroups) * gw, 0u);
            for (uint32_t g = 0; g < sd.rgroups; ++g) {
                std::vector<std::pair<uint64_t, uint64_t>> iv;  // inclusive key intervals
                for (uint32_t k = 32 * g; k < std::min(nr, 32 * g + 32); ++k)
                    iv.push_back(range_keys(uterms[order[sd.rbeg + k]], sd.dtype));
                build_range_tree(iv, is64, ps.pool.data() + sd.roff + static_cast<size_t>(g) * gw);
            }
        }
    }
    // a wide pass's lanes take every 32nd predicate: ordered by term count,
    // the lanes of one step AND as many masks each
    if (!narrow)
        std::stable_sort(ps.preds.begin(), ps.preds.end(),
                         [&](uint32_t x, uint32_t y) { return pred_u[x].size() > pred_u[y].size(); });
    ps.poff.assign(1, 0);
    ps.pterm.clear();
    for (uint32_t p : ps.preds) {
        for (uint32_t u : pred_u[p]) ps.pterm.push_back(local[u]);
        ps.poff.push_back(static_cast<uint32_t>(ps.pterm.size()));
    }
    A.nrows = tab.nrows;
    A.nslots = nslots;
    A.nsets = static_cast<uint32_t>(sets.size());
    for (uint32_t q = 0; q < sets.size(); ++q) A.sets[q] = sets[q].d;
    A.nterms = static_cast<uint32_t>(ps.dterms.size());
    A.npreds = static_cast<uint32_t>(ps.preds.size());
    A.npool = static_cast<uint32_t>(ps.pool.size());
    A.npredterms = static_cast<uint32_t>(ps.pterm.size());
    A.want_marg = want_marg && !ps.hist_marg ? 1u : 0u;
    A.timeout_ns = ctx->timeout_ns;
    A.nwarps = narrow ? static_cast<uint32_t>(kProbeWarps) : wide_warps;

    // Narrow passes (the gate's single probes) stream staged tiles of about
    // 32 KB through a bulk-copy pipeline two or three stages deep (at most
    // 64 KB per CTA, so that three or four CTAs fit on an SM); wide passes are
    // ALU-bound and load directly.
    uint32_t rowbytes = 0;  // a rank-coded slot reads the rows' 16-bit ranks
    for (uint32_t s = 0; s < nslots; ++s) rowbytes += A.slots[s].rstride ? 2u : A.slots[s].width;
    ps.rowbytes = rowbytes;
    A.narrow = narrow ? 1u : 0u;
    const uint32_t sweep = (A.narrow ? 2u : 1u) * kSliceRows * kProbeWarps;  // rows of one CTA sweep
#ifndef GACE_STAGE_TARGET_KB
#define GACE_STAGE_TARGET_KB 32
#endif
    uint32_t tile_rows = sweep;
    if (rowbytes > 0)
        while (tile_rows * 2 * rowbytes <= (GACE_STAGE_TARGET_KB << 10) && tile_rows < 8 * sweep)
            tile_rows *= 2;  // stages of about GACE_STAGE_TARGET_KB
    else
        tile_rows = 8 * sweep;
    A.tile_rows = tile_rows;
    bool aligned = true;
    for (uint32_t s = 0; s < nslots; ++s)
        if (reinterpret_cast<uintptr_t>(A.slots[s].ptr) & 15u) aligned = false;
    bool staged = A.narrow && aligned && nslots > 0;
    // At most kStageBudget bytes of stages per CTA, so that three or four CTAs
    // fit on an SM whatever the referenced columns (a fused pass over many
    // wide columns would otherwise hold a whole SM's shared memory); rows too
    // wide for two stages are read with plain loads.
#ifndef GACE_STAGE_BUDGET_KB
#define GACE_STAGE_BUDGET_KB 64
#endif
    constexpr uint32_t kStageBudget = static_cast<uint32_t>(GACE_STAGE_BUDGET_KB) << 10;
    uint32_t nst = 3;
    while (staged && nst > 2 && nst * tile_rows * rowbytes > kStageBudget) --nst;
    if (staged && nst * tile_rows * rowbytes > kStageBudget) staged = false;
    for (;;) {
        A.nstages = staged ? nst : 1;
        A.stage_bytes = staged ? tile_rows * rowbytes : 0;
        uint32_t off = 0;
        for (uint32_t s = 0; s < nslots; ++s) {
            A.slots[s].soff = off;
            off += tile_rows * A.slots[s].width;
        }
        probe_layout(A);
        if (A.smem_bytes <= static_cast<uint32_t>(ctx->smem_optin)) break;
        if (staged && nst > 2) {
            --nst;
        } else if (staged) {
            staged = false;
        } else {
            return fail(GACE_EINVAL, "probe pass needs %u bytes of shared memory (limit %d)",
                        A.smem_bytes, ctx->smem_optin);
        }
    }
    A.ntiles = (tab.nrows + A.tile_rows - 1) / A.tile_rows;
    A.nstaged = staged ? tab.nrows / A.tile_rows : 0;
    // A narrow pass whose row sets are all block samples reads only the tiles
    // that hold a sampled block (the point of sampling whole blocks), when a
    // tile spans few enough blocks to test them all.
    bool blocks_only = A.narrow && A.nsets > 0;
    for (uint32_t q = 0; q < A.nsets; ++q) {
        const SetDesc& d = A.sets[q];
        blocks_only = blocks_only && d.kind == 2 && d.mode == 2 && d.block_rows * kSkipBlocksPerTile >= A.tile_rows;
    }
    A.skip_tiles = blocks_only ? 1u : 0u;
    return GACE_OK;
}


double hll_estimate_host(const uint8_t* regs, uint32_t p) {
    const uint64_t m = 1ull << p;
    uint64_t hist[66] = {0};
    for (uint64_t j = 0; j < m; ++j) hist[regs[j] < 65 ? regs[j] : 65]++;
    return hll_estimate_from_hist(hist, p);
}

}  // namespace host

double hll_estimate_from_hist(const uint64_t (&c)[66], uint32_t p) {
    const double dm = static_cast<double>(1ull << p);
    double alpha;
    if (p == 4) alpha = 0.673;
    else if (p == 5) alpha = 0.697;
    else if (p == 6) alpha = 0.709;
    else alpha = 0.7213 / (1.0 + 1.079 / dm);
    double z = 0.0;
    for (int k = 0; k <= 65; ++k) z += static_cast<double>(c[k]) * std::ldexp(1.0, -k);
    double e = alpha * dm * dm / z;
    if (e <= 2.5 * dm && c[0] > 0) e = dm * std::log(dm / static_cast<double>(c[0]));
    return e;
}

namespace host {

// Staged side scans (k_side_staged) stream tiles of about 32 KB per stage
// through two or three stages (at most 64 KB per CTA, three CTAs per SM), like
// the narrow probes; columns that are not 16-byte aligned, or rows too wide
// for two stages, keep the direct-load kernel (stage_bytes = 0).
#ifndef GACE_SIDE_STAGED
#define GACE_SIDE_STAGED 1
#endif
#ifndef GACE_SIDE_TARGET_KB
#define GACE_SIDE_TARGET_KB 32
#endif
#ifndef GACE_SIDE_BUDGET_KB
#define GACE_SIDE_BUDGET_KB 64
#endif
#ifndef GACE_SIDE_STAGES
#define GACE_SIDE_STAGES 3
#endif
void plan_side_stages(SideArgs& a) {
    constexpr uint32_t kTarget = GACE_SIDE_TARGET_KB << 10, kBudget = GACE_SIDE_BUDGET_KB << 10;
    static_assert(GACE_SIDE_STAGES >= 2 && GACE_SIDE_STAGES <= kMaxStages, "stage count");
    const uint32_t sweep = kSideSlice * kSideWarps;
    uint32_t rowbytes = 0;
    bool aligned = true;
    for (uint32_t s = 0; s < a.nslots; ++s) {
        rowbytes += a.slot_width[s];
        aligned = aligned && a.slot_aligned[s];
    }
    a.stage_bytes = 0;
    a.nstages = 1;
    a.tile_rows = sweep;
    uint32_t tile = sweep;
    while (tile * 2 * rowbytes <= kTarget && tile < 8 * sweep) tile *= 2;
    uint32_t nst = GACE_SIDE_STAGES;
    while (nst > 2 && nst * tile * rowbytes > kBudget) --nst;
    if (!GACE_SIDE_STAGED || !aligned || rowbytes == 0 || nst * tile * rowbytes > kBudget) return;
    a.tile_rows = tile;
    a.nstages = nst;
    a.stage_bytes = tile * rowbytes;
    uint32_t off = 0;
    for (uint32_t s = 0; s < a.nslots; ++s) {
        a.slot_soff[s] = off;
        off += tile * a.slot_width[s];
    }
    a.smem_bytes = kSideStageOff + nst * a.stage_bytes;
    a.ntiles = (a.nrows + tile - 1) / tile;
    a.nstaged = a.nrows / tile;
}

gace_status build_side(gace_ctx* ctx, const gace_join_side& js, const char* name, int extra_col,
                              SideArgs& a, std::vector<uint32_t>& pool, TableRec** tab_out, uint32_t* extra_slot,
                              SideWork& work) {
    TableRec* tab = find_table(ctx, js.table_id);
    if (!tab) return fail(GACE_ENOTFOUND, "%s table %u is not loaded", name, js.table_id);
    if (js.key_col >= tab->cols.size()) return fail(GACE_EINVAL, "%s key column %u out of range", name, js.key_col);
    if (tab->cols[js.key_col].dtype == GACE_F32) return fail(GACE_EINVAL, "%s key column is float32", name);
    if (js.nterms && !js.terms) return fail(GACE_EINVAL, "%s terms is NULL", name);
    if (js.nterms > static_cast<uint32_t>(kMaxFilterTerms))
        return fail(GACE_EINVAL, "%s filter has %u terms (max %d)", name, js.nterms, kMaxFilterTerms);
    a = SideArgs{};
    a.nrows = tab->nrows;
    std::vector<uint32_t> slot_col;
    auto slot_of = [&](uint32_t col) -> int {
        for (uint32_t s = 0; s < slot_col.size(); ++s)
            if (slot_col[s] == col) return static_cast<int>(s);
        if (slot_col.size() == static_cast<size_t>(kMaxFilterSlots)) return -1;
        slot_col.push_back(col);
        return static_cast<int>(slot_col.size() - 1);
    };
    a.key_slot = static_cast<uint32_t>(slot_of(js.key_col));
    if (extra_col >= 0) {
        if (static_cast<uint32_t>(extra_col) >= tab->cols.size() || tab->cols[extra_col].dtype == GACE_F32)
            return fail(GACE_EINVAL, "%s fk2 column %d invalid", name, extra_col);
        *extra_slot = static_cast<uint32_t>(slot_of(static_cast<uint32_t>(extra_col)));
    }
    uint32_t nt = 0;
    bool never = false;
    for (uint32_t t = 0; t < js.nterms; ++t) {
        if (js.terms[t].col >= tab->cols.size())
            return fail(GACE_EINVAL, "%s term %u references column %u", name, t, js.terms[t].col);
        NTerm n;
        if (gace_status st = normalize_term(js.terms[t], tab->cols[js.terms[t].col].dtype, js.in_values, js.nin, n))
            return st;
        if (n.kind == kFalse) {
            never = true;
            continue;
        }
        const int s = slot_of(n.col);
        if (s < 0) return fail(GACE_EINVAL, "%s filter references more than %d columns", name, kMaxFilterSlots);
        FilterTerm& ft = a.terms[nt++];
        ft.slot = static_cast<uint32_t>(s);
        ft.kind = n.kind;
        work.ops_per_row += term_cost(n);
        uint32_t poff = static_cast<uint32_t>(pool.size());
        if (is_in_kind(n.kind)) pool.insert(pool.end(), n.in.begin(), n.in.end());
        ft.c = make_devterm(n, poff);
    }
    if (never) {  // an always-false term: a range no value satisfies on the key column
        nt = 0;
        FilterTerm& ft = a.terms[nt++];
        ft.slot = a.key_slot;
        ft.kind = kInI32;
        ft.c = DevTerm{0, 0, 0, 0};  // empty IN list
    }
    a.nterms = nt;
    a.nslots = static_cast<uint32_t>(slot_col.size());
    work.rows = tab->nrows;
    for (uint32_t c : slot_col) work.rowbytes += dtype_width(tab->cols[c].dtype);
    for (uint32_t s = 0; s < slot_col.size(); ++s) {
        a.slot_ptr[s] = tab->cols[slot_col[s]].dptr;
        a.slot_dtype[s] = static_cast<uint32_t>(tab->cols[slot_col[s]].dtype);
        a.slot_aligned[s] = (reinterpret_cast<uintptr_t>(a.slot_ptr[s]) & 15u) == 0;
        a.slot_width[s] = dtype_width(tab->cols[slot_col[s]].dtype);
    }
    a.timeout_ns = ctx->timeout_ns;
    plan_side_stages(a);
    *tab_out = tab;
    return GACE_OK;
}

// ---------------------------------------------------------------- probe

gace_status check_probe_request(const ProbeRequest& r) {
    if (!r.samples || r.nsamples == 0 || r.nsamples > kMaxSets)
        return fail(GACE_EINVAL, "nsamples %u outside 1..%d", r.nsamples, kMaxSets);
    if (r.npreds && (!r.preds || !r.results)) return fail(GACE_EINVAL, "preds or results is NULL");
    if (r.nterms && !r.terms) return fail(GACE_EINVAL, "terms is NULL");
    if (r.nterms > (1u << 24) || r.npreds > (1u << 24)) return fail(GACE_EINVAL, "batch too large");
    return GACE_OK;
}

// Distinct 64-bit keys in insertion order with an open-addressing index
// (linear probing on a splitmix64 hash) from each key to a value.
struct KeyIndex {
    std::vector<uint64_t> key;
    std::vector<uint32_t> val;
    std::vector<uint8_t> used;
    std::vector<uint64_t> distinct;
    uint64_t mask = 0;
    void init(uint64_t n) {
        uint64_t cap = 16;
        while (cap < 2 * n) cap <<= 1;
        key.assign(cap, 0);
        val.assign(cap, 0);
        used.assign(cap, 0);
        distinct.clear();
        mask = cap - 1;
    }
    uint64_t slot_of(uint64_t k) const {
        uint64_t i = splitmix64_host(k) & mask;
        while (used[i] && key[i] != k) i = (i + 1) & mask;
        return i;
    }
    void insert(uint64_t k) {
        const uint64_t i = slot_of(k);
        if (used[i]) return;
        used[i] = 1;
        key[i] = k;
        distinct.push_back(k);
    }
    void set(uint64_t k, uint32_t v) { val[slot_of(k)] = v; }
    uint32_t find(uint64_t k) const { return val[slot_of(k)]; }  // k was inserted
};

// The search tree of a rank-coded column's endpoints (RankArgs): the
// perfect tree whose in-order is the sorted keys padded with the largest key,
// in level order (node i of level L, 2^L <= i < 2^(L+1), is in-order element
// ((2 (i - 2^L) + 1) << (levels - 1 - L)) - 1).
void build_rank_tree(RankCode& rc) {
    const bool is64 = rc.dtype == GACE_I64;
    const uint64_t kmax = is64 ? ~0ull : 0xFFFFFFFFull;
    const uint32_t m = static_cast<uint32_t>(rc.keys.size());
    uint32_t levels = 1;
    while ((1u << levels) - 1 < m) ++levels;
    rc.levels = levels;
    const uint32_t nkeys = (1u << levels) - 1;
    std::vector<uint64_t> sorted(rc.keys);
    sorted.resize(nkeys, kmax);
    rc.tree.assign(is64 ? 2 * nkeys : nkeys, 0u);
    for (uint32_t L = 0; L < levels; ++L)
        for (uint32_t i = 1u << L; i < (2u << L); ++i) {
            const uint64_t key = sorted[((2 * (i - (1u << L)) + 1) << (levels - 1 - L)) - 1];
            if (is64) {
                rc.tree[2 * (i - 1)] = static_cast<uint32_t>(key);
                rc.tree[2 * (i - 1) + 1] = static_cast<uint32_t>(key >> 32);
            } else {
                rc.tree[i - 1] = static_cast<uint32_t>(key);
            }
        }
}

// Bucket of key distance d (RankArgs): linear buckets of 2^smin keys up to
// 2^(smin + mbits + 1), then 2^mbits buckets per doubling of d.
static inline uint64_t rank_bucket(uint64_t d, uint32_t smin, uint32_t mbits) {
    const int len = d ? 64 - __builtin_clzll(d) : 0;
    const uint32_t s = std::max<int>(static_cast<int>(smin), len - static_cast<int>(mbits) - 1);
    return (static_cast<uint64_t>(s - smin) << mbits) + (d >> s);
}

// A bucket index of a rank-coded column's endpoints instead of its search
// tree (search: gace_config.rank_search): of linear buckets and of buckets
// growing with the distance from the smallest endpoint (at most kRankBuckets
// of either), the one whose fullest bucket needs the fewest halvings, taken
// when it needs at least two fewer dependent shared-memory loads than the
// tree (always under search 2, never under search 1).
void build_rank_buckets(RankCode& rc, uint32_t search) {
    constexpr uint64_t kRankBuckets = 8192;
    const uint32_t m = static_cast<uint32_t>(rc.keys.size());
    if (search == 1 || m == 0) return;
    const bool is64 = rc.dtype == GACE_I64;
    const uint32_t maxbits = is64 ? 63u : 31u;
    const uint64_t base = rc.keys.front(), span = rc.keys.back() - base;
    struct Cand {
        uint32_t smin = 0, mbits = 0, steps = 99;
        uint64_t nb = 0;
    } best;
    for (uint32_t mbits : {maxbits, 8u, 6u}) {
        uint32_t smin = 0;
        while (rank_bucket(span, smin, mbits) >= kRankBuckets) ++smin;
        const uint64_t nb = rank_bucket(span, smin, mbits) + 1;
        uint64_t fullest = 0, run = 0, prev = ~0ull;
        for (uint64_t k : rc.keys) {
            const uint64_t b = rank_bucket(k - base, smin, mbits);
            run = b == prev ? run + 1 : 1;
            prev = b;
            fullest = std::max(fullest, run);
        }
        uint32_t steps = 0;
        while ((1ull << steps) < fullest + 1) ++steps;
        if (steps < best.steps || (steps == best.steps && nb < best.nb)) best = {smin, mbits, steps, nb};
    }
    if (search == 0 && best.steps + 1 + 2 > rc.levels) return;
    const uint64_t kmax = is64 ? ~0ull : 0xFFFFFFFFull;
    const uint64_t nends = m + (1ull << best.steps);
    // the 16-bit first indices take whole 8-byte units, so that the (lo, hi)
    // endpoint pairs of an int64 column start 8-byte aligned
    const uint64_t start_words = rank_start_words(static_cast<uint32_t>(best.nb));
    std::vector<uint32_t> words(start_words + nends * (is64 ? 2 : 1), 0u);
    uint16_t* start = reinterpret_cast<uint16_t*>(words.data());
    std::vector<uint32_t> bucket(m);  // each endpoint's bucket (non-decreasing)
    for (uint32_t k = 0; k < m; ++k)
        bucket[k] = static_cast<uint32_t>(rank_bucket(rc.keys[k] - base, best.smin, best.mbits));
    uint32_t i = 0;
    for (uint64_t b = 0; b < best.nb; ++b) {  // first endpoint at or after bucket b
        while (i < m && bucket[i] < b) ++i;
        start[b] = static_cast<uint16_t>(i);
    }
    uint32_t* ends = words.data() + start_words;
    for (uint64_t e = 0; e < nends; ++e) {
        const uint64_t key = e < m ? rc.keys[e] : kmax;
        if (is64) {
            ends[2 * e] = static_cast<uint32_t>(key);
            ends[2 * e + 1] = static_cast<uint32_t>(key >> 32);
        } else {
            ends[e] = static_cast<uint32_t>(key);
        }
    }
    rc.tree = std::move(words);
    rc.levels = 0;
    rc.bbase = base;
    rc.bnb = static_cast<uint32_t>(best.nb);
    rc.bsmin = best.smin;
    rc.bmbits = best.mbits;
    rc.bsteps = best.steps;
}

gace_status plan_probe(gace_ctx* ctx, const TableRec& tab, const ProbeRequest& r, bool force_wide,
                       ProbePlan& plan, uint32_t wide_warps, bool rank_code, bool trace) {
    auto phase = [&](const char* name) {
        if (trace) ctx->host_phase(name);
    };
    plan = ProbePlan();
    plan.tab = &tab;
    const uint32_t nsamples = r.nsamples, nterms = r.nterms, npreds = r.npreds;
    // Device row sets: one set for every sample that keeps all rows (full
    // scans, rate >= 1), then one per distinct hashed sample, ordered so that
    // sets sharing a hash input are adjacent.  Samples of rate <= 0 need no
    // device work.
    std::vector<SetDesc> sdesc(nsamples);
    for (uint32_t s = 0; s < nsamples; ++s)
        if (gace_status st = make_set(r.samples[s], sdesc[s])) return st;
    std::vector<SetPlan>& sets = plan.sets;
    std::vector<int32_t>& set_dev = plan.set_dev;
    set_dev.assign(nsamples, -1);
    for (uint32_t s = 0; s < nsamples; ++s)
        if (sdesc[s].mode == 1) {
            if (sets.empty()) {
                SetPlan v;
                v.d = SetDesc{};
                v.d.kind = 0;
                v.d.mode = 1;
                v.d.block_shift = -1;
                v.orig = s;
                sets.push_back(v);
            }
            set_dev[s] = 0;
        }
    std::vector<SetPlan> hashed;
    for (uint32_t s = 0; s < nsamples; ++s)
        if (sdesc[s].mode == 2) hashed.push_back({sdesc[s], s});
    std::stable_sort(hashed.begin(), hashed.end(), [](const SetPlan& a, const SetPlan& b) {
        return std::tie(a.d.kind, a.d.seedhash, a.d.block_rows, a.d.thresh) <
               std::tie(b.d.kind, b.d.seedhash, b.d.block_rows, b.d.thresh);
    });
    for (const SetPlan& h : hashed) {
        const SetDesc* last = sets.empty() ? nullptr : &sets.back().d;
        if (last && last->mode == 2 && last->kind == h.d.kind && last->seedhash == h.d.seedhash &&
            last->block_rows == h.d.block_rows && last->thresh == h.d.thresh) {
            set_dev[h.orig] = static_cast<int32_t>(sets.size() - 1);  // identical sample
            continue;
        }
        SetPlan c = h;
        c.d.share_prev = (last && last->mode == 2 && last->kind == c.d.kind && last->seedhash == c.d.seedhash &&
                          last->block_rows == c.d.block_rows)
                             ? 1u
                             : 0u;
        set_dev[h.orig] = static_cast<int32_t>(sets.size());
        sets.push_back(c);
    }

    phase("host_plan_sets");
    // normalise and deduplicate terms
    std::vector<NTerm>& uterms = plan.uterms;
    uterms.reserve(nterms);
    std::unordered_map<NTerm, uint32_t, NTermHash> dedup;
    dedup.reserve(nterms);
    plan.t2u.assign(nterms, 0);
    for (uint32_t t = 0; t < nterms; ++t) {
        if (r.terms[t].col >= tab.cols.size())
            return fail(GACE_EINVAL, "term %u references column %u of a %zu-column table", t, r.terms[t].col,
                        tab.cols.size());
        NTerm n;
        if (gace_status st = normalize_term(r.terms[t], tab.cols[r.terms[t].col].dtype, r.in_values, r.nin, n))
            return st;
        if (n.kind == kFalse) {
            plan.t2u[t] = UINT32_MAX;
            continue;
        }
        const auto ins = dedup.try_emplace(n, static_cast<uint32_t>(uterms.size()));
        if (ins.second) uterms.push_back(std::move(n));
        plan.t2u[t] = ins.first->second;
    }
    // predicates: 0 device, 1 never true, 2 always true (no terms)
    plan.pstate.assign(npreds, 0);
    plan.pred_u.assign(npreds, {});
    bool any_pair = false;
    for (uint32_t p = 0; p < npreds; ++p) {
        const gace_pred& pr = r.preds[p];
        if ((uint64_t)pr.term_off + pr.term_cnt > nterms)
            return fail(GACE_EINVAL, "predicate %u terms [%u, %u) outside terms[%u]", p, pr.term_off,
                        pr.term_off + pr.term_cnt, nterms);
        if (pr.term_cnt == 2) any_pair = true;
        if (pr.term_cnt == 0) {
            plan.pstate[p] = 2;
            continue;
        }
        std::vector<uint32_t>& pu = plan.pred_u[p];
        for (uint32_t k = 0; k < pr.term_cnt; ++k) {
            const uint32_t u = plan.t2u[pr.term_off + k];
            if (u == UINT32_MAX) {
                plan.pstate[p] = 1;
                break;
            }
            pu.push_back(u);
        }
        std::sort(pu.begin(), pu.end());
        pu.erase(std::unique(pu.begin(), pu.end()), pu.end());
        if (plan.pstate[p] == 1) pu.clear();
    }
    plan.want_marg = r.term_marginals != nullptr || any_pair;

    phase("host_plan_terms");
    // rank coding: every column's distinct range endpoints over the whole plan
    plan.code_of_col.assign(tab.cols.size(), -1);
    // ranks pay for their pre-pass when several wide passes read them: a
    // batch of more predicates than a narrow pass holds, with more terms than
    // one wide pass holds, over a table of at least kRankMinRows rows
    rank_code = rank_code && npreds > static_cast<uint32_t>(kNarrowMax) && uterms.size() >= kRankMinTerms &&
                tab.nrows >= (ctx->rank_min_rows ? ctx->rank_min_rows : kRankMinRows);
    if (rank_code) {
        // per column, the distinct endpoints of all its terms' key intervals
        // (all terms are coded when they fit), else of its multi-value ranges
        const size_t ncols = tab.cols.size();
        std::vector<uint32_t> ivo(uterms.size() + 1, 0);  // term u's intervals: iv[ivo[u] .. ivo[u + 1])
        std::vector<std::pair<uint64_t, uint64_t>> iv, ivs;
        std::vector<uint64_t> nends(ncols, 0);
        for (uint32_t u = 0; u < uterms.size(); ++u) {
            const NTerm& t = uterms[u];
            term_intervals(t, static_cast<uint32_t>(tab.cols[t.col].dtype), ivs);
            iv.insert(iv.end(), ivs.begin(), ivs.end());
            ivo[u + 1] = static_cast<uint32_t>(iv.size());
            nends[t.col] += 2 * ivs.size();
        }
        std::vector<KeyIndex> all(ncols);
        for (uint32_t c = 0; c < ncols; ++c)
            if (nends[c]) all[c].init(nends[c]);
        std::vector<std::vector<uint64_t>> rng(ncols);
        for (uint32_t u = 0; u < uterms.size(); ++u) {
            const NTerm& t = uterms[u];
            const uint64_t kmax = tab.cols[t.col].dtype == GACE_I64 ? ~0ull : 0xFFFFFFFFull;
            const bool range = !is_in_kind(t.kind) && term_cost(t) == 2;
            for (uint32_t i = ivo[u]; i < ivo[u + 1]; ++i) {
                all[t.col].insert(iv[i].first);
                if (iv[i].second < kmax) all[t.col].insert(iv[i].second + 1);
                if (range) {
                    rng[t.col].push_back(iv[i].first);
                    if (iv[i].second < kmax) rng[t.col].push_back(iv[i].second + 1);
                }
            }
        }
        // each column's code (its endpoints sorted, their search tree or
        // bucket index): independent per column, so on the context's host
        // workers (the caller holds the context's mutex)
        std::vector<RankCode> percol(ncols);
        std::vector<uint8_t> coded(ncols, 0);
        auto code_col = [&](uint32_t c) {
            RankCode& rc = percol[c];
            if (!all[c].distinct.empty() && all[c].distinct.size() <= kRankPlanMax) {
                rc.keys = all[c].distinct;
                rc.all_terms = true;
            } else {
                std::vector<uint64_t>& e = rng[c];
                std::sort(e.begin(), e.end());
                e.erase(std::unique(e.begin(), e.end()), e.end());
                if (e.empty() || e.size() > kRankPlanMax) return;
                rc.keys = std::move(e);
                all[c].init(rc.keys.size());
                for (uint64_t k : rc.keys) all[c].insert(k);
            }
            std::sort(rc.keys.begin(), rc.keys.end());
            for (uint32_t i = 0; i < rc.keys.size(); ++i) all[c].set(rc.keys[i], i);
            rc.col = c;
            rc.dtype = static_cast<uint32_t>(tab.cols[c].dtype);
            build_rank_tree(rc);
            build_rank_buckets(rc, ctx->rank_search);
            // marginals (and single-term counts) by rank histogram: one
            // shared-memory counter per set and rank
            rc.hist_fits = rc.tree.size() * 4 + sets.size() * (rc.keys.size() + 1) * 4 <= kRankHistSmem;
            rc.hist = plan.want_marg && rc.hist_fits;
            coded[c] = 1;
        };
        if (ncols >= 2)
            ctx->workers.run(static_cast<uint32_t>(ncols), code_col);
        else
            for (uint32_t c = 0; c < ncols; ++c) code_col(c);
        for (uint32_t c = 0; c < ncols; ++c) {
            if (!coded[c]) continue;
            plan.code_of_col[c] = static_cast<int32_t>(plan.codes.size());
            plan.codes.push_back(std::move(percol[c]));
        }
        // each coded term's intervals as column endpoint indices: an
        // interval [lo, hi] holds the endpoints from lo's index up to that of
        // hi + 1 (or to the last, when hi is the largest key)
        plan.span_off.assign(1, 0);
        for (uint32_t u = 0; u < uterms.size(); ++u) {
            const NTerm& t = uterms[u];
            const int32_t code = plan.code_of_col[t.col];
            const bool range = !is_in_kind(t.kind) && term_cost(t) == 2;
            if (code >= 0 && (range || plan.codes[code].all_terms)) {
                const uint64_t kmax = tab.cols[t.col].dtype == GACE_I64 ? ~0ull : 0xFFFFFFFFull;
                const uint32_t m = static_cast<uint32_t>(plan.codes[code].keys.size());
                const KeyIndex& ki = all[t.col];
                for (uint32_t i = ivo[u]; i < ivo[u + 1]; ++i)
                    plan.span.push_back({ki.find(iv[i].first), iv[i].second < kmax ? ki.find(iv[i].second + 1) : m});
            }
            plan.span_off.push_back(static_cast<uint32_t>(plan.span.size()));
        }
        // a batch's single-term predicates on such columns are counted from
        // the rank histograms (their count is their term's marginal)
        {
            for (uint32_t p = 0; p < npreds; ++p) {
                if (plan.pstate[p] != 0 || plan.pred_u[p].size() != 1) continue;
                const uint32_t u = plan.pred_u[p][0];
                const int32_t code = plan.code_of_col[uterms[u].col];
                if (code < 0 || !plan.codes[code].hist_fits || plan.span_off[u + 1] == plan.span_off[u]) continue;
                plan.pstate[p] = 3;
                plan.codes[code].hist = true;
            }
        }
    }

    phase("host_plan_rank");
    // pack predicates into passes that fit the kernel's shared-memory tables
    std::vector<Pass>& passes = plan.passes;
    std::vector<int32_t> u_pass(uterms.size(), -1);
    {
        Pass cur;
        std::vector<uint8_t> in_cur(uterms.size(), 0);  // unique terms placed in the current pass
        uint32_t pool_words = 0;
        uint64_t pred_terms = 0;  // predicate-term entries of the pass
        // the pass's columns and their tables (a table has at most 64 columns)
        std::vector<ColPool> cols_cur(tab.cols.size());
        std::vector<uint8_t> has_col(tab.cols.size(), 0);
        size_t ncols_cur = 0;
        using Touched = std::vector<std::pair<uint32_t, ColPool>>;
        auto flush = [&]() {
            if (!cur.preds.empty() || !cur.uterms.empty()) passes.push_back(cur);
            for (uint32_t u : cur.uterms) in_cur[u] = 0;
            cur = Pass();
            std::fill(has_col.begin(), has_col.end(), 0);
            ncols_cur = 0;
            pool_words = 0;
            pred_terms = 0;
        };
        // shared memory of a wide pass of nt terms, np predicates, npt
        // predicate-term entries and `pool` pool words (the layout of
        // probe_layout), against what keeps kWideCtas CTAs per SM (1 KB of
        // each CTA's share is reserved by the hardware)
        const uint64_t nsets_dev = sets.size();
        const int ctas = wide_warps >= 16 ? 2 : kWideCtas;
        const uint64_t smem_budget = static_cast<uint64_t>(ctx->smem_per_sm) / ctas - 1024;
        // (no marginal counters when the rank histograms count every term's)
        bool marg_counters = plan.want_marg;
        if (marg_counters) {
            bool all_hist = true;
            for (uint32_t u = 0; u < uterms.size() && all_hist; ++u) all_hist = plan.hist_term(u);
            marg_counters = !all_hist;
        }
        auto wide_smem = [&](uint64_t nt, uint64_t np, uint64_t npt, uint64_t pool) {
            uint64_t off = 128 + nt * 16;
            off = round_up(off + pool * 4, 16) + (np + 1) * 4;
            off = round_up(off + npt * 4, 16);
            off += static_cast<uint64_t>(wide_warps) * (nt + nsets_dev) * 16 + nsets_dev * np * 4;
            off += marg_counters ? nsets_dev * nt * 4 : 0;
            return round_up(off + nsets_dev * 4, 16);
        };
        // the pass's columns and pool words with the terms `add` added
        auto with_terms = [&](const std::vector<uint32_t>& add, Touched& touched) {
            uint64_t total = pool_words;
            for (uint32_t u : add) {
                const uint32_t col = uterms[u].col;
                size_t k = 0;
                while (k < touched.size() && touched[k].first != col) ++k;
                if (k == touched.size()) {
                    ColPool c;
                    if (has_col[col]) {
                        c = cols_cur[col];
                    } else {
                        c.is64 = tab.cols[col].dtype == GACE_I64;
                        const int32_t code = plan.code_of_col[col];
                        c.rstride = code < 0 ? 0u : static_cast<uint32_t>(plan.codes[code].keys.size()) + 1;
                        c.rank_all = code >= 0 && plan.codes[code].all_terms;
                    }
                    touched.emplace_back(col, c);
                }
                touched[k].second.add(uterms[u]);
            }
            for (const auto& kv : touched)
                total += kv.second.words() - (has_col[kv.first] ? cols_cur[kv.first].words() : 0u);
            return total;
        };
        // slots of a wide pass: a column with only its ranges rank-coded may take two (ranges, EQ/IN)
        auto col_slots = [&](uint32_t col) -> size_t {
            const int32_t code = plan.code_of_col[col];
            return code >= 0 && !plan.codes[code].all_terms ? 2 : 1;
        };
        auto new_cols = [&](const Touched& touched) {
            size_t n = 0;
            for (const auto& kv : touched) n += has_col[kv.first] ? 0 : col_slots(kv.first);
            return n;
        };
        auto commit = [&](const std::vector<uint32_t>& add, const Touched& touched, uint64_t total) {
            for (uint32_t u : add) {
                in_cur[u] = 1;
                cur.uterms.push_back(u);
                u_pass[u] = static_cast<int32_t>(passes.size());
            }
            for (const auto& kv : touched) {
                if (!has_col[kv.first]) {
                    has_col[kv.first] = 1;
                    ncols_cur += col_slots(kv.first);
                }
                cols_cur[kv.first] = kv.second;
            }
            pool_words = static_cast<uint32_t>(total);
        };
        std::vector<uint32_t> add;
        Touched touched;
        for (uint32_t p = 0; p < npreds; ++p) {
            if (plan.pstate[p] != 0) continue;
            const std::vector<uint32_t>& pu = plan.pred_u[p];
            if (pu.size() > kPassTerms) return fail(GACE_EINVAL, "predicate %u has too many terms", p);
            add.clear();
            for (uint32_t u : pu)
                if (!in_cur[u]) add.push_back(u);
            touched.clear();
            uint64_t total = with_terms(add, touched);
            // a predicate too large for a shared pass gets one of its own (a
            // single predicate evaluates IN lists by compare, with no tables)
            const size_t ncols = ncols_cur + new_cols(touched);
            if (!cur.preds.empty() &&
                (cur.uterms.size() + add.size() > kPassTerms || cur.preds.size() + 1 > kPassPreds ||
                 total > kPassPool || ncols > static_cast<size_t>(kMaxSlots) ||
                 wide_smem(cur.uterms.size() + add.size(), cur.preds.size() + 1, pred_terms + pu.size(), total) >
                     smem_budget)) {
                flush();
                add.assign(pu.begin(), pu.end());
                touched.clear();
                total = with_terms(add, touched);
            }
            commit(add, touched, total);
            cur.preds.push_back(p);
            pred_terms += pu.size();
        }
        // terms whose marginals are wanted but that no device predicate placed
        // (and that no rank histogram counts)
        if (plan.want_marg) {
            for (uint32_t u = 0; u < uterms.size(); ++u) {
                if (u_pass[u] >= 0 || plan.hist_term(u)) continue;
                add.assign(1, u);
                touched.clear();
                uint64_t total = with_terms(add, touched);
                const size_t ncols = ncols_cur + (has_col[uterms[u].col] ? 0 : col_slots(uterms[u].col));
                if (!cur.uterms.empty() &&
                    (cur.uterms.size() + 1 > kPassTerms || total > kPassPool ||
                     ncols > static_cast<size_t>(kMaxSlots) ||
                     wide_smem(cur.uterms.size() + 1, cur.preds.size(), pred_terms, total) > smem_budget)) {
                    flush();
                    touched.clear();
                    total = with_terms(add, touched);
                }
                commit(add, touched, total);
            }
        }
        flush();
    }
    phase("host_plan_pack");
    bool need_ns = false;
    for (auto& s : sets)
        if (s.d.mode == 2) need_ns = true;
    if (sets.empty()) passes.clear();  // every sample is empty: nothing to count
    if (passes.empty() && need_ns) passes.push_back(Pass());  // counts sample rows only
    // the passes of a split batch are all wide: a small last pass in the
    // narrow layout would evaluate its IN lists by compare
    const bool all_wide = force_wide || passes.size() > 1;
    for (auto& ps : passes) {
        if (gace_status st = build_pass(ctx, tab, ps, uterms, plan.pred_u, sets, plan.want_marg, all_wide,
                                        wide_warps, plan))
            return st;
        pass_sizes(ps);
    }
    phase("host_plan_build");
    return GACE_OK;
}

void pass_sizes(Pass& ps) {
    const ProbeArgs& A = ps.args;
    ps.in_bytes = round_up(A.nterms * 16ull, 16) + round_up(A.npool * 4ull, 16) + round_up((A.npreds + 1) * 4ull, 16) +
                  round_up(A.npredterms * 4ull, 16);
    ps.out_bytes =
        (static_cast<uint64_t>(A.nsets) * A.npreds + static_cast<uint64_t>(A.nsets) * A.nterms + A.nsets) * 8ull;
}

void stage_pass(Pass& ps, unsigned char* pin, unsigned char* dws, unsigned int* status) {
    ProbeArgs& A = ps.args;
    uint64_t o = ps.in_off;
    auto put = [&](const void* src, uint64_t bytes) {
        const uint64_t at = o;
        if (bytes) memcpy(pin + o, src, bytes);
        o += round_up(bytes, 16);
        return at;
    };
    const uint64_t o_terms = put(ps.dterms.data(), ps.dterms.size() * 16ull);
    const uint64_t o_pool = put(ps.pool.data(), ps.pool.size() * 4ull);
    const uint64_t o_poff = put(ps.poff.data(), ps.poff.size() * 4ull);
    const uint64_t o_pterm = put(ps.pterm.data(), ps.pterm.size() * 4ull);
    A.terms = reinterpret_cast<const DevTerm*>(dws + o_terms);
    A.pool = reinterpret_cast<const uint32_t*>(dws + o_pool);
    A.pred_off = reinterpret_cast<const uint32_t*>(dws + o_poff);
    A.pred_terms = reinterpret_cast<const uint32_t*>(dws + o_pterm);
    unsigned long long* out = reinterpret_cast<unsigned long long*>(dws + ps.out_off);
    A.counts = out;
    A.marg = out + static_cast<uint64_t>(A.nsets) * A.npreds;
    A.nsamp = A.marg + static_cast<uint64_t>(A.nsets) * A.nterms;
    A.status = status;
}

void assemble_probe(const ProbePlan& plan, const ProbeRequest& r,
                    const std::vector<const unsigned long long*>& pass_out) {
    const uint32_t nsamples = r.nsamples, npreds = r.npreds;
    const std::vector<Pass>& passes = plan.passes;
    std::vector<uint64_t> ns(nsamples, 0);
    for (uint32_t s = 0; s < nsamples; ++s) {
        if (plan.set_dev[s] < 0) continue;
        const SetDesc& d = plan.sets[plan.set_dev[s]].d;
        if (d.mode == 1) {
            ns[s] = plan.tab->nrows;
        } else {
            const Pass& ps = passes.front();
            ns[s] = pass_out[0][static_cast<uint64_t>(ps.args.nsets) * ps.args.npreds +
                                static_cast<uint64_t>(ps.args.nsets) * ps.args.nterms + plan.set_dev[s]];
        }
    }
    // per unique term: (pass, local index)
    std::vector<std::pair<int32_t, uint32_t>> uloc(plan.uterms.size(), {-1, 0});
    for (uint32_t k = 0; k < passes.size(); ++k)
        for (uint32_t i = 0; i < passes[k].uterms.size(); ++i)
            uloc[passes[k].uterms[i]] = {static_cast<int32_t>(k), i};
    // rank-histogram marginals: per coded column and set, pre[r] = the set's
    // rows of rank < r; a row of rank r holds a term whose interval spans
    // column endpoints [r0, r1) when r0 < r <= r1
    std::vector<std::vector<uint64_t>> pre(plan.codes.size());
    auto hist_marg = [&](uint32_t u, uint32_t ds) -> uint64_t {
        const int32_t code = plan.code_of_col[plan.uterms[u].col];
        const RankCode& rc = plan.codes[code];
        const uint64_t bins = rc.keys.size() + 1;
        std::vector<uint64_t>& p = pre[code];
        if (p.empty()) {
            p.assign(plan.sets.size() * (bins + 1), 0);
            for (size_t q = 0; q < plan.sets.size(); ++q)
                for (uint64_t r = 0; r < bins; ++r)
                    p[q * (bins + 1) + r + 1] = p[q * (bins + 1) + r] + rc.hist_host[q * bins + r];
        }
        const uint64_t* pq = p.data() + ds * (bins + 1);
        uint64_t n = 0;
        for (uint32_t i = plan.span_off[u]; i < plan.span_off[u + 1]; ++i)
            n += pq[plan.span[i].second + 1] - pq[plan.span[i].first + 1];
        return n;
    };
    auto marg_of = [&](uint32_t t, uint32_t s) -> uint64_t {
        const uint32_t u = plan.t2u[t];
        if (u == UINT32_MAX || plan.set_dev[s] < 0) return 0;
        if (plan.hist_term(u)) return hist_marg(u, static_cast<uint32_t>(plan.set_dev[s]));
        const auto& L = uloc[u];
        if (L.first < 0) return 0;
        const Pass& ps = passes[L.first];
        return pass_out[L.first][static_cast<uint64_t>(ps.args.nsets) * ps.args.npreds +
                                 static_cast<uint64_t>(plan.set_dev[s]) * ps.args.nterms + L.second];
    };
    std::vector<std::pair<int32_t, uint32_t>> ploc(npreds, {-1, 0});
    for (uint32_t k = 0; k < passes.size(); ++k)
        for (uint32_t i = 0; i < passes[k].preds.size(); ++i)
            ploc[passes[k].preds[i]] = {static_cast<int32_t>(k), i};
    assemble_probe_counts(
        plan, r, [&](uint32_t s) { return ns[s]; },
        [&](uint32_t p, uint32_t s) -> uint64_t {
            if (plan.pstate[p] == 3) return hist_marg(plan.pred_u[p][0], static_cast<uint32_t>(plan.set_dev[s]));
            const Pass& ps = passes[ploc[p].first];
            return pass_out[ploc[p].first][static_cast<uint64_t>(plan.set_dev[s]) * ps.args.npreds + ploc[p].second];
        },
        marg_of);
}

namespace {

// The launch of one pass over rows [row0, row0 + rows) of its table (all of
// it when rows == 0): the pass's arguments narrowed to those rows (row ids
// stay table-global for the samples' hashes), the grid sized for them.
// ranks: per column, the ranks of the rows launched (rank-coded slots).
gace_status launch_pass(gace_ctx* ctx, const Pass& ps, uint64_t row0, uint64_t rows, const uint4* setmask,
                        const std::vector<const uint16_t*>& ranks) {
    ProbeArgs a = ps.args;
    if (rows) {
        a.nrows = rows;
        a.row0 = row0;
        for (uint32_t s = 0; s < a.nslots; ++s)
            a.slots[s].ptr = static_cast<const unsigned char*>(a.slots[s].ptr) + row0 * a.slots[s].width;
        a.ntiles = (rows + a.tile_rows - 1) / a.tile_rows;
        a.nstaged = a.stage_bytes ? rows / a.tile_rows : 0;
    }
    if (!a.narrow && setmask) a.setmask = setmask;
    for (uint32_t s = 0; s < a.nslots; ++s) {
        if (!a.slots[s].rstride) continue;
        const uint32_t col = ps.slots[s].first;
        if (col >= ranks.size() || !ranks[col]) return fail(GACE_EINVAL, "rank-coded column %u has no ranks", col);
        a.slots[s].rank = ranks[col];
    }
    const int occ = probe_occupancy(a);
    if (occ < 1)
        return fail(GACE_ECUDA, "probe kernel cannot be resident with %u bytes of shared memory", a.smem_bytes);
    // work units: tiles (narrow) or warp sweeps of 128-row slices (wide)
    const uint64_t n = a.nrows;
    const uint64_t unit_rows = a.narrow ? a.tile_rows : static_cast<uint64_t>(kSliceRows) * a.nwarps;
    const uint64_t units = (n + unit_rows - 1) / unit_rows;
    uint64_t grid = static_cast<uint64_t>(ctx->sms) * occ;
    if (ctx->max_ctas && grid > ctx->max_ctas) grid = ctx->max_ctas;
    if (grid > units) grid = units;
    if (grid < 1) grid = 1;
    // each CTA keeps 32-bit row counters
    while ((units + grid - 1) / grid * unit_rows >= (1ull << 31)) grid *= 2;
    if (grid > 0x7FFFFFFFull) return fail(GACE_EINVAL, "table too large for one probe grid");
    CK(ctx->traced(a.narrow ? "probe_narrow" : "probe_wide", n, n * ps.rowbytes, n * ps.ops_per_row,
                   [&] { return probe_launch(a, static_cast<int>(grid), ctx->stream); }));
    return GACE_OK;
}

}  // namespace

gace_status run_planned(gace_ctx* ctx, std::vector<PlannedProbe>& parts, TableRec* lazy) {
    // workspace: status | inputs and outputs of every part's passes, the
    // rank-coded columns' search trees (copied in, read back) | device-only
    // scratch: row-set masks and ranks of one chunk of rows per part
    Ws ws;
    const uint64_t status_off = ws.take(256);
    bool any_pass = false;
    for (auto& pp : parts)
        for (auto& ps : pp.plan.passes) {
            ps.in_off = ws.take(ps.in_bytes);
            ps.out_off = ws.take(ps.out_bytes);
            any_pass = true;
        }
    // rank histograms of the row sets (marginals), zeroed and read back
    std::vector<std::vector<uint64_t>> tree_off(parts.size()), hist_off(parts.size());
    for (size_t i = 0; i < parts.size(); ++i)
        for (const RankCode& rc : parts[i].plan.codes) {
            tree_off[i].push_back(rc.used || rc.hist ? ws.take(rc.tree.size() * 4ull) : 0);
            const uint64_t bins = parts[i].plan.sets.size() * (rc.keys.size() + 1);
            hist_off[i].push_back(rc.hist ? ws.take(bins * 8) : 0);
        }
    const uint64_t io_end = ws.off;
    // Rows per chunk: a table whose copy is pending (one part) streams in
    // chunks of rows, a multiple of every pass's tile, each chunk running
    // every pass; so does a table whose ranks would not fit kRankScratch.
    std::vector<uint64_t> chunk(parts.size(), 0), mask_off(parts.size(), 0), qmask_off(parts.size(), 0);
    std::vector<std::vector<uint64_t>> rank_off(parts.size());
    for (size_t i = 0; i < parts.size(); ++i) {
        const ProbePlan& pl = parts[i].plan;
        const uint64_t n = parts[i].tab->nrows;
        uint64_t coded = 0;
        for (const RankCode& rc : pl.codes) coded += rc.used ? 1 : 0;
        uint64_t rows = n;
        if (lazy)
            rows = round_up(std::max<uint64_t>(n / kLoadChunks, 1ull << 20), 1ull << 16);
        else if (coded && coded * round_up(n, kSliceRows) * 2 > kRankScratch)
            rows = std::max<uint64_t>(kRankScratch / (coded * 2) / (1ull << 16) * (1ull << 16), 1ull << 16);
        chunk[i] = std::min(rows, n);
        const uint64_t crows = round_up(chunk[i], kSliceRows);
        // A part with several wide passes over hashed row sets computes every
        // slice's row-set masks once (per chunk), for all its passes to load.
        // (and so does a rank pass that counts hashed sets)
        uint32_t wide = 0;
        for (const auto& ps : pl.passes) wide += ps.args.narrow ? 0u : 1u;
        bool hashed = false, hist = false;
        for (const auto& sp : pl.sets) hashed = hashed || sp.d.mode == 2;
        for (const RankCode& rc : pl.codes) hist = hist || rc.hist;
        if ((wide >= 2 || hist) && hashed) mask_off[i] = ws.take((crows / kSliceRows) * pl.sets.size() * 16);
        if (hist && hashed) qmask_off[i] = ws.take(crows);  // one word per quad
        for (const RankCode& rc : pl.codes) rank_off[i].push_back(rc.used ? ws.take(crows * 2) : 0);
    }
    if (gace_status st = ctx->ensure_ws(ws.off)) return st;
    if (gace_status st = ctx->ensure_pin(io_end + 256)) return st;

    // stage inputs into pinned memory, one H2D copy, zero outputs
    unsigned char* pin = ctx->pin;
    unsigned char* dws = ctx->ws;
    unsigned int* dstatus = reinterpret_cast<unsigned int*>(dws + status_off);
    for (auto& pp : parts)
        for (auto& ps : pp.plan.passes) stage_pass(ps, pin, dws, dstatus);
    for (size_t i = 0; i < parts.size(); ++i)
        for (size_t c = 0; c < parts[i].plan.codes.size(); ++c) {
            const RankCode& rc = parts[i].plan.codes[c];
            if (rc.used || rc.hist) memcpy(pin + tree_off[i][c], rc.tree.data(), rc.tree.size() * 4ull);
        }
    const uint64_t first_in = status_off + 256;
    if (io_end > first_in) {
        CK(cudaMemcpyAsync(dws + first_in, pin + first_in, io_end - first_in, cudaMemcpyHostToDevice, ctx->stream));
        for (auto& pp : parts)
            for (auto& ps : pp.plan.passes) CK(cudaMemsetAsync(dws + ps.out_off, 0, ps.out_bytes, ctx->stream));
        for (size_t i = 0; i < parts.size(); ++i)
            for (size_t c = 0; c < parts[i].plan.codes.size(); ++c)
                if (hist_off[i][c])
                    CK(cudaMemsetAsync(dws + hist_off[i][c], 0,
                                       parts[i].plan.sets.size() * (parts[i].plan.codes[c].keys.size() + 1) * 8,
                                       ctx->stream));
    }
    CK(cudaMemsetAsync(dws + status_off, 0, 256, ctx->stream));
    ctx->host_phase("host_probe_stage");
    uint64_t nload = 0;  // chunks of the pending copy
    if (lazy) {
        // every chunk's copy on the copy stream, all at once (they run back to
        // back); the context stream waits for each before that chunk's passes
        if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        const uint64_t n = lazy->nrows, step = chunk[0];
        nload = step ? (n + step - 1) / step : 0;
        while (ctx->chunk_events.size() < std::max<uint64_t>(nload, 1)) {
            cudaEvent_t ev = nullptr;
            CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            ctx->chunk_events.push_back(ev);
        }
        // the copy stream starts after what the context stream has queued (the
        // columns' stream-ordered allocations)
        CK(cudaEventRecord(ctx->chunk_events[0], ctx->stream));
        CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->chunk_events[0], 0));
        for (uint64_t k = 0; k < nload; ++k) {
            const uint64_t r0 = k * step, rows = std::min(step, n - r0);
            for (size_t c = 0; c < lazy->cols.size(); ++c) {
                const uint64_t w = dtype_width(lazy->cols[c].dtype);
                CK(cudaMemcpyAsync(static_cast<unsigned char*>(lazy->cols[c].dptr) + r0 * w,
                                   static_cast<const unsigned char*>(lazy->pending[c]) + r0 * w, rows * w,
                                   cudaMemcpyHostToDevice, ctx->copy_stream));
            }
            CK(cudaEventRecord(ctx->chunk_events[k], ctx->copy_stream));
        }
    }
    for (size_t i = 0; i < parts.size(); ++i) {
        auto& pp = parts[i];
        const TableRec* tab = pp.tab;
        const uint64_t n = tab->nrows, step = chunk[i];
        const bool whole = step >= n;  // one chunk: the passes' own row counts
        const uint64_t nchunks = whole ? 1 : (n + step - 1) / step;
        std::vector<const uint16_t*> ranks(tab->cols.size(), nullptr);
        for (uint64_t k = 0; k < nchunks; ++k) {
            const uint64_t r0 = whole ? 0 : k * step, rows = whole ? n : std::min(step, n - r0);
            if (lazy && k < nload) CK(cudaStreamWaitEvent(ctx->stream, ctx->chunk_events[k], 0));
            uint4* masks = nullptr;
            uint32_t* qmask = qmask_off[i] ? reinterpret_cast<uint32_t*>(dws + qmask_off[i]) : nullptr;
            if (mask_off[i]) {
                masks = reinterpret_cast<uint4*>(dws + mask_off[i]);
                ProbeArgs a0 = pp.plan.passes.front().args;
                a0.nrows = rows;
                a0.row0 = r0;
                CK(ctx->traced("probe_setmask", rows, 0, rows,
                               [&] { return setmask_launch(a0, masks, qmask, ctx->sms, ctx->stream); }));
            }
            for (size_t c = 0; c < pp.plan.codes.size(); ++c) {
                const RankCode& rc = pp.plan.codes[c];
                if (!rc.used && !rc.hist) continue;  // ranks for the passes, or histograms only
                RankArgs ra{};
                const uint32_t w = dtype_width(static_cast<int>(rc.dtype));
                ra.col = static_cast<const unsigned char*>(tab->cols[rc.col].dptr) + r0 * w;
                ra.nrows = rows;
                ra.nout = round_up(rows, kSliceRows);
                ra.tree = reinterpret_cast<const uint32_t*>(dws + tree_off[i][c]);
                ra.out = rc.used ? reinterpret_cast<uint16_t*>(dws + rank_off[i][c]) : nullptr;
                ra.dtype = rc.dtype;
                ra.levels = rc.levels;
                ra.words = static_cast<uint32_t>(rc.tree.size());
                ra.base = rc.bbase;
                ra.nb = rc.bnb;
                ra.smin = rc.bsmin;
                ra.mbits = rc.bmbits;
                ra.steps = rc.bsteps;
                ra.m = static_cast<uint32_t>(rc.keys.size());
                if (hist_off[i][c]) {
                    ra.hist = reinterpret_cast<unsigned long long*>(dws + hist_off[i][c]);
                    ra.qmask = qmask;
                    ra.nsets = static_cast<uint32_t>(pp.plan.sets.size());
                    for (uint32_t q = 0; q < ra.nsets; ++q) {
                        const SetDesc& d = pp.plan.sets[q].d;
                        if (d.kind == 0 || d.mode == 1) ra.full_sets |= 1u << q;
                    }
                    if (!qmask && ra.full_sets != (1u << ra.nsets) - 1u)
                        return fail(GACE_EINVAL, "rank histograms of hashed sets without their masks");
                }
                ranks[rc.col] = ra.out;
                CK(ctx->traced("probe_rank", rows, rows * (w + (rc.used ? 2 : 0)), rows,
                               [&] { return rank_launch(ra, ctx->sms, ctx->stream); }));
            }
            for (auto& ps : pp.plan.passes)
                if (gace_status st = launch_pass(ctx, ps, r0, whole ? 0 : rows, masks, ranks)) return st;
        }
    }
    const uint64_t rb_hi = any_pass ? io_end : status_off + 256;
    CK(cudaMemcpyAsync(pin + status_off, dws + status_off, rb_hi - status_off, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->host_phase("host_probe_launch");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->host_phase("host_probe_wait");
    ctx->collect();
    if (lazy) lazy->pending.clear();  // the stream waited for every chunk's copy
    if (gace_status st = read_status(ctx, *reinterpret_cast<unsigned int*>(pin + status_off))) return st;
    for (size_t i = 0; i < parts.size(); ++i)
        for (size_t c = 0; c < parts[i].plan.codes.size(); ++c)
            parts[i].plan.codes[c].hist_host =
                hist_off[i][c] ? reinterpret_cast<const unsigned long long*>(pin + hist_off[i][c]) : nullptr;
    for (auto& pp : parts) {
        std::vector<const unsigned long long*> outs;
        for (auto& ps : pp.plan.passes) outs.push_back(reinterpret_cast<const unsigned long long*>(pin + ps.out_off));
        assemble_probe(pp.plan, pp.r, outs);
    }
    ctx->host_phase("host_probe_finish");
    return GACE_OK;
}

}  // namespace host
}  // namespace gace

// ======================================================================== ABI

extern "C" {

uint32_t gace_abi_version(void) { return GACE_ABI_VERSION; }

const char* gace_last_error(void) { return g_last_error.c_str(); }

const char* gace_status_string(gace_status s) {
    switch (s) {
        case GACE_OK: return "GACE_OK";
        case GACE_EINVAL: return "GACE_EINVAL";
        case GACE_ENOMEM: return "GACE_ENOMEM";
        case GACE_EBUSY: return "GACE_EBUSY";
        case GACE_EPENDING: return "GACE_EPENDING";
        case GACE_ETIMEDOUT: return "GACE_ETIMEDOUT";
        case GACE_ENOTFOUND: return "GACE_ENOTFOUND";
        case GACE_EOVERFLOW: return "GACE_EOVERFLOW";
        case GACE_ECUDA: return "GACE_ECUDA";
    }
    return "GACE_UNKNOWN";
}

gace_status gace_create(gace_ctx** out, const gace_config* cfg) {
    if (!out) return fail(GACE_EINVAL, "out is NULL");
    gace_config c{};
    if (cfg) c = *cfg;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0)
        return fail(GACE_ECUDA, "no CUDA device: %s", e != cudaSuccess ? cudaGetErrorString(e) : "count is 0");
    if (c.device < 0 || c.device >= n) return fail(GACE_EINVAL, "device %d outside 0..%d", c.device, n - 1);
    if (c.rank_search > 2) return fail(GACE_EINVAL, "rank_search = %u (0, 1 or 2)", c.rank_search);
    DeviceGuard g(c.device);
    gace_ctx* ctx = new gace_ctx();
    ctx->device = c.device;
    ctx->budget = c.hbm_budget_bytes;
    ctx->max_ctas = c.max_ctas;
    ctx->rank_min_rows = c.rank_min_rows;
    ctx->rank_search = c.rank_search;
    if (c.wait_timeout_ms) ctx->timeout_ns = static_cast<uint64_t>(c.wait_timeout_ms) * 1000000ull;
    auto bail = [&](gace_status s) {
        gace_destroy(ctx);
        return s;
    };
    if ((e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, c.device)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaDeviceGetAttribute(SM count)"));
    if ((e = cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device)) !=
        cudaSuccess)
        return bail(cuda_fail(e, "cudaDeviceGetAttribute(smem opt-in)"));
    if ((e = cudaDeviceGetAttribute(&ctx->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c.device)) !=
        cudaSuccess)
        return bail(cuda_fail(e, "cudaDeviceGetAttribute(smem per SM)"));
    if (c.stream) {
        ctx->stream = static_cast<cudaStream_t>(c.stream);
    } else {
        if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaStreamCreateWithFlags"));
        ctx->own_stream = true;
    }
    if ((e = probe_configure()) != cudaSuccess) return bail(cuda_fail(e, "probe kernel attributes"));
    {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = c.device;
        if ((e = cudaMemPoolCreate(&ctx->pool, &props)) != cudaSuccess) {
            ctx->pool = nullptr;
            return bail(cuda_fail(e, "cudaMemPoolCreate"));
        }
        // freed blocks stay in the pool up to the HBM budget (all of them without one)
        uint64_t keep = ctx->budget ? ctx->budget : ~0ull;
        if ((e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMemPoolSetAttribute"));
    }
    if ((e = cudaMalloc(&ctx->d_status, 256)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(status)"));
    *out = ctx;
    return GACE_OK;
}

gace_status gace_destroy(gace_ctx* ctx) {
    if (!ctx) return GACE_OK;
    serve_shutdown(ctx);
    {
        DeviceGuard g(ctx->device);
        if (ctx->stream) {
            resident_clear(ctx);
            for (auto& kv : ctx->tables) free_table_columns(ctx, kv.second);
            cudaStreamSynchronize(ctx->stream);
        }
        if (ctx->ws) cudaFree(ctx->ws);
        if (ctx->pin) cudaFreeHost(ctx->pin);
        if (ctx->d_status) cudaFree(ctx->d_status);
        ctx->collect();
        for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
        if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
        if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
        for (cudaStream_t a : ctx->batch_aux)
            if (a) cudaStreamDestroy(a);
        for (int ph = 0; ph < kPhases; ++ph) {
            if (ctx->batch_fork[ph]) cudaEventDestroy(ctx->batch_fork[ph]);
            for (cudaEvent_t j : ctx->batch_join[ph])
                if (j) cudaEventDestroy(j);
        }
        if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        for (cudaEvent_t e : ctx->chunk_events) cudaEventDestroy(e);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    }
    delete ctx;
    return GACE_OK;
}

gace_status gace_load_columns(gace_ctx* ctx, uint64_t nrows, uint32_t ncols, const gace_column* cols,
                              uint32_t flags, uint32_t* table_id_out) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (!cols || !table_id_out) return fail(GACE_EINVAL, "cols or table_id_out is NULL");
    if (ncols == 0 || ncols > 64) return fail(GACE_EINVAL, "ncols %u outside 1..64", ncols);
    if (flags > GACE_COPY_ON_FIRST_PROBE) return fail(GACE_EINVAL, "flags %u is not a gace_load_flags value", flags);
    if (nrows > (1ull << 40)) return fail(GACE_EINVAL, "nrows %llu above 2^40", (unsigned long long)nrows);
    for (uint32_t c = 0; c < ncols; ++c) {
        if (cols[c].dtype < GACE_I32 || cols[c].dtype > GACE_F32)
            return fail(GACE_EINVAL, "column %u has dtype %d", c, cols[c].dtype);
        if (nrows > 0 && !cols[c].data) return fail(GACE_EINVAL, "column %u data is NULL", c);
        if (flags == GACE_BORROW && !cols[c].on_device)
            return fail(GACE_EINVAL, "GACE_BORROW needs device columns (column %u is on the host)", c);
        if (flags == GACE_COPY_ON_FIRST_PROBE && cols[c].on_device)
            return fail(GACE_EINVAL, "GACE_COPY_ON_FIRST_PROBE needs host columns (column %u is on the device)", c);
    }
    const bool lazy = flags == GACE_COPY_ON_FIRST_PROBE;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (flags == GACE_COPY && nrows > 0) {
        // device sources are read on the context stream: whatever produced
        // them on other streams must have finished first
        bool from_device = false;
        for (uint32_t c = 0; c < ncols; ++c) from_device = from_device || cols[c].on_device;
        if (from_device) CK(cudaDeviceSynchronize());
    }
    TableRec tab;
    tab.nrows = nrows;
    uint64_t need = 0;
    if (flags != GACE_BORROW)
        for (uint32_t c = 0; c < ncols; ++c) need += round_up(nrows * dtype_width(cols[c].dtype) + 16, 256);
    if (!ctx->fits(need))
        return fail(GACE_ENOMEM, "table of %llu bytes exceeds the HBM budget (%llu of %llu used)",
                    (unsigned long long)need, (unsigned long long)ctx->used,
                    (unsigned long long)ctx->budget);
    for (uint32_t c = 0; c < ncols; ++c) {
        ColumnRec r;
        r.dtype = cols[c].dtype;
        const uint64_t bytes = nrows * dtype_width(r.dtype);
        r.bytes = bytes;
        if (flags == GACE_BORROW) {
            r.dptr = const_cast<void*>(cols[c].data);
        } else {
            const uint64_t alloc = round_up(bytes + 16, 256);
            // stream-ordered: no device-wide synchronisation
            cudaError_t e = ctx->alloc_async(&r.dptr, alloc);
            if (e != cudaSuccess) {
                for (auto& x : tab.cols) cudaFreeAsync(x.dptr, ctx->stream);
                return fail(GACE_ENOMEM, "cudaMallocAsync(%llu) for column %u: %s", (unsigned long long)alloc, c,
                            cudaGetErrorString(e));
            }
            r.owned = true;
            tab.owned_bytes += alloc;
            if (lazy) {
                tab.pending.push_back(cols[c].data);  // copied by the first call that reads the table
            } else if (bytes) {
                e = cudaMemcpyAsync(r.dptr, cols[c].data, bytes,
                                    cols[c].on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    ctx->stream);
                if (e != cudaSuccess) {
                    cudaFreeAsync(r.dptr, ctx->stream);
                    for (auto& x : tab.cols) cudaFreeAsync(x.dptr, ctx->stream);
                    return cuda_fail(e, "cudaMemcpyAsync(column)");
                }
            }
        }
        tab.cols.push_back(r);
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        for (auto& x : tab.cols)
            if (x.owned) cudaFreeAsync(x.dptr, ctx->stream);
        return cuda_fail(e, "cudaStreamSynchronize(load)");
    }
    ctx->used += tab.owned_bytes;
    const uint32_t id = ctx->next_id++;
    ctx->tables.emplace(id, std::move(tab));
    *table_id_out = id;
    return GACE_OK;
}

gace_status gace_unload(gace_ctx* ctx, uint32_t table_id) {
    if (gace_status s = check_ctx(ctx)) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    auto it = ctx->tables.find(table_id);
    if (it == ctx->tables.end()) return fail(GACE_ENOTFOUND, "table %u is not loaded", table_id);
    if (gace_status s = serve_forget_table(ctx, table_id)) return s;
    if (resident_samples_busy(ctx, table_id))
        return fail(GACE_EBUSY, "served requests read a resident sample of table %u", table_id);
    if (it->second.in_store) {  // a resident sample unloaded by hand leaves the store
        ResidentStore& R = ctx->resident;
        for (auto e = R.samples.begin(); e != R.samples.end(); ++e)
            if (e->second.sample_table == table_id) {
                R.used -= e->second.bytes;
                R.samples.erase(e);
                break;
            }
    }
    resident_forget_table(ctx, table_id);
    // stream-ordered frees: after the work already queued on the context stream
    it = ctx->tables.find(table_id);
    free_table_columns(ctx, it->second);
    ctx->tables.erase(it);
    return GACE_OK;
}

gace_status gace_probe_batch(gace_ctx* ctx, uint32_t table_id, const gace_sample* samples, uint32_t nsamples,
                             const gace_term* terms, uint32_t nterms, const gace_scalar* in_values, uint32_t nin,
                             const gace_pred* preds, uint32_t npreds, gace_pred_result* results,
                             uint64_t* term_marginals) {
    if (gace_status s = check_ctx(ctx)) return s;
    ProbeRequest r;
    r.samples = samples;
    r.nsamples = nsamples;
    r.terms = terms;
    r.nterms = nterms;
    r.in_values = in_values;
    r.nin = nin;
    r.preds = preds;
    r.npreds = npreds;
    r.results = results;
    r.term_marginals = term_marginals;
    if (gace_status s = check_probe_request(r)) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->phase_t = std::chrono::steady_clock::now();
    TableRec* tab = find_table_raw(ctx, table_id);  // a pending copy may overlap the probe
    if (!tab) return fail(GACE_ENOTFOUND, "table %u is not loaded", table_id);
    DeviceGuard g(ctx->device);
    for (uint32_t s = 0; s < nsamples; ++s) {
        SetDesc d;
        if (gace_status st = make_set(samples[s], d)) return st;
    }
    // Row sets held by the resident store are counted by full scans of their
    // resident samples; the others on the base table.
    std::vector<uint32_t> where(nsamples, 0), pinned;
    bool any = false;
    if (ctx->resident.samples_on()) {
        for (uint32_t s = 0; s < nsamples; ++s) {
            SetDesc d;
            make_set(samples[s], d);
            where[s] = resident_sample(ctx, table_id, d, true, pinned);
            any = any || where[s] != 0;
        }
    }
    std::vector<PlannedProbe> parts;
    if (!any) {
        parts.emplace_back();
        parts.back().tab = tab;
        parts.back().r = r;
        if (gace_status st = plan_probe(ctx, *tab, r, false, parts.back().plan, kWideWarps, true, true)) return st;
        ctx->host_phase("host_probe_plan");
        return run_planned(ctx, parts, tab->pending.empty() ? nullptr : tab);
    }
    if (gace_status st = complete_load(ctx, *tab)) return st;
    // one part per table: the base table with the samples that are not
    // resident, and each resident sample table with one full scan; each part
    // writes its own results, scattered to the caller's rows afterwards
    static const gace_sample kFull{GACE_FULL, 0, 1.0, 0};
    std::vector<uint32_t> order;  // the tables of the parts, base first
    std::vector<std::vector<uint32_t>> members;
    auto part_of = [&](uint32_t t) {
        for (size_t i = 0; i < order.size(); ++i)
            if (order[i] == t) return i;
        order.push_back(t);
        members.emplace_back();
        return order.size() - 1;
    };
    for (uint32_t s = 0; s < nsamples; ++s) members[part_of(where[s] ? where[s] : table_id)].push_back(s);
    parts.resize(order.size());
    std::vector<std::vector<gace_sample>> psamples(order.size());
    std::vector<std::vector<gace_pred_result>> pres(order.size());
    std::vector<std::vector<uint64_t>> pmarg(order.size());
    for (size_t i = 0; i < order.size(); ++i) {
        PlannedProbe& pp = parts[i];
        const bool resident = order[i] != table_id;
        pp.tab = find_table(ctx, order[i]);
        if (resident)
            psamples[i].push_back(kFull);  // identical samples of one part share its counts
        else
            for (uint32_t s : members[i]) psamples[i].push_back(samples[s]);
        const uint32_t ns = static_cast<uint32_t>(psamples[i].size());
        pres[i].resize(static_cast<size_t>(ns) * npreds);
        if (term_marginals) pmarg[i].resize(static_cast<size_t>(ns) * nterms);
        pp.r = r;
        pp.r.samples = psamples[i].data();
        pp.r.nsamples = ns;
        pp.r.results = npreds ? pres[i].data() : nullptr;
        pp.r.term_marginals = term_marginals ? pmarg[i].data() : nullptr;
        if (gace_status st = plan_probe(ctx, *pp.tab, pp.r, false, pp.plan, kWideWarps, true, true)) return st;
    }
    ctx->host_phase("host_probe_plan");
    if (gace_status st = run_planned(ctx, parts)) return st;
    for (size_t i = 0; i < order.size(); ++i) {
        const bool resident = order[i] != table_id;
        for (size_t k = 0; k < members[i].size(); ++k) {
            const uint32_t s = members[i][k];
            const size_t from = resident ? 0 : k;
            if (npreds)
                memcpy(results + static_cast<size_t>(s) * npreds, pres[i].data() + from * npreds,
                       npreds * sizeof(gace_pred_result));
            if (term_marginals && nterms)
                memcpy(term_marginals + static_cast<size_t>(s) * nterms, pmarg[i].data() + from * nterms,
                       nterms * sizeof(uint64_t));
        }
    }
    return GACE_OK;
}

// ---------------------------------------------------------------- HLL


gace_status gace_ndv(gace_ctx* ctx, uint32_t table_id, uint32_t col, uint32_t p, uint64_t hash_seed,
                     uint8_t* registers_out, double* estimate_out) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (p < 4 || p > 18) return fail(GACE_EINVAL, "p = %u outside 4..18", p);
    std::lock_guard<std::mutex> lk(ctx->mu);
    TableRec* tab = find_table(ctx, table_id);
    if (!tab) return fail(GACE_ENOTFOUND, "table %u is not loaded", table_id);
    if (col >= tab->cols.size()) return fail(GACE_EINVAL, "column %u of a %zu-column table", col, tab->cols.size());
    DeviceGuard g(ctx->device);
    const uint64_t m = 1ull << p;
    {  // a resident sketch of this column, p and seed answers without a scan
        std::vector<uint8_t> regs(m);
        if (resident_sketch_get(ctx, table_id, col, p, hash_seed, regs.data())) {
            if (registers_out) memcpy(registers_out, regs.data(), m);
            if (estimate_out) *estimate_out = hll_estimate_host(regs.data(), p);
            return GACE_OK;
        }
    }
    Ws ws;
    const uint64_t status_off = ws.take(256);
    const uint64_t regs_off = ws.take(m * 4);
    if (gace_status st = ctx->ensure_ws(ws.off)) return st;
    if (gace_status st = ctx->ensure_pin(ws.off)) return st;
    CK(cudaMemsetAsync(ctx->ws, 0, ws.off, ctx->stream));
    HllArgs a{};
    a.col = tab->cols[col].dptr;
    a.nrows = tab->nrows;
    a.dtype = static_cast<uint32_t>(tab->cols[col].dtype);
    a.p = p;
    a.seedhash = splitmix64_host(hash_seed);
    a.aligned = (reinterpret_cast<uintptr_t>(a.col) & 15u) == 0;
    a.regs = reinterpret_cast<uint32_t*>(ctx->ws + regs_off);
    a.status = reinterpret_cast<unsigned int*>(ctx->ws + status_off);
    if (tab->nrows > 0) {
        const uint64_t n = tab->nrows;
        CK(ctx->traced("hll", n, n * dtype_width(tab->cols[col].dtype), n,
                       [&] { return hll_launch(a, ctx->sms, ctx->stream); }));
    }
    CK(cudaMemcpyAsync(ctx->pin, ctx->ws, ws.off, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->collect();
    if (gace_status st = read_status(ctx, *reinterpret_cast<unsigned int*>(ctx->pin + status_off))) return st;
    const uint32_t* r32 = reinterpret_cast<const uint32_t*>(ctx->pin + regs_off);
    std::vector<uint8_t> regs(m);
    for (uint64_t j = 0; j < m; ++j) regs[j] = static_cast<uint8_t>(r32[j]);
    if (registers_out) memcpy(registers_out, regs.data(), m);
    if (estimate_out) *estimate_out = hll_estimate_host(regs.data(), p);
    resident_sketch_put(ctx, table_id, col, p, hash_seed, regs.data());
    return GACE_OK;
}

// ---------------------------------------------------------------- joins



gace_status gace_join_card(gace_ctx* ctx, const gace_join* spec, gace_join_result* out) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (!spec || !out) return fail(GACE_EINVAL, "spec or out is NULL");
    if (spec->hops != 1 && spec->hops != 2) return fail(GACE_EINVAL, "hops = %u (1 or 2)", spec->hops);
    if (spec->method > GACE_JOIN_GATHER) return fail(GACE_EINVAL, "method %u invalid", spec->method);
    if (spec->key_domain == 0 || spec->key_domain > (1ull << 32))
        return fail(GACE_EINVAL, "key_domain %llu outside 1..2^32", (unsigned long long)spec->key_domain);
    if (spec->hops == 2 && (spec->key_domain2 == 0 || spec->key_domain2 > (1ull << 32)))
        return fail(GACE_EINVAL, "key_domain2 %llu outside 1..2^32", (unsigned long long)spec->key_domain2);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    std::vector<uint32_t> pool;
    SideArgs F, D, D2;
    TableRec *tf = nullptr, *td = nullptr, *td2 = nullptr;
    uint32_t fk2_slot = 0;
    SideWork wf, wd, wd2;
    if (gace_status st = build_side(ctx, spec->fact, "fact", -1, F, pool, &tf, nullptr, wf)) return st;
    if (gace_status st = build_side(ctx, spec->dim, "dim", spec->hops == 2 ? static_cast<int>(spec->dim_fk2_col) : -1, D,
                                    pool, &td, &fk2_slot, wd))
        return st;
    if (spec->hops == 2)
        if (gace_status st = build_side(ctx, spec->dim2, "dim2", -1, D2, pool, &td2, nullptr, wd2)) return st;
    auto side = [&](const char* nm, const SideWork& w, auto&& f) {
        return ctx->traced(nm, w.rows, w.rows * w.rowbytes, w.rows * w.ops_per_row, f);
    };
    auto vec = [&](const char* nm, uint64_t n, uint64_t bytes_per, auto&& f) {
        return ctx->traced(nm, n, n * bytes_per, n, f);
    };
    const bool hist_dot = spec->method == GACE_JOIN_HIST_DOT;
    if (td->nrows >= (1ull << 32) || (td2 && td2->nrows >= (1ull << 32)))
        return fail(GACE_EINVAL, "a histogrammed dimension has 2^32 or more rows");
    if (hist_dot && tf->nrows >= (1ull << 32))
        return fail(GACE_EINVAL, "GACE_JOIN_HIST_DOT needs a fact table below 2^32 rows");
    const uint64_t K = spec->key_domain, K2 = spec->hops == 2 ? spec->key_domain2 : 0;

    // workspace: status | scalars | pool | h_D (or h_D2 + w) | h_F
    Ws ws;
    const uint64_t status_off = ws.take(256);
    const uint64_t sc_off = ws.take(8 * 8);  // fact_pass dim_pass dim2_pass sum max_h max_w
    const uint64_t pool_off = ws.take(pool.size() * 4 + 16);
    const uint64_t hd_off = ws.take((spec->hops == 2 ? K2 : K) * 4);
    const uint64_t w_off = spec->hops == 2 ? ws.take(K * 8) : 0;
    const uint64_t hf_off = hist_dot ? ws.take(K * 4) : 0;
    if (gace_status st = ctx->ensure_ws(ws.off)) return st;
    if (gace_status st = ctx->ensure_pin(pool_off + pool.size() * 4 + 16)) return st;
    unsigned char* w = ctx->ws;
    unsigned long long* sc = reinterpret_cast<unsigned long long*>(w + sc_off);
    unsigned int* status = reinterpret_cast<unsigned int*>(w + status_off);
    const uint32_t* dpool = reinterpret_cast<const uint32_t*>(w + pool_off);
    if (!pool.empty()) {
        memcpy(ctx->pin + pool_off, pool.data(), pool.size() * 4);
        CK(cudaMemcpyAsync(w + pool_off, ctx->pin + pool_off, pool.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaMemsetAsync(w, 0, pool_off, ctx->stream));
    CK(cudaMemsetAsync(w + hd_off, 0, ws.off - hd_off, ctx->stream));
    for (SideArgs* s : {&F, &D, &D2}) {
        s->pool = dpool;
        s->status = status;
    }
    F.domain = K;
    F.pass_count = sc + 0;
    D.domain = K;
    D.pass_count = sc + 1;
    const int sms = ctx->sms;
    uint32_t* hD = reinterpret_cast<uint32_t*>(w + hd_off);
    if (spec->hops == 1) {
        CK(side("join_hist", wd, [&] { return hist_launch(D, hD, 1, 1, sms, ctx->stream); }));
        CK(vec("join_max", K, 4, [&] { return max_launch(hD, 0, K, sc + 4, sms, ctx->stream); }));
        if (hist_dot) {
            uint32_t* hF = reinterpret_cast<uint32_t*>(w + hf_off);
            CK(side("join_hist", wf, [&] { return hist_launch(F, hF, 0, 1, sms, ctx->stream); }));
            CK(vec("join_dot", K, 8, [&] { return dot_launch(hF, hD, 0, K, sc + 3, sms, ctx->stream); }));
        } else {
            CK(side("join_gather", wf, [&] { return gather_launch(F, hD, 0, sc + 3, sms, ctx->stream); }));
        }
    } else {
        D2.domain = K2;
        D2.pass_count = sc + 2;
        unsigned long long* wk = reinterpret_cast<unsigned long long*>(w + w_off);
        CK(side("join_hist", wd2, [&] { return hist_launch(D2, hD, 1, 1, sms, ctx->stream); }));
        CK(vec("join_max", K2, 4, [&] { return max_launch(hD, 0, K2, sc + 4, sms, ctx->stream); }));
        CK(side("join_chain", wd, [&] { return chain_weight_launch(D, fk2_slot, K2, hD, wk, sms, ctx->stream); }));
        CK(vec("join_max", K, 8, [&] { return max_launch(wk, 1, K, sc + 5, sms, ctx->stream); }));
        if (hist_dot) {
            uint32_t* hF = reinterpret_cast<uint32_t*>(w + hf_off);
            CK(side("join_hist", wf, [&] { return hist_launch(F, hF, 0, 1, sms, ctx->stream); }));
            CK(vec("join_dot", K, 12, [&] { return dot_launch(hF, wk, 1, K, sc + 3, sms, ctx->stream); }));
        } else {
            CK(side("join_gather", wf, [&] { return gather_launch(F, wk, 1, sc + 3, sms, ctx->stream); }));
        }
    }
    CK(cudaMemcpyAsync(ctx->pin, w, sc_off + 64, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->collect();
    const unsigned int st = *reinterpret_cast<unsigned int*>(ctx->pin + status_off);
    if (st & kStatusKeyDomain) return fail(GACE_EINVAL, "a filtered dimension row has a key outside its domain");
    if (gace_status s = read_status(ctx, st)) return s;
    const unsigned long long* h = reinterpret_cast<const unsigned long long*>(ctx->pin + sc_off);
    const unsigned __int128 lim = static_cast<unsigned __int128>(1) << 63;
    if (spec->hops == 1) {
        if (static_cast<unsigned __int128>(h[0]) * h[4] >= lim)
            return fail(GACE_EOVERFLOW, "fact_rows * max h_D >= 2^63");
    } else {
        if (static_cast<unsigned __int128>(h[1]) * h[4] >= lim)
            return fail(GACE_EOVERFLOW, "dim_rows * max h_D2 >= 2^63");
        if (static_cast<unsigned __int128>(h[0]) * h[5] >= lim)
            return fail(GACE_EOVERFLOW, "fact_rows * max w >= 2^63");
    }
    out->card = static_cast<int64_t>(h[3]);
    out->fact_rows = h[0];
    out->dim_rows = h[1];
    out->dim2_rows = spec->hops == 2 ? h[2] : 0;
    return GACE_OK;
}

gace_status gace_stats_reset(gace_ctx* ctx, uint32_t time_kernels) {
    if (gace_status s = check_ctx(ctx)) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->collect();
    ctx->stats.clear();
    ctx->timing = time_kernels != 0;
    return GACE_OK;
}

gace_status gace_stats_read(gace_ctx* ctx, gace_kernel_stat* out, uint32_t cap, uint32_t* n_out) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (!n_out || (cap && !out)) return fail(GACE_EINVAL, "out or n_out is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->collect();
    uint32_t i = 0;
    for (const auto& kv : ctx->stats) {
        if (i < cap) {
            gace_kernel_stat& o = out[i];
            memset(&o, 0, sizeof(o));
            strncpy(o.name, kv.first.c_str(), sizeof(o.name) - 1);
            o.launches = kv.second.launches;
            o.rows = kv.second.rows;
            o.bytes = kv.second.bytes;
            o.ops = kv.second.ops;
            o.total_ms = kv.second.ms;
        }
        ++i;
    }
    *n_out = i;
    return GACE_OK;
}

}  // extern "C"
