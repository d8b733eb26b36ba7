// gace_gate.cpp -- the Risky Gate's trust metrics (Section III-C, Eq. 1-3)
// and the break-even cost model (Section V, item 2; Eq. 4), on the host.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "gace_host.h"

using namespace gace;
using namespace gace::host;

namespace {

// Default rates, measured on GB300 with this library's kernels: a narrow
// probe streams about 5 TB/s of referenced columns, the wide passes evaluate
// about 1.3e13 compare operations per second, a pinned host-to-device copy
// (allocation included) runs near 200 GB/s, hashing a row for a sample costs
// about 1.5 ps per row
// and set, and a synchronous call's fixed cost is about 30 us.
constexpr double kDefaultHbmRate = 5e12;
constexpr double kDefaultOpsRate = 1.3e13;
constexpr double kDefaultH2dRate = 2e11;
constexpr double kDefaultHashNs = 1.5e-3;
constexpr double kDefaultCallMs = 0.03;

// The paper's thresholds.
constexpr double kDriftMin = 0.25;   // Eq. 1
constexpr double kSelErrMax = 0.01;  // Eq. 2
constexpr double kPcsHigh = 1.6;     // Eq. 3
constexpr double kPcsLow = 0.7;

bool bad_threshold(double x) { return std::isnan(x) || std::isinf(x) || x < 0.0; }

}  // namespace

extern "C" {

gace_status gace_gate_eval(const gace_gate_config* cfg, const gace_gate_input* in, uint32_t n,
                           gace_gate_result* out) {
    if (n > 0 && (!in || !out)) return fail(GACE_EINVAL, "in or out is NULL");
    gace_gate_config c{kDriftMin, kSelErrMax, kPcsHigh, kPcsLow};
    if (cfg) {
        if (bad_threshold(cfg->drift_min) || bad_threshold(cfg->sel_err_max) || bad_threshold(cfg->pcs_high) ||
            bad_threshold(cfg->pcs_low))
            return fail(GACE_EINVAL, "gate thresholds must be finite and >= 0");
        if (cfg->drift_min != 0.0) c.drift_min = cfg->drift_min;
        if (cfg->sel_err_max != 0.0) c.sel_err_max = cfg->sel_err_max;
        if (cfg->pcs_high != 0.0) c.pcs_high = cfg->pcs_high;
        if (cfg->pcs_low != 0.0) c.pcs_low = cfg->pcs_low;
    }
    if (c.pcs_low > c.pcs_high) return fail(GACE_EINVAL, "pcs_low %g > pcs_high %g", c.pcs_low, c.pcs_high);
    const double nan = std::nan("");
    for (uint32_t i = 0; i < n; ++i) {
        const gace_gate_input& x = in[i];
        gace_gate_result r{};
        r.drift = nan;
        r.sel_err = nan;
        // Eq. 1: relative NDV drift against the histogram's NDV
        if (std::isfinite(x.ndv_hist) && x.ndv_hist > 0.0 && !std::isnan(x.ndv_est)) {
            r.drift = std::fabs(x.ndv_hist - x.ndv_est) / x.ndv_hist;
            if (r.drift >= c.drift_min) r.flags |= GACE_RISK_DRIFT;
        }
        // Eq. 2: the estimate misses the measured selectivity
        if (!std::isnan(x.sel_est) && !std::isnan(x.sel_probe)) {
            r.sel_err = std::fabs(x.sel_est - x.sel_probe);
            if (r.sel_err > c.sel_err_max) r.flags |= GACE_RISK_SELECTIVITY;
        }
        // Eq. 3: joint vs independent selectivity out of the trusted band
        if (!std::isnan(x.pcs) && (x.pcs > c.pcs_high || x.pcs < c.pcs_low)) r.flags |= GACE_RISK_CORRELATION;
        out[i] = r;
    }
    return GACE_OK;
}

gace_status gace_break_even(gace_ctx* ctx, const gace_cost_query* q, gace_cost_answer* out) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (!q || !out) return fail(GACE_EINVAL, "query or answer is NULL");
    if (q->nsets == 0) return fail(GACE_EINVAL, "nsets is 0");
    if (q->hashed_sets > q->nsets) return fail(GACE_EINVAL, "hashed_sets %u > nsets %u", q->hashed_sets, q->nsets);
    if (std::isnan(q->alt_ms) || q->alt_ms < 0.0) return fail(GACE_EINVAL, "alt_ms must be >= 0");
    if (std::isnan(q->ops_per_row) || q->ops_per_row < 0.0) return fail(GACE_EINVAL, "ops_per_row must be >= 0");
    gace_cost_answer a{};
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        const gace_ctx::CostRec& cn = ctx->cost_narrow;
        const gace_ctx::CostRec& cw = ctx->cost_wide;
        a.hbm_rate = kDefaultHbmRate;
        a.ops_rate = kDefaultOpsRate;
        if (cn.launches && cn.ms > 0.0 && cn.bytes > 0.0) {
            a.hbm_rate = cn.bytes / (cn.ms * 1e-3);
            a.measured |= 1u;
        }
        if (cw.launches && cw.ms > 0.0 && cw.ops > 0.0) {
            a.ops_rate = cw.ops / (cw.ms * 1e-3);
            a.measured |= 2u;
        }
    }
    a.h2d_rate = kDefaultH2dRate;
    a.hash_ns = kDefaultHashNs;
    a.call_ms = kDefaultCallMs;
    const double n = static_cast<double>(q->nrows);
    const double bytes = n * q->row_bytes;
    a.narrow = q->npreds <= static_cast<uint32_t>(kNarrowMax) && q->nterms <= static_cast<uint32_t>(kNarrowMax) ? 1u
                                                                                                                 : 0u;
    if (a.narrow) {
        a.kernel_ms = bytes / a.hbm_rate * 1e3 + n * q->hashed_sets * a.hash_ns * 1e-6;
    } else {
        const double ops = q->ops_per_row > 0.0 ? q->ops_per_row : 2.0 * q->nterms;
        a.kernel_ms = n * ops / a.ops_rate * 1e3;
    }
    a.transfer_ms = q->resident ? 0.0 : bytes / a.h2d_rate * 1e3;
    a.total_ms = a.call_ms + a.kernel_ms + a.transfer_ms;
    a.offload = a.total_ms < q->alt_ms ? 1u : 0u;
    *out = a;
    return GACE_OK;
}

gace_status gace_check_wait_limit(gace_ctx* ctx, uint32_t timeout_us) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (timeout_us == 0 || timeout_us > 10000000u) return fail(GACE_EINVAL, "timeout_us %u outside 1..10^7", timeout_us);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (gace_status s = ctx->ensure_ws(256)) return s;
    if (gace_status s = ctx->ensure_pin(256)) return s;
    unsigned int* status = reinterpret_cast<unsigned int*>(ctx->ws);
    cudaError_t e = cudaMemsetAsync(status, 0, 4, ctx->stream);
    if (e == cudaSuccess) e = wait_check_launch(status, static_cast<uint64_t>(timeout_us) * 1000ull, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->pin, status, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "wait check");
    const unsigned int st = *reinterpret_cast<const unsigned int*>(ctx->pin);
    if (st & kStatusTimeout) return fail(GACE_ETIMEDOUT, "the check's device wait gave up after %u us", timeout_us);
    return fail(GACE_ECUDA, "the check's device wait ended without giving up");
}

gace_status gace_calibrate_int(gace_ctx* ctx, uint32_t kind, uint32_t ms, double* ops_per_s) {
    if (gace_status s = check_ctx(ctx)) return s;
    if (kind > 1) return fail(GACE_EINVAL, "calibration kind %u (0 or 1)", kind);
    if (ms == 0 || ms > 1000) return fail(GACE_EINVAL, "ms %u outside 1..1000", ms);
    if (!ops_per_s) return fail(GACE_EINVAL, "ops_per_s is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (gace_status s = ctx->ensure_ws(256)) return s;
    const int occ = int_peak_occupancy(static_cast<int>(kind));
    if (occ < 1) return fail(GACE_ECUDA, "calibration kernel cannot be resident");
    const int grid = ctx->sms * occ;
    uint32_t* sink = reinterpret_cast<uint32_t*>(ctx->ws);
    cudaEvent_t a = ctx->take_event(), b = ctx->take_event();
    if (!a || !b) return fail(GACE_ECUDA, "cudaEventCreate");
    auto timed = [&](uint32_t iters, float* out_ms) -> cudaError_t {
        cudaError_t e = cudaEventRecord(a, ctx->stream);
        if (e == cudaSuccess) e = int_peak_launch(static_cast<int>(kind), iters, grid, sink, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(b, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(out_ms, a, b);
        return e;
    };
    float t = 0.f;
    uint32_t iters = 64;
    cudaError_t e = timed(iters, &t);  // warm-up and first estimate
    // grow the launch until it lasts about `ms` (at most 2^24 iterations)
    while (e == cudaSuccess && t < 0.25f * ms && iters < (1u << 24)) {
        iters *= 4;
        e = timed(iters, &t);
    }
    double best = 0.0;
    for (int rep = 0; e == cudaSuccess && rep < 3; ++rep) {
        e = timed(iters, &t);
        if (e == cudaSuccess && t > 0.f) {
            const double ops = static_cast<double>(grid) * 256.0 * iters * int_peak_ops_per_iter(static_cast<int>(kind));
            best = std::max(best, ops / (t * 1e-3));
        }
    }
    ctx->ev_free.push_back(a);
    ctx->ev_free.push_back(b);
    if (e != cudaSuccess) return cuda_fail(e, "calibration kernel");
    *ops_per_s = best;
    return GACE_OK;
}

}  // extern "C"
