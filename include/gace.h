/*
 * gace.h -- C ABI of libgace, the GPU probe engine of GACE on GB300 (sm_103a).
 *
 * GACE (I.-S. Chang, "Risk-Aware GPU-Assisted Cardinality Estimation for
 * Cost-Based Query Optimizers", arXiv 2512.19750) pairs a Risky Gate with a
 * Measurement Engine that measures, on the GPU, the selectivity and the
 * distribution of an optimizer's candidate conditions (Section III-B) using
 * full scans, sampling and block-level summaries.  This library is that
 * measurement path over device-resident columnar tables:
 *
 *   gace_probe_batch  counts of conjunctive EQ / RANGE / IN predicates over the
 *                     full table, a seeded row sample or a seeded block sample,
 *                     with per-term marginals and the PCS signal (Eq. 3);
 *   gace_ndv          HyperLogLog registers and NDV estimate of a column (the
 *                     NDV_est of the drift signal, Eq. 1);
 *   gace_join_card    exact join cardinality of two filtered tables (and a
 *                     three-table chain) as the dot product of filtered
 *                     key-frequency histograms (join workload, Section IV-F).
 *
 * Conventions for every call:
 *   - The return value is a gace_status; nothing aborts or exits.  On an error
 *     the outputs are left untouched and gace_last_error() describes it.
 *   - Caller-provided output arrays are HOST memory.
 *   - A context serialises its calls on its own CUDA stream; calls on one
 *     context from several threads are safe (they take a lock).
 *   - Counts are exact unsigned 64-bit integers.  Doubles derived from them
 *     (selectivity, PCS) come from one IEEE expression each, stated below.
 */
#ifndef GACE_H
#define GACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GACE_ABI_VERSION 4

typedef enum {
    GACE_OK = 0,
    GACE_EINVAL = 1,    /* an argument is invalid (message in gace_last_error) */
    GACE_ENOMEM = 2,    /* device or pinned memory exhausted, or HBM budget exceeded */
    GACE_EBUSY = 3,     /* a queue is full */
    GACE_EPENDING = 4,  /* the result is not ready yet */
    GACE_ETIMEDOUT = 5, /* a device-side wait gave up after the context's wait limit */
    GACE_ENOTFOUND = 6, /* unknown table id or ticket */
    GACE_EOVERFLOW = 7, /* a join cardinality could exceed 2^63 - 1 */
    GACE_ECUDA = 8      /* a CUDA runtime call failed (no GPU, launch error, ...) */
} gace_status;

typedef enum { GACE_I32 = 0, GACE_I64 = 1, GACE_F32 = 2 } gace_dtype;
typedef enum { GACE_EQ = 0, GACE_RANGE = 1, GACE_IN = 2 } gace_op;
typedef enum { GACE_FULL = 0, GACE_ROWS = 1, GACE_BLOCKS = 2 } gace_sample_kind;
typedef enum { GACE_COPY = 0, GACE_BORROW = 1, GACE_COPY_ON_FIRST_PROBE = 2 } gace_load_flags;

typedef struct gace_ctx gace_ctx;

/* A constant: integer columns read .i, float32 columns read .f. */
typedef union {
    int64_t i;
    double f;
} gace_scalar;

typedef struct {
    int32_t device;            /* CUDA device ordinal */
    uint32_t wait_timeout_ms;  /* limit of every device-side wait; 0 selects 2000 ms */
    uint64_t hbm_budget_bytes; /* device bytes the context may hold (tables it copies,
                                  workspaces); 0 = no limit */
    void* stream;              /* cudaStream_t for all work; NULL = a private
                                  non-blocking stream */
    uint32_t max_ctas;         /* most CTAs one gace_probe_batch launch uses, to
                                  leave SMs to other work on the GPU (0 = as
                                  many as are resident at once); raised where a
                                  CTA would otherwise count 2^31 rows or more
                                  in its 32-bit counters */
    uint32_t rank_min_rows;    /* a gace_probe_batch call over a table of fewer
                                  rows does not rank-code its columns
                                  (0 selects 1048576; the call must also have
                                  more than 32 predicates and at least 384
                                  distinct terms).  Rank coding changes no
                                  result, only the kernels that compute it */
    uint32_t rank_search;      /* how the rank pass finds a value's rank among a
                                  column's endpoints: 0 = per column, a bucket
                                  index (the value's bucket gives the first
                                  candidate endpoint, a few halvings the rank)
                                  where it takes at least two fewer dependent
                                  lookups than the search tree, else the tree;
                                  1 = the search tree; 2 = the bucket index.
                                  Changes no result; other values: GACE_EINVAL */
} gace_config;

/* One column of a table: nrows elements of dtype, densely packed. */
typedef struct {
    int32_t dtype;      /* gace_dtype */
    int32_t on_device;  /* 1: data is a device pointer; 0: host pointer */
    const void* data;
} gace_column;

/*
 * A candidate condition on one column (Section III-B):
 *   GACE_EQ     x == a
 *   GACE_RANGE  a <= x < b                        (half-open; a >= b matches nothing)
 *   GACE_IN     x equals one of in_values[in_off .. in_off + in_len)
 * Integer columns compare exact integers (a constant outside the column's
 * range simply matches nothing).  Float32 columns compare the value, widened
 * to double, with double constants under IEEE rules: NaN matches nothing and
 * -0 equals +0.  in_len is 1..4096.
 */
typedef struct {
    uint32_t col;
    uint32_t op;        /* gace_op */
    gace_scalar a;
    gace_scalar b;
    uint32_t in_off;
    uint32_t in_len;
} gace_term;

/* A predicate is the conjunction of terms[term_off .. term_off + term_cnt);
 * term_cnt == 0 matches every row. */
typedef struct {
    uint32_t term_off;
    uint32_t term_cnt;
} gace_pred;

/*
 * The rows a probe counts over (dynamic sampling, Sections II-A and III-B):
 *   GACE_FULL    every row.
 *   GACE_ROWS    row i (0-based, table-global) is kept iff H(i, seed) < T(rate).
 *   GACE_BLOCKS  block b = floor(i / block_rows) is kept iff H(b, seed) < T(rate);
 *                all rows of a kept block count (the last block may be short).
 * H(x, s) = splitmix64(x XOR splitmix64(s)) with the splitmix64 output function
 * of Steele, Lea & Flood (OOPSLA 2014).  T(rate) = floor(rate * 2^64); rate <= 0
 * keeps nothing and rate >= 1 keeps everything.  Samples are nested in rate.
 */
typedef struct {
    uint32_t kind;        /* gace_sample_kind */
    uint32_t block_rows;  /* GACE_BLOCKS: rows per block, >= 1 */
    double rate;
    uint64_t seed;
} gace_sample;

/*
 * Result of one predicate on one row set:
 *   match        rows of the set on which every term holds
 *   sample_rows  rows in the set
 *   sel          match / sample_rows as doubles (0 when sample_rows == 0)
 *   pcs          for a predicate of exactly two terms A and B:
 *                (double)c_AB * (double)n / ((double)c_A * (double)c_B),
 *                with n = sample_rows and c_A, c_B the terms' marginal counts on
 *                the same set (PCS = P(A,B)/(P(A)P(B)), Section III-C, Eq. 3);
 *                NaN for other predicates or when c_A or c_B is zero.
 */
typedef struct {
    uint64_t match;
    uint64_t sample_rows;
    double sel;
    double pcs;
} gace_pred_result;

/* Creates a context on cfg->device (cfg may be NULL: device 0, defaults).
 * Fails with GACE_ECUDA when no usable GPU is present. */
gace_status gace_create(gace_ctx** out, const gace_config* cfg);

/* Frees every table the context copied and every workspace.  NULL is a no-op. */
gace_status gace_destroy(gace_ctx* ctx);

/*
 * Registers a table of nrows rows and ncols (1..64) columns.
 * flags == GACE_COPY: the context copies each column (host or device source)
 *   into device memory it owns, 256-byte aligned; counted against the budget.
 * flags == GACE_BORROW: the context keeps the device pointers; the caller keeps
 *   them alive and unchanged until gace_unload.  Every column must be on_device.
 * flags == GACE_COPY_ON_FIRST_PROBE: host columns the context copies, like
 *   GACE_COPY, but not before the first call that reads the table; when that
 *   call is gace_probe_batch, the copy streams in row chunks on a second
 *   stream while the probe's passes run on the chunks already copied (a probe
 *   of columns that were not resident costs about the larger of the copy and
 *   the kernels, not their sum; the paper's prototype copies key columns per
 *   probe, Section IV-B).  The host columns must stay valid and unchanged
 *   until that call returns (or the table is unloaded); pinned memory lets the
 *   copy run at full speed.  Any other call completes the copy first.
 * Device columns are read on the context's stream: work on other streams that
 * writes them must be complete (or ordered before that stream) when they are
 * read.  A GACE_COPY load from device memory waits for the whole device first;
 * a borrowed column is read by every later call on the table.
 * The probe reads each column with 16-byte bulk copies when its base address is
 * 16-byte aligned, and with plain loads otherwise (same results, slower).
 */
gace_status gace_load_columns(gace_ctx* ctx, uint64_t nrows, uint32_t ncols,
                              const gace_column* cols, uint32_t flags,
                              uint32_t* table_id_out);

/* Forgets a table (frees its copies when it was loaded with GACE_COPY). */
gace_status gace_unload(gace_ctx* ctx, uint32_t table_id);

/*
 * Measurement Engine probe (Section III-B; Key-Only + Bitmask evaluation,
 * Section IV-H): fused passes over the referenced columns evaluate every
 * predicate on every requested row set (one pass unless the batch outgrows a
 * pass's shared-memory tables; each pass reads only its own columns).  When
 * every row set is a block sample, only the tiles that hold a sampled block
 * are read.
 *   samples[nsamples]   1..8 row sets
 *   terms[nterms]       the terms the predicates index; identical terms are
 *                       evaluated once
 *   in_values[nin]      IN lists
 *   preds[npreds]       conjunctions
 *   results             out, nsamples * npreds entries, results[s * npreds + p]
 *   term_marginals      out or NULL, nsamples * nterms entries: rows of set s
 *                       on which term t holds
 */
gace_status gace_probe_batch(gace_ctx* ctx, uint32_t table_id,
                             const gace_sample* samples, uint32_t nsamples,
                             const gace_term* terms, uint32_t nterms,
                             const gace_scalar* in_values, uint32_t nin,
                             const gace_pred* preds, uint32_t npreds,
                             gace_pred_result* results, uint64_t* term_marginals);

/*
 * HyperLogLog NDV of one column (the NDV_est of the drift signal D, Eq. 1;
 * sketch of Flajolet, Fusy, Gandouet & Meunier, AofA 2007) with m = 2^p
 * registers, p in 4..18.  Each value's canonical 64-bit key (int32
 * sign-extended, int64 as is, float32 bit pattern zero-extended after mapping
 * -0 to +0 and every NaN to 0x7FC00000) is hashed h = H(key, hash_seed);
 * register j = top p bits of h; rho = 1-based position of the leftmost 1 in
 * the remaining 64 - p bits (64 - p + 1 if they are all zero); M[j] = max rho.
 *   registers_out  out or NULL, 2^p bytes
 *   estimate_out   out or NULL: alpha_m m^2 / sum_j 2^-M[j] (alpha_m = 0.673,
 *                  0.697, 0.709 for m = 16, 32, 64, else 0.7213/(1 + 1.079/m)),
 *                  replaced by m ln(m / V) when it is <= 2.5 m and V, the number
 *                  of zero registers, is positive.
 */
gace_status gace_ndv(gace_ctx* ctx, uint32_t table_id, uint32_t col, uint32_t p,
                     uint64_t hash_seed, uint8_t* registers_out, double* estimate_out);

/* One side of a join: a table, its key column (int32 or int64) and a
 * conjunctive filter (nterms may be 0). */
typedef struct {
    uint32_t table_id;
    uint32_t key_col;
    const gace_term* terms;
    uint32_t nterms;
    uint32_t nin;
    const gace_scalar* in_values;
} gace_join_side;

typedef enum { GACE_JOIN_AUTO = 0, GACE_JOIN_HIST_DOT = 1, GACE_JOIN_GATHER = 2 } gace_join_method;

/*
 * Join cardinality (the join-correlation failures of Sections I and IV-F):
 *   hops == 1:  J = |sigma(fact) JOIN_{fact.key = dim.key} sigma(dim)|
 *             = sum_k h_F[k] * h_D[k] over k in [0, key_domain), where h_X[k]
 *               counts the filtered rows of X whose key equals k.
 *   hops == 2:  chain fact -> dim -> dim2 through dim's column dim_fk2_col:
 *               J = sum_k h_F[k] * w[k], w[k] = sum over filtered dim rows d
 *               with d.key = k of h_D2[d.fk2], h_D2 over [0, key_domain2).
 * Every filtered dim (and dim2) row must have its key inside its domain, else
 * GACE_EINVAL; fact (and dim.fk2) keys outside the domain match nothing.
 * GACE_EOVERFLOW when fact_rows * max_k h_D[k] >= 2^63 (hops == 1), or when
 * dim_rows * max h_D2 >= 2^63 or fact_rows * max_k w[k] >= 2^63 (hops == 2).
 * A histogrammed side must have fewer than 2^32 rows.
 * method: GACE_JOIN_HIST_DOT builds both histograms and takes their dot
 * product; GACE_JOIN_GATHER builds h_D (or w) only and sums h_D[fact.key] over
 * the filtered fact rows, the same integer; GACE_JOIN_AUTO picks.
 */
typedef struct {
    gace_join_side fact;
    gace_join_side dim;
    uint64_t key_domain;
    gace_join_side dim2;
    uint64_t key_domain2;
    uint32_t dim_fk2_col;
    uint32_t hops;      /* 1 or 2 */
    uint32_t method;    /* gace_join_method */
    uint32_t reserved;
} gace_join;

typedef struct {
    int64_t card;       /* join cardinality */
    uint64_t fact_rows; /* fact rows passing the fact filter */
    uint64_t dim_rows;  /* dim rows passing the dim filter */
    uint64_t dim2_rows; /* dim2 rows passing the dim2 filter (hops == 2) */
} gace_join_result;

gace_status gace_join_card(gace_ctx* ctx, const gace_join* spec, gace_join_result* out);

/*
 * HyperLogLog of one device column WITHOUT ANY ALLOCATION, for callers that
 * cannot allocate device memory: an optimizer's planning hook that must not
 * trigger cudaMalloc's device-wide synchronisation and unbounded latency while
 * a query is planned, or a process whose device memory belongs to another
 * allocator (a database buffer manager, a framework's caching allocator under
 * a hard cap).  The paper has no counterpart for this entry point; it computes
 * exactly what gace_ndv computes, without a context.
 *
 * Scratch: one fixed array of 328,448 bytes inside the library (32-bit and byte
 * registers for up to 2^GACE_NOALLOC_MAX_P of them, a value histogram, a status
 * word); every GPU that loads the library holds it until the process exits.
 * Every call uses all of it and clears what must start at zero, so calls that
 * overlap on the GPU (other streams or host threads) race and must be
 * serialised by the caller.  Each call looks up the array's device address on
 * the current device (cudaGetSymbolAddress, which allocates nothing once the
 * library's module is loaded there).  With CUDA's default lazy module loading,
 * the FIRST call on each device loads the module, which may allocate and
 * synchronise: warm the entry point up once per device before the code that
 * must not allocate, or run with CUDA_MODULE_LOADING=EAGER.  Every call waits
 * for its stream and copies its results to host memory, so it must never be
 * called while a stream is being captured into a CUDA graph.  No cudaMalloc,
 * cudaFree or allocating library routine is called.
 *   column         device pointer to nrows elements of dtype (the current device)
 *   p              4..GACE_NOALLOC_MAX_P; larger p is rejected with GACE_EINVAL
 *   stream         cudaStream_t to run on (NULL: the default stream); the call
 *                  waits for it before returning
 *   registers_out  HOST, 2^p bytes, or NULL (may be written even if a device
 *                  wait then reports GACE_ETIMEDOUT)
 *   estimate_out   HOST or NULL, as in gace_ndv
 */
#define GACE_NOALLOC_MAX_P 16
gace_status gace_ndv_noalloc(const void* column, int32_t dtype, uint64_t nrows, uint32_t p,
                             uint64_t hash_seed, void* stream, uint8_t* registers_out,
                             double* estimate_out);

/* ------------------------------------------------- resident samples and sketches */

/*
 * Materialised sample (the Measurement Engine's sampling, Section III-B, kept
 * for the gate's repeated invocations while queries are planned, Section
 * III-A): the rows of `sample` of table_id (GACE_ROWS or GACE_BLOCKS with
 * 0 < rate < 1), every column, in row order, copied into a new table that the
 * context owns (counted against the HBM budget).  A GACE_FULL probe of the new
 * table returns exactly the counts, sample_rows, selectivities, PCS and
 * marginals that the same probe of table_id with `sample` returns, and its
 * row count (rows_out, may be NULL) is that sample_rows.  Two passes decide
 * membership as the probe does (one hash per row or block); the second loads
 * only the kept rows.  gace_unload frees the new table; unloading table_id
 * does not.  GACE_EINVAL for another sample kind or rate, GACE_ENOMEM beyond
 * the budget.
 */
gace_status gace_sample_materialize(gace_ctx* ctx, uint32_t table_id, const gace_sample* sample,
                                    uint32_t* sample_table_out, uint64_t* rows_out);

/*
 * The resident store: samples and HyperLogLog sketches kept in device memory
 * under a byte budget and used by every form of the calls (gace_probe_batch,
 * gace_ndv, batched and served requests) without a change to the requests:
 *  - a row set that is a row or block sample (0 < rate < 1) held by the store
 *    is counted by a full scan of the resident sample (the same integers as a
 *    scan of the base table that hashes every row).  A sample not held is
 *    admitted (materialised) once it has been asked for admit_after times
 *    (0 or 1: at its first use) if it fits the budget after the least recently
 *    used entries that no request in flight is using are evicted; otherwise
 *    (refused) the probe scans the base table;
 *  - an NDV request whose (table, column, p, seed) sketch is held is answered
 *    from the resident registers (2^p bytes read back); a sketch a call
 *    computes is kept, admitted and evicted the same way.
 * The served form rewrites a probe at submission only when all its row sets
 * are one sample; the synchronous call splits any mix of row sets.
 * budget_bytes = 0 turns the store off (the default) and frees its entries;
 * a changed configuration frees them and restarts the statistics.  Unloading
 * a table drops what the store drew from it.
 */
#define GACE_RESIDENT_SAMPLES 1u
#define GACE_RESIDENT_SKETCHES 2u
typedef struct {
    uint64_t budget_bytes;  /* device bytes for resident samples and sketches; 0 = off */
    uint32_t admit_after;   /* uses of a sample before it is materialised (0 or 1: the first) */
    uint32_t flags;         /* GACE_RESIDENT_SAMPLES | GACE_RESIDENT_SKETCHES; 0 = both */
} gace_resident_config;

typedef struct {
    uint64_t budget_bytes, used_bytes;
    uint64_t samples, sketches;          /* entries held */
    uint64_t sample_hits, sample_misses; /* row sets counted on / not on a resident sample */
    uint64_t admitted, refused, evicted; /* samples materialised into the store, refused, evicted */
    uint64_t sketch_hits, sketch_misses, sketch_evicted;
} gace_resident_stats;

gace_status gace_resident_configure(gace_ctx* ctx, const gace_resident_config* cfg);

/* Materialises a sample into the store now (admission and eviction as above);
 * GACE_ENOMEM when it cannot fit, GACE_EINVAL when the store is off or the
 * sample is not a row or block sample with 0 < rate < 1.  A sample already
 * held is only refreshed. */
gace_status gace_resident_prefetch(gace_ctx* ctx, uint32_t table_id, const gace_sample* sample);

gace_status gace_resident_stats_read(gace_ctx* ctx, gace_resident_stats* out);

/* ------------------------------------------------------------ batched form */

typedef enum { GACE_REQ_PROBE = 0, GACE_REQ_NDV = 1, GACE_REQ_JOIN = 2 } gace_req_kind;

/*
 * One request of a batch (gace_run_batch): the arguments and outputs of the
 * matching synchronous call (gace_probe_batch, gace_ndv or gace_join_card),
 * fields of the other kinds ignored.  Output pointers are HOST memory.  The
 * paper's Risky Gate issues many such probes per query workload (Section
 * III-A); the batch runs them together.
 */
typedef struct {
    uint32_t kind;                /* gace_req_kind */
    uint32_t table_id;            /* PROBE, NDV */
    const gace_sample* samples;   /* PROBE */
    uint32_t nsamples;
    uint32_t nterms;
    const gace_term* terms;
    const gace_scalar* in_values;
    uint32_t nin;
    uint32_t npreds;
    const gace_pred* preds;
    gace_pred_result* results;    /* out, nsamples * npreds */
    uint64_t* term_marginals;     /* out or NULL */
    uint32_t col;                 /* NDV */
    uint32_t p;
    uint64_t hash_seed;
    uint8_t* registers_out;       /* out or NULL */
    double* estimate_out;         /* out or NULL */
    const gace_join* join;        /* JOIN */
    gace_join_result* join_out;   /* out */
} gace_request;

/*
 * Runs n requests as one batch: every request is compiled into jobs, each job
 * split into row chunks, and one persistent kernel per dependency phase (join
 * histograms before the sums that read them) drains the chunks from a device
 * work queue.  The upload of the compiled batch, the clearing of its
 * counters, the phase launches and the read-back form one CUDA graph that is
 * replayed while batches keep the same shape.  Chunk size and grid come from
 * the context's tuning table (gace_tune_batch), else defaults, and so does the
 * rule by which probes on one table are fused.  A batch of 64 or more
 * requests is planned, and its results assembled, on a few host threads of
 * the context.  With kernel timing on (gace_stats_reset), the host phases
 * (host_batch_resident, _compile, _build, _run, _finish) are added to the
 * statistics, launches = calls and total_ms = wall time.  Results are
 * identical to the synchronous calls'.  statuses (out, n entries, may be NULL)
 * receives each request's status; the return value is GACE_OK when every
 * request succeeded, else the first failing request's status.
 */
gace_status gace_run_batch(gace_ctx* ctx, const gace_request* reqs, uint32_t n, gace_status* statuses);

/*
 * Autotuner: runs the batch under each of four fusion rules (probes on one
 * table fused only when they share their row sets and columns and are not
 * single predicates on one row set; single predicates fused too; groups that
 * take the union of their members' row sets and columns; single predicates
 * fused only on a shared row sample, with the union of their columns), each
 * with every
 * candidate chunk size (128K..8M rows) and grid (1, 2 or the maximum of CTAs
 * per SM), times every candidate with CUDA events (and each rule's planning
 * of the batch on the host), and records the fastest (planning plus device
 * time):
 * the fusion rule for batches of this request shape (requests and the rows of
 * the tables they read, each bucketed by powers of two), chunk and grid for
 * batches of the compiled shape (jobs and rows).  Results are the same
 * integers under every rule.  Each rule's best device time is added to the
 * kernel statistics as tune_batch_fuse0..3, its planning time as
 * tune_batch_plan0..3.
 */
gace_status gace_tune_batch(gace_ctx* ctx, const gace_request* reqs, uint32_t n);

/* The tuning table as JSON lines (save) / merged from such a file (load). */
gace_status gace_tune_save(gace_ctx* ctx, const char* path);
gace_status gace_tune_load(gace_ctx* ctx, const char* path);

/* ------------------------------------------------------------ served form */

/*
 * Serving: requests arrive one by one (the Risky Gate's invocations while
 * queries are planned, Section III-A) and are answered with continuous
 * batching.  gace_submit copies a request's inputs, checks and compiles it
 * (as a batch would) and queues it.  A scheduler thread owns a device arena
 * for the state of requests in flight; a queued request is admitted, in
 * arrival order, once its state fits in the arena and fewer than
 * max_inflight requests are in flight (admission by memory).  Each
 * scheduling step is one persistent launch of the batch kernel over up to
 * step_rows units of chunks taken round-robin from every request in flight,
 * so a small probe that arrives while a long scan is on the GPU is answered
 * after the next step, not after the scan.  Steps are issued back to back,
 * two in flight, each with one upload, one scatter of the newly admitted
 * requests' inputs, the batch launch, one gather of the finished requests'
 * counters and one read-back.  A request completes when its last chunk has
 * run; its results are identical to the synchronous call's.  A request that
 * arrives at an idle server (nothing in flight, nothing else queued) is run
 * at once through its synchronous call on the context's stream: with nothing
 * to batch it with, a step would only add latency.  Results of
 * NDV requests are kept on the host as a sketch cache (LRU) that answers
 * later requests for the same table, column, p and seed at submission.
 * Probe results are cached the same way by bind value (Section V, item 3):
 * the count of every predicate, term and sample size a finished probe
 * returned is kept under (table, row set, the predicate's normalised terms in
 * canonical order), so a later probe whose every count is known (the same
 * predicates in another batch, order or spelling) is answered at submission
 * with the synchronous call's results.  Only small probes take part: at most
 * 256 (predicates + terms) x samples counts.  gace_unload forgets a table's
 * sketches and counts and fails with GACE_EBUSY while requests on that table
 * are queued or in flight.
 */
typedef struct {
    uint64_t arena_bytes;   /* device bytes for the state of requests in flight; 0 = 1 GiB */
    uint32_t max_inflight;  /* requests admitted at once; 0 = 4096 */
    int32_t sketch_cache;   /* NDV results kept for reuse (entries); 0 = 1024, < 0 = no cache */
    uint64_t step_rows;     /* units (rows) per scheduling step; 0 = 2^29 */
    uint64_t chunk_rows;    /* rows per chunk (at most 2^30), rounded up to a multiple of 128, and
                               for a narrow probe pass to a multiple of its tile; 0 = 2^18 */
    uint32_t flags;         /* GACE_SERVE_* */
    int32_t probe_cache;    /* probe counts kept for reuse (entries); 0 = 65536, < 0 = no cache */
    uint32_t idle_spin_us;  /* an idle scheduler watches its queue this long (yielding its
                               thread) before it sleeps, so that a request arriving meanwhile
                               does not wait out a thread wake-up; 0 = 10000 */
} gace_serve_config;

/* Never run a request alone through its synchronous call: every request goes
 * through the steps (tests of the batching machinery). */
#define GACE_SERVE_ALWAYS_STEP 1u
/* Fuse admitted one-predicate probes on one table that share a hashed row
 * sample (then one hash per row serves the group, with the union of their
 * columns), as the batched form's fusion rule 3 does; without it such probes
 * run alone.  Changes no result. */
#define GACE_SERVE_FUSE_SAMPLES 2u

/* Starts the scheduler (cfg may be NULL: defaults); its arena counts against
 * the context's HBM budget.  GACE_EBUSY when it is already running: stop it
 * first to change the configuration. */
gace_status gace_serve_start(gace_ctx* ctx, const gace_serve_config* cfg);

/* Stops the scheduler after every queued and in-flight request has finished,
 * and frees its arena.  A no-op when it is not running. */
gace_status gace_serve_stop(gace_ctx* ctx);

/* Queues a request and returns its ticket.  Its inputs are copied; its output
 * pointers must stay valid until gace_poll reports completion.  Argument
 * errors (the checks of the synchronous call) are returned here and no ticket
 * is made; GACE_ENOMEM when the request's state exceeds the whole arena.
 * Starts the scheduler with defaults when it is not running. */
gace_status gace_submit(gace_ctx* ctx, const gace_request* req, uint64_t* ticket_out);

/* Waits up to timeout_us for a request: GACE_OK when it has completed (its
 * outputs are written; the ticket is then forgotten), GACE_EPENDING if it has
 * not yet, its error status if it failed (also forgotten), GACE_ENOTFOUND for
 * an unknown ticket. */
gace_status gace_poll(gace_ctx* ctx, uint64_t ticket, uint64_t timeout_us);

/*
 * Open-loop load driver: submits reqs[i] at arrival_ns[i] (nanoseconds from
 * the start of the call, non-decreasing) from the calling thread and records
 * in done_ns[i] the time, on the same clock, at which its outputs were
 * written.  mode 0 goes through the served form (starting it with defaults
 * if needed); mode 1 is the plain path for comparison: one synchronous call
 * per request (gace_probe_batch, gace_ndv or gace_join_card), in arrival
 * order, each starting when both its arrival time and the previous call have
 * passed.  statuses (may be NULL) receives each request's status; the return
 * value is GACE_OK when every request succeeded, else the first failing
 * request's status.
 */
gace_status gace_serve_replay(gace_ctx* ctx, const gace_request* reqs, uint32_t n, const uint64_t* arrival_ns,
                              uint32_t mode, uint64_t* done_ns, gace_status* statuses);

/*
 * The plain path with its calls overlapped (the baseline a caller gets by
 * issuing synchronous probes from several threads): request i runs through
 * its synchronous call (gace_probe_batch, gace_ndv or gace_join_card) on
 * context ctxs[i % nctx]; each context's requests run in order on a host
 * thread of its own (the calling thread takes context 0), so calls on
 * different contexts, each on its own stream, overlap on the GPU.  The
 * table ids of request i must name tables registered on ctxs[i % nctx] (the
 * same borrowed columns may be registered on every context).  statuses (out,
 * n entries, may be NULL) receives each request's status; the return value is
 * GACE_OK when every request succeeded, else the first failing request's
 * status.  No context may be used by another thread during the call.
 */
gace_status gace_run_plain_async(gace_ctx* const* ctxs, uint32_t nctx, const gace_request* reqs, uint32_t n,
                                 gace_status* statuses);

/* ------------------------------------------------------------ Risky Gate */
/*
 * The trust metrics that decide whether a query goes to the GPU path
 * (Section III-A, III-C), evaluated on host doubles; no GPU is used.
 *
 *   drift D = |NDV_hist - NDV_est| / NDV_hist                 (Eq. 1), flagged
 *             when D >= drift_min (0.25 in the paper);
 *   selectivity error |S_est - S_probe|                       (Eq. 2), flagged
 *             when > sel_err_max (0.01);
 *   PCS = P(A,B) / (P(A) P(B))                                (Eq. 3), flagged
 *             when > pcs_high (1.6) or < pcs_low (0.7).
 *
 * A zero field of the config takes the paper's value; a NULL config takes all
 * four.  An input that is NaN leaves its signal out (its flag clear, its
 * output NaN); so does ndv_hist <= 0 or infinite (D is undefined), and a NaN
 * PCS (a zero marginal, gace_pred_result.pcs).  Errors: GACE_EINVAL for NULL
 * in/out with n > 0, or a threshold that is negative, NaN or infinite, or
 * pcs_low > pcs_high; outputs are then untouched.
 */
typedef struct {
    double drift_min;    /* 0 -> 0.25 */
    double sel_err_max;  /* 0 -> 0.01 */
    double pcs_high;     /* 0 -> 1.6 */
    double pcs_low;      /* 0 -> 0.7 */
} gace_gate_config;

typedef struct {
    double ndv_hist;   /* the optimizer's histogram NDV (NaN: no drift signal) */
    double ndv_est;    /* the measured NDV, e.g. gace_ndv's estimate */
    double sel_est;    /* the optimizer's selectivity (NaN: no selectivity signal) */
    double sel_probe;  /* the measured selectivity, gace_pred_result.sel */
    double pcs;        /* gace_pred_result.pcs of a 2-term predicate (NaN: none) */
} gace_gate_input;

#define GACE_RISK_DRIFT 1u
#define GACE_RISK_SELECTIVITY 2u
#define GACE_RISK_CORRELATION 4u

typedef struct {
    uint32_t flags;    /* OR of GACE_RISK_* */
    uint32_t reserved;
    double drift;      /* D, NaN when the signal is left out */
    double sel_err;    /* |S_est - S_probe|, NaN when left out */
} gace_gate_result;

gace_status gace_gate_eval(const gace_gate_config* cfg, const gace_gate_input* in, uint32_t n,
                           gace_gate_result* out);

/*
 * Break-even logic (Section V, item 2; Eq. 4 models the measurement cost as
 * the kernel time): predicted cost of one synchronous probe of npreds
 * predicates (K) on nsets row sets (M) over nrows rows (N), and whether it
 * beats the caller's alternative (alt_ms, e.g. the CPU's dynamic sampling).
 *
 *   batches of at most 32 predicates and 32 terms (narrow):
 *     kernel_ms = N * row_bytes / hbm_rate + N * hashed_sets * hash_ns
 *   larger batches (wide passes, ALU-bound):
 *     kernel_ms = N * ops_per_row / ops_rate
 *   transfer_ms = resident ? 0 : N * row_bytes / h2d_rate   (key-only copy)
 *   total_ms = call_ms + kernel_ms + transfer_ms;  offload = total_ms < alt_ms
 *
 * ops_per_row is the batch's compare operations per row (1 per equality, 2
 * per range, k per IN list of k values); 0 takes 2 per term.  The rates are
 * the context's own measurements: every probe launch timed while
 * gace_stats_reset(ctx, 1) is in effect adds to a cost table that
 * gace_stats_reset does not clear (narrow launches give hbm_rate, wide ones
 * ops_rate); a rate without measurements takes its GB300 default (hbm 5e12 B/s,
 * ops 1.3e13 /s, h2d 2e11 B/s, hash 1.5e-3 ns per row and set, call 0.03 ms).
 * The answer reports the rates it used.  Errors: GACE_EINVAL for NULL
 * arguments, nsets = 0, hashed_sets > nsets, or a NaN / negative alt_ms.
 */
typedef struct {
    uint64_t nrows;        /* N */
    uint32_t npreds;       /* K */
    uint32_t nsets;        /* M: row sets (full scan and samples) */
    uint32_t hashed_sets;  /* of which row or block samples (hashed per row) */
    uint32_t nterms;       /* distinct terms of the batch */
    uint32_t row_bytes;    /* bytes per row of the referenced columns */
    uint32_t resident;     /* 1: columns in HBM; 0: copied from host per probe */
    double ops_per_row;    /* 0: 2 * nterms */
    double alt_ms;         /* the alternative's cost */
} gace_cost_query;

typedef struct {
    double total_ms;
    double kernel_ms;
    double transfer_ms;
    double call_ms;
    double hbm_rate;       /* bytes/s */
    double ops_rate;       /* compare ops/s */
    double h2d_rate;       /* bytes/s */
    double hash_ns;        /* per row and hashed set */
    uint32_t narrow;       /* 1: the narrow kernels' model was used */
    uint32_t offload;      /* 1: total_ms < alt_ms */
    uint32_t measured;     /* bit 0: hbm_rate measured, bit 1: ops_rate measured */
    uint32_t reserved;
} gace_cost_answer;

gace_status gace_break_even(gace_ctx* ctx, const gace_cost_query* q, gace_cost_answer* out);

/*
 * Failure detection without a fault: launches one kernel whose single
 * device-side wait (an mbarrier phase that nothing completes) uses the same
 * bounded wait as every pipeline, with a limit of timeout_us (1..10^7) instead
 * of the context's.  Returns GACE_ETIMEDOUT when the wait gave up, set its
 * status and returned, as it must; the context stays usable afterwards.
 * GACE_EINVAL for a timeout outside its range; GACE_ECUDA if the wait did not
 * give up.
 */
gace_status gace_check_wait_limit(gace_ctx* ctx, uint32_t timeout_us);

/*
 * Roofline calibration (a measurement of the GPU; the paper has no counterpart):
 * the rate at which this GPU retires simple 32-bit integer operations, the
 * denominator of the integer-bound probe kernels' roofline.
 *   kind 0  independent chains of alternating 32-bit xor and add (two
 *           operations per step that no single instruction fuses): integer
 *           lane operations per second;
 *   kind 1  32-bit range tests (x - lo) <= span whose outcomes are added to
 *           counts, one operation per test: the best rate of the simplest
 *           term evaluation.
 * Every SM runs as many 256-thread CTAs as fit; the launch is grown until it
 * lasts about ms milliseconds (1..1000), then timed three times with CUDA
 * events on the context stream; *ops_per_s receives the best.  GACE_EINVAL for
 * another kind, ms outside its range or a NULL output.
 */
gace_status gace_calibrate_int(gace_ctx* ctx, uint32_t kind, uint32_t ms, double* ops_per_s);

/*
 * Kernel statistics of a context (tracing; the paper decomposes probe time
 * into transfer, kernel and reduction phases, Section IV-B).  Every launch is
 * counted with the algorithmic work it was given: rows scanned, bytes of the
 * referenced columns (the key-only bytes a scan must read), and compare
 * operations (per row: 1 for an equality, 2 for a range, k for an IN list of
 * k values, 1 per hashed key or histogram update).  When time_kernels is set,
 * each launch is also bracketed by CUDA events on the context stream and its
 * device time accumulated.  The served form adds "serve_step" (its batch
 * launches, timed on the scheduler's stream), "serve_copy" (scatter and
 * gather launches) and four entries that split the latency of completed
 * requests, with launches = requests and total_ms = the summed wall time:
 * serve_req_queue (submission to admission), serve_req_run (admission to the
 * step with the request's last chunk), serve_req_gpu (that step's enqueue to
 * the scheduler seeing it complete, or the synchronous call of a request run
 * alone), serve_req_finish (outputs assembled and the ticket completed); and
 * "serve_alone", whose launches count the requests an idle server ran
 * through their synchronous call.
 */
typedef struct {
    char name[24];      /* kernel family, NUL-terminated */
    uint64_t launches;
    uint64_t rows;
    uint64_t bytes;
    uint64_t ops;
    double total_ms;    /* 0 unless timing was enabled */
} gace_kernel_stat;

/* Clears the statistics; time_kernels = 1 turns event timing on. */
gace_status gace_stats_reset(gace_ctx* ctx, uint32_t time_kernels);

/* Copies up to cap entries (one per kernel family seen) into out; *n_out is
 * the number of families.  Waits for the context stream first. */
gace_status gace_stats_read(gace_ctx* ctx, gace_kernel_stat* out, uint32_t cap, uint32_t* n_out);

/* Message of the last failing call on this thread ("" if none). */
const char* gace_last_error(void);

/* Name of a status code. */
const char* gace_status_string(gace_status s);

/* GACE_ABI_VERSION of the loaded library; needs no GPU. */
uint32_t gace_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GACE_H */
