// gace_internal.h -- structures shared by the host runtime and the sm_103a
// kernels of libgace.  Not part of the public ABI (include/gace.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gace {

// ---------------------------------------------------------------- limits
constexpr int kProbeWarps = 8;                  // warps per probe CTA
constexpr int kRowsPerLane = 4;                 // consecutive rows per lane
constexpr int kSliceRows = 32 * kRowsPerLane;   // rows per warp step (128)
constexpr int kMaxSlots = 32;                   // distinct columns in one pass
constexpr int kMaxSets = 8;                     // row sets in one probe
constexpr int kMaxStages = 4;                   // bulk-copy pipeline depth
constexpr int kNarrowMax = 32;                  // narrow kernel: predicates and terms per pass
// Warps of the synchronous wide-pass CTA and its CTAs per SM (the shared-memory
// tables of a pass are read by every warp of its CTA; each warp keeps its own
// term masks).
#ifndef GACE_WIDE_WARPS
#define GACE_WIDE_WARPS 8
#endif
constexpr int kWideWarps = GACE_WIDE_WARPS;
// CTAs per SM the compiler must fit the wide kernel's registers to (0: no
// bound; at 8 warps its registers allow three CTAs unbounded, and a bound made
// it spill).
#ifndef GACE_WIDE_MINCTAS
#define GACE_WIDE_MINCTAS (GACE_WIDE_WARPS >= 16 ? 2 : 0)
#endif

// device status word bits (first error wins for the code, bits accumulate)
constexpr unsigned kStatusTimeout = 1u;         // an mbarrier wait gave up
constexpr unsigned kStatusKeyDomain = 2u;       // a dimension key outside its domain
constexpr unsigned kStatusCasLimit = 4u;        // a bounded CAS loop gave up

// ---------------------------------------------------------------- terms
// Normalised term kinds.  Every RANGE/EQ becomes an inclusive interval in the
// column's own domain; IN lists are deduplicated values of the column type.
enum TermKind : uint32_t {
    kRangeI32 = 0,  // (uint32)(x - a) <= b       a = lo, b = hi - lo
    kRangeI64 = 1,  // (uint64)(x - a) <= b
    kRangeF32 = 2,  // x >= a && x <= b            a, b float bit patterns
    kInI32 = 3,     // x in pool32[a .. a + b)
    kInI64 = 4,     // x in pool64 words [a .. a + 2b)
    kInF32 = 5,     // x == any float in pool32[a .. a + b)
    kFalse = 6      // matches nothing (host short-circuits it)
};

// 16-byte device term: 32-bit kinds read (a_lo, b_lo); 64-bit kinds read all.
struct DevTerm {
    uint32_t a_lo, b_lo, a_hi, b_hi;
};

// ---------------------------------------------------------------- probe
struct SlotDesc {
    const void* ptr;     // column base (device)
    uint32_t dtype;      // 0 i32, 1 i64, 2 f32
    uint32_t width;      // bytes per element
    uint32_t rbeg;       // range terms of this slot: [rbeg, rend)
    uint32_t rend;
    uint32_t iend;       // narrow passes: IN terms [rend, iend); wide passes: EQ and
                         // IN terms [rend, iend), looked up in the slot's hash tables
    uint32_t soff;       // byte offset of the slot's tile inside a stage buffer
    uint32_t toff;       // wide passes: pool word offset of the slot's hash tables
    uint32_t tlog;       // log2 of each table's capacity (entries)
    uint32_t ngroups;    // tables (groups of up to 32 EQ/IN terms)
    uint32_t roff;       // wide passes: pool word offset of the slot's range trees
    uint32_t rgroups;    // range trees (groups of up to 32 range terms)
    uint32_t rtree;      // range terms [rbeg, rbeg + rtree) by tree, the rest by compare
    uint32_t vm1, vm2;   // wide passes: the multipliers of the hash tables' two slot functions
    // Rank-coded ranges (wide passes of a synchronous call): every row's rank
    // among the column's range endpoints, written by k_probe_rank; the slot's
    // range terms [rbeg, rend) are then read as rgroups groups of 32, group g's
    // mask of local rank r at pool[roff + g * rstride + r], where a row's local
    // rank (among the endpoints of this slot's terms) is its rank among the
    // column's endpoints, mapped by the table at pool word (rmap & ~kRankMap16)
    // - 1, of bytes, or of 16-bit entries when rmap has kRankMap16 (rmap 0: no
    // map, the two ranks are the same).  Such a slot holds no EQ/IN terms of
    // its own: they take a second slot of the column, or the column is coded
    // with all its terms, each an interval list in [rbeg, rend).  It reads no
    // values.  nullptr: not coded.
    const uint16_t* rank;
    uint32_t rstride;    // words per group (the local endpoints + 1)
    uint32_t rmap;
};

// A wide pass's range terms of one column, 32 at a time, as an interval tree:
// the group's distinct interval endpoints (order-preserving unsigned keys,
// padded with the largest key to 127) in level order, then the 128 term masks
// indexed by the number of endpoints <= a key.  A row takes 7 comparisons and
// one mask load for the whole group.
constexpr int kTreeLevels = 7;
constexpr uint32_t kTreeNodes = 127;
constexpr uint32_t kTreeWords32 = 256;  // 127 keys, 1 pad, 128 masks
constexpr uint32_t kTreeWords64 = 384;  // 127 key pairs, 2 pad, 128 masks

// A wide pass's EQ and IN terms of one column, 32 at a time, as two-choice
// (cuckoo) hash tables of 2^tlog entries: every distinct value of the group's
// terms is stored once, with the mask of the group's terms that contain it,
// at one of its two candidate slots vs_slot(key, vm1) and vs_slot(key, vm2);
// an empty slot has mask 0.  A lookup reads both slots and ORs the masks of
// those whose key matches: two independent loads, whatever the occupancy.
// A 64-bit key folds to 32 bits as lo ^ rotl16(hi * m): the rotation keeps
// keys such as 2^31 and -2^63, whose words are 2^31 and 0 swapped, apart for
// every odd m (without it both would fold to 2^31 and share every slot).
// Host and device compute the slots with this one function.
#if defined(__CUDACC__)
__host__ __device__
#endif
inline uint32_t vs_slot(uint32_t lo, uint32_t hi, uint32_t m, uint32_t tlog) {
    const uint32_t h = hi * m;
    return ((lo ^ ((h << 16) | (h >> 16))) * m) >> (32 - tlog);
}

struct SetDesc {
    uint32_t kind;       // 0 full, 1 rows, 2 blocks
    uint32_t mode;       // 0 keep none, 1 keep all, 2 threshold
    uint64_t thresh;     // keep iff hash < thresh
    uint64_t seedhash;   // splitmix64(seed)
    uint64_t block_rows;
    int32_t block_shift; // log2(block_rows) when a power of two, else -1
    uint32_t share_prev; // 1: same hash input as the previous set (reuse it)
};

struct alignas(16) ProbeArgs {
    uint64_t nrows;
    uint64_t row0;          // table-global id of the first row scanned (rows are hashed by global id)
    uint64_t ntiles;        // ceil(nrows / tile_rows)
    uint64_t nstaged;       // tiles loaded by bulk copy (full tiles when staged)
    uint32_t tile_rows;     // multiple of kSliceRows * kProbeWarps (narrow kernel)
    uint32_t stage_bytes;   // bytes of one stage buffer (all slots)
    uint32_t nstages;
    uint32_t nslots, nsets, nterms, npreds, npool, npredterms;
    uint32_t want_marg;
    uint32_t narrow;        // 1: lane-owned counters, staged tiles; 0: wide batch kernel
    uint32_t skip_tiles;    // 1: every row set is a block sample; tiles with no sampled block are skipped
    uint32_t smem_bytes;
    uint32_t nwarps;        // warps of the CTA that runs the pass (per-warp mask buffers)
    uint32_t ranks_only;    // wide passes: every slot with range terms is rank-coded
    uint32_t pad_[2];
    // smem byte offsets
    uint32_t off_stage, off_terms, off_pool, off_poff, off_pterm, off_tm, off_keep,
        off_cnt, off_marg, off_ns;
    uint64_t timeout_ns;
    SlotDesc slots[kMaxSlots];
    SetDesc sets[kMaxSets];
    const DevTerm* terms;
    const uint32_t* pool;
    const uint32_t* pred_off;    // npreds + 1
    const uint32_t* pred_terms;
    const uint4* setmask;        // wide passes: row-set masks of every 128-row slice, [slice][nsets],
                                 // computed once for all passes of a call (nullptr: hashed per pass)
    unsigned long long* counts;  // [nsets][npreds]
    unsigned long long* marg;    // [nsets][nterms]
    unsigned long long* nsamp;   // [nsets]
    unsigned int* status;
};

#ifdef __CUDACC__
#define GACE_HD __host__ __device__
#else
#define GACE_HD
#endif

// Which evaluation a pass takes: 0 wide, 1 narrow on all rows, 2 narrow on
// one hashed set, 3 narrow on several sets with a hashed one, 4 single
// predicate on all rows, 5 single predicate on one hashed set.
GACE_HD inline int probe_variant(const ProbeArgs& a) {
    if (!a.narrow) return 0;
    bool hash = false;
    for (uint32_t q = 0; q < a.nsets; ++q)
        if (a.sets[q].mode == 2) hash = true;
    // the single evaluation ANDs every term of the pass: only when the one predicate uses them all
    if (a.npreds == 1 && a.nsets == 1 && a.npredterms == a.nterms) return hash ? 5 : 4;
    if (!hash) return 1;
    return a.nsets == 1 ? 2 : 3;
}

static_assert(sizeof(ProbeArgs) % 16 == 0, "ProbeArgs is copied in 16-byte words");

// Fills the smem layout fields of `a` (given counts) and returns total bytes.
uint32_t probe_layout(ProbeArgs& a);
cudaError_t probe_configure();  // one-time kernel attributes
cudaError_t probe_launch(const ProbeArgs& a, int grid, cudaStream_t s);
// Rank coding of one column for the wide passes of a call: out[r] = the number
// of the column's range endpoints <= the order-preserving key of row r (at most
// m), for rows [0, nout) (rows >= nrows get 0), from the endpoints' search tree
// (level order, 2^levels - 1 keys padded with the largest key; 32-bit keys, or
// (lo, hi) word pairs for 64-bit columns).  With hist, also the histogram of
// the ranks of each row set's rows, added to hist[q * (m + 1) + rank]: set q
// holds every row when bit q of full_sets is set, else the rows of each quad
// (rows 4 j .. 4 j + 3) whose bit 4 q + i is set in qmask[j].
struct RankArgs {
    const void* col;        // the column's first row of the range scanned
    uint64_t nrows;
    uint64_t nout;          // nrows rounded up to a multiple of 128
    const uint32_t* tree;
    uint16_t* out;             // nullptr: histograms only
    unsigned long long* hist;  // nullptr: no histograms
    const uint32_t* qmask;     // nullptr when every set holds every row
    uint32_t dtype;
    uint32_t levels;        // search tree: 1..13 levels; 0: bucket index
    uint32_t m;             // endpoints (<= 8191)
    uint32_t nsets;         // row sets of the histograms (<= kMaxSets)
    uint32_t full_sets;
    uint32_t words;         // 32-bit words at tree (staged in shared memory)
    // Bucket index (levels == 0): a key k >= base falls in bucket
    // ((s - smin) << mbits) + ((k - base) >> s), s = max(smin, bit length of
    // k - base - mbits - 1), at most nb - 1 (keys below base: bucket 0);
    // tree holds the nb 16-bit first-endpoint indices of the buckets in
    // rank_start_words(nb) words (whole 8-byte units), then the sorted
    // endpoints (words, or 8-byte aligned (lo, hi) pairs for int64) padded
    // with the largest key to m + 2^steps entries; the rank is the bucket's
    // first index plus `steps` halvings over those entries.
    uint64_t base;
    uint32_t nb, smin, mbits, steps;
};
// Words of a bucket index's first-endpoint indices: nb 16-bit entries
// rounded up to whole 8-byte units.
__host__ __device__ constexpr uint32_t rank_start_words(uint32_t nb) { return 2u * ((nb + 3u) / 4u); }
constexpr uint32_t kRankMaxEndpoints = 8191;
constexpr uint32_t kRankMap16 = 0x80000000u;  // SlotDesc::rmap: the map has 16-bit entries
cudaError_t rank_launch(const RankArgs& a, int sms, cudaStream_t s);
uint32_t rank_smem(const RankArgs& a);  // shared memory of a rank launch (bytes)

// The row-set masks of every 128-row slice of a pass's table into out, for
// the wide passes that follow to load instead of hashing, and (qmask not
// nullptr) each quad's membership word for the rank histograms.
cudaError_t setmask_launch(const ProbeArgs& a, uint4* out, uint32_t* qmask, int sms, cudaStream_t s);
int probe_occupancy(const ProbeArgs& a);  // CTAs per SM for this kernel and smem size

// ---------------------------------------------------------------- materialised samples
// A row or block sample compacted into its own columns (k_sample_count, then
// k_sample_scatter), in tiles of kSampleTileRows rows.
constexpr uint32_t kSampleTileRows = 4096;
constexpr int kMaxSampleCols = 64;

struct alignas(16) SampleArgs {
    uint64_t nrows;
    uint64_t ntiles;              // ceil(nrows / kSampleTileRows)
    SetDesc set;                  // kind 1 (rows) or 2 (blocks), mode 2 (threshold)
    uint32_t ncols;
    uint32_t pad;
    const void* src[kMaxSampleCols];
    void* dst[kMaxSampleCols];    // scatter only
    uint32_t width[kMaxSampleCols];
    uint32_t* tile_count;         // [ntiles], written by the count pass
    const uint64_t* tile_off;     // [ntiles], exclusive prefix sums (scatter)
};

cudaError_t sample_count_launch(const SampleArgs& a, int grid, cudaStream_t s);
cudaError_t sample_scatter_launch(const SampleArgs& a, int grid, cudaStream_t s);

// ---------------------------------------------------------------- HyperLogLog
struct HllArgs {
    const void* col;
    uint64_t nrows;
    uint32_t dtype;
    uint32_t p;
    uint64_t seedhash;
    uint32_t aligned;     // column base 16-byte aligned
    uint32_t* regs;       // 2^p uint32 (global, zeroed)
    unsigned int* status;
};
cudaError_t hll_launch(const HllArgs& a, int sms, cudaStream_t s);

// Raw HyperLogLog estimate (Flajolet, Fusy, Gandouet & Meunier, AofA 2007)
// from the histogram of register values: c[k] registers hold k, for
// k = 0..65 (64 - p + 1 <= 61 is the largest a register can hold).  The sum
// runs in ascending k, so the estimate depends only on the histogram, not on
// the order of the registers.  alpha_m = 0.673, 0.697, 0.709 for m = 16, 32,
// 64, else 0.7213 / (1 + 1.079 / m); the linear-counting estimate m ln(m / V)
// replaces E when E <= 2.5 m and V = c[0] > 0.  Every entry point that
// returns an estimate calls this one function, so their doubles agree bit for
// bit.
double hll_estimate_from_hist(const uint64_t (&c)[66], uint32_t p);

// Sets the thread-local message returned by gace_last_error().
void set_last_error_message(const char* msg);

// ---------------------------------------------------------------- joins
constexpr int kMaxFilterTerms = 64;
constexpr int kMaxFilterSlots = 8;

struct FilterTerm {
    uint32_t slot;
    uint32_t kind;
    DevTerm c;
};

struct alignas(16) SideArgs {
    uint64_t nrows;
    uint32_t nslots;
    uint32_t nterms;
    uint32_t npool;
    uint32_t key_slot;
    const void* slot_ptr[kMaxFilterSlots];
    uint32_t slot_dtype[kMaxFilterSlots];
    uint32_t slot_aligned[kMaxFilterSlots];
    FilterTerm terms[kMaxFilterTerms];
    const uint32_t* pool;    // device
    uint64_t domain;         // keys must lie in [0, domain)
    unsigned long long* pass_count;
    unsigned int* status;
    // Staged scans (stage_bytes > 0): tiles of tile_rows rows of every slot
    // pass through shared memory, slot s at byte slot_soff[s] of a stage
    // buffer; tiles below nstaged are bulk-copied, the rest read directly.
    uint64_t ntiles;
    uint64_t nstaged;
    uint32_t tile_rows;
    uint32_t stage_bytes;
    uint32_t nstages;
    uint32_t smem_bytes;     // dynamic shared memory of a staged launch
    uint32_t slot_width[kMaxFilterSlots];
    uint32_t slot_soff[kMaxFilterSlots];
    uint64_t timeout_ns;
};

static_assert(sizeof(SideArgs) % 16 == 0, "SideArgs is copied in 16-byte words");

// Rows of one warp step of a staged side scan (8 per lane) and its CTA shape.
constexpr uint32_t kSideSlice = 256;
constexpr int kSideWarps = 8;
constexpr uint32_t kSideStageOff = 128;  // stage buffers follow the mbarriers

// h[key] += 1 for filtered rows; strict: out-of-domain key sets kStatusKeyDomain
cudaError_t hist_launch(const SideArgs& a, uint32_t* hist, int strict, int aggregate,
                        int sms, cudaStream_t s);
// w[key] += h2[fk2] for filtered rows of dim1 (key checked strictly)
cudaError_t chain_weight_launch(const SideArgs& a, uint32_t fk2_slot, uint64_t domain2,
                                const uint32_t* h2, unsigned long long* w, int sms,
                                cudaStream_t s);
// sum over filtered rows of weight[key] (uint32 or uint64 weights)
cudaError_t gather_launch(const SideArgs& a, const void* weight, int weight64,
                          unsigned long long* sum, int sms, cudaStream_t s);
// sum_k a[k] * b[k]
cudaError_t dot_launch(const uint32_t* a, const void* b, int b64, uint64_t n,
                       unsigned long long* sum, int sms, cudaStream_t s);
// max_k a[k]
cudaError_t max_launch(const void* a, int a64, uint64_t n, unsigned long long* mx, int sms,
                       cudaStream_t s);

// ---------------------------------------------------------------- batch
// A batch is a set of jobs (one probe pass, one HLL sketch, one join side or
// histogram reduction each) cut into items of rows (or histogram elements)
// that a persistent kernel takes from a device work queue.
enum BatchJobKind : uint32_t {
    kJobProbe = 0,
    kJobHll = 1,
    kJobHist = 2,      // h[key] += 1 over filtered rows
    kJobHistAgg = 3,   // the same, equal keys of a warp combined first
    kJobGather32 = 4,  // out += h[key] over filtered rows
    kJobGather64 = 5,  // out += w[key]
    kJobChain = 6,     // w[key] += h2[fk2]
    kJobMax32 = 7,     // out = max h[i]
    kJobMax64 = 8,
    kJobDot32 = 9,     // out += a[i] * b32[i]
    kJobDot64 = 10     // out += a[i] * b64[i]
};

struct BatchJob {
    uint32_t kind;
    uint32_t strict;            // join histograms: key outside the domain is an error
    uint32_t fk2_slot;          // chain
    uint32_t pad;
    uint64_t domain2;           // chain
    const ProbeArgs* probe;     // kJobProbe (device copy, wide layout)
    const SideArgs* side;       // join sides (device copy)
    HllArgs hll;                // kJobHll
    uint32_t* hist;             // histogram built (Hist*), or a of a dot product
    const void* weight;         // weights read (gather, chain), b of a dot, input of a max
    unsigned long long* out;    // sum (gather, dot) or maximum
    unsigned long long* w64;    // chain weights
};

struct BatchItem {
    uint32_t job;
    uint32_t pad;
    uint64_t begin;             // rows (elements for max and dot); a multiple of 128
    uint64_t end;
};

// One 16-byte-granular copy (src == nullptr: zero fill) of the served form's
// scatter and gather launches; dst, src and bytes are multiples of 16.
struct CopyDesc {
    unsigned char* dst;
    const unsigned char* src;
    uint64_t bytes;
    uint64_t pad;
};

// Item classes, each drained by its own persistent kernel: narrow and
// single-predicate probe items (k_batch_probe), join histograms over small
// key domains counted in shared memory (k_batch_hist), join sides whose
// columns stream through the staged tile pipeline (k_batch_side), everything
// else (k_batch).
constexpr int kClassProbe = 0;
constexpr int kClassGeneral = 1;
constexpr int kClassHist = 2;
constexpr int kClassSide = 3;
constexpr int kClasses = 4;
constexpr int kPhases = 3;  // dependency phases of a batch (a join's histogram before its readers)

// Key domains up to this many entries are histogrammed per CTA in shared
// memory (hierarchical atomics: skewed keys do not serialise on one global
// address), the CTA's nonzero bins then added to the global histogram.
constexpr uint64_t kSmemHistMax = 1u << 15;
constexpr int kHistThreads = 1024;

cudaError_t batch_configure(int smem_optin);
int batch_occupancy(uint32_t smem_bytes, int cls);
cudaError_t batch_launch(const BatchItem* items, uint32_t nitems, const BatchJob* jobs, unsigned int* head,
                         int grid, uint32_t smem_bytes, int cls, cudaStream_t s);
cudaError_t copy_launch(const CopyDesc* descs, uint32_t n, int grid, cudaStream_t s);

// Roofline calibration kernel of the integer pipes (gace_calibrate_int).
cudaError_t int_peak_launch(int kind, uint32_t iters, int grid, uint32_t* sink, cudaStream_t s);
uint64_t int_peak_ops_per_iter(int kind);
int int_peak_occupancy(int kind);

}  // namespace gace
