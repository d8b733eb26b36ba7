/*
 * gace_oracle.h -- plain, single-threaded CPU oracle for the GACE probe path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no header, helper or constant table with the
 * CUDA library; the two meet only through the seeded input generators.
 *
 * Every function states the passage of the paper (Chang, "Risk-Aware
 * GPU-Assisted Cardinality Estimation for Cost-Based Query Optimizers",
 * arXiv 2512.19750) or the published algorithm it follows.  Each is written as
 * the plain definition: loops over rows, no blocking, no reordering.
 */
#ifndef GACE_ORACLE_H
#define GACE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* column element types */
enum { ORC_I32 = 0, ORC_I64 = 1, ORC_F32 = 2 };
/* term operators: x == a ; a <= x < b ; x in {values} */
enum { ORC_EQ = 0, ORC_RANGE = 1, ORC_IN = 2 };
/* row sets a probe counts over */
enum { ORC_FULL = 0, ORC_ROWS = 1, ORC_BLOCKS = 2 };
/* return codes (numerically equal to the library's, but defined here) */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_EOVERFLOW = 7 };

typedef struct {
    int32_t dtype;      /* ORC_I32 / ORC_I64 / ORC_F32 */
    int32_t pad;
    const void* data;   /* host array of nrows elements */
} orc_column;

/* One term.  Integer columns read ia/ib and in_i; float columns read fa/fb and
 * in_f.  IN lists are in_{i,f}[in_off .. in_off + in_len). */
typedef struct {
    uint32_t col;
    uint32_t op;
    int64_t ia, ib;
    double fa, fb;
    uint32_t in_off, in_len;
} orc_term;

typedef struct {
    uint32_t kind;        /* ORC_FULL / ORC_ROWS / ORC_BLOCKS */
    uint32_t pad;
    uint64_t block_rows;  /* ORC_BLOCKS: rows per block (>= 1) */
    double rate;          /* ORC_ROWS / ORC_BLOCKS: sampling rate */
    uint64_t seed;
} orc_sample;

/* splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014). */
uint64_t orc_splitmix64(uint64_t x);
/* H(x, seed) = splitmix64(x XOR splitmix64(seed)). */
uint64_t orc_hash(uint64_t x, uint64_t seed);
/* Sampling threshold: returns 0 (keep none), 1 (keep all) or 2 (compare with *t). */
int orc_threshold(double rate, uint64_t* t);
/* 1 if row `row` belongs to the sample, else 0. */
int orc_row_in_sample(const orc_sample* s, uint64_t row);

/* Measurement Engine probe of candidate conditions (Section III-B; the
 * Key-Only + Bitmask evaluation of Experiment D).  Predicate p is the
 * conjunction of terms[pred_off[p] .. pred_off[p+1]).
 * Outputs: *n_sample = rows in the sample; counts[p] = sample rows matching p;
 * marginals[t] (optional, may be NULL) = sample rows matching term t alone. */
int orc_probe(uint64_t nrows, const orc_column* cols, uint32_t ncols,
              const orc_sample* sample,
              const orc_term* terms, uint32_t nterms,
              const int64_t* in_i, const double* in_f, uint32_t nin,
              const uint32_t* pred_off, uint32_t npreds,
              uint64_t* n_sample, uint64_t* counts, uint64_t* marginals);

/* Selectivity estimate count / n (0 when n == 0). */
double orc_selectivity(uint64_t count, uint64_t n);
/* PCS = P(A,B) / (P(A) P(B)) (Section III-C, Eq. 3) on one row set of n rows. */
double orc_pcs(uint64_t c_ab, uint64_t c_a, uint64_t c_b, uint64_t n);

/* HyperLogLog registers (Flajolet, Fusy, Gandouet, Meunier, AofA 2007) with a
 * 64-bit hash.  regs has 2^p entries and is overwritten. */
int orc_hll_registers(uint64_t nrows, const orc_column* col, uint32_t p,
                      uint64_t seed, uint8_t* regs);
/* Raw HyperLogLog estimate with the small-range (linear counting) rule. */
double orc_hll_estimate(const uint8_t* regs, uint32_t p);
/* Exact number of distinct values (float: -0 == +0, all NaNs one value). */
uint64_t orc_ndv_exact(uint64_t nrows, const orc_column* col);

/* One side of a join: a table, its join-key column and a conjunctive filter. */
typedef struct {
    uint64_t nrows;
    const orc_column* cols;
    uint32_t ncols;
    uint32_t key_col;
    const orc_term* terms;
    uint32_t nterms;
    uint32_t pad;
    const int64_t* in_i;
    const double* in_f;
} orc_side;

/* |sigma_f(F) JOIN_{F.fk = D.key} sigma_g(D)| (Section IV-F, join workload). */
int orc_join_card(const orc_side* fact, const orc_side* dim, uint64_t key_domain,
                  int64_t* card, uint64_t* fact_pass, uint64_t* dim_pass);
/* |sigma(F) JOIN sigma(D1) JOIN sigma(D2)| on F.fk = D1.key, D1.fk2 = D2.key. */
int orc_chain_card(const orc_side* fact, const orc_side* dim1, uint32_t dim1_fk2_col,
                   const orc_side* dim2, uint64_t key_domain1, uint64_t key_domain2,
                   int64_t* card, uint64_t* fact_pass, uint64_t* dim1_pass,
                   uint64_t* dim2_pass);

#ifdef __cplusplus
}
#endif
#endif
