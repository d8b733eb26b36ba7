/*
 * gace_oracle.c -- plain, single-threaded CPU oracle for the GACE probe path.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline of the benchmark; never by the product path.  It shares no code with
 * the CUDA library.  Each function is the plain definition of what the probe
 * computes, written as loops over rows in the order the definition states.
 *
 * Paper: I.-S. Chang, "Risk-Aware GPU-Assisted Cardinality Estimation for
 * Cost-Based Query Optimizers", arXiv 2512.19750.
 *   - Section III-B: the Measurement Engine measures the selectivity of
 *     candidate conditions by full scans, sampling or block-level summaries.
 *   - Section III-C, Eq. 3: PCS = P(A,B) / (P(A) P(B)).
 *   - Section IV-H (Experiment D): candidate conditions evaluated row by row
 *     ("Key-Only + Bitmask").
 *   - Section IV-F (join workload): join cardinality is the measured quantity.
 * The paper names no sampler, no sketch and no join formula; the readings used
 * here (splitmix64 sampling, HyperLogLog, histogram dot product) are stated
 * next to each function.
 */
#include "gace_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- hashing */

/* splitmix64 output function, as published by Steele, Lea & Flood,
 * "Fast Splittable Pseudorandom Number Generators", OOPSLA 2014: add the
 * golden-ratio increment, then two xor-shift-multiply rounds and a final
 * xor-shift, all modulo 2^64. */
uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* H(x, seed) = splitmix64(x XOR splitmix64(seed)): the counter-based hash of
 * a row id, block id or canonical value under a seed. */
uint64_t orc_hash(uint64_t x, uint64_t seed) {
    return orc_splitmix64(x ^ orc_splitmix64(seed));
}

/* ---------------------------------------------------------------- sampling */

/* Threshold T(r) of a Bernoulli sample of rate r: an element whose hash h
 * satisfies h < T is kept.  T = floor(r * 2^64), computed exactly as
 * ldexp(r, 64) truncated; r <= 0 (or NaN) keeps nothing and r >= 1 keeps
 * everything (T would be 2^64, which does not fit). */
int orc_threshold(double rate, uint64_t* t) {
    if (!(rate > 0.0)) {
        *t = 0;
        return 0;
    }
    if (rate >= 1.0) {
        *t = UINT64_MAX;
        return 1;
    }
    *t = (uint64_t)ldexp(rate, 64);
    return 2;
}

/* Row sample: row i kept iff H(i, seed) < T(r).
 * Block sample: block b = floor(i / B) kept iff H(b, seed) < T(r), and then
 * every row of the block is kept (dynamic sampling at row or block level,
 * Section II-A item 5 and Section III-B). */
int orc_row_in_sample(const orc_sample* s, uint64_t row) {
    uint64_t t;
    int mode;
    if (s->kind == ORC_FULL) return 1;
    mode = orc_threshold(s->rate, &t);
    if (mode == 0) return 0;
    if (mode == 1) return 1;
    if (s->kind == ORC_ROWS) return orc_hash(row, s->seed) < t;
    return orc_hash(row / s->block_rows, s->seed) < t;
}

/* ---------------------------------------------------------------- terms */

static int64_t int_value(const orc_column* c, uint64_t row) {
    if (c->dtype == ORC_I32) return (int64_t)((const int32_t*)c->data)[row];
    return ((const int64_t*)c->data)[row];
}

static double float_value(const orc_column* c, uint64_t row) {
    return (double)((const float*)c->data)[row];
}

/* A term on one column (the candidate conditions of Section III-B):
 *   EQ:    x == a
 *   RANGE: a <= x < b           (half-open)
 *   IN:    x equals one of the listed values
 * Integer columns compare exact integers; float columns compare the float
 * value, widened to double, with the double constants under IEEE rules, so a
 * NaN matches nothing and -0 equals +0. */
static int term_holds(const orc_column* cols, const orc_term* t,
                      const int64_t* in_i, const double* in_f, uint64_t row) {
    const orc_column* c = &cols[t->col];
    uint32_t k;
    if (c->dtype == ORC_F32) {
        double x = float_value(c, row);
        if (t->op == ORC_EQ) return x == t->fa;
        if (t->op == ORC_RANGE) return t->fa <= x && x < t->fb;
        for (k = 0; k < t->in_len; k++)
            if (x == in_f[t->in_off + k]) return 1;
        return 0;
    } else {
        int64_t x = int_value(c, row);
        if (t->op == ORC_EQ) return x == t->ia;
        if (t->op == ORC_RANGE) return t->ia <= x && x < t->ib;
        for (k = 0; k < t->in_len; k++)
            if (x == in_i[t->in_off + k]) return 1;
        return 0;
    }
}

static int check_terms(const orc_column* cols, uint32_t ncols, const orc_term* terms,
                       uint32_t nterms, uint32_t nin) {
    uint32_t i;
    for (i = 0; i < nterms; i++) {
        if (terms[i].col >= ncols) return ORC_EINVAL;
        if (terms[i].op > ORC_IN) return ORC_EINVAL;
        if (cols[terms[i].col].dtype < ORC_I32 || cols[terms[i].col].dtype > ORC_F32)
            return ORC_EINVAL;
        if (terms[i].op == ORC_IN &&
            (uint64_t)terms[i].in_off + terms[i].in_len > nin)
            return ORC_EINVAL;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- probe */

/* count[p] = #{ rows i in the sample : every term of predicate p holds on i }
 * marginal[t] = #{ rows i in the sample : term t holds on i }
 * n_sample = #{ rows i in the sample }.
 * A predicate with no terms matches every sampled row. */
int orc_probe(uint64_t nrows, const orc_column* cols, uint32_t ncols,
              const orc_sample* sample,
              const orc_term* terms, uint32_t nterms,
              const int64_t* in_i, const double* in_f, uint32_t nin,
              const uint32_t* pred_off, uint32_t npreds,
              uint64_t* n_sample, uint64_t* counts, uint64_t* marginals) {
    uint64_t row, ns = 0;
    uint32_t p, t;
    unsigned char* holds;
    int rc = check_terms(cols, ncols, terms, nterms, nin);
    if (rc != ORC_OK) return rc;
    if (sample->kind > ORC_BLOCKS) return ORC_EINVAL;
    if (sample->kind == ORC_BLOCKS && sample->block_rows == 0) return ORC_EINVAL;
    for (p = 0; p < npreds; p++)
        if (pred_off[p] > pred_off[p + 1] || pred_off[p + 1] > nterms) return ORC_EINVAL;

    holds = (unsigned char*)malloc(nterms ? nterms : 1);
    if (!holds) return ORC_EINVAL;
    for (p = 0; p < npreds; p++) counts[p] = 0;
    if (marginals)
        for (t = 0; t < nterms; t++) marginals[t] = 0;

    for (row = 0; row < nrows; row++) {
        if (!orc_row_in_sample(sample, row)) continue;
        ns++;
        for (t = 0; t < nterms; t++) holds[t] = (unsigned char)term_holds(cols, &terms[t], in_i, in_f, row);
        for (p = 0; p < npreds; p++) {
            int all = 1;
            for (t = pred_off[p]; t < pred_off[p + 1]; t++)
                if (!holds[t]) { all = 0; break; }
            counts[p] += (uint64_t)all;
        }
        if (marginals)
            for (t = 0; t < nterms; t++) marginals[t] += holds[t];
    }
    *n_sample = ns;
    free(holds);
    return ORC_OK;
}

/* Selectivity of a condition on a row set: matching rows / rows in the set
 * (the S_probe of Section III-C, Eq. 2).  An empty set yields 0. */
double orc_selectivity(uint64_t count, uint64_t n) {
    if (n == 0) return 0.0;
    return (double)count / (double)n;
}

/* PCS = P(A,B) / (P(A) P(B)) with P(X) = c_X / n on one row set
 * (Section III-C, Eq. 3), written as (c_AB * n) / (c_A * c_B).  Undefined
 * (NaN) when either marginal count is zero. */
double orc_pcs(uint64_t c_ab, uint64_t c_a, uint64_t c_b, uint64_t n) {
    if (c_a == 0 || c_b == 0) return NAN;
    return ((double)c_ab * (double)n) / ((double)c_a * (double)c_b);
}

/* ---------------------------------------------------------------- HyperLogLog */

/* Canonical 64-bit key of a value: int32 sign-extended, int64 as is, float32
 * by its bit pattern zero-extended after mapping -0 to +0 and every NaN to
 * the one pattern 0x7FC00000, so that values equal under the column's
 * equality hash equally. */
static uint64_t canonical_key(const orc_column* c, uint64_t row) {
    if (c->dtype == ORC_I32) return (uint64_t)(int64_t)((const int32_t*)c->data)[row];
    if (c->dtype == ORC_I64) return (uint64_t)((const int64_t*)c->data)[row];
    {
        float x = ((const float*)c->data)[row];
        uint32_t bits;
        if (x == 0.0f) return 0;
        if (x != x) return 0x7FC00000ULL;
        memcpy(&bits, &x, 4);
        return (uint64_t)bits;
    }
}

/* HyperLogLog (Flajolet et al. 2007) with the 64-bit hash h = H(key, seed):
 * the register index j is the top p bits of h, w is the remaining 64 - p
 * bits, and rho(w) is the 1-based position of the leftmost 1-bit of w
 * (64 - p + 1 when w is all zeros).  M[j] = max over all values of rho. */
int orc_hll_registers(uint64_t nrows, const orc_column* col, uint32_t p,
                      uint64_t seed, uint8_t* regs) {
    uint64_t row, m;
    if (p < 4 || p > 18) return ORC_EINVAL;
    if (col->dtype < ORC_I32 || col->dtype > ORC_F32) return ORC_EINVAL;
    m = 1ULL << p;
    memset(regs, 0, m);
    for (row = 0; row < nrows; row++) {
        uint64_t h = orc_hash(canonical_key(col, row), seed);
        uint64_t j = h >> (64 - p);
        uint64_t w = h << p;
        uint32_t rho;
        if (w == 0) {
            rho = 64 - p + 1;
        } else {
            uint64_t bit = 1ULL << 63;
            rho = 1;
            while ((w & bit) == 0) {
                rho++;
                bit >>= 1;
            }
        }
        if (rho > regs[j]) regs[j] = (uint8_t)rho;
    }
    return ORC_OK;
}

/* Raw HyperLogLog estimate E = alpha_m * m^2 / Z with Z = sum_j 2^-M[j]
 * (Flajolet et al. 2007, Fig. 3).  alpha_m takes the published constants
 * 0.673, 0.697, 0.709 for m = 16, 32, 64 and 0.7213 / (1 + 1.079/m) above.
 * Z is summed through the histogram c[k] = #{j : M[j] = k} in ascending k so
 * that the result does not depend on register order.  Small-range rule: if
 * E <= 5m/2 and V = c[0] > 0, E = m ln(m / V) (linear counting).  The hash
 * has 64 bits, so the paper's large-range correction for 32-bit hashes does
 * not apply. */
double orc_hll_estimate(const uint8_t* regs, uint32_t p) {
    uint64_t m = 1ULL << p, j;
    uint64_t c[66];
    double alpha, z = 0.0, e, dm = (double)m;
    uint32_t k;
    memset(c, 0, sizeof(c));
    for (j = 0; j < m; j++) c[regs[j] < 65 ? regs[j] : 65]++;
    if (m == 16) alpha = 0.673;
    else if (m == 32) alpha = 0.697;
    else if (m == 64) alpha = 0.709;
    else alpha = 0.7213 / (1.0 + 1.079 / dm);
    for (k = 0; k <= 65; k++) z += (double)c[k] * ldexp(1.0, -(int)k);
    e = alpha * dm * dm / z;
    if (e <= 2.5 * dm && c[0] > 0) e = dm * log(dm / (double)c[0]);
    return e;
}

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

/* Exact NDV: sort the canonical keys and count the distinct ones. */
uint64_t orc_ndv_exact(uint64_t nrows, const orc_column* col) {
    uint64_t* keys, row, ndv = 0;
    if (nrows == 0) return 0;
    keys = (uint64_t*)malloc(nrows * sizeof(uint64_t));
    if (!keys) return 0;
    for (row = 0; row < nrows; row++) keys[row] = canonical_key(col, row);
    qsort(keys, nrows, sizeof(uint64_t), cmp_u64);
    for (row = 0; row < nrows; row++)
        if (row == 0 || keys[row] != keys[row - 1]) ndv++;
    free(keys);
    return ndv;
}

/* ---------------------------------------------------------------- joins */

static int side_passes(const orc_side* s, uint64_t row) {
    uint32_t t;
    for (t = 0; t < s->nterms; t++)
        if (!term_holds(s->cols, &s->terms[t], s->in_i, s->in_f, row)) return 0;
    return 1;
}

static int side_check(const orc_side* s) {
    uint32_t t;
    if (s->key_col >= s->ncols) return ORC_EINVAL;
    if (s->cols[s->key_col].dtype == ORC_F32) return ORC_EINVAL;
    for (t = 0; t < s->nterms; t++) {
        if (s->terms[t].col >= s->ncols || s->terms[t].op > ORC_IN) return ORC_EINVAL;
    }
    return ORC_OK;
}

/* h[k] = #{ rows of the side passing its filter whose key column equals k },
 * k in [0, domain).  A passing row whose key lies outside the domain is an
 * error when strict (a dimension key), else it is skipped (a foreign key that
 * cannot match any dimension key). */
static int build_hist(const orc_side* s, uint64_t domain, int strict, uint64_t* h,
                      uint64_t* pass) {
    uint64_t row, np = 0;
    for (row = 0; row < s->nrows; row++) {
        int64_t k;
        if (!side_passes(s, row)) continue;
        np++;
        k = int_value(&s->cols[s->key_col], row);
        if (k < 0 || (uint64_t)k >= domain) {
            if (strict) return ORC_EINVAL;
            continue;
        }
        h[k]++;
    }
    *pass = np;
    return ORC_OK;
}

static uint64_t max_of(const uint64_t* h, uint64_t n) {
    uint64_t i, mx = 0;
    for (i = 0; i < n; i++)
        if (h[i] > mx) mx = h[i];
    return mx;
}

/* Join cardinality |sigma_f(F) JOIN_{F.fk = D.key} sigma_g(D)| as the dot
 * product of the two filtered key-frequency histograms,
 * J = sum_k h_F[k] * h_D[k], over the key domain [0, key_domain).
 * Overflow rule: EOVERFLOW when fact_pass * max_k h_D[k] >= 2^63. */
int orc_join_card(const orc_side* fact, const orc_side* dim, uint64_t key_domain,
                  int64_t* card, uint64_t* fact_pass, uint64_t* dim_pass) {
    uint64_t *hf, *hd, k, sum = 0;
    int rc;
    if (side_check(fact) != ORC_OK || side_check(dim) != ORC_OK) return ORC_EINVAL;
    if (key_domain == 0) return ORC_EINVAL;
    hf = (uint64_t*)calloc(key_domain, sizeof(uint64_t));
    hd = (uint64_t*)calloc(key_domain, sizeof(uint64_t));
    if (!hf || !hd) {
        free(hf);
        free(hd);
        return ORC_EINVAL;
    }
    rc = build_hist(fact, key_domain, 0, hf, fact_pass);
    if (rc == ORC_OK) rc = build_hist(dim, key_domain, 1, hd, dim_pass);
    if (rc == ORC_OK &&
        (unsigned __int128)(*fact_pass) * max_of(hd, key_domain) >= ((unsigned __int128)1 << 63))
        rc = ORC_EOVERFLOW;
    if (rc == ORC_OK) {
        for (k = 0; k < key_domain; k++) sum += hf[k] * hd[k];
        *card = (int64_t)sum;
    }
    free(hf);
    free(hd);
    return rc;
}

/* Three-table chain F -> D1 -> D2 (snowflake reading of the chain join):
 * J3 = sum over rows r of sigma(F), rows d of sigma(D1) with d.key = r.fk,
 * rows e of sigma(D2) with e.key = d.fk2, of 1.  Grouped by the first key:
 * w[k1] = sum_{d in sigma(D1), d.key = k1} h_D2[d.fk2] and J3 = sum_k h_F[k] w[k].
 * Overflow rule: EOVERFLOW when dim1_pass * max h_D2 >= 2^63 or
 * fact_pass * max w >= 2^63. */
int orc_chain_card(const orc_side* fact, const orc_side* dim1, uint32_t dim1_fk2_col,
                   const orc_side* dim2, uint64_t key_domain1, uint64_t key_domain2,
                   int64_t* card, uint64_t* fact_pass, uint64_t* dim1_pass,
                   uint64_t* dim2_pass) {
    uint64_t *hf = NULL, *hd2 = NULL, *w = NULL, row, k, sum = 0, np1 = 0;
    int rc = ORC_OK;
    if (side_check(fact) != ORC_OK || side_check(dim1) != ORC_OK || side_check(dim2) != ORC_OK)
        return ORC_EINVAL;
    if (dim1_fk2_col >= dim1->ncols || dim1->cols[dim1_fk2_col].dtype == ORC_F32)
        return ORC_EINVAL;
    if (key_domain1 == 0 || key_domain2 == 0) return ORC_EINVAL;
    hf = (uint64_t*)calloc(key_domain1, sizeof(uint64_t));
    w = (uint64_t*)calloc(key_domain1, sizeof(uint64_t));
    hd2 = (uint64_t*)calloc(key_domain2, sizeof(uint64_t));
    if (!hf || !w || !hd2) rc = ORC_EINVAL;
    if (rc == ORC_OK) rc = build_hist(dim2, key_domain2, 1, hd2, dim2_pass);
    if (rc == ORC_OK) {
        for (row = 0; row < dim1->nrows; row++) {
            int64_t k1, k2;
            if (!side_passes(dim1, row)) continue;
            np1++;
            k1 = int_value(&dim1->cols[dim1->key_col], row);
            if (k1 < 0 || (uint64_t)k1 >= key_domain1) {
                rc = ORC_EINVAL;
                break;
            }
            k2 = int_value(&dim1->cols[dim1_fk2_col], row);
            if (k2 < 0 || (uint64_t)k2 >= key_domain2) continue;
            w[k1] += hd2[k2];
        }
        *dim1_pass = np1;
    }
    if (rc == ORC_OK &&
        (unsigned __int128)np1 * max_of(hd2, key_domain2) >= ((unsigned __int128)1 << 63))
        rc = ORC_EOVERFLOW;
    if (rc == ORC_OK) rc = build_hist(fact, key_domain1, 0, hf, fact_pass);
    if (rc == ORC_OK &&
        (unsigned __int128)(*fact_pass) * max_of(w, key_domain1) >= ((unsigned __int128)1 << 63))
        rc = ORC_EOVERFLOW;
    if (rc == ORC_OK) {
        for (k = 0; k < key_domain1; k++) sum += hf[k] * w[k];
        *card = (int64_t)sum;
    }
    free(hf);
    free(w);
    free(hd2);
    return rc;
}
