/*
 * Oracle for sampled sub-block Toeplitz hashing (arXiv 2308.02856).
 *
 * TEST INFRASTRUCTURE ONLY (tests, the package smoke check and the benchmark's
 * CPU-baseline leg).  Plain C, one bit at a time; shares no code with the CUDA
 * library.  The definitions are stated in oracle.h; each function below cites
 * the passage of the paper it follows.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* Philox4x32-10, from its published definition (Salmon et al., SC'11):    */
/* a 4-word counter is passed through 10 rounds; each round multiplies     */
/* words 0 and 2 by fixed 32-bit constants, takes the 64-bit products      */
/* apart into high and low halves, and recombines them with words 1 and 3  */
/* and the round key; the 2-word key is advanced by the two Weyl constants */
/* between rounds.  The paper (Sec. IV) only says "a PRNG" decides the     */
/* sampling; Philox is the generator chosen for it here.                   */
/* ---------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ---------------------------------------------------------------------- */
/* Sampling (Sec. III.B step 1).  The paper draws an i.i.d. label per round */
/* and lets sub-block sizes vary; the reading used here gives each position */
/* a 64-bit Philox label and cuts the sorted order into equal sub-blocks.   */
/* ---------------------------------------------------------------------- */
uint64_t oracle_sampling_key(uint64_t i, uint64_t sampling_key, uint32_t flags)
{
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), 0u, 0u};
    uint32_t key[2] = {(uint32_t)sampling_key, (uint32_t)(sampling_key >> 32)};
    uint32_t x[4];
    oracle_philox4x32_10(ctr, key, x);
    uint64_t label = ((uint64_t)x[0] << 32) | (uint64_t)x[1];
    uint32_t kb = (flags >> 8) & 0x3fu;
    if (kb != 0u)
        label &= ~((1ull << (64u - kb)) - 1ull); /* keep the top kb bits */
    return label;
}

typedef struct {
    uint64_t lo, hi, sampling_key;
    uint32_t flags;
    uint64_t *keys;
} keys_job;

static void *keys_worker(void *arg)
{
    keys_job *job = (keys_job *)arg;
    for (uint64_t i = job->lo; i < job->hi; ++i)
        job->keys[i] = oracle_sampling_key(i, job->sampling_key, job->flags);
    return NULL;
}

void oracle_sampling_keys(uint64_t n, uint64_t sampling_key, uint32_t flags,
                          uint64_t *keys, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    pthread_t th[256];
    keys_job jobs[256];
    if (nthreads > 256) nthreads = 256;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].lo = n * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
        jobs[t].sampling_key = sampling_key;
        jobs[t].flags = flags;
        jobs[t].keys = keys;
        pthread_create(&th[t], NULL, keys_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t)
        pthread_join(th[t], NULL);
}

typedef struct {
    uint64_t key;
    uint32_t idx;
} keyed_pos;

/* Total order of the sampled positions: by label, then by position. */
static int keyed_pos_cmp(const void *a, const void *b)
{
    const keyed_pos *x = (const keyed_pos *)a, *y = (const keyed_pos *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

int oracle_perm(uint64_t n, const uint64_t *keys, uint32_t *perm)
{
    if (n > (1ull << 32)) return -1;
    keyed_pos *r = (keyed_pos *)malloc((size_t)(n ? n : 1) * sizeof(keyed_pos));
    if (!r) return -2;
    for (uint64_t i = 0; i < n; ++i) {
        r[i].key = keys[i];
        r[i].idx = (uint32_t)i;
    }
    qsort(r, (size_t)n, sizeof(keyed_pos), keyed_pos_cmp);
    for (uint64_t i = 0; i < n; ++i)
        perm[i] = r[i].idx;
    free(r);
    return 0;
}

int oracle_perm_range(uint64_t n, const uint64_t *keys, uint64_t lo, uint64_t cnt,
                      uint32_t *out)
{
    if (n > (1ull << 32) || lo + cnt > n) return -1;
    if (cnt == 0) return 0;
    /* rank of the first element of each 16-bit label bucket */
    uint64_t *start = (uint64_t *)calloc(65537, sizeof(uint64_t));
    if (!start) return -2;
    for (uint64_t i = 0; i < n; ++i)
        start[(keys[i] >> 48) + 1]++;
    for (int b = 0; b < 65536; ++b)
        start[b + 1] += start[b];
    /* buckets that hold ranks lo .. lo+cnt-1 */
    int blo = 0, bhi = 65535;
    while (start[blo + 1] <= lo) ++blo;
    while (start[bhi] >= lo + cnt) --bhi;
    uint64_t base = start[blo], m = start[bhi + 1] - start[blo];
    keyed_pos *r = (keyed_pos *)malloc((size_t)m * sizeof(keyed_pos));
    if (!r) { free(start); return -2; }
    uint64_t t = 0;
    for (uint64_t i = 0; i < n; ++i) {
        int b = (int)(keys[i] >> 48);
        if (b >= blo && b <= bhi) {
            r[t].key = keys[i];
            r[t].idx = (uint32_t)i;
            ++t;
        }
    }
    qsort(r, (size_t)m, sizeof(keyed_pos), keyed_pos_cmp);
    for (uint64_t q = 0; q < cnt; ++q)
        out[q] = r[lo - base + q].idx;
    free(r);
    free(start);
    return 0;
}

typedef struct {
    uint64_t n, lo, hi;
    const uint64_t *keys;
    const uint32_t *perm;
    int64_t bad;
} check_job;

static void *check_worker(void *arg)
{
    check_job *c = (check_job *)arg;
    c->bad = -1;
    for (uint64_t t = c->lo; t < c->hi; ++t) {
        if (c->perm[t] >= c->n) { c->bad = (int64_t)t; return NULL; }
        if (t + 1 < c->n) {
            uint32_t a = c->perm[t], b = c->perm[t + 1];
            if (b >= c->n) { c->bad = (int64_t)(t + 1); return NULL; }
            int ok = c->keys[a] < c->keys[b] || (c->keys[a] == c->keys[b] && a < b);
            if (!ok) { c->bad = (int64_t)t; return NULL; }
        }
    }
    return NULL;
}

int64_t oracle_check_order(uint64_t n, const uint64_t *keys, const uint32_t *perm, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    check_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].n = n; jobs[t].keys = keys; jobs[t].perm = perm;
        jobs[t].lo = n * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
        pthread_create(&th[t], NULL, check_worker, &jobs[t]);
    }
    int64_t bad = -1;
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].bad >= 0 && (bad < 0 || jobs[t].bad < bad)) bad = jobs[t].bad;
    }
    return bad;
}

/* ---------------------------------------------------------------------- */
/* Bits, sub-blocks and the Toeplitz product (Sec. I: K = T . A';           */
/* Sec. III.B steps 3-4).                                                  */
/* ---------------------------------------------------------------------- */
static inline uint8_t bit(const uint32_t *x, uint64_t i)
{
    return (uint8_t)((x[i >> 5] >> (i & 31u)) & 1u);
}

void oracle_subblock(const uint32_t *in, const uint32_t *pos, uint64_t s, uint8_t *A)
{
    for (uint64_t c = 0; c < s; ++c)
        A[c] = bit(in, pos[c]);
}

void oracle_subblock_padded(const uint32_t *in, const uint32_t *pos, uint64_t s, uint8_t *A)
{
    for (uint64_t c = 0; c < s; ++c)
        A[c] = pos[c] == ORACLE_NO_POS ? 0 : bit(in, pos[c]);
}

/* ---------------------------------------------------------------------- */
/* The paper's own sampling law (Sec. III.B step 1): every position draws  */
/* an i.i.d. uniform label V_i in [0, m) and S_j = {i : V_i = j}, so the   */
/* sub-block sizes are binomial.  V_i is the integer part of key_i m/2^64  */
/* for the 64-bit label key_i of definition 1.  A sub-block is the input   */
/* restricted to S_j in increasing position order (the order in which the  */
/* paper's hardware stores the sampled bits, Sec. IV), zero-padded to the  */
/* block size limit s = L_S^UB; the protocol aborts when some |S_j| > s    */
/* (Sec. III.D).                                                           */
/* ---------------------------------------------------------------------- */
uint32_t oracle_iid_label(uint64_t key, uint64_t m)
{
    return (uint32_t)(((unsigned __int128)key * m) >> 64);
}

uint64_t oracle_iid_order(uint64_t n, const uint64_t *keys, uint64_t m, uint64_t s,
                          uint64_t *sizes, uint32_t *order)
{
    memset(sizes, 0, (size_t)m * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; ++i)
        sizes[oracle_iid_label(keys[i], m)]++;
    uint64_t largest = 0;
    for (uint64_t j = 0; j < m; ++j)
        if (sizes[j] > largest) largest = sizes[j];
    if (largest > s || !order) return largest;
    for (uint64_t t = 0; t < m * s; ++t)
        order[t] = ORACLE_NO_POS;
    uint64_t *fill = (uint64_t *)calloc((size_t)m, sizeof(uint64_t));
    if (!fill) return UINT64_MAX;
    for (uint64_t i = 0; i < n; ++i) {  /* increasing positions */
        uint32_t j = oracle_iid_label(keys[i], m);
        order[(uint64_t)j * s + fill[j]++] = (uint32_t)i;
    }
    free(fill);
    return largest;
}

/* Eq. 7 (Sec. III.D): with H(x, p) = x ln(x/p) + (1-x) ln((1-x)/(1-p)) and
   Phi the standard normal CDF, the chance that one binomial(N, p) sub-block
   size exceeds L is at most 1 - Phi(sqrt(2 N H(L/N, p))) for L >= N p (the
   Zubkov-Serov bound); the limit is the smallest L at which m times that
   bound is at most eps.  For L < N p the bound's argument changes sign. */
static double binary_relative_entropy(double x, double p)
{
    double a = x > 0.0 ? x * log(x / p) : 0.0;
    double b = x < 1.0 ? (1.0 - x) * log((1.0 - x) / (1.0 - p)) : 0.0;
    return a + b;
}

double oracle_size_tail_bound(uint64_t N, uint64_t L, double p)
{
    double x = (double)L / (double)N;
    double z = sqrt(2.0 * (double)N * binary_relative_entropy(x, p));
    if (x < p) z = -z;
    return 0.5 * erfc(z / sqrt(2.0));  /* 1 - Phi(z) */
}

uint64_t oracle_block_limit(uint64_t N, uint64_t m, double eps, double p)
{
    if (N == 0 || m == 0 || !(p > 0.0 && p < 1.0) || !(eps > 0.0)) return N;
    double target = eps / (double)m;
    if (oracle_size_tail_bound(N, N, p) > target) return N;  /* no size can exceed N */
    uint64_t lo = 0, hi = N;  /* the bound fails at lo - 1 ... holds at hi */
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (oracle_size_tail_bound(N, mid, p) <= target) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

uint8_t oracle_toeplitz_bit(const uint32_t *seed, uint64_t off, uint64_t s,
                            const uint8_t *A, uint64_t i)
{
    uint8_t acc = 0;
    for (uint64_t c = 0; c < s; ++c) {
        uint8_t t_ic = bit(seed, off + i - c + s - 1); /* T[i][c] */
        acc ^= (uint8_t)(t_ic & A[c]);
    }
    return acc;
}

void oracle_toeplitz(const uint32_t *seed, uint64_t off, uint64_t s,
                     const uint8_t *A, uint64_t i0, uint64_t cnt, uint8_t *K)
{
    for (uint64_t i = i0; i < i0 + cnt; ++i)
        K[i - i0] = oracle_toeplitz_bit(seed, off, s, A, i);
}

typedef struct {
    const uint32_t *in, *pos, *seed;
    uint64_t s, k, j0, nj, i0, ni, jlo, jhi;
    uint32_t flags;
    uint8_t *out;
} window_job;

static void *window_worker(void *arg)
{
    window_job *w = (window_job *)arg;
    uint8_t *A = (uint8_t *)malloc((size_t)(w->s ? w->s : 1));
    if (!A) return (void *)1;
    for (uint64_t j = w->jlo; j < w->jhi; ++j) {
        if (w->flags & ORACLE_SAMPLING_IID)
            oracle_subblock_padded(w->in, w->pos + (j - w->j0) * w->s, w->s, A);
        else
            oracle_subblock(w->in, w->pos + (j - w->j0) * w->s, w->s, A);
        uint64_t off = (w->flags & ORACLE_SEED_PER_SUBBLOCK) ? j * (w->s + w->k - 1) : 0;
        oracle_toeplitz(w->seed, off, w->s, A, w->i0, w->ni, w->out + (j - w->j0) * w->ni);
    }
    free(A);
    return NULL;
}

static int run_window(const uint32_t *in, const uint32_t *pos, uint64_t s, uint64_t k,
                      const uint32_t *seed, uint32_t flags, uint64_t j0, uint64_t nj,
                      uint64_t i0, uint64_t ni, uint8_t *out, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((uint64_t)nthreads > nj) nthreads = (int)(nj ? nj : 1);
    pthread_t th[256];
    window_job jobs[256];
    int bad = 0;
    for (int t = 0; t < nthreads; ++t) {
        window_job *w = &jobs[t];
        w->in = in; w->pos = pos; w->seed = seed;
        w->s = s; w->k = k; w->j0 = j0; w->nj = nj; w->i0 = i0; w->ni = ni;
        w->jlo = j0 + nj * (uint64_t)t / (uint64_t)nthreads;
        w->jhi = j0 + nj * (uint64_t)(t + 1) / (uint64_t)nthreads;
        w->flags = flags;
        w->out = out;
        pthread_create(&th[t], NULL, window_worker, w);
    }
    for (int t = 0; t < nthreads; ++t) {
        void *ret = NULL;
        pthread_join(th[t], &ret);
        if (ret) bad = 1;
    }
    return bad ? -2 : 0;
}

void oracle_extract_window(const uint32_t *in, const uint32_t *pos, uint64_t s, uint64_t k,
                           const uint32_t *seed, uint32_t flags, uint64_t j0, uint64_t nj,
                           uint64_t i0, uint64_t ni, uint8_t *out, int nthreads)
{
    run_window(in, pos, s, k, seed, flags, j0, nj, i0, ni, out, nthreads);
}

int oracle_extract(uint64_t n, uint64_t m, uint64_t s, uint64_t k,
                   const uint32_t *in, const uint32_t *seed, uint64_t sampling_key,
                   uint32_t flags, uint32_t *out, int nthreads)
{
    const int iid = (flags & ORACLE_SAMPLING_IID) != 0;
    if (m < 1 || s < 1 || k < 1 || k > s || n > (1ull << 32)) return -1;
    if (iid ? (n >= (1ull << 32) || (flags & ORACLE_IDENTITY_PERM)) : m * s > n) return -1;
    uint32_t *perm = (uint32_t *)malloc((size_t)(iid ? m * s : n) * sizeof(uint32_t));
    uint8_t *K = (uint8_t *)malloc((size_t)(m * k));
    if (!perm || !K) { free(perm); free(K); return -2; }
    if (iid) {
        uint64_t *keys = (uint64_t *)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
        uint64_t *sizes = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
        if (!keys || !sizes) { free(keys); free(sizes); free(perm); free(K); return -2; }
        oracle_sampling_keys(n, sampling_key, flags, keys, nthreads);
        uint64_t largest = oracle_iid_order(n, keys, m, s, sizes, perm);
        free(keys);
        free(sizes);
        if (largest == UINT64_MAX) { free(perm); free(K); return -2; }
        if (largest > s) { free(perm); free(K); return -3; }  /* the protocol aborts */
    } else if (flags & ORACLE_IDENTITY_PERM) {
        for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    } else {
        uint64_t *keys = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
        if (!keys) { free(perm); free(K); return -2; }
        oracle_sampling_keys(n, sampling_key, flags, keys, nthreads);
        int rc = oracle_perm(n, keys, perm);
        free(keys);
        if (rc) { free(perm); free(K); return rc; }
    }
    int rc = run_window(in, perm, s, k, seed, flags, 0, m, 0, k, K, nthreads);
    if (rc == 0) {
        uint64_t words = (m * k + 31) / 32;
        memset(out, 0, (size_t)words * sizeof(uint32_t));
        for (uint64_t t = 0; t < m * k; ++t)   /* bit j*k + i = K_j[i] */
            out[t >> 5] |= (uint32_t)K[t] << (t & 31u);
    }
    free(perm);
    free(K);
    return rc;
}
