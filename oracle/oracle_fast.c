/*
 * Word-packed oracle for sampled sub-block Toeplitz hashing (arXiv 2308.02856).
 *
 * TEST INFRASTRUCTURE ONLY (tests, the package smoke check and the benchmark's
 * CPU legs).  Plain C; shares no code with the CUDA library.
 *
 * The same definitions as oracle.c (stated in oracle.h), with steps 5-6 of
 * the method - sub-block assembly (Sec. III.B step 1) and the Toeplitz
 * product (Sec. I, K = T . A'; Sec. III.B step 3) - restated on 64-bit
 * words instead of single bits:
 *
 *   K_j[i] = XOR_{c<s} seed_j[i - c + s - 1] AND A_j[c]
 *          = XOR_{c'<s} seed_j[i + c'] AND R_j[c']        (R_j[c'] = A_j[s-1-c'])
 *          = parity( XOR_w  W_i[w] AND R_j[w] ),
 *
 * where R_j is the sub-block reversed and packed 64 bits to a word (bits past
 * s are 0), and W_i[w] is the 64-bit word of seed_j that starts at bit
 * i + 64 w.  Reversing A turns T's anti-diagonal index into a window that
 * slides with the output row: row i reads the s seed bits starting at bit i.
 * An AND of two words forms 64 bit-products at once, XOR adds them over
 * GF(2), and the parity of the final word's population count is the row's
 * bit.  Nothing else is reordered: each output bit is one pass over the
 * words of its window.  Its results are pinned to the bit loop of oracle.c.
 */
#include "oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

static inline uint32_t bit32(const uint32_t *x, uint64_t i)
{
    return (x[i >> 5] >> (i & 31u)) & 1u;
}

/* R[w] (64-bit words): bit c' of R = A[s - 1 - c'] = bit(in, pos[s - 1 - c']);
   padding slots (ORACLE_NO_POS, only with ORACLE_SAMPLING_IID) read as 0. */
static void pack_reversed(const uint32_t *in, const uint32_t *pos, uint64_t s, int padded, uint64_t *R,
                          uint64_t nwords)
{
    memset(R, 0, (size_t)nwords * sizeof(uint64_t));
    for (uint64_t c = 0; c < s; ++c) {
        const uint32_t p = pos[c];
        if (padded && p == ORACLE_NO_POS) continue;
        const uint64_t cr = s - 1 - c;
        R[cr >> 6] |= (uint64_t)bit32(in, p) << (cr & 63u);
    }
}

/* One output bit: parity of XOR_w (W_i[w] AND R[w]), where W_i[w] is the 64
   seed bits from bit t0 + 64 w, t0 = off + i (S: little-endian 64-bit words,
   zero past the end of the seed string).  A window word is the two seed
   words it straddles, funnel-shifted by t0 mod 64, or one word when the
   window starts on a word boundary. */
static uint8_t fast_row(const uint64_t *S, uint64_t off, const uint64_t *R, uint64_t nwords, uint64_t i)
{
    const uint64_t t0 = off + i, q = t0 >> 6, b = t0 & 63u;
    uint64_t acc = 0;
    if (b == 0) {
        for (uint64_t w = 0; w < nwords; ++w)
            acc ^= S[q + w] & R[w];
    } else {
        for (uint64_t w = 0; w < nwords; ++w)
            acc ^= ((S[q + w] >> b) | (S[q + w + 1] << (64u - b))) & R[w];
    }
    return (uint8_t)(__builtin_popcountll(acc) & 1);
}

typedef struct {
    const uint32_t *in, *pos;
    const uint64_t *S, *js;
    uint64_t s, k, nj, i0, ni, nwords, seed_len;
    uint32_t flags;
    uint64_t *R;       /* nj * nwords packed reversed sub-blocks */
    uint8_t *out;      /* nj * ni, one byte per bit */
    uint64_t lo, hi;   /* this thread's share: sub-blocks (pack) or rows (hash) */
    int phase;
} fast_job;

static void *fast_worker(void *arg)
{
    fast_job *f = (fast_job *)arg;
    if (f->phase == 0) {  /* step 5: assemble and pack sub-blocks lo .. hi */
        for (uint64_t t = f->lo; t < f->hi; ++t)
            pack_reversed(f->in, f->pos + t * f->s, f->s, (f->flags & ORACLE_SAMPLING_IID) != 0,
                          f->R + t * f->nwords, f->nwords);
        return NULL;
    }
    /* step 6: flattened rows lo .. hi of the nj x ni window */
    for (uint64_t r = f->lo; r < f->hi; ++r) {
        const uint64_t t = r / f->ni, i = f->i0 + r % f->ni;
        const uint64_t off = (f->flags & ORACLE_SEED_PER_SUBBLOCK) ? f->js[t] * f->seed_len : 0;
        f->out[r] = fast_row(f->S, off, f->R + t * f->nwords, f->nwords, i);
    }
    return NULL;
}

int oracle_fast_window(const uint32_t *in, const uint32_t *pos, uint64_t s, uint64_t k, const uint32_t *seed,
                       uint64_t seed_bits, uint32_t flags, const uint64_t *js, uint64_t nj, uint64_t i0,
                       uint64_t ni, uint8_t *out, int nthreads)
{
    if (s < 1 || k < 1 || k > s || i0 + ni > k) return -1;
    if (nj == 0 || ni == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    const uint64_t nwords = (s + 63) / 64;
    /* seed string as 64-bit words, two zero words past its end so that every
       window word (up to bit seed_bits - 1 + 63) is in bounds */
    const uint64_t sw32 = (seed_bits + 31) / 32, sw64 = (seed_bits + 63) / 64 + 2;
    uint64_t *S = (uint64_t *)calloc((size_t)sw64, sizeof(uint64_t));
    uint64_t *R = (uint64_t *)malloc((size_t)(nj * nwords) * sizeof(uint64_t));
    if (!S || !R) { free(S); free(R); return -2; }
    for (uint64_t w = 0; w < sw32; ++w)
        S[w >> 1] |= (uint64_t)seed[w] << (32u * (w & 1u));
    if (seed_bits & 63u)  /* bits past the end of the string are 0 */
        S[seed_bits >> 6] &= (1ull << (seed_bits & 63u)) - 1ull;
    pthread_t th[256];
    fast_job jobs[256];
    for (int phase = 0; phase < 2; ++phase) {
        const uint64_t units = phase == 0 ? nj : nj * ni;
        int nt = (uint64_t)nthreads > units ? (int)units : nthreads;
        for (int t = 0; t < nt; ++t) {
            fast_job *f = &jobs[t];
            f->in = in; f->pos = pos; f->S = S; f->js = js;
            f->s = s; f->k = k; f->nj = nj; f->i0 = i0; f->ni = ni; f->nwords = nwords;
            f->seed_len = s + k - 1;
            f->flags = flags; f->R = R; f->out = out; f->phase = phase;
            f->lo = units * (uint64_t)t / (uint64_t)nt;
            f->hi = units * (uint64_t)(t + 1) / (uint64_t)nt;
            pthread_create(&th[t], NULL, fast_worker, f);
        }
        for (int t = 0; t < nt; ++t)
            pthread_join(th[t], NULL);
    }
    free(S);
    free(R);
    return 0;
}

typedef struct {
    uint64_t key;
    uint32_t idx;
} kp;

/* Total order of the sampled positions: by label, then by position. */
static int kp_cmp(const void *a, const void *b)
{
    const kp *x = (const kp *)a, *y = (const kp *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

int oracle_perm_ranges(uint64_t n, const uint64_t *keys, uint64_t nr, const uint64_t *lo, const uint64_t *cnt,
                       uint32_t *out)
{
    if (n > (1ull << 32)) return -1;
    uint64_t total = 0;
    for (uint64_t r = 0; r < nr; ++r) {
        if (lo[r] + cnt[r] > n) return -1;
        total += cnt[r];
    }
    if (total == 0) return 0;
    /* rank of the first label of each 16-bit label bucket */
    uint64_t *start = (uint64_t *)calloc(65537, sizeof(uint64_t));
    uint8_t *need = (uint8_t *)calloc(65536, 1);
    if (!start || !need) { free(start); free(need); return -2; }
    for (uint64_t i = 0; i < n; ++i)
        start[(keys[i] >> 48) + 1]++;
    for (int b = 0; b < 65536; ++b)
        start[b + 1] += start[b];
    /* the buckets that hold any requested rank */
    for (uint64_t r = 0; r < nr; ++r) {
        if (!cnt[r]) continue;
        for (int b = 0; b < 65536; ++b)
            if (start[b + 1] > lo[r] && start[b] < lo[r] + cnt[r]) need[b] = 1;
    }
    uint64_t m = 0;
    for (int b = 0; b < 65536; ++b)
        if (need[b]) m += start[b + 1] - start[b];
    kp *c = (kp *)malloc((size_t)m * sizeof(kp));
    uint64_t *fill = (uint64_t *)calloc(65536, sizeof(uint64_t));  /* candidates so far per bucket */
    uint64_t *base = (uint64_t *)calloc(65537, sizeof(uint64_t));  /* first candidate slot per bucket */
    if (!c || !fill || !base) { free(c); free(fill); free(base); free(start); free(need); return -2; }
    for (int b = 0; b < 65536; ++b)
        base[b + 1] = base[b] + (need[b] ? start[b + 1] - start[b] : 0);
    for (uint64_t i = 0; i < n; ++i) {
        const int b = (int)(keys[i] >> 48);
        if (!need[b]) continue;
        kp *e = &c[base[b] + fill[b]++];
        e->key = keys[i];
        e->idx = (uint32_t)i;
    }
    for (int b = 0; b < 65536; ++b)  /* sort each needed bucket by (label, position) */
        if (need[b]) qsort(c + base[b], (size_t)(base[b + 1] - base[b]), sizeof(kp), kp_cmp);
    uint64_t o = 0;
    for (uint64_t r = 0; r < nr; ++r)
        for (uint64_t q = 0; q < cnt[r]; ++q) {
            const uint64_t rank = lo[r] + q;
            int lo_b = 0, hi_b = 65535;  /* the bucket holding rank */
            while (lo_b < hi_b) {  /* first bucket with start[b + 1] > rank */
                const int mid = (lo_b + hi_b) / 2;
                if (start[mid + 1] > rank) hi_b = mid;
                else lo_b = mid + 1;
            }
            out[o++] = c[base[lo_b] + (rank - start[lo_b])].idx;
        }
    free(c); free(fill); free(base); free(start); free(need);
    return 0;
}
