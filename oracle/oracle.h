/*
 * Oracle for sampled sub-block Toeplitz hashing (arXiv 2308.02856).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously correct CPU
 * statement of what the hashing path computes.  Only the test suite, the
 * package smoke check and the CPU-baseline leg of the benchmark may load it;
 * the CUDA library never links, includes or calls it, and the two share no
 * code.  oracle.c computes every bit of the path one bit at a time, exactly
 * as the definitions below state them; oracle_fast.c restates steps 5-6 on
 * 64-bit words (for full-size checks and the timed CPU baseline) and is
 * pinned to the bit loop.
 *
 * Bit convention (the paper fixes none; this is the reading used throughout):
 *   bit(x, i) = (x[i >> 5] >> (i & 31)) & 1 for every packed string
 *   (input block, Toeplitz seed, output).
 *
 * Definitions, in the order of the sub-block protocol of Sec. III.B:
 *   1. Sampling (Sec. III.B step 1).  Position i gets the 64-bit label
 *        key_i = (x0 << 32) | x1,  (x0..x3) = Philox4x32-10(ctr = (i_lo, i_hi, 0, 0),
 *                                                        key = (K_lo, K_hi))
 *      where K is the sampling key.  The sampled order is the stable argsort
 *      of key_i (equal keys: lower index first); sub-block j is made of the
 *      positions at sorted ranks [j*s, (j+1)*s), in rank order.
 *   2. Extraction (Sec. I, Sec. III.B step 3): K_j = T * A_j mod 2 with the
 *      k x s diagonal-constant matrix T[i][c] = seed_j[i - c + s - 1], i.e.
 *        K_j[i] = XOR_{c < s} seed_j[i - c + s - 1] AND A_j[c].
 *      seed_j is the shared seed (s + k - 1 bits), or, with
 *      ORACLE_SEED_PER_SUBBLOCK, the j-th consecutive (s + k - 1)-bit span
 *      of the seed string.
 *   1b. With ORACLE_SAMPLING_IID, the paper's own law instead: position i
 *      joins sub-block V_i = floor(key_i * m / 2^64) (i.i.d. uniform on
 *      [0, m)); sub-block j is the input at S_j = {i : V_i = j} in
 *      increasing position order, zero-padded to s = L_S^UB, and the run
 *      aborts (returns -3) when some |S_j| > s (Sec. III.D).
 *   3. Concatenation (Sec. III.B step 4): output bit j*k + i = K_j[i]; the
 *      tail bits of the last output word are 0.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Flags, same meaning as the library's create flags. */
#define ORACLE_SEED_PER_SUBBLOCK 0x1u
#define ORACLE_IDENTITY_PERM     0x2u
/* The paper's i.i.d. sampling law (definition 1b). */
#define ORACLE_SAMPLING_IID      0x10u
/* Order entry of a padding slot (reads as a 0 bit). */
#define ORACLE_NO_POS            0xffffffffu
/* Test hook: keep only the top b (1..63) bits of every sampling key. */
#define ORACLE_KEY_BITS(b)       (((uint32_t)(b) & 0x3fu) << 8)

/* Philox4x32-10 block function (Salmon, Moraes, Dror, Shaw, SC'11). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Sampling label of position i (definition 1 above). */
uint64_t oracle_sampling_key(uint64_t i, uint64_t sampling_key, uint32_t flags);

/* keys[i] = oracle_sampling_key(i) for i < n, split over nthreads threads. */
void oracle_sampling_keys(uint64_t n, uint64_t sampling_key, uint32_t flags,
                          uint64_t *keys, int nthreads);

/* perm = stable argsort of keys[0..n) (qsort on (key, index) pairs). 0 = ok. */
int oracle_perm(uint64_t n, const uint64_t *keys, uint32_t *perm);

/* out[r] = perm[lo + r] for r < cnt, without sorting all n positions
   (rank selection through a 16-bit key histogram, then a sort of the
   candidates).  0 = ok. */
int oracle_perm_range(uint64_t n, const uint64_t *keys, uint64_t lo, uint64_t cnt,
                      uint32_t *out);

/* Property check of a claimed sampled order (for sizes where sorting all n
   positions on the CPU is too slow): returns -1 when every perm entry is
   < n and the labels keys[perm[t]] increase strictly in (label, position)
   order - which makes perm a bijection and the unique stable argsort -
   else the first offending t. */
int64_t oracle_check_order(uint64_t n, const uint64_t *keys, const uint32_t *perm, int nthreads);

/* Sub-block assembly: A[c] = bit(in, pos[c]) for c < s (one byte per bit). */
void oracle_subblock(const uint32_t *in, const uint32_t *pos, uint64_t s, uint8_t *A);
/* The same with ORACLE_NO_POS entries read as 0 (padded i.i.d. sub-blocks). */
void oracle_subblock_padded(const uint32_t *in, const uint32_t *pos, uint64_t s, uint8_t *A);

/* i.i.d. law (definition 1b): the sub-block of a position with label key. */
uint32_t oracle_iid_label(uint64_t key, uint64_t m);

/* sizes[j] = |S_j| for j < m; returns the largest size.  When it is <= s
   and order is not NULL, order[j*s + c] = the c-th smallest position of S_j
   for c < sizes[j] and ORACLE_NO_POS for sizes[j] <= c < s.  UINT64_MAX on
   allocation failure. */
uint64_t oracle_iid_order(uint64_t n, const uint64_t *keys, uint64_t m, uint64_t s,
                          uint64_t *sizes, uint32_t *order);

/* Eq. 7: 1 - Phi(sign(L - N p) sqrt(2 N H(L/N, p))), the Zubkov-Serov bound
   on the chance that a binomial(N, p) sub-block size exceeds L. */
double oracle_size_tail_bound(uint64_t N, uint64_t L, double p);

/* Eq. 7: the smallest L with m * oracle_size_tail_bound(N, L, p) <= eps
   (N when no L below N qualifies or the arguments are degenerate). */
uint64_t oracle_block_limit(uint64_t N, uint64_t m, double eps, double p);

/* One Toeplitz output bit: XOR_{c<s} bit(seed, off + i - c + s - 1) AND A[c]. */
uint8_t oracle_toeplitz_bit(const uint32_t *seed, uint64_t off, uint64_t s,
                            const uint8_t *A, uint64_t i);

/* K[i - i0] for i in [i0, i0 + cnt) (one byte per bit). */
void oracle_toeplitz(const uint32_t *seed, uint64_t off, uint64_t s,
                     const uint8_t *A, uint64_t i0, uint64_t cnt, uint8_t *K);

/* The whole method (definitions 1-3): out gets ceil(m*k/32) words.
   Sub-blocks are processed on nthreads threads.  0 = ok, -1 = bad args,
   -2 = out of memory, -3 = the i.i.d. law aborts (a sub-block exceeds s). */
int oracle_extract(uint64_t n, uint64_t m, uint64_t s, uint64_t k,
                   const uint32_t *in, const uint32_t *seed, uint64_t sampling_key,
                   uint32_t flags, uint32_t *out, int nthreads);

/* A window of the method: K_j[i] for j in [j0, j0+nj), i in [i0, i0+ni),
   given the sampled positions of those sub-blocks (pos[(j-j0)*s + c]).
   out[(j-j0)*ni + (i-i0)] is one byte per bit.  Threads split the j range. */
void oracle_extract_window(const uint32_t *in, const uint32_t *pos, uint64_t s, uint64_t k,
                           const uint32_t *seed, uint32_t flags, uint64_t j0, uint64_t nj,
                           uint64_t i0, uint64_t ni, uint8_t *out, int nthreads);

/* ---- word-packed restatement (oracle_fast.c) ---------------------------
   Steps 5-6 on 64-bit words: with R_j the sub-block reversed and packed
   (bit c' = A_j[s-1-c']) and W_i[w] the 64 seed bits from bit i + 64 w,
   K_j[i] = parity(XOR_w W_i[w] AND R_j[w]).  Pinned to the bit loop above. */

/* K_j[i] for the nj sub-blocks js[0..nj) and rows i in [i0, i0 + ni), given
   their sampled positions pos[t*s + c] (sub-block js[t]).  seed holds
   seed_bits bits (s + k - 1, or m (s + k - 1) with ORACLE_SEED_PER_SUBBLOCK,
   where sub-block j's seed starts at bit j (s + k - 1)).  With
   ORACLE_SAMPLING_IID, ORACLE_NO_POS entries read as 0.
   out[t*ni + (i - i0)] is one byte per bit.  Threads split the rows.
   0 = ok, -1 = bad args, -2 = out of memory. */
int oracle_fast_window(const uint32_t *in, const uint32_t *pos, uint64_t s, uint64_t k, const uint32_t *seed,
                       uint64_t seed_bits, uint32_t flags, const uint64_t *js, uint64_t nj, uint64_t i0,
                       uint64_t ni, uint8_t *out, int nthreads);

/* Ranks [lo[r], lo[r] + cnt[r]) of the stable argsort of keys[0..n) for
   r < nr, concatenated into out, in one pass over the keys (a 16-bit label
   histogram, then a sort of the candidates of the needed buckets).
   0 = ok, -1 = bad args, -2 = out of memory. */
int oracle_perm_ranges(uint64_t n, const uint64_t *keys, uint64_t nr, const uint64_t *lo, const uint64_t *cnt,
                       uint32_t *out);

#ifdef __cplusplus
}
#endif
#endif
