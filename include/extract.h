/*
 * extract.h - C ABI of the GB300 (sm_103a) sampled sub-block Toeplitz hashing
 * library, libextract.so.
 *
 * What it computes (arXiv 2308.02856, "Sampled sub-block hashing for large
 * input randomness extraction"):
 *
 *   1. Sampling (Sec. III.B step 1).  Every input position i gets a 64-bit
 *      label, (x0 << 32) | x1 of Philox4x32-10 with counter (i_lo, i_hi, 0, 0)
 *      and key = the 64-bit sampling key (lo, hi).  The sampled order is the
 *      stable argsort of the labels (equal labels: lower position first).
 *      Sub-block j, for j < m, is the s positions at sorted ranks
 *      [j*s, (j+1)*s), taken in rank order: A_j[c] = in[perm[j*s + c]].
 *      Positions at ranks >= m*s are not hashed.  (The paper draws an i.i.d.
 *      label per round and so gets sub-blocks of varying size; this library
 *      cuts the sampled order into m equal sub-blocks instead.)
 *   2. Extraction (Sec. I, K = T . A'; Sec. III.B step 3).  Each sub-block is
 *      multiplied over GF(2) by the k x s diagonal-constant (Toeplitz) matrix
 *      T[i][c] = seed_j[i - c + s - 1], built from an (s + k - 1)-bit seed:
 *        K_j[i] = XOR_{c<s} seed_j[i - c + s - 1] AND A_j[c],   i < k.
 *      T is never materialised.
 *   3. Concatenation (Sec. III.B step 4).  Output bit j*k + i = K_j[i].
 *
 * Bit strings (input, seed, output) are packed LSB-first in uint32 words:
 * bit t of a string is (w[t >> 5] >> (t & 31)) & 1.  Output bits past m*k in
 * the last word are written as 0.
 *
 * Errors: every entry point returns EXTRACT_OK (0) or a negative code and
 * never aborts the process; extract_last_error() gives the message of the
 * last failure on the calling thread.  CUDA failures map to EXTRACT_ECUDA.
 *
 * Streams are passed as `void *` holding a cudaStream_t (NULL = the legacy
 * default stream); all device work of a run is asynchronous on that stream.
 */
#ifndef EXTRACT_H
#define EXTRACT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define EXTRACT_OK         0
#define EXTRACT_EINVAL    (-1)  /* bad argument (shape, null pointer, flag) */
#define EXTRACT_ENOMEM    (-2)  /* device or host allocation failed          */
#define EXTRACT_ECUDA     (-3)  /* a CUDA call failed; see extract_last_error */
#define EXTRACT_ETIMEDOUT (-4)  /* a bounded wait ran out                     */
#define EXTRACT_EBUDGET   (-5)  /* the job does not fit the memory budget     */
#define EXTRACT_EBUSY     (-6)  /* no free slot / resource in use             */
#define EXTRACT_EINTERNAL (-7)  /* an internal consistency check failed       */
#define EXTRACT_EABORT    (-8)  /* i.i.d. sampling: a sub-block exceeds the
                                   block size limit s, so the protocol aborts
                                   (Sec. III.D); nothing is created        */

/* ---- create flags ---------------------------------------------------- */
/* seed_bits holds m consecutive (s + k - 1)-bit seeds, one independent
   Toeplitz matrix per sub-block (Sec. III.B step 3 draws f_RE,j
   independently).  Without it, all sub-blocks share one seed. */
#define EXTRACT_SEED_PER_SUBBLOCK 0x1u
/* Skip sampling: perm = identity, so sub-block j is input bits
   [j*s, (j+1)*s).  With m = 1 and s = n this is direct whole-block Toeplitz
   hashing, the "traditional" method of Sec. IV.C. */
#define EXTRACT_IDENTITY_PERM     0x2u
/* Hashing method.  Default (neither flag): the library picks the faster of
   the two exact methods for the shape.  EXTRACT_METHOD_DIRECT forces the
   direct GF(2) product (bit-sliced AND/XOR, work m*k*s); EXTRACT_METHOD_NTT
   forces the number-theoretic-transform middle product modulo the prime
   7*2^26+1.  It splits each sub-block into P pieces (1 <= P <= 16) of h
   bits (h = s for P = 1, else ceil(s/P) rounded up to a multiple of 32) and
   costs P + 1 transforms of the power of two N >= h+k-1 per sub-block; P
   is the one with the least predicted work.  With
   EXTRACT_SEED_PER_SUBBLOCK (then N >= 2^16) the spectra of every
   sub-block's seed windows are built at create and kept (4 m P N bytes)
   when they take at most a quarter of the free device memory, else their
   windows are transformed in every run (2P + 1 transforms).  It needs
   s+k-1 > 2^11, s < 7*2^26+1 and
   N <= 2^22 for some P <= 16 (EXTRACT_EINVAL otherwise).  Both methods
   give the same bits. */
#define EXTRACT_METHOD_DIRECT     0x4u
#define EXTRACT_METHOD_NTT        0x8u
/* NTT method: use P = 2^l pieces per sub-block (l = 0 .. 4) instead of the
   split with the least predicted work; EXTRACT_EINVAL if that split has no
   transform length <= 2^22 or leaves a piece empty.  Tuning and test hook. */
#define EXTRACT_NTT_SPLIT(l)      ((((uint32_t)(l) + 1u) & 0x7u) << 16)
/* Test hook: keep only the top b (1..63) bits of every sampling label, which
   forces many equal labels so that the index tie-break is exercised. */
#define EXTRACT_KEY_BITS(b)       ((((uint32_t)(b)) & 0x3fu) << 8)
/* The paper's own sampling law (Sec. III.B step 1) instead of the sorted
   order: position i joins sub-block V_i = floor(label_i * m / 2^64), an
   i.i.d. uniform draw on [0, m), so sub-block sizes are binomial(n, 1/m).
   Sub-block j is the input at S_j = {i : V_i = j} in increasing position
   order, zero-padded to s, which now plays the block size limit L_S^UB
   (extract_block_limit computes it from Eq. 7): the Toeplitz matrix is
   k x s and the seed s + k - 1 bits as usual.  Every position is hashed
   (m*s >= n is not required).  extract_create fails with EXTRACT_EABORT
   when some |S_j| > s (a batch fails to create, naming the job; a served
   job fails and extract_server_wait returns EXTRACT_EABORT).  Needs
   n < 2^32 and m <= 2^16; not combinable with EXTRACT_IDENTITY_PERM. */
#define EXTRACT_SAMPLING_IID      0x10u
/* Gather (step 1's bit movement).  Default (neither flag): for inputs of at
   least 2^22 bits the library compiles the order into bucket tables at
   create time (a two-stage gather: each 2^16-bit input chunk regrouped by
   sub-block in shared memory, then each sub-block permuted in shared
   memory), which costs 2 bytes per sampled bit plus 4 bytes per stored
   sub-block bit of extra device memory and makes no random global reads; it
   needs n <= 25600 input chunks of 2^16 bits, or of 2^18 bits with 18-bit
   table entries (2.25 bytes per sampled bit), and every sub-block's regrouped
   bits within 220 KiB; otherwise (or without room) the plain gather is
   kept.
   EXTRACT_GATHER_PLAIN keeps the plain gather (one random input read per
   gathered bit); EXTRACT_GATHER_BUCKETS asks for the tables at any input
   size (EXTRACT_EINVAL if the shape does not suit them).  Both give the
   same sub-blocks.  Not combinable with EXTRACT_IDENTITY_PERM. */
#define EXTRACT_GATHER_PLAIN      0x20u
#define EXTRACT_GATHER_BUCKETS    0x40u
/* Bucket tables over 2^18-bit input chunks (18-bit table entries) even where
   2^16-bit chunks fit; the library itself takes them when the input has more
   than 25600 chunks of 2^16 bits or its runs are too short to fit.  Tuning
   and test hook. */
#define EXTRACT_GATHER_WIDE_CHUNKS 0x80u

/* The direct GF(2) product on the tensor cores instead (the dense form of
   Sec. I's K = T . A' with all sub-blocks sharing T): D = T . [A_1 .. A_m]
   over the integers with 0/1 e4m3 operands on tcgen05.mma (kind::f8f6f4,
   f32 accumulators in tensor memory), K_j[i] = D[i][j] mod 2.  The sums are
   read back and reduced to parities every K chunk (4096 by default), so
   every partial sum stays an exact small integer.  Needs one shared seed
   (EXTRACT_EINVAL with EXTRACT_SEED_PER_SUBBLOCK); exclusive with the other
   method flags.  Gives the same bits as the other methods.  A kernel that
   gives up on a wait (about a second) sets an error word that
   extract_status reports. */
#define EXTRACT_METHOD_TENSOR     0x100000u
/* Tensor-core method: 2^l K blocks of 128 (l = 0 .. 14) summed before each
   parity read-back instead of 2^5.  Test hook. */
#define EXTRACT_TC_CHUNK(l)       ((((uint32_t)(l) + 1u) & 0xfu) << 24)
/* Tensor-core method, test hook of the error path: every CTA of the hash
   kernel first waits on a barrier that nothing arrives on, so the wait runs
   out after about a second; the kernel then sets the context's error word
   and returns without multiplying (extract_status reports
   EXTRACT_ETIMEDOUT; the output is not valid). */
#define EXTRACT_TC_TEST_STALL     0x10000000u

typedef struct extract_ctx extract_ctx;

/*
 * extract_create - validate the shape, copy the seed to the device and build
 * the sampled order (step 1) on the GPU, resident until extract_destroy.
 *
 *   out            receives the new context (owned by the library).
 *   n              input bits, m*s <= n <= 2^32 (i.i.d. law: n < 2^32).
 *   m, s, k        sub-blocks, bits per sub-block, output bits per sub-block;
 *                  1 <= m, 1 <= k <= s.
 *   seed_bits_host host pointer to ceil(L/32) words with L = s + k - 1 (or
 *                  m*(s + k - 1) with EXTRACT_SEED_PER_SUBBLOCK); copied, the
 *                  caller keeps ownership.
 *   sampling_key   64-bit Philox key of the sampling labels.
 *   flags          EXTRACT_* create flags.
 *
 * Synchronous: it returns once the order (and the tables below) are built.
 * Device memory held: 4n bytes of order (4ms with EXTRACT_SAMPLING_IID, none
 * with EXTRACT_IDENTITY_PERM) plus about n/8 bytes of sub-block buffer and
 * the seed; with the bucketed gather about 5 more bytes per sampled bit (see
 * EXTRACT_GATHER_PLAIN); with the NTT method its tables and one work buffer
 * of at most 128 MB per lane; with EXTRACT_SEED_PER_SUBBLOCK and the NTT
 * method possibly the resident seed spectra (see EXTRACT_METHOD_NTT).
 * Errors: EINVAL, ENOMEM, ECUDA, EABORT (i.i.d. law only).
 */
int extract_create(extract_ctx **out, uint64_t n, uint32_t m, uint32_t s, uint32_t k,
                   const uint32_t *seed_bits_host, uint64_t sampling_key, uint32_t flags);

/*
 * extract_run - steps 1-3 on one input block: gather the m sub-blocks in
 * sampled order, hash each one and write the concatenated output.
 *
 *   stream        cudaStream_t (void *) the work is queued on.
 *   in_bits_dev   device pointer, ceil(n/32) words, caller-owned, read only.
 *   out_bits_dev  device pointer, ceil(m*k/32) words, caller-owned; fully
 *                 overwritten.
 *
 * Asynchronous.  Both buffers must stay valid until the stream reaches the
 * end of the run.  The context's sub-block buffer is reused by every run, so
 * runs on one context must be ordered on one stream (or by events).
 * Errors: EINVAL (null pointers), ECUDA (launch failure).
 */
int extract_run(extract_ctx *h, void *stream, const uint32_t *in_bits_dev,
                uint32_t *out_bits_dev);

/*
 * extract_run_host - extract_run on host buffers, end to end: copies the
 * ceil(n/32) input words from in_bits_host to the device, runs steps 1-3 and
 * copies the ceil(m*k/32) output words back to out_bits_host, ordered after
 * earlier work on `stream`; returns once the output is in host memory.  With
 * the bucketed gather the copies run on an internal stream of the context and
 * overlap the work (input pieces feed the gather as they land; the NTT
 * hash's finished output words go back while later ones are computed).  The
 * device staging buffers are allocated on the first call and kept until
 * extract_destroy.  Page-locked host buffers give full copy bandwidth;
 * pageable ones work.  Calls on one context must not overlap.
 * Errors: EINVAL (null pointers), ENOMEM, ECUDA.
 */
int extract_run_host(extract_ctx *h, void *stream, const uint32_t *in_bits_host,
                     uint32_t *out_bits_host);

/*
 * extract_run_host_many - extract_run_host on `count` blocks in a row (a
 * stream of blocks, as QKD and QRNG post-processing deliver them): block b's
 * input comes from in_bits_host[b] (ceil(n/32) words) and its output goes to
 * out_bits_host[b] (ceil(m*k/32) words); the two host arrays of pointers are
 * read before the call returns.  The copies run on two internal streams of
 * the context and overlap the work of the neighbouring blocks: block b+1's
 * input goes up while block b is hashed, block b's output comes down while
 * block b+1 is gathered and hashed.  Each block is gathered and hashed in
 * order on `stream`, with the same results as extract_run_host one block at
 * a time.  Returns once every output is in host memory.  Two device staging
 * buffers each way are allocated on the first call and kept until
 * extract_destroy.  Page-locked host buffers give full copy bandwidth and
 * the overlap; calls on one context must not overlap.
 * Errors: EINVAL (null pointers), ENOMEM, ECUDA.
 */
int extract_run_host_many(extract_ctx *h, void *stream, const uint32_t *const *in_bits_host,
                          uint32_t *const *out_bits_host, uint32_t count);

/* extract_gather - step 1's gather alone: fills the context's sub-block
   buffer from in_bits_dev (same contract as extract_run). */
int extract_gather(extract_ctx *h, void *stream, const uint32_t *in_bits_dev);

/* extract_hash - steps 2-3 alone on the sub-block buffer filled by the last
   extract_gather on the same stream; writes out_bits_dev as extract_run does. */
int extract_hash(extract_ctx *h, void *stream, uint32_t *out_bits_dev);

/*
 * extract_run_plain - the same result as extract_run through the plain
 * per-block path: after the gather, one kernel launch per sub-block, one
 * thread per output bit, no register tiling and no seed reuse across
 * sub-blocks.  It is the baseline the tuned path is measured against.
 */
int extract_run_plain(extract_ctx *h, void *stream, const uint32_t *in_bits_dev,
                      uint32_t *out_bits_dev);

/* extract_read_perm - copy ranks [start, start+count) of the sampled order
   to host memory (synchronous).  With EXTRACT_IDENTITY_PERM it writes the
   identity.  With EXTRACT_SAMPLING_IID the order has m*s slots: slot
   j*s + c is the c-th position of sub-block j, 0xffffffff past its size.
   Errors: EINVAL if start + count exceeds the order. */
int extract_read_perm(extract_ctx *h, uint64_t start, uint64_t count, uint32_t *dst_host);

/* extract_subblock_sizes - sizes_host[j] = |S_j| for j < m: the number of
   input bits in each sub-block (s for every j under the sorted order; the
   binomial sizes under EXTRACT_SAMPLING_IID).  Host memory, synchronous. */
int extract_subblock_sizes(extract_ctx *h, uint64_t *sizes_host);

/*
 * extract_block_limit - the block size limit of Eq. 7 (Sec. III.D): the
 * smallest L with
 *     m * (1 - Phi(sign(L - N p) sqrt(2 N H(L/N, p)))) <= eps,
 * H(x, p) = x ln(x/p) + (1-x) ln((1-x)/(1-p)), Phi the standard normal CDF
 * (the Zubkov-Serov bound on a binomial tail, union over the m
 * sub-blocks).  N = n input bits, p = the chance that a bit lands in a given
 * sub-block (1/m without sifting), eps = the allowed abort probability
 * eps_Omega'.  Writes N when no smaller L qualifies.  Host only (no GPU).
 * Errors: EINVAL for N = 0, m = 0, p outside (0, 1), eps <= 0 or a null
 * limit_out.
 */
int extract_block_limit(uint64_t N, uint32_t m, double eps, double p, uint64_t *limit_out);

/* extract_read_subblock - copy sub-block j as gathered by the last run or
   gather, ceil(s/32) words, to host memory (synchronous, waits for the
   device).  Word layout: bit t of the copy is A_j[s - 1 - t], the sub-block
   reversed, which is the order the hashing kernel consumes. */
int extract_read_subblock(extract_ctx *h, uint32_t j, uint32_t *dst_host);

/* extract_describe - write a one-line text description of the context's
   kernel configuration (tile shape, split, grid) into buf. */
int extract_describe(extract_ctx *h, char *buf, uint32_t buflen);

/* extract_status - synchronise the device and report whether a kernel of
   this context gave up on a bounded wait since the last call
   (EXTRACT_ETIMEDOUT, then cleared) or not (EXTRACT_OK). */
int extract_status(extract_ctx *h);

/* extract_gather_bytes - the device-memory bytes one extract_gather of this
   context reads and writes by design: with the bucket tables, the input
   once, the tables (chunk starts, in-chunk positions, destinations, member
   fields), the run buffer written and read, and the sub-block buffer; with
   the window-major order, its entries and slots, the input once and the
   sub-block buffer; with the plain gather, the order entries (once per
   input window pass), one 32-byte sector of input per gathered bit and the
   sub-block buffer.  Host only, no device work. */
int extract_gather_bytes(extract_ctx *h, uint64_t *bytes);

/*
 * extract_run_static - extract_run for callers that must not allocate device
 * memory.  The paper has no counterpart; this is a library convenience.
 *
 * Who needs it: code that runs with a device-memory budget handed out by
 * someone else (an embedding application's own pool, a post-processing
 * pipeline sized up front) and so may not call cudaMalloc, and loops that
 * cannot afford the implicit device-wide synchronisation cudaMalloc and
 * cudaFree can cause.  Such callers own all of their buffers; this call only
 * borrows them and never calls cudaMalloc, cudaFree or any allocating
 * library routine.
 *
 * Its scratch (the padded seed plus the gathered sub-blocks) is one fixed
 * array of EXTRACT_STATIC_SCRATCH_WORDS 32-bit words (16 MiB) in the
 * library's static device memory.  A device holds that array from the first
 * use of the library's device code there (with CUDA's lazy module loading,
 * the first call of this entry point or of any other on that device) until
 * the process exits.
 *   n, m, s, k    as for extract_create; one shared seed (no per-sub-block
 *                 seeds).  Shapes whose scratch would exceed the array,
 *                 about m*s > 2^27 bits, are rejected with EXTRACT_EINVAL
 *                 and a message giving the words needed.
 *   perm_dev      device pointer to the sampled order as extract_read_perm
 *                 returns it (its first m*s entries are read), or NULL for
 *                 the identity order (direct hashing of consecutive s-bit
 *                 blocks; then m*s <= n).  Every entry must be a position
 *                 < n or, when n < 2^32, the padding value 0xffffffff,
 *                 which reads as a 0 bit: an EXTRACT_SAMPLING_IID
 *                 context's order (m*s slots, which may exceed n) is
 *                 accepted as it is.
 *   seed_dev      device pointer, ceil((s+k-1)/32) words of seed bits.
 *   in_bits_dev   device pointer, ceil(n/32) input words.
 *   out_bits_dev  device pointer, ceil(m*k/32) words, fully overwritten.
 *   stream        cudaStream_t the work is queued on.
 *
 * Every call looks up the array's device address with cudaGetSymbolAddress
 * while the calling device is current (a host-side lookup, nothing is
 * allocated).  The first call on a device may load the library's device
 * code there and reserve the array, with the implicit synchronisation that
 * module loading brings, so make one call at setup, before any stream
 * capture.  All calls share the one array and each call rewrites all of the
 * scratch it reads, so results never depend on earlier calls; but two calls
 * whose work overlaps on the GPU (different streams, or different host
 * threads, without ordering between them) race on the array and give wrong
 * results.  Order them on one stream.
 */
#define EXTRACT_STATIC_SCRATCH_WORDS (4u * 1024u * 1024u)
int extract_run_static(uint64_t n, uint32_t m, uint32_t s, uint32_t k, const uint32_t *perm_dev,
                       const uint32_t *seed_dev, const uint32_t *in_bits_dev, uint32_t *out_bits_dev,
                       void *stream);

/* ---- batching: many blocks of uneven n, s, k in one persistent launch -- */

/* One block of a batch or a served job: the arguments of extract_create. */
typedef struct extract_job_desc {
    uint64_t n;
    uint32_t m, s, k;
    uint32_t flags;                  /* EXTRACT_* create flags */
    uint64_t sampling_key;
    const uint32_t *seed_bits_host;  /* as in extract_create; copied */
} extract_job_desc;

typedef struct extract_batch extract_batch;

/* batch flags */
#define EXTRACT_BATCH_NO_GRAPH 0x1u  /* launch the kernels directly instead of replaying a CUDA graph */
#define EXTRACT_BATCH_NO_TUNE  0x2u  /* use the single-block heuristic tile instead of the autotuned one */
#define EXTRACT_BATCH_DIRECT_ONLY 0x4u  /* hash every job with the direct method (no NTT jobs) */
#define EXTRACT_BATCH_TENSOR 0x8u       /* test hook: hash every shared-seed job with the tensor-core product */

/*
 * extract_batch_create - set up njobs independent blocks (the method of
 * Sec. III.B applied to each) for hashing in one persistent launch.
 *
 * Builds every job's sampled order (synchronous) and picks each job's
 * method by least predicted time: the NTT method where it is eligible, the
 * tensor-core product where the job has one shared seed (those jobs run on
 * four concurrent lanes of the batch, each with its own stream and work
 * buffer, longest predicted first to the least-loaded lane, concurrent with
 * the rest), else the direct method, whose tile shape the autotuner chooses
 * (measured cost per tile variant, cached per device, then the least
 * predicted time including padding).  Direct jobs' word ranges are split so
 * the tiles balance across SMs, the tiles are ordered longest first, and
 * their per-run kernels (zero outputs, gather, persistent hash) are
 * captured into a CUDA graph.  Device memory held: per job as
 * extract_create (plus the NTT tables of NTT jobs and one NTT work buffer
 * per lane).
 * Errors: EINVAL (empty list, a bad job shape or flags), ENOMEM, ECUDA.
 */
int extract_batch_create(extract_batch **out, const extract_job_desc *jobs, uint32_t njobs,
                         uint32_t flags);

/*
 * extract_batch_run - hash every job's input into its output on `stream`
 * (asynchronous).  in_bits_dev[i] / out_bits_dev[i] are job i's device
 * buffers with the sizes of extract_run; the two host arrays of pointers are
 * read before the call returns.  Output i is fully overwritten with exactly
 * what extract_run would give for job i.  Runs of one batch must be ordered
 * on one stream.  Errors: EINVAL, ECUDA.
 */
int extract_batch_run(extract_batch *b, void *stream, const uint32_t *const *in_bits_dev,
                      uint32_t *const *out_bits_dev);

/* extract_batch_run_sequential - the same result with one gather and one
   hash launch per block, each with the single-block heuristic tile: the
   baseline the persistent launch is measured against. */
int extract_batch_run_sequential(extract_batch *b, void *stream, const uint32_t *const *in_bits_dev,
                                 uint32_t *const *out_bits_dev);

/* extract_batch_status - synchronise the device and report whether a
   tensor-core kernel of the batch gave up on a bounded wait since the last
   call (EXTRACT_ETIMEDOUT, then cleared) or not (EXTRACT_OK). */
int extract_batch_status(extract_batch *b);

/* extract_batch_describe - one line: jobs, tiles, graph, chosen variants and
   their measured cost. */
int extract_batch_describe(extract_batch *b, char *buf, uint32_t buflen);

/* extract_batch_destroy - synchronise the device and free the batch. */
int extract_batch_destroy(extract_batch *b);

/* ---- serving: continuous batching under a device-memory budget -------- */

typedef struct extract_server extract_server;

typedef struct extract_stats {
    uint64_t submitted, admitted, completed, failed, rejected;
    uint64_t queued, active, waves;
    uint64_t bytes_in_use, bytes_peak;  /* budget charge now / at most */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* latency: submit -> done */
    double input_bits_done;                  /* sum of n over completed jobs */
    double span_s;                           /* first submit -> last completion */
    double gbit_per_s;                       /* input_bits_done / span_s / 1e9 */
} extract_stats;

/*
 * extract_server_create - start a serving loop on the current device.
 *
 *   hbm_budget_bytes  device memory the admitted jobs may hold at once: each
 *                     job is charged its order (4n bytes, returned once its
 *                     sub-blocks are gathered), sub-block buffer, seed, and
 *                     its input and output buffers.
 *   max_slots         most jobs admitted at once.
 *   wave_us           GPU time of one hashing wave in microseconds (0: 2000).
 *   flags             must be 0.
 *
 * Jobs are admitted first come first served while budget and slots allow;
 * admitted jobs are set up (order, gather) on their own stream while others
 * hash, and every hashing launch ("wave") mixes tiles of all ready jobs,
 * shortest remaining work first, so jobs join and leave the running work
 * continuously.  Two host threads run the loop.  Errors: EINVAL, ENOMEM,
 * ECUDA.
 */
int extract_server_create(extract_server **out, uint64_t hbm_budget_bytes, uint32_t max_slots,
                          uint32_t wave_us, uint32_t flags);

/*
 * extract_server_submit - queue one job (thread-safe).  The seed is copied;
 * in_bits_dev (ceil(n/32) words) and out_bits_dev (ceil(m*k/32) words) are
 * the caller's device buffers and must stay valid until the job completes;
 * the output is fully overwritten with exactly what extract_run gives.
 * *ticket identifies the job.  Errors: EINVAL (shape, flags, null),
 * EBUDGET (the job alone exceeds the budget), EBUSY (server stopping).
 */
int extract_server_submit(extract_server *srv, const extract_job_desc *job, const uint32_t *in_bits_dev,
                          uint32_t *out_bits_dev, uint64_t *ticket);

/*
 * extract_server_wait - block until the job completes or timeout_ms passes.
 * EXTRACT_OK: done (latency_ms, if not NULL, gets submit -> completion);
 * EXTRACT_ETIMEDOUT: not yet (the ticket stays valid); otherwise the job's
 * own error.  A completed ticket is forgotten after a successful wait.
 */
int extract_server_wait(extract_server *srv, uint64_t ticket, uint32_t timeout_ms, double *latency_ms);

/* extract_server_stats - counters, budget use and latency percentiles of
   all jobs completed so far. */
int extract_server_stats(extract_server *srv, extract_stats *st);

/* extract_server_destroy - finish every submitted job, stop the loop and
   free everything. */
int extract_server_destroy(extract_server *srv);

/* extract_destroy - free the context and all device memory it holds
   (synchronises the device first).  NULL is accepted. */
int extract_destroy(extract_ctx *h);

/* extract_last_error - message of the last failure on this thread ("" if
   none); valid until the next failing call on the same thread. */
const char *extract_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EXTRACT_H */
