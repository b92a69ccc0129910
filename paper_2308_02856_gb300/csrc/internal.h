// Host-side launchers shared between the translation units of libextract.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

namespace ex {

// ---- step 1: the sampled order ------------------------------------------
// Builds perm[0..n) = stable argsort of the Philox sampling labels (index
// tie-break) on `st`, then synchronises it.  `mask` keeps the top label bits
// (all ones unless the test hook is set).  Allocates and frees its own
// scratch.  Returns EXTRACT_OK or a negative code.
int build_perm(uint64_t n, uint64_t sampling_key, uint64_t mask, uint32_t *perm,
               cudaStream_t st, int num_sms);

// start[0..nb) = exclusive prefix sums of cnt[0..nb), start[nb] = total
// (which must equal the sum), on `st`.
int exclusive_scan_counts(const uint32_t *cnt, uint32_t nb, uint64_t total, uint64_t *start, cudaStream_t st);

// Order entry of a padding slot of the i.i.d. law (reads as a 0 bit).
constexpr uint32_t kNoPos = 0xffffffffu;

// The paper's i.i.d. sampling law (iid.cu): sub-block V_i =
// floor(label_i * m / 2^64); order[j*s + c] = the c-th smallest position with
// V_i = j, kNoPos past |S_j|; sizes_out[j] = |S_j|.  EXTRACT_EABORT (order
// untouched) when some |S_j| > s.  Needs n < 2^32.  Synchronises `st`.
int build_iid_order(uint64_t n, uint64_t sampling_key, uint64_t mask, uint32_t m, uint32_t s, uint32_t *order,
                    std::vector<uint64_t> *sizes_out, cudaStream_t st, int num_sms);

// ---- step 1 (gather) ----------------------------------------------------
// arev[j * w_pad + w], for j < m and w < w_pad: bit b of the word is
// in[perm[j*s + s-1-(32w+b)]] when 32w+b < s, else 0 (sub-block j reversed).
// perm == nullptr means the identity order.
// rank0: rank of the first position of sub-block 0 of this launch (arev
// then holds sub-blocks starting at that rank).
// padded: kNoPos entries of perm read as 0 (i.i.d. law).  input_bits: the
// input's length; sorted-order inputs of one to two half-L2 windows are
// gathered in one pass per window (0: one pass).  windows_when_padded: a
// padded order takes the window passes too (padded orders are otherwise
// gathered in one pass: the i.i.d. law's increasing positions read with
// locality).
int launch_gather(const uint32_t *in, const uint32_t *perm, uint32_t m, uint32_t s,
                  uint32_t w_pad, uint32_t *arev, cudaStream_t st, int num_sms, uint64_t rank0 = 0,
                  bool padded = false, uint64_t input_bits = 0, bool windows_when_padded = false);
// True when the gather of an input of this length runs best as one launch
// (at most two windows); larger inputs are better overlapped with hashing.
bool gather_prefers_whole_block(uint64_t input_bits);

// Gather for inputs of more than two 64 MiB windows (gather_windows.cu): the
// order entries of every 1024-bit group of stored sub-block words re-laid by
// input window, so a run takes one pass per window with all random reads in
// L2.  Same words as launch_gather.
struct GatherWindows {
    uint32_t *pos = nullptr;   // groups x 1024 positions, window-major per group
    uint16_t *slot = nullptr;  // their slots in the group (32 t + lane)
    uint16_t *off = nullptr;   // groups x (R + 1) window starts
    uint32_t R = 0;            // windows
    uint64_t groups = 0;       // m * w_pad / 32
};
bool gather_windows_wanted(uint64_t input_bits);
// Builds the re-laid order from the sorted order perm (on st, asynchronous).
int gather_windows_build(const uint32_t *perm, uint32_t m, uint32_t s, uint32_t w_pad, uint64_t input_bits,
                         GatherWindows *gw, cudaStream_t st, int num_sms);
int gather_windows_run(const GatherWindows &gw, const uint32_t *in, uint32_t w_pad, uint32_t *arev, cudaStream_t st,
                       int num_sms);
void gather_windows_free(GatherWindows *gw);
// Device-memory bytes one run of the window-major gather reads and writes by design.
uint64_t gather_windows_bytes(const GatherWindows &gw, uint64_t n, uint32_t w_pad);

// Bucketed two-stage gather (gather_buckets.cu): per sampling key, tables
// that regroup every input chunk's bits by sub-block (stage 1) and then
// permute each sub-block's members in shared memory (stage 2), so a run
// reads the input once and makes no random global reads.  Same words as
// launch_gather.
struct GatherBuckets {
    uint32_t *qc = nullptr;     // chunks + 1: first run word of each chunk
    uint32_t *pi = nullptr;     // 16 (or 32) words per run word: in-chunk positions of its 32 bits
    uint32_t *dst = nullptr;    // run words: word index into B (kNoPos: padding)
    uint32_t *sigma = nullptr;  // m * w_pad * 32: member bit of every stored bit
    uint32_t *B = nullptr;      // m * bstride words: the runs of each sub-block
    uint32_t nch = 0;           // input chunks
    uint32_t clog = 16;         // chunk bits log2 (16: 16-bit pi entries, 18: 32-bit)
    uint32_t bstride = 0;       // words per sub-block region of B
    uint64_t run_words = 0;     // run words over all chunks
};
// Returned by gather_buckets_build when the shape does not suit the tables
// (too many input chunks, a region wider than shared memory, no room); the
// caller keeps the plain gather.
constexpr int kBucketsNotEligible = 1;
// Sub-block j's slots are perm[j s .. j s + s) (either sampling law).
int gather_buckets_build(const uint32_t *perm, uint64_t n, uint32_t m, uint32_t s, uint32_t w_pad, GatherBuckets *gb,
                         cudaStream_t st, int num_sms, bool wide_chunks = false);
int gather_buckets_run(const GatherBuckets &gb, const uint32_t *in, uint64_t n, uint32_t m, uint32_t w_pad,
                       uint32_t *arev, cudaStream_t st, int num_sms);
// The two stages alone: stage 1 over input chunks [c_begin, c_end) (of
// 2^gb.clog bits each), stage 2 over every sub-block.
int gather_buckets_stage1(const GatherBuckets &gb, const uint32_t *in, uint64_t n, uint32_t c_begin, uint32_t c_end,
                          cudaStream_t st, int num_sms);
int gather_buckets_stage2(const GatherBuckets &gb, uint32_t m, uint32_t w_pad, uint32_t *arev, cudaStream_t st,
                          int num_sms);
void gather_buckets_free(GatherBuckets *gb);
// Device-memory bytes one run of the bucketed gather reads and writes by
// design: input, chunk starts, pi, destinations, run words (written and
// read), sigma and the sub-block buffer.
uint64_t gather_buckets_bytes(const GatherBuckets &gb, uint64_t n, uint32_t m, uint32_t w_pad);

// ---- steps 2-3: the Toeplitz product and concatenation ------------------
struct HashPlan {
    int variant = 7;      // tile variant (see hash_tile.cuh)
    int q = 4;            // row groups of 32 per warp (rows per warp = 32 q)
    int j = 32;           // sub-blocks per CTA sharing the seed windows
    int warps = 8;        // warps per CTA, each on its own rows
    int wc = 128;         // words of sub-block data staged per chunk
    uint32_t gx = 0;      // row tiles
    uint32_t gy = 0;      // sub-block tiles
    uint32_t nchunks = 0; // w_pad / wc
    uint32_t cps = 0;     // chunks per split
    uint32_t splits = 0;  // split-K factor (gridDim.z)
    uint32_t rows() const { return (uint32_t)(warps * 32 * q); }
};

// Word layout shared by the gather and the hash kernels.
constexpr uint32_t kWordChunk = 128;

// Pick the tile shape and split for (m, k, w_pad) on `num_sms` SMs.
HashPlan plan_hash(uint32_t m, uint32_t k, uint32_t w_pad, bool per_subblock_seed, int num_sms);

// Seed words each (realigned) seed needs for this plan: the kernels read
// seed word (row >> 5) + w + 1 for every row tile and word chunk.
uint32_t seed_stride_words(const HashPlan &p, uint32_t k, uint32_t w_pad);

// out (ceil(m*k/32) words) is zeroed on `st` and then receives every K_j.
// seed_stride = 0: one shared seed; else seed j starts at seed + j*seed_stride.
int launch_hash(const HashPlan &p, const uint32_t *seed, uint32_t seed_stride,
                const uint32_t *arev, uint32_t w_pad, uint32_t m, uint32_t k,
                uint32_t *out, cudaStream_t st);

// The direct product on the tensor cores (tc_hash.cu): one shared seed of
// seed_words realigned words; out is zeroed on st and receives every K_j;
// err is set to 1 when a kernel wait gave up.  chunk_blocks: K blocks of 128
// summed before each parity read-back.
// test_stall: every CTA first waits on a barrier nothing arrives on, so the
// wait runs out, err is set and the kernel returns (the error path's test).
int launch_hash_tc(const uint32_t *seed, uint64_t seed_words, const uint32_t *arev, uint32_t w_pad, uint32_t m,
                   uint32_t s, uint32_t k, uint32_t *out, uint32_t *err, cudaStream_t st, uint32_t chunk_blocks,
                   bool test_stall = false);
// Sub-blocks per tile of the tensor-core product for m sub-blocks.
uint32_t tc_tile_n(uint32_t m);

// The plain per-block path: one launch per sub-block, one thread per row.
int launch_hash_plain(const uint32_t *seed, uint32_t seed_stride, const uint32_t *arev,
                      uint32_t w_pad, uint32_t s, uint32_t m, uint32_t k, uint32_t *out,
                      cudaStream_t st);

// ---- batching and serving: the persistent multi-job hash kernel ----------
struct BatchJobDev {
    const uint32_t *perm;  // null: identity order
    const uint32_t *in;    // refreshed per run
    uint32_t *out;         // refreshed per run
    const uint32_t *seed;  // realigned seeds
    uint32_t *arev;
    uint64_t groups_before;  // prefix of gather groups (m * w_pad / 32)
    uint64_t outw_before;    // prefix of output words
    uint32_t seed_stride;    // 0: one shared seed
    uint32_t m, s, k, w_pad;
    uint32_t padded;         // 1: the i.i.d. law's padded order (kNoPos reads as 0)
};

// One CTA work item: rows [r0, r0 + rows(variant)) x sub-blocks
// [j0, j0 + J(variant)) x word chunks [c_begin, c_end) of job `job`.
struct BatchTileDev {
    uint32_t job, variant, r0, j0, c_begin, c_end;
};

// GPU nanoseconds per (CTA, 128-word chunk) of each tile variant, measured
// once per device inside the persistent kernel and cached.
int tile_costs(int dev, int sms, const double **ns_per_chunk);

// The variant with the least predicted time (tiles x chunks x cost).
int choose_variant(uint32_t m, uint32_t k, uint32_t w_pad, bool per_sub, const double *ns_per_chunk);

// One CTA per SM pulls tiles[0..ntiles) through *counter (which must be 0).
int launch_batch_hash(const BatchJobDev *jobs, const BatchTileDev *tiles, uint32_t ntiles, uint32_t *counter,
                      int sms, cudaStream_t st);

// ---- exact NTT middle product (ntt.cu) -----------------------------------
struct NttPlan;
// Transform length N, pieces per sub-block P and coefficients per piece h.
// split_log2 < 0 picks P = 2^l (l <= 4) with the least predicted work; N = 0
// when no shape exists (s + k - 1 <= 2^11, s >= the prime, N > 2^22 or
// P N > ntt_max_work_words()).
struct NttShape {
    uint32_t N = 0, P = 1, h = 0;
};
// per_block_seeds: one seed per sub-block (its windows are transformed in
// every run: 2P + 1 transforms per sub-block; N >= 2^16).
NttShape ntt_shape(uint32_t s, uint32_t k, int split_log2 = -1, bool per_block_seeds = false);
bool ntt_eligible(uint32_t s, uint32_t k);
// Words of the work buffer a plan for (m, s, k) uses, and the most any uses.
uint64_t ntt_work_words(uint32_t m, uint32_t s, uint32_t k, int split_log2 = -1, bool per_block_seeds = false);
uint64_t ntt_max_work_words();
// Radix-2 butterflies of one hash of m sub-blocks ((P + 1) transforms each).
double ntt_work_butterflies(uint32_t m, uint32_t s, uint32_t k, int split_log2 = -1, bool per_block_seeds = false);
// Builds the twiddle tables and the seed spectra (synchronous on st).  work:
// a caller-owned buffer of ntt_work_words() words shared by plans that never
// run concurrently, or null to allocate one.
// seed_stride > 0: one seed per sub-block, seed_stride words apart; with
// resident_spectra the spectra of all m sub-blocks' seed windows are built
// here and kept (m P N words), else every run transforms them again.
int ntt_create(NttPlan **out, uint32_t m, uint32_t s, uint32_t k, const uint32_t *seed_dev, cudaStream_t st,
               uint32_t *work = nullptr, int split_log2 = -1, uint64_t seed_stride = 0,
               bool resident_spectra = false);
// Words of the resident per-sub-block spectra (m P N) of a plan for (m, s, k)
// with one seed per sub-block.
uint64_t ntt_resident_spectra_words(uint32_t m, uint32_t s, uint32_t k, int split_log2 = -1);
// True when the plan keeps every sub-block's seed spectrum.
bool ntt_spectra_resident(const NttPlan *p);
// Extra streams and work buffers for ntt_hash: launch group i runs on lane
// i mod (1 + n) (lane 0 = the caller's stream and buffer), so one group's
// passes fill the others' last waves.  Events owned by the caller.
constexpr int kMaxNttLanes = 8;
struct NttLanes {
    int n = 0;  // extra lanes (0 .. kMaxNttLanes - 1)
    cudaStream_t st[kMaxNttLanes - 1] = {};
    uint32_t *work[kMaxNttLanes - 1] = {};  // ntt_work_words() words each
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kMaxNttLanes - 1] = {};
};
// Hashes all m gathered sub-blocks; zeroes and fills out.  work: a buffer
// of ntt_work_words() words to use instead of the plan's own (null: the
// plan's).  lanes: optional extra lanes (ordered after prior work on st and
// joined back into st).
// Host copy of the output while later groups still run: after launch group
// i (and group i - 1, which may share its first word) the words that no
// later group touches go to host on stream st; the rest after the last one.
struct NttHostOut {
    uint32_t *host = nullptr;   // ceil(m k / 32) words
    cudaStream_t st = nullptr;  // copy stream
    cudaEvent_t *ev = nullptr;  // one event per launch group
    uint32_t nev = 0;
    cudaEvent_t ev_end = nullptr;
};
int ntt_hash(const NttPlan *p, const uint32_t *arev, uint32_t w_pad, uint32_t m, uint32_t s, uint32_t k,
             uint32_t *out, cudaStream_t st, uint32_t *work = nullptr, const NttLanes *lanes = nullptr,
             const NttHostOut *host_out = nullptr);
// Gather and hash with the gather of each launch group on `aux` overlapping
// the transforms of the previous group on `st`; ordered after prior work on
// st and fully ordered before later work on st.  ev_fork, ev_group: events
// owned by the caller.
int ntt_run_overlapped(const NttPlan *p, const uint32_t *in, const uint32_t *perm, uint32_t *arev, uint32_t w_pad,
                       uint32_t m, uint32_t s, uint32_t k, uint32_t *out, cudaStream_t st, cudaStream_t aux,
                       cudaEvent_t ev_fork, cudaEvent_t ev_group, int num_sms, bool padded = false,
                       uint64_t input_bits = 0);
void ntt_destroy(NttPlan *p);
// Stream-ordered release (no device-wide synchronisation).
void ntt_destroy_async(NttPlan *p, cudaStream_t st);
// Device bytes a plan holds besides the shared work buffer.
uint64_t ntt_plan_bytes(uint32_t s, uint32_t k, int split_log2 = -1, bool per_block_seeds = false);
// Predicted seconds of the two hashing methods for m sub-blocks (direct: the
// LOP3 rate the tiled kernel reaches; NTT: the measured cost per transformed
// element and stage).
double predict_direct_s(uint32_t m, uint32_t k, uint32_t s);
double predict_ntt_s(uint32_t m, uint32_t s, uint32_t k, int split_log2 = -1, bool per_block_seeds = false);
double predict_tc_s(uint32_t m, uint32_t k, uint32_t s);
// Relative cost of the NTT method's transforms (ntt_shape's and
// predict_ntt_s's unit).
double ntt_cost_units(uint32_t transforms, uint32_t N);
uint32_t ntt_group(const NttPlan *p);
uint32_t ntt_size(const NttPlan *p);
// pass A runs on the tensor cores (transform lengths 2^16 .. 2^18)
bool ntt_uses_tensor_cores(const NttPlan *p);
// the plan's device error word (nonzero: a tensor-core wait gave up)
uint32_t *ntt_error_word(const NttPlan *p);
// EXTRACT_ETIMEDOUT (once) when a tensor-core kernel of the plan gave up on
// a wait since the last call; synchronises the device
int ntt_status(const NttPlan *p);
uint32_t ntt_pieces(const NttPlan *p);

}  // namespace ex
