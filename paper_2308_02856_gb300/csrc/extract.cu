// C ABI of libextract (declared in include/extract.h): context lifetime,
// argument validation, device memory and the composition of the kernels.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>
#include <vector>

namespace ex {

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char *what)
{
    return set_error(e == cudaErrorMemoryAllocation ? EXTRACT_ENOMEM : EXTRACT_ECUDA,
                     "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

double predict_direct_s(uint32_t m, uint32_t k, uint32_t s)
{
    return (double)m * k * ((s + 31) / 32) / 19e12;
}

// The tensor-core product pays for its padded tile: 128 rows x nt
// sub-blocks x 128 K per stage.  0.66 - 0.86 PMAC/s measured with 256
// sub-blocks per tile; narrower tiles spend relatively more on building the
// Toeplitz operand.
double predict_tc_s(uint32_t m, uint32_t k, uint32_t s)
{
    const double nt = tc_tile_n(m);
    const double macs = (double)round_up(k, 128) * (double)round_up(m, (uint64_t)nt) * (double)round_up(s, 128);
    return macs / (8e14 * (0.3 + 0.7 * nt / 256.0)) + 5e-6;
}

double predict_ntt_s(uint32_t m, uint32_t s, uint32_t k, int split_log2, bool per_block_seeds)
{
    const NttShape sh = ntt_shape(s, k, split_log2, per_block_seeds);
    const double N = (double)sh.N;
    const double transforms = (per_block_seeds ? 2.0 : 1.0) * sh.P + 1.0;
    // seconds per cost unit, from the measured hash times of shapes between
    // s = 2^16 and 2^20 (1.9 - 34.7 ms, to within about 20 %)
    return (double)m * ntt_cost_units((uint32_t)transforms, sh.N) * 0.19e-12;
}

}  // namespace ex

using namespace ex;

struct extract_ctx {
    uint64_t n = 0;
    uint32_t m = 0, s = 0, k = 0, flags = 0;
    uint64_t sampling_key = 0;
    int device = 0, num_sms = 0;
    uint32_t w_pad = 0;        // words per stored sub-block (multiple of kWordChunk)
    uint32_t seed_stride = 0;  // words per realigned seed
    uint32_t nseeds = 0;
    uint32_t *perm = nullptr;  // n entries (null with EXTRACT_IDENTITY_PERM; m*s padded slots with
                               // EXTRACT_SAMPLING_IID)
    uint64_t perm_len = 0;     // entries of perm (n, or m*s)
    bool iid = false;          // EXTRACT_SAMPLING_IID: padded order, kNoPos slots read as 0
    std::vector<uint64_t> sizes;  // |S_j| (i.i.d. law; empty for the sorted order)
    uint32_t *arev = nullptr;  // m * w_pad words
    uint32_t *seed = nullptr;  // nseeds * seed_stride words
    uint32_t *stage_in = nullptr;   // extract_run_host staging, ceil(n/32) words
    uint32_t *stage_out = nullptr;  // extract_run_host staging, ceil(m*k/32) words
    HashPlan plan;
    NttPlan *ntt = nullptr;  // set when the NTT method hashes this shape
    bool tc = false;         // the tensor-core direct product hashes this shape
    uint32_t *dev_err = nullptr;  // device error word of the tensor-core kernel (a wait that gave up)
    cudaStream_t aux = nullptr;                       // gather stream of the overlapped NTT run
    cudaEvent_t ev_fork = nullptr, ev_group = nullptr;
    NttLanes lanes;                                   // extra lanes of the NTT hash (own streams, buffers)
    GatherWindows gw;                                 // window-major order for inputs far above L2
    GatherBuckets gb;                                 // bucketed two-stage gather tables
    // extract_run_host with the bucket tables: copies on their own stream,
    // overlapped with stage 1 (input pieces) and the hash (output groups)
    cudaStream_t copy_st = nullptr;
    cudaEvent_t ev_copy0 = nullptr, ev_out_end = nullptr, ev_copy_done = nullptr;
    cudaEvent_t ev_piece[8] = {};
    std::vector<cudaEvent_t> ev_groups;
    // extract_run_host_many: two staging buffers each way, copies in and out
    // on their own streams; stage_in / stage_out serve as buffer 0
    uint32_t *stage_in1 = nullptr, *stage_out1 = nullptr;
    cudaStream_t copy_in_st = nullptr, copy_out_st = nullptr;
    cudaEvent_t ev_many0 = nullptr, ev_in[2] = {}, ev_gathered[2] = {}, ev_hashed[2] = {}, ev_out[2] = {};
};

namespace {

// NTT hash lanes (launch groups dealt round robin over streams)
#ifndef EX_NTT_LANES
#define EX_NTT_LANES 2
#endif
constexpr uint32_t kNttLanes = EX_NTT_LANES;
static_assert(kNttLanes >= 1 && kNttLanes <= (uint32_t)kMaxNttLanes, "NTT lane count");

constexpr uint32_t kKnownFlags = EXTRACT_SEED_PER_SUBBLOCK | EXTRACT_IDENTITY_PERM | EXTRACT_METHOD_DIRECT |
                                  EXTRACT_METHOD_NTT | EXTRACT_SAMPLING_IID | EXTRACT_GATHER_PLAIN |
                                  EXTRACT_GATHER_BUCKETS | EXTRACT_GATHER_WIDE_CHUNKS | (0x3fu << 8) | (0x7u << 16) |
                                  EXTRACT_METHOD_TENSOR | (0xfu << 24) | EXTRACT_TC_TEST_STALL;

// K blocks of 128 per accumulation chunk of the tensor-core product
// (EXTRACT_TC_CHUNK(l): 2^l blocks; default 2^5 = 4096 K per chunk)
constexpr uint32_t kTcChunkLog2Default = 5;

// Smallest input that gets the bucketed gather by default
constexpr uint64_t kBucketsMinBits = 1ull << 22;

void free_ctx(extract_ctx *h)
{
    if (!h) return;
    cudaFree(h->perm);
    cudaFree(h->arev);
    cudaFree(h->seed);
    cudaFree(h->dev_err);
    cudaFree(h->stage_in);
    cudaFree(h->stage_out);
    cudaFree(h->stage_in1);
    cudaFree(h->stage_out1);
    for (cudaStream_t s : {h->copy_in_st, h->copy_out_st})
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t ev : {h->ev_many0, h->ev_in[0], h->ev_in[1], h->ev_gathered[0], h->ev_gathered[1],
                           h->ev_hashed[0], h->ev_hashed[1], h->ev_out[0], h->ev_out[1]})
        if (ev) cudaEventDestroy(ev);
    ntt_destroy(h->ntt);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_group) cudaEventDestroy(h->ev_group);
    if (h->aux) cudaStreamDestroy(h->aux);
    gather_windows_free(&h->gw);
    gather_buckets_free(&h->gb);
    for (cudaEvent_t ev : {h->ev_copy0, h->ev_out_end, h->ev_copy_done})
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : h->ev_piece)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : h->ev_groups)
        if (ev) cudaEventDestroy(ev);
    if (h->copy_st) cudaStreamDestroy(h->copy_st);
    for (int l = 0; l < kMaxNttLanes - 1; ++l) {
        cudaFree(h->lanes.work[l]);
        if (h->lanes.ev_join[l]) cudaEventDestroy(h->lanes.ev_join[l]);
        if (h->lanes.st[l]) cudaStreamDestroy(h->lanes.st[l]);
    }
    if (h->lanes.ev_fork) cudaEventDestroy(h->lanes.ev_fork);
    delete h;
}

// Bits [off, off + len) of a packed string, realigned to start at bit 0 of
// dst (dst_words words, zero past len).
void realign_bits(const uint32_t *src, uint64_t src_words, uint64_t off, uint64_t len,
                  uint32_t *dst, uint64_t dst_words)
{
    std::memset(dst, 0, dst_words * 4);
    const uint64_t w0 = off >> 5;
    const uint32_t sh = (uint32_t)(off & 31u);
    const uint64_t nw = (len + 31) / 32;
    for (uint64_t t = 0; t < nw && t < dst_words; ++t) {
        const uint64_t a = w0 + t;
        uint32_t lo = a < src_words ? src[a] : 0u;
        uint32_t hi = a + 1 < src_words ? src[a + 1] : 0u;
        dst[t] = sh ? ((lo >> sh) | (hi << (32u - sh))) : lo;
    }
    if (len % 32 && nw - 1 < dst_words) dst[nw - 1] &= (1u << (len % 32)) - 1u;
}

int check_ctx(const extract_ctx *h)
{
    if (!h) return set_error(EXTRACT_EINVAL, "null context");
    return EXTRACT_OK;
}

// extract_run_host over the bucket tables.  The input goes up in pieces of
// whole input chunks on the copy stream and stage 1 takes each piece as
// soon as it is in; the NTT hash sends each launch group's finished output
// words down while later groups run (the direct hash's output goes down at
// the end).  Same results as copy in, extract_run, copy out.
int run_host_overlapped(extract_ctx *h, cudaStream_t st, const uint32_t *in_host, uint32_t *out_host)
{
    constexpr uint32_t kPieces = 8;
    if (!h->copy_st) {
        EX_CUDA(cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking));
        EX_CUDA(cudaEventCreateWithFlags(&h->ev_copy0, cudaEventDisableTiming));
        EX_CUDA(cudaEventCreateWithFlags(&h->ev_out_end, cudaEventDisableTiming));
        EX_CUDA(cudaEventCreateWithFlags(&h->ev_copy_done, cudaEventDisableTiming));
        for (cudaEvent_t &ev : h->ev_piece) EX_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        if (h->ntt) {
            h->ev_groups.assign(ceil_div(h->m, ntt_group(h->ntt)), nullptr);
            for (cudaEvent_t &ev : h->ev_groups) EX_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        }
    }
    const uint64_t words = ceil_div(h->n, 32), out_words = ceil_div((uint64_t)h->m * h->k, 32);
    const uint64_t kChunkWords = (1ull << h->gb.clog) / 32;
    EX_CUDA(cudaEventRecord(h->ev_copy0, st));  // after the caller's earlier work on st
    EX_CUDA(cudaStreamWaitEvent(h->copy_st, h->ev_copy0, 0));
    const uint32_t nch = h->gb.nch, np = std::min<uint32_t>(kPieces, nch);
    for (uint32_t i = 0; i < np; ++i) {
        const uint32_t c0 = (uint32_t)((uint64_t)nch * i / np), c1 = (uint32_t)((uint64_t)nch * (i + 1) / np);
        const uint64_t w0 = std::min<uint64_t>(words, c0 * kChunkWords), w1 = std::min<uint64_t>(words, c1 * kChunkWords);
        if (w1 > w0)
            EX_CUDA(cudaMemcpyAsync(h->stage_in + w0, in_host + w0, (w1 - w0) * 4, cudaMemcpyHostToDevice, h->copy_st));
        EX_CUDA(cudaEventRecord(h->ev_piece[i], h->copy_st));
        EX_CUDA(cudaStreamWaitEvent(st, h->ev_piece[i], 0));
        if (int rc = gather_buckets_stage1(h->gb, h->stage_in, h->n, c0, c1, st, h->num_sms)) return rc;
    }
    if (int rc = gather_buckets_stage2(h->gb, h->m, h->w_pad, h->arev, st, h->num_sms)) return rc;
    if (h->ntt) {
        const NttHostOut ho{out_host, h->copy_st, h->ev_groups.data(), (uint32_t)h->ev_groups.size(), h->ev_out_end};
        if (int rc = ntt_hash(h->ntt, h->arev, h->w_pad, h->m, h->s, h->k, h->stage_out, st, nullptr, &h->lanes, &ho))
            return rc;
    } else {
        if (int rc = launch_hash(h->plan, h->seed, h->nseeds > 1 ? h->seed_stride : 0u, h->arev, h->w_pad, h->m, h->k,
                                 h->stage_out, st))
            return rc;
        EX_CUDA(cudaEventRecord(h->ev_out_end, st));
        EX_CUDA(cudaStreamWaitEvent(h->copy_st, h->ev_out_end, 0));
        EX_CUDA(cudaMemcpyAsync(out_host, h->stage_out, out_words * 4, cudaMemcpyDeviceToHost, h->copy_st));
    }
    EX_CUDA(cudaEventRecord(h->ev_copy_done, h->copy_st));
    EX_CUDA(cudaStreamWaitEvent(st, h->ev_copy_done, 0));
    EX_CUDA(cudaStreamSynchronize(st));
    return EXTRACT_OK;
}

}  // namespace

extern "C" {

const char *extract_last_error(void) { return g_err; }

int extract_create(extract_ctx **out, uint64_t n, uint32_t m, uint32_t s, uint32_t k,
                   const uint32_t *seed_bits_host, uint64_t sampling_key, uint32_t flags)
{
    g_err[0] = 0;
    if (!out) return set_error(EXTRACT_EINVAL, "out is null");
    *out = nullptr;
    if (!seed_bits_host) return set_error(EXTRACT_EINVAL, "seed_bits_host is null");
    if (flags & ~kKnownFlags) return set_error(EXTRACT_EINVAL, "unknown flags 0x%x", flags);
    if (m < 1 || s < 1 || k < 1 || k > s)
        return set_error(EXTRACT_EINVAL, "need m >= 1 and 1 <= k <= s (m=%u s=%u k=%u)", m, s, k);
    if (n > (1ull << 32)) return set_error(EXTRACT_EINVAL, "n = %llu exceeds 2^32", (unsigned long long)n);
    const bool per_sub = (flags & EXTRACT_SEED_PER_SUBBLOCK) != 0;
    const bool ident = (flags & EXTRACT_IDENTITY_PERM) != 0;
    const bool iid = (flags & EXTRACT_SAMPLING_IID) != 0;
    if (iid) {
        if (ident) return set_error(EXTRACT_EINVAL, "EXTRACT_SAMPLING_IID and EXTRACT_IDENTITY_PERM are exclusive");
        if (n >= (1ull << 32)) return set_error(EXTRACT_EINVAL, "the i.i.d. law needs n < 2^32");
        if (m > (1u << 16)) return set_error(EXTRACT_EINVAL, "the i.i.d. law needs m <= 2^16 (m = %u)", m);
    } else if ((uint64_t)m * s > n) {
        return set_error(EXTRACT_EINVAL, "m*s = %llu exceeds n = %llu",
                         (unsigned long long)((uint64_t)m * s), (unsigned long long)n);
    }
    if (((flags & EXTRACT_METHOD_DIRECT) != 0) + ((flags & EXTRACT_METHOD_NTT) != 0) +
            ((flags & EXTRACT_METHOD_TENSOR) != 0) > 1)
        return set_error(EXTRACT_EINVAL, "EXTRACT_METHOD_DIRECT, EXTRACT_METHOD_NTT and EXTRACT_METHOD_TENSOR are "
                                         "exclusive");
    if ((flags & EXTRACT_METHOD_TENSOR) && per_sub)
        return set_error(EXTRACT_EINVAL, "EXTRACT_METHOD_TENSOR needs one shared seed");
    if ((flags & EXTRACT_GATHER_PLAIN) && (flags & (EXTRACT_GATHER_BUCKETS | EXTRACT_GATHER_WIDE_CHUNKS)))
        return set_error(EXTRACT_EINVAL, "EXTRACT_GATHER_PLAIN excludes EXTRACT_GATHER_BUCKETS and "
                                         "EXTRACT_GATHER_WIDE_CHUNKS");
    if (ident && (flags & EXTRACT_GATHER_BUCKETS))
        return set_error(EXTRACT_EINVAL, "EXTRACT_GATHER_BUCKETS needs a sampled order (not EXTRACT_IDENTITY_PERM)");
    const uint32_t split_field = (flags >> 16) & 0x7u;
    if (split_field > 5) return set_error(EXTRACT_EINVAL, "EXTRACT_NTT_SPLIT takes 0 .. 4");
    const int split = (int)split_field - 1;  // -1: automatic
    const bool ntt_ok = ntt_shape(s, k, split, per_sub).N != 0;
    if ((flags & EXTRACT_METHOD_NTT) && !ntt_ok)
        return set_error(EXTRACT_EINVAL,
                         "the NTT method needs s+k-1 > 2^11, s < 7*2^26+1 and a split with transform length "
                         "<= 2^22 (>= 2^16 with one seed per sub-block) (s=%u k=%u split=%d)", s, k, split);
    // automatic choice: the least predicted time among the exact methods
    // (the tensor-core product only with a shared seed)
    const uint32_t forced = flags & (EXTRACT_METHOD_DIRECT | EXTRACT_METHOD_NTT | EXTRACT_METHOD_TENSOR);
    const double t_direct = predict_direct_s(m, k, s);
    const double t_ntt = ntt_ok ? predict_ntt_s(m, s, k, split, per_sub) : 1e30;
    const double t_tc = per_sub ? 1e30 : predict_tc_s(m, k, s);
    const bool use_ntt = forced ? (forced == EXTRACT_METHOD_NTT) : (t_ntt < t_direct && t_ntt <= t_tc);
    const bool use_tc = forced ? (forced == EXTRACT_METHOD_TENSOR) : (!use_ntt && t_tc < t_direct);

    extract_ctx *h = new (std::nothrow) extract_ctx();
    if (!h) return set_error(EXTRACT_ENOMEM, "host allocation failed");
    h->n = n; h->m = m; h->s = s; h->k = k; h->flags = flags; h->sampling_key = sampling_key;
    h->iid = iid;
    h->perm_len = ident ? 0 : iid ? (uint64_t)m * s : n;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) { delete h; return cuda_error(e, "device query"); }

    h->w_pad = (uint32_t)round_up(ceil_div(s, 32), kWordChunk);
    h->plan = plan_hash(m, k, h->w_pad, per_sub, h->num_sms);
    if ((uint64_t)h->plan.gx * h->plan.gy >= (1ull << 31)) {
        delete h;
        return set_error(EXTRACT_EINVAL, "too many tiles for one launch (m=%u k=%u)", m, k);
    }
    h->seed_stride = seed_stride_words(h->plan, k, h->w_pad);
    h->nseeds = per_sub ? m : 1u;

    // seeds, realigned to word boundaries and zero padded
    const uint64_t L = (uint64_t)s + k - 1;
    const uint64_t src_words = ceil_div(L * h->nseeds, 32);
    std::vector<uint32_t> host;
    try {
        host.resize((size_t)h->nseeds * h->seed_stride);
    } catch (...) {
        delete h;
        return set_error(EXTRACT_ENOMEM, "host allocation failed");
    }
    for (uint32_t j = 0; j < h->nseeds; ++j)
        realign_bits(seed_bits_host, src_words, (uint64_t)j * L, L, host.data() + (size_t)j * h->seed_stride,
                     h->seed_stride);

    if ((e = cudaMalloc(&h->seed, host.size() * 4)) != cudaSuccess) { free_ctx(h); return cuda_error(e, "cudaMalloc(seed)"); }
    if ((e = cudaMemcpy(h->seed, host.data(), host.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) {
        free_ctx(h); return cuda_error(e, "copy seed");
    }
    if (use_tc) {
        h->tc = true;
        if ((e = cudaMalloc(&h->dev_err, 4)) != cudaSuccess || (e = cudaMemset(h->dev_err, 0, 4)) != cudaSuccess) {
            free_ctx(h);
            return cuda_error(e, "tensor-core error word");
        }
    }
    if (use_ntt) {
        cudaStream_t st;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) { free_ctx(h); return cuda_error(e, "stream"); }
        // independent seeds: keep every sub-block's seed spectrum when it
        // takes at most a quarter of the free device memory (P + 1 transforms
        // per run instead of 2P + 1)
        bool resident = false;
        if (per_sub) {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
                resident = ntt_resident_spectra_words(m, s, k, split) * 4 <= free_b / 4;
        }
        int rc = ntt_create(&h->ntt, m, s, k, h->seed, st, nullptr, split, per_sub ? h->seed_stride : 0, resident);
        cudaStreamDestroy(st);
        if (rc != EXTRACT_OK) { free_ctx(h); return rc; }
        if ((e = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_group, cudaEventDisableTiming)) != cudaSuccess) {
            free_ctx(h);
            return cuda_error(e, "overlap stream");
        }
        const uint32_t groups = (uint32_t)ceil_div(m, ntt_group(h->ntt));
        NttLanes &L = h->lanes;
        L.n = (int)std::min<uint32_t>(kNttLanes - 1, groups - 1);
        if (L.n > 0 && (e = cudaEventCreateWithFlags(&L.ev_fork, cudaEventDisableTiming)) != cudaSuccess) {
            free_ctx(h);
            return cuda_error(e, "NTT lanes");
        }
        for (int l = 0; l < L.n; ++l)
            if ((e = cudaStreamCreateWithFlags(&L.st[l], cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&L.ev_join[l], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaMalloc(&L.work[l], ntt_work_words(m, s, k, split, per_sub) * 4)) != cudaSuccess) {
                free_ctx(h);
                return cuda_error(e, "NTT lanes");
            }
    }
    if ((e = cudaMalloc(&h->arev, (size_t)m * h->w_pad * 4)) != cudaSuccess) { free_ctx(h); return cuda_error(e, "cudaMalloc(sub-blocks)"); }
    if ((e = cudaMemset(h->arev, 0, (size_t)m * h->w_pad * 4)) != cudaSuccess) { free_ctx(h); return cuda_error(e, "memset(sub-blocks)"); }
    if (!ident) {
        if ((e = cudaMalloc(&h->perm, (size_t)std::max<uint64_t>(h->perm_len, 1) * 4)) != cudaSuccess) {
            free_ctx(h);
            return cuda_error(e, "cudaMalloc(order)");
        }
        const uint32_t kb = (flags >> 8) & 0x3fu;
        const uint64_t mask = kb ? ~((1ull << (64u - kb)) - 1ull) : ~0ull;
        cudaStream_t st;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) { free_ctx(h); return cuda_error(e, "stream"); }
        int rc = iid ? build_iid_order(n, sampling_key, mask, m, s, h->perm, &h->sizes, st, h->num_sms)
                     : build_perm(n, sampling_key, mask, h->perm, st, h->num_sms);
        const bool want_buckets = (flags & EXTRACT_GATHER_BUCKETS) ||
                                  (!(flags & EXTRACT_GATHER_PLAIN) && n >= kBucketsMinBits);
        bool have_buckets = false;
        if (rc == EXTRACT_OK && want_buckets) {
            rc = gather_buckets_build(h->perm, n, m, s, h->w_pad, &h->gb, st, h->num_sms,
                                      (flags & EXTRACT_GATHER_WIDE_CHUNKS) != 0);
            if (rc == kBucketsNotEligible) {
                rc = (flags & EXTRACT_GATHER_BUCKETS)
                         ? set_error(EXTRACT_EINVAL, "EXTRACT_GATHER_BUCKETS: the shape does not suit the bucket "
                                                     "tables (n <= 25600 * 2^18, regions within 220 KiB)")
                         : EXTRACT_OK;
            } else {
                have_buckets = rc == EXTRACT_OK;
            }
        }
        if (rc == EXTRACT_OK && !have_buckets && !iid && gather_windows_wanted(n))
            rc = gather_windows_build(h->perm, m, s, h->w_pad, n, &h->gw, st, h->num_sms);
        cudaStreamDestroy(st);
        if (rc != EXTRACT_OK) { free_ctx(h); return rc; }
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) { free_ctx(h); return cuda_error(e, "create"); }
    *out = h;
    return EXTRACT_OK;
}

int extract_gather(extract_ctx *h, void *stream, const uint32_t *in_bits_dev)
{
    if (int rc = check_ctx(h)) return rc;
    if (!in_bits_dev) return set_error(EXTRACT_EINVAL, "in_bits_dev is null");
    if (h->gb.pi)
        return gather_buckets_run(h->gb, in_bits_dev, h->n, h->m, h->w_pad, h->arev, (cudaStream_t)stream, h->num_sms);
    if (h->gw.pos) return gather_windows_run(h->gw, in_bits_dev, h->w_pad, h->arev, (cudaStream_t)stream, h->num_sms);
    return launch_gather(in_bits_dev, h->perm, h->m, h->s, h->w_pad, h->arev, (cudaStream_t)stream,
                         h->num_sms, 0, h->iid, h->n);
}

int extract_hash(extract_ctx *h, void *stream, uint32_t *out_bits_dev)
{
    if (int rc = check_ctx(h)) return rc;
    if (!out_bits_dev) return set_error(EXTRACT_EINVAL, "out_bits_dev is null");
    if (h->ntt)
        return ntt_hash(h->ntt, h->arev, h->w_pad, h->m, h->s, h->k, out_bits_dev, (cudaStream_t)stream, nullptr,
                        &h->lanes);
    if (h->tc) {
        const uint32_t cl = (h->flags >> 24) & 0xfu;
        return launch_hash_tc(h->seed, h->seed_stride, h->arev, h->w_pad, h->m, h->s, h->k, out_bits_dev, h->dev_err,
                              (cudaStream_t)stream, 1u << (cl ? cl - 1 : kTcChunkLog2Default),
                              (h->flags & EXTRACT_TC_TEST_STALL) != 0);
    }
    return launch_hash(h->plan, h->seed, h->nseeds > 1 ? h->seed_stride : 0u, h->arev, h->w_pad, h->m,
                       h->k, out_bits_dev, (cudaStream_t)stream);
}

int extract_run(extract_ctx *h, void *stream, const uint32_t *in_bits_dev, uint32_t *out_bits_dev)
{
    if (int rc = check_ctx(h)) return rc;
    if (!out_bits_dev) return set_error(EXTRACT_EINVAL, "out_bits_dev is null");
    // NTT method: the whole block is gathered first (2^30-bit block 25.4
    // ms/step against 26.7 overlapped), except for large inputs without the
    // window-major order (the i.i.d. law), whose gather waits on DRAM and is
    // overlapped group by group with the transforms.
    if (h->ntt && !h->gw.pos && !h->gb.pi && !gather_prefers_whole_block(h->n)) {
        if (!in_bits_dev) return set_error(EXTRACT_EINVAL, "in_bits_dev is null");
        return ntt_run_overlapped(h->ntt, in_bits_dev, h->perm, h->arev, h->w_pad, h->m, h->s, h->k, out_bits_dev,
                                  (cudaStream_t)stream, h->aux, h->ev_fork, h->ev_group, h->num_sms, h->iid, h->n);
    }
    if (int rc = extract_gather(h, stream, in_bits_dev)) return rc;
    return extract_hash(h, stream, out_bits_dev);
}

int extract_run_host(extract_ctx *h, void *stream, const uint32_t *in_bits_host, uint32_t *out_bits_host)
{
    if (int rc = check_ctx(h)) return rc;
    if (!in_bits_host || !out_bits_host) return set_error(EXTRACT_EINVAL, "null host buffer");
    const size_t in_bytes = ceil_div(h->n, 32) * 4, out_bytes = ceil_div((uint64_t)h->m * h->k, 32) * 4;
    if (!h->stage_in) EX_CUDA(cudaMalloc(&h->stage_in, in_bytes ? in_bytes : 4));
    if (!h->stage_out) EX_CUDA(cudaMalloc(&h->stage_out, out_bytes));
    cudaStream_t st = (cudaStream_t)stream;
    if (h->gb.pi) return run_host_overlapped(h, st, in_bits_host, out_bits_host);
    EX_CUDA(cudaMemcpyAsync(h->stage_in, in_bits_host, in_bytes, cudaMemcpyHostToDevice, st));
    if (int rc = extract_run(h, stream, h->stage_in, h->stage_out)) return rc;
    EX_CUDA(cudaMemcpyAsync(out_bits_host, h->stage_out, out_bytes, cudaMemcpyDeviceToHost, st));
    EX_CUDA(cudaStreamSynchronize(st));
    return EXTRACT_OK;
}

int extract_run_host_many(extract_ctx *h, void *stream, const uint32_t *const *in_bits_host,
                          uint32_t *const *out_bits_host, uint32_t count)
{
    if (int rc = check_ctx(h)) return rc;
    if (!count) return EXTRACT_OK;
    if (!in_bits_host || !out_bits_host) return set_error(EXTRACT_EINVAL, "null pointer array");
    for (uint32_t b = 0; b < count; ++b)
        if (!in_bits_host[b] || !out_bits_host[b]) return set_error(EXTRACT_EINVAL, "null host buffer %u", b);
    const size_t in_bytes = ceil_div(h->n, 32) * 4, out_bytes = ceil_div((uint64_t)h->m * h->k, 32) * 4;
    for (uint32_t **buf : {&h->stage_in, &h->stage_in1})
        if (!*buf) EX_CUDA(cudaMalloc(buf, in_bytes ? in_bytes : 4));
    for (uint32_t **buf : {&h->stage_out, &h->stage_out1})
        if (!*buf) EX_CUDA(cudaMalloc(buf, out_bytes));
    if (!h->copy_in_st) {
        EX_CUDA(cudaStreamCreateWithFlags(&h->copy_in_st, cudaStreamNonBlocking));
        EX_CUDA(cudaStreamCreateWithFlags(&h->copy_out_st, cudaStreamNonBlocking));
        EX_CUDA(cudaEventCreateWithFlags(&h->ev_many0, cudaEventDisableTiming));
        for (int i = 0; i < 2; ++i)
            for (cudaEvent_t *ev : {&h->ev_in[i], &h->ev_gathered[i], &h->ev_hashed[i], &h->ev_out[i]})
                EX_CUDA(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    }
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *const sin[2] = {h->stage_in, h->stage_in1};
    uint32_t *const sout[2] = {h->stage_out, h->stage_out1};
    EX_CUDA(cudaEventRecord(h->ev_many0, st));  // after the caller's earlier work on st
    EX_CUDA(cudaStreamWaitEvent(h->copy_in_st, h->ev_many0, 0));
    EX_CUDA(cudaStreamWaitEvent(h->copy_out_st, h->ev_many0, 0));
    for (uint32_t b = 0; b < count; ++b) {
        const int i = (int)(b & 1u);
        // block b's input into staging buffer i once block b - 2's gather has read it
        if (b >= 2) EX_CUDA(cudaStreamWaitEvent(h->copy_in_st, h->ev_gathered[i], 0));
        EX_CUDA(cudaMemcpyAsync(sin[i], in_bits_host[b], in_bytes, cudaMemcpyHostToDevice, h->copy_in_st));
        EX_CUDA(cudaEventRecord(h->ev_in[i], h->copy_in_st));
        EX_CUDA(cudaStreamWaitEvent(st, h->ev_in[i], 0));
        if (int rc = extract_gather(h, st, sin[i])) return rc;
        EX_CUDA(cudaEventRecord(h->ev_gathered[i], st));
        // its output into staging buffer i once block b - 2's output is in host memory
        if (b >= 2) EX_CUDA(cudaStreamWaitEvent(st, h->ev_out[i], 0));
        if (int rc = extract_hash(h, st, sout[i])) return rc;
        EX_CUDA(cudaEventRecord(h->ev_hashed[i], st));
        EX_CUDA(cudaStreamWaitEvent(h->copy_out_st, h->ev_hashed[i], 0));
        EX_CUDA(cudaMemcpyAsync(out_bits_host[b], sout[i], out_bytes, cudaMemcpyDeviceToHost, h->copy_out_st));
        EX_CUDA(cudaEventRecord(h->ev_out[i], h->copy_out_st));
    }
    EX_CUDA(cudaStreamWaitEvent(st, h->ev_out[(count - 1) & 1u], 0));
    if (count >= 2) EX_CUDA(cudaStreamWaitEvent(st, h->ev_out[count & 1u], 0));
    EX_CUDA(cudaStreamSynchronize(st));
    return EXTRACT_OK;
}

int extract_run_plain(extract_ctx *h, void *stream, const uint32_t *in_bits_dev, uint32_t *out_bits_dev)
{
    if (int rc = check_ctx(h)) return rc;
    if (!out_bits_dev) return set_error(EXTRACT_EINVAL, "out_bits_dev is null");
    if (int rc = extract_gather(h, stream, in_bits_dev)) return rc;
    return launch_hash_plain(h->seed, h->nseeds > 1 ? h->seed_stride : 0u, h->arev, h->w_pad, h->s, h->m,
                             h->k, out_bits_dev, (cudaStream_t)stream);
}

int extract_read_perm(extract_ctx *h, uint64_t start, uint64_t count, uint32_t *dst_host)
{
    if (int rc = check_ctx(h)) return rc;
    if (!dst_host && count) return set_error(EXTRACT_EINVAL, "dst_host is null");
    const uint64_t len = h->perm ? h->perm_len : h->n;
    if (start > len || count > len - start)
        return set_error(EXTRACT_EINVAL, "range [%llu, +%llu) outside the order of %llu entries",
                         (unsigned long long)start, (unsigned long long)count, (unsigned long long)len);
    if (!h->perm) {
        for (uint64_t t = 0; t < count; ++t) dst_host[t] = (uint32_t)(start + t);
        return EXTRACT_OK;
    }
    EX_CUDA(cudaDeviceSynchronize());
    EX_CUDA(cudaMemcpy(dst_host, h->perm + start, count * 4, cudaMemcpyDeviceToHost));
    return EXTRACT_OK;
}

int extract_subblock_sizes(extract_ctx *h, uint64_t *sizes_host)
{
    if (int rc = check_ctx(h)) return rc;
    if (!sizes_host) return set_error(EXTRACT_EINVAL, "sizes_host is null");
    for (uint32_t j = 0; j < h->m; ++j) sizes_host[j] = h->iid ? h->sizes[j] : h->s;
    return EXTRACT_OK;
}

// Eq. 7 (Sec. III.D), restated from the paper for the library: the chance
// that a binomial(N, p) sub-block size exceeds L is at most
// 1 - Phi(sign(L - N p) sqrt(2 N H(L/N, p))), H the binary relative entropy;
// the limit is the smallest L at which m times that bound is <= eps.
static double eq7_tail(uint64_t N, uint64_t L, double p)
{
    const double x = (double)L / (double)N;
    const double h = (x > 0.0 ? x * std::log(x / p) : 0.0) + (x < 1.0 ? (1.0 - x) * std::log((1.0 - x) / (1.0 - p)) : 0.0);
    const double z = (x < p ? -1.0 : 1.0) * std::sqrt(2.0 * (double)N * std::max(h, 0.0));
    return 0.5 * std::erfc(z / std::sqrt(2.0));
}

int extract_block_limit(uint64_t N, uint32_t m, double eps, double p, uint64_t *limit_out)
{
    if (!limit_out) return set_error(EXTRACT_EINVAL, "limit_out is null");
    if (N == 0 || m == 0 || !(p > 0.0 && p < 1.0) || !(eps > 0.0))
        return set_error(EXTRACT_EINVAL, "need N > 0, m > 0, 0 < p < 1 and eps > 0");
    const double target = eps / (double)m;
    if (eq7_tail(N, N, p) > target) {
        *limit_out = N;
        return EXTRACT_OK;
    }
    uint64_t lo = 0, hi = N;  // smallest L in [lo, hi] with eq7_tail(L) <= target
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (eq7_tail(N, mid, p) <= target) hi = mid;
        else lo = mid + 1;
    }
    *limit_out = lo;
    return EXTRACT_OK;
}

int extract_read_subblock(extract_ctx *h, uint32_t j, uint32_t *dst_host)
{
    if (int rc = check_ctx(h)) return rc;
    if (!dst_host) return set_error(EXTRACT_EINVAL, "dst_host is null");
    if (j >= h->m) return set_error(EXTRACT_EINVAL, "sub-block %u >= m = %u", j, h->m);
    EX_CUDA(cudaDeviceSynchronize());
    EX_CUDA(cudaMemcpy(dst_host, h->arev + (size_t)j * h->w_pad, ceil_div(h->s, 32) * 4,
                       cudaMemcpyDeviceToHost));
    return EXTRACT_OK;
}

int extract_describe(extract_ctx *h, char *buf, uint32_t buflen)
{
    if (int rc = check_ctx(h)) return rc;
    if (!buf || !buflen) return set_error(EXTRACT_EINVAL, "empty buffer");
    const HashPlan &p = h->plan;
    char gather[96];
    if (h->gb.pi)
        snprintf(gather, sizeof gather, "gather=buckets (2^%u-bit chunks, %u-word sub-block regions)", h->gb.clog,
                 h->gb.bstride);
    else if (h->gw.pos)
        snprintf(gather, sizeof gather, "gather=windows (%u input windows)", h->gw.R);
    else
        snprintf(gather, sizeof gather, "gather=plain");
    if (h->ntt) {
        snprintf(buf, buflen,
                 "ntt: N=%u (%u x 2048) P=%u pieces per sub-block, %u sub-blocks per launch group, "
                 "prime 7*2^26+1, %s, column pass A %s; sms=%d; %s",
                 ntt_size(h->ntt), ntt_size(h->ntt) / 2048, ntt_pieces(h->ntt), ntt_group(h->ntt),
                 h->nseeds > 1 ? (ntt_spectra_resident(h->ntt) ? "seed spectra resident (one seed per sub-block)"
                                                                : "seed windows transformed per run (one seed per sub-block)")
                               : "shared seed spectrum",
                 ntt_uses_tensor_cores(h->ntt) ? "on the tensor cores (f16 slices of the DFT matrix)" : "by butterflies",
                 h->num_sms, gather);
        return EXTRACT_OK;
    }
    if (h->tc) {
        const uint32_t cl = (h->flags >> 24) & 0xfu;
        snprintf(buf, buflen,
                 "tensor: tcgen05.mma kind::f8f6f4 e4m3 0/1 operands, f32 accumulator, tiles of 128 rows x %u "
                 "sub-blocks, K chunk %u; sms=%d; %s",
                 tc_tile_n(h->m), 128u << (cl ? cl - 1 : kTcChunkLog2Default), h->num_sms, gather);
        return EXTRACT_OK;
    }
    snprintf(buf, buflen,
             "lop3 tile: rows=%u (q=%d x %d warps x 32) subblocks=%d words/chunk=%d grid=%ux%ux%u "
             "(row tiles %u, sub-block tiles %u, split-K %u x %u chunks) w_pad=%u sms=%d; %s",
             p.rows(), p.q, p.warps, p.j, p.wc, p.gx * p.gy, 1u, p.splits, p.gx, p.gy, p.splits, p.cps,
             h->w_pad, h->num_sms, gather);
    return EXTRACT_OK;
}

int extract_status(extract_ctx *h)
{
    if (int rc = check_ctx(h)) return rc;
    if (h->ntt)
        if (int rc = ntt_status(h->ntt)) return rc;
    if (!h->dev_err) return EXTRACT_OK;
    uint32_t v = 0;
    EX_CUDA(cudaDeviceSynchronize());
    EX_CUDA(cudaMemcpy(&v, h->dev_err, 4, cudaMemcpyDeviceToHost));
    if (!v) return EXTRACT_OK;
    EX_CUDA(cudaMemset(h->dev_err, 0, 4));
    return set_error(EXTRACT_ETIMEDOUT, "a tensor-core hash kernel gave up waiting for its multiplies");
}

int extract_gather_bytes(extract_ctx *h, uint64_t *bytes)
{
    if (int rc = check_ctx(h)) return rc;
    if (!bytes) return set_error(EXTRACT_EINVAL, "bytes is null");
    const uint64_t sub = (uint64_t)h->m * h->w_pad * 4;
    if (h->gb.pi) {
        *bytes = gather_buckets_bytes(h->gb, h->n, h->m, h->w_pad);
    } else if (h->gw.pos) {
        *bytes = gather_windows_bytes(h->gw, h->n, h->w_pad);
    } else {
        // order entries of the m*s slots, one 32-byte sector of input per
        // gathered bit (random reads), the sub-block buffer; the order is
        // read again by every window pass
        const uint64_t slots = (uint64_t)h->m * h->s;
        const uint64_t passes = (h->perm && !h->iid && h->n > (1ull << 29) && h->n <= (1ull << 30)) ? 2 : 1;
        *bytes = (h->perm ? passes * slots * 4 : 0) + slots * 32 + sub;
    }
    return EXTRACT_OK;
}

int extract_destroy(extract_ctx *h)
{
    if (!h) return EXTRACT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_ctx(h);
    if (e != cudaSuccess) return cuda_error(e, "destroy");
    return EXTRACT_OK;
}

}  // extern "C"
