// Bucketed gather of the sub-blocks (Sec. III.B step 1), in two stages.
//
// The plain gather reads one random input bit per sub-block bit, and every
// such read costs a whole 32-byte sector: the gather is bound by the sector
// rate, not by bytes.  Here, once per sampling key, the fixed map from input
// positions to sub-block slots is compiled into two tables so that a run
// reads every input word once and does its random bit reads in shared
// memory:
//
//   stage 1, per input chunk of 2^16 positions (2^18 when the input has too
//     many 2^16-bit chunks or too short runs; one CTA, the chunk's
//     words in shared memory): the chunk's sampled bits are regrouped by
//     sub-block into runs padded to whole words (the order inside a run is
//     fixed when the tables are built); every run word is stored into that
//     sub-block's region of the run buffer B.  Table: for every run word, the
//     32 in-chunk positions of its bits (16-bit, pairs in one 32-bit word;
//     18-bit fields for 2^18-bit chunks) and the word's place in B.
//   stage 2, per sub-block j (one CTA, B_j in shared memory): B_j holds the
//     members of sub-block j, chunk by chunk; stored bit c of the sub-block
//     is the member sigma_j[c] of B_j.  Table: sigma, one 21-bit index per
//     stored bit (all ones: a zero bit, past s or past |S_j|).
//
// Both tables are read in order (each warp instruction loads 128 contiguous
// bytes), the input and B move once each, and the stored words equal the
// plain gather's: word w of sub-block j has bit l = in[perm[j s + s-1 - c]]
// with c = 32 w + l (0 when c >= s or the slot is padding).
//
// The tables come from the order in five steps: a per-(chunk, sub-block)
// count, two scans (run offsets inside a chunk and inside B_j), the run
// words' destinations, and one CTA per sub-block that places each slot's
// position in its run (pi, first in B's layout) and records where (sigma).
//
// Layouts (a group = 32 consecutive words, lane l = word 32 g + l):
//   pi   [word group g][bit pair b2 < 16][lane]   (bit 2 b2 | bit 2 b2+1 << 16),
//        or [word group g][word i < 18][lane] for 2^18-bit chunks (the
//        lane's 32 positions, 18 bits each, entry b at stream bit 18 b)
//   dst  [run word]                                word index into B, or kNoPos
//   qc   [chunk + 1]                               first run word of a chunk
//                                                  (multiples of 32)
//   sigma[j][word group g][word i < 21][lane]      the lane's 32 member bit
//                                                  indices in B_j, 21 bits each,
//                                                  entry b at stream bit 21 b
//   B    [j][bstride words]
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <vector>

namespace ex {
namespace {

constexpr size_t kAssignSmemMax = 200 * 1024;    // two counters per chunk in shared memory
constexpr size_t kStage2SmemMax = 220 * 1024;    // bytes of B_j a stage-2 CTA holds
constexpr int kStage1Warps = 8;
// sigma entries are 21-bit fields: a lane's 32 entries fill 21 words
constexpr uint32_t kSigBits = 21, kSigMask = (1u << kSigBits) - 1u, kSigNone = kSigMask;
constexpr uint32_t kSigWords = kSigBits;  // 32 entries x 21 bits / 32
static_assert((kStage2SmemMax / 4) * 32 <= kSigNone, "member bit indices must stay below the sentinel");
constexpr int kStage2Warps = 32;
// pi of 2^18-bit chunks: 18-bit in-chunk positions, a run word's 32 in 18 words
constexpr uint32_t kPi18Words = 18, kPi18Mask = (1u << 18) - 1u;

__host__ __device__ __forceinline__ uint32_t words_of(uint32_t bits) { return (bits + 31u) >> 5; }

// One CTA per sub-block: cnt[c * m + j] = #{slots of sub-block j whose
// position lies in chunk c} (a shared-memory histogram over the chunks).
__global__ void __launch_bounds__(1024)
bk_count_kernel(const uint32_t *__restrict__ perm, uint32_t s, uint32_t m, uint32_t nch, uint32_t clog,
                uint32_t *__restrict__ cnt)
{
    extern __shared__ uint32_t hist[];  // nch
    for (uint32_t j = blockIdx.x; j < m; j += gridDim.x) {
        for (uint32_t c = threadIdx.x; c < nch; c += blockDim.x) hist[c] = 0;
        __syncthreads();
        const uint32_t *pj = perm + (size_t)j * s;
        for (uint32_t x = threadIdx.x; x < s; x += blockDim.x) {
            const uint32_t p = __ldcs(pj + x);
            if (p != kNoPos) atomicAdd(&hist[p >> clog], 1u);
        }
        __syncthreads();
        for (uint32_t c = threadIdx.x; c < nch; c += blockDim.x) cnt[(size_t)c * m + j] = hist[c];
        __syncthreads();
    }
}

// Per chunk (one CTA): wpre[c * (m + 1) + j] = run words of sub-blocks < j
// in chunk c; chunk_words[c] = round_up(all of them, 32).
__global__ void __launch_bounds__(1024)
bk_chunk_scan_kernel(const uint32_t *__restrict__ cnt, uint32_t m, uint32_t nch, uint32_t *__restrict__ wpre,
                     uint32_t *__restrict__ chunk_words)
{
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (uint32_t j0 = 0; j0 < m; j0 += blockDim.x) {
            const uint32_t j = j0 + threadIdx.x;
            const uint32_t v = j < m ? words_of(cnt[(size_t)c * m + j]) : 0u;
            uint32_t x = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, x, d);
                if ((int)lane >= d) x += o;
            }
            if (lane == 31) warp_tot[warp] = x;
            __syncthreads();
            uint32_t wb = 0;
            for (uint32_t w = 0; w < warp; ++w) wb += warp_tot[w];
            const uint32_t base = carry;
            if (j < m) wpre[(size_t)c * (m + 1) + j] = base + wb + x - v;
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) carry = base + wb + x;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            wpre[(size_t)c * (m + 1) + m] = carry;
            chunk_words[c] = (carry + 31u) & ~31u;
        }
        __syncthreads();
    }
}

// Per sub-block (one thread): mw[c * m + j] = run words of sub-block j in
// chunks < c; total[j] = all of them.  Loads go 16 chunks ahead.
__global__ void bk_block_scan_kernel(const uint32_t *__restrict__ cnt, uint32_t m, uint32_t nch,
                                     uint32_t *__restrict__ mw, uint32_t *__restrict__ total)
{
    constexpr uint32_t kAhead = 16;
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    uint32_t run = 0;
    for (uint32_t c0 = 0; c0 < nch; c0 += kAhead) {
        uint32_t v[kAhead];
#pragma unroll
        for (uint32_t t = 0; t < kAhead; ++t) v[t] = c0 + t < nch ? cnt[(size_t)(c0 + t) * m + j] : 0u;
#pragma unroll
        for (uint32_t t = 0; t < kAhead; ++t) {
            if (c0 + t < nch) mw[(size_t)(c0 + t) * m + j] = run;
            run += words_of(v[t]);
        }
    }
    total[j] = run;
}

// dst of every run word: chunk c's run of sub-block j, word t -> j * bstride
// + mw[c][j] + t (padding words of a chunk keep kNoPos from the memset).
__global__ void __launch_bounds__(256)
bk_dst_kernel(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ wpre, const uint32_t *__restrict__ mw,
              const uint32_t *__restrict__ qc, uint32_t m, uint32_t nch, uint32_t bstride, uint32_t *__restrict__ dst)
{
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const uint32_t q0 = qc[c];
        for (uint32_t j = threadIdx.x; j < m; j += blockDim.x) {
            const uint32_t nw = words_of(cnt[(size_t)c * m + j]);
            const uint32_t at = q0 + wpre[(size_t)c * (m + 1) + j];
            const uint32_t to = j * bstride + mw[(size_t)c * m + j];
            for (uint32_t t = 0; t < nw; ++t) dst[at + t] = to + t;
        }
    }
}

// One CTA per sub-block places its members: the slot x with position p in
// chunk c takes the next free bit r of the run (c, j) (a shared-memory
// counter per chunk; the order inside a run is whatever the atomics give,
// which is fine because pi and sigma are written from the same choice):
//   pib[32 (j bstride + mw[c][j]) + r] = p mod 2^16   (B-space layout)
//   sigma: stored bit s-1-x of sub-block j        -> 32 mw[c][j] + r.
// pib writes scatter inside the sub-block's region only.
template <typename PiT>
__global__ void __launch_bounds__(1024)
bk_assign_kernel(const uint32_t *__restrict__ perm, uint32_t s, uint32_t m, uint32_t nch, uint32_t clog,
                 uint32_t w_pad, uint32_t bstride, const uint32_t *__restrict__ mw, PiT *__restrict__ pib,
                 uint32_t *__restrict__ sigma)
{
    extern __shared__ uint32_t sm[];  // nch counters, nch run starts (member bits)
    uint32_t *ctr = sm, *start = sm + nch;
    const uint32_t gps = w_pad >> 5;
    for (uint32_t j = blockIdx.x; j < m; j += gridDim.x) {
        for (uint32_t c = threadIdx.x; c < nch; c += blockDim.x) {
            ctr[c] = 0;
            start[c] = mw[(size_t)c * m + j] << 5;
        }
        __syncthreads();
        const uint32_t *pj = perm + (size_t)j * s;
        PiT *pb = pib + (size_t)j * bstride * 32u;
        uint32_t *sg = sigma + (size_t)j * gps * (kSigWords * 32u);
        for (uint32_t x = threadIdx.x; x < s; x += blockDim.x) {
            const uint32_t p = __ldcs(pj + x);
            if (p == kNoPos) continue;
            const uint32_t c = p >> clog;
            const uint32_t mem = start[c] + atomicAdd(&ctr[c], 1u);
            pb[mem] = (PiT)(p & ((1u << clog) - 1u));
            const uint32_t cs = s - 1u - x, wd = cs >> 5;
            // field cs % 32 of the lane's stream: clear the bits where mem
            // has zeros (the tables start as all ones, the sentinel)
            uint32_t *lw = sg + (wd >> 5) * (kSigWords * 32u) + (wd & 31u);
            const uint32_t o = kSigBits * (cs & 31u), zeros = ~mem & kSigMask;
            atomicAnd(lw + (o >> 5) * 32u, ~(zeros << (o & 31u)));
            if ((o & 31u) + kSigBits > 32u) atomicAnd(lw + ((o >> 5) + 1u) * 32u, ~(zeros >> (32u - (o & 31u))));
        }
        __syncthreads();
    }
}

// pi in the stage-1 layout from the B-space entries: run word q with
// destination d takes the 32 entries of B word d (kWords 32-bit words: 16
// for 16-bit entries, 32 for 32-bit ones; padding words: zeros).  With
// 2^18-bit chunks the layout is bk_pi_pack18_kernel's instead.
template <int kWords>
__global__ void __launch_bounds__(256)
bk_pi_kernel(const uint32_t *__restrict__ pib32, const uint32_t *__restrict__ dst, uint64_t run_words,
             uint32_t *__restrict__ pi)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; g < run_words / 32; g += nwarps) {
        const uint32_t d = dst[g * 32u + lane];
        uint4 v[kWords / 4];
#pragma unroll
        for (int i = 0; i < kWords / 4; ++i) v[i] = make_uint4(0u, 0u, 0u, 0u);
        if (d != kNoPos) {
            const uint4 *src = reinterpret_cast<const uint4 *>(pib32 + (size_t)d * kWords);
#pragma unroll
            for (int i = 0; i < kWords / 4; ++i) v[i] = __ldcs(src + i);
        }
        uint32_t *o = pi + g * 32u * kWords + lane;
#pragma unroll
        for (int i = 0; i < kWords / 4; ++i) {
            o[(4 * i + 0) * 32] = v[i].x;
            o[(4 * i + 1) * 32] = v[i].y;
            o[(4 * i + 2) * 32] = v[i].z;
            o[(4 * i + 3) * 32] = v[i].w;
        }
    }
}

// pi for 2^18-bit chunks: the 32 in-chunk positions of a run word (18 bits
// each) packed into 18 words, entry b at stream bit 18 b, so stage 1 reads
// 72 instead of 128 bytes per run word.  Layout [word group g][word i < 18]
// [lane], like sigma's.
__global__ void __launch_bounds__(256)
bk_pi_pack18_kernel(const uint32_t *__restrict__ pib32, const uint32_t *__restrict__ dst, uint64_t run_words,
                    uint32_t *__restrict__ pi)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; g < run_words / 32; g += nwarps) {
        const uint32_t d = dst[g * 32u + lane];
        uint32_t e[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) e[i] = 0u;
        if (d != kNoPos) {
            const uint4 *src = reinterpret_cast<const uint4 *>(pib32 + (size_t)d * 32u);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint4 v = __ldcs(src + i);
                e[4 * i] = v.x & kPi18Mask;
                e[4 * i + 1] = v.y & kPi18Mask;
                e[4 * i + 2] = v.z & kPi18Mask;
                e[4 * i + 3] = v.w & kPi18Mask;
            }
        }
        uint32_t o[kPi18Words];
#pragma unroll
        for (int i = 0; i < (int)kPi18Words; ++i) o[i] = 0u;
#pragma unroll
        for (int b = 0; b < 32; ++b) {
            const int bit = 18 * b, wi = bit >> 5, sh = bit & 31;
            o[wi] |= e[b] << sh;
            if (sh > 14) o[wi + 1] |= e[b] >> (32 - sh);
        }
        uint32_t *out = pi + g * 32u * kPi18Words + lane;
#pragma unroll
        for (int i = 0; i < (int)kPi18Words; ++i) out[i * 32] = o[i];
    }
}

// Stage 1: one chunk of 2^kLog bits per CTA iteration; one warp per group of
// 32 run words.  pi entries: 16-bit pairs (kLog = 16) or 18-bit fields
// (kLog = 18).
template <int kLog>
__global__ void __launch_bounds__(kStage1Warps * 32)
bk_stage1_kernel(const uint32_t *__restrict__ in, uint64_t in_words, const uint32_t *__restrict__ pi,
                 const uint32_t *__restrict__ dst, const uint32_t *__restrict__ qc, uint32_t c_begin, uint32_t c_end,
                 uint32_t *__restrict__ B)
{
    constexpr uint32_t kWords = (1u << kLog) / 32;          // chunk words
    constexpr int kPiWords = kLog <= 16 ? 16 : (int)kPi18Words;  // pi words per run word
    __shared__ __align__(16) uint32_t cw[kWords];
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const bool aligned = (reinterpret_cast<uintptr_t>(in) & 15u) == 0;
    for (uint32_t c = c_begin + blockIdx.x; c < c_end; c += gridDim.x) {
        const uint64_t w0 = (uint64_t)c * kWords;
        if (aligned && w0 + kWords <= in_words) {
            const uint4 *src = reinterpret_cast<const uint4 *>(in + w0);
            for (uint32_t t = threadIdx.x; t < kWords / 4; t += blockDim.x)
                reinterpret_cast<uint4 *>(cw)[t] = __ldcs(src + t);
        } else {
            for (uint32_t t = threadIdx.x; t < kWords; t += blockDim.x)
                cw[t] = w0 + t < in_words ? __ldcs(in + w0 + t) : 0u;
        }
        __syncthreads();
        const uint32_t g0 = qc[c] >> 5, g1 = qc[c + 1] >> 5;
        for (uint32_t g = g0 + w; g < g1; g += kStage1Warps) {
            const uint32_t *pg = pi + (size_t)g * kPiWords * 32u + lane;
            uint32_t pr[kPiWords];
#pragma unroll
            for (int i = 0; i < kPiWords; ++i) pr[i] = __ldcs(pg + i * 32);
            const uint32_t to = __ldcs(dst + (size_t)g * 32u + lane);
            uint32_t word = 0;
            if (kPiWords == 16) {
#pragma unroll
                for (int b2 = 0; b2 < kPiWords; ++b2) {
                    const uint32_t lo = pr[b2] & 0xffffu, hi = pr[b2] >> 16;
                    word |= ((cw[lo >> 5] >> (lo & 31u)) & 1u) << (2 * b2);
                    word |= ((cw[hi >> 5] >> (hi & 31u)) & 1u) << (2 * b2 + 1);
                }
            } else {
#pragma unroll
                for (int b = 0; b < 32; ++b) {
                    const int bit = 18 * b, wi = bit >> 5, sh = bit & 31;
                    uint32_t p = pr[wi] >> sh;
                    if (sh > 14) p |= pr[wi + 1] << (32 - sh);
                    p &= kPi18Mask;
                    word |= ((cw[p >> 5] >> (p & 31u)) & 1u) << b;
                }
            }
            if (to != kNoPos) B[to] = word;
        }
        __syncthreads();
    }
}

// Stage 2: one sub-block per CTA iteration (B_j in shared memory); one warp
// per group of 32 stored words.
__global__ void __launch_bounds__(kStage2Warps * 32)
bk_stage2_kernel(const uint32_t *__restrict__ B, uint32_t bstride, const uint32_t *__restrict__ sigma, uint32_t m,
                 uint32_t w_pad, uint32_t *__restrict__ arev)
{
    extern __shared__ __align__(16) uint32_t bj[];  // bstride words
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t gps = w_pad >> 5;
    for (uint32_t j = blockIdx.x; j < m; j += gridDim.x) {
        const uint4 *src = reinterpret_cast<const uint4 *>(B + (size_t)j * bstride);
        for (uint32_t t = threadIdx.x; t < bstride / 4; t += blockDim.x) reinterpret_cast<uint4 *>(bj)[t] = __ldcs(src + t);
        __syncthreads();
        for (uint32_t g = w; g < gps; g += kStage2Warps) {
            const uint32_t *sg = sigma + ((size_t)j * gps + g) * (kSigWords * 32u) + lane;
            uint32_t u[kSigWords];
#pragma unroll
            for (int i = 0; i < (int)kSigWords; ++i) u[i] = __ldcs(sg + i * 32);
            uint32_t word = 0;
#pragma unroll
            for (int b = 0; b < 32; ++b) {
                constexpr uint32_t kB = kSigBits;
                const uint32_t o = kB * b, i = o >> 5, sh = o & 31u;
                uint32_t v = u[i] >> sh;
                if (sh + kB > 32u) v |= u[i + 1] << (32u - sh);
                v &= kSigMask;
                if (v != kSigNone) word |= ((bj[v >> 5] >> (v & 31u)) & 1u) << b;
            }
            __stcs(arev + (size_t)j * w_pad + (size_t)g * 32u + lane, word);
        }
        __syncthreads();
    }
}

}  // namespace

namespace {

// The tables for chunks of 2^clog bits (16: 16-bit pi entries; 18: 32-bit).
int build_tables(const uint32_t *perm, uint64_t n, uint32_t m, uint32_t s, uint32_t w_pad, uint32_t clog,
                 GatherBuckets *gb, cudaStream_t st, int num_sms)
{
    gather_buckets_free(gb);
    const uint32_t nch = (uint32_t)ceil_div(n, 1ull << clog);
    if ((size_t)nch * 8 > kAssignSmemMax || (uint64_t)nch * (m + 1) >= (1ull << 32)) return kBucketsNotEligible;
    const uint32_t pi_words = clog <= 16 ? 16 : kPi18Words;  // 32-bit words of pi per run word
    const uint32_t pib_words = clog <= 16 ? 16 : 32;         // the same in the B-space staging copy
    uint32_t *cnt = nullptr, *wpre = nullptr, *mw = nullptr, *cwords = nullptr, *total = nullptr;
    uint32_t *pib = nullptr;
    int rc = EXTRACT_OK;
    cudaError_t e = cudaSuccess;
    auto fail = [&](int code) { if (rc == EXTRACT_OK) rc = code; };
    do {
        if ((e = cudaMallocAsync(&cnt, (size_t)nch * m * 4, st)) != cudaSuccess ||
            (e = cudaMallocAsync(&wpre, (size_t)nch * (m + 1) * 4, st)) != cudaSuccess ||
            (e = cudaMallocAsync(&mw, (size_t)nch * m * 4, st)) != cudaSuccess ||
            (e = cudaMallocAsync(&cwords, (size_t)(nch + 1) * 4, st)) != cudaSuccess ||
            (e = cudaMallocAsync(&total, (size_t)m * 4, st)) != cudaSuccess) {
            cudaGetLastError();
            fail(kBucketsNotEligible);  // no room for the tables
            break;
        }
        if ((e = cudaFuncSetAttribute(bk_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(nch * 4))) !=
            cudaSuccess) { fail(cuda_error(e, "smem attribute")); break; }
        bk_count_kernel<<<std::min<uint32_t>(m, (uint32_t)num_sms * 2), 1024, nch * 4, st>>>(perm, s, m, nch, clog, cnt);
        bk_chunk_scan_kernel<<<std::min<uint32_t>(nch, (uint32_t)num_sms * 2), 1024, 0, st>>>(cnt, m, nch, wpre, cwords);
        bk_block_scan_kernel<<<(uint32_t)ceil_div(m, 128), 128, 0, st>>>(cnt, m, nch, mw, total);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(cuda_error(e, "bucket scans")); break; }
        // host: the chunk starts (qc) and the widest sub-block region
        std::vector<uint32_t> hw(nch), ht(m);
        if ((e = cudaMemcpyAsync(hw.data(), cwords, (size_t)nch * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(ht.data(), total, (size_t)m * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) { fail(cuda_error(e, "bucket sizes")); break; }
        const uint32_t widest = *std::max_element(ht.begin(), ht.end());
        const uint32_t bstride = std::max<uint32_t>(4, (widest + 3u) & ~3u);
        if ((size_t)bstride * 4 > kStage2SmemMax) { fail(kBucketsNotEligible); break; }  // B_j too wide
        std::vector<uint32_t> hq(nch + 1);
        uint64_t q = 0;
        for (uint32_t c = 0; c < nch; ++c) {
            hq[c] = (uint32_t)q;
            q += hw[c];
        }
        if (q >= (1ull << 32) || (uint64_t)m * bstride >= (1ull << 32)) { fail(kBucketsNotEligible); break; }
        hq[nch] = (uint32_t)q;
        gb->nch = nch;
        gb->clog = clog;
        gb->bstride = bstride;
        gb->run_words = q;
        const uint64_t sig_len = (uint64_t)m * w_pad * kSigWords;  // 21-bit fields, 32 per 21 words
        const size_t pib_bytes = (size_t)m * bstride * 4 * pib_words;
        if ((e = cudaMalloc(&gb->qc, (size_t)(nch + 1) * 4)) != cudaSuccess ||
            (e = cudaMalloc(&gb->pi, std::max<uint64_t>(q, 1) * 4 * pi_words)) != cudaSuccess ||
            (e = cudaMalloc(&gb->dst, std::max<uint64_t>(q, 1) * 4)) != cudaSuccess ||
            (e = cudaMalloc(&gb->sigma, sig_len * 4)) != cudaSuccess ||
            (e = cudaMalloc(&gb->B, (size_t)m * bstride * 4)) != cudaSuccess ||
            (e = cudaMallocAsync(&pib, pib_bytes, st)) != cudaSuccess) {
            cudaGetLastError();
            fail(kBucketsNotEligible);  // no room for the tables
            break;
        }
        if ((e = cudaMemcpyAsync(gb->qc, hq.data(), (size_t)(nch + 1) * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(gb->dst, 0xff, std::max<uint64_t>(q, 1) * 4, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(gb->sigma, 0xff, sig_len * 4, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(gb->B, 0, (size_t)m * bstride * 4, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(pib, 0, pib_bytes, st)) != cudaSuccess) {
            fail(cuda_error(e, "bucket tables init"));
            break;
        }
        bk_dst_kernel<<<std::min<uint32_t>(nch, (uint32_t)num_sms * 8), 256, 0, st>>>(cnt, wpre, mw, gb->qc, m, nch,
                                                                                 bstride, gb->dst);
        if ((e = cudaFuncSetAttribute(bk_assign_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(nch * 8))) != cudaSuccess ||
            (e = cudaFuncSetAttribute(bk_assign_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(nch * 8))) != cudaSuccess) { fail(cuda_error(e, "smem attribute")); break; }
        // one sub-block per SM at a time (a cap at about 128 MB of regions in
        // flight, to keep the scattered pib writes in L2, measured slower:
        // 100.6 against 96.3 ms of create at n = 2^30)
        const uint32_t agrid = std::min<uint32_t>(m, (uint32_t)num_sms);
        const uint32_t pgrid = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(1, q / 256), (uint64_t)num_sms * 16);
        if (pi_words == 16) {
            bk_assign_kernel<uint16_t><<<agrid, 1024, nch * 8, st>>>(perm, s, m, nch, clog, w_pad, bstride, mw,
                                                                    reinterpret_cast<uint16_t *>(pib), gb->sigma);
            bk_pi_kernel<16><<<pgrid, 256, 0, st>>>(pib, gb->dst, q, gb->pi);
        } else {
            bk_assign_kernel<uint32_t><<<agrid, 1024, nch * 8, st>>>(perm, s, m, nch, clog, w_pad, bstride, mw, pib,
                                                                    gb->sigma);
            bk_pi_pack18_kernel<<<pgrid, 256, 0, st>>>(pib, gb->dst, q, gb->pi);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(cuda_error(e, "bucket tables")); break; }
        if ((e = cudaFuncSetAttribute(bk_stage2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kStage2SmemMax)) != cudaSuccess) { fail(cuda_error(e, "smem attribute")); break; }
    } while (0);
    for (void *ptr : {(void *)cnt, (void *)wpre, (void *)mw, (void *)cwords, (void *)total, (void *)pib})
        if (ptr) cudaFreeAsync(ptr, st);
    const cudaError_t se = cudaStreamSynchronize(st);
    if (rc == EXTRACT_OK && se != cudaSuccess) rc = cuda_error(se, "bucket gather build");
    if (rc != EXTRACT_OK) gather_buckets_free(gb);
    return rc;
}

}  // namespace

int gather_buckets_build(const uint32_t *perm, uint64_t n, uint32_t m, uint32_t s, uint32_t w_pad, GatherBuckets *gb,
                         cudaStream_t st, int num_sms, bool wide_chunks)
{
    gather_buckets_free(gb);
    if (n > (1ull << 32) || w_pad % 32u || n == 0) return kBucketsNotEligible;
    // 2^16-bit chunks (16-bit pi entries) unless they are too many or leave
    // runs so short that a sub-block's padded runs overflow shared memory;
    // then 2^18-bit chunks (32-bit entries, four times longer runs)
    int rc = wide_chunks ? kBucketsNotEligible : build_tables(perm, n, m, s, w_pad, 16, gb, st, num_sms);
    if (rc == kBucketsNotEligible) rc = build_tables(perm, n, m, s, w_pad, 18, gb, st, num_sms);
    return rc;
}

int gather_buckets_stage1(const GatherBuckets &gb, const uint32_t *in, uint64_t n, uint32_t c_begin, uint32_t c_end,
                          cudaStream_t st, int num_sms)
{
    if (c_end <= c_begin) return EXTRACT_OK;
    const uint32_t grid = std::min<uint32_t>(c_end - c_begin, (uint32_t)num_sms * 8);
    if (gb.clog == 16)
        bk_stage1_kernel<16><<<grid, kStage1Warps * 32, 0, st>>>(in, ceil_div(n, 32), gb.pi, gb.dst, gb.qc, c_begin,
                                                                 c_end, gb.B);
    else
        bk_stage1_kernel<18><<<grid, kStage1Warps * 32, 0, st>>>(in, ceil_div(n, 32), gb.pi, gb.dst, gb.qc, c_begin,
                                                                 c_end, gb.B);
    EX_LAUNCH("bk_stage1_kernel");
    return EXTRACT_OK;
}

int gather_buckets_stage2(const GatherBuckets &gb, uint32_t m, uint32_t w_pad, uint32_t *arev, cudaStream_t st,
                          int num_sms)
{
    bk_stage2_kernel<<<std::min<uint32_t>(m, (uint32_t)num_sms), kStage2Warps * 32, (size_t)gb.bstride * 4, st>>>(
        gb.B, gb.bstride, gb.sigma, m, w_pad, arev);
    EX_LAUNCH("bk_stage2_kernel");
    return EXTRACT_OK;
}

int gather_buckets_run(const GatherBuckets &gb, const uint32_t *in, uint64_t n, uint32_t m, uint32_t w_pad,
                       uint32_t *arev, cudaStream_t st, int num_sms)
{
    if (int rc = gather_buckets_stage1(gb, in, n, 0, gb.nch, st, num_sms)) return rc;
    return gather_buckets_stage2(gb, m, w_pad, arev, st, num_sms);
}

uint64_t gather_buckets_bytes(const GatherBuckets &gb, uint64_t n, uint32_t m, uint32_t w_pad)
{
    const uint64_t q = gb.run_words, pi_words = gb.clog <= 16 ? 16 : kPi18Words;
    const uint64_t stage1 = ceil_div(n, 32) * 4 + (uint64_t)(gb.nch + 1) * 4 + q * 4 * pi_words + q * 4  // in, qc, pi, dst
                            + q * 4;                                                                      // run words to B
    const uint64_t stage2 = q * 4 + (uint64_t)m * w_pad * kSigWords * 4 + (uint64_t)m * w_pad * 4;        // B, sigma, arev
    return stage1 + stage2;
}

void gather_buckets_free(GatherBuckets *gb)
{
    cudaFree(gb->qc);
    cudaFree(gb->pi);
    cudaFree(gb->dst);
    cudaFree(gb->sigma);
    cudaFree(gb->B);
    *gb = GatherBuckets{};
}

}  // namespace ex
