// Step 1 of the sub-block protocol (Sec. III.B, "Sampling"): the sampled
// order of the n input positions, perm = stable argsort of 64-bit Philox
// labels with the lower position first on equal labels.
//
// GPU design (no sort library): the labels are never stored; every pass
// recomputes them from the position with Philox.  The order is an MSD sort
// on the top b = ceil(log2 n) - 10 label bits (buckets of about 512-1024
// positions) finished by a sort inside each bucket:
//   1. a histogram of the top C <= 10 label bits (coarse bins) in shared
//      memory per CTA;
//   2. coarse scatter: each CTA sorts a tile of 8192 positions by coarse bin
//      in shared memory and writes one contiguous run per bin (coalesced),
//      reserving its place in the bin with one atomic per (tile, bin);
//   3. fine pass, one CTA per coarse bin: a shared-memory histogram of the
//      next b - C bits, then the scatter of the bin's positions into their
//      buckets; a coarse bin spans at most a few MB of the order, so these
//      random writes stay in L2;
//   4. one CTA per bucket sorts it in shared memory by (label, position):
//      a counting pass on the next 10 label bits, then insertion sort of
//      each of those small bins;
//   5. buckets too large for shared memory (only possible when the
//      test hook forces equal labels) are ranked by all-pairs comparison.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <vector>

namespace ex {
namespace {

constexpr int kSortCap = 2048;      // positions per bucket sorted in smem
constexpr int kSubBits = 8;         // counting-pass digit inside a bucket (== kSortThreads bins)
constexpr int kSubBins = 1 << kSubBits;
constexpr int kSortThreads = 256;
constexpr int kScanPerBlock = 4096; // elements per scan block (1024 x 4)

// Inclusive scan of one value per thread across a block of 1024 threads.
__device__ __forceinline__ uint64_t block_inclusive_scan(uint64_t v, uint64_t *warp_tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint64_t t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t o = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += o;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    if (warp > 0) v += warp_tot[warp - 1];
    return v;
}

// start[i] = exclusive prefix of cnt within the block; bsum[block] = total.
__global__ void __launch_bounds__(1024) scan_blocks_kernel(const uint32_t *cnt, uint32_t nb,
                                                           uint64_t *start, uint64_t *bsum)
{
    __shared__ uint64_t warp_tot[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanPerBlock + threadIdx.x * 4u;
    uint64_t v[4];
    uint64_t tsum = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        v[t] = (base + t < nb) ? cnt[base + t] : 0u;
        tsum += v[t];
    }
    const uint64_t incl = block_inclusive_scan(tsum, warp_tot);
    uint64_t run = incl - tsum;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (base + t < nb) start[base + t] = run;
        run += v[t];
    }
    if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = incl;
}

// Exclusive scan of the block sums in place (one block, any count).
__global__ void __launch_bounds__(1024) scan_bsum_kernel(uint64_t *bsum, uint32_t nblk)
{
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nblk; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint64_t v = i < nblk ? bsum[i] : 0;
        const uint64_t incl = block_inclusive_scan(v, warp_tot);
        const uint64_t c = carry;
        if (i < nblk) bsum[i] = c + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + incl;
        __syncthreads();
    }
}

__global__ void scan_add_kernel(uint64_t *start, uint32_t nb, const uint64_t *bsum, uint64_t n)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < nb) start[i] += bsum[i / kScanPerBlock];
    if (i == 0) start[nb] = n;
}

constexpr int kCoarseMax = 10;              // coarse bins: at most 1024
constexpr uint32_t kCoarseBins = 1u << kCoarseMax;
constexpr int kTileThreads = 512;
constexpr int kTilePerThread = 16;
constexpr uint32_t kTile = kTileThreads * kTilePerThread;  // positions per coarse-scatter tile
constexpr int kFineThreads = 1024;

__device__ __forceinline__ uint32_t coarse_of(uint64_t label, int C)
{
    return C ? (uint32_t)(label >> (64 - C)) : 0u;
}
__device__ __forceinline__ uint32_t fine_of(uint64_t label, int C, int F)
{
    return F ? (uint32_t)((label << C) >> (64 - F)) : 0u;
}

// ccnt[d] += #{i : coarse digit d}
__global__ void __launch_bounds__(512) perm_coarse_hist_kernel(uint64_t n, uint2 key, uint64_t mask, int C,
                                                               uint32_t *ccnt)
{
    __shared__ uint32_t h[kCoarseBins];
    for (uint32_t d = threadIdx.x; d < kCoarseBins; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        atomicAdd(&h[coarse_of(sampling_label(i, key, mask), C)], 1u);
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < (1u << C); d += blockDim.x)
        if (h[d]) atomicAdd(&ccnt[d], h[d]);
}

// Exclusive scan of kCoarseBins values (2 per thread, 512 threads) in place;
// returns nothing, tot: scratch of 16 words.
__device__ __forceinline__ void scan_coarse_bins(uint32_t *v, uint32_t *tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t a = v[2 * threadIdx.x], b = v[2 * threadIdx.x + 1];
    uint32_t x = a + b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += o;
    }
    if (lane == 31) tot[warp] = x;
    __syncthreads();
    uint32_t base = 0;
    for (int w = 0; w < warp; ++w) base += tot[w];
    const uint32_t excl = base + x - (a + b);
    __syncthreads();
    v[2 * threadIdx.x] = excl;
    v[2 * threadIdx.x + 1] = excl + a;
    __syncthreads();
}

// Coarse scatter: tile t holds positions [t kTile, (t+1) kTile); they are
// sorted by coarse digit in shared memory and each digit's run is written
// to tmp[cstart[d] + (the run's reserved offset in bin d)].
__global__ void __launch_bounds__(kTileThreads) perm_coarse_scatter_kernel(uint64_t n, uint2 key, uint64_t mask,
                                                                           int C, const uint64_t *cstart,
                                                                           uint32_t *cfill, uint32_t *tmp)
{
    __shared__ uint32_t cnt[kCoarseBins], tstart[kCoarseBins], gbase[kCoarseBins], tot[16];
    extern __shared__ uint32_t sorted_pos[];  // kTile positions, then kTile 16-bit digits
    uint16_t *sorted_dig = reinterpret_cast<uint16_t *>(sorted_pos + kTile);
    const uint32_t nbins = 1u << C;
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t i0 = t * kTile;
        const uint32_t cnt_t = (uint32_t)min((uint64_t)kTile, n - i0);
        for (uint32_t d = threadIdx.x; d < kCoarseBins; d += blockDim.x) cnt[d] = 0;
        __syncthreads();
        uint16_t dig[kTilePerThread], rnk[kTilePerThread];
#pragma unroll
        for (int q = 0; q < kTilePerThread; ++q) {
            const uint32_t e = threadIdx.x + q * kTileThreads;
            if (e < cnt_t) {
                const uint32_t d = coarse_of(sampling_label(i0 + e, key, mask), C);
                dig[q] = (uint16_t)d;
                rnk[q] = (uint16_t)atomicAdd(&cnt[d], 1u);
            }
        }
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < kCoarseBins; d += blockDim.x) {
            tstart[d] = cnt[d];
            gbase[d] = (d < nbins && cnt[d]) ? atomicAdd(&cfill[d], cnt[d]) : 0u;
        }
        __syncthreads();
        scan_coarse_bins(tstart, tot);
#pragma unroll
        for (int q = 0; q < kTilePerThread; ++q) {
            const uint32_t e = threadIdx.x + q * kTileThreads;
            if (e < cnt_t) {
                const uint32_t at = tstart[dig[q]] + rnk[q];
                sorted_pos[at] = (uint32_t)(i0 + e);
                sorted_dig[at] = dig[q];
            }
        }
        __syncthreads();
        for (uint32_t u = threadIdx.x; u < cnt_t; u += blockDim.x) {
            const uint32_t d = sorted_dig[u];
            tmp[cstart[d] + gbase[d] + (u - tstart[d])] = sorted_pos[u];
        }
        __syncthreads();
    }
}

// Fine pass: CTA per coarse bin c (grid-stride).  The bin's positions
// tmp[cstart[c] .. cstart[c+1]) go to their buckets (c << F) + f, whose
// starts it also writes (start[bucket] = first rank of the bucket).
__global__ void __launch_bounds__(kFineThreads) perm_fine_kernel(uint2 key, uint64_t mask, int C, int F,
                                                                 const uint64_t *cstart, const uint32_t *tmp,
                                                                 uint64_t *start, uint32_t *perm)
{
    extern __shared__ uint32_t fsm[];  // hist[1 << F], fill[1 << F]
    __shared__ uint64_t warp_tot[32];
    const uint32_t nf = 1u << F;
    uint32_t *hist = fsm, *fill = fsm + nf;
    for (uint32_t c = blockIdx.x; c < (1u << C); c += gridDim.x) {
        const uint64_t lo = cstart[c], L = cstart[c + 1] - lo;
        for (uint32_t f = threadIdx.x; f < nf; f += blockDim.x) {
            hist[f] = 0;
            fill[f] = 0;
        }
        __syncthreads();
        for (uint64_t e = threadIdx.x; e < L; e += blockDim.x)
            atomicAdd(&hist[fine_of(sampling_label(tmp[lo + e], key, mask), C, F)], 1u);
        __syncthreads();
        // exclusive scan of nf (<= 4 * blockDim) counts, 4 per thread
        {
            uint32_t v[4], tsum = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t f = threadIdx.x * 4 + q;
                v[q] = f < nf ? hist[f] : 0u;
                tsum += v[q];
            }
            const uint64_t incl = block_inclusive_scan(tsum, warp_tot);
            uint32_t run = (uint32_t)(incl - tsum);
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t f = threadIdx.x * 4 + q;
                if (f < nf) {
                    hist[f] = run;
                    start[((uint64_t)c << F) + f] = lo + run;
                }
                run += v[q];
            }
        }
        __syncthreads();
        for (uint64_t e = threadIdx.x; e < L; e += blockDim.x) {
            const uint32_t pos = tmp[lo + e];
            const uint32_t f = fine_of(sampling_label(pos, key, mask), C, F);
            perm[lo + hist[f] + atomicAdd(&fill[f], 1u)] = pos;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ bool less_pair(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib)
{
    return ka < kb || (ka == kb && ia < ib);
}

__device__ __forceinline__ uint32_t sub_digit(uint64_t label, int b)
{
    return (uint32_t)((label << b) >> (64 - kSubBits));
}

// One CTA per bucket (grid-stride over buckets).  Each thread keeps its
// (up to kSortCap / kSortThreads) entries in registers; shared memory holds
// only the counting-pass bins and the binned copy k2 / i2, so 8 CTAs fit on
// an SM.  A counting pass on the next kSubBits label bits leaves about 4
// entries per bin; each entry's rank inside its bin by (label, position)
// then places it directly.
__global__ void __launch_bounds__(kSortThreads)
perm_local_sort_kernel(uint32_t nb, int b, uint2 key, uint64_t mask, const uint64_t *start,
                       uint32_t *perm, uint32_t *big_list, uint32_t *big_count)
{
    constexpr int kPer = kSortCap / kSortThreads;
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *k2 = reinterpret_cast<uint64_t *>(smem);
    uint32_t *i2 = reinterpret_cast<uint32_t *>(k2 + kSortCap);
    uint32_t *hist = i2 + kSortCap;         // kSubBins + 1
    uint32_t *cur = hist + kSubBins + 1;    // kSubBins
    __shared__ uint32_t warp_tot[kSortThreads / 32];

    for (uint32_t bk = blockIdx.x; bk < nb; bk += gridDim.x) {
        const uint64_t lo = start[bk];
        const uint64_t L = start[bk + 1] - lo;
        if (L <= 1) continue;
        if (L > (uint64_t)kSortCap) {
            if (threadIdx.x == 0) big_list[atomicAdd(big_count, 1u)] = bk;
            continue;
        }
        for (int t = threadIdx.x; t < kSubBins; t += blockDim.x) {
            hist[t] = 0;
            cur[t] = 0;
        }
        __syncthreads();
        uint64_t lab[kPer];
        uint32_t idx[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t e = threadIdx.x + q * kSortThreads;
            if (e < L) {
                idx[q] = perm[lo + e];
                lab[q] = sampling_label(idx[q], key, mask);
                atomicAdd(&hist[sub_digit(lab[q], b)], 1u);
            }
        }
        __syncthreads();
        // exclusive scan of the kSubBins (== kSortThreads) counts
        {
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            const uint32_t v = hist[threadIdx.x];
            uint32_t x = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += o;
            }
            if (lane == 31) warp_tot[warp] = x;
            __syncthreads();
            uint32_t wbase = 0;
            for (int w = 0; w < warp; ++w) wbase += warp_tot[w];
            __syncthreads();
            hist[threadIdx.x] = wbase + x - v;
            if (threadIdx.x == 0) hist[kSubBins] = (uint32_t)L;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t e = threadIdx.x + q * kSortThreads;
            if (e < L) {
                const uint32_t d = sub_digit(lab[q], b);
                const uint32_t p = hist[d] + atomicAdd(&cur[d], 1u);
                k2[p] = lab[q];
                i2[p] = idx[q];
            }
        }
        __syncthreads();
        // every entry's place: its bin's start plus the number of entries of
        // the bin that sort before it (positions are distinct, so no ties);
        // all reads of this bucket's perm entries happened before the barriers
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t e = threadIdx.x + q * kSortThreads;
            if (e < L) {
                const uint32_t d = sub_digit(lab[q], b);
                const uint32_t a = hist[d], z = hist[d + 1];
                uint32_t rank = 0;
                for (uint32_t f = a; f < z; ++f) rank += less_pair(k2[f], i2[f], lab[q], idx[q]) ? 1u : 0u;
                perm[lo + a + rank] = idx[q];
            }
        }
        __syncthreads();
    }
}

// ---- fallback for buckets larger than kSortCap -----------------------------
__global__ void big_load_kernel(const uint32_t *perm_seg, uint64_t L, uint2 key, uint64_t mask,
                                uint64_t *lab, uint32_t *idx)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < L; e += stride) {
        const uint32_t p = perm_seg[e];
        idx[e] = p;
        lab[e] = sampling_label(p, key, mask);
    }
}

// rank(e) = #{f : (lab[f], idx[f]) < (lab[e], idx[e])}; dst[rank] = idx[e].
__global__ void __launch_bounds__(256) big_rank_kernel(const uint64_t *lab, const uint32_t *idx,
                                                       uint64_t L, uint32_t *dst)
{
    __shared__ uint64_t tk[256];
    __shared__ uint32_t ti[256];
    const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const bool live = e < L;
    const uint64_t ke = live ? lab[e] : 0;
    const uint32_t ie = live ? idx[e] : 0;
    uint64_t rank = 0;
    for (uint64_t base = 0; base < L; base += 256) {
        const uint64_t f = base + threadIdx.x;
        if (f < L) {
            tk[threadIdx.x] = lab[f];
            ti[threadIdx.x] = idx[f];
        }
        __syncthreads();
        const uint32_t cnt = (uint32_t)((L - base) < 256 ? (L - base) : 256);
        if (live)
            for (uint32_t t = 0; t < cnt; ++t) rank += less_pair(tk[t], ti[t], ke, ie) ? 1u : 0u;
        __syncthreads();
    }
    if (live) dst[rank] = ie;
}

int ceil_log2_u64(uint64_t n)
{
    int l = 0;
    while ((1ull << l) < n) ++l;
    return l;
}

}  // namespace

int exclusive_scan_counts(const uint32_t *cnt, uint32_t nb, uint64_t total, uint64_t *start, cudaStream_t st)
{
    const uint32_t nblk = (uint32_t)ceil_div(nb, kScanPerBlock);
    uint64_t *bsum = nullptr;
    cudaError_t e = cudaMallocAsync(&bsum, sizeof(uint64_t) * std::max<uint32_t>(nblk, 1), st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(scan)");
    scan_blocks_kernel<<<nblk, 1024, 0, st>>>(cnt, nb, start, bsum);
    scan_bsum_kernel<<<1, 1024, 0, st>>>(bsum, nblk);
    scan_add_kernel<<<(uint32_t)ceil_div((uint64_t)nb + 1, 256), 256, 0, st>>>(start, nb, bsum, total);
    e = cudaGetLastError();
    cudaFreeAsync(bsum, st);
    return e == cudaSuccess ? EXTRACT_OK : cuda_error(e, "scan kernels");
}

int build_perm(uint64_t n, uint64_t sampling_key, uint64_t mask, uint32_t *perm,
               cudaStream_t st, int num_sms)
{
    if (n == 0) return EXTRACT_OK;
    int b = ceil_log2_u64(n) - 10;
    if (b < 0) b = 0;
    if (b > 22) b = 22;
    const int C = std::min(b, kCoarseMax), F = b - C;
    const uint32_t nb = 1u << b, ncb = 1u << C;
    const uint2 key = make_uint2((uint32_t)sampling_key, (uint32_t)(sampling_key >> 32));

    uint32_t *ccnt = nullptr, *cfill = nullptr, *tmp = nullptr, *big_list = nullptr, *big_count = nullptr;
    uint64_t *start = nullptr, *cstart = nullptr;
    int rc = EXTRACT_OK;
    auto fail = [&](int code) { rc = code; };
    do {
        cudaError_t e;
        if ((e = cudaMallocAsync(&ccnt, sizeof(uint32_t) * kCoarseBins * 2, st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm coarse)")); break; }
        cfill = ccnt + kCoarseBins;
        if ((e = cudaMallocAsync(&cstart, sizeof(uint64_t) * (kCoarseBins + 1), st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm cstart)")); break; }
        if ((e = cudaMallocAsync(&start, sizeof(uint64_t) * (nb + 1), st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm start)")); break; }
        if ((e = cudaMallocAsync(&tmp, sizeof(uint32_t) * n, st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm tmp)")); break; }
        if ((e = cudaMallocAsync(&big_list, sizeof(uint32_t) * nb, st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm big)")); break; }
        if ((e = cudaMallocAsync(&big_count, sizeof(uint32_t), st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm bigc)")); break; }
        if ((e = cudaMemsetAsync(ccnt, 0, sizeof(uint32_t) * kCoarseBins * 2, st)) != cudaSuccess) { fail(cuda_error(e, "memset")); break; }
        if ((e = cudaMemsetAsync(big_count, 0, sizeof(uint32_t), st)) != cudaSuccess) { fail(cuda_error(e, "memset")); break; }

        // 1. coarse histogram, scanned on the host (1024 values)
        const uint32_t hgrid = (uint32_t)std::min<uint64_t>(ceil_div(n, 512), (uint64_t)num_sms * 4);
        perm_coarse_hist_kernel<<<hgrid, 512, 0, st>>>(n, key, mask, C, ccnt);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(cuda_error(e, "perm_coarse_hist_kernel")); break; }
        std::vector<uint32_t> hc(ncb);
        std::vector<uint64_t> hs(kCoarseBins + 1, n);
        if ((e = cudaMemcpyAsync(hc.data(), ccnt, sizeof(uint32_t) * ncb, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) { fail(cuda_error(e, "perm coarse counts")); break; }
        uint64_t run = 0;
        for (uint32_t d = 0; d < ncb; ++d) {
            hs[d] = run;
            run += hc[d];
        }
        if (run != n) { fail(set_error(EXTRACT_EINTERNAL, "perm: coarse counts sum to %llu, not n", (unsigned long long)run)); break; }
        if ((e = cudaMemcpyAsync(cstart, hs.data(), sizeof(uint64_t) * (kCoarseBins + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(start + nb, &n, sizeof(uint64_t), cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            fail(cuda_error(e, "perm coarse starts"));
            break;
        }
        // 2. coarse scatter in tiles
        const size_t tsmem = (size_t)kTile * (4 + 2);
        if ((e = cudaFuncSetAttribute(perm_coarse_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)tsmem)) != cudaSuccess) { fail(cuda_error(e, "smem attr")); break; }
        const uint32_t tgrid = (uint32_t)std::min<uint64_t>(ceil_div(n, kTile), (uint64_t)num_sms * 3);
        perm_coarse_scatter_kernel<<<tgrid, kTileThreads, tsmem, st>>>(n, key, mask, C, cstart, cfill, tmp);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(cuda_error(e, "perm_coarse_scatter_kernel")); break; }
        // 3. fine pass, one CTA per coarse bin
        perm_fine_kernel<<<ncb, kFineThreads, sizeof(uint32_t) * 2 * (1u << F), st>>>(key, mask, C, F, cstart, tmp,
                                                                                      start, perm);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(cuda_error(e, "perm_fine_kernel")); break; }
        cudaFreeAsync(tmp, st);
        tmp = nullptr;

        const size_t smem = (size_t)kSortCap * (8 + 4) + (size_t)(2 * kSubBins + 1) * 4;
        if ((e = cudaFuncSetAttribute(perm_local_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess) { fail(cuda_error(e, "smem attr")); break; }
        const uint32_t sgrid = std::min<uint32_t>(nb, (uint32_t)num_sms * 16);
        perm_local_sort_kernel<<<sgrid, kSortThreads, smem, st>>>(nb, b, key, mask, start, perm,
                                                                  big_list, big_count);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(cuda_error(e, "perm_local_sort_kernel")); break; }

        uint32_t nbig = 0;
        if ((e = cudaMemcpyAsync(&nbig, big_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess) { fail(cuda_error(e, "read big count")); break; }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { fail(cuda_error(e, "perm build")); break; }
        if (nbig == 0) break;

        // rare path: all-pairs ranking of the oversized buckets
        uint32_t *blist = new uint32_t[nbig];
        if ((e = cudaMemcpyAsync(blist, big_list, sizeof(uint32_t) * nbig, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            delete[] blist; fail(cuda_error(e, "read big list")); break;
        }
        for (uint32_t t = 0; t < nbig && rc == EXTRACT_OK; ++t) {
            uint64_t se[2];
            if ((e = cudaMemcpyAsync(se, start + blist[t], sizeof(se), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess) { fail(cuda_error(e, "read bucket")); break; }
            const uint64_t L = se[1] - se[0];
            uint64_t *lab = nullptr;
            uint32_t *idx = nullptr, *dst = nullptr;
            if (cudaMallocAsync(&lab, L * 8, st) != cudaSuccess || cudaMallocAsync(&idx, L * 4, st) != cudaSuccess ||
                cudaMallocAsync(&dst, L * 4, st) != cudaSuccess) {
                if (lab) cudaFreeAsync(lab, st);
                if (idx) cudaFreeAsync(idx, st);
                if (dst) cudaFreeAsync(dst, st);
                fail(set_error(EXTRACT_ENOMEM, "perm: no memory for an oversized bucket of %llu",
                               (unsigned long long)L));
                break;
            }
            big_load_kernel<<<(uint32_t)std::min<uint64_t>(ceil_div(L, 256), 65535), 256, 0, st>>>(
                perm + se[0], L, key, mask, lab, idx);
            big_rank_kernel<<<(uint32_t)ceil_div(L, 256), 256, 0, st>>>(lab, idx, L, dst);
            cudaMemcpyAsync(perm + se[0], dst, L * 4, cudaMemcpyDeviceToDevice, st);
            cudaFreeAsync(lab, st);
            cudaFreeAsync(idx, st);
            cudaFreeAsync(dst, st);
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) fail(cuda_error(e, "oversized bucket rank"));
        }
        delete[] blist;
    } while (0);
    // stream-ordered frees: no device-wide synchronisation, so an order can
    // be built while other streams keep hashing
    if (ccnt) cudaFreeAsync(ccnt, st);
    if (cstart) cudaFreeAsync(cstart, st);
    if (tmp) cudaFreeAsync(tmp, st);
    if (start) cudaFreeAsync(start, st);
    if (big_list) cudaFreeAsync(big_list, st);
    if (big_count) cudaFreeAsync(big_count, st);
    cudaError_t fe = cudaStreamSynchronize(st);
    if (rc == EXTRACT_OK && fe != cudaSuccess) rc = cuda_error(fe, "perm build");
    return rc;
}

}  // namespace ex
