// Step 1 of the sub-block protocol (Sec. III.B, "Sampling"): the sampled
// order of the n input positions, perm = stable argsort of 64-bit Philox
// labels with the lower position first on equal labels.
//
// GPU design (no sort library): the labels are never stored; every pass
// recomputes them from the position with Philox, which keeps the device
// footprint at the 4n-byte order itself.
//   1. histogram of the top b label bits (b = ceil(log2 n) - 10, so a bucket
//      holds about 512-1024 positions);
//   2. exclusive scan of the bucket counts;
//   3. scatter of every position into its bucket (any order inside it);
//   4. one CTA per bucket sorts it in shared memory by (label, position):
//      a counting pass on the next 10 label bits, then insertion sort of
//      each of those small bins;
//   5. buckets too large for shared memory (only possible when the
//      test hook forces equal labels) are ranked by all-pairs comparison.
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace ex {
namespace {

constexpr int kSortCap = 2048;      // positions per bucket sorted in smem
constexpr int kSubBits = 10;        // counting-pass digit inside a bucket
constexpr int kSubBins = 1 << kSubBits;
constexpr int kSortThreads = 256;
constexpr int kScanPerBlock = 4096; // elements per scan block (1024 x 4)

__device__ __forceinline__ uint32_t bucket_of(uint64_t label, int b)
{
    return b ? (uint32_t)(label >> (64 - b)) : 0u;
}

__global__ void perm_hist_kernel(uint64_t n, uint2 key, uint64_t mask, int b, uint32_t *cnt)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        atomicAdd(&cnt[bucket_of(sampling_label(i, key, mask), b)], 1u);
}

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

__global__ void perm_scatter_kernel(uint64_t n, uint2 key, uint64_t mask, int b,
                                    const uint64_t *start, uint32_t *fill, uint32_t *perm)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t bk = bucket_of(sampling_label(i, key, mask), b);
        const uint64_t pos = start[bk] + atomicAdd(&fill[bk], 1u);
        perm[pos] = (uint32_t)i;
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

// One CTA per bucket (grid-stride over buckets).  Shared memory:
//   k1, k2: labels (2 x cap x 8 B), i1, i2: positions (2 x cap x 4 B),
//   hist, cur: counting-pass bins.
__global__ void __launch_bounds__(kSortThreads)
perm_local_sort_kernel(uint32_t nb, int b, uint2 key, uint64_t mask, const uint64_t *start,
                       uint32_t *perm, uint32_t *big_list, uint32_t *big_count)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *k1 = reinterpret_cast<uint64_t *>(smem);
    uint64_t *k2 = k1 + kSortCap;
    uint32_t *i1 = reinterpret_cast<uint32_t *>(k2 + kSortCap);
    uint32_t *i2 = i1 + kSortCap;
    uint32_t *hist = i2 + kSortCap;         // kSubBins + 1
    uint32_t *cur = hist + kSubBins + 1;    // kSubBins
    __shared__ uint64_t warp_tot[32];

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
        for (uint32_t e = threadIdx.x; e < L; e += blockDim.x) {
            const uint32_t idx = perm[lo + e];
            const uint64_t lab = sampling_label(idx, key, mask);
            k1[e] = lab;
            i1[e] = idx;
            atomicAdd(&hist[sub_digit(lab, b)], 1u);
        }
        __syncthreads();
        // exclusive scan of the kSubBins counts, 4 per thread
        {
            uint32_t v[4];
            uint32_t tsum = 0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                v[t] = hist[threadIdx.x * 4 + t];
                tsum += v[t];
            }
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            uint32_t x = tsum;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += o;
            }
            if (lane == 31) warp_tot[warp] = x;
            __syncthreads();
            uint32_t wbase = 0;
            for (int w = 0; w < warp; ++w) wbase += (uint32_t)warp_tot[w];
            uint32_t run = wbase + x - tsum;
            __syncthreads();
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                hist[threadIdx.x * 4 + t] = run;
                run += v[t];
            }
            if (threadIdx.x == 0) hist[kSubBins] = (uint32_t)L;
        }
        __syncthreads();
        for (uint32_t e = threadIdx.x; e < L; e += blockDim.x) {
            const uint64_t lab = k1[e];
            const uint32_t d = sub_digit(lab, b);
            const uint32_t p = hist[d] + atomicAdd(&cur[d], 1u);
            k2[p] = lab;
            i2[p] = i1[e];
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kSubBins; d += blockDim.x) {
            const uint32_t a = hist[d], z = hist[d + 1];
            for (uint32_t x = a + 1; x < z; ++x) {
                const uint64_t kx = k2[x];
                const uint32_t ix = i2[x];
                uint32_t y = x;
                while (y > a && less_pair(kx, ix, k2[y - 1], i2[y - 1])) {
                    k2[y] = k2[y - 1];
                    i2[y] = i2[y - 1];
                    --y;
                }
                k2[y] = kx;
                i2[y] = ix;
            }
        }
        __syncthreads();
        for (uint32_t e = threadIdx.x; e < L; e += blockDim.x) perm[lo + e] = i2[e];
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
    const uint32_t nb = 1u << b;
    const uint2 key = make_uint2((uint32_t)sampling_key, (uint32_t)(sampling_key >> 32));
    const uint32_t nblk = (uint32_t)ceil_div(nb, kScanPerBlock);

    uint32_t *cnt = nullptr, *big_list = nullptr, *big_count = nullptr;
    uint64_t *start = nullptr, *bsum = nullptr;
    int rc = EXTRACT_OK;
    auto fail = [&](int code) { rc = code; };
    do {
        cudaError_t e;
        if ((e = cudaMallocAsync(&cnt, sizeof(uint32_t) * nb, st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm hist)")); break; }
        if ((e = cudaMallocAsync(&start, sizeof(uint64_t) * (nb + 1), st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm start)")); break; }
        if ((e = cudaMallocAsync(&bsum, sizeof(uint64_t) * nblk, st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm bsum)")); break; }
        if ((e = cudaMallocAsync(&big_list, sizeof(uint32_t) * nb, st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm big)")); break; }
        if ((e = cudaMallocAsync(&big_count, sizeof(uint32_t), st)) != cudaSuccess) { fail(cuda_error(e, "cudaMalloc(perm bigc)")); break; }
        if ((e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * nb, st)) != cudaSuccess) { fail(cuda_error(e, "memset")); break; }
        if ((e = cudaMemsetAsync(big_count, 0, sizeof(uint32_t), st)) != cudaSuccess) { fail(cuda_error(e, "memset")); break; }

        const uint32_t grid = (uint32_t)std::min<uint64_t>(ceil_div(n, 256), (uint64_t)num_sms * 16);
        perm_hist_kernel<<<grid, 256, 0, st>>>(n, key, mask, b, cnt);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(cuda_error(e, "perm_hist_kernel")); break; }
        scan_blocks_kernel<<<nblk, 1024, 0, st>>>(cnt, nb, start, bsum);
        scan_bsum_kernel<<<1, 1024, 0, st>>>(bsum, nblk);
        scan_add_kernel<<<(uint32_t)ceil_div(nb, 256), 256, 0, st>>>(start, nb, bsum, n);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(cuda_error(e, "perm scan")); break; }
        if ((e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * nb, st)) != cudaSuccess) { fail(cuda_error(e, "memset")); break; }
        perm_scatter_kernel<<<grid, 256, 0, st>>>(n, key, mask, b, start, cnt, perm);
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(cuda_error(e, "perm_scatter_kernel")); break; }

        const size_t smem = (size_t)kSortCap * (8 + 8 + 4 + 4) + (size_t)(2 * kSubBins + 1) * 4;
        if ((e = cudaFuncSetAttribute(perm_local_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess) { fail(cuda_error(e, "smem attr")); break; }
        const uint32_t sgrid = std::min<uint32_t>(nb, (uint32_t)num_sms * 8);
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
    if (cnt) cudaFreeAsync(cnt, st);
    if (start) cudaFreeAsync(start, st);
    if (bsum) cudaFreeAsync(bsum, st);
    if (big_list) cudaFreeAsync(big_list, st);
    if (big_count) cudaFreeAsync(big_count, st);
    cudaError_t fe = cudaStreamSynchronize(st);
    if (rc == EXTRACT_OK && fe != cudaSuccess) rc = cuda_error(fe, "perm build");
    return rc;
}

}  // namespace ex
