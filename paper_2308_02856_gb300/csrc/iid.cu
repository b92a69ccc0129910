// The paper's own sampling law (Sec. III.B step 1): position i joins
// sub-block V_i = floor(label_i * m / 2^64), an i.i.d. uniform draw on
// [0, m) from the same 64-bit Philox label as the sorted order; sub-block j
// is the input at S_j = {i : V_i = j} in increasing position order (the
// order in which the paper's hardware stores sampled bits, Sec. IV),
// zero-padded to the block size limit s = L_S^UB, and the protocol aborts
// when some |S_j| > s (Sec. III.D).
//
// The result is an order of m*s slots in the layout of the sorted order
// (slot j*s + c = the c-th position of S_j, or kNoPos past |S_j|), so the
// gather and both hashing methods run on it unchanged.  Built without a
// sort, from positions cut into chunks of kChunk:
//   1. per chunk, a shared-memory histogram of V -> count[j * nchunks + c];
//   2. an exclusive scan of the counts (j-major) gives every (bin, chunk)
//      its first slot inside the bin, and the bin sizes;
//   3. the host checks the sizes against s (abort) and fills the order with
//      kNoPos;
//   4. one warp per chunk walks its positions in increasing order, 32 at a
//      time: lanes with equal V find each other with a match, take ranks
//      among themselves, and a per-bin counter in shared memory (started at
//      the chunk's first rank in the bin) carries the rank across steps, so
//      each bin's positions land in increasing order.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <vector>

namespace ex {
namespace {

constexpr uint32_t kChunk = 1u << 16;      // positions per chunk (one warp in the scatter)
constexpr uint32_t kSmemBins = 16384;      // bins kept in shared memory by the count pass
constexpr int kCountThreads = 512;

__device__ __forceinline__ uint32_t iid_label(uint64_t label, uint32_t m)
{
    return (uint32_t)__umul64hi(label, (uint64_t)m);
}

// count[j * nchunks + c] = #{i in chunk c : V_i = j}
__global__ void __launch_bounds__(kCountThreads)
iid_count_kernel(uint64_t n, uint2 key, uint64_t mask, uint32_t m, uint32_t nchunks, uint32_t *count)
{
    extern __shared__ uint32_t hist[];  // m bins when m <= kSmemBins
    const bool in_smem = m <= kSmemBins;
    for (uint32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        if (in_smem) {
            for (uint32_t j = threadIdx.x; j < m; j += blockDim.x) hist[j] = 0;
            __syncthreads();
        }
        const uint64_t i0 = (uint64_t)c * kChunk, i1 = min(n, i0 + kChunk);
        for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const uint32_t j = iid_label(sampling_label(i, key, mask), m);
            if (in_smem) atomicAdd(&hist[j], 1u);
            else atomicAdd(&count[(size_t)j * nchunks + c], 1u);
        }
        if (in_smem) {
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < m; j += blockDim.x) count[(size_t)j * nchunks + c] = hist[j];
            __syncthreads();
        }
    }
}

// sizes[j] = start[(j + 1) * nchunks] - start[j * nchunks]
__global__ void iid_sizes_kernel(const uint64_t *start, uint32_t m, uint32_t nchunks, uint64_t *sizes)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
        sizes[j] = start[(size_t)(j + 1) * nchunks] - start[(size_t)j * nchunks];
}

// One warp per chunk (kWarps per CTA, each with m counters in shared memory).
template <int kWarps>
__global__ void __launch_bounds__(kWarps * 32)
iid_scatter_kernel(uint64_t n, uint2 key, uint64_t mask, uint32_t m, uint32_t nchunks, const uint64_t *start,
                   uint32_t s, uint32_t *order)
{
    extern __shared__ uint32_t ctr_all[];  // kWarps x m
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *ctr = ctr_all + (size_t)w * m;
    const uint32_t below = (1u << lane) - 1u;
    for (uint32_t c = blockIdx.x * kWarps + w; c < nchunks; c += gridDim.x * kWarps) {
        // ctr[j]: rank inside bin j of the chunk's next position with V = j
        for (uint32_t j = lane; j < m; j += 32)
            ctr[j] = (uint32_t)(start[(size_t)j * nchunks + c] - start[(size_t)j * nchunks]);
        __syncwarp();
        const uint64_t i0 = (uint64_t)c * kChunk, i1 = min(n, i0 + kChunk);
        for (uint64_t b = i0; b < i1; b += 32) {
            const uint64_t i = b + lane;
            const bool live = i < i1;
            // dead lanes take bin m, which no live lane has
            const uint32_t j = live ? iid_label(sampling_label(i, key, mask), m) : m;
            const uint32_t peers = __match_any_sync(0xffffffffu, j);
            const uint32_t base = live ? ctr[j] : 0u;
            __syncwarp();
            if (live) {
                order[(uint64_t)j * s + base + __popc(peers & below)] = (uint32_t)i;
                if ((peers & below) == 0) ctr[j] = base + __popc(peers);  // the lowest lane of each bin
            }
            __syncwarp();
        }
        __syncwarp();
    }
}

}  // namespace

int build_iid_order(uint64_t n, uint64_t sampling_key, uint64_t mask, uint32_t m, uint32_t s, uint32_t *order,
                    std::vector<uint64_t> *sizes_out, cudaStream_t st, int num_sms)
{
    sizes_out->assign(m, 0);
    if (n == 0) return EXTRACT_OK;
    const uint32_t nchunks = (uint32_t)ceil_div(n, kChunk);
    const uint64_t nb = (uint64_t)m * nchunks;
    if (nb >= (1ull << 31)) return set_error(EXTRACT_EINVAL, "i.i.d. sampling: m x chunks = %llu too large",
                                             (unsigned long long)nb);
    const uint2 key = make_uint2((uint32_t)sampling_key, (uint32_t)(sampling_key >> 32));
    uint32_t *count = nullptr;
    uint64_t *start = nullptr, *sizes = nullptr;
    int rc = EXTRACT_OK;
    do {
        cudaError_t e;
        if ((e = cudaMallocAsync(&count, nb * 4, st)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(iid counts)"); break; }
        if ((e = cudaMallocAsync(&start, (nb + 1) * 8, st)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(iid starts)"); break; }
        if ((e = cudaMallocAsync(&sizes, (size_t)m * 8, st)) != cudaSuccess) { rc = cuda_error(e, "cudaMalloc(iid sizes)"); break; }
        if (m > kSmemBins && (e = cudaMemsetAsync(count, 0, nb * 4, st)) != cudaSuccess) { rc = cuda_error(e, "memset"); break; }
        const size_t hsmem = m <= kSmemBins ? (size_t)m * 4 : 0;
        if ((e = cudaFuncSetAttribute(iid_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)std::max<size_t>(hsmem, 1))) != cudaSuccess) { rc = cuda_error(e, "smem attribute"); break; }
        iid_count_kernel<<<std::min<uint32_t>(nchunks, (uint32_t)num_sms * 4), kCountThreads, hsmem, st>>>(
            n, key, mask, m, nchunks, count);
        if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_error(e, "iid_count_kernel"); break; }
        if ((rc = exclusive_scan_counts(count, (uint32_t)nb, n, start, st)) != EXTRACT_OK) break;
        iid_sizes_kernel<<<(uint32_t)ceil_div(m, 256), 256, 0, st>>>(start, m, nchunks, sizes);
        if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_error(e, "iid_sizes_kernel"); break; }
        if ((e = cudaMemcpyAsync(sizes_out->data(), sizes, (size_t)m * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_error(e, "iid sizes"); break; }
        uint32_t worst = 0;
        for (uint32_t j = 1; j < m; ++j)
            if ((*sizes_out)[j] > (*sizes_out)[worst]) worst = j;
        if ((*sizes_out)[worst] > s) {
            rc = set_error(EXTRACT_EABORT, "i.i.d. sampling: sub-block %u holds %llu bits > limit s = %u (abort)", worst,
                           (unsigned long long)(*sizes_out)[worst], s);
            break;
        }
        if ((e = cudaMemsetAsync(order, 0xff, (size_t)m * s * 4, st)) != cudaSuccess) { rc = cuda_error(e, "memset(order)"); break; }
        // as many warps per CTA as the per-warp counters allow (<= 16)
        const size_t per_warp = (size_t)m * 4;
        int warps = (int)std::min<size_t>(16, std::max<size_t>(1, (size_t)(96 * 1024) / per_warp));
        if (per_warp > (size_t)200 * 1024) { rc = set_error(EXTRACT_EINVAL, "i.i.d. sampling: m = %u too large", m); break; }
#define EX_IID_SCATTER(W)                                                                                           \
    if (warps >= W) {                                                                                               \
        const size_t smem = per_warp * W;                                                                           \
        if ((e = cudaFuncSetAttribute(iid_scatter_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != \
            cudaSuccess) { rc = cuda_error(e, "smem attribute"); break; }                                            \
        iid_scatter_kernel<W><<<(uint32_t)std::min<uint64_t>(ceil_div(nchunks, W), (uint64_t)num_sms * 8), W * 32, smem, st>>>( \
            n, key, mask, m, nchunks, start, s, order);                                                              \
    } else
        EX_IID_SCATTER(16) EX_IID_SCATTER(8) EX_IID_SCATTER(4) EX_IID_SCATTER(2) EX_IID_SCATTER(1) {}
#undef EX_IID_SCATTER
        if (rc != EXTRACT_OK) break;
        if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_error(e, "iid_scatter_kernel"); break; }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_error(e, "iid order"); break; }
    } while (0);
    if (count) cudaFreeAsync(count, st);
    if (start) cudaFreeAsync(start, st);
    if (sizes) cudaFreeAsync(sizes, st);
    cudaStreamSynchronize(st);
    return rc;
}

}  // namespace ex
