// extract_run_static: a run of the gather + hash path that allocates no
// device memory.  Its scratch (the padded Toeplitz seed and the gathered
// sub-blocks) lives in one file-scope __device__ array of fixed size that the
// CUDA driver reserves on every GPU that loads this library, for as long as
// the process lives.
//
// Host code must not use the array's name as a device address (on the host
// it names a host-side shadow); every call fetches the device address with
// cudaGetSymbolAddress, with the calling device current, and hands it to the
// kernels.  The lookup is not cached: after a cudaDeviceReset the module is
// loaded again and the array may sit at a new address.
#include "common.cuh"
#include "internal.h"

namespace ex {
namespace {

constexpr uint64_t kScratchWords = EXTRACT_STATIC_SCRATCH_WORDS;

static __device__ __align__(256) uint32_t g_static_scratch[kScratchWords];

// Device address of the scratch array on the current device.  The first
// lookup on a device loads this library's device code there (lazy module
// loading), which reserves the array.
int scratch_for_device(uint32_t **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
    if (!p) return set_error(EXTRACT_EINTERNAL, "static scratch has no device address");
    *out = static_cast<uint32_t *>(p);
    return EXTRACT_OK;
}

// dst[t] for t < stride: the seed's words with the bits past L cleared, then
// zeros (the hashing kernel reads up to stride words).
__global__ void stage_seed_kernel(const uint32_t *__restrict__ seed, uint64_t L, uint32_t stride,
                                  uint32_t *__restrict__ dst)
{
    const uint32_t words = (uint32_t)((L + 31) / 32);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < stride; t += gridDim.x * blockDim.x) {
        uint32_t v = 0;
        if (t < words) {
            v = seed[t];
            if (t == words - 1 && (L & 31u)) v &= (1u << (L & 31u)) - 1u;
        }
        dst[t] = v;
    }
}

}  // namespace
}  // namespace ex

using namespace ex;

extern "C" int extract_run_static(uint64_t n, uint32_t m, uint32_t s, uint32_t k, const uint32_t *perm_dev,
                                  const uint32_t *seed_dev, const uint32_t *in_bits_dev,
                                  uint32_t *out_bits_dev, void *stream)
{
    if (!seed_dev || !in_bits_dev || !out_bits_dev)
        return set_error(EXTRACT_EINVAL, "extract_run_static: null seed, input or output pointer");
    if (m < 1 || s < 1 || k < 1 || k > s)
        return set_error(EXTRACT_EINVAL, "need m >= 1 and 1 <= k <= s (m=%u s=%u k=%u)", m, s, k);
    if (n > (1ull << 32))
        return set_error(EXTRACT_EINVAL, "need n <= 2^32 (n=%llu)", (unsigned long long)n);
    // a padded order (the i.i.d. law's) may hold more slots than positions;
    // padding slots exist only when n < 2^32, where no position equals them
    if ((uint64_t)m * s > n && (!perm_dev || n == (1ull << 32)))
        return set_error(EXTRACT_EINVAL, "need m*s <= n (n=%llu m=%u s=%u)%s", (unsigned long long)n, m, s,
                         perm_dev ? "" : " for the identity order");

    int dev = 0, sms = 0;
    EX_CUDA(cudaGetDevice(&dev));
    EX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint32_t w_pad = (uint32_t)round_up(ceil_div(s, 32), kWordChunk);
    const HashPlan plan = plan_hash(m, k, w_pad, false, sms);
    const uint32_t stride = seed_stride_words(plan, k, w_pad);
    const uint64_t seed_part = round_up(stride, 64);  // keeps the sub-block part 256-byte aligned
    const uint64_t need = seed_part + (uint64_t)m * w_pad;
    if (need > kScratchWords)
        return set_error(EXTRACT_EINVAL,
                         "extract_run_static: this shape needs %llu scratch words, the static limit is %llu "
                         "(%llu MiB); use extract_create/extract_run",
                         (unsigned long long)need, (unsigned long long)kScratchWords,
                         (unsigned long long)(kScratchWords * 4 >> 20));
    uint32_t *scratch = nullptr;
    if (int rc = scratch_for_device(&scratch)) return rc;
    uint32_t *seed_stage = scratch;
    uint32_t *arev = scratch + seed_part;

    cudaStream_t st = (cudaStream_t)stream;
    stage_seed_kernel<<<(uint32_t)ceil_div(stride, 256), 256, 0, st>>>(seed_dev, (uint64_t)s + k - 1, stride,
                                                                       seed_stage);
    EX_LAUNCH("stage_seed_kernel");
    // Below 2^32 input bits no position equals the padding value, so order
    // entries that hold it are read as 0: the i.i.d. law's padded orders, and
    // never a real position of a sorted order.
    const bool padded = perm_dev && n < (1ull << 32);
    if (int rc = launch_gather(in_bits_dev, perm_dev, m, s, w_pad, arev, st, sms, 0, padded, n, true)) return rc;
    return launch_hash(plan, seed_stage, 0u, arev, w_pad, m, k, out_bits_dev, st);
}
