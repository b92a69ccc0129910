// extract_run_static: a run of the gather + hash path that allocates no
// device memory.  Its scratch (the padded Toeplitz seed and the gathered
// sub-blocks) lives in one file-scope __device__ array of fixed size that the
// CUDA driver reserves on every GPU that loads this library, for as long as
// the process lives.
//
// Host code must not use the array's name as a device address (on the host
// it names a host-side shadow); the device address is fetched once per
// device with cudaGetSymbolAddress, with that device current, and handed to
// the kernels.
#include "common.cuh"
#include "internal.h"

#include <mutex>

namespace ex {
namespace {

constexpr uint64_t kScratchWords = EXTRACT_STATIC_SCRATCH_WORDS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint32_t g_static_scratch[kScratchWords];

std::mutex g_setup_mu;
uint32_t *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call for that device).
int scratch_for_device(int dev, uint32_t **out)
{
    if (dev < 0 || dev >= kMaxDevices) return set_error(EXTRACT_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
        if (!p) return set_error(EXTRACT_EINTERNAL, "static scratch has no device address");
        g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_scratch_ptr[dev];
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
    if (n > (1ull << 32) || (uint64_t)m * s > n)
        return set_error(EXTRACT_EINVAL, "need m*s <= n <= 2^32 (n=%llu m=%u s=%u)", (unsigned long long)n, m, s);

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
    if (int rc = scratch_for_device(dev, &scratch)) return rc;
    uint32_t *seed_stage = scratch;
    uint32_t *arev = scratch + seed_part;

    cudaStream_t st = (cudaStream_t)stream;
    stage_seed_kernel<<<(uint32_t)ceil_div(stride, 256), 256, 0, st>>>(seed_dev, (uint64_t)s + k - 1, stride,
                                                                       seed_stage);
    EX_LAUNCH("stage_seed_kernel");
    if (int rc = launch_gather(in_bits_dev, perm_dev, m, s, w_pad, arev, st, sms, 0, false, n)) return rc;
    return launch_hash(plan, seed_stage, 0u, arev, w_pad, m, k, out_bits_dev, st);
}
