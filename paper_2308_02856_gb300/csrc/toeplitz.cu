// Toeplitz hashing of the gathered sub-blocks and concatenation of the
// outputs (Sec. I: K = T . A'; Sec. III.B steps 3 and 4).
//
// The tile body and its design notes are in hash_tile.cuh; this file holds
// the single-block launch, the plan heuristic and the plain per-block
// baseline kernel.
#include "common.cuh"
#include "hash_tile.cuh"
#include "internal.h"

#include <algorithm>

namespace ex {
namespace {

constexpr int kWarps = kHashWarps;
constexpr int kWC = kHashWC;

template <int Q, int J>
__global__ void __launch_bounds__(kHashThreads, 1)
toeplitz_lop3_kernel(const uint32_t *__restrict__ seed, uint32_t seed_stride,
                     const uint32_t *__restrict__ arev, uint32_t w_pad, uint32_t m, uint32_t k,
                     uint32_t gx, uint32_t nchunks, uint32_t cps, uint32_t *__restrict__ out)
{
    constexpr int kRows = kWarps * 32 * Q;
    __shared__ __align__(16) uint32_t a_s[J * kWC];
    __shared__ __align__(16) uint32_t s_s[kSeedSmemWords];
    const uint32_t bx = blockIdx.x % gx, by = blockIdx.x / gx;
    const uint32_t r0 = bx * kRows;
    const uint32_t j0 = by * J;
    const uint32_t c_begin = blockIdx.z * cps;
    const uint32_t c_end = min(nchunks, c_begin + cps);
    const uint32_t *sd = seed + (size_t)(seed_stride ? j0 : 0u) * seed_stride + (r0 >> 5);
    hash_tile<Q, J>(sd, arev, w_pad, m, k, r0, j0, c_begin, c_end, out, a_s, s_s);
}

// Plain per-block baseline: one thread per output row of one sub-block.
__global__ void __launch_bounds__(256)
toeplitz_plain_kernel(const uint32_t *__restrict__ seed, const uint32_t *__restrict__ arev_j,
                      uint32_t sw, uint32_t k, uint64_t bitoff, uint32_t *__restrict__ out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t *sd = seed + (i >> 5);
    const uint32_t sh = i & 31u;
    uint32_t acc = 0;
    for (uint32_t w = 0; w < sw; ++w) acc ^= __funnelshift_r(sd[w], sd[w + 1], sh) & arev_j[w];
    uint32_t word = __ballot_sync(0xffffffffu, __popc(acc) & 1u);
    if ((threadIdx.x & 31u) == 0 && i < k && word) {
        if (k - i < 32u) word &= (1u << (k - i)) - 1u;
        const uint64_t P = bitoff + i;
        const uint32_t s2 = (uint32_t)(P & 31u);
        atomicXor(out + (P >> 5), word << s2);
        if (s2 && (word >> (32u - s2))) atomicXor(out + (P >> 5) + 1, word >> (32u - s2));
    }
}

template <int Q, int J>
void launch_tile(const HashPlan &p, const uint32_t *seed, uint32_t seed_stride, const uint32_t *arev,
                 uint32_t w_pad, uint32_t m, uint32_t k, uint32_t *out, cudaStream_t st)
{
    dim3 grid(p.gx * p.gy, 1, p.splits);
    toeplitz_lop3_kernel<Q, J><<<grid, kWarps * 32, 0, st>>>(seed, seed_stride, arev, w_pad, m, k,
                                                              p.gx, p.nchunks, p.cps, out);
}

template <int Q>
bool dispatch_j(const HashPlan &p, const uint32_t *seed, uint32_t seed_stride, const uint32_t *arev,
                uint32_t w_pad, uint32_t m, uint32_t k, uint32_t *out, cudaStream_t st)
{
    switch (p.j) {
    case 1: launch_tile<Q, 1>(p, seed, seed_stride, arev, w_pad, m, k, out, st); return true;
    case 4: launch_tile<Q, 4>(p, seed, seed_stride, arev, w_pad, m, k, out, st); return true;
    case 8: launch_tile<Q, 8>(p, seed, seed_stride, arev, w_pad, m, k, out, st); return true;
    case 16: launch_tile<Q, 16>(p, seed, seed_stride, arev, w_pad, m, k, out, st); return true;
    case 32: launch_tile<Q, 32>(p, seed, seed_stride, arev, w_pad, m, k, out, st); return true;
    default: return false;
    }
}

}  // namespace

HashPlan plan_hash(uint32_t m, uint32_t k, uint32_t w_pad, bool per_subblock_seed, int num_sms)
{
    HashPlan p;
    p.warps = kWarps;
    p.wc = kWC;
    if (per_subblock_seed) p.j = 1;
    else p.j = m >= 32 ? 32 : m >= 16 ? 16 : m >= 8 ? 8 : m >= 4 ? 4 : 1;
    p.q = k > 512 ? 4 : 1;
    p.gx = (uint32_t)ceil_div(k, p.rows());
    p.gy = (uint32_t)ceil_div(m, (uint32_t)p.j);
    p.nchunks = w_pad / (uint32_t)p.wc;
    const uint64_t tiles = (uint64_t)p.gx * p.gy;
    const uint64_t target = 2ull * (uint64_t)num_sms;
    uint64_t splits = std::max<uint64_t>(1, ceil_div(target, tiles));
    splits = std::min<uint64_t>(splits, p.nchunks);
    p.cps = (uint32_t)ceil_div(p.nchunks, splits);
    p.splits = (uint32_t)ceil_div(p.nchunks, p.cps);
    return p;
}

uint32_t seed_stride_words(const HashPlan &p, uint32_t k, uint32_t w_pad)
{
    const uint64_t rows = std::max<uint64_t>((uint64_t)p.gx * p.rows(), round_up(k, 256));
    return (uint32_t)round_up(rows / 32 + w_pad + 2, 4);
}

int launch_hash(const HashPlan &p, const uint32_t *seed, uint32_t seed_stride, const uint32_t *arev,
                uint32_t w_pad, uint32_t m, uint32_t k, uint32_t *out, cudaStream_t st)
{
    const uint64_t out_words = ceil_div((uint64_t)m * k, 32);
    EX_CUDA(cudaMemsetAsync(out, 0, out_words * sizeof(uint32_t), st));
    bool ok = false;
    if (p.q == 4) ok = dispatch_j<4>(p, seed, seed_stride, arev, w_pad, m, k, out, st);
    else if (p.q == 1) ok = dispatch_j<1>(p, seed, seed_stride, arev, w_pad, m, k, out, st);
    if (!ok) return set_error(EXTRACT_EINTERNAL, "no kernel for tile q=%d j=%d", p.q, p.j);
    EX_LAUNCH("toeplitz_lop3_kernel");
    return EXTRACT_OK;
}

int launch_hash_plain(const uint32_t *seed, uint32_t seed_stride, const uint32_t *arev,
                      uint32_t w_pad, uint32_t s, uint32_t m, uint32_t k, uint32_t *out,
                      cudaStream_t st)
{
    const uint64_t out_words = ceil_div((uint64_t)m * k, 32);
    EX_CUDA(cudaMemsetAsync(out, 0, out_words * sizeof(uint32_t), st));
    const uint32_t sw = (uint32_t)ceil_div(s, 32);
    const uint32_t grid = (uint32_t)ceil_div(k, 256);
    for (uint32_t j = 0; j < m; ++j) {
        toeplitz_plain_kernel<<<grid, 256, 0, st>>>(seed + (size_t)(seed_stride ? j : 0u) * seed_stride,
                                                    arev + (size_t)j * w_pad, sw, k,
                                                    (uint64_t)j * k, out);
    }
    EX_LAUNCH("toeplitz_plain_kernel");
    return EXTRACT_OK;
}

}  // namespace ex
