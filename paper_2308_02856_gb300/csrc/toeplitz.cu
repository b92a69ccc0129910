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

}  // namespace

HashPlan plan_hash(uint32_t m, uint32_t k, uint32_t w_pad, bool per_subblock_seed, int num_sms)
{
    // Model: padded work of the tile grid divided by the share of ALU issue
    // slots that are LOP3 (one SHF per distinct window: Q + kWinBlock - 1
    // SHF per Q x J x kWinBlock LOP3).
    HashPlan p;
    double best = 1e300;
    for (int v = 0; v < kNumVariants; ++v) {
        const int q = variant_q(v), j = variant_j(v);
        if (per_subblock_seed && j != 1) continue;
        const double tiles = (double)ceil_div(k, variant_rows(v)) * (double)ceil_div(m, (uint32_t)j);
        const double lop3 = (double)q * j * kWinBlock;
        const double eff = lop3 / (lop3 + q + kWinBlock - 1);
        const double t = tiles * variant_rows(v) * j / eff;
        if (t < best * 0.999) {
            best = t;
            p.variant = v;
        }
    }
    p.q = variant_q(p.variant);
    p.j = variant_j(p.variant);
    p.warps = kWarps;
    p.wc = kWC;
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
    if (p.variant < 0 || p.variant >= kNumVariants || variant_q(p.variant) != p.q || variant_j(p.variant) != p.j)
        return set_error(EXTRACT_EINTERNAL, "no kernel for tile q=%d j=%d", p.q, p.j);
#define EX_LAUNCH_TILE(Q_, J_) launch_tile<Q_, J_>(p, seed, seed_stride, arev, w_pad, m, k, out, st)
    EX_FOR_VARIANT(p.variant, EX_LAUNCH_TILE)
#undef EX_LAUNCH_TILE
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
