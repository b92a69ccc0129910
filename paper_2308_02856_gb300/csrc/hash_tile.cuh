// The CTA tile of the Toeplitz hash (Sec. I: K = T . A'; Sec. III.B steps 3-4),
// shared by the single-block kernel (toeplitz.cu) and the persistent
// multi-block kernel (batch.cu).
//
// With sub-block j stored reversed (gather), output bit i is
//     K_j[i] = parity( XOR_w  win(seed_j, i + 32 w) AND Arev_j[w] )
// where win(x, p) is the 32 seed bits starting at bit p: one LOP3 per 32
// bit-products of T . A.
//
// Lane l of warp v owns the rows r0 + 32 (v Q + q) + l, q < Q.  The window
// that row group q needs at word w starts at word (v Q + q + w) with the
// constant shift l, so it depends on q + w only: over a block of B words a
// lane computes the Q + B - 1 distinct windows once (one SHF each) and reuses
// them for every (row group, word) pair and for all J sub-blocks of the tile,
// which share the seed.  Sub-block words come from shared memory as 16-byte
// broadcasts; the Q x J accumulators stay in registers; popc + ballot pack 32
// rows into a word that is XORed into the output at bit j*k + i (partial
// parities of a split word range combine by XOR).
#pragma once

#include "common.cuh"
#include "internal.h"

namespace ex {

constexpr int kHashWarps = 8;
constexpr int kHashThreads = kHashWarps * 32;
constexpr int kHashWC = (int)kWordChunk;  // words staged per chunk
constexpr int kWinBlock = 8;              // words sharing one set of windows
constexpr int kMaxQ = 16;
// seed words staged per chunk: every row group of the CTA plus the chunk
constexpr int kSeedSmemWords = ((kHashWarps * kMaxQ + kHashWC + 1) + 3) & ~3;

// Tile variants (row groups per lane Q, sub-blocks per tile J).  A CTA covers
// 256 Q rows x J sub-blocks.  Large J reuses each window most; large Q keeps
// small-J tiles efficient; Q = 1 serves short outputs.
constexpr int kNumVariants = 13;
__host__ __device__ constexpr int variant_q(int v)
{
    return v < 3 ? 1 : v < 8 ? 4 : v < 10 ? 8 : 16;
}
__host__ __device__ constexpr int variant_j(int v)
{
    return v == 0 ? 1 : v == 1 ? 8 : v == 2 ? 32 : v == 3 ? 1 : v == 4 ? 4 : v == 5 ? 8 : v == 6 ? 16
         : v == 7 ? 32 : v == 8 ? 8 : v == 9 ? 16 : v == 10 ? 1 : v == 11 ? 4 : 8;
}
__host__ __device__ constexpr int variant_id(int q, int j)
{
    int id = -1;
    for (int v = 0; v < kNumVariants; ++v)
        if (variant_q(v) == q && variant_j(v) == j) id = v;
    return id;
}
__host__ __device__ constexpr uint32_t variant_rows(int v) { return (uint32_t)(kHashWarps * 32 * variant_q(v)); }

// sd: the tile's seed starting at word (r0 >> 5); arev: all sub-blocks of the
// job (row stride w_pad words); a_s: J * kHashWC words; s_s: kSeedSmemWords.
template <int Q, int J>
__device__ __forceinline__ void hash_tile(const uint32_t *__restrict__ sd, const uint32_t *__restrict__ arev,
                                          uint32_t w_pad, uint32_t m, uint32_t k, uint32_t r0, uint32_t j0,
                                          uint32_t c_begin, uint32_t c_end, uint32_t *__restrict__ out,
                                          uint32_t *__restrict__ a_s, uint32_t *__restrict__ s_s)
{
    constexpr int kSeedW = kHashWarps * Q + kHashWC + 1;
    constexpr int kW = Q + kWinBlock - 1;  // distinct windows per block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    uint32_t acc[Q][J];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int j = 0; j < J; ++j) acc[q][j] = 0u;

    for (uint32_t c = c_begin; c < c_end; ++c) {
        const uint32_t wc = c * kHashWC;
        for (int t = threadIdx.x; t < kSeedW; t += blockDim.x) s_s[t] = __ldg(sd + wc + t);
        for (int t = threadIdx.x; t < J * kHashWC / 4; t += blockDim.x) {
            const int jj = t / (kHashWC / 4), ww = t % (kHashWC / 4);
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (j0 + jj < m)
                v = __ldg(reinterpret_cast<const uint4 *>(arev + (size_t)(j0 + jj) * w_pad + wc) + ww);
            *reinterpret_cast<uint4 *>(a_s + jj * kHashWC + ww * 4) = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int wb = 0; wb < kHashWC; wb += kWinBlock) {
            uint32_t win[kW];
            {
                uint32_t sw[kW + 1];
#pragma unroll
                for (int t = 0; t <= kW; ++t) sw[t] = s_s[warp * Q + wb + t];
#pragma unroll
                for (int t = 0; t < kW; ++t) win[t] = __funnelshift_r(sw[t], sw[t + 1], lane);
            }
#pragma unroll
            for (int w = 0; w < kWinBlock; w += 4) {
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const uint4 a = *reinterpret_cast<const uint4 *>(a_s + j * kHashWC + wb + w);
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        acc[q][j] ^= win[q + w] & a.x;
                        acc[q][j] ^= win[q + w + 1] & a.y;
                        acc[q][j] ^= win[q + w + 2] & a.z;
                        acc[q][j] ^= win[q + w + 3] & a.w;
                    }
                }
            }
        }
        __syncthreads();
    }

#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const uint32_t ib = r0 + (uint32_t)(warp * Q + q) * 32u;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            uint32_t word = __ballot_sync(0xffffffffu, __popc(acc[q][j]) & 1u);
            const uint32_t jj = j0 + j;
            if (lane == (j & 31) && jj < m && ib < k && word) {
                if (k - ib < 32u) word &= (1u << (k - ib)) - 1u;
                const uint64_t P = (uint64_t)jj * k + ib;
                const uint32_t sh = (uint32_t)(P & 31u);
                atomicXor(out + (P >> 5), word << sh);
                if (sh && (word >> (32u - sh))) atomicXor(out + (P >> 5) + 1, word >> (32u - sh));
            }
        }
    }
}

// Dispatch a functor templated on the variant: f.template operator()<Q, J>().
#define EX_FOR_VARIANT(v, CALL)                                             \
    switch (v) {                                                            \
    case 0: CALL(1, 1); break;                                              \
    case 1: CALL(1, 8); break;                                              \
    case 2: CALL(1, 32); break;                                             \
    case 3: CALL(4, 1); break;                                              \
    case 4: CALL(4, 4); break;                                              \
    case 5: CALL(4, 8); break;                                              \
    case 6: CALL(4, 16); break;                                             \
    case 7: CALL(4, 32); break;                                             \
    case 8: CALL(8, 8); break;                                              \
    case 9: CALL(8, 16); break;                                             \
    case 10: CALL(16, 1); break;                                            \
    case 11: CALL(16, 4); break;                                            \
    default: CALL(16, 8); break;                                            \
    }

}  // namespace ex
