// The CTA tile of the Toeplitz hash (Sec. I: K = T . A'; Sec. III.B steps 3-4),
// shared by the single-block kernel (toeplitz.cu) and the persistent
// multi-block kernel (batch.cu).
//
// With sub-block j stored reversed (gather), output bit i is
//     K_j[i] = parity( XOR_w  win(seed_j, i + 32 w) AND Arev_j[w] )
// where win(x, p) is the 32 seed bits starting at bit p: one LOP3 per 32
// bit-products of T . A.  Lane l of warp v owns rows r0 + 32 (v Q + q) + l,
// so its funnel-shift amount is the constant l and one SHF serves all J
// sub-blocks of the tile; sub-block words come from shared memory as 16-byte
// broadcasts; Q x J accumulators per lane stay in registers; popc + ballot
// pack 32 rows into a word that is XORed into the output at bit j*k + i
// (partial parities of a split word range combine by XOR).
#pragma once

#include "common.cuh"
#include "internal.h"

namespace ex {

constexpr int kHashWarps = 8;
constexpr int kHashThreads = kHashWarps * 32;
constexpr int kHashWC = (int)kWordChunk;
// seed words staged per chunk for row groups Q <= 4
constexpr int kSeedSmemWords = ((kHashWarps * 4 + kHashWC + 1) + 3) & ~3;

// sd: the tile's seed starting at word (r0 >> 5); arev: all sub-blocks of the
// job (row stride w_pad words); a_s: J * kHashWC words; s_s: kSeedSmemWords.
template <int Q, int J>
__device__ __forceinline__ void hash_tile(const uint32_t *__restrict__ sd, const uint32_t *__restrict__ arev,
                                          uint32_t w_pad, uint32_t m, uint32_t k, uint32_t r0, uint32_t j0,
                                          uint32_t c_begin, uint32_t c_end, uint32_t *__restrict__ out,
                                          uint32_t *__restrict__ a_s, uint32_t *__restrict__ s_s)
{
    constexpr int kSeedW = kHashWarps * Q + kHashWC + 1;
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
        for (int w = 0; w < kHashWC; w += 4) {
            uint32_t sw[Q + 4];
#pragma unroll
            for (int t = 0; t < Q + 4; ++t) sw[t] = s_s[warp * Q + w + t];
            uint32_t win[Q][4];
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int u = 0; u < 4; ++u) win[q][u] = __funnelshift_r(sw[q + u], sw[q + u + 1], lane);
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const uint4 a = *reinterpret_cast<const uint4 *>(a_s + j * kHashWC + w);
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    acc[q][j] ^= win[q][0] & a.x;
                    acc[q][j] ^= win[q][1] & a.y;
                    acc[q][j] ^= win[q][2] & a.z;
                    acc[q][j] ^= win[q][3] & a.w;
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

// Tile variants: q in {1, 4} (256 or 1024 rows per CTA) x j in {1, 4, 8, 16, 32}.
constexpr int kNumVariants = 10;
__host__ __device__ constexpr int variant_id(int q, int j)
{
    return (q == 4 ? 5 : 0) + (j == 1 ? 0 : j == 4 ? 1 : j == 8 ? 2 : j == 16 ? 3 : 4);
}
__host__ __device__ constexpr int variant_q(int v) { return v >= 5 ? 4 : 1; }
__host__ __device__ constexpr int variant_j(int v)
{
    return (v % 5) == 0 ? 1 : (v % 5) == 1 ? 4 : (v % 5) == 2 ? 8 : (v % 5) == 3 ? 16 : 32;
}

}  // namespace ex
