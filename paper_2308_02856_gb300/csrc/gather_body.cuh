// One warp's share of the sub-block gather (Sec. III.B step 1; the sampled
// bits are stored before hashing, Sec. IV), shared by the single-block and
// the batched gather kernels.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace ex {

// Words [w0, w0 + 32) of sub-block j, stored reversed: bit b of word w is
// in[perm[rank0 + j*s + s-1-(32w+b)]] when 32w+b < s, else 0 (rank0: the
// first rank of sub-block 0 of this launch).  The warp issues 32
// coalesced 128-byte loads of the order, then 32 independent input loads
// per lane, packs each word with a ballot and stores the 32 words with one
// coalesced store.  kIdentity: perm is the identity (perm unused).
// kPadded: order entries equal to kNoPos are padding and read as 0 (the
// i.i.d. law's sub-blocks shorter than s; n < 2^32 there, so no position
// has that value).
// kWindowed: only positions in [wlo, wlo + wlen) are read (the others
// count as 0) and, when `accumulate`, the words are OR-ed into what earlier
// windows stored: passes over windows of the input that fit in L2 turn the
// random input reads into L2 hits at the cost of re-reading the order.
template <bool kIdentity, bool kPadded = false, bool kWindowed = false>
__device__ __forceinline__ void gather_group(const uint32_t *__restrict__ in, const uint32_t *__restrict__ perm,
                                             uint32_t s, uint32_t w_pad, uint32_t j, uint32_t w0, uint32_t lane,
                                             uint32_t *__restrict__ arev, uint64_t rank0 = 0, uint32_t wlo = 0,
                                             uint32_t wlen = 0, bool accumulate = false)
{
    const uint64_t top = rank0 + (uint64_t)j * s + (s - 1);  // rank of A_j[s-1]
    uint32_t pos[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        const uint64_t cr = (uint64_t)(w0 + t) * 32u + lane;  // reversed index s-1-c
        if (cr < s) {
            const uint64_t rank = top - cr;
            // the order is streamed once: evict it first so that the input
            // words, read at random, stay in L2
            pos[t] = kIdentity ? (uint32_t)rank : __ldcs(perm + rank);
        } else {
            pos[t] = 0xffffffffu;
        }
    }
    uint32_t mine = 0;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        const uint64_t cr = (uint64_t)(w0 + t) * 32u + lane;
        uint32_t bit = 0;
        const bool in_window = !kWindowed || pos[t] - wlo < wlen;
        if (cr < s && (!kPadded || pos[t] != kNoPos) && in_window)
            bit = (__ldg(in + (pos[t] >> 5)) >> (pos[t] & 31u)) & 1u;
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == (uint32_t)t) mine = word;
    }
    uint32_t *dst = arev + (uint64_t)j * w_pad + w0 + lane;
    if (kWindowed && accumulate) mine |= *dst;
    __stcs(dst, mine);
}

}  // namespace ex
