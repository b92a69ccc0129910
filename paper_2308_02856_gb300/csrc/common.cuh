// Shared device helpers and the host-side error state of libextract.
#pragma once

#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "../../include/extract.h"

namespace ex {

// ---------------------------------------------------------------------------
// Host-side error reporting (thread-local message, negative return codes).
// ---------------------------------------------------------------------------
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);

#define EX_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::ex::cuda_error(_e, #call);      \
    } while (0)

#define EX_LAUNCH(what)                                                 \
    do {                                                                \
        cudaError_t _e = cudaGetLastError();                            \
        if (_e != cudaSuccess) return ::ex::cuda_error(_e, what);       \
    } while (0)

static inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
static inline uint64_t round_up(uint64_t a, uint64_t b) { return ceil_div(a, b) * b; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64-bit
// multiplies mixed with the other two counter words and the round key; the
// key advances by the two Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += W0;
        k.y += W1;
    }
    return c;
}

// 64-bit sampling label of input position i (Sec. III.B step 1 as a keyed
// order): (x0 << 32) | x1 of Philox(ctr = (i_lo, i_hi, 0, 0), key), with the
// test-hook mask applied (all ones unless EXTRACT_KEY_BITS is set).
__device__ __forceinline__ uint64_t sampling_label(uint64_t i, uint2 key, uint64_t mask)
{
    const uint4 x = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, 0u), key);
    return ((((uint64_t)x.x) << 32) | (uint64_t)x.y) & mask;
}

}  // namespace ex
