// Gather of the sampled sub-blocks (Sec. III.B step 1: bit A_i goes to
// sub-block j when its label ranks it there; Sec. IV: the sampled bits are
// stored before hashing).
//
// Output layout, read by the hashing kernels: sub-block j occupies words
// [j * w_pad, (j+1) * w_pad) and is stored REVERSED, bit b of word w being
// A_j[s - 1 - (32 w + b)] (0 past s).  With that order the Toeplitz row i is
// the plain dot product of seed bits [i, i + s) with the stored string, so
// the hashing kernel reads the seed forwards with funnel shifts only.
//
// One warp builds 32 consecutive output words: for each word every lane
// fetches one order entry (32 consecutive entries: one coalesced 128-byte
// load), then the input word that holds its bit (random 4-byte loads, 32 in
// flight per lane), and a ballot packs the 32 bits.  The 32 words are stored
// with one coalesced 128-byte store.
#include "common.cuh"
#include "gather_body.cuh"
#include "internal.h"

#include <algorithm>

namespace ex {
namespace {

// input window of one gather pass: 2^29 bits = 64 MiB, half the L2
// (measured on the 2^30-bit block: 8.6 ms in one pass, 5.5 ms in two)
constexpr uint64_t kGatherWindowBits = 1ull << 29;

template <bool kIdentity, bool kPadded, bool kWindowed>
__global__ void __launch_bounds__(256)
gather_kernel(const uint32_t *__restrict__ in, const uint32_t *__restrict__ perm, uint32_t m,
              uint32_t s, uint32_t w_pad, uint64_t groups, uint32_t *__restrict__ arev, uint64_t rank0,
              uint32_t wlo, uint32_t wlen, bool accumulate)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gstride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t gpr = w_pad >> 5;  // 32-word groups per sub-block
    for (uint64_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; g < groups;
         g += gstride)
        gather_group<kIdentity, kPadded, kWindowed>(in, perm, s, w_pad, (uint32_t)(g / gpr), (uint32_t)(g % gpr) * 32u,
                                                    lane, arev, rank0, wlo, wlen, accumulate);
}

}  // namespace

bool gather_prefers_whole_block(uint64_t input_bits) { return input_bits <= 2 * kGatherWindowBits; }

int launch_gather(const uint32_t *in, const uint32_t *perm, uint32_t m, uint32_t s,
                  uint32_t w_pad, uint32_t *arev, cudaStream_t st, int num_sms, uint64_t rank0, bool padded,
                  uint64_t input_bits, bool windows_when_padded)
{
    if (w_pad % 32u) return set_error(EXTRACT_EINTERNAL, "gather: w_pad %u not a multiple of 32", w_pad);
    const uint64_t groups = (uint64_t)m * (w_pad / 32u);
    if (groups == 0) return EXTRACT_OK;
    const uint64_t want = ceil_div(groups, 8);  // 8 warps per block
    const uint32_t grid = (uint32_t)std::min<uint64_t>(want, (uint64_t)num_sms * 64);
    if (!perm) {
        gather_kernel<true, false, false><<<grid, 256, 0, st>>>(in, perm, m, s, w_pad, groups, arev, rank0, 0, 0, false);
        EX_LAUNCH("gather_kernel");
        return EXTRACT_OK;
    }
    // inputs of one to two windows (sorted order): one pass per window of the
    // input, so the random reads stay in L2.  More passes cost more in order
    // re-reads than they save, and the i.i.d. law's increasing positions
    // already read with locality.
    const bool two_windows = input_bits > kGatherWindowBits && input_bits <= 2 * kGatherWindowBits;
    if (!two_windows || (padded && !windows_when_padded)) {
        if (padded)
            gather_kernel<false, true, false><<<grid, 256, 0, st>>>(in, perm, m, s, w_pad, groups, arev, rank0, 0, 0, false);
        else
            gather_kernel<false, false, false><<<grid, 256, 0, st>>>(in, perm, m, s, w_pad, groups, arev, rank0, 0, 0, false);
    } else {
        for (uint64_t lo = 0; lo < input_bits; lo += kGatherWindowBits) {
            const uint32_t len = (uint32_t)std::min<uint64_t>(kGatherWindowBits, input_bits - lo);
            if (padded)
                gather_kernel<false, true, true><<<grid, 256, 0, st>>>(in, perm, m, s, w_pad, groups, arev, rank0,
                                                                       (uint32_t)lo, len, lo > 0);
            else
                gather_kernel<false, false, true><<<grid, 256, 0, st>>>(in, perm, m, s, w_pad, groups, arev, rank0,
                                                                        (uint32_t)lo, len, lo > 0);
        }
    }
    EX_LAUNCH("gather_kernel");
    return EXTRACT_OK;
}

}  // namespace ex
