// Gather of sub-blocks from inputs much larger than L2 (Sec. III.B step 1).
//
// The plain gather reads one random input bit per sub-block bit; once the
// input is several times the L2, most of those reads go to DRAM.  Here the
// input is cut into windows of 2^29 bits (64 MiB) and, once per sampling key,
// the order entries of every group of 1024 output bits (32 words of one
// stored sub-block, the unit one warp of the plain gather builds) are
// re-laid window by window, each entry with its slot in the group:
//   pos[g*1024 + e], slot[g*1024 + e]  entries of group g, window-major,
//                                      slot order inside a window;
//   off[g*(R+1) + r]                   first entry of window r (off[..R] =
//                                      the group's entry count).
// A run is then one pass per window: every warp takes groups, ORs the bits of
// the group's entries in that window into its 32 words in shared memory and
// stores them (reading back the previous windows' words first).  All random
// reads of a pass fall in one window, which stays in L2, and every order
// entry is read once per run.  The stored words are the same as the plain
// gather's: word w0 + t of sub-block j has bit l = in[perm[j s + s-1 - c]]
// with c = 32 (w0 + t) + l (0 when c >= s).
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace ex {
namespace {

constexpr int kWindowLog2 = 29;
constexpr uint32_t kGroupSlots = 1024;
constexpr int kPassWarps = 8;
constexpr int kUnroll = 4;  // rounds of 32 entries in flight per warp

// One warp per group: its 1024 slots' windows, counts, then the stable
// placement of the entries (slot order inside each window).
__global__ void __launch_bounds__(256)
gw_build_kernel(const uint32_t *__restrict__ perm, uint32_t s, uint32_t w_pad, uint64_t groups, uint32_t R,
                uint32_t *__restrict__ pos_out, uint16_t *__restrict__ slot_out, uint16_t *__restrict__ off_out)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t gpr = w_pad >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; g < groups; g += nwarps) {
        const uint64_t j = g / gpr;
        const uint32_t w0 = (uint32_t)(g % gpr) * 32u;
        const uint64_t top = j * s + (s - 1);
        uint32_t p[32], win[32];
        uint32_t cnt = 0;  // lane r < R: entries in window r
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const uint32_t cr = (w0 + t) * 32u + lane;
            const bool valid = cr < s;
            p[t] = valid ? __ldg(perm + (top - cr)) : 0u;
            win[t] = valid ? (p[t] >> kWindowLog2) : R;
            for (uint32_t r = 0; r < R; ++r) {
                const uint32_t c = __popc(__ballot_sync(0xffffffffu, win[t] == r));
                if (lane == r) cnt += c;
            }
        }
        // exclusive scan of the counts over lanes 0..R-1
        uint32_t x = lane < R ? cnt : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, x, d);
            if ((int)lane >= d) x += o;
        }
        uint32_t next = x - (lane < R ? cnt : 0u);  // lane r: next entry of window r
        if (lane <= R) off_out[g * (R + 1) + lane] = (uint16_t)next;
        const uint64_t ebase = g * kGroupSlots;
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            for (uint32_t r = 0; r < R; ++r) {
                const uint32_t mask = __ballot_sync(0xffffffffu, win[t] == r);
                const uint32_t at = __shfl_sync(0xffffffffu, next, r);
                if (win[t] == r) {
                    const uint32_t e = at + __popc(mask & below);
                    pos_out[ebase + e] = p[t];
                    slot_out[ebase + e] = (uint16_t)(t * 32 + lane);
                }
                if (lane == r) next += __popc(mask);
            }
        }
    }
}

// Pass r: the group words gain the bits of their entries in window r.
__global__ void __launch_bounds__(kPassWarps * 32)
gw_pass_kernel(const uint32_t *__restrict__ in, const uint32_t *__restrict__ pos, const uint16_t *__restrict__ slot,
               const uint16_t *__restrict__ off, uint32_t R, uint32_t r, uint64_t groups, uint32_t w_pad,
               uint32_t *__restrict__ arev)
{
    __shared__ uint32_t words[kPassWarps][32];
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t gpr = w_pad >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; g < groups; g += nwarps) {
        uint32_t *dst = arev + (g / gpr) * w_pad + (uint32_t)(g % gpr) * 32u;
        words[w][lane] = r == 0 ? 0u : dst[lane];
        __syncwarp();
        const uint32_t a = off[g * (R + 1) + r], b = off[g * (R + 1) + r + 1];
        const uint64_t ebase = g * kGroupSlots;
        // kUnroll rounds of 32 entries at a time: all their loads are issued
        // before the first bit is used
        for (uint32_t e0 = a; e0 < b; e0 += 32 * kUnroll) {
            uint32_t q[kUnroll], u[kUnroll], v[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                const uint32_t e = e0 + 32u * k + lane;
                q[k] = e < b ? __ldcs(pos + ebase + e) : 0u;
                u[k] = e < b ? __ldcs(slot + ebase + e) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) v[k] = e0 + 32u * k + lane < b ? __ldg(in + (q[k] >> 5)) : 0u;
#pragma unroll
            for (int k = 0; k < kUnroll; ++k)
                if ((v[k] >> (q[k] & 31u)) & 1u) atomicOr(&words[w][u[k] >> 5], 1u << (u[k] & 31u));
        }
        __syncwarp();
        __stcs(dst + lane, words[w][lane]);
        __syncwarp();
    }
}

}  // namespace

bool gather_windows_wanted(uint64_t input_bits) { return input_bits > (2ull << kWindowLog2); }

int gather_windows_build(const uint32_t *perm, uint32_t m, uint32_t s, uint32_t w_pad, uint64_t input_bits,
                         GatherWindows *gw, cudaStream_t st, int num_sms)
{
    gather_windows_free(gw);
    if (w_pad % 32u) return set_error(EXTRACT_EINTERNAL, "gather windows: w_pad %u not a multiple of 32", w_pad);
    gw->R = (uint32_t)ceil_div(input_bits, 1ull << kWindowLog2);
    if (gw->R > 31) return set_error(EXTRACT_EINVAL, "gather windows: %u windows", gw->R);
    gw->groups = (uint64_t)m * (w_pad / 32u);
    cudaError_t e;
    if ((e = cudaMalloc(&gw->pos, gw->groups * kGroupSlots * 4)) != cudaSuccess ||
        (e = cudaMalloc(&gw->slot, gw->groups * kGroupSlots * 2)) != cudaSuccess ||
        (e = cudaMalloc(&gw->off, gw->groups * (gw->R + 1) * 2)) != cudaSuccess) {
        gather_windows_free(gw);
        return cuda_error(e, "cudaMalloc(gather windows)");
    }
    const uint32_t grid = (uint32_t)std::min<uint64_t>(ceil_div(gw->groups, 8), (uint64_t)num_sms * 16);
    gw_build_kernel<<<grid, 256, 0, st>>>(perm, s, w_pad, gw->groups, gw->R, gw->pos, gw->slot, gw->off);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        gather_windows_free(gw);
        return cuda_error(e, "gw_build_kernel");
    }
    return EXTRACT_OK;
}

int gather_windows_run(const GatherWindows &gw, const uint32_t *in, uint32_t w_pad, uint32_t *arev, cudaStream_t st,
                       int num_sms)
{
    const uint32_t grid = (uint32_t)std::min<uint64_t>(ceil_div(gw.groups, kPassWarps), (uint64_t)num_sms * 16);
    for (uint32_t r = 0; r < gw.R; ++r)
        gw_pass_kernel<<<grid, kPassWarps * 32, 0, st>>>(in, gw.pos, gw.slot, gw.off, gw.R, r, gw.groups, w_pad, arev);
    EX_LAUNCH("gw_pass_kernel");
    return EXTRACT_OK;
}

uint64_t gather_windows_bytes(const GatherWindows &gw, uint64_t n, uint32_t w_pad)
{
    // every pass reads its window's entries (4-byte position, 2-byte slot)
    // and window starts; the input once; every group's 32 words OR-ed in
    // shared memory and stored once
    const uint64_t slots = gw.groups * 1024;
    return slots * 6 + gw.groups * (gw.R + 1) * 2 * gw.R + ceil_div(n, 32) * 4 + gw.groups * 32 * 4;
}

void gather_windows_free(GatherWindows *gw)
{
    cudaFree(gw->pos);
    cudaFree(gw->slot);
    cudaFree(gw->off);
    *gw = GatherWindows{};
}

}  // namespace ex
