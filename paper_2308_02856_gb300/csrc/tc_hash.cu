// Direct Toeplitz hashing on the fifth-generation tensor cores (tcgen05).
//
// With a shared seed the hash of all sub-blocks is one dense product over
// the integers followed by a parity (Sec. I: K = T . A' over GF(2)):
//
//   D[i][j] = sum_{b < s} seed[i + b] * R_j[b],   K_j[i] = D[i][j] mod 2,
//
// where R_j is sub-block j stored reversed (bit b = A_j[s-1-b], as the
// gather writes it), so that row i of the (Hankel-ordered) Toeplitz matrix is
// the seed window starting at bit i.  This is a GEMM with M = k output rows,
// N = m sub-blocks and K = s, on 0/1 operands.
//
// Operands are e4m3 bytes (0x38 = 1.0, 0x00 = 0.0) that the CTA expands from
// the bit strings straight into shared memory, in the canonical K-major
// layout without swizzle: 8-row x 16-byte core matrices, core matrices along
// K 128 bytes apart (LBO), groups of 8 rows 1024 bytes apart (SBO).  One
// thread issues tcgen05.mma kind::f8f6f4 (M = 128, N = nt <= 256, K = 32)
// with an f32 accumulator in tensor memory.  Products of 0/1 are exact and
// every partial sum of a K-chunk is an integer no larger than the chunk
// length (4096 by default), so the f32 sums are exact; at the end of each
// chunk the accumulator is read back (tcgen05.ld), its parities are XOR-ed
// into per-thread bit masks, and the next chunk starts from zero.  The
// parities go to output bit j k + i with word-wise atomic XORs (the output
// is zeroed first).
//
// Pipeline: two shared-memory stages; while the tensor core multiplies one
// stage, all 256 threads build the next.  tcgen05.commit arrives on the
// stage's mbarrier when the multiplies that read it are done.  Every
// mbarrier wait gives up after about a second: the kernel then sets the
// error word, waits (again bounded) for its last multiplies, frees its
// tensor memory and returns.
#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

#include <algorithm>
#include <mutex>

namespace ex {
namespace {

constexpr uint32_t kTcM = 128;                 // output rows per tile (tensor-memory lanes)
constexpr uint32_t kTcKB = 128;                // K elements (e4m3 bytes) per stage
constexpr uint32_t kTcThreads = 256;
constexpr uint32_t kTcMaxN = 256;              // sub-blocks per tile
constexpr uint32_t kTcStageA = kTcM * kTcKB;   // 16 KB of Toeplitz rows per stage
constexpr uint32_t kE4M3One = 0x38u;           // 1.0 in e4m3

// Instruction descriptor of kind::f8f6f4: f32 accumulator, A and B e4m3,
// both K-major, N = nt, M = 128.
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t nt) { return tc_idesc_mn(kTcM, nt); }

// 16 bits -> 16 e4m3 bytes (byte t = 1.0 when bit t is set, else 0)
__device__ __forceinline__ uint4 expand16(uint32_t b)
{
    uint4 r;
    r.x = (((b & 0xfu) * 0x00204081u) & 0x01010101u) * kE4M3One;
    r.y = ((((b >> 4) & 0xfu) * 0x00204081u) & 0x01010101u) * kE4M3One;
    r.z = ((((b >> 8) & 0xfu) * 0x00204081u) & 0x01010101u) * kE4M3One;
    r.w = ((((b >> 12) & 0xfu) * 0x00204081u) & 0x01010101u) * kE4M3One;
    return r;
}

// byte offset of element (row r, k) in a stage operand (core matrices)
__device__ __forceinline__ uint32_t core_off(uint32_t r, uint32_t kk)
{
    return (r >> 3) * 1024u + (kk >> 4) * 128u + (r & 7u) * 16u + (kk & 15u);
}

struct TcArgs {
    const uint32_t *seed;  // realigned seed bits, seed_words words (zero past the end)
    uint64_t seed_words;
    const uint32_t *arev;  // sub-block j at arev + j w_pad, stored reversed
    uint32_t w_pad;
    uint32_t m, k;         // sub-blocks, output rows
    uint32_t nkb;          // K blocks of 128
    uint32_t nt;           // sub-blocks per tile: 64, 128, 192 or 256
    uint32_t ncols;        // tensor-memory columns allocated (power of two >= nt)
    uint32_t tiles_m;      // row tiles
    uint32_t chunk;        // K blocks per accumulation chunk
    uint32_t *out;         // zeroed; receives K_j[i] at bit j k + i
    uint32_t *err;         // set to 1 when a wait gave up
    uint32_t stall;        // test hook: first wait on a barrier nothing arrives on
};

__device__ __forceinline__ uint32_t seed_word(const TcArgs &a, uint64_t w) { return w < a.seed_words ? __ldg(a.seed + w) : 0u; }

// The global words one thread needs to build one stage: three seed words for
// its Toeplitz row segment and the 128 bits of its sub-block row.  Loaded a
// stage ahead, so their latency hides behind the current stage's build.
struct StageWords {
    uint32_t s0, s1, s2;  // seed words from T0 / 32 (T0 below)
    uint32_t sh;          // T0 mod 32
    uint4 bits;           // sub-block row jj = threadIdx.x (0 past m or nt)
};

// Words for K block kb: Toeplitz row r = t / 2, elements 64 (t % 2) .. +63
// (seed bits from T0 = i0 + r + 128 kb + 64 (t % 2)); sub-block row t.
__device__ __forceinline__ StageWords load_stage(const TcArgs &a, uint32_t i0, uint32_t j0, uint32_t kb)
{
    const uint32_t t = threadIdx.x;
    StageWords v;
    const uint64_t T0 = (uint64_t)i0 + (t >> 1) + (uint64_t)kb * kTcKB + 64u * (t & 1u);
    const uint64_t w = T0 >> 5;
    v.sh = (uint32_t)(T0 & 31u);
    v.s0 = seed_word(a, w);
    v.s1 = seed_word(a, w + 1);
    v.s2 = seed_word(a, w + 2);
    v.bits = make_uint4(0, 0, 0, 0);
    const uint32_t j = j0 + t;
    if (t < a.nt && j < a.m) v.bits = __ldg(reinterpret_cast<const uint4 *>(a.arev + (size_t)j * a.w_pad + 4u * kb));
    return v;
}

// Build stage `st` from the loaded words: Toeplitz rows i0 .. i0+127 (row r,
// element kk = seed bit i0 + r + 128 kb + kk) and sub-blocks j0 .. j0+nt-1
// (row jj, element kk = bit 128 kb + kk of R_{j0+jj}; zero past m).
__device__ __forceinline__ void build_stage(const TcArgs &a, uint8_t *st, const StageWords &v)
{
    const uint32_t t = threadIdx.x;
    {   // A: thread t -> row t / 2, elements 64 (t % 2) .. +63
        const uint32_t r = t >> 1, h = t & 1u;
        const uint32_t lo = __funnelshift_r(v.s0, v.s1, v.sh), hi = __funnelshift_r(v.s1, v.s2, v.sh);
        const uint32_t g4[4] = {lo & 0xffffu, lo >> 16, hi & 0xffffu, hi >> 16};
#pragma unroll
        for (int g = 0; g < 4; ++g)
            *reinterpret_cast<uint4 *>(st + core_off(r, 64u * h + 16u * g)) = expand16(g4[g]);
    }
    if (t < a.nt) {  // B: one sub-block row per thread
        uint8_t *sb = st + kTcStageA;
        const uint32_t wv[4] = {v.bits.x, v.bits.y, v.bits.z, v.bits.w};
#pragma unroll
        for (int q = 0; q < 8; ++q)
            *reinterpret_cast<uint4 *>(sb + core_off(t, 16u * q)) = expand16((wv[q >> 1] >> (16u * (q & 1))) & 0xffffu);
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) tc_hash_kernel(TcArgs a)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    const uint32_t stage_bytes = kTcStageA + a.nt * kTcKB;
    uint8_t *stage0 = sm, *stage1 = sm + stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + 2 * stage_bytes);  // 2 stages + 1 never arrived on
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 3);
    volatile uint32_t *abort_flag = tslot + 1;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t i0 = (blockIdx.x % a.tiles_m) * kTcM, j0 = (blockIdx.x / a.tiles_m) * a.nt;
    const uint32_t idesc = tc_idesc(a.nt);
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        mbar_init(smem_u32(&bars[2]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tslot), a.ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // this thread's rows and columns in the read-back: lane quarter w % 4,
    // column half w / 4 (nt / 2 columns, a multiple of 32)
    const uint32_t lq = warp & 3u, half = a.nt >> 1, c0 = (warp >> 2) * half;
    uint32_t par[kTcMaxN / 2 / 32] = {0, 0, 0, 0};
    int64_t last_commit = -1;
    // test hook: a wait that runs out (its barrier's first phase never
    // completes), exercising the error path without any multiply in flight
    if (a.stall && !mbar_wait(smem_u32(&bars[2]), 0u)) *abort_flag = 1;
    __syncthreads();
    StageWords next = load_stage(a, i0, j0, 0);
    for (uint32_t kb = 0; kb < a.nkb && !*abort_flag; ++kb) {
        const uint32_t b = kb & 1u;
        uint8_t *st = b ? stage1 : stage0;
        const StageWords cur = next;
        if (kb + 1 < a.nkb) next = load_stage(a, i0, j0, kb + 1);  // in flight during this stage
        // the multiplies of K block kb - 2 read this stage: wait for them
        if (kb >= 2 && !mbar_wait(smem_u32(&bars[b]), ((kb - 2) >> 1) & 1u)) *abort_flag = 1;
        build_stage(a, st, cur);
        fence_async_smem();  // the stage's generic writes, visible to the tensor core
        __syncthreads();
        if (*abort_flag) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t sa = smem_u32(st), sbm = sa + kTcStageA;
            const bool fresh = (kb % a.chunk) == 0;
#pragma unroll
            for (uint32_t q = 0; q < kTcKB / 32; ++q)  // K = 32 per multiply: two core matrices
                tc_mma(tmem, smem_desc(sa + 256u * q, 128u, 1024u), smem_desc(sbm + 256u * q, 128u, 1024u), idesc,
                       (fresh && q == 0) ? 0u : 1u);
            tc_commit(smem_u32(&bars[b]));
        }
        last_commit = kb;
        if ((kb + 1) % a.chunk == 0 || kb + 1 == a.nkb) {
            // end of a chunk: its sums are complete once its last multiplies are
            if (!mbar_wait(smem_u32(&bars[b]), (kb >> 1) & 1u)) *abort_flag = 1;
            __syncthreads();  // one view of the abort flag before the warp-wide loads
            if (*abort_flag) break;
            tc_fence_after();
            for (uint32_t cb = 0; cb < half / 32; ++cb) {
                uint32_t v[32];
                tmem_ld32(tmem + ((32u * lq) << 16) + c0 + 32u * cb, v);
                tmem_wait_ld();
                uint32_t bits = 0;
#pragma unroll
                for (int c = 0; c < 32; ++c) bits |= (__float2uint_rz(__uint_as_float(v[c])) & 1u) << c;
                par[cb] ^= bits;
            }
            tc_fence_before();
            __syncthreads();  // the next chunk's first multiply overwrites the accumulator
        }
    }
    if (*abort_flag) {
        if (tid == 0) atomicOr(a.err, 1u);
        // let the last committed multiplies finish before the memory is freed
        if (last_commit >= 0) mbar_wait(smem_u32(&bars[last_commit & 1]), (uint32_t)(last_commit >> 1) & 1u);
    } else {
        // K_j[i] for rows i0 + 32 lq + lane and columns j0 + c0 + c: one ballot
        // per column gives 32 consecutive output bits of sub-block j
        const uint32_t i = i0 + 32u * lq + lane;
        for (uint32_t cb = 0; cb < half / 32; ++cb)
            for (uint32_t c = 0; c < 32; ++c) {
                const uint32_t j = j0 + c0 + 32u * cb + c;
                const uint32_t word = __ballot_sync(0xffffffffu, i < a.k && ((par[cb] >> c) & 1u));
                if (lane == c && j < a.m && word) {
                    const uint64_t P = (uint64_t)j * a.k + (i0 + 32u * lq);
                    const uint32_t sh = (uint32_t)(P & 31u);
                    atomicXor(a.out + (P >> 5), word << sh);
                    if (sh && (word >> (32u - sh))) atomicXor(a.out + (P >> 5) + 1, word >> (32u - sh));
                }
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, a.ncols);
    }
}

std::mutex g_tc_mu;
uint64_t g_tc_smem_set = 0;  // devices whose kernel attribute is set

}  // namespace

uint32_t tc_tile_n(uint32_t m) { return m >= kTcMaxN ? kTcMaxN : (uint32_t)std::max<uint64_t>(64, round_up(m, 64)); }

int launch_hash_tc(const uint32_t *seed, uint64_t seed_words, const uint32_t *arev, uint32_t w_pad, uint32_t m,
                   uint32_t s, uint32_t k, uint32_t *out, uint32_t *err, cudaStream_t st, uint32_t chunk_blocks,
                   bool test_stall)
{
    if (w_pad % 4u) return set_error(EXTRACT_EINTERNAL, "tensor-core hash: w_pad %u not a multiple of 4", w_pad);
    TcArgs a{};
    a.seed = seed;
    a.seed_words = seed_words;
    a.arev = arev;
    a.w_pad = w_pad;
    a.m = m;
    a.k = k;
    a.nkb = (uint32_t)ceil_div(s, kTcKB);
    if ((uint64_t)a.nkb * 4u > w_pad) return set_error(EXTRACT_EINTERNAL, "tensor-core hash: K blocks past w_pad");
    a.nt = tc_tile_n(m);
    a.ncols = a.nt <= 32 ? 32u : a.nt <= 64 ? 64u : a.nt <= 128 ? 128u : 256u;
    a.tiles_m = (uint32_t)ceil_div(k, kTcM);
    a.chunk = std::max<uint32_t>(1, chunk_blocks);
    a.out = out;
    a.err = err;
    a.stall = test_stall ? 1u : 0u;
    const uint64_t tiles = (uint64_t)a.tiles_m * ceil_div(m, a.nt);
    if (tiles >= (1ull << 31)) return set_error(EXTRACT_EINVAL, "tensor-core hash: too many tiles");
    // shared memory: two stages and the barriers; at least enough that no
    // more CTAs share an SM than its 512 tensor-memory columns hold
    const uint32_t need = 2 * (kTcStageA + a.nt * kTcKB) + 64;  // stages, 3 barriers, tensor address, flag
    const uint32_t per_sm = 512u / a.ncols;
    const uint32_t smem = std::max<uint32_t>(need, kSmemPerSM / (per_sm + 1) + 1);
    int dev = 0;
    EX_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lock(g_tc_mu);
        if (dev < 64 && !((g_tc_smem_set >> dev) & 1u)) {
            EX_CUDA(cudaFuncSetAttribute(tc_hash_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
            g_tc_smem_set |= 1ull << dev;
        }
    }
    if (smem > 200 * 1024) return set_error(EXTRACT_EINTERNAL, "tensor-core hash: %u bytes of shared memory", smem);
    EX_CUDA(cudaMemsetAsync(out, 0, ceil_div((uint64_t)m * k, 32) * 4, st));
    tc_hash_kernel<<<(uint32_t)tiles, kTcThreads, smem, st>>>(a);
    EX_LAUNCH("tc_hash_kernel");
    return EXTRACT_OK;
}

}  // namespace ex
