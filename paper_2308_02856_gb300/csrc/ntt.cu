// Exact fast Toeplitz hashing by number-theoretic transform: the FFT-based
// direction the paper names for CPUs and GPUs (Sec. I, Sec. V), done exactly
// in integer arithmetic.
//
// K_j[i] = XOR_c seed[i - c + s - 1] A_j[c] is the parity of coefficient
// i + s - 1 of the integer product sigma(x) a_j(x), sigma = sum seed[t] x^t
// (L = s + k - 1 terms), a_j = sum A_j[c] x^c (s terms).  That coefficient
// is at most s < p = 7 * 2^26 + 1, so one NTT modulo p gives it exactly.  A
// cyclic convolution of length N = 2^e >= s + k - 1 leaves coefficients
// s-1 .. s+k-2 free of wrap-around (no index pair reaches N + s - 1).
//
// Splitting: a sub-block may be cut into P = 2^l pieces of h coefficients;
// piece q is its own middle product against the seed window starting at
// q h, the P products add up in the frequency domain, and one inverse
// transform of length N >= h + k - 1 gives their sum (work P + 1 transforms
// of N instead of 2 of the length for s + k - 1).
//
// Four-step layout, N = R1 x R2 with R2 = 2048 (element t = t1 R2 + t2):
//   pass A  (columns t2 of one piece per CTA): load the bits, R1-point DIF
//           NTT along t1, multiply by w_N^(k1 t2); for R1 = 32, 64, 128 the
//           column DFTs of the bits run on the tensor cores instead, as an
//           exact integer GEMM (ntt_cols_fwd_tc_kernel);
//   pass B  (two warps per row): 2048-point DIF NTT of each piece's row,
//           multiply by that piece's seed spectrum (laid out the same way,
//           1/N folded in), sum over pieces, 2048-point inverse DIT NTT;
//   pass A' (columns per CTA): multiply by w_N^(-k1 t2), R1-point inverse
//           DIT NTT along t1, then the parity of every coefficient t in
//           [h-1, h+k-1) goes straight to output bit j k + t - (h-1).
// DIF leaves bit-reversed order and DIT consumes it, so nothing is permuted.
//
// Warp transforms: a warp holds 32 EPL values, lane l / register j at
// position 32 j + l (for R1 < 1024, 32 / E whole columns of 32 E); stages
// with pair distance >= 32 run inside registers, then a shared-memory
// transpose (padded rows: word 33 j + l; the transposed-warp kernels for
// R1 >= 1024 use the XOR swizzle 32 j + (l ^ j)) gives each lane whole rows
// of 32 and the distance < 32 stages run in registers too, with their
// twiddles as constant-bank operands.
//
// Arithmetic (Harvey's lazy butterflies): 4p < 2^31, so DIF values stay in
// [0, 2p) and DIT values in [0, 4p) with one conditional subtraction per
// sum; fixed multipliers use Shoup's precomputed quotient (result in
// [0, 2p)), computed twist factors use Montgomery form.  Values are reduced
// to [0, p) only where a parity is taken.
#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

namespace ex {
namespace {

constexpr uint32_t kP = 469762049u;   // 7 * 2^26 + 1
constexpr uint32_t k2P = 2u * kP;
constexpr uint32_t kGen = 3u;         // a primitive root modulo p
constexpr int kR2Log = 11;
constexpr uint32_t kR2 = 1u << kR2Log;
constexpr int kCW = 16;               // columns per pass-A CTA
constexpr int kCS = kCW + 1;          // padded smem row (no bank conflicts)
constexpr int kRowsB = 2;             // rows per pass-B CTA
constexpr int kThreads = 256;
constexpr int kMaxSplitLog2 = 4;      // at most 16 pieces per sub-block
constexpr uint64_t kMaxWorkWords = 16ull << 20;    // one sub-block's pieces (and windows), <= 64 MB
// One launch group's work buffer: up to 1 GB (140 sub-blocks of the QKD shape,
// 128 of the QRNG shape).  Large groups amortise each launch's set-up and
// fill the GPU in every pass; the QKD-shaped block's hash takes 26.9 ms with
// 1 GB groups against 30.9 ms with 128 MB (18 sub-blocks), 28.3 with 192 MB
// and 27.0 with 512 MB (two lanes; a third lane gains nothing at 1 GB).
#ifndef EX_NTT_GROUP_WORDS
#define EX_NTT_GROUP_WORDS (256ull << 20)
#endif
constexpr uint64_t kGroupWorkWords = EX_NTT_GROUP_WORDS;

// -p^{-1} mod 2^32 by Newton iteration
constexpr uint32_t neg_inv32(uint32_t p)
{
    uint32_t x = p;  // p * p == 1 mod 8
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    return 0u - x;
}
constexpr uint32_t kPNegInv = neg_inv32(kP);

__device__ __forceinline__ uint32_t add_p(uint32_t a, uint32_t b)
{
    const uint32_t r = a + b;
    return min(r, r - kP);
}
__device__ __forceinline__ uint32_t sub_p(uint32_t a, uint32_t b)
{
    const uint32_t r = a - b + kP;
    return min(r, r - kP);
}
// a * w mod p with wq = floor(w 2^32 / p) (Shoup)
__device__ __forceinline__ uint32_t mul_shoup(uint32_t a, uint32_t w, uint32_t wq)
{
    const uint32_t q = __umulhi(a, wq);
    const uint32_t r = a * w - q * kP;
    return min(r, r - kP);
}
// a * b * 2^-32 mod p (Montgomery)
__device__ __forceinline__ uint32_t mul_mont(uint32_t a, uint32_t b)
{
    const uint64_t t = (uint64_t)a * b;
    const uint32_t m = (uint32_t)t * kPNegInv;
    const uint32_t u = (uint32_t)((t + (uint64_t)m * kP) >> 32);
    return min(u, u - kP);
}

// lazy forms
__device__ __forceinline__ uint32_t red2p(uint32_t x) { return min(x, x - k2P); }  // [0,4p) -> [0,2p)
__device__ __forceinline__ uint32_t redp(uint32_t x) { return min(x, x - kP); }    // [0,2p) -> [0,p)
__device__ __forceinline__ uint32_t shoup_lazy(uint32_t a, uint32_t w, uint32_t wq)  // any a: [0,2p)
{
    return a * w - __umulhi(a, wq) * kP;
}
__device__ __forceinline__ uint32_t mont_lazy(uint32_t a, uint32_t b)  // a < 4p, b < 2p: [0,2p)
{
    const uint64_t t = (uint64_t)a * b;
    const uint32_t m = (uint32_t)t * kPNegInv;
    return (uint32_t)((t + (uint64_t)m * kP) >> 32);
}
// DIF butterfly, inputs and outputs in [0, 2p)
__device__ __forceinline__ void bf_dif(uint32_t &x, uint32_t &y, uint32_t w, uint32_t wq)
{
    const uint32_t d = x - y + k2P;
    x = red2p(x + y);
    y = shoup_lazy(d, w, wq);
}
// DIF butterflies with looser bounds (8p < 2^32): inputs in [0, 4p) give
// x' in [0, 4p) and y' in [0, 2p); inputs in [0, 2p) give the same bounds
// with no reduction at all (x' = x + y).
constexpr uint32_t k4P = 4u * kP;
__device__ __forceinline__ uint32_t red4p(uint32_t x) { return min(x, x - k4P); }  // [0,8p) -> [0,4p)
__device__ __forceinline__ void bf_dif_4p(uint32_t &x, uint32_t &y, uint32_t w, uint32_t wq)
{
    const uint32_t d = x - y + k4P;
    x = red4p(x + y);
    y = shoup_lazy(d, w, wq);
}
__device__ __forceinline__ void bf_dif_2p(uint32_t &x, uint32_t &y, uint32_t w, uint32_t wq)
{
    const uint32_t d = x - y + k2P;
    x = x + y;
    y = shoup_lazy(d, w, wq);
}
// DIT butterfly, inputs and outputs in [0, 4p)
__device__ __forceinline__ void bf_dit(uint32_t &x, uint32_t &y, uint32_t w, uint32_t wq)
{
    const uint32_t a = red2p(x), t = shoup_lazy(y, w, wq);
    x = a + t;
    y = a - t + k2P;
}

__device__ __forceinline__ uint32_t bitrev(uint32_t x, int bits)
{
    return bits ? __brev(x) >> (32 - bits) : 0u;
}

// Twiddle tables in device memory (one plan per context).
struct Tables {
    // stage twiddles w_R^i, i < R/2, and their Shoup quotients, for the
    // column (R1) and row (R2) transforms, forward and inverse
    const uint32_t *col_f, *col_fq, *col_i, *col_iq;
    const uint32_t *row_f, *row_fq, *row_i, *row_iq;
    // twist factors in Montgomery form: w_N^x = lo[x & 2047] * hi[x >> 11]
    const uint32_t *tw_lo_f, *tw_hi_f, *tw_lo_i, *tw_hi_i;
    // per-stage tables for the warp transforms: entry (h - 1) + r holds
    // (w_2h^r, Shoup quotient) for r < h, every h = 1, 2, 4, ... < R
    const uint2 *row_stage_f, *row_stage_i;  // R = 2048
    const uint2 *col_stage_f, *col_stage_i;  // R = R1
    // full twist tables for R1 >= 32 (Montgomery form): entry t2 * R1 + r
    // is w_N^(+-bitrev(r) t2)
    const uint32_t *twist_f, *twist_i;
};

// Where pass A finds the bits of virtual block v = g P + q: piece q of
// source row g, starting 32 step q bits in.  A piece holds len coefficients;
// only its first lim(q) = min(len, total - 32 step q) positions are data,
// the rest read as 0.  Sub-block pieces have len = 32 step; a seed window of
// a piece is longer (len = h + k - 1) and overlaps the next one.
struct Pieces {
    uint64_t stride;  // words between source rows
    uint32_t P;       // pieces per row
    uint32_t step;    // words between pieces (h / 32 when P > 1)
    uint32_t len;     // coefficients per piece
    uint32_t total;   // data bits per row
};

__device__ __forceinline__ const uint32_t *piece_src(const uint32_t *bits, const Pieces &pc, uint32_t v,
                                                     uint32_t &lim)
{
    const uint32_t q = v % pc.P;
    lim = min(pc.len, pc.total - q * pc.step * 32u);
    return bits + (size_t)(v / pc.P) * pc.stride + (size_t)q * pc.step;
}

// The bits a pass-A CTA loads, staged once per CTA: rb[t1] bit c is element
// t = t1 R2 + c0 + c, read from position len - 1 - t (kReversed) or t of b,
// and 0 where t >= len or the position is >= lim.  The CTA's 16 columns of
// one row are 16 adjacent bits of the source (at most two words), so a row
// costs one or two word loads instead of one load per column.
template <bool kReversed>
__device__ __forceinline__ void stage_row_bits(uint32_t *rb, const uint32_t *__restrict__ b, uint32_t len,
                                               uint32_t lim, uint32_t R1, uint32_t c0)
{
    for (uint32_t t1 = threadIdx.x; t1 < R1; t1 += blockDim.x) {
        const uint32_t t0 = t1 * kR2 + c0;  // element of column c0
        uint32_t f = 0;
        if (t0 < len) {
            if (kReversed) {
                // element t0 + c sits at position hi - c; keep positions <= top
                const int32_t hi = (int32_t)(len - 1 - t0), lo = hi - (kCW - 1);
                const int32_t top = min(hi, (int32_t)lim - 1);
                if (top >= max(lo, 0)) {
                    const int32_t w0 = lo >> 5, w1 = top >> 5;  // floor; w1 >= 0
                    const uint32_t a = w0 >= 0 ? __ldg(b + w0) : 0u;
                    const uint32_t c = w1 != w0 ? __ldg(b + w1) : 0u;
                    const uint64_t v = ((uint64_t)c << 32) | a;
                    const int32_t nb = top - lo + 1;  // 1 .. 16 positions kept
                    const uint32_t f16 = (uint32_t)(v >> (lo - 32 * w0)) & (nb >= 16 ? 0xffffu : (1u << nb) - 1u);
                    f = __brev(f16 << 16);  // position lo + i -> column 15 - i
                }
            } else {
                const uint32_t end = min(len, lim);
                if (t0 < end) {
                    f = (__ldg(b + (t0 >> 5)) >> (t0 & 31u)) & 0xffffu;  // c0 % 16 == 0: one word
                    if (end - t0 < (uint32_t)kCW) f &= (1u << (end - t0)) - 1u;
                }
            }
        }
        rb[t1] = f;
    }
}

__device__ __forceinline__ uint32_t twist_mont(const uint32_t *lo, const uint32_t *hi, uint32_t x)
{
    return mul_mont(__ldg(lo + (x & (kR2 - 1))), __ldg(hi + (x >> kR2Log)));
}

// DIF NTT of length R over the first index of x[r * kCS + c], c < kCW.
__device__ __forceinline__ void dif_cols(uint32_t *x, uint32_t R, const uint32_t *tw, const uint32_t *twq)
{
    for (uint32_t h = R >> 1; h >= 1; h >>= 1) {
        const uint32_t stride = R / (2 * h);
        for (uint32_t it = threadIdx.x; it < (R >> 1) * kCW; it += blockDim.x) {
            const uint32_t c = it % kCW, b = it / kCW;
            const uint32_t off = b & (h - 1), i = ((b - off) << 1) + off;
            uint32_t *pu = x + i * kCS + c, *pv = x + (i + h) * kCS + c;
            const uint32_t u = *pu, v = *pv;
            const uint32_t ti = off * stride;
            *pu = add_p(u, v);
            *pv = mul_shoup(sub_p(u, v), __ldg(tw + ti), __ldg(twq + ti));
        }
        __syncthreads();
    }
}

// DIT inverse NTT of length R (bit-reversed in, natural out) over columns.
__device__ __forceinline__ void dit_cols(uint32_t *x, uint32_t R, const uint32_t *tw, const uint32_t *twq)
{
    for (uint32_t h = 1; h < R; h <<= 1) {
        const uint32_t stride = R / (2 * h);
        for (uint32_t it = threadIdx.x; it < (R >> 1) * kCW; it += blockDim.x) {
            const uint32_t c = it % kCW, b = it / kCW;
            const uint32_t off = b & (h - 1), i = ((b - off) << 1) + off;
            uint32_t *pu = x + i * kCS + c, *pv = x + (i + h) * kCS + c;
            const uint32_t ti = off * stride;
            const uint32_t u = *pu, v = mul_shoup(*pv, __ldg(tw + ti), __ldg(twq + ti));
            *pu = add_p(u, v);
            *pv = sub_p(u, v);
        }
        __syncthreads();
    }
}

// Pass A: bits -> column DIF -> twist -> buf (row-major R1 x R2), one
// virtual block (piece) per blockIdx.y.
// kReversed: bits are a gathered sub-block stored reversed (bit s-1-t of
// row j holds A_j[t]); else bit t holds coefficient t (the seed).
template <bool kReversed>
__global__ void __launch_bounds__(kThreads)
ntt_pass_a_kernel(const uint32_t *__restrict__ bits, Pieces pc, uint32_t R1, int r1_log, uint32_t N, Tables T,
                  uint32_t *__restrict__ buf)
{
    extern __shared__ uint32_t x[];  // R1 * kCS + R1
    const uint32_t g = blockIdx.y;
    const uint32_t c0 = blockIdx.x * kCW;
    uint32_t lim;
    const uint32_t *b = piece_src(bits, pc, g, lim);
    uint32_t *rb = x + R1 * kCS;
    stage_row_bits<kReversed>(rb, b, pc.len, lim, R1, c0);
    __syncthreads();
    for (uint32_t it = threadIdx.x; it < R1 * kCW; it += blockDim.x) {
        const uint32_t c = it % kCW, t1 = it / kCW;
        x[t1 * kCS + c] = (rb[t1] >> c) & 1u;
    }
    __syncthreads();
    dif_cols(x, R1, T.col_f, T.col_fq);
    // row r now holds frequency k1 = bitrev(r); multiply by w_N^(k1 t2)
    for (uint32_t it = threadIdx.x; it < R1 * kCW; it += blockDim.x) {
        const uint32_t c = it % kCW, r = it / kCW;
        const uint32_t e = bitrev(r, r1_log) * (c0 + c);  // < N
        x[r * kCS + c] = mul_mont(x[r * kCS + c], twist_mont(T.tw_lo_f, T.tw_hi_f, e));
    }
    __syncthreads();
    uint32_t *o = buf + (size_t)g * N;
    for (uint32_t it = threadIdx.x; it < R1 * kCW; it += blockDim.x) {
        const uint32_t c = it % kCW, r = it / kCW;
        o[(size_t)r * kR2 + c0 + c] = x[r * kCS + c];
    }
}

// Pass A': untwist, column inverse DIT, parity of coefficients
// [len-1, len+k-1) (len: coefficients per piece) into output bits
// j k + t - (len-1).  Sub-block g's summed rows start g sub_stride words in.
__global__ void __launch_bounds__(kThreads)
ntt_pass_a_inv_kernel(const uint32_t *__restrict__ buf, uint64_t sub_stride, uint32_t R1, int r1_log, Tables T, uint32_t j0,
                      uint32_t len, uint32_t k, uint32_t *__restrict__ out)
{
    extern __shared__ uint32_t x[];  // R1 * kCS
    const uint32_t g = blockIdx.y;
    const uint32_t c0 = blockIdx.x * kCW;
    const uint32_t *in = buf + (size_t)g * sub_stride;
    for (uint32_t it = threadIdx.x; it < R1 * kCW; it += blockDim.x) {
        const uint32_t c = it % kCW, r = it / kCW;
        const uint32_t e = bitrev(r, r1_log) * (c0 + c);
        x[r * kCS + c] = mul_mont(in[(size_t)r * kR2 + c0 + c], twist_mont(T.tw_lo_i, T.tw_hi_i, e));
    }
    __syncthreads();
    dit_cols(x, R1, T.col_i, T.col_iq);
    const uint64_t jk = (uint64_t)(j0 + g) * k;
    const uint32_t lo_t = len - 1, hi_t = len - 1 + k;  // wanted coefficients
    for (uint32_t t1 = threadIdx.x; t1 < R1; t1 += blockDim.x) {
        const uint32_t base = t1 * kR2 + c0;
        if (base + kCW <= lo_t || base >= hi_t) continue;
        uint32_t bits16 = 0;
#pragma unroll
        for (int c = 0; c < kCW; ++c) {
            const uint32_t t = base + c;
            if (t >= lo_t && t < hi_t) bits16 |= (x[t1 * kCS + c] & 1u) << c;
        }
        uint64_t P;  // output bit of the lowest kept coefficient
        if (base < lo_t) {
            bits16 >>= (lo_t - base);
            P = jk;
        } else {
            P = jk + (base - lo_t);
        }
        if (!bits16) continue;
        const uint32_t sh = (uint32_t)(P & 31u);
        atomicXor(out + (P >> 5), bits16 << sh);
        if (sh > 16 && (bits16 >> (32u - sh))) atomicXor(out + (P >> 5) + 1, bits16 >> (32u - sh));
    }
}

// Full twist tables: tw[t2 * R1 + r] = w_N^(+-bitrev(r) t2), Montgomery form.
__global__ void ntt_twist_table_kernel(uint32_t *twf, uint32_t *twi, uint32_t R1, int r1_log, Tables T)
{
    const uint32_t total = R1 * kR2;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t t2 = i / R1, r = i % R1;
        const uint32_t e = bitrev(r, r1_log) * t2;
        twf[i] = twist_mont(T.tw_lo_f, T.tw_hi_f, e);
        twi[i] = twist_mont(T.tw_lo_i, T.tw_hi_i, e);
    }
}

// The shared seed spectrum's pointwise products: Montgomery form (one word
// per element) or Shoup form (value and quotient, two words).
constexpr bool kSpectrumMont = true;

// S = spectrum * N^-1 (Shoup: c = N^-1, with quotients Sq) or spectrum *
// N^-1 * 2^32 (Montgomery form: c = N^-1 2^32, Sq unused).
__global__ void ntt_finish_spectrum_kernel(uint32_t *S, uint32_t *Sq, uint32_t N, uint32_t c, uint32_t c_q)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const uint32_t v = mul_shoup(S[i], c, c_q);
        S[i] = v;
        if (!kSpectrumMont) Sq[i] = (uint32_t)(((uint64_t)v << 32) / kP);
    }
}


// ---- transposed warp transforms (32 EPL values, EPL in {32, 64}) ---------
// distance < 32 stages: twiddle w_2h^r for r < h at (h - 1) + r, h = 1..16
__constant__ uint2 c_low_f[31];
__constant__ uint2 c_low_i[31];

__device__ __forceinline__ uint32_t swz(uint32_t t) { return (t & ~31u) | ((t ^ (t >> 5)) & 31u); }


// DIF: layout A in (e[j] = position 32 j + l), layout B out (e[32 q + i] =
// position 32 (l + 32 q) + i).  sw: this warp's 32 EPL-word scratch.  HP0:
// the largest register-stage distance / 32 (EPL / 2 for one column; E / 2
// when the 32 EPL positions are 32 / E columns of 32 E, which the register
// stages then never mix).
// kZeroTop: e[j] are bits and the upper half of every column is zero, so the
// first stage's butterflies (x, 0) -> (x, x w) are one multiply each.
// kLazy (inputs in [0, 2p); outputs in [0, 4p), for a Montgomery product
// that takes them): every stage leaves its sums x + y in [0, 4p) and its
// differences in [0, 2p), so a pair of two earlier differences needs no
// reduction; which earlier branch a pair comes from is fixed by its register
// index, except across the transpose (the lane's parity), where the 4p form
// is used.  The last stage (twiddle 1) of a difference pair is x + y,
// x - y + 2p with no multiply.
// kPad: the transpose scratch is padded (row stride 33 words) instead of
// XOR-swizzled: every access is a lane-dependent base plus a constant offset,
// so no index arithmetic per element; 33 EPL words of scratch.
template <int EPL, int HP0 = EPL / 2, bool kZeroTop = false, bool kLazy = false, bool kPad = false>
__device__ __forceinline__ void dif_warp_t(uint32_t (&e)[EPL], uint32_t *sw, const uint2 *__restrict__ tw, int lane)
{
#pragma unroll
    for (int hp = HP0; hp >= 1; hp >>= 1) {
#pragma unroll
        for (int j = 0; j < EPL; ++j) {
            if (j & hp) continue;
            const uint2 w = __ldg(tw + (32 * hp - 1) + lane + 32 * (j & (hp - 1)));
            if (kZeroTop && hp == HP0) {
                e[j + hp] = e[j] * w.x;
            } else if (!kLazy) {
                bf_dif(e[j], e[j + hp], w.x, w.y);
            } else {
                // inputs below 2p: the first stage, the stage after the
                // zero-top one, or two differences of the previous stage
                const bool low = hp == HP0 || (kZeroTop && 2 * hp == HP0) || (j & (2 * hp));
                if (low) bf_dif_2p(e[j], e[j + hp], w.x, w.y);
                else bf_dif_4p(e[j], e[j + hp], w.x, w.y);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < EPL; ++j) sw[kPad ? 33u * j + lane : swz(32u * j + lane)] = e[j];
    __syncwarp();
#pragma unroll
    for (int q = 0; q < EPL / 32; ++q)
#pragma unroll
        for (int i = 0; i < 32; ++i)
            e[32 * q + i] = sw[kPad ? 33u * (lane + 32 * q) + i : swz(32u * (lane + 32 * q) + i)];
    __syncwarp();
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1)
#pragma unroll
        for (int q = 0; q < EPL / 32; ++q)
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (i & h) continue;
                const uint2 w = c_low_f[(h - 1) + (i & (h - 1))];
                if (!kLazy) {
                    bf_dif(e[32 * q + i], e[32 * q + i + h], w.x, w.y);
                    continue;
                }
                // h = 16 follows the register stages across the transpose
                const bool low = h == 16 ? (HP0 == 0 || (kZeroTop && HP0 == 1)) : (i & (2 * h)) != 0;
                if (h == 1 && low) {
                    const uint32_t a = e[32 * q + i], b = e[32 * q + i + 1];
                    e[32 * q + i] = a + b;
                    e[32 * q + i + 1] = a - b + k2P;
                } else if (low) {
                    bf_dif_2p(e[32 * q + i], e[32 * q + i + h], w.x, w.y);
                } else {
                    bf_dif_4p(e[32 * q + i], e[32 * q + i + h], w.x, w.y);
                }
            }
}

// DIT: layout B in, layout A out (the exact reverse of dif_warp_t).
// kFirstUnit: inputs are in [0, 2p), so the first stage (twiddle 1) is
// x + y, x - y + 2p with no reduction and no multiply.
template <int EPL, int HP0 = EPL / 2, bool kFirstUnit = false, bool kPad = false>
__device__ __forceinline__ void dit_warp_t(uint32_t (&e)[EPL], uint32_t *sw, const uint2 *__restrict__ tw, int lane)
{
#pragma unroll
    for (int h = 1; h <= 16; h <<= 1)
#pragma unroll
        for (int q = 0; q < EPL / 32; ++q)
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (i & h) continue;
                if (kFirstUnit && h == 1) {
                    const uint32_t a = e[32 * q + i], b = e[32 * q + i + 1];
                    e[32 * q + i] = a + b;
                    e[32 * q + i + 1] = a - b + k2P;
                    continue;
                }
                const uint2 w = c_low_i[(h - 1) + (i & (h - 1))];
                bf_dit(e[32 * q + i], e[32 * q + i + h], w.x, w.y);
            }
#pragma unroll
    for (int q = 0; q < EPL / 32; ++q)
#pragma unroll
        for (int i = 0; i < 32; ++i)
            sw[kPad ? 33u * (lane + 32 * q) + i : swz(32u * (lane + 32 * q) + i)] = e[32 * q + i];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < EPL; ++j) e[j] = sw[kPad ? 33u * j + lane : swz(32u * j + lane)];
    __syncwarp();
#pragma unroll
    for (int hp = 1; hp <= HP0; hp <<= 1) {
#pragma unroll
        for (int j = 0; j < EPL; ++j) {
            if (j & hp) continue;
            const uint2 w = __ldg(tw + (32 * hp - 1) + lane + 32 * (j & (hp - 1)));
            bf_dit(e[j], e[j + hp], w.x, w.y);
        }
    }
}

// Pass B's per-warp transpose scratch: padded rows (EX_ROW_PAD), else XOR swizzle
#ifndef EX_ROW_PAD
#define EX_ROW_PAD 1
#endif
constexpr bool kRowPad = EX_ROW_PAD != 0;
constexpr uint32_t kRowSw = kRowPad ? 33u * 32u : 1024u;

// Pass B: one CTA of two warps per 2048-word row; warp w owns half
// [1024 w, 1024 w + 1024).  The distance-1024 DIF stage is done while
// loading (each warp reads both halves), the distance-1024 DIT stage by an
// exchange through shared memory.
//   kInverse false: forward DIF only (the seed spectrum), stored in layout B.
//   kInverse true:  for each of the P pieces q of a sub-block (its rows
//                   q N words after piece 0's), DIF and multiply by
//                   spectrum q; the products are summed, transformed back,
//                   and the row is stored in piece 0's place.  kMulti
//                   false is the P = 1 form.
// kLazy: outputs in [0, 4p) (for the spectrum product), else [0, 2p)
template <bool kLazy>
__device__ __forceinline__ void row_dif(uint32_t (&e)[32], const uint32_t *x, uint32_t *sw, const Tables &T,
                                        int lane, int w)
{
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const uint32_t pos = 32u * j + lane;
        const uint32_t a = x[pos], b = x[pos + 1024];
        if (w == 0) {
            e[j] = red2p(a + b);
        } else {
            const uint2 tw = __ldg(T.row_stage_f + 1023 + pos);
            e[j] = shoup_lazy(a - b + k2P, tw.x, tw.y);
        }
    }
    dif_warp_t<32, 16, false, kLazy, kRowPad>(e, sw, T.row_stage_f, lane);
}

// e[i] (layout B, from base) times a spectrum row computed in the same run
// (no Shoup quotients): Montgomery products, e * s * 2^-32; the inverse
// twist table of such a plan carries the factor 2^32 back.  kAcc: added.
template <bool kAcc>
__device__ __forceinline__ void row_mul_mont(uint32_t (&e)[32], uint32_t (&acc)[32], const uint32_t *sv)
{
#pragma unroll
    for (int i = 0; i < 32; i += 4) {
        const uint4 a = *reinterpret_cast<const uint4 *>(sv + i);
        const uint32_t m0 = mont_lazy(e[i], a.x), m1 = mont_lazy(e[i + 1], a.y);
        const uint32_t m2 = mont_lazy(e[i + 2], a.z), m3 = mont_lazy(e[i + 3], a.w);
        if (kAcc) {
            acc[i] = red2p(acc[i] + m0);
            acc[i + 1] = red2p(acc[i + 1] + m1);
            acc[i + 2] = red2p(acc[i + 2] + m2);
            acc[i + 3] = red2p(acc[i + 3] + m3);
        } else {
            acc[i] = m0;
            acc[i + 1] = m1;
            acc[i + 2] = m2;
            acc[i + 3] = m3;
        }
    }
}

// e[i] (layout B, from base) times the spectrum; kAcc: added to acc
template <bool kAcc>
__device__ __forceinline__ void row_mul(uint32_t (&e)[32], uint32_t (&acc)[32], const uint32_t *sv,
                                        const uint32_t *sq)
{
#pragma unroll
    for (int i = 0; i < 32; i += 4) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(sv + i)), b = __ldg(reinterpret_cast<const uint4 *>(sq + i));
        const uint32_t m0 = shoup_lazy(e[i], a.x, b.x), m1 = shoup_lazy(e[i + 1], a.y, b.y);
        const uint32_t m2 = shoup_lazy(e[i + 2], a.z, b.z), m3 = shoup_lazy(e[i + 3], a.w, b.w);
        if (kAcc) {
            acc[i] = red2p(acc[i] + m0);
            acc[i + 1] = red2p(acc[i + 1] + m1);
            acc[i + 2] = red2p(acc[i + 2] + m2);
            acc[i + 3] = red2p(acc[i + 3] + m3);
        } else {
            acc[i] = m0;
            acc[i + 1] = m1;
            acc[i + 2] = m2;
            acc[i + 3] = m3;
        }
    }
}

// inverse DIT of acc (layout B) and the distance-1024 stage, stored to x
__device__ __forceinline__ void row_dit_store(uint32_t (&e)[32], uint32_t *x, uint32_t (*sw)[kRowSw], const Tables &T,
                                              int lane, int w)
{
    dit_warp_t<32, 16, true, kRowPad>(e, sw[w], T.row_stage_i, lane);  // the products are in [0, 2p)
    // distance-1024 DIT stage: x' = x + w y, y' = x - w y (w = w_2048^-pos)
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const uint32_t pos = 32u * j + lane;
        if (w == 0) {
            sw[0][pos] = red2p(e[j]);
        } else {
            const uint2 tw = __ldg(T.row_stage_i + 1023 + pos);
            sw[1][pos] = shoup_lazy(e[j], tw.x, tw.y);
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const uint32_t pos = 32u * j + lane;
        const uint32_t a = sw[0][pos], t = sw[1][pos];
        x[pos + 1024u * w] = w == 0 ? a + t : a - t + k2P;
    }
}

// kPerBlock: the spectra are per sub-block (independent seeds), transformed
// in the same run: piece q of sub-block g uses S + (g P + q) N, without
// quotients (Montgomery products).
// The distance-1024 DIF stage of a row held in shared memory (xs): warp 0
// keeps the sums, warp 1 the twisted differences (layout A, [0, 2p)).
__device__ __forceinline__ void row_first_stage(uint32_t (&e)[32], const uint32_t *xs, const Tables &T, int lane,
                                                int w)
{
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const uint32_t pos = 32u * j + lane;
        const uint32_t a = xs[pos], b = xs[pos + 1024];
        if (w == 0) {
            e[j] = red2p(a + b);
        } else {
            const uint2 tw = __ldg(T.row_stage_f + 1023 + pos);
            e[j] = shoup_lazy(a - b + k2P, tw.x, tw.y);
        }
    }
}

// kMulti (the P-piece inverse form): each piece's row comes into shared
// memory by one bulk copy, issued while the previous piece is transformed;
// a copy that does not land within about a second sets *err and the row is
// left unwritten.
template <bool kInverse, bool kMulti, bool kPerBlock = false>
__global__ void __launch_bounds__(64, kMulti ? 10 : 12)
ntt_rows_kernel(uint32_t *__restrict__ buf, uint32_t N, uint32_t R1, uint32_t P, const uint32_t *__restrict__ S,
                const uint32_t *__restrict__ Sq, Tables T, uint32_t *err)
{
    __shared__ __align__(16) uint32_t sw[2][kRowSw];
    __shared__ __align__(16) uint32_t xs[kInverse && kMulti ? kR2 : 4];
    __shared__ uint64_t xbar;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t row = blockIdx.x, g = row / R1, r = row % R1;
    uint32_t *x = buf + (size_t)g * P * N + (size_t)r * kR2;
    const uint32_t base = 1024u * w + 32u * lane;  // layout B: e[i] at base + i
    const size_t so = (size_t)r * kR2 + base;
    const uint32_t *Sb = kPerBlock ? S + (size_t)g * P * N : S;
    uint32_t e[32];
    if (!(kInverse && kMulti)) row_dif<kInverse>(e, x, sw[w], T, lane, w);
    if (!kInverse) {
        // both warps read both halves of the row in row_dif: no half is
        // overwritten before the other warp has loaded it
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 32; i += 4)
            *reinterpret_cast<uint4 *>(x + base + i) = make_uint4(e[i], e[i + 1], e[i + 2], e[i + 3]);
        return;
    }
    constexpr bool kMont = kPerBlock || kSpectrumMont;
    if (!kMulti) {
        if (kMont) row_mul_mont<false>(e, e, Sb + so);
        else row_mul<false>(e, e, S + so, Sq + so);
        row_dit_store(e, x, sw, T, lane, w);
        return;
    }
    // one copy of the piece loop's code (fewer instruction-fetch stalls than
    // peeling the first piece: 66.7 against 66.1 Gbit/s on the 2^30-bit
    // block); the first piece's products are added to zero
    uint32_t acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0;
    const uint32_t xb = smem_u32(xs), mb = smem_u32(&xbar);
    if (threadIdx.x == 0) {
        mbar_init(mb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bulk_load(xb, x, kR2 * 4, mb);
    }
    __syncthreads();
    uint32_t q = 0;
#pragma unroll 1
    for (; q < P; ++q) {
        if (!__syncthreads_and(mbar_wait(mb, q & 1u))) break;  // the same view in both warps
        row_first_stage(e, xs, T, lane, w);
        // the next piece's copy overwrites the row through the async proxy: every
        // load of it must have returned first (a barrier alone does not wait for
        // loads in flight), and the reads are ordered before the copy's writes
#pragma unroll
        for (int j = 0; j < 32; ++j) asm volatile("" ::"r"(e[j]));
        fence_async_smem();
        __syncthreads();  // both warps have read the row: the next piece's copy may land
        if (threadIdx.x == 0 && q + 1 < P) bulk_load(xb, x + (size_t)(q + 1) * N, kR2 * 4, mb);
        dif_warp_t<32, 16, false, true, kRowPad>(e, sw[w], T.row_stage_f, lane);
        if (kMont) row_mul_mont<true>(e, acc, Sb + (size_t)q * N + so);
        else row_mul<true>(e, acc, S + (size_t)q * N + so, Sq + (size_t)q * N + so);
    }
    if (q < P) {
        // no copy may still be landing in shared memory when the CTA exits
        if (threadIdx.x == 0) {
            atomicOr(err, 1u);
            mbar_wait(mb, q & 1u);
        }
        return;
    }
    row_dit_store(acc, x, sw, T, lane, w);
}

// Pass A with transposed warps (R1 = 32 EPL, EPL in {32, 64}): one warp per
// column; the CTA's 16 columns are staged (column-major, swizzled) in shared
// memory for coalesced row-major stores.
template <int EPL, bool kReversed>
__global__ void __launch_bounds__(kCW * 32)
ntt_cols_fwd_t_kernel(const uint32_t *__restrict__ bits, Pieces pc, int r1_log, uint32_t N, Tables T,
                      uint32_t *__restrict__ buf)
{
    constexpr uint32_t R1 = 32u * EPL, kStr = R1 + 1;
    extern __shared__ uint32_t xs[];  // kCW * kStr + R1
    const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
    const uint32_t g = blockIdx.y, c0 = blockIdx.x * kCW, t2 = c0 + c;
    uint32_t *col = xs + c * kStr;
    uint32_t *rb = xs + kCW * kStr;  // R1 staged row bits
    uint32_t lim;
    const uint32_t *b = piece_src(bits, pc, g, lim);
    stage_row_bits<kReversed>(rb, b, pc.len, lim, R1, c0);
    __syncthreads();
    uint32_t e[EPL];
#pragma unroll
    for (int j = 0; j < EPL; ++j) e[j] = (rb[32u * j + lane] >> c) & 1u;
    dif_warp_t<EPL, EPL / 2, false, true>(e, col, T.col_stage_f, lane);  // the twist takes [0, 4p)
    // layout B: e[32 q + i] is row r = 32 (lane + 32 q) + i, frequency bitrev(r)
    const uint32_t *twr = T.twist_f + (size_t)t2 * R1;
#pragma unroll
    for (int q = 0; q < EPL / 32; ++q)
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
            const uint32_t rr = 32u * (lane + 32 * q) + i;
            const uint4 tw = __ldg(reinterpret_cast<const uint4 *>(twr + rr));
            col[swz(rr)] = mont_lazy(e[32 * q + i], tw.x);
            col[swz(rr + 1)] = mont_lazy(e[32 * q + i + 1], tw.y);
            col[swz(rr + 2)] = mont_lazy(e[32 * q + i + 2], tw.z);
            col[swz(rr + 3)] = mont_lazy(e[32 * q + i + 3], tw.w);
        }
    __syncthreads();
    uint32_t *o = buf + (size_t)g * N;
    for (uint32_t it = threadIdx.x; it < R1 * kCW; it += blockDim.x) {
        const uint32_t cc = it % kCW, rr = it / kCW;
        o[(size_t)rr * kR2 + c0 + cc] = xs[cc * kStr + swz(rr)];
    }
}

// Pass A' with transposed warps: coalesced tile load, untwist, inverse DIT
// along t1, parity of the wanted coefficients into the output.
template <int EPL>
__global__ void __launch_bounds__(kCW * 32, EPL <= 32 ? 2 : 1)
ntt_cols_inv_t_kernel(const uint32_t *__restrict__ buf, uint64_t sub_stride, int r1_log, Tables T, uint32_t j0, uint32_t len,
                      uint32_t k, uint32_t *__restrict__ out)
{
    constexpr uint32_t R1 = 32u * EPL, kStr = R1 + 1;
    extern __shared__ uint32_t xs[];  // kCW * kStr
    const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
    const uint32_t g = blockIdx.y, c0 = blockIdx.x * kCW, t2 = c0 + c;
    uint32_t *col = xs + c * kStr;
    const uint32_t *in = buf + (size_t)g * sub_stride;
    for (uint32_t it = threadIdx.x; it < R1 * kCW; it += blockDim.x) {
        const uint32_t cc = it % kCW, rr = it / kCW;
        xs[cc * kStr + swz(rr)] = in[(size_t)rr * kR2 + c0 + cc];
    }
    __syncthreads();
    uint32_t e[EPL];
    const uint32_t *twr = T.twist_i + (size_t)t2 * R1;
#pragma unroll
    for (int q = 0; q < EPL / 32; ++q)
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
            const uint32_t rr = 32u * (lane + 32 * q) + i;
            const uint4 tw = __ldg(reinterpret_cast<const uint4 *>(twr + rr));
            e[32 * q + i] = mont_lazy(col[swz(rr)], tw.x);
            e[32 * q + i + 1] = mont_lazy(col[swz(rr + 1)], tw.y);
            e[32 * q + i + 2] = mont_lazy(col[swz(rr + 2)], tw.z);
            e[32 * q + i + 3] = mont_lazy(col[swz(rr + 3)], tw.w);
        }
    dit_warp_t<EPL, EPL / 2, true>(e, col, T.col_stage_i, lane);  // untwisted values are in [0, 2p)
    // layout A: e[j] is coefficient row t1 = 32 j + lane; store its parity
#pragma unroll
    for (int j = 0; j < EPL; ++j) col[swz(32u * j + lane)] = redp(red2p(e[j])) & 1u;
    __syncthreads();
    const uint64_t jk = (uint64_t)(j0 + g) * k;
    const uint32_t lo_t = len - 1, hi_t = len - 1 + k;
    for (uint32_t t1 = threadIdx.x; t1 < R1; t1 += blockDim.x) {
        const uint32_t base = t1 * kR2 + c0;
        if (base + kCW <= lo_t || base >= hi_t) continue;
        uint32_t bits16 = 0;
#pragma unroll
        for (int cc = 0; cc < kCW; ++cc) {
            const uint32_t t = base + cc;
            if (t >= lo_t && t < hi_t) bits16 |= xs[cc * kStr + swz(t1)] << cc;
        }
        uint64_t P;
        if (base < lo_t) {
            bits16 >>= (lo_t - base);
            P = jk;
        } else {
            P = jk + (base - lo_t);
        }
        if (!bits16) continue;
        const uint32_t sh = (uint32_t)(P & 31u);
        atomicXor(out + (P >> 5), bits16 << sh);
        if (sh > 16 && (bits16 >> (32u - sh))) atomicXor(out + (P >> 5) + 1, bits16 >> (32u - sh));
    }
}

// 32 x 32 bit transpose across a warp: on return bit c of lane r is bit r
// of lane c's input (five exchange rounds of swapping off-diagonal blocks).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane)
{
    const uint32_t masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int sft = 16 >> k;
        const uint32_t m = masks[k];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sft);
        x = (lane & sft) ? ((x & ~m) | ((y >> sft) & m)) : ((x & m) | ((y << sft) & ~m));
    }
    return x;
}

// ---- multi-column warps (R1 = 32 E, E in {1, 2, 4, 8, 16}) ---------------
// A warp transforms COLS = 32 / E columns at once: lane l, register j holds
// element 32 (j % E) + l of column j / E (layout A).  The distance >= 32
// stages pair registers of one column; the swizzled transpose then gives
// lane l the 32 consecutive elements 32 (l % E) .. 32 (l % E) + 31 of column
// l / E (layout B), where the distance < 32 stages run: no shuffles.  A CTA
// of NW warps covers CW = NW COLS adjacent columns; its R1 x CW tile sits in
// shared memory row-major, the column of row r XOR-ed with COLS (r / 32) so
// that both the per-lane column writes and the row-wise copies are
// conflict-free.
#ifndef EX_NTT_TC_COLS
#define EX_NTT_TC_COLS 1  // pass A on the tensor cores where R1 is 32, 64 or 128
#endif
#ifndef EX_COLS_WARPS
#define EX_COLS_WARPS 8
#endif
// Warps per CTA of the multi-column kernels for R1 = 32 E: EX_COLS_WARPS
// (8 or 16) where E allows it (the row swizzle needs COLS (E - 1) < CW, so
// at least E warps), else 16.  The R1 x CW tile is 1024 words per warp.
// Eight warps let four CTAs share an SM instead of two, so one CTA's loads
// and stores overlap another's butterflies: the 2^32-bit block's hash takes
// 38.4 instead of 40.3 ms (no change on the 2^30-bit block, E = 16).
// Per-warp transpose scratch of the multi-column kernels: padded rows
// (EX_COL_PAD; 33 x 32 words), else XOR swizzle (1024 words).  The R1 x CW
// tile (1024 words per warp) shares the region.
#ifndef EX_COL_PAD
#define EX_COL_PAD 1
#endif
constexpr bool kColPad = EX_COL_PAD != 0;
constexpr uint32_t kColSw = kColPad ? 33u * 32u : 1024u;
template <int E>
__host__ __device__ constexpr uint32_t col_warps() { return (EX_COLS_WARPS >= E) ? EX_COLS_WARPS : 16; }
template <int E>
constexpr uint32_t tile_words() { return col_warps<E>() * kColSw; }
template <int E>
size_t smem_multi() { return (size_t)(tile_words<E>() + 1024) * 4; }

template <int E>
__device__ __forceinline__ uint32_t tile_at(uint32_t r, uint32_t c)
{
    constexpr uint32_t COLS = 32u / E, CW = col_warps<E>() * COLS;
    return r * CW + (c ^ (COLS * (r >> 5)));
}

// The word whose bit c is element t0 + c of a piece (t0 % 32 == 0): read
// from position len - 1 - t (kReversed) or t of b, 0 where t >= len or the
// position is >= lim.  In two steps, so that the loads can be issued well
// before the word is needed: row_fetch loads the (at most two) source words,
// row_finish assembles the word from them.
template <bool kReversed>
__device__ __forceinline__ void row_fetch(const uint32_t *__restrict__ b, uint32_t len, uint32_t lim, uint32_t t0,
                                          uint32_t &a, uint32_t &c)
{
    a = c = 0u;
    if (t0 >= len) return;
    if (kReversed) {
        const int32_t hi = (int32_t)(len - 1 - t0), lo = hi - 31;
        const int32_t top = min(hi, (int32_t)lim - 1);
        if (top < max(lo, 0)) return;
        const int32_t w0 = lo >> 5, w1 = top >> 5;  // floor; w1 >= 0
        if (w0 >= 0) a = __ldg(b + w0);
        if (w1 != w0) c = __ldg(b + w1);
    } else if (t0 < min(len, lim)) {
        a = __ldg(b + (t0 >> 5));
    }
}
template <bool kReversed>
__device__ __forceinline__ uint32_t row_finish(uint32_t len, uint32_t lim, uint32_t t0, uint32_t a, uint32_t c)
{
    if (t0 >= len) return 0u;
    if (kReversed) {
        const int32_t hi = (int32_t)(len - 1 - t0), lo = hi - 31;
        const int32_t top = min(hi, (int32_t)lim - 1);
        if (top < max(lo, 0)) return 0u;
        const int32_t w0 = lo >> 5;
        const uint64_t v = ((uint64_t)c << 32) | a;
        const int32_t nb = top - lo + 1;  // 1 .. 32 positions kept
        const uint32_t f32 = (uint32_t)(v >> (lo - 32 * w0)) & (nb >= 32 ? ~0u : (1u << nb) - 1u);
        return __brev(f32);  // position lo + i -> column 31 - i
    }
    const uint32_t end = min(len, lim);
    if (t0 >= end) return 0u;
    return end - t0 < 32u ? a & ((1u << (end - t0)) - 1u) : a;
}
template <bool kReversed>
__device__ __forceinline__ uint32_t row_word(const uint32_t *__restrict__ b, uint32_t len, uint32_t lim, uint32_t t0)
{
    uint32_t a, c;
    row_fetch<kReversed>(b, len, lim, t0, a, c);
    return row_finish<kReversed>(len, lim, t0, a, c);
}

// Staged bits for CW >= 32 columns: rb[t1 * CW/32 + w] bit c is element
// t = t1 R2 + c0 + 32 w + c (c0 % 32 == 0).
template <bool kReversed, uint32_t WPR>
__device__ __forceinline__ void stage_row_words(uint32_t *rb, const uint32_t *__restrict__ b, uint32_t len,
                                                uint32_t lim, uint32_t R1, uint32_t c0)
{
    for (uint32_t it = threadIdx.x; it < R1 * WPR; it += blockDim.x) {
        const uint32_t t1 = it / WPR, wi = it % WPR;
        rb[it] = row_word<kReversed>(b, len, lim, t1 * kR2 + c0 + 32u * wi);
    }
}

// Pass A: bits -> DIF along t1 -> twist -> buf, for CW columns per CTA.
// kZeroTop: pieces of at most N / 2 coefficients (rows t1 >= R1 / 2 zero).
template <int E, bool kReversed, bool kZeroTop>
__global__ void __launch_bounds__(col_warps<E>() * 32, 32 / col_warps<E>())
ntt_cols_fwd_m_kernel(const uint32_t *__restrict__ bits, Pieces pc, uint32_t N, Tables T, uint32_t *__restrict__ buf)
{
    constexpr uint32_t COLS = 32u / E, R1 = 32u * E, CW = col_warps<E>() * COLS, WPR = CW / 32;
    extern __shared__ uint32_t xs[];  // tile (and warp scratch), then R1 * WPR staged bit words
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t g = blockIdx.y, c0 = blockIdx.x * CW;
    uint32_t *rb = xs + tile_words<E>();
    uint32_t lim;
    const uint32_t *b = piece_src(bits, pc, g, lim);
    stage_row_words<kReversed, WPR>(rb, b, pc.len, lim, R1, c0);
    __syncthreads();
    uint32_t e[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const uint32_t cc = w * COLS + j / E, t1 = 32u * (j % E) + lane;
        e[j] = (rb[t1 * WPR + (cc >> 5)] >> (cc & 31u)) & 1u;
    }
    dif_warp_t<32, E / 2, kZeroTop && (E >= 2), true, kColPad>(e, xs + w * kColSw, T.col_stage_f, lane);  // the twist takes [0, 4p)
    // layout B: e[i] is frequency row r = 32 a + i of column cc
    const uint32_t a = lane % E, cc = w * COLS + lane / E;
    const uint32_t *twr = T.twist_f + (size_t)(c0 + cc) * R1 + 32u * a;
#pragma unroll
    for (int i = 0; i < 32; i += 4) {
        const uint4 tw = __ldg(reinterpret_cast<const uint4 *>(twr + i));
        e[i] = mont_lazy(e[i], tw.x);
        e[i + 1] = mont_lazy(e[i + 1], tw.y);
        e[i + 2] = mont_lazy(e[i + 2], tw.z);
        e[i + 3] = mont_lazy(e[i + 3], tw.w);
    }
    __syncthreads();  // every warp is done with its scratch
#pragma unroll
    for (int i = 0; i < 32; ++i) xs[tile_at<E>(32u * a + i, cc)] = e[i];
    __syncthreads();
    // column pairs stay adjacent under the swizzle (COLS >= 2): 8-byte moves
    uint32_t *o = buf + (size_t)g * N;
    for (uint32_t it = threadIdx.x; it < R1 * CW / 2; it += blockDim.x) {
        const uint32_t r = it / (CW / 2), c = 2u * (it % (CW / 2));
        *reinterpret_cast<uint2 *>(o + (size_t)r * kR2 + c0 + c) =
            *reinterpret_cast<const uint2 *>(xs + tile_at<E>(r, c));
    }
}

// Pass A': coalesced tile load, untwist, inverse DIT along t1, parity of the
// wanted coefficients [len-1, len+k-1) into output bits j k + t - (len-1).
// The parities of a column are ballot-packed per 32 rows into column words
// (through shared memory), and each warp turns one 32 x 32 block of them
// into row words of 32 adjacent columns with a shuffle transpose.
template <int E>
__global__ void __launch_bounds__(col_warps<E>() * 32, 32 / col_warps<E>())
ntt_cols_inv_m_kernel(const uint32_t *__restrict__ buf, uint64_t sub_stride, Tables T, uint32_t j0, uint32_t len,
                      uint32_t k, uint32_t *__restrict__ out)
{
    constexpr uint32_t COLS = 32u / E, R1 = 32u * E, CW = col_warps<E>() * COLS, WPR = CW / 32;
    extern __shared__ uint32_t xs[];  // tile (and warp scratch), then CW x (E + 1) column words
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t g = blockIdx.y, c0 = blockIdx.x * CW;
    uint32_t *colw = xs + tile_words<E>();
    const uint32_t *in = buf + (size_t)g * sub_stride;
    for (uint32_t it = threadIdx.x; it < R1 * CW / 2; it += blockDim.x) {
        const uint32_t r = it / (CW / 2), c = 2u * (it % (CW / 2));
        *reinterpret_cast<uint2 *>(xs + tile_at<E>(r, c)) =
            __ldg(reinterpret_cast<const uint2 *>(in + (size_t)r * kR2 + c0 + c));
    }
    __syncthreads();
    const uint32_t a = lane % E, cc = w * COLS + lane / E;
    const uint32_t *twr = T.twist_i + (size_t)(c0 + cc) * R1 + 32u * a;
    uint32_t e[32];
#pragma unroll
    for (int i = 0; i < 32; i += 4) {
        const uint4 tw = __ldg(reinterpret_cast<const uint4 *>(twr + i));
        e[i] = mont_lazy(xs[tile_at<E>(32u * a + i, cc)], tw.x);
        e[i + 1] = mont_lazy(xs[tile_at<E>(32u * a + i + 1, cc)], tw.y);
        e[i + 2] = mont_lazy(xs[tile_at<E>(32u * a + i + 2, cc)], tw.z);
        e[i + 3] = mont_lazy(xs[tile_at<E>(32u * a + i + 3, cc)], tw.w);
    }
    __syncthreads();  // the tile is consumed; warps reuse it as scratch
    dit_warp_t<32, E / 2, true, kColPad>(e, xs + w * kColSw, T.col_stage_i, lane);  // untwisted values are in [0, 2p)
    // layout A: e[j] is coefficient row 32 (j % E) + lane of column w COLS + j / E;
    // only row blocks holding a wanted coefficient [len-1, len+k-1) are packed
    const uint32_t row_lo = (len - 1) / kR2, row_hi = (uint32_t)(((uint64_t)len + k - 2) / kR2);
    uint32_t mine = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (32u * (j % E) + 31u >= row_lo && 32u * (j % E) <= row_hi) {  // warp-uniform
            const uint32_t word = __ballot_sync(0xffffffffu, redp(red2p(e[j])) & 1u);
            if (lane == j) mine = word;
        }
    }
    colw[(w * COLS + lane / E) * (E + 1) + lane % E] = mine;  // column, 32-row block
    __syncthreads();
    // one 32 x 32 bit block per warp (E * CW / 32 = one per warp): rows
    // 32 b .. 32 b + 31 of columns 32 wi .. 32 wi + 31
    const uint32_t b = w % E, wi = w / E;
    uint32_t x = colw[(32u * wi + lane) * (E + 1) + b];  // lane c: column 32 wi + c
    x = transpose32(x, lane);                              // lane r: row 32 b + r
    const uint32_t t1 = 32u * b + lane;
    const uint32_t base = t1 * kR2 + c0 + 32u * wi;  // element of bit 0
    const uint32_t lo_t = len - 1, hi_t = len - 1 + k;
    if (base + 32 <= lo_t || base >= hi_t) return;
    if (hi_t - base < 32u) x &= (1u << (hi_t - base)) - 1u;
    uint64_t P = (uint64_t)(j0 + g) * k;  // output bit of element base (or of lo_t)
    if (base < lo_t) x >>= (lo_t - base);
    else P += base - lo_t;
    if (!x) return;
    const uint32_t sh = (uint32_t)(P & 31u);
    atomicXor(out + (P >> 5), x << sh);
    if (sh && (x >> (32u - sh))) atomicXor(out + (P >> 5) + 1, x >> (32u - sh));
}

// ---- pass A on the tensor cores (R1 in {32, 64, 128}) -------------------
// Pass A's inputs are bits, so its column DFTs are one exact integer GEMM per
// piece:
//   buf[r][t2] = w_N^(K t2) * sum_{t1} F[r][t1] x[t1 R2 + t2]  (mod p),
//   F[r][t1] = w_R1^(K t1),  K = bitrev(r),
// the values the butterfly kernels above write (in [0, 2p)).  F is cut into
// three 11-bit slices, F = F_0 + 2^11 F_1 + 2^22 F_2, each exact in f16; the
// bits are 0/1 in f16; every slice's sum has at most R1 terms below 2^11, so
// its f32 accumulator holds it exactly (below 2^18).  tcgen05.mma kind::f16
// with M = 128 columns t2 (one tensor-memory lane each), N = the three
// slices' rows of one half of the rows r (3 R1 / 2; each half has its own
// accumulators), K = the rows t1 that can hold data, rounded up to 16 (a
// piece of len coefficients has data in rows t1 < len / R2 only).  Each
// half's accumulators start at 2^23 (one multiply of two constant tiles,
// 256 x 32768), so a sum S < 2^18 reads back as the f32 bits 2^23 + S: the
// integer S sits in the low bits with no conversion.  F's slices stay in
// shared memory; the epilogue joins the three sums mod p, applies the twist
// and stores rows of buf with the lanes on consecutive columns.
//
// Persistent CTAs, one per SM, 21 warps in three roles:
//   warp 0      tensor-memory allocation; lane 0 issues the multiplies
//   warps 1-4   bits -> f16 operand (two shared-memory stages): warp 1 + w
//               expands columns 32 w .. 32 w + 31 of the 128-column tile
//   warps 5-20  epilogue: warp 5 + e takes a quarter of the rows (half
//               e / 8, its first or second R1 / 4 rows by (e / 4) % 2) in the
//               columns of its lane quarter (warp % 4)
// Each CTA keeps one 128-column block cb = blockIdx.x % 16 and walks the
// pieces blockIdx.x / 16, + g, + 2 g, ... (16 g CTAs), so an epilogue thread
// holds the twists of its column and rows in registers, loaded once.
// Every wait gives up after about a second (error word set, tensor memory
// freed after the last multiplies, return).
struct TcColsArgs {
    const uint32_t *bits;
    Pieces pc;
    uint32_t N;
    uint32_t npieces;     // pieces (virtual blocks) of the launch
    uint32_t g;           // CTAs per column block
    uint32_t k16;         // K steps of 16 rows t1
    const uint4 *fimg;    // F's slices in the shared-memory layout (6 R1^2 bytes)
    const uint32_t *twt;  // twist w_N^(bitrev(r) t2) at r R2 + t2, Montgomery form
    uint32_t *buf;
    uint32_t *err;
};

constexpr uint32_t kTcColsThreads = 21 * 32;
constexpr uint32_t kTcColsTile = 128;                    // columns t2 per tile
constexpr uint32_t kTcColBlocks = kR2 / kTcColsTile;     // 16 column blocks per row
constexpr uint32_t kHalfOne = 0x3C00u;                   // 1.0 in f16
constexpr uint16_t kHalf256 = 0x5C00u, kHalf32768 = 0x7800u;  // 2^8, 2^15 in f16: product 2^23
constexpr uint32_t kF32Int = 0x4B000000u;                // bits of 2^23: v + 2^23 holds integer v < 2^23
constexpr uint32_t kJoin = kF32Int * (1u + (1u << 11));  // the two offsets of u0 + 2^11 u1 (mod 2^32)
constexpr uint32_t kQ22 = (uint32_t)((1ull << 54) / kP); // Shoup quotient of 2^22

__host__ __device__ constexpr uint32_t tc_cols_ncols(uint32_t R1)
{
    return 3 * R1 <= 128 ? 128u : 3 * R1 <= 256 ? 256u : 512u;
}
// shared memory: F's slices, two stages, the two 16-column constant tiles
// (128 and 3 R1 / 2 rows), 8 barriers, tensor address, flag; at least half
// an SM's, so that one CTA holds an SM's tensor memory
__host__ __device__ constexpr uint32_t tc_cols_smem_need(uint32_t R1)
{
    return 6 * R1 * R1 + 512 * R1 + 4096 + 48 * R1 + 72;
}
__host__ __device__ constexpr uint32_t tc_cols_smem(uint32_t R1)
{
    return tc_cols_smem_need(R1) > kSmemPerSM / 2 + 1 ? tc_cols_smem_need(R1) : kSmemPerSM / 2 + 1;
}

// two bits -> two f16 (1.0 where set): element 2 i in the low half
__device__ __forceinline__ uint32_t two_halves(uint32_t y) { return (((y & 3u) * 0x8001u) & 0x10001u) * kHalfOne; }

template <uint32_t R1, bool kReversed>
__global__ void __launch_bounds__(kTcColsThreads, 1) ntt_cols_fwd_tc_kernel(TcColsArgs a)
{
    constexpr uint32_t NH = R1 / 2, kF = 6 * R1 * R1, kStage = 256 * R1, SBO = 16 * R1;
    constexpr uint32_t kCols = tc_cols_ncols(R1), kBiasA = 4096, kBiasB = 48 * R1;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *fs = sm, *as = sm + kF, *ba = sm + kF + 2 * kStage, *bb = ba + kBiasA;
    uint64_t *bars = reinterpret_cast<uint64_t *>(bb + kBiasB);  // a_full[2] a_empty[2] d_full[2] d_empty[2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 8);
    volatile uint32_t *abort_flag = tslot + 1;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t cb = blockIdx.x % kTcColBlocks, v0 = blockIdx.x / kTcColBlocks;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&bars[i]), 128);      // the four operand warps
            mbar_init(smem_u32(&bars[2 + i]), 1);    // tcgen05.commit
            mbar_init(smem_u32(&bars[4 + i]), 1);    // tcgen05.commit
            mbar_init(smem_u32(&bars[6 + i]), 256);  // the eight epilogue warps of the half
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (uint32_t i = tid; i < kF / 16; i += blockDim.x) reinterpret_cast<uint4 *>(fs)[i] = __ldg(a.fimg + i);
    // constant tiles (K = 16, K-major, core matrices of 8 rows x 16 bytes):
    // column 0 is 256 (rows of A) and 32768 (rows of B), the rest 0
    for (uint32_t i = tid; i < (kBiasA + kBiasB) / 16; i += blockDim.x) reinterpret_cast<uint4 *>(ba)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    if (tid < 128) *reinterpret_cast<uint16_t *>(ba + (tid >> 3) * 256 + (tid & 7) * 16) = kHalf256;
    if (tid < 3 * NH) *reinterpret_cast<uint16_t *>(bb + (tid >> 3) * 256 + (tid & 7) * 16) = kHalf32768;
    fence_async_smem();
    if (warp == 0) {
        tmem_alloc(smem_u32(tslot), kCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // descriptors advance by 256 bytes (16 in the address field) per
            // K step; the address field does not overflow (shared memory < 256 KB)
            const uint32_t idesc = tc_idesc_mn(128, 3 * NH);
            const uint64_t ad0 = smem_desc(smem_u32(as), 128, SBO), fd0 = smem_desc(smem_u32(fs), 128, SBO);
            const uint64_t bad = smem_desc(smem_u32(ba), 128, 256), bbd = smem_desc(smem_u32(bb), 128, 256);
            int64_t last = -1;  // last tile whose multiplies were committed
            uint32_t i = 0;
            for (uint32_t v = v0; v < a.npieces; v += a.g, ++i) {
                const uint32_t s = i & 1u;
                if (!mbar_wait(smem_u32(&bars[s]), (i >> 1) & 1u)) { *abort_flag = 1; break; }
                bool ok = true;
                for (uint32_t h = 0; h < 2 && ok; ++h) {
                    if (i >= 1 && !mbar_wait(smem_u32(&bars[6 + h]), (i - 1) & 1u)) { ok = false; break; }
                    tc_fence_after();
                    // the three slices of half h are rows 3 h NH .. 3 h NH + 3 NH - 1 of
                    // the F image: one multiply with N = 3 NH gives all three sums
                    uint64_t ad = ad0 + ((s * kStage) >> 4), bd = fd0 + ((3 * h * NH / 8 * SBO) >> 4);
                    tc_mma_f16(tmem + 3 * h * NH, bad, bbd, idesc, 0u);  // 2^23 everywhere
                    for (uint32_t ks = 0; ks < a.k16; ++ks) {
                        tc_mma_f16(tmem + 3 * h * NH, ad, bd, idesc, 1u);
                        ad += 16;
                        bd += 16;
                    }
                    tc_commit(smem_u32(&bars[4 + h]));
                }
                tc_commit(smem_u32(&bars[2 + s]));
                last = i;
                if (!ok) { *abort_flag = 1; break; }
            }
            // the stage barrier of the last commit arrives once every multiply is done
            if (last >= 0) mbar_wait(smem_u32(&bars[2 + (last & 1)]), (uint32_t)(last >> 1) & 1u);
        }
        __syncwarp();
    } else if (warp <= 4) {
        constexpr uint32_t RB = R1 / 32;  // 32-row blocks
        const uint32_t wc = warp - 1, m = 32 * wc + lane;  // this lane's tile column (row m of A)
        const uint32_t c0 = cb * kTcColsTile + 32 * wc, nrb = (16 * a.k16 + 31) / 32;
        // source words of the pieces two tiles ahead are in flight while a
        // stage is built (lane: row 32 u + lane of this warp's 32 columns)
        uint32_t wa0[RB], wb0[RB], wa1[RB], wb1[RB];
        auto fetch = [&](uint32_t v, uint32_t (&wa)[RB], uint32_t (&wb)[RB]) {
            if (v >= a.npieces) return;
            uint32_t lim;
            const uint32_t *src = piece_src(a.bits, a.pc, v, lim);
#pragma unroll
            for (uint32_t u = 0; u < RB; ++u)
                if (u < nrb) row_fetch<kReversed>(src, a.pc.len, lim, (32 * u + lane) * kR2 + c0, wa[u], wb[u]);
        };
        // build stage i & 1 from piece v; false when a wait gave up
        auto build = [&](uint32_t v, uint32_t i, const uint32_t (&wa)[RB], const uint32_t (&wb)[RB]) -> bool {
            const uint32_t s = i & 1u;
            if (i >= 2 && !__all_sync(~0u, mbar_wait(smem_u32(&bars[2 + s]), ((i >> 1) - 1) & 1u))) return false;
            uint32_t lim;
            piece_src(a.bits, a.pc, v, lim);
            uint8_t *st = as + s * kStage + (m >> 3) * SBO + (m & 7u) * 16;
#pragma unroll
            for (uint32_t u = 0; u < RB; ++u) {
                if (u >= nrb) break;
                const uint32_t t0 = (32 * u + lane) * kR2 + c0;
                // lane = row 32 u + lane -> lane = column c0 + lane, bit i = row 32 u + i
                const uint32_t x = transpose32(row_finish<kReversed>(a.pc.len, lim, t0, wa[u], wb[u]), lane);
#pragma unroll
                for (uint32_t q = 0; q < 4; ++q) {
                    const uint32_t y = x >> (8 * q);
                    *reinterpret_cast<uint4 *>(st + (4 * u + q) * 128) =
                        make_uint4(two_halves(y), two_halves(y >> 2), two_halves(y >> 4), two_halves(y >> 6));
                }
            }
            fence_async_smem();  // the stage's generic writes, visible to the tensor core
            mbar_arrive(smem_u32(&bars[s]));
            return true;
        };
        fetch(v0, wa0, wb0);
        fetch(v0 + a.g, wa1, wb1);
        uint32_t i = 0;
        for (uint32_t v = v0; v < a.npieces;) {
            if (!build(v, i, wa0, wb0)) { *abort_flag = 1; break; }
            fetch(v + 2 * a.g, wa0, wb0);
            v += a.g;
            ++i;
            if (v >= a.npieces) break;
            if (!build(v, i, wa1, wb1)) { *abort_flag = 1; break; }
            fetch(v + 2 * a.g, wa1, wb1);
            v += a.g;
            ++i;
        }
    } else {
        constexpr uint32_t NQ = NH / 2;  // rows per epilogue warp
        const uint32_t e = warp - 5, h = e >> 3, q = warp & 3u, r0 = h * NH + ((e >> 2) & 1u) * NQ;
        const uint32_t tl = tmem + ((32u * q) << 16) + 3 * h * NH + (r0 - h * NH);
        const uint32_t t2 = cb * kTcColsTile + 32 * q + lane;
        uint32_t tw[NQ];  // twists of rows r0 .. r0 + NQ - 1 in this lane's column
#pragma unroll
        for (uint32_t j = 0; j < NQ; ++j) tw[j] = __ldg(a.twt + (size_t)(r0 + j) * kR2 + t2);
        uint32_t i = 0;
        for (uint32_t v = v0; v < a.npieces; v += a.g, ++i) {
            if (!__all_sync(~0u, mbar_wait(smem_u32(&bars[4 + h]), i & 1u))) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            uint32_t *o = a.buf + (size_t)v * a.N + (size_t)r0 * kR2 + t2;
#pragma unroll
            for (uint32_t rc = 0; rc < NQ; rc += 8) {
                uint32_t s0[8], s1[8], s2[8];  // f32 bits of 2^23 + S: S in the low bits
                tmem_ld8(tl + rc, s0);
                tmem_ld8(tl + NH + rc, s1);
                tmem_ld8(tl + 2 * NH + rc, s2);
                tmem_wait_ld();
#pragma unroll
                for (uint32_t j = 0; j < 8; ++j) {
                    // F_0 x + 2^11 F_1 x + (2^22 F_2 x mod p) < 2^18 + 2^29 + 2p < 4p
                    const uint32_t val = s0[j] + (s1[j] << 11) + shoup_lazy(s2[j] - kF32Int, 1u << 22, kQ22) - kJoin;
                    o[(size_t)(rc + j) * kR2] = mont_lazy(val, tw[rc + j]);
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&bars[6 + h]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && tid == 0) atomicOr(a.err, 1u);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// Transposed twist table for the tensor-core pass A: twt[r R2 + t2] =
// w_N^(bitrev(r) t2), Montgomery form.
__global__ void ntt_twist_t_kernel(uint32_t *twt, uint32_t R1, int r1_log, Tables T)
{
    const uint32_t total = R1 * kR2;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        twt[i] = twist_mont(T.tw_lo_f, T.tw_hi_f, bitrev(i / kR2, r1_log) * (i % kR2));
}

// ---- host side -----------------------------------------------------------
uint32_t powmod(uint64_t b, uint64_t e)
{
    uint64_t r = 1;
    b %= kP;
    while (e) {
        if (e & 1) r = r * b % kP;
        b = b * b % kP;
        e >>= 1;
    }
    return (uint32_t)r;
}
uint32_t shoup_q(uint32_t w) { return (uint32_t)(((uint64_t)w << 32) / kP); }
uint32_t to_mont(uint32_t w) { return (uint32_t)(((uint64_t)w << 32) % kP); }
uint32_t host_bitrev(uint32_t x, int bits)
{
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}
// f16 bits of an integer 0 <= v < 2048 (exact: at most 11 significant bits)
uint16_t half_of_int(uint32_t v)
{
    if (!v) return 0;
    int e = 0;
    while ((v >> (e + 1)) != 0) ++e;
    return (uint16_t)(((uint32_t)(e + 15) << 10) | ((v << (10 - e)) & 0x3ffu));
}

}  // namespace

struct NttPlan {
    int e = 0, r1_log = 0;
    uint32_t N = 0, R1 = 0, G = 0;
    uint32_t P = 1, h = 0;  // pieces per sub-block and coefficients per piece
    uint32_t *buf = nullptr, *S = nullptr, *Sq = nullptr, *tables = nullptr, *twist = nullptr;
    bool own_buf = true;
    // independent seeds: every sub-block's windows are transformed per run,
    // or (resident) once at create into S, m P N words
    bool per_block = false;
    bool resident = false;
    const uint32_t *seed = nullptr;  // sub-block j's seed at seed + j seed_stride words
    uint64_t seed_stride = 0;
    uint32_t L = 0;                  // bits per seed (s + k - 1)
    Tables T{};
    // tensor-core pass A (R1 in {32, 64, 128}): transposed twist (N words),
    // then F's slices in the shared-memory layout (6 R1^2 bytes)
    bool tc_cols = false;
    uint32_t *tc_mem = nullptr;
    uint32_t sms = 0;
    uint32_t *err = nullptr;  // device word: a tensor-core wait gave up
};

namespace {

// dynamic shared memory of the column kernels (+ R1 words of staged row
// bits); 32 <= R1 < 1024 kernels take smem_multi<E>()
size_t smem_generic(uint32_t R1) { return (size_t)R1 * (kCS + 1) * 4; }         // R1 < 32 kernels
size_t smem_transposed(uint32_t R1) { return ((size_t)kCW * (R1 + 1) + R1) * 4; }  // R1 >= 1024 kernels

// The tensor-core pass A for the g * pc.P pieces of g source rows.
int ntt_launch_a_tc(const NttPlan *p, const uint32_t *bits, const Pieces &pc, bool reversed, uint32_t g,
                    uint32_t *dst, cudaStream_t st)
{
    const uint32_t R1 = p->R1;
    const uint64_t pieces = (uint64_t)g * pc.P;
    if (pieces >= (1ull << 31)) return set_error(EXTRACT_EINTERNAL, "ntt: %llu pieces", (unsigned long long)pieces);
    TcColsArgs a{};
    a.bits = bits;
    a.pc = pc;
    a.N = p->N;
    a.npieces = (uint32_t)pieces;
    a.g = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(p->sms / kTcColBlocks, pieces));
    a.k16 = (uint32_t)std::min<uint64_t>(R1 / 16, std::max<uint64_t>(1, ceil_div(pc.len, 16ull * kR2)));
    a.twt = p->tc_mem;
    a.fimg = reinterpret_cast<const uint4 *>(p->tc_mem + p->N);
    a.buf = dst;
    a.err = p->err;
    const uint32_t grid = a.g * kTcColBlocks;
#define EX_TC_COLS(R)                                                                                       \
    if (R1 == R) {                                                                                          \
        if (reversed) ntt_cols_fwd_tc_kernel<R, true><<<grid, kTcColsThreads, tc_cols_smem(R), st>>>(a);    \
        else ntt_cols_fwd_tc_kernel<R, false><<<grid, kTcColsThreads, tc_cols_smem(R), st>>>(a);            \
        return EXTRACT_OK;                                                                                  \
    }
    EX_TC_COLS(32)
    EX_TC_COLS(64)
    EX_TC_COLS(128)
#undef EX_TC_COLS
    return set_error(EXTRACT_EINTERNAL, "ntt: no tensor-core column kernel for R1=%u", R1);
}

// pass A for the g * pc.P pieces of g source rows into dst (N words each)
int ntt_launch_a(const NttPlan *p, const uint32_t *bits, const Pieces &pc, bool reversed, uint32_t g, uint32_t *dst,
                 cudaStream_t st)
{
    if (p->tc_cols) return ntt_launch_a_tc(p, bits, pc, reversed, g, dst, st);
    const dim3 grid(kR2 / kCW, g * pc.P);
    const uint32_t R1 = p->R1;
    if (R1 < 32) {
        const size_t smem = smem_generic(R1);
        if (reversed)
            ntt_pass_a_kernel<true><<<grid, kThreads, smem, st>>>(bits, pc, R1, p->r1_log, p->N, p->T, dst);
        else
            ntt_pass_a_kernel<false><<<grid, kThreads, smem, st>>>(bits, pc, R1, p->r1_log, p->N, p->T, dst);
        return EXTRACT_OK;
    }
    const int epl = (int)(R1 / 32);
#define EX_COLS_FWD_M(E)                                                                                     \
    if (epl == E) {                                                                                          \
        constexpr uint32_t nt = col_warps<E>() * 32;                                                        \
        const dim3 gm(kR2 / (nt / E), g * pc.P);                                                             \
        const size_t sm = smem_multi<E>();                                                                   \
        if (2ull * pc.len <= p->N) {                                                                         \
            if (reversed) ntt_cols_fwd_m_kernel<E, true, true><<<gm, nt, sm, st>>>(bits, pc, p->N, p->T, dst); \
            else ntt_cols_fwd_m_kernel<E, false, true><<<gm, nt, sm, st>>>(bits, pc, p->N, p->T, dst);       \
        } else {                                                                                             \
            if (reversed) ntt_cols_fwd_m_kernel<E, true, false><<<gm, nt, sm, st>>>(bits, pc, p->N, p->T, dst); \
            else ntt_cols_fwd_m_kernel<E, false, false><<<gm, nt, sm, st>>>(bits, pc, p->N, p->T, dst);      \
        }                                                                                                    \
        return EXTRACT_OK;                                                                                   \
    }
#define EX_COLS_FWD(E, K, SMEM)                                                                 \
    if (epl == E) {                                                                             \
        if (reversed) K<E, true><<<grid, kCW * 32, SMEM, st>>>(bits, pc, p->r1_log, p->N, p->T, dst); \
        else K<E, false><<<grid, kCW * 32, SMEM, st>>>(bits, pc, p->r1_log, p->N, p->T, dst);       \
        return EXTRACT_OK;                                                                      \
    }
    EX_COLS_FWD_M(1)
    EX_COLS_FWD_M(2)
    EX_COLS_FWD_M(4)
    EX_COLS_FWD_M(8)
    EX_COLS_FWD_M(16)
    EX_COLS_FWD(32, ntt_cols_fwd_t_kernel, smem_transposed(R1))
    EX_COLS_FWD(64, ntt_cols_fwd_t_kernel, smem_transposed(R1))
#undef EX_COLS_FWD_M
#undef EX_COLS_FWD
    return set_error(EXTRACT_EINTERNAL, "ntt: no column kernel for R1=%u", R1);
}

// pass B over the g * R1 output rows of dst; one CTA of two warps per row.
// inverse: the P pieces of each sub-block times their spectra, summed and
// transformed back; else the forward DIF of one piece (P = 1).
void ntt_launch_rows(const NttPlan *p, uint32_t *dst, uint32_t g, uint32_t P, const uint32_t *S, const uint32_t *Sq,
                     bool inverse, cudaStream_t st, bool per_block = false)
{
    const uint32_t rows = p->R1 * g;
    uint32_t *e = p->err;
    if (!inverse) ntt_rows_kernel<false, false><<<rows, 64, 0, st>>>(dst, p->N, p->R1, 1, S, Sq, p->T, e);
    else if (per_block && P == 1) ntt_rows_kernel<true, false, true><<<rows, 64, 0, st>>>(dst, p->N, p->R1, 1, S, Sq, p->T, e);
    else if (per_block) ntt_rows_kernel<true, true, true><<<rows, 64, 0, st>>>(dst, p->N, p->R1, P, S, Sq, p->T, e);
    else if (P == 1) ntt_rows_kernel<true, false><<<rows, 64, 0, st>>>(dst, p->N, p->R1, 1, S, Sq, p->T, e);
    else ntt_rows_kernel<true, true><<<rows, 64, 0, st>>>(dst, p->N, p->R1, P, S, Sq, p->T, e);
}

// pass A' for g sub-blocks of buf (P N words apart), output bits of
// sub-blocks j0 .. j0+g-1
int ntt_launch_a_inv(const NttPlan *p, const uint32_t *buf, uint32_t g, uint32_t j0, uint32_t k, uint32_t *out,
                     cudaStream_t st)
{
    const dim3 grid(kR2 / kCW, g);
    const uint32_t R1 = p->R1;
    const uint64_t sub = (uint64_t)p->P * p->N;
    if (R1 < 32) {
        ntt_pass_a_inv_kernel<<<grid, kThreads, smem_generic(R1), st>>>(buf, sub, R1, p->r1_log, p->T, j0, p->h, k, out);
        return EXTRACT_OK;
    }
    const int epl = (int)(R1 / 32);
#define EX_COLS_INV_M(E)                                                                                 \
    if (epl == E) {                                                                                      \
        constexpr uint32_t nt = col_warps<E>() * 32;                                                    \
        const dim3 gm(kR2 / (nt / E), g);                                                                \
        ntt_cols_inv_m_kernel<E><<<gm, nt, smem_multi<E>(), st>>>(buf, sub, p->T, j0, p->h, k, out);     \
        return EXTRACT_OK;                                                                               \
    }
#define EX_COLS_INV(E, K, SMEM)                                                          \
    if (epl == E) {                                                                      \
        K<E><<<grid, kCW * 32, SMEM, st>>>(buf, sub, p->r1_log, p->T, j0, p->h, k, out); \
        return EXTRACT_OK;                                                               \
    }
    EX_COLS_INV_M(1)
    EX_COLS_INV_M(2)
    EX_COLS_INV_M(4)
    EX_COLS_INV_M(8)
    EX_COLS_INV_M(16)
    EX_COLS_INV(32, ntt_cols_inv_t_kernel, smem_transposed(R1))
    EX_COLS_INV(64, ntt_cols_inv_t_kernel, smem_transposed(R1))
#undef EX_COLS_INV_M
#undef EX_COLS_INV
    return set_error(EXTRACT_EINTERNAL, "ntt: no column kernel for R1=%u", R1);
}

}  // namespace

// Relative cost of `transforms` transforms of length N.  Lengths below 2^16
// (R1 < 32 columns) run the generic column kernels, with one barrier per
// stage, measured 3.7x slower per butterfly than the warp-transposed ones.
double ntt_cost_units(uint32_t transforms, uint32_t N)
{
    const double c = (double)transforms * (double)N * (std::log2((double)N) + 4.0);
    return N < (1u << 16) ? 3.7 * c : c;
}

// Split of a sub-block into P pieces (1 <= P <= 16) of h coefficients (h a
// multiple of 32 when P > 1, so pieces start on word boundaries): each piece
// is its own middle product with seed window q h .. q h + h + k - 2, and the
// P products add up in the frequency domain, so one inverse transform serves
// them all.  Length N = 2^e >= h + k - 1 (2^12 .. 2^22); work P + 1
// transforms of N instead of 2 of the length for s + k - 1.  P need not be a
// power of two: with k = 0.1 s, seven pieces fit N = 2^18 as eight do (8
// transforms instead of 9).  split_log2 >= 0 forces P = 2^split_log2.
NttShape ntt_shape(uint32_t s, uint32_t k, int split_log2, bool per_block_seeds)
{
    NttShape best{};
    if ((uint64_t)s + k - 1 <= kR2 || s >= kP) return best;
    const uint32_t bufs = per_block_seeds ? 2u : 1u;  // data pieces (+ seed windows)
    double best_cost = 0;
    for (uint32_t P = 1; P <= (1u << kMaxSplitLog2); ++P) {
        if (split_log2 >= 0 && P != (1u << split_log2)) continue;
        const uint64_t h = P == 1 ? s : (((uint64_t)s + P - 1) / P + 31) / 32 * 32;
        if ((uint64_t)(P - 1) * h >= s) continue;  // the last piece would be empty
        uint64_t N = 2 * kR2;
        while (N < h + k - 1) N <<= 1;
        if (N > (1ull << 22) || bufs * P * N > kMaxWorkWords) continue;
        if (per_block_seeds && N < (1u << 16)) continue;  // needs the full twist tables (R1 >= 32)
        // transforms per sub-block: P data pieces (+ P seed windows) + 1 inverse
        const double cost = ntt_cost_units(bufs * P + 1, (uint32_t)N);
        if (best.N == 0 || cost < best_cost) {
            best = NttShape{(uint32_t)N, P, (uint32_t)h};
            best_cost = cost;
        }
    }
    return best;
}

bool ntt_eligible(uint32_t s, uint32_t k) { return ntt_shape(s, k).N != 0; }

void ntt_destroy_async(NttPlan *p, cudaStream_t st)
{
    if (!p) return;
    if (p->own_buf && p->buf) cudaFreeAsync(p->buf, st);
    if (p->S) cudaFreeAsync(p->S, st);
    if (p->Sq) cudaFreeAsync(p->Sq, st);
    if (p->tables) cudaFreeAsync(p->tables, st);
    if (p->twist) cudaFreeAsync(p->twist, st);
    if (p->tc_mem) cudaFreeAsync(p->tc_mem, st);
    delete p;
}

void ntt_destroy(NttPlan *p)
{
    if (!p) return;
    if (p->own_buf) cudaFree(p->buf);
    cudaFree(p->S);
    cudaFree(p->Sq);
    cudaFree(p->tables);
    cudaFree(p->twist);
    cudaFree(p->tc_mem);
    delete p;
}


uint64_t ntt_plan_bytes(uint32_t s, uint32_t k, int split_log2, bool per_block_seeds)
{
    const NttShape sh = ntt_shape(s, k, split_log2, per_block_seeds);
    // P spectra + quotients (shared seed) or the scaled inverse twist table
    // (independent seeds), twist tables, stage tables
    return (per_block_seeds ? 3ull : 2ull * sh.P + 2) * sh.N * 4 + 64 * 1024;
}

// sub-blocks per launch group: keep the working buffer near 64 MB (L2-sized)
static uint32_t group_size(uint32_t m, const NttShape &sh, bool per_block_seeds)
{
    const uint64_t per_sub = (per_block_seeds ? 2ull : 1ull) * sh.P * sh.N;
    // pass A launches one CTA row per piece (grid y = sub-blocks x P < 2^16)
    const uint64_t cap = 32768u / sh.P;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(std::min<uint64_t>(m, cap), kGroupWorkWords / per_sub));
}

uint64_t ntt_max_work_words() { return kGroupWorkWords; }

uint64_t ntt_work_words(uint32_t m, uint32_t s, uint32_t k, int split_log2, bool per_block_seeds)
{
    const NttShape sh = ntt_shape(s, k, split_log2, per_block_seeds);
    return (uint64_t)group_size(m, sh, per_block_seeds) * (per_block_seeds ? 2u : 1u) * sh.P * sh.N;
}

double ntt_work_butterflies(uint32_t m, uint32_t s, uint32_t k, int split_log2, bool per_block_seeds)
{
    const NttShape sh = ntt_shape(s, k, split_log2, per_block_seeds);
    const uint32_t transforms = (per_block_seeds ? 2u : 1u) * sh.P + 1;
    return (double)m * transforms * (sh.N / 2) * std::log2((double)std::max<uint32_t>(sh.N, 2));
}

// tw'[i] = tw[i] c 2^-32 (Montgomery product): the per-block plans' inverse
// twist, scaled by 1/N and by 2^32 to undo their Montgomery row products.
__global__ void ntt_scale_table_kernel(const uint32_t *tw, uint32_t *out, uint32_t n, uint32_t c)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = mul_mont(tw[i], c);
}

// Once per device: every column kernel's dynamic shared-memory limit (set
// to the most any plan launches it with, so plans of different lengths can
// share the kernels) and the distance < 32 twiddles in the constant bank
// (they depend only on the prime).  Complete before it returns.
static int device_setup(cudaStream_t st)
{
    static std::mutex mu;
    static uint64_t done = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "ntt device");
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && ((done >> dev) & 1u)) return EXTRACT_OK;
    auto attr = [&](const void *f, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    const size_t small = smem_generic(16);  // R1 < 32
    attr((const void *)ntt_pass_a_kernel<false>, small);
    attr((const void *)ntt_pass_a_kernel<true>, small);
    attr((const void *)ntt_pass_a_inv_kernel, small);
#define EX_SET_SMEM(E, KF, KI, SMEM)          \
    attr((const void *)KF<E, true>, SMEM);  \
    attr((const void *)KF<E, false>, SMEM); \
    attr((const void *)KI<E>, SMEM);
#define EX_SET_SMEM_M(E)                                                            \
    attr((const void *)ntt_cols_fwd_m_kernel<E, true, true>, smem_multi<E>());    \
    attr((const void *)ntt_cols_fwd_m_kernel<E, false, true>, smem_multi<E>());   \
    attr((const void *)ntt_cols_fwd_m_kernel<E, true, false>, smem_multi<E>());   \
    attr((const void *)ntt_cols_fwd_m_kernel<E, false, false>, smem_multi<E>());  \
    attr((const void *)ntt_cols_inv_m_kernel<E>, smem_multi<E>());
    EX_SET_SMEM_M(1)
    EX_SET_SMEM_M(2)
    EX_SET_SMEM_M(4)
    EX_SET_SMEM_M(8)
    EX_SET_SMEM_M(16)
    EX_SET_SMEM(32, ntt_cols_fwd_t_kernel, ntt_cols_inv_t_kernel, smem_transposed(1024))
    EX_SET_SMEM(64, ntt_cols_fwd_t_kernel, ntt_cols_inv_t_kernel, smem_transposed(2048))
#undef EX_SET_SMEM
#undef EX_SET_SMEM_M
#define EX_SET_SMEM_TC(R)                                                         \
    attr((const void *)ntt_cols_fwd_tc_kernel<R, true>, tc_cols_smem(R));  \
    attr((const void *)ntt_cols_fwd_tc_kernel<R, false>, tc_cols_smem(R));
    EX_SET_SMEM_TC(32)
    EX_SET_SMEM_TC(64)
    EX_SET_SMEM_TC(128)
#undef EX_SET_SMEM_TC
    if (e != cudaSuccess) return cuda_error(e, "ntt smem attribute");
    uint2 lf[31], li[31];
    for (uint32_t hh = 1; hh <= 16; hh <<= 1) {
        const uint32_t wf = powmod(kGen, (kP - 1) / (2 * hh)), wi = powmod(wf, kP - 2);
        for (uint32_t r = 0; r < hh; ++r) {
            const uint32_t a = powmod(wf, r), b = powmod(wi, r);
            lf[hh - 1 + r] = make_uint2(a, shoup_q(a));
            li[hh - 1 + r] = make_uint2(b, shoup_q(b));
        }
    }
    // complete before the flag is set: another thread may launch at once
    if ((e = cudaMemcpyToSymbolAsync(c_low_f, lf, sizeof(lf), 0, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyToSymbolAsync(c_low_i, li, sizeof(li), 0, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_error(e, "ntt constant twiddles");
    if (dev < 64) done |= 1ull << dev;
    return EXTRACT_OK;
}

// seed_dev: realigned seed bits (bit t = seed[t]), L = s + k - 1 bits; with
// seed_stride > 0 one seed per sub-block, seed_stride words apart.
static Pieces seed_pieces(const NttPlan *p, uint32_t k);

int ntt_create(NttPlan **out, uint32_t m, uint32_t s, uint32_t k, const uint32_t *seed_dev, cudaStream_t st,
               uint32_t *work, int split_log2, uint64_t seed_stride, bool resident_spectra)
{
    *out = nullptr;
    const bool per_block = seed_stride > 0;
    const NttShape sh = ntt_shape(s, k, split_log2, per_block);
    if (!sh.N) return set_error(EXTRACT_EINVAL, "no NTT shape for s=%u k=%u (split %d)", s, k, split_log2);
    NttPlan *p = new NttPlan();
    p->N = sh.N;
    p->P = sh.P;
    p->h = sh.h;
    p->per_block = per_block;
    p->seed = seed_dev;
    p->seed_stride = seed_stride;
    p->L = s + k - 1;
    p->e = 0;
    while ((1u << p->e) < p->N) ++p->e;
    p->R1 = p->N / kR2;
    p->r1_log = p->e - kR2Log;
    p->G = group_size(m, sh, per_block);
    const uint32_t R1 = p->R1;
    // table layout (words): col_f, col_fq, col_i, col_iq (R1/2 each, >= 1),
    // row_f, row_fq, row_i, row_iq (1024 each), tw_lo_f, tw_lo_i (2048),
    // tw_hi_f, tw_hi_i (R1 each, >= 1)
    const uint32_t ch = std::max<uint32_t>(1, R1 / 2);
    std::vector<uint32_t> h;
    auto push_stage = [&](uint32_t R, uint32_t count, bool inverse) {
        const uint32_t w = powmod(kGen, (kP - 1) / R);
        const uint32_t wi = powmod(w, kP - 2);
        std::vector<uint32_t> f(count), q(count);
        uint64_t cur = 1;
        for (uint32_t i = 0; i < count; ++i) {
            f[i] = (uint32_t)cur;
            q[i] = shoup_q(f[i]);
            cur = cur * (inverse ? wi : w) % kP;
        }
        h.insert(h.end(), f.begin(), f.end());
        h.insert(h.end(), q.begin(), q.end());
    };
    const size_t o_col_f = 0;
    push_stage(std::max<uint32_t>(2, R1), ch, false);
    const size_t o_col_i = h.size();
    push_stage(std::max<uint32_t>(2, R1), ch, true);
    const size_t o_row_f = h.size();
    push_stage(kR2, kR2 / 2, false);
    const size_t o_row_i = h.size();
    push_stage(kR2, kR2 / 2, true);
    // per-stage (w_2h^r, quotient) tables for the warp transforms, 8-byte aligned
    auto push_per_stage = [&](uint32_t R, bool inverse) {
        if (h.size() & 1) h.push_back(0);
        const size_t at = h.size();
        for (uint32_t hh = 1; hh < R; hh <<= 1) {
            const uint32_t w = powmod(kGen, (kP - 1) / (2 * hh));
            const uint32_t step = inverse ? powmod(w, kP - 2) : w;
            uint64_t cur = 1;
            for (uint32_t r = 0; r < hh; ++r) {
                h.push_back((uint32_t)cur);
                h.push_back(shoup_q((uint32_t)cur));
                cur = cur * step % kP;
            }
        }
        return at;
    };
    const size_t o_rs_f = push_per_stage(kR2, false), o_rs_i = push_per_stage(kR2, true);
    const size_t o_cs_f = push_per_stage(std::max<uint32_t>(2, R1), false);
    const size_t o_cs_i = push_per_stage(std::max<uint32_t>(2, R1), true);
    const uint32_t wN = powmod(kGen, (kP - 1) / p->N), wNi = powmod(wN, kP - 2);
    const size_t o_tw = h.size();
    for (int inv = 0; inv < 2; ++inv) {
        const uint32_t w = inv ? wNi : wN;
        for (uint32_t x = 0; x < kR2; ++x) h.push_back(to_mont(powmod(w, x)));
        const uint32_t w2 = powmod(w, kR2);
        for (uint32_t x = 0; x < std::max<uint32_t>(1, R1); ++x) h.push_back(to_mont(powmod(w2, x)));
    }
    const size_t o_err = h.size();
    h.push_back(0);
    int rc = EXTRACT_OK;
    do {
        cudaError_t e;
        if ((e = cudaMallocAsync(&p->tables, h.size() * 4, st)) != cudaSuccess) { rc = cuda_error(e, "ntt tables"); break; }
        if ((e = cudaMemcpyAsync(p->tables, h.data(), h.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_error(e, "ntt tables copy"); break; }
        const uint32_t *t = p->tables;
        p->err = p->tables + o_err;
        p->T.col_f = t + o_col_f; p->T.col_fq = t + o_col_f + ch;
        p->T.col_i = t + o_col_i; p->T.col_iq = t + o_col_i + ch;
        p->T.row_f = t + o_row_f; p->T.row_fq = t + o_row_f + kR2 / 2;
        p->T.row_i = t + o_row_i; p->T.row_iq = t + o_row_i + kR2 / 2;
        const uint32_t hiN = std::max<uint32_t>(1, R1);
        p->T.tw_lo_f = t + o_tw; p->T.tw_hi_f = t + o_tw + kR2;
        p->T.tw_lo_i = t + o_tw + kR2 + hiN; p->T.tw_hi_i = t + o_tw + 2 * kR2 + hiN;
        p->T.row_stage_f = reinterpret_cast<const uint2 *>(t + o_rs_f);
        p->T.row_stage_i = reinterpret_cast<const uint2 *>(t + o_rs_i);
        p->T.col_stage_f = reinterpret_cast<const uint2 *>(t + o_cs_f);
        p->T.col_stage_i = reinterpret_cast<const uint2 *>(t + o_cs_i);
        const size_t spec = (size_t)p->P * p->N;
        if (work) {
            p->buf = work;
            p->own_buf = false;
        } else if ((e = cudaMallocAsync(&p->buf, (size_t)p->G * spec * (per_block ? 2 : 1) * 4, st)) != cudaSuccess) {
            rc = cuda_error(e, "ntt buffer");
            break;
        }
        if (R1 >= 32) {
            if ((e = cudaMallocAsync(&p->twist, (size_t)(per_block ? 3 : 2) * p->N * 4, st)) != cudaSuccess) { rc = cuda_error(e, "ntt twist tables"); break; }
            p->T.twist_f = p->twist;
            p->T.twist_i = p->twist + p->N;
            ntt_twist_table_kernel<<<(uint32_t)std::min<uint64_t>(ceil_div(p->N, 256), 8192), 256, 0, st>>>(
                p->twist, p->twist + p->N, R1, p->r1_log, p->T);
            if (per_block) {  // inverse twist x 1/N x 2^32 (the row products are Montgomery)
                const uint64_t two32 = (1ull << 32) % kP, two64 = two32 * two32 % kP;
                const uint32_t c = (uint32_t)((uint64_t)powmod(p->N, kP - 2) * two64 % kP);
                ntt_scale_table_kernel<<<(uint32_t)std::min<uint64_t>(ceil_div(p->N, 256), 8192), 256, 0, st>>>(
                    p->twist + p->N, p->twist + 2 * (size_t)p->N, p->N, c);
                p->T.twist_i = p->twist + 2 * (size_t)p->N;
            }
        } else if (per_block) {
            rc = set_error(EXTRACT_EINVAL, "independent seeds need N >= 2^16");
            break;
        }
        if (EX_NTT_TC_COLS && (R1 == 32 || R1 == 64 || R1 == 128)) {
            // F's three 11-bit slices as f16 in the layout of the kernel's
            // shared memory: row r of slice l is image row n = (3 h + l) R1/2
            // + r - h R1/2 for the half h = r / (R1/2) it falls in (the three
            // slices of a half are consecutive rows, one multiply's N), at
            // byte (n / 8) 16 R1 + (kk / 8) 128 + (n % 8) 16 + (kk % 8) 2 for
            // column kk = t1
            const size_t fwords = (size_t)3 * R1 * R1 / 2;
            std::vector<uint16_t> img((size_t)3 * R1 * R1);
            const uint32_t wr = powmod(kGen, (kP - 1) / R1);
            const uint32_t NH = R1 / 2;
            for (uint32_t r = 0; r < R1; ++r) {
                const uint64_t K = host_bitrev(r, p->r1_log);
                const uint32_t h = r / NH;
                for (uint32_t kk = 0; kk < R1; ++kk) {
                    const uint32_t f = powmod(wr, K * kk % R1);
                    for (uint32_t l = 0; l < 3; ++l) {
                        const uint32_t n = (3 * h + l) * NH + (r - h * NH);
                        const size_t byte = (size_t)(n >> 3) * 16 * R1 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2;
                        img[byte / 2] = half_of_int((f >> (11 * l)) & 2047u);
                    }
                }
            }
            int dev = 0, sms = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
                (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
                (e = cudaMallocAsync(&p->tc_mem, ((size_t)p->N + fwords) * 4, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(p->tc_mem + p->N, img.data(), fwords * 4, cudaMemcpyHostToDevice, st)) !=
                    cudaSuccess) {
                rc = cuda_error(e, "ntt tensor-core tables");
                break;
            }
            ntt_twist_t_kernel<<<(uint32_t)std::min<uint64_t>(ceil_div(p->N, 256), 8192), 256, 0, st>>>(
                p->tc_mem, R1, p->r1_log, p->T);
            p->sms = (uint32_t)sms;
            p->tc_cols = true;
        }
        if ((rc = device_setup(st)) != EXTRACT_OK) break;
        if (per_block && resident_spectra) {
            // every sub-block's seed windows, group by group, through pass A
            // and the forward row pass into S (sub-block j's piece q at
            // (j P + q) N), the layout the inverse row pass reads
            if ((e = cudaMallocAsync(&p->S, (size_t)m * spec * 4, st)) != cudaSuccess) {
                cudaGetLastError();
                rc = set_error(EXTRACT_ENOMEM, "ntt: no room for %u resident seed spectra", m);
                break;
            }
            p->resident = true;
            for (uint32_t j0 = 0; j0 < m && rc == EXTRACT_OK; j0 += p->G) {
                const uint32_t g = std::min(p->G, m - j0);
                uint32_t *sj = p->S + (size_t)j0 * spec;
                if (int lrc = ntt_launch_a(p, p->seed + (size_t)j0 * p->seed_stride, seed_pieces(p, k), false, g, sj, st)) rc = lrc;
                else ntt_launch_rows(p, sj, g * p->P, 1, nullptr, nullptr, false, st);
            }
            if (rc != EXTRACT_OK) break;
        }
        if (per_block) {
            if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_error(e, "ntt tables"); break; }
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_error(e, "ntt tables"); break; }
            break;  // no shared spectrum
        }
        if ((e = cudaMallocAsync(&p->S, spec * 4, st)) != cudaSuccess) { rc = cuda_error(e, "ntt spectrum"); break; }
        if (!kSpectrumMont && (e = cudaMallocAsync(&p->Sq, spec * 4, st)) != cudaSuccess) { rc = cuda_error(e, "ntt spectrum"); break; }
        // seed spectra: for piece q, the window seed[q h .. q h + h + k - 1)
        // (zero past L = s + k - 1) through pass A + row DIF into S + q N;
        // then all are scaled by 1/N
        const uint32_t L = s + k - 1;
        for (uint32_t q = 0; q < p->P && rc == EXTRACT_OK; ++q) {
            const uint32_t off = q * p->h;  // a multiple of 32 when P > 1
            const uint32_t len = std::min(p->h + k - 1, L - off);
            const Pieces pc{0, 1, 0, len, len};
            if (int lrc = ntt_launch_a(p, seed_dev + off / 32, pc, false, 1, p->S + (size_t)q * p->N, st)) rc = lrc;
            else ntt_launch_rows(p, p->S + (size_t)q * p->N, 1, 1, nullptr, nullptr, false, st);
        }
        if (rc != EXTRACT_OK) break;
        const uint32_t ninv = powmod(p->N, kP - 2);
        const uint32_t c = kSpectrumMont ? (uint32_t)((uint64_t)ninv * ((1ull << 32) % kP) % kP) : ninv;
        ntt_finish_spectrum_kernel<<<(uint32_t)std::min<uint64_t>(ceil_div(spec, 256), 4096), 256, 0, st>>>(
            p->S, p->Sq, (uint32_t)spec, c, shoup_q(c));
        if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_error(e, "ntt spectrum kernels"); break; }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_error(e, "ntt spectrum"); break; }
    } while (0);
    if (rc != EXTRACT_OK) { ntt_destroy(p); return rc; }
    *out = p;
    return EXTRACT_OK;
}

// The pieces of stored sub-blocks: row g at g w_pad words, piece q from
// row bit q h (the reversed row's bit b holds A[s-1-b], so piece q holds
// coefficients s-(q+1)h .. s-q h-1, and bits past s read as 0).
static Pieces sub_block_pieces(const NttPlan *p, uint32_t w_pad, uint32_t s)
{
    return Pieces{w_pad, p->P, p->P > 1 ? p->h / 32 : 0u, p->h, s};
}

// The seed windows of sub-blocks j0 .. (independent seeds): window q of
// sub-block j starts at bit q h of its seed and holds h + k - 1 coefficients
// (0 past L): the seed window that meets piece q of the sub-block.
static Pieces seed_pieces(const NttPlan *p, uint32_t k)
{
    return Pieces{p->seed_stride, p->P, p->P > 1 ? p->h / 32 : 0u, std::min(p->h + k - 1, p->L), p->L};
}

// One launch group: the g sub-blocks from j0, in gb (the group's buffer).
static int ntt_group_run(const NttPlan *p, const uint32_t *arev, uint32_t w_pad, uint32_t j0, uint32_t g,
                         uint32_t k, const Pieces &pc, uint32_t *gb, uint32_t *out, cudaStream_t gs)
{
    if (int rc = ntt_launch_a(p, arev + (size_t)j0 * w_pad, pc, true, g, gb, gs)) return rc;
    if (!p->per_block) {
        ntt_launch_rows(p, gb, g, p->P, p->S, p->Sq, true, gs);
    } else if (p->resident) {
        ntt_launch_rows(p, gb, g, p->P, p->S + (size_t)j0 * p->P * p->N, nullptr, true, gs, true);
    } else {
        // the seed windows' spectra, transformed into the second half
        uint32_t *sb = gb + (size_t)p->G * p->P * p->N;
        if (int rc = ntt_launch_a(p, p->seed + (size_t)j0 * p->seed_stride, seed_pieces(p, k), false, g, sb, gs)) return rc;
        ntt_launch_rows(p, sb, g * p->P, 1, nullptr, nullptr, false, gs);
        ntt_launch_rows(p, gb, g, p->P, sb, nullptr, true, gs, true);
    }
    return ntt_launch_a_inv(p, gb, g, j0, k, out, gs);
}

// Hash every sub-block: out (zeroed here) gets K_j at bit j*k.
int ntt_hash(const NttPlan *p, const uint32_t *arev, uint32_t w_pad, uint32_t m, uint32_t s, uint32_t k,
             uint32_t *out, cudaStream_t st, uint32_t *work, const NttLanes *lanes, const NttHostOut *host_out)
{
    uint32_t *buf = work ? work : p->buf;
    const uint64_t out_words = ceil_div((uint64_t)m * k, 32);
    EX_CUDA(cudaMemsetAsync(out, 0, out_words * 4, st));
    const Pieces pc = sub_block_pieces(p, w_pad, s);
    const uint32_t groups = (uint32_t)ceil_div(m, p->G);
    // lanes past the group count stay idle
    const uint32_t L = 1u + (lanes ? std::min<uint32_t>((uint32_t)lanes->n, groups - 1u) : 0u);
    // per-group host copies need every word shared by at most two groups
    const bool per_group = host_out && host_out->nev >= groups && (uint64_t)p->G * k >= 64;
    if (L > 1) {
        EX_CUDA(cudaEventRecord(lanes->ev_fork, st));
        for (uint32_t l = 1; l < L; ++l) EX_CUDA(cudaStreamWaitEvent(lanes->st[l - 1], lanes->ev_fork, 0));
    }
    uint32_t gi = 0;
    uint64_t copied = 0;  // host words done
    for (uint32_t j0 = 0; j0 < m; j0 += p->G, ++gi) {
        const uint32_t g = std::min(p->G, m - j0);
        const uint32_t l = gi % L;
        cudaStream_t gs = l ? lanes->st[l - 1] : st;
        uint32_t *gb = l ? lanes->work[l - 1] : buf;
        if (int rc = ntt_group_run(p, arev, w_pad, j0, g, k, pc, gb, out, gs)) return rc;
        if (per_group) {
            EX_CUDA(cudaEventRecord(host_out->ev[gi], gs));
            EX_CUDA(cudaStreamWaitEvent(host_out->st, host_out->ev[gi], 0));
            if (gi) EX_CUDA(cudaStreamWaitEvent(host_out->st, host_out->ev[gi - 1], 0));
            const uint64_t hi = (uint64_t)(j0 + g) * k / 32;  // words below hold no later group's bits
            if (hi > copied)
                EX_CUDA(cudaMemcpyAsync(host_out->host + copied, out + copied, (hi - copied) * 4,
                                        cudaMemcpyDeviceToHost, host_out->st));
            copied = std::max(copied, hi);
        }
    }
    for (uint32_t l = 1; l < L; ++l) {
        EX_CUDA(cudaEventRecord(lanes->ev_join[l - 1], lanes->st[l - 1]));
        EX_CUDA(cudaStreamWaitEvent(st, lanes->ev_join[l - 1], 0));
    }
    if (host_out && copied < out_words) {
        EX_CUDA(cudaEventRecord(host_out->ev_end, st));
        EX_CUDA(cudaStreamWaitEvent(host_out->st, host_out->ev_end, 0));
        EX_CUDA(cudaMemcpyAsync(host_out->host + copied, out + copied, (out_words - copied) * 4,
                                cudaMemcpyDeviceToHost, host_out->st));
    }
    EX_LAUNCH("ntt kernels");
    return EXTRACT_OK;
}

int ntt_run_overlapped(const NttPlan *p, const uint32_t *in, const uint32_t *perm, uint32_t *arev, uint32_t w_pad,
                       uint32_t m, uint32_t s, uint32_t k, uint32_t *out, cudaStream_t st, cudaStream_t aux,
                       cudaEvent_t ev_fork, cudaEvent_t ev_group, int num_sms, bool padded, uint64_t input_bits)
{
    EX_CUDA(cudaEventRecord(ev_fork, st));
    EX_CUDA(cudaStreamWaitEvent(aux, ev_fork, 0));
    EX_CUDA(cudaMemsetAsync(out, 0, ceil_div((uint64_t)m * k, 32) * 4, st));
    const Pieces pc = sub_block_pieces(p, w_pad, s);
    for (uint32_t j0 = 0; j0 < m; j0 += p->G) {
        const uint32_t g = std::min(p->G, m - j0);
        uint32_t *ar = arev + (size_t)j0 * w_pad;
        if (int rc = launch_gather(in, perm, g, s, w_pad, ar, aux, num_sms, (uint64_t)j0 * s, padded, input_bits))
            return rc;
        // each wait binds to the record just before it, so one event serves every group
        EX_CUDA(cudaEventRecord(ev_group, aux));
        EX_CUDA(cudaStreamWaitEvent(st, ev_group, 0));
        if (int rc = ntt_group_run(p, arev, w_pad, j0, g, k, pc, p->buf, out, st)) return rc;
    }
    EX_LAUNCH("ntt kernels");
    return EXTRACT_OK;
}

uint32_t ntt_group(const NttPlan *p) { return p->G; }
bool ntt_spectra_resident(const NttPlan *p) { return p->resident; }
uint64_t ntt_resident_spectra_words(uint32_t m, uint32_t s, uint32_t k, int split_log2)
{
    const NttShape sh = ntt_shape(s, k, split_log2, true);
    return (uint64_t)m * sh.P * sh.N;
}
uint32_t ntt_size(const NttPlan *p) { return p->N; }
bool ntt_uses_tensor_cores(const NttPlan *p) { return p->tc_cols; }
uint32_t *ntt_error_word(const NttPlan *p) { return p ? p->err : nullptr; }

int ntt_status(const NttPlan *p)
{
    if (!p || !p->err) return EXTRACT_OK;
    uint32_t v = 0;
    EX_CUDA(cudaDeviceSynchronize());
    EX_CUDA(cudaMemcpy(&v, p->err, 4, cudaMemcpyDeviceToHost));
    if (!v) return EXTRACT_OK;
    EX_CUDA(cudaMemset(p->err, 0, 4));
    return set_error(EXTRACT_ETIMEDOUT, "a tensor-core NTT pass gave up waiting for its multiplies");
}
uint32_t ntt_pieces(const NttPlan *p) { return p->P; }

}  // namespace ex
