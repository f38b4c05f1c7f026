// The innermost part of BasisCvt / iBasisCvt (Alg. 1, Sec. 2.3.1): the
// conversion of every aligned 2^16-bit block on its own.
//
// For a length 2^K with 16 <= K <= 32, Alg. 1 splits at tau = 2^16 (the
// largest 2^i with i a power of two and i <= K - 1), so its last part is the
// same algorithm inside every block of 2^16 bits; for K >= 33 it splits at
// 2^32 and the 2^32-bit blocks again end with it.  Its step list, the
// flattening described in cvt.cu, is fixed: 32 (h, d) steps, generated below
// at compile time.
//
// GPU mapping: one warp per block, registers only.  Lane L holds the 32
// consecutive words 32L .. 32L+31 (2048 bits).  A step whose segments fit in
// 2048 bits (2h <= 2048) runs inside every lane with fixed register indices;
// a wider step (h >= 2^11, 15 of the 32) pairs lane L of the lower half of a
// segment with lane L + h/2048 of the upper half and moves the words it needs
// with warp shuffles.  No shared-memory barrier is taken between steps; shared
// memory only turns the coalesced load (lane L gets words L, L+32, ...) into
// the per-lane layout and back, with an XOR swizzle that keeps both sides free
// of bank conflicts.
#include "gf2x_common.cuh"

namespace gf2x {
namespace {

constexpr int kUnitWords = 1024;        // 2^16 bits

struct StepList {
    int n;
    signed char lh[40], ld[40];         // log2 h, log2 d (bits)
};

// Same recursion as the host planner: Taylor steps at s_i = x^tau + x, then
// the outer conversion (unit tau), then the inner one (unit 1).
constexpr void gen_steps(StepList &s, int K, int ulog)
{
    if (K <= 1) return;
    int i = 1;
    while (2 * i <= K - 1) i *= 2;
    for (int k = K - i - 1; k >= 0; --k) {
        s.lh[s.n] = (signed char)(i + k + ulog);
        s.ld[s.n] = (signed char)(k + ulog);
        ++s.n;
    }
    gen_steps(s, K - i, ulog + i);
    gen_steps(s, i, ulog);
}

constexpr StepList make_steps16()
{
    StepList s{};
    gen_steps(s, 16, 0);
    return s;
}

constexpr StepList kSteps16 = make_steps16();
static_assert(kSteps16.n == 32, "BasisCvt of 2^16 bits has 32 steps");

constexpr u64 seg_mask(int h, int lo_bit, int hi_bit)
{
    // bits [lo_bit, hi_bit) of every 2h-bit segment of a word (h < 64)
    u64 one = ((1ull << (hi_bit - lo_bit)) - 1) << lo_bit;
    u64 m = 0;
    for (int s = 0; s < 64; s += 2 * h) m |= one << s;
    return m;
}

__device__ __forceinline__ u64 shfl(u64 v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// One step (h = 2^LH, d = 2^LD bits) on the block held by the warp.
// Forward: hi' = hi with its quotient fix, lo ^= (hi' << d) mod x^h.
// Inverse: lo ^= (hi << d) mod x^h with the current hi, then the fix.
template <int LH, int LD, bool INV>
__device__ __forceinline__ void step(u64 (&w)[32], int lane)
{
    if constexpr (LH < 6) {
        // segments inside one word
        constexpr int h = 1 << LH, d = 1 << LD, sh = h - d;
        constexpr u64 ma = seg_mask(h, h, h + d);      // bottom d bits of hi
        constexpr u64 mb = seg_mask(h, d, h);          // lo bits [d, h)
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            u64 x = w[j];
            if (!INV) {
                x ^= (x >> sh) & ma;
                x ^= (x >> sh) & mb;
            } else {
                x ^= (x >> sh) & mb;
                x ^= (x >> sh) & ma;
            }
            w[j] = x;
        }
    } else if constexpr (LH <= 10) {
        // segments of 2hw <= 32 words, inside one lane
        constexpr int hw = 1 << (LH - 6);
#pragma unroll
        for (int b = 0; b < 32; b += 2 * hw) {
            if constexpr (LD >= 6) {
                constexpr int dw = 1 << (LD - 6);
                if (!INV) {
#pragma unroll
                    for (int r = 0; r < dw; ++r) w[b + hw + r] ^= w[b + 2 * hw - dw + r];
                }
#pragma unroll
                for (int q = dw; q < hw; ++q) w[b + q] ^= w[b + hw + q - dw];
                if (INV) {
#pragma unroll
                    for (int r = 0; r < dw; ++r) w[b + hw + r] ^= w[b + 2 * hw - dw + r];
                }
            } else {
                constexpr int d = 1 << LD;
                if (!INV) w[b + hw] ^= w[b + 2 * hw - 1] >> (64 - d);
#pragma unroll
                for (int q = hw - 1; q >= 0; --q) {
                    u64 t = w[b + hw + q] << d;
                    if (q > 0) t |= w[b + hw + q - 1] >> (64 - d);
                    w[b + q] ^= t;
                }
                if (INV) w[b + hw] ^= w[b + 2 * hw - 1] >> (64 - d);
            }
        }
    } else {
        // segments of 2P lanes: lane s < P of a segment holds lo words, lane
        // s >= P the hi words at the same offsets
        constexpr int P = 1 << (LH - 11);
        const int s = lane & (2 * P - 1);
        const int base = lane - s;
        const u64 lo_mask = s < P ? ~0ull : 0ull;
        if constexpr (LD < 6) {
            constexpr int d = 1 << LD;
            // the fix: hi[0] ^= hi[hw-1] >> (64 - d), on the first hi lane
            auto fix = [&]() {
                const u64 top = shfl(w[31], base + 2 * P - 1);
                if (s == P) w[0] ^= top >> (64 - d);
            };
            if (!INV) fix();
            // lo[q] ^= (hi[q] << d) | (hi[q-1] >> (64 - d))
            u64 prev = shfl(w[31], lane + P - 1);
            if (s == 0) prev = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const u64 v = shfl(w[j], lane + P);
                w[j] ^= ((v << d) | (prev >> (64 - d))) & lo_mask;
                prev = v;
            }
            if (INV) fix();
        } else {
            constexpr int dw = 1 << (LD - 6);
            if constexpr (dw < 32) {
                // hi[r] ^= hi[hw - dw + r] for r < dw: first hi lane, from the last one
                auto fix = [&]() {
#pragma unroll
                    for (int r = 0; r < dw; ++r) {
                        const u64 t = shfl(w[32 - dw + r], base + 2 * P - 1);
                        if (s == P) w[r] ^= t;
                    }
                };
                if (!INV) fix();
                // lo[q] ^= hi[q - dw]: word j of lo lane s takes word j - dw of
                // hi lane s (or word 32 + j - dw of hi lane s - 1)
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    u64 v;
                    if (j >= dw) {
                        v = shfl(w[j - dw], lane + P);
                    } else {
                        v = shfl(w[32 + j - dw], lane + P - 1);
                        if (s == 0) v = 0;
                    }
                    w[j] ^= v & lo_mask;
                }
                if (INV) fix();
            } else {
                // whole lanes: D = dw/32.  Lo lane s >= D takes hi lane s - D
                // (lane + P - D); hi lane s < P + D is fixed from lane + P - D.
                constexpr int D = dw / 32;
                const u64 fix_mask = (s >= P && s < P + D) ? ~0ull : 0ull;
                const u64 lo_take = (s >= D && s < P) ? ~0ull : 0ull;
                if (!INV) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) w[j] ^= shfl(w[j], lane + P - D) & fix_mask;
#pragma unroll
                    for (int j = 0; j < 32; ++j) w[j] ^= shfl(w[j], lane + P - D) & lo_take;
                } else {
                    // sources of both updates are unfixed hi lanes
#pragma unroll
                    for (int j = 0; j < 32; ++j) w[j] ^= shfl(w[j], lane + P - D) & (fix_mask | lo_take);
                }
            }
        }
    }
}

template <bool INV, int I>
__device__ __forceinline__ void run_steps(u64 (&w)[32], int lane)
{
    if constexpr (I < 32) {
        // forward order, or the reversed list for the inverse
        constexpr int k = INV ? 31 - I : I;
        step<kSteps16.lh[k], kSteps16.ld[k], INV>(w, lane);
        run_steps<INV, I + 1>(w, lane);
    }
}

// One warp per 2^16-bit block; blockIdx.y is the job of a batch.
template <bool INV>
__global__ void __launch_bounds__(32) k_cvt_unit16(u64 *bits, u64 stride)
{
    __shared__ u64 stage[kUnitWords];
    const int lane = threadIdx.x;
    u64 *g = bits + (u64)blockIdx.y * stride + (u64)blockIdx.x * kUnitWords;
    // word 32i + j is kept at 32i + (j ^ i)
#pragma unroll 8
    for (int i = 0; i < 32; ++i) stage[32 * i + (lane ^ i)] = g[32 * i + lane];
    __syncwarp();
    u64 w[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) w[j] = stage[32 * lane + (j ^ lane)];
    run_steps<INV, 0>(w, lane);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j) stage[32 * lane + (j ^ lane)] = w[j];
    __syncwarp();
#pragma unroll 8
    for (int i = 0; i < 32; ++i) g[32 * i + lane] = stage[32 * i + (lane ^ i)];
}

}  // namespace

cudaError_t basis_cvt_unit16(gf2x_ctx *ctx, u64 *bits, u64 L, bool inverse, int count, u64 stride, cudaStream_t st)
{
    const u64 units = L >> 16;
    if (units == 0) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)units, (unsigned)count);
    if (inverse) k_cvt_unit16<true><<<grid, 32, 0, st>>>(bits, stride);
    else k_cvt_unit16<false><<<grid, 32, 0, st>>>(bits, stride);
    count_launch(ctx);
    return cudaGetLastError();
}

}  // namespace gf2x
