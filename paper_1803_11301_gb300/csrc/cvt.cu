// BasisCvt / iBasisCvt (Alg. 1, Sec. 2.3.1) on packed bit arrays.
//
// Flattening of Alg. 1.  For a length L = 2^K, let i be the largest power of
// two with 2^i <= L-1 and tau = 2^i.  Alg. 1 is (1) the Taylor expansion of f
// at s_i = x^tau + x, (2) the same algorithm on the L/tau blocks of tau bits
// ("outer"), (3) the same algorithm inside each block ("inner").  The Taylor
// expansion divides by s_i^(2^k) = x^(tau 2^k) + x^(2^k) for k = K-i-1 .. 0,
// on every aligned segment of 2h = 2 tau 2^k bits.  Writing a segment as
// lo + x^h hi, one division is
//       hi ^= hi >> (h - d)          (only the top d bits move: quotient fix)
//       lo ^= (hi << d) mod x^h      (remainder)
// with d = 2^k.  The outer and inner conversions are the same steps with h and
// d scaled by the unit (tau bits, resp. 1 bit).  So BasisCvt is a fixed list
// of (h, d) steps, each applied to every aligned 2h-bit segment; iBasisCvt is
// the list reversed with each step inverted (lo update first, then the hi fix,
// which is its own inverse).
//
// GPU mapping.  Steps with 2h <= one tile (2^16 bits) run back to back in
// shared memory, one HBM read and write per run of such steps.  Wider steps
// (segments larger than a tile) run as global passes over the array.
#include <vector>

#include "gf2x_common.cuh"

namespace gf2x {
namespace {

constexpr int kTileWordsLog = 10;               // 1024 words = 2^16 bits = 8 KiB
constexpr int kMaxRun = 48;

struct Step {
    u64 h, d;   // bits
};

struct StepRun {
    int count;
    u32 h[kMaxRun];
    u32 d[kMaxRun];
};

void build_steps(int K, u64 unit, std::vector<Step> &out)
{
    if (K <= 1) return;                          // deg f <= 1: identity
    int i = 1;
    while (2 * i <= K - 1) i *= 2;
    u64 tau = 1ull << i;
    for (int k = K - i - 1; k >= 0; --k) out.push_back({tau * (1ull << k) * unit, (1ull << k) * unit});
    build_steps(K - i, unit * tau, out);         // outer: blocks of tau bits
    build_steps(i, unit, out);                   // inner: inside every block
}

__device__ __forceinline__ u64 seg_mask(u32 h, u32 lo_bit, u32 hi_bit)
{
    // bits [lo_bit, hi_bit) of every 2h-bit segment of a 64-bit word
    u64 one = (hi_bit - lo_bit >= 64) ? ~0ull : (((1ull << (hi_bit - lo_bit)) - 1) << lo_bit);
    u64 m = 0;
    for (u32 s = 0; s < 64; s += 2 * h) m |= one << s;
    return m;
}

// hi'(r): word r of the hi half after the quotient fix (forward only).
__device__ __forceinline__ u64 hi_fixed(const u64 *seg, u64 hw, u64 d, u64 r, bool fix)
{
    u64 v = seg[hw + r];
    if (fix) {
        if (d >= 64) {
            u64 dw = d >> 6;
            if (r < dw) v ^= seg[2 * hw - dw + r];
        } else if (r == 0) {
            v ^= seg[2 * hw - 1] >> (64 - d);
        }
    }
    return v;
}

// lo[q] update of one step (word-level, h >= 64 bits): lo ^= (hi' << d) mod x^h.
__device__ __forceinline__ u64 lo_term(const u64 *seg, u64 hw, u64 d, u64 q, bool fix)
{
    if (d >= 64) {
        u64 dw = d >> 6;
        return q >= dw ? hi_fixed(seg, hw, d, q - dw, fix) : 0;
    }
    u64 v = hi_fixed(seg, hw, d, q, fix) << d;
    if (q > 0) v |= hi_fixed(seg, hw, d, q - 1, fix) >> (64 - d);
    return v;
}

__global__ void k_cvt_tile(u64 *bits, int tw_log, StepRun run, int inverse)
{
    extern __shared__ u64 sm[];
    const u64 tw = 1ull << tw_log;
    u64 *g = bits + (u64)blockIdx.x * tw;
    for (u64 w = threadIdx.x; w < tw; w += blockDim.x) sm[w] = g[w];
    __syncthreads();
    for (int s = 0; s < run.count; ++s) {
        const u32 h = run.h[s], d = run.d[s];
        if (h < 64) {                            // segments inside one word
            const u64 ma = seg_mask(h, h, h + d);        // hi bottom d bits
            const u64 mb = seg_mask(h, d, h);            // lo bits [d, h)
            const u32 sh = h - d;
            for (u64 w = threadIdx.x; w < tw; w += blockDim.x) {
                u64 x = sm[w];
                if (!inverse) {
                    x ^= (x >> sh) & ma;
                    x ^= (x >> sh) & mb;
                } else {
                    x ^= (x >> sh) & mb;
                    x ^= (x >> sh) & ma;
                }
                sm[w] = x;
            }
            __syncthreads();
        } else {
            const u64 hw = h >> 6;
            const int hl = __ffsll((long long)hw) - 1;
            for (u64 t = threadIdx.x; t < tw / 2; t += blockDim.x) {
                u64 seg = t >> hl, q = t & (hw - 1);
                u64 *sp = sm + seg * 2 * hw;
                sp[q] ^= lo_term(sp, hw, d, q, !inverse);
            }
            __syncthreads();
            const u64 nfix = d >= 64 ? (d >> 6) : 1;
            const int fl = __ffsll((long long)nfix) - 1;
            const u64 nseg = tw / (2 * hw);
            for (u64 t = threadIdx.x; t < nseg * nfix; t += blockDim.x) {
                u64 seg = t >> fl, r = t & (nfix - 1);
                u64 *sp = sm + seg * 2 * hw;
                if (d >= 64) sp[hw + r] ^= sp[2 * hw - nfix + r];
                else sp[hw] ^= sp[2 * hw - 1] >> (64 - d);
            }
            __syncthreads();
        }
    }
    for (u64 w = threadIdx.x; w < tw; w += blockDim.x) g[w] = sm[w];
}

// One wide step, lo half: every lo word of every segment.
__global__ void k_cvt_lo(u64 *bits, u64 total_lo, u64 hw, u64 d, int inverse)
{
    u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total_lo) return;
    const int hl = __ffsll((long long)hw) - 1;
    u64 seg = t >> hl, q = t & (hw - 1);
    u64 *sp = bits + seg * 2 * hw;
    sp[q] ^= lo_term(sp, hw, d, q, !inverse);
}

// One wide step, the quotient fix of the hi half (runs after k_cvt_lo).
__global__ void k_cvt_fix(u64 *bits, u64 nseg, u64 hw, u64 d)
{
    u64 nfix = d >= 64 ? (d >> 6) : 1;
    u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nseg * nfix) return;
    const int fl = __ffsll((long long)nfix) - 1;
    u64 seg = t >> fl, r = t & (nfix - 1);
    u64 *sp = bits + seg * 2 * hw;
    if (d >= 64) sp[hw + r] ^= sp[2 * hw - nfix + r];
    else sp[hw] ^= sp[2 * hw - 1] >> (64 - d);
}

inline unsigned blocks_for(u64 n, unsigned threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t basis_cvt(gf2x_ctx *ctx, u64 *bits, u64 L, bool inverse, cudaStream_t st)
{
    int K = 0;
    while ((1ull << K) < L) ++K;
    std::vector<Step> steps;
    build_steps(K, 1, steps);
    if (inverse) std::vector<Step>(steps.rbegin(), steps.rend()).swap(steps);

    const u64 words = L >> 6;
    int tw_log = 0;
    while ((1ull << tw_log) < words && tw_log < kTileWordsLog) ++tw_log;
    const u64 tile_bits = 64ull << tw_log;
    const unsigned tile_threads = 256;

    StepRun run;
    run.count = 0;
    auto flush = [&]() {
        if (!run.count) return;
        unsigned nblk = (unsigned)(words >> tw_log);
        k_cvt_tile<<<nblk, tile_threads, (size_t)(8ull << tw_log), st>>>(bits, tw_log, run, inverse ? 1 : 0);
        count_launch(ctx);
        run.count = 0;
    };
    for (const Step &s : steps) {
        if (2 * s.h <= tile_bits) {
            if (run.count == kMaxRun) flush();
            run.h[run.count] = (u32)s.h;
            run.d[run.count] = (u32)s.d;
            ++run.count;
            continue;
        }
        flush();
        const u64 hw = s.h >> 6;
        const u64 total_lo = words / 2;
        const u64 nseg = words / (2 * hw);
        const u64 nfix = s.d >= 64 ? (s.d >> 6) : 1;
        k_cvt_lo<<<blocks_for(total_lo, 256), 256, 0, st>>>(bits, total_lo, hw, s.d, inverse ? 1 : 0);
        k_cvt_fix<<<blocks_for(nseg * nfix, 256), 256, 0, st>>>(bits, nseg, hw, s.d);
        count_launch(ctx, 2);
    }
    flush();
    return cudaGetLastError();
}

}  // namespace gf2x
