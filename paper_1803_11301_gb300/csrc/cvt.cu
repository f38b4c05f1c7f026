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
// the list reversed with each step inverted (lo update with the current hi,
// then the hi fix, which is its own inverse).
//
// GPU mapping: one kernel per phase (kernel boundaries order the phases; in a
// CUDA graph a boundary costs about 0.5 us, less than a software grid barrier,
// measured at 1.7-2.7 us on GB300).
//
// For 17 <= K <= 32 the split is at tau = 2^16 and the phases follow the
// structure of Alg. 1 (basis_cvt_structured): the low Taylor layers in one
// window kernel (below), the others as wide steps, the outer conversion
// on whole 2^16-bit blocks and the inner conversion of every block in the
// register kernels of cvt_reg.cu.  Other lengths, and the parts of that path
// that are plain lists of steps, go through the generic planner:
//  * a run of consecutive steps with 2h <= one tile (2^18 bits) is one kernel:
//    each block loads a tile into shared memory, applies the whole run, and
//    writes it back (one HBM/L2 read and write per run);
//  * a run of steps that all move whole units of U >= 256 bits is one column
//    kernel (each word column of the units is independent);
//  * a wider step is one kernel, in place: each lo word is owned by one
//    thread, which also writes the quotient fix of the one hi word whose only
//    reader it is (for d < 64 bits a thread owns four lo words, so hi[0],
//    read by the owners of lo[0] and lo[1], has a single owner).
//
// The bounded grid barrier below is used by the wait self-test: a wait that
// runs out records GF2X_ETIMEOUT in the context status word and returns.
#include <vector>

#include "cvt_dev.cuh"

namespace gf2x {
namespace {
using namespace cvtk;

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

// ------------------------------------------------------------- grid barrier
// Arrive-and-wait on the barrier in `gs` for `nblocks` blocks.  Returns false
// (on every thread of the block) when the wait ran out or another block gave
// up; the block must then return.
__device__ bool grid_sync(GridSync *gs, unsigned nblocks, int *status, unsigned long long limit)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = &gs->gen;
        volatile unsigned *vabort = &gs->abort;
        const unsigned my = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&gs->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&gs->count, 0u);
            __threadfence();
            atomicAdd(&gs->gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (*vgen == my) {
                if (*vabort) { ok = 0; break; }
                if (++spins > limit) {
                    atomicExch(&gs->abort, 1u);
                    atomicCAS(status, (int)GF2X_OK, (int)GF2X_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}


__global__ void __launch_bounds__(256) k_cvt_wide(u64 *bits, const u64 *src, u64 words, u64 h, u64 d, int inverse,
                                                  u64 stride)
{
    cvt_wide_body(launch_block(), bits, src, words, h, d, inverse, stride);
}

__global__ void __launch_bounds__(kThreads) k_cvt_tile(u64 *bits, const u64 *src, CvtPlan P, int phase, u64 stride)
{
    extern __shared__ u64 sm[];
    cvt_tile_body(launch_block(), sm, bits, src, P, phase, stride);
}

__global__ void __launch_bounds__(kThreads) k_cvt_col(u64 *bits, const u64 *src, CvtPlan P, int phase, u64 stride)
{
    extern __shared__ u64 sm[];
    cvt_col_body(launch_block(), sm, bits, src, P, phase, stride);
}

__global__ void __launch_bounds__(kTaylorThreads) k_cvt_taylor(u64 *bits, const u64 *src, int mw, int W, int inverse,
                                                                u64 stride)
{
    extern __shared__ u64 win[];
    cvt_taylor_body(launch_block(), win, bits, src, mw, W, inverse, stride);
}

// Bounded-wait self-test: one block waits for a second arrival that never
// comes, so the wait runs out and records GF2X_ETIMEOUT.
__global__ void k_wait_timeout_probe(GridSync *gs, int *status, unsigned long long limit)
{
    grid_sync(gs, gridDim.x + 1, status, limit);
}

bool g_configured = false;

void configure_kernels()
{
    if (g_configured) return;
    cudaFuncSetAttribute(k_cvt_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((size_t)8 << kTileWordsLog));
    cudaFuncSetAttribute(k_cvt_col, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((size_t)8 << kTileWordsLog));
    cudaFuncSetAttribute(k_cvt_taylor, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    g_configured = true;
}

// Any list of steps (in execution order) on an L-bit array: runs of in-tile
// steps, column runs and single wide steps, one kernel each.
// The first phase reads `src` (which may differ from `bits`, each job's buffer
// `stride` words apart in both), every phase writes `bits`.
cudaError_t run_steps_generic(gf2x_ctx *ctx, u64 *bits, const u64 *src, u64 L, const std::vector<Step> &steps,
                              bool inverse, int count, u64 stride, cudaStream_t st)
{
    if (steps.empty()) return src == bits ? cudaSuccess : cudaErrorInvalidValue;
    configure_kernels();
    CvtPlan P;
    P.inverse = inverse ? 1 : 0;
    P.words = L >> 6;
    int tw_log = 0;
    while ((1ull << tw_log) < P.words && tw_log < kTileWordsLog) ++tw_log;
    P.tw_log = tw_log;
    const u64 tile_bits = 64ull << tw_log;
    const u64 tile_words = 1ull << kTileWordsLog;
    // a column run with unit U and longest half H fits when each block can hold
    // 4 words of 2H/U units (U >= 256 bits)
    auto fits = [&](u64 U, u64 H) { return U >= 256 && 2 * H / U <= tile_words / 4 && 2 * H / U <= L / U; };
    P.nphase = 0;
    const size_t n = steps.size();
    for (size_t k = 0; k < n; ++k) { P.h[k] = steps[k].h; P.d[k] = steps[k].d; }
    for (size_t k = 0; k < n;) {
        const int ph = P.nphase++;
        P.first[ph] = (unsigned char)k;
        if (2 * steps[k].h <= tile_bits) {              // run of in-tile steps
            size_t j = k;
            while (j < n && 2 * steps[j].h <= tile_bits && j - k < 255) ++j;
            P.kind[ph] = PHASE_TILE;
            P.count[ph] = (unsigned char)(j - k);
            k = j;
            continue;
        }
        u64 U = steps[k].d, H = steps[k].h;
        size_t j = k + 1;
        while (j < n) {
            const u64 U2 = steps[j].d < U ? steps[j].d : U, H2 = steps[j].h > H ? steps[j].h : H;
            if (!fits(U2, H2)) break;
            U = U2; H = H2; ++j;
        }
        if (j - k >= 2 && fits(U, H)) {                 // column run
            int ulog = 0, slog = 0;
            while ((1ull << ulog) < U) ++ulog;
            while ((1ull << slog) < 2 * H / U) ++slog;
            int wlog = 2;                               // widest rows that still fit
            while (wlog < 4 && (1ull << (wlog + 1)) <= (U >> 6) && ((2 * H / U) << (wlog + 1)) <= tile_words) ++wlog;
            // as many units per block as fit (>= the run's segments)
            while ((1ull << (slog + 1)) <= L / U && (1ull << (slog + 1 + wlog)) <= tile_words) ++slog;
            P.kind[ph] = PHASE_COLUMN;
            P.ulog[ph] = (unsigned char)ulog;
            P.wlog[ph] = (unsigned char)wlog;
            P.slog[ph] = (unsigned char)slog;
            P.count[ph] = (unsigned char)(j - k);
            k = j;
        } else {                                        // one wide step
            P.kind[ph] = PHASE_WIDE;
            P.count[ph] = 1;
            ++k;
        }
    }
    const u64 ntiles = P.words >> tw_log;
    const u64 wide_threads = P.words / 8;         // four lo words per thread
    if (recording(ctx)) {
        const int blob = record_blob(ctx, &P, sizeof P);
        if (blob < 0) return cudaErrorInvalidValue;
        for (int ph = 0; ph < P.nphase; ++ph) {
            const u64 *in = ph == 0 ? src : bits;
            SegRec r{};
            r.gy = (unsigned)count;
            r.blob = blob;
            r.a[0] = (u64)bits;
            r.a[1] = (u64)in;
            r.a[2] = stride;
            r.i[0] = ph;
            if (P.kind[ph] == PHASE_WIDE) {
                const int s0 = P.first[ph];
                r.kind = SEG_CVT_WIDE;
                r.gx = (unsigned)((wide_threads + 255) / 256);
                r.threads = 256;
                r.a[3] = P.words;
                r.a[4] = P.h[s0];
                r.a[5] = P.d[s0];
                r.i[1] = P.inverse;
            } else if (P.kind[ph] == PHASE_TILE) {     // the bodies loop over any thread count
                r.kind = SEG_CVT_TILE;
                r.gx = (unsigned)ntiles;
                r.threads = kPersistThreads;
                r.smem = 8u << tw_log;
            } else {
                r.kind = SEG_CVT_COL;
                r.gx = (unsigned)((P.words >> (P.ulog[ph] - 6 + P.slog[ph])) * ((1ull << (P.ulog[ph] - 6)) >> P.wlog[ph]));
                r.threads = kPersistThreads;
                r.smem = 8u << (P.slog[ph] + P.wlog[ph]);
            }
            r.per_job = r.gx;
            if (!record(ctx, r)) return cudaErrorInvalidValue;
        }
        return cudaSuccess;
    }
    for (int ph = 0; ph < P.nphase; ++ph) {
        const u64 *in = ph == 0 ? src : bits;
        if (P.kind[ph] == PHASE_WIDE) {
            const int s0 = P.first[ph];
            k_cvt_wide<<<dim3((unsigned)((wide_threads + 255) / 256), count), 256, 0, st>>>(
                bits, in, P.words, P.h[s0], P.d[s0], P.inverse, stride);
        } else if (P.kind[ph] == PHASE_TILE) {
            k_cvt_tile<<<dim3((unsigned)ntiles, count), kThreads, (size_t)8 << tw_log, st>>>(bits, in, P, ph, stride);
        } else {
            const u64 blocks = (P.words >> (P.ulog[ph] - 6 + P.slog[ph] - 0)) * ((1ull << (P.ulog[ph] - 6)) >> P.wlog[ph]);
            k_cvt_col<<<dim3((unsigned)blocks, count), kThreads, (size_t)8 << (P.slog[ph] + P.wlog[ph]), st>>>(
                bits, in, P, ph, stride);
        }
        count_launch(ctx);
    }
    return cudaGetLastError();
}

#define TRY_CUDA(x)                                  \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return e_;            \
    } while (0)

// Taylor window kernel over every group of 2^mw blocks: src -> bits (distinct).
cudaError_t taylor_window_launch(gf2x_ctx *ctx, u64 *bits, const u64 *src, u64 L, int mw, bool inverse, int count,
                                 u64 stride, cudaStream_t st)
{
    configure_kernels();
    const u64 groups = (L >> 16) >> mw;
    const int halo = taylor_halo(mw);
    // widest window that fits in shared memory, narrowed (down to 8 columns)
    // while there are fewer than two blocks per SM
    auto bytes = [&](int w) { return (size_t)((1 << mw) + 1) * (w + halo) * 8; };
    const size_t cap = recording(ctx) ? kPersistSmem : 180 * 1024;   // a block of the persistent kernel holds less
    int W = 32;
    while (W > 8 && bytes(W) > cap) W >>= 1;
    while (W > 8 && ((1u << kUnitWordsLog) / W) * groups * (u64)count < 2 * (u64)ctx->num_sms) W >>= 1;
    const size_t smem = bytes(W);
    const dim3 grid((unsigned)(((1u << kUnitWordsLog) / W) * groups), (unsigned)count);
    if (recording(ctx)) {
        SegRec r{SEG_CVT_TAYLOR, {mw, W, inverse ? 1 : 0, 0}, grid.x, grid.y, kPersistThreads, (unsigned)smem, grid.x, -1,
                 {(u64)bits, (u64)src, stride}};
        return record(ctx, r) ? cudaSuccess : cudaErrorInvalidValue;
    }
    k_cvt_taylor<<<grid, kTaylorThreads, smem, st>>>(bits, src, mw, W, inverse ? 1 : 0, stride);
    count_launch(ctx);
    return cudaGetLastError();
}

// 18 <= K <= 32: Alg. 1 splits at tau = 2^16 with m = K - 16 >= 2:
//   (a) Taylor expansion, steps (2^(16+k), 2^k) for k = m-1 .. 0: the low
//       layers (up to 8) in the window kernel, the rest as wide steps;
//   (b) outer BasisCvt(2^m) on blocks of 2^16 bits (1024 words): the
//       register kernel for m <= 9; for m >= 10 its own split at 2^8 blocks:
//       Taylor steps (2^(24+k), 2^(16+k)), k = m-9 .. 0 (generic planner),
//       outer BasisCvt(2^(m-8)) on units of 2^24 bits, inner BasisCvt(2^8) on
//       every group of 256 blocks;
//   (c) BasisCvt(2^16) inside every block (register kernel).
// The inverse runs the same parts in the reverse order, each inverted.  The
// window kernel runs out of place through `scratch` (a buffer laid out like
// `bits`), and the part next to it moves the data back: forward, window
// bits -> scratch and (b) scratch -> bits; inverse, (b) bits -> scratch and
// the window scratch -> bits.
//
// With a side buffer and m >= 9 (where (a) needs wide steps), (a) is instead
// the two superset-sum passes of cvt_zeta.cu (bits -> scratch and side ->
// bits), (b) runs in place on bits, and for m >= 10 the Taylor steps of (b)
// are the row-level superset sum and carry passes of cvt_zeta.cu.
// Whether the structured path takes the two-pass Taylor part for 2^(m+16) bits.
bool two_pass_taylor(gf2x_ctx *ctx, int m, bool has_side, u64 side_words)
{
    const u64 need = taylor_zeta_side_words(m);
    static const int cands[2] = {0, 1};
    return has_side && need && need <= side_words && !recording(ctx) &&
           tune_pinned(ctx, TUNE_CVT_TAYLOR, cands, 2, 1) == 1;
}

cudaError_t basis_cvt_structured(gf2x_ctx *ctx, u64 *bits, u64 *scratch, u64 L, int K, bool inverse, int count,
                                 u64 stride, cudaStream_t st, u64 *side = nullptr, u64 side_stride = 0,
                                 u64 side_words = 0, const ZetaIO *io = nullptr)
{
    const int m = K - 16;
    if (two_pass_taylor(ctx, m, side != nullptr, side_words)) {
        {
            if (!inverse) {
                TRY_CUDA(taylor_zeta(ctx, bits, scratch, side, side_stride, m, false, count, stride, st, io));
                if (m <= 9) {
                    TRY_CUDA(basis_cvt_outer(ctx, bits, bits, L, m, kUnitWordsLog, false, count, stride, st));
                } else {
                    TRY_CUDA(outer_taylor_zeta(ctx, bits, side, side_stride, m, false, count, stride, st));
                    TRY_CUDA(basis_cvt_outer(ctx, bits, bits, L, m - 8, kUnitWordsLog + 8, false, count, stride, st));
                    TRY_CUDA(basis_cvt_outer(ctx, bits, bits, L, 8, kUnitWordsLog, false, count, stride, st));
                }
                return basis_cvt_unit16(ctx, bits, L, false, count, stride, scratch, st);
            }
            TRY_CUDA(basis_cvt_unit16(ctx, bits, L, true, count, stride, scratch, st));
            if (m <= 9) {
                TRY_CUDA(basis_cvt_outer(ctx, bits, bits, L, m, kUnitWordsLog, true, count, stride, st));
            } else {
                TRY_CUDA(basis_cvt_outer(ctx, bits, bits, L, 8, kUnitWordsLog, true, count, stride, st));
                TRY_CUDA(basis_cvt_outer(ctx, bits, bits, L, m - 8, kUnitWordsLog + 8, true, count, stride, st));
                TRY_CUDA(outer_taylor_zeta(ctx, bits, side, side_stride, m, true, count, stride, st));
            }
            return taylor_zeta(ctx, bits, scratch, side, side_stride, m, true, count, stride, st, io);
        }
    }
    if (io && (io->src[0] || io->dst)) return cudaErrorInvalidValue;   // only the two-pass part reads or writes in place
    // Layers in the window kernel (at most 8; the rest are wide steps): its
    // cost grows faster than linearly with the depth (the halo and the rows
    // per block double with each layer), so deep windows pay most while the
    // array sits in L2.  The tuner compares depths 6, 7 and 8 on the layers
    // below 8 (window from bits into scratch, then the remaining wide steps
    // in place on scratch); the default found on GB300 is 8 for K <= 25 and 7
    // above.
    int cap = K <= 25 ? 8 : 7;
    if (m > 6) {
        static const int cands[3] = {6, 7, 8};
        const int top = m < 8 ? m : 8;
        cap = tune_choice(ctx, TUNE_WINDOW_DEPTH, ((u64)K << 33) | (tune_bucket((u64)count) << 1) | (inverse ? 1u : 0u), cands,
                          top - 5, cap, [&](int c) -> cudaError_t {
                              std::vector<Step> w;
                              for (int k = top - 1; k >= c; --k) w.push_back({1ull << (16 + k), 1ull << k});
                              TRY_CUDA(taylor_window_launch(ctx, scratch, bits, L, c, inverse, count, stride, st));
                              return run_steps_generic(ctx, scratch, scratch, L, w, inverse, count, stride, st);
                          }, st);
    }
    const int mw = m < cap ? m : cap;
    std::vector<Step> taylor_wide, outer_taylor;
    for (int k = m - 1; k >= mw; --k) taylor_wide.push_back({1ull << (16 + k), 1ull << k});
    if (m >= 10)
        for (int k = m - 9; k >= 0; --k) outer_taylor.push_back({1ull << (24 + k), 1ull << (16 + k)});
    const std::vector<Step> taylor_wide_inv(taylor_wide.rbegin(), taylor_wide.rend());
    const std::vector<Step> outer_taylor_inv(outer_taylor.rbegin(), outer_taylor.rend());
    if (!inverse) {
        TRY_CUDA(run_steps_generic(ctx, bits, bits, L, taylor_wide, false, count, stride, st));
        TRY_CUDA(taylor_window_launch(ctx, scratch, bits, L, mw, false, count, stride, st));
        if (m <= 9) {
            TRY_CUDA(basis_cvt_outer(ctx, bits, scratch, L, m, kUnitWordsLog, false, count, stride, st));
        } else {
            TRY_CUDA(run_steps_generic(ctx, bits, scratch, L, outer_taylor, false, count, stride, st));
            TRY_CUDA(basis_cvt_outer(ctx, bits, bits, L, m - 8, kUnitWordsLog + 8, false, count, stride, st));
            TRY_CUDA(basis_cvt_outer(ctx, bits, bits, L, 8, kUnitWordsLog, false, count, stride, st));
        }
        return basis_cvt_unit16(ctx, bits, L, false, count, stride, scratch, st);
    }
    TRY_CUDA(basis_cvt_unit16(ctx, bits, L, true, count, stride, scratch, st));
    if (m <= 9) {
        TRY_CUDA(basis_cvt_outer(ctx, scratch, bits, L, m, kUnitWordsLog, true, count, stride, st));
    } else {
        TRY_CUDA(basis_cvt_outer(ctx, bits, bits, L, 8, kUnitWordsLog, true, count, stride, st));
        TRY_CUDA(basis_cvt_outer(ctx, bits, bits, L, m - 8, kUnitWordsLog + 8, true, count, stride, st));
        TRY_CUDA(run_steps_generic(ctx, scratch, bits, L, outer_taylor_inv, true, count, stride, st));
    }
    TRY_CUDA(taylor_window_launch(ctx, bits, scratch, L, mw, true, count, stride, st));
    return run_steps_generic(ctx, bits, bits, L, taylor_wide_inv, true, count, stride, st);
}

}  // namespace

bool basis_cvt_two_pass(gf2x_ctx *ctx, u64 L, u64 side_words)
{
    int K = 0;
    while ((1ull << K) < L) ++K;
    return K >= 18 && K <= 32 && two_pass_taylor(ctx, K - 16, true, side_words);
}

cudaError_t basis_cvt(gf2x_ctx *ctx, u64 *bits, u64 L, bool inverse, int count, u64 stride, u64 *scratch,
                      cudaStream_t st, u64 *side, u64 side_stride, u64 side_words, const ZetaIO *io)
{
    int K = 0;
    while ((1ull << K) < L) ++K;
    if (scratch && K >= 18 && K <= 32)
        return basis_cvt_structured(ctx, bits, scratch, L, K, inverse, count, stride, st, side, side_stride, side_words,
                                    io);
    if (io && (io->src[0] || io->dst)) return cudaErrorInvalidValue;
    std::vector<Step> steps;
    build_steps(K, 1, steps);
    if (scratch && K > 32) {
        // Alg. 1 with i = 32 (tau = 2^32): its K - 32 Taylor layers and the outer
        // conversion of the 2^(K-32) units of 2^32 bits are the generic steps
        // before the last |build_steps(32)| ones; those are the inner conversion
        // of every unit, run by the structured K = 32 path (outer and inner commute).
        std::vector<Step> inner;
        build_steps(32, 1, inner);
        steps.resize(steps.size() - inner.size());
        const u64 unit_words = 1ull << 26, units = L >> 32;
        auto inner_all = [&]() -> cudaError_t {
            if (count == 1 || stride == units * unit_words)
                return basis_cvt_structured(ctx, bits, scratch, 1ull << 32, 32, inverse, (int)(units * (u64)count),
                                            unit_words, st);
            for (int j = 0; j < count; ++j)
                TRY_CUDA(basis_cvt_structured(ctx, bits + (u64)j * stride, scratch + (u64)j * stride, 1ull << 32, 32,
                                              inverse, (int)units, unit_words, st));
            return cudaSuccess;
        };
        if (inverse) {
            TRY_CUDA(inner_all());
            return run_steps_generic(ctx, bits, bits, L, std::vector<Step>(steps.rbegin(), steps.rend()), true, count,
                                     stride, st);
        }
        TRY_CUDA(run_steps_generic(ctx, bits, bits, L, steps, false, count, stride, st));
        return inner_all();
    }
    if (steps.empty()) return cudaSuccess;
    // For K >= 16 the list ends with the 32 steps of BasisCvt inside every
    // 2^16-bit block, run by the register kernel (first for the inverse, last
    // for the forward transform).
    const bool unit16 = K >= 16;
    if (unit16) steps.resize(steps.size() - 32);
    if (inverse) {
        if (unit16) TRY_CUDA(basis_cvt_unit16(ctx, bits, L, true, count, stride, scratch, st));
        return run_steps_generic(ctx, bits, bits, L, std::vector<Step>(steps.rbegin(), steps.rend()), true, count,
                                 stride, st);
    }
    TRY_CUDA(run_steps_generic(ctx, bits, bits, L, steps, false, count, stride, st));
    return unit16 ? basis_cvt_unit16(ctx, bits, L, false, count, stride, scratch, st) : cudaSuccess;
}

cudaError_t wait_timeout_probe(gf2x_ctx *ctx, GridSync *gs, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(gs, 0, sizeof(GridSync), st);
    if (e != cudaSuccess) return e;
    k_wait_timeout_probe<<<1, 32, 0, st>>>(gs, ctx->d_status, 1ull << 14);
    count_launch(ctx);
    return cudaGetLastError();
}

GF2X_OUT_OF_RANGE_READER(out_of_range_cvt)

}  // namespace gf2x
