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

#include "gf2x_common.cuh"

namespace gf2x {
namespace {

constexpr int kTileWordsLog = 12;               // 4096 words = 2^18 bits = 32 KiB
constexpr int kMaxSteps = 96;                   // K <= 37 gives at most 90 steps
constexpr int kThreads = 512;

struct Step {
    u64 h, d;   // bits
};

enum PhaseKind { PHASE_TILE = 0, PHASE_WIDE = 1, PHASE_COLUMN = 2 };

struct CvtPlan {
    int nphase;
    int inverse;
    int tw_log;                     // tile = 2^tw_log words
    u64 words;                      // L / 64
    unsigned char kind[kMaxSteps];  // PhaseKind of phase p
    unsigned char first[kMaxSteps], count[kMaxSteps];
    unsigned char ulog[kMaxSteps];  // column phase: unit of 2^ulog bits
    unsigned char wlog[kMaxSteps];  // column phase: 2^wlog words per unit per block
    unsigned char slog[kMaxSteps];  // column phase: 2^slog units per block
    u64 h[kMaxSteps], d[kMaxSteps];
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

// Asynchronous global -> shared copies (cp.async, 8 bytes: the arrays are only
// required to be 8-byte aligned): a thread issues all of its loads of a tile
// before waiting, instead of one dependent load at a time.
__device__ __forceinline__ void copy_async8(void *dst_shared, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst_shared)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void copy_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ u64 seg_mask(u32 h, u32 lo_bit, u32 hi_bit)
{
    // bits [lo_bit, hi_bit) of every 2h-bit segment of a 64-bit word (h < 64)
    u64 one = ((1ull << (hi_bit - lo_bit)) - 1) << lo_bit;
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

// A run of steps (all with 2h <= tile) on a tile in shared memory.
__device__ void tile_run(u64 *sm, u64 tw, const CvtPlan &P, int first, int count)
{
    const bool inverse = P.inverse != 0;
    for (int s = first; s < first + count; ++s) {
        const u64 h = P.h[s], d = P.d[s];
        if (h < 64) {                            // segments inside one word
            const u64 ma = seg_mask((u32)h, (u32)h, (u32)(h + d));   // hi bottom d bits
            const u64 mb = seg_mask((u32)h, (u32)d, (u32)h);         // lo bits [d, h)
            const u32 sh = (u32)(h - d);
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
}

// One wide step in place (segments larger than a tile, so h >= 2^18 bits, hw >= 4096 words).
// Each thread owns four consecutive lo words.
// Out of place (src != bits): every word is read from src and the thread
// writes lo[q] and hi[q] of its four indices q to bits (the fix of hi[q] is
// computed from src by its own thread).
__global__ void __launch_bounds__(256) k_cvt_wide(u64 *bits, const u64 *src, u64 words, u64 h, u64 d, int inverse,
                                                  u64 stride)
{
    bits += (u64)blockIdx.y * stride;             // job of a batch
    src += (u64)blockIdx.y * stride;
    const u64 hw = h >> 6;
    const int hl = __ffsll((long long)hw) - 1;
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * t >= words / 2) return;
    const u64 w = 4 * t;                          // index among all lo words
    const u64 seg = w >> hl, q0 = w & (hw - 1);
    if (src != bits) {
        const u64 *sp = src + seg * 2 * hw;
        u64 *op = bits + seg * 2 * hw;
        if (d >= 64) {
            const u64 dw = d >> 6;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const u64 q = q0 + k;
                const u64 hq = sp[hw + q];
                op[hw + q] = q < dw ? hq ^ sp[2 * hw - dw + q] : hq;
                u64 term = 0;
                if (q >= dw) {
                    const u64 r = q - dw;
                    term = sp[hw + r];
                    if (!inverse && r < dw) term ^= sp[2 * hw - dw + r];
                }
                op[q] = sp[q] ^ term;
            }
        } else {
            const u64 top = sp[2 * hw - 1] >> (64 - d);
            u64 hv[5];
            hv[0] = q0 > 0 ? sp[hw + q0 - 1] : 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) hv[k + 1] = sp[hw + q0 + k];
            op[hw + q0] = q0 == 0 ? hv[1] ^ top : hv[1];
#pragma unroll
            for (int k = 1; k < 4; ++k) op[hw + q0 + k] = hv[k + 1];
            if (q0 == 0 && !inverse) hv[1] ^= top;
#pragma unroll
            for (int k = 0; k < 4; ++k) op[q0 + k] = sp[q0 + k] ^ ((hv[k + 1] << d) | (hv[k] >> (64 - d)));
        }
        return;
    }
    u64 *sp = bits + seg * 2 * hw;
    u64 lo[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) lo[k] = sp[q0 + k];
    if (d >= 64) {
        // lo[q] ^= hi'[q - dw]; the owner of lo[q] is the only reader of
        // hi[q - dw] and writes its fix hi[r] ^= hi[2hw - dw + r] (r < dw)
        const u64 dw = d >> 6;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const u64 q = q0 + k;
            if (q < dw) continue;
            const u64 r = q - dw;
            const u64 hv = sp[hw + r];
            u64 term = hv;
            if (r < dw) {
                const u64 top = sp[2 * hw - dw + r];
                if (!inverse) term ^= top;       // the forward step uses the fixed hi
                sp[hw + r] = hv ^ top;           // the fix is its own inverse
            }
            lo[k] ^= term;
        }
    } else {
        // lo[q] ^= (hi'[q] << d) | (hi'[q-1] >> (64-d)); only hi[0] is fixed
        u64 hv[5];
        hv[0] = q0 > 0 ? sp[hw + q0 - 1] : 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) hv[k + 1] = sp[hw + q0 + k];
        if (q0 == 0) {
            const u64 top = sp[2 * hw - 1] >> (64 - d);
            sp[hw] = hv[1] ^ top;
            if (!inverse) hv[1] ^= top;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) lo[k] ^= (hv[k + 1] << d) | (hv[k] >> (64 - d));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) sp[q0 + k] = lo[k];
}

// A run of tile steps: one block per tile of 2^tw_log words.
__global__ void __launch_bounds__(kThreads) k_cvt_tile(u64 *bits, const u64 *src, CvtPlan P, int phase, u64 stride)
{
    extern __shared__ u64 sm[];
    bits += (u64)blockIdx.y * stride;
    src += (u64)blockIdx.y * stride;
    const u64 tw = 1ull << P.tw_log;
    u64 *g = bits + (u64)blockIdx.x * tw;
    const u64 *gs = src + (u64)blockIdx.x * tw;
    for (u64 w = threadIdx.x; w < tw; w += blockDim.x) copy_async8(sm + w, gs + w);
    copy_async_wait();
    __syncthreads();
    tile_run(sm, tw, P, P.first[phase], P.count[phase]);
    for (u64 w = threadIdx.x; w < tw; w += blockDim.x) g[w] = sm[w];
}

// A run of steps whose d are all multiples of a unit U (>= 4 words): every step
// moves whole units, so the same step applies to each word column of the units
// independently.  A block holds 2^wlog word columns of 2^slog consecutive
// units (a segment-aligned range at least as long as the run's segments).
__global__ void __launch_bounds__(kThreads) k_cvt_col(u64 *bits, const u64 *src, CvtPlan P, int phase, u64 stride)
{
    extern __shared__ u64 sm[];
    bits += (u64)blockIdx.y * stride;
    src += (u64)blockIdx.y * stride;
    const int ulog = P.ulog[phase], wlog = P.wlog[phase], slog = P.slog[phase];
    const u64 uw = 1ull << (ulog - 6);                  // words per unit
    const u64 W = 1ull << wlog, S = 1ull << slog;
    const u64 cols = uw >> wlog;                        // column blocks per unit
    const u64 u0 = ((u64)blockIdx.x / cols) << slog, c0 = ((u64)blockIdx.x % cols) << wlog;
    for (u64 k = threadIdx.x; k < S * W; k += blockDim.x)
        copy_async8(sm + k, src + (u0 + (k >> wlog)) * uw + c0 + (k & (W - 1)));
    copy_async_wait();
    __syncthreads();
    const bool inverse = P.inverse != 0;
    for (int s = P.first[phase]; s < P.first[phase] + P.count[phase]; ++s) {
        const u64 H = P.h[s] >> ulog, D = P.d[s] >> ulog;      // in units
        const int hl = __ffsll((long long)H) - 1;
        // lo[q] ^= hi'[q - D], hi' = hi with the quotient fix (forward)
        for (u64 k = threadIdx.x; k < (S / 2) * W; k += blockDim.x) {
            const u64 e = k >> wlog, w = k & (W - 1);
            const u64 base = (e >> hl) << (hl + 1), q = e & (H - 1);
            if (q < D) continue;
            const u64 r = q - D;
            u64 hv = sm[((base + H + r) << wlog) + w];
            if (!inverse && r < D) hv ^= sm[((base + 2 * H - D + r) << wlog) + w];
            sm[((base + q) << wlog) + w] ^= hv;
        }
        __syncthreads();
        // hi[r] ^= hi[H - D + r], r < D
        const int dl = __ffsll((long long)D) - 1;
        for (u64 k = threadIdx.x; k < (S >> (hl + 1)) * D * W; k += blockDim.x) {
            const u64 w = k & (W - 1), rest = k >> wlog;
            const u64 r = rest & (D - 1), seg = rest >> dl;
            const u64 base = seg << (hl + 1);
            sm[((base + H + r) << wlog) + w] ^= sm[((base + 2 * H - D + r) << wlog) + w];
        }
        __syncthreads();
    }
    for (u64 k = threadIdx.x; k < S * W; k += blockDim.x)
        bits[(u0 + (k >> wlog)) * uw + c0 + (k & (W - 1))] = sm[k];
}

// ------------------------------------------------------ Taylor window kernel
// Layers k = mw-1 .. 0 (forward) of the Taylor expansion at x^tau + x with
// tau = 2^16: step (h, d) = (tau 2^k, 2^k) bits on every group of 2^mw blocks
// of 2^16 bits (1024 words each).  Seen as a table of blocks (rows u) by word
// columns c, every dependency of a step goes from a column to columns on its
// left, cyclically: lo[p] reads hi'[p - dw] (or hi'[p], hi'[p-1] for d < 64
// bits), and the quotient fix brings the top dw words of the hi half to its
// bottom.  A block of threads holds, for every row of the group, a window of W
// output columns plus `halo` columns to their left (wrapping around to the top
// of the row), runs all mw layers on it in shared memory, and writes back the
// W output columns, which are then exact (taylor_halo).  The
// halo columns of one block are output columns of its neighbour, so the
// kernel runs out of place (src != bits): no block reads what another writes.
constexpr int kUnitWordsLog = 10;               // 2^16 bits
constexpr int kTaylorThreads = 512;

// Columns of halo for mw layers: the layers together shift by less than 2^mw
// bits (the Taylor expansion at x^tau + x of a 2^mw-block group, written as
// sums of x^(q-r) f_q, reaches q - r < 2^mw bits to the left, cyclically), so
// ceil(2^mw / 64) + 1 words, rounded up to even (the kernel works on column
// pairs).  Checked exact, against the step list, for every window position,
// window widths 8, 16 and 32, and the depths in use (mw <= 8).
__host__ __device__ constexpr int taylor_halo(int mw)
{
    const int h = ((1 << mw) + 63) / 64 + 1;
    return (h + 1) & ~1;
}

__global__ void __launch_bounds__(kTaylorThreads) k_cvt_taylor(u64 *bits, const u64 *src, int mw, int W, int inverse,
                                                                u64 stride)
{
    // window storage, column-major: win[j * (G + 1) + u] (row u, window column
    // j).  The odd column stride keeps both the load (consecutive columns of
    // one row) and the steps (consecutive rows of one column) conflict-free.
    extern __shared__ u64 win[];
    const int halo = taylor_halo(mw);
    const int WW = W + halo, G = 1 << mw, CS = G + 1;
    const int nwin = (1 << kUnitWordsLog) / W;
    const int c0 = (int)(blockIdx.x % nwin) * W;
    const int cw0 = c0 - halo;                  // true column of window column 0 (mod 1024)
    const int cmask = (1 << kUnitWordsLog) - 1;
    const u64 goff = (u64)blockIdx.y * stride + ((u64)(blockIdx.x / nwin) << (mw + kUnitWordsLog));
    u64 *g = bits + goff;
    const u64 *gs = src + goff;
    int lwp = 0;
    while ((1 << lwp) < WW) ++lwp;
    for (int e = threadIdx.x; e < (G << lwp); e += blockDim.x) {
        const int u = e >> lwp, j = e & ((1 << lwp) - 1);
        if (j < WW) copy_async8(win + j * CS + u, gs + ((u64)u << kUnitWordsLog) + ((cw0 + j) & cmask));
    }
    copy_async_wait();
    __syncthreads();
    // one layer per pass over the window: item = (column pair, lo row); the
    // thread that updates lo[p] also writes the quotient fix of the hi word
    // that only lo[p] reads (for d < 64 bits, hi[0] is read by lo[0] and
    // lo[1], which form one pair), so each layer takes a single barrier
    const int nitems = (WW >> 1) << (mw - 1);
    for (int it = 0; it < mw; ++it) {
        const int k = inverse ? it : mw - 1 - it;
        const int hu = 1 << k;                  // rows per half segment
        const int d = 1 << k;                   // bits
        for (int item = threadIdx.x; item < nitems; item += blockDim.x) {
            const int q = item & ((G >> 1) - 1), j = (item >> (mw - 1)) << 1;
            const int u = ((q >> k) << (k + 1)) | (q & (hu - 1));
            const bool first = (q & (hu - 1)) == 0;   // first lo row of its segment
            const int uh = u + hu;                    // hi row at the same offset
            const int ul = u - (q & (hu - 1)) + 2 * hu - 1;   // last hi row of the segment
            const int c = (cw0 + j) & cmask;          // true column of j (even)
            u64 lo[2] = {win[j * CS + u], win[(j + 1) * CS + u]};
            if (d >= 64) {
                const int dw = d >> 6;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int jt = j + t, ct = c + t;
                    if (jt < dw || (first && ct < dw)) continue;   // outside the valid window / lo[p], p < dw
                    const int srow = ct < dw ? uh - 1 : uh;
                    u64 v = win[(jt - dw) * CS + srow];
                    if (first && ct < 2 * dw) {
                        // the source hi[ct - dw] (< dw) takes the fix from hi[hw - dw + ct - dw]
                        if (jt < 2 * dw) continue;
                        const u64 top = win[(jt - 2 * dw) * CS + ul];
                        win[(jt - dw) * CS + uh] = v ^ top;
                        if (!inverse) v ^= top;
                    }
                    lo[t] ^= v;
                }
            } else {
                u64 h0 = win[j * CS + uh];
                const u64 h1 = win[(j + 1) * CS + uh];
                u64 pv = 0;
                if (j >= 1 && !(first && c == 0)) pv = win[(j - 1) * CS + (c == 0 ? uh - 1 : uh)];
                if (first && c == 0 && j >= 1) {
                    // hi[0] ^= hi[hw - 1] >> (64 - d)
                    const u64 top = win[(j - 1) * CS + ul] >> (64 - d);
                    win[j * CS + uh] = h0 ^ top;
                    if (!inverse) h0 ^= top;
                }
                lo[0] ^= (h0 << d) | (pv >> (64 - d));
                lo[1] ^= (h1 << d) | (h0 >> (64 - d));
            }
            win[j * CS + u] = lo[0];
            win[(j + 1) * CS + u] = lo[1];
        }
        __syncthreads();
    }
    const int lw = __ffs(W) - 1;                // W is a power of two
    for (int e = threadIdx.x; e < G * W; e += blockDim.x) {
        const int u = e >> lw, j = e & (W - 1);
        g[((u64)u << kUnitWordsLog) + c0 + j] = win[(halo + j) * CS + u];
    }
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
    int W = 32;
    while (W > 8 && bytes(W) > 180 * 1024) W >>= 1;
    while (W > 8 && ((1u << kUnitWordsLog) / W) * groups * (u64)count < 2 * (u64)ctx->num_sms) W >>= 1;
    const size_t smem = bytes(W);
    const dim3 grid((unsigned)(((1u << kUnitWordsLog) / W) * groups), (unsigned)count);
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
cudaError_t basis_cvt_structured(gf2x_ctx *ctx, u64 *bits, u64 *scratch, u64 L, int K, bool inverse, int count,
                                 u64 stride, cudaStream_t st)
{
    const int m = K - 16;
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

cudaError_t basis_cvt(gf2x_ctx *ctx, u64 *bits, u64 L, bool inverse, int count, u64 stride, u64 *scratch,
                      cudaStream_t st)
{
    int K = 0;
    while ((1ull << K) < L) ++K;
    if (scratch && K >= 18 && K <= 32) return basis_cvt_structured(ctx, bits, scratch, L, K, inverse, count, stride, st);
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

}  // namespace gf2x
