// BasisCvt / iBasisCvt (Alg. 1, Sec. 2.3.1) on packed bit arrays: the step
// plan and the block bodies of cvt.cu's step kernels (in-tile runs, column
// runs, wide steps, the Taylor window), shared with the persistent batch
// kernel (persist.cu).  cvt.cu explains the flattening of Alg. 1 into
// (h, d) steps and plans them.  Each body runs as one block described by a
// VBlock.
#pragma once

#include "gf2x_common.cuh"

namespace gf2x {
namespace cvtk {

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
static __device__ void tile_run(const VBlock &vb, u64 *sm, u64 tw, const CvtPlan &P, int first, int count)
{
    const bool inverse = P.inverse != 0;
    for (int s = first; s < first + count; ++s) {
        const u64 h = P.h[s], d = P.d[s];
        if (h < 64) {                            // segments inside one word
            const u64 ma = seg_mask((u32)h, (u32)h, (u32)(h + d));   // hi bottom d bits
            const u64 mb = seg_mask((u32)h, (u32)d, (u32)h);         // lo bits [d, h)
            const u32 sh = (u32)(h - d);
            for (u64 w = vb.t; w < tw; w += vb.nt) {
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
            vb.sync();
        } else {
            const u64 hw = h >> 6;
            const int hl = __ffsll((long long)hw) - 1;
            for (u64 t = vb.t; t < tw / 2; t += vb.nt) {
                u64 seg = t >> hl, q = t & (hw - 1);
                u64 *sp = sm + seg * 2 * hw;
                sp[q] ^= lo_term(sp, hw, d, q, !inverse);
            }
            vb.sync();
            const u64 nfix = d >= 64 ? (d >> 6) : 1;
            const int fl = __ffsll((long long)nfix) - 1;
            const u64 nseg = tw / (2 * hw);
            for (u64 t = vb.t; t < nseg * nfix; t += vb.nt) {
                u64 seg = t >> fl, r = t & (nfix - 1);
                u64 *sp = sm + seg * 2 * hw;
                if (d >= 64) sp[hw + r] ^= sp[2 * hw - nfix + r];
                else sp[hw] ^= sp[2 * hw - 1] >> (64 - d);
            }
            vb.sync();
        }
    }
}

// One wide step in place (segments larger than a tile, so h >= 2^18 bits, hw >= 4096 words).
// Each thread owns four consecutive lo words.
// Out of place (src != bits): every word is read from src and the thread
// writes lo[q] and hi[q] of its four indices q to bits (the fix of hi[q] is
// computed from src by its own thread).
__device__ __forceinline__ void cvt_wide_body(const VBlock &vb, u64 *bits, const u64 *src, u64 words, u64 h, u64 d,
                                              int inverse, u64 stride)
{
    bits += (u64)vb.by * stride;             // job of a batch
    src += (u64)vb.by * stride;
    const u64 hw = h >> 6;
    const int hl = __ffsll((long long)hw) - 1;
    const u64 t = (u64)vb.bx * vb.nt + vb.t;
    if (4 * t >= words / 2) return;
    const u64 w = 4 * t;                          // index among all lo words
    const u64 seg = w >> hl, q0 = w & (hw - 1);
    if (!in_range(seg * 2 * hw + 2 * hw - 1, words)) return;   // the thread's segment lies in the array
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
__device__ __forceinline__ void cvt_tile_body(const VBlock &vb, u64 *sm, u64 *bits, const u64 *src, const CvtPlan &P,
                                              int phase, u64 stride)
{
    bits += (u64)vb.by * stride;
    src += (u64)vb.by * stride;
    const u64 tw = 1ull << P.tw_log;
    if (!in_range((u64)vb.bx * tw + tw - 1, P.words)) return;   // the tile lies in the array
    u64 *g = bits + (u64)vb.bx * tw;
    const u64 *gs = src + (u64)vb.bx * tw;
    for (u64 w = vb.t; w < tw; w += vb.nt) copy_async8(sm + w, gs + w);
    copy_async_wait();
    vb.sync();
    tile_run(vb, sm, tw, P, P.first[phase], P.count[phase]);
    for (u64 w = vb.t; w < tw; w += vb.nt) g[w] = sm[w];
}

// A run of steps whose d are all multiples of a unit U (>= 4 words): every step
// moves whole units, so the same step applies to each word column of the units
// independently.  A block holds 2^wlog word columns of 2^slog consecutive
// units (a segment-aligned range at least as long as the run's segments).
__device__ __forceinline__ void cvt_col_body(const VBlock &vb, u64 *sm, u64 *bits, const u64 *src, const CvtPlan &P,
                                             int phase, u64 stride)
{
    bits += (u64)vb.by * stride;
    src += (u64)vb.by * stride;
    const int ulog = P.ulog[phase], wlog = P.wlog[phase], slog = P.slog[phase];
    const u64 uw = 1ull << (ulog - 6);                  // words per unit
    const u64 W = 1ull << wlog, S = 1ull << slog;
    const u64 cols = uw >> wlog;                        // column blocks per unit
    const u64 u0 = ((u64)vb.bx / cols) << slog, c0 = ((u64)vb.bx % cols) << wlog;
    if (!in_range((u0 + S - 1) * uw + c0 + W - 1, P.words)) return;   // the block's units lie in the array
    for (u64 k = vb.t; k < S * W; k += vb.nt)
        copy_async8(sm + k, src + (u0 + (k >> wlog)) * uw + c0 + (k & (W - 1)));
    copy_async_wait();
    vb.sync();
    const bool inverse = P.inverse != 0;
    for (int s = P.first[phase]; s < P.first[phase] + P.count[phase]; ++s) {
        const u64 H = P.h[s] >> ulog, D = P.d[s] >> ulog;      // in units
        const int hl = __ffsll((long long)H) - 1;
        // lo[q] ^= hi'[q - D], hi' = hi with the quotient fix (forward)
        for (u64 k = vb.t; k < (S / 2) * W; k += vb.nt) {
            const u64 e = k >> wlog, w = k & (W - 1);
            const u64 base = (e >> hl) << (hl + 1), q = e & (H - 1);
            if (q < D) continue;
            const u64 r = q - D;
            u64 hv = sm[((base + H + r) << wlog) + w];
            if (!inverse && r < D) hv ^= sm[((base + 2 * H - D + r) << wlog) + w];
            sm[((base + q) << wlog) + w] ^= hv;
        }
        vb.sync();
        // hi[r] ^= hi[H - D + r], r < D
        const int dl = __ffsll((long long)D) - 1;
        for (u64 k = vb.t; k < (S >> (hl + 1)) * D * W; k += vb.nt) {
            const u64 w = k & (W - 1), rest = k >> wlog;
            const u64 r = rest & (D - 1), seg = rest >> dl;
            const u64 base = seg << (hl + 1);
            sm[((base + H + r) << wlog) + w] ^= sm[((base + 2 * H - D + r) << wlog) + w];
        }
        vb.sync();
    }
    for (u64 k = vb.t; k < S * W; k += vb.nt)
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

__device__ __forceinline__ void cvt_taylor_body(const VBlock &vb, u64 *win, u64 *bits, const u64 *src, int mw, int W,
                                                int inverse, u64 stride)
{
    // window storage, column-major: win[j * (G + 1) + u] (row u, window column
    // j).  The odd column stride keeps both the load (consecutive columns of
    // one row) and the steps (consecutive rows of one column) conflict-free.
    const int halo = taylor_halo(mw);
    const int WW = W + halo, G = 1 << mw, CS = G + 1;
    const int nwin = (1 << kUnitWordsLog) / W;
    const int c0 = (int)(vb.bx % nwin) * W;
    const int cw0 = c0 - halo;                  // true column of window column 0 (mod 1024)
    const int cmask = (1 << kUnitWordsLog) - 1;
    const u64 goff = (u64)vb.by * stride + ((u64)(vb.bx / nwin) << (mw + kUnitWordsLog));
    u64 *g = bits + goff;
    const u64 *gs = src + goff;
    int lwp = 0;
    while ((1 << lwp) < WW) ++lwp;
    for (int e = vb.t; e < (G << lwp); e += vb.nt) {
        const int u = e >> lwp, j = e & ((1 << lwp) - 1);
        if (j < WW) copy_async8(win + j * CS + u, gs + ((u64)u << kUnitWordsLog) + ((cw0 + j) & cmask));
    }
    copy_async_wait();
    vb.sync();
    // one layer per pass over the window: item = (column pair, lo row); the
    // thread that updates lo[p] also writes the quotient fix of the hi word
    // that only lo[p] reads (for d < 64 bits, hi[0] is read by lo[0] and
    // lo[1], which form one pair), so each layer takes a single barrier
    const int nitems = (WW >> 1) << (mw - 1);
    for (int it = 0; it < mw; ++it) {
        const int k = inverse ? it : mw - 1 - it;
        const int hu = 1 << k;                  // rows per half segment
        const int d = 1 << k;                   // bits
        for (int item = vb.t; item < nitems; item += vb.nt) {
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
        vb.sync();
    }
    const int lw = __ffs(W) - 1;                // W is a power of two
    for (int e = vb.t; e < G * W; e += vb.nt) {
        const int u = e >> lw, j = e & (W - 1);
        g[((u64)u << kUnitWordsLog) + c0 + j] = win[(halo + j) * CS + u];
    }
}

}  // namespace cvtk
}  // namespace gf2x
