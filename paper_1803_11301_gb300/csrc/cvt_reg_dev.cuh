// Register-resident parts of BasisCvt / iBasisCvt (Alg. 1, Sec. 2.3.1).
//
// (1) The conversion of every aligned 2^16-bit block on its own.  For a
// length 2^K with 16 <= K <= 32, Alg. 1 splits at tau = 2^16 (the largest 2^i
// with i a power of two and i <= K - 1), so its last part is the same
// algorithm inside every block of 2^16 bits; for K >= 33 it splits at 2^32
// and the 2^32-bit blocks again end with it.  Its step list, the flattening
// described in cvt.cu, is fixed: 32 (h, d) steps, generated below at compile
// time.  One warp per block: lane L holds the 32 consecutive words 32L ..
// 32L+31 (2048 bits).  A step whose segments fit in 2048 bits runs inside
// every lane with fixed register indices; a wider step (h >= 2^11, 15 of the
// 32) pairs lane L of the lower half of a segment with lane L + h/2048 of the
// upper half and moves the words it needs with warp shuffles.  No barrier is
// taken between steps; shared memory only turns the coalesced load (lane L
// gets words L, L+32, ...) into the per-lane layout and back, with an XOR
// swizzle that keeps both sides free of bank conflicts.
//
// (2) The "outer" conversion of Alg. 1 on whole units: BasisCvt of length
// 2^M whose coefficients are units of U words (the outer step of a split at
// tau = U bits).  Every step then moves whole units, lo[q] ^= hi'[q - D], so
// each of the U word columns is an independent BasisCvt of 2^M words.  A lane
// group of min(2^M, 32) lanes holds one column, 2^M / 32 units per lane, and
// runs the compile-time step list of BasisCvt(2^M) with the same
// register/shuffle scheme as (1), here without bit shifts.
//
// The block bodies below are shared with the persistent batch kernel
// (persist.cu); cvt_reg.cu launches them.  Each body runs as one block
// described by a VBlock.
#pragma once

#include "gf2x_common.cuh"

namespace gf2x {
namespace cvtrk {

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

constexpr StepList make_steps(int K)
{
    StepList s{};
    gen_steps(s, K, 0);
    return s;
}

constexpr StepList kSteps16 = make_steps(16);
static_assert(kSteps16.n == 32, "BasisCvt of 2^16 bits has 32 steps");

template <int M>
struct StepsOf {
    static constexpr StepList list = make_steps(M);
};

constexpr u64 seg_mask(int h, int lo_bit, int hi_bit)
{
    // bits [lo_bit, hi_bit) of every 2h-bit segment of a word (h < 64)
    u64 one = ((1ull << (hi_bit - lo_bit)) - 1) << lo_bit;
    u64 m = 0;
    for (int s = 0; s < 64; s += 2 * h) m |= one << s;
    return m;
}

__device__ __forceinline__ u64 shfl(u64 v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// One step of a conversion whose elements are whole words (h = H = 2^LH and
// d = D = 2^LD elements), on a column held by a group of lanes with R
// consecutive elements per lane; gl is the lane's index in its group.
// Forward: hi' = hi with its quotient fix hi[r] ^= hi[H - D + r] (r < D),
// then lo[q] ^= hi'[q - D].  Inverse: the lo update with the current hi, then
// the fix.
template <int R, int LH, int LD, bool INV>
__device__ __forceinline__ void wstep(u64 (&w)[R], int gl, int lane)
{
    constexpr int H = 1 << LH, D = 1 << LD;
    if constexpr (2 * H <= R) {
        // segments inside one lane
#pragma unroll
        for (int b = 0; b < R; b += 2 * H) {
            if (!INV) {
#pragma unroll
                for (int r = 0; r < D; ++r) w[b + H + r] ^= w[b + 2 * H - D + r];
            }
#pragma unroll
            for (int q = D; q < H; ++q) w[b + q] ^= w[b + H + q - D];
            if (INV) {
#pragma unroll
                for (int r = 0; r < D; ++r) w[b + H + r] ^= w[b + 2 * H - D + r];
            }
        }
    } else {
        // segments of 2P lanes: lane s < P of a segment holds lo elements,
        // lane s >= P the hi elements at the same offsets
        constexpr int P = H / R;
        const int s = gl & (2 * P - 1);
        const int base = lane - s;
        const u64 lo_mask = s < P ? ~0ull : 0ull;
        if constexpr (D < R) {
            // hi[r] ^= hi[H - D + r] for r < D: first hi lane, from the last one
            auto fix = [&]() {
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    const u64 t = shfl(w[R - D + r], base + 2 * P - 1);
                    if (s == P) w[r] ^= t;
                }
            };
            if (!INV) fix();
            // element j of lo lane s takes element j - D of hi lane s (or
            // element R + j - D of hi lane s - 1)
#pragma unroll
            for (int j = 0; j < R; ++j) {
                u64 v;
                if (j >= D) {
                    v = shfl(w[j - D], lane + P);
                } else {
                    v = shfl(w[R + j - D], lane + P - 1);
                    if (s == 0) v = 0;
                }
                w[j] ^= v & lo_mask;
            }
            if (INV) fix();
        } else {
            // whole lanes: DL = D/R.  Lo lane s >= DL takes hi lane s - DL
            // (lane + P - DL); hi lane s < P + DL is fixed from lane + P - DL.
            constexpr int DL = D / R;
            const u64 fix_mask = (s >= P && s < P + DL) ? ~0ull : 0ull;
            const u64 lo_take = (s >= DL && s < P) ? ~0ull : 0ull;
            if (!INV) {
#pragma unroll
                for (int j = 0; j < R; ++j) w[j] ^= shfl(w[j], lane + P - DL) & fix_mask;
#pragma unroll
                for (int j = 0; j < R; ++j) w[j] ^= shfl(w[j], lane + P - DL) & lo_take;
            } else {
                // sources of both updates are unfixed hi lanes
#pragma unroll
                for (int j = 0; j < R; ++j) w[j] ^= shfl(w[j], lane + P - DL) & (fix_mask | lo_take);
            }
        }
    }
}

// Word index p of a 2^16-bit block -> its slot in shared memory: word 32a + b
// at 32a + (b ^ a).  Lanes that hold R consecutive words each (R = 8, 16 or
// 32) and read or write their j-th word together hit 16 bank pairs, two lanes
// each; so do 32 lanes that take 32 consecutive words.
__device__ __forceinline__ int unit_slot(int p) { return (p & ~31) | ((p & 31) ^ ((p >> 5) & 31)); }

// A step whose segments span several warps, through shared memory: every
// thread stores its words, then takes what it needs from that snapshot
// (forward: lo[q] ^= hi'[q - dw], hi' = hi with the quotient fix; inverse: the
// lo update with the snapshot hi; both: the fix of hi[r] for r < dw).
template <int R, int LH, int LD, bool INV>
__device__ __forceinline__ void xstep(const VBlock &vb, u64 (&w)[R], int t, u64 *sm)
{
    constexpr int hw = 1 << (LH - 6);
    vb.sync();                                    // the previous readers of sm are done
#pragma unroll
    for (int j = 0; j < R; ++j) sm[unit_slot(t * R + j)] = w[j];
    vb.sync();
    const int p0 = t * R;
    const int q0 = p0 & (2 * hw - 1);                   // offset in the segment; all R words in one half
    const int sb = p0 - q0;
    auto at = [&](int x) { return sm[unit_slot(sb + x)]; };
    if (q0 < hw) {
        if constexpr (LD >= 6) {
            constexpr int dw = 1 << (LD - 6);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const int q = q0 + j;
                if (q < dw) continue;
                const int x = q - dw;
                u64 v = at(hw + x);
                if (!INV && x < dw) v ^= at(2 * hw - dw + x);
                w[j] ^= v;
            }
        } else {
            constexpr int d = 1 << LD;
            const u64 fix0 = INV ? 0 : at(2 * hw - 1) >> (64 - d);   // hi'[0] = hi[0] ^ fix0
            u64 prev = q0 > 0 ? at(hw + q0 - 1) : 0;
            if (q0 == 1) prev ^= fix0;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                u64 v = at(hw + q0 + j);
                if (q0 + j == 0) v ^= fix0;
                w[j] ^= (v << d) | (prev >> (64 - d));
                prev = v;
            }
        }
    } else {
        const int r0 = q0 - hw;
        if constexpr (LD >= 6) {
            constexpr int dw = 1 << (LD - 6);
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (r0 + j < dw) w[j] ^= at(2 * hw - dw + r0 + j);
        } else {
            constexpr int d = 1 << LD;
            if (r0 == 0) w[0] ^= at(2 * hw - 1) >> (64 - d);
        }
    }
}

// One step (h = 2^LH, d = 2^LD bits) on a 2^16-bit block held by 1024/R
// threads, R consecutive words each (thread t: words tR .. tR + R - 1).
// Forward: hi' = hi with its quotient fix, lo ^= (hi' << d) mod x^h.
// Inverse: lo ^= (hi << d) mod x^h with the current hi, then the fix.
// Steps with d >= 64 bits move whole words (wstep); wider than a warp: xstep.
template <int R, int LH, int LD, bool INV>
__device__ __forceinline__ void step(const VBlock &vb, u64 (&w)[R], int t, int lane, u64 *sm)
{
    if constexpr (LH >= 6 && (2 << (LH - 6)) > 32 * R) {
        xstep<R, LH, LD, INV>(vb, w, t, sm);
    } else if constexpr (LD >= 6) {
        wstep<R, LH - 6, LD - 6, INV>(w, lane, lane);
    } else if constexpr (LH < 6) {
        // segments inside one word
        constexpr int h = 1 << LH, d = 1 << LD, sh = h - d;
        constexpr u64 ma = seg_mask(h, h, h + d);      // bottom d bits of hi
        constexpr u64 mb = seg_mask(h, d, h);          // lo bits [d, h)
#pragma unroll
        for (int j = 0; j < R; ++j) {
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
    } else if constexpr ((2 << (LH - 6)) <= R) {
        // segments of 2hw <= R words inside one lane; d < 64 bits
        constexpr int hw = 1 << (LH - 6), d = 1 << LD;
#pragma unroll
        for (int b = 0; b < R; b += 2 * hw) {
            if (!INV) w[b + hw] ^= w[b + 2 * hw - 1] >> (64 - d);
#pragma unroll
            for (int q = hw - 1; q >= 0; --q) {
                u64 t2 = w[b + hw + q] << d;
                if (q > 0) t2 |= w[b + hw + q - 1] >> (64 - d);
                w[b + q] ^= t2;
            }
            if (INV) w[b + hw] ^= w[b + 2 * hw - 1] >> (64 - d);
        }
    } else {
        // segments of 2P lanes (lane s < P of a segment holds lo words, lane
        // s >= P the hi words at the same offsets); d < 64 bits
        constexpr int P = (1 << (LH - 6)) / R, d = 1 << LD;
        const int s = lane & (2 * P - 1);
        const int base = lane - s;
        const u64 lo_mask = s < P ? ~0ull : 0ull;
        // the fix: hi[0] ^= hi[hw-1] >> (64 - d), on the first hi lane
        auto fix = [&]() {
            const u64 top = shfl(w[R - 1], base + 2 * P - 1);
            if (s == P) w[0] ^= top >> (64 - d);
        };
        if (!INV) fix();
        // lo[q] ^= (hi[q] << d) | (hi[q-1] >> (64 - d))
        u64 prev = shfl(w[R - 1], lane + P - 1);
        if (s == 0) prev = 0;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const u64 v = shfl(w[j], lane + P);
            w[j] ^= ((v << d) | (prev >> (64 - d))) & lo_mask;
            prev = v;
        }
        if (INV) fix();
    }
}

template <int R, bool INV, int I>
__device__ __forceinline__ void run_steps(const VBlock &vb, u64 (&w)[R], int t, int lane, u64 *sm)
{
    if constexpr (I < 32) {
        // forward order, or the reversed list for the inverse
        constexpr int k = INV ? 31 - I : I;
        step<R, kSteps16.lh[k], kSteps16.ld[k], INV>(vb, w, t, lane, sm);
        run_steps<R, INV, I + 1>(vb, w, t, lane, sm);
    }
}

// One block of 1024/R threads per 2^16-bit block; vb.by is the job of a
// batch.  Words go through shared memory in both directions so that global
// accesses are coalesced (thread t takes words t, t + 1024/R, ...).
// sm: kUnitWords words of shared memory; the block has 1024/R threads.
template <bool INV, int R>
__device__ __forceinline__ void cvt_unit16_body(const VBlock &vb, u64 *sm, u64 *bits, u64 stride)
{
    constexpr int NT = 1024 / R;
    const int t = vb.t, lane = t & 31;
    u64 *g = bits + (u64)vb.by * stride + (u64)vb.bx * kUnitWords;
#pragma unroll 8
    for (int i = 0; i < R; ++i) sm[unit_slot(NT * i + t)] = g[NT * i + t];
    vb.sync();
    u64 w[R];
#pragma unroll
    for (int j = 0; j < R; ++j) w[j] = sm[unit_slot(t * R + j)];
    run_steps<R, INV, 0>(vb, w, t, lane, sm);
    vb.sync();
#pragma unroll
    for (int j = 0; j < R; ++j) sm[unit_slot(t * R + j)] = w[j];
    vb.sync();
#pragma unroll 8
    for (int i = 0; i < R; ++i) g[NT * i + t] = sm[unit_slot(NT * i + t)];
}

template <int M, bool INV, int I>
__device__ __forceinline__ void run_outer_steps(u64 (&w)[(1 << M) >= 32 ? (1 << M) / 32 : 1], int gl, int lane)
{
    constexpr StepList S = StepsOf<M>::list;
    if constexpr (I < S.n) {
        constexpr int k = INV ? S.n - 1 - I : I;
        wstep<((1 << M) >= 32 ? (1 << M) / 32 : 1), S.lh[k], S.ld[k], INV>(w, gl, lane);
        run_outer_steps<M, INV, I + 1>(w, gl, lane);
    }
}

// Block shape of the outer kernel: 16 warps (8 for M = 9, whose 16 units per
// lane take more registers), one column per warp for M >= 5.  The persistent
// batch kernel runs blocks of 8 warps (WARPS_ = 8) for every M.
template <int M, int WARPS_ = (M >= 9 ? 8 : 16)>
struct OuterShape {
    static constexpr int NU = 1 << M;                   // units per column
    static constexpr int LPC = NU < 32 ? NU : 32;       // lanes per column
    static constexpr int R = NU / LPC;                  // units per lane
    static constexpr int CPW = 32 / LPC;                // columns per warp
    static constexpr int WARPS = WARPS_;
    static constexpr int THREADS = WARPS * 32;
    static constexpr int CW = WARPS * CPW;              // columns per block
    static constexpr int S = NU + 1;                    // shared-memory column stride (odd)
    static constexpr int SMEM_WORDS = CW * S;
    // lanes of a column hold units gl R .. gl R + R - 1; unit j of lane gl sits
    // at gl R + (j ^ sigma(gl)), so the 32 lanes reading their j-th unit hit
    // 16 different bank pairs (two lanes each)
    static __device__ __forceinline__ int slot(int gl, int j)
    {
        constexpr int spread = R >= 16 ? 1 : 16 / R;
        return gl * R + (j ^ ((gl / spread) & (R - 1)));
    }
};

// Outer BasisCvt(2^M) on units of 2^ulog words: unit r, column c of chunk ch
// is word (ch 2^M + r) 2^ulog + c.  A block takes CW adjacent columns: their
// unit rows are staged through shared memory (coalesced 8-byte cp.async, one
// row segment of CW words per unit), each lane group takes one column into
// registers, runs the steps, and the rows go back the same way.
// st: CW S words of shared memory (OuterShape<M, WARPS>::SMEM_WORDS); the block has OuterShape<M, WARPS>::THREADS
// threads.
template <int M, bool INV, int WARPS = OuterShape<M>::WARPS>
__device__ __forceinline__ void cvt_outer_body(const VBlock &vb, u64 *st, u64 *bits, const u64 *src, int ulog,
                                               u64 stride)
{
    using Sh = OuterShape<M, WARPS>;
    constexpr int NU = Sh::NU, LPC = Sh::LPC, R = Sh::R, CW = Sh::CW, S = Sh::S;
    const u64 col0 = (u64)vb.bx * CW;
    const u64 ch = col0 >> ulog, c0 = col0 & ((1ull << ulog) - 1);
    const u64 off = (u64)vb.by * stride + ((ch << M) << ulog) + c0;
    u64 *g = bits + off;
    const u64 *gs = src + off;
    // rows in: element (unit r, column w) -> st[w S + slot(r / R, r % R)]
    for (int e = vb.t; e < NU * CW; e += Sh::THREADS) {
        const int r = e / CW, w = e % CW;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(st + w * S + Sh::slot(r / R, r % R));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(gs + ((u64)r << ulog) + w)
                     : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    vb.sync();
    const int lane = vb.t & 31;
    const int gl = lane & (LPC - 1);
    const int w0 = (vb.t >> 5) * Sh::CPW + lane / LPC;   // this lane group's column
    u64 w[R];
#pragma unroll
    for (int j = 0; j < R; ++j) w[j] = st[w0 * S + Sh::slot(gl, j)];
    run_outer_steps<M, INV, 0>(w, gl, lane);
#pragma unroll
    for (int j = 0; j < R; ++j) st[w0 * S + Sh::slot(gl, j)] = w[j];
    vb.sync();
    for (int e = vb.t; e < NU * CW; e += Sh::THREADS) {
        const int r = e / CW, w = e % CW;
        g[((u64)r << ulog) + w] = st[w * S + Sh::slot(r / R, r % R)];
    }
}

}  // namespace cvtrk
}  // namespace gf2x
