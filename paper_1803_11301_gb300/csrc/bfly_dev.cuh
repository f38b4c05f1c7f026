// Butterfly / iButterfly (Alg. 2, Sec. 2.3.2) with several layers per pass:
// the block bodies of bfly.cu's kernels, shared with the persistent batch
// kernel (persist.cu).  Each body runs as one block described by a VBlock.
//
// Layer i works on blocks of 2^(i+1) points starting at s = blk 2^(i+1) and
// multiplies by c = s_i(alpha + u_s).  By Eq. 4 (s_i shifts Cantor
// coordinates right by i) and alpha = v_{l+32}:
//     c = v_{l+32-i} + (element with Cantor coordinates 2 blk).
//
// Top passes (layers >= bt, the bottom depth): a pass covers m <= 4 consecutive layers
// [p, p+m).  The points it touches are split into columns: for fixed high
// bits (>= p+m) and fixed low bits (< p), the 2^m points that differ in bits
// [p, p+m) form one column, held by one thread in registers through all m
// layers.  All columns of one group (same high bits) share the 2^m - 1
// twiddles of the pass, so the block builds one multiplication table per
// twiddle and reuses it for every column of the group.
//
// Bottom tile (layers < bt; bt = l up to l = 8, else 8 <= bt <= kBottom): 2^bt points in
// shared memory.  Layers i >= kTableMin (twiddle shared by 2^i butterflies per
// array) use tables, packed so that the top layers' tables are built in one
// round and the inverse starts with the tables the forward pass left; layers
// 0..kTableMin-1 multiply with the integer form, in registers (one
// shared-memory pass each for tiles under 64 points).  In the fused
// mode the tile holds the matching tiles of both transforms: forward A,
// forward B, pointwise product, inverse (the Butterfly, pointwise and
// iButterfly steps of Alg. 5 on the low layers) in one pass over HBM.
//
// Multiplication table (method of four Russians, Sec. 4.5): for a fixed c,
// tab[w][e] = c * (e x^(4w)) for the 16 four-bit windows w and e < 16, so
// c*x = XOR_w tab[w][nibble_w(x)].  A window table is 16 x 8 bytes, exactly
// the 32 shared-memory banks, so the 32 lanes of a warp never conflict.  A
// table is built from the 64 powers c x^k: each entry XORs at most four.
#pragma once

#include "gf2x_common.cuh"
#include "gf2x_tables.cuh"

namespace gf2x {
namespace bflyk {


#ifndef GF2X_BOTTOM_LAYERS
#define GF2X_BOTTOM_LAYERS 11        // compile-time override to measure other tile depths
#endif
constexpr int kBottom = GF2X_BOTTOM_LAYERS;   // bottom tile: 2^11 points (16 KiB per transform)
#ifndef GF2X_TABLE_MIN
#define GF2X_TABLE_MIN 4             // compile-time override to measure other thresholds
#endif
constexpr int kTableMin = GF2X_TABLE_MIN;   // bottom layers >= 4 multiply through tables
// Layers per top pass (<= 4; compile-time override to measure others).  On
// GB300 three-layer passes run at 0.82-0.86 of the table-product peak against
// 0.75-0.76 for four-layer ones (half the tables per group, half the values per
// column), which outweighs the extra pass: 9.25 against 9.42 ms per 2^30 x 2^30
// product, 0.085 against 0.091 ms at 2^22, even at 2^24; 5 layers (176 to 255
// registers, one block per SM) measured 10% slower.
#ifndef GF2X_TOP_LAYERS
#define GF2X_TOP_LAYERS 3
#endif
constexpr int kTopLayers = GF2X_TOP_LAYERS;
constexpr int kThreads = 256;
// Element with Cantor coordinates u (window tables of the context).
__device__ __forceinline__ u64 cantor(const u64 *__restrict__ cvt, u64 u)
{
    u64 r = 0;
    for (int k = 0; u; ++k, u >>= 8) r ^= cvt[k * 256 + (u & 255)];
    return r;
}

// ------------------------------------------------------------------ top pass
// Layers [p, p+M) of one or two transforms (vb.by selects x0 or x1).
// Grid.x covers (group, column chunk) pairs: `chunks` chunks of kThreads
// columns per group, each block handling `per_block` consecutive chunks of
// one group.  Tables: layer p + r has 2^(M-1-r) twiddles, stored from table
// 2^(M-1-r) - 1 on; table j of that layer serves rows u with u >> (r+1) = j.
template <int M, bool INV>
__device__ __forceinline__ void bfly_top_body(const VBlock &vb, u64 *smem_raw, u64 *x0, u64 *x1, int l, int p,
                                              u64 chunks, int per_block, const u64 *__restrict__ cvt,
                                              const u64 *__restrict__ vcan, int arrays, u64 stride)
{
    u64 *tabs = align128(smem_raw);
    constexpr int ntab = (1 << M) - 1;
    // vb.by = job * arrays + array; jobs of a batch are `stride` words apart
    const u64 job = vb.by / arrays;
    u64 *x = ((vb.by % arrays) ? x1 : x0) + job * stride;
    const u64 first = (u64)vb.bx * per_block;
    const u64 group = first / chunks;
    pdl_allow();
    build_tables(vb, tabs, ntab, [&](int t) {
        const int lvl = 31 - __clz(t + 1);              // layer r = M-1-lvl holds 2^lvl tables
        const int r = M - 1 - lvl;
        const int j = t - ((1 << lvl) - 1);
        const u64 blk = (group << lvl) | (u64)j;        // block index at layer p + r
        return vcan[l + 32 - (p + r)] ^ cantor(cvt, blk << 1);
    });
    const u64 rstride = 1ull << p;                      // distance between the rows of a column
    pdl_wait();                                         // the twiddle tables need no earlier data
    for (int ch = 0; ch < per_block; ++ch) {
        const u64 chunk = first + ch;
        if (chunk / chunks != group) break;
        const u64 col = (chunk % chunks) * kThreads + vb.t;
        const u64 base = (group << (p + M)) + col;
        u64 v[1 << M];
#pragma unroll
        for (int u = 0; u < (1 << M); ++u) {
            const u64 i = base + (u64)u * rstride;
            v[u] = in_range(i, 1ull << l) ? x[i] : 0;
        }
#pragma unroll
        for (int s2 = 0; s2 < M; ++s2) {
            const int r = INV ? s2 : M - 1 - s2;
            const int half = 1 << r;
            const unsigned tl = smem_addr(tabs) + (unsigned)(((1 << (M - 1 - r)) - 1) * kTab * 8);
#pragma unroll
            for (int u = 0; u < (1 << M); ++u) {
                if (u & half) continue;
                const unsigned tb = tl + (unsigned)((u >> (r + 1)) * kTab * 8);
                if (!INV) {
                    v[u] ^= mul_tab(tb, v[u | half]);
                    v[u | half] ^= v[u];
                } else {
                    v[u | half] ^= v[u];
                    v[u] ^= mul_tab(tb, v[u | half]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < (1 << M); ++u) {
            const u64 i = base + (u64)u * rstride;
            if (in_range(i, 1ull << l)) x[i] = v[u];
        }
    }
}

// -------------------------------------------------------------- bottom tile
// BOTTOM_FUSED: Y holds the top-layer output of the second forward transform;
// BOTTOM_FUSED_PRE: Y already holds a complete forward transform (a reused
// operand), so only X's low layers run before the pointwise product.
enum BottomMode { BOTTOM_FWD = 0, BOTTOM_INV = 1, BOTTOM_FUSED = 2, BOTTOM_FUSED_PRE = 3 };

// One layer i (< bt) on a tile held in shared memory.  ctop = v_{l+32-i} +
// Cantor((tile base) >> i); the block of local start s_lo adds Cantor(s_lo >> i).
template <bool H4>
__device__ __forceinline__ void tile_layer(const VBlock &vb, u64 *a, int bt, int i, u64 ctop, const u64 *__restrict__ cvt, bool inverse)
{
    const int nb = 1 << (bt - 1);                       // butterflies per layer
    const int span = 1 << i;
    for (int t = vb.t; t < nb; t += vb.nt) {
        int blk = t >> i, j = t & (span - 1);
        int s0 = (blk << (i + 1)) + j;
        u64 x0 = a[s0], x1 = a[s0 + span];
        u64 c = ctop ^ cvt[(blk << 1) & 255] ^ cvt[256 + ((blk << 1) >> 8)];   // Cantor(2 blk), 2 blk < 2^11
        if (!inverse) {
            x0 ^= gf64_mul_t<H4>(c, x1);
            x1 ^= x0;
        } else {
            x1 ^= x0;
            x0 ^= gf64_mul_t<H4>(c, x1);
        }
        a[s0] = x0;
        a[s0 + span] = x1;
    }
}

// Butterflies of layer i for the blocks j0 .. j0 + nt - 1 of the tile(s),
// block j's table at slot slot0 + j - j0 of tabs; on A and, if given, B.
__device__ __forceinline__ void table_butterflies(const VBlock &vb, u64 *a, u64 *b, int i, int j0, int nt, int slot0, const u64 *tabs,
                                                  bool inverse)
{
    const int span = 1 << i;
    for (int t = vb.t; t < (nt << i); t += vb.nt) {
        const int blk = j0 + (t >> i), jj = t & (span - 1);
        const int s0 = (blk << (i + 1)) + jj;
        const unsigned tb = smem_addr(tabs) + (unsigned)((slot0 + blk - j0) * kTab * 8);
        u64 x0 = a[s0], x1 = a[s0 + span];
        if (!inverse) {
            x0 ^= mul_tab(tb, x1);
            x1 ^= x0;
        } else {
            x1 ^= x0;
            x0 ^= mul_tab(tb, x1);
        }
        a[s0] = x0;
        a[s0 + span] = x1;
        if (b) {
            u64 y0 = b[s0], y1 = b[s0 + span];
            y0 ^= mul_tab(tb, y1);
            y1 ^= y0;
            b[s0] = y0;
            b[s0 + span] = y1;
        }
    }
}

// The table layers bt-1 .. kTableMin of a tile in the order of the pass
// (forward top down, inverse bottom up), twiddle tables packed.  The layers
// i >= bt - log2(CHUNK) have 2^(bt-i) - 1 tables together (layer i's block j
// at slot 2^(bt-1-i) - 1 + j), built in one round by the whole block; each
// lower layer has 2^(bt-1-i) >= CHUNK tables, built CHUNK at a time.  The
// inverse takes the groups in reverse order, so its first group is the last
// one of the forward pass: with `kept` those tables are still in tabs and are
// not built again.  ctops[i] = v_{l+32-i} + Cantor((tile base) >> i), and the
// block j of layer i adds Cantor(2j), 2j < 2^(bt-i) <= 2^11 (two byte windows).
template <int CHUNK>
__device__ void table_layers(const VBlock &vb, u64 *a, u64 *b, int bt, const u64 *__restrict__ cvt, const u64 *ctops, u64 *tabs,
                             bool inverse, bool kept)
{
    static_assert(CHUNK == 8 || CHUNK == 16 || CHUNK == 32, "chunk of 8, 16 or 32 tables");
    constexpr int kLogChunk = CHUNK == 8 ? 3 : CHUNK == 16 ? 4 : 5;
    if (bt <= kTableMin) return;
    const int lo_top = bt - kLogChunk > kTableMin ? bt - kLogChunk : kTableMin;
    auto twid = [&](int i, int j) {
        const unsigned j2 = (unsigned)j << 1;
        return ctops[i] ^ cvt[j2 & 255] ^ cvt[256 + (j2 >> 8)];
    };
    auto packed = [&](bool build) {
        if (build)
            build_tables(vb, tabs, (1 << (bt - lo_top)) - 1, [&](int t) {
                const int r = 31 - __clz(t + 1);            // slot t: block t + 1 - 2^r of layer bt-1-r
                return twid(bt - 1 - r, t + 1 - (1 << r));
            });
        for (int k = 0; k < bt - lo_top; ++k) {
            const int i = inverse ? lo_top + k : bt - 1 - k;
            table_butterflies(vb, a, b, i, 0, 1 << (bt - 1 - i), (1 << (bt - 1 - i)) - 1, tabs, inverse);
            vb.sync();
        }
    };
    auto chunked = [&](int i, bool first_kept) {
        const int nc = (1 << (bt - 1 - i)) / CHUNK;
        for (int c = 0; c < nc; ++c) {
            const int j0 = (inverse ? nc - 1 - c : c) * CHUNK;
            if (!(first_kept && c == 0)) build_tables(vb, tabs, CHUNK, [&](int t) { return twid(i, j0 + t); });
            table_butterflies(vb, a, b, i, j0, CHUNK, 0, tabs, inverse);
            vb.sync();
        }
    };
    if (!inverse) {
        packed(true);
        for (int i = lo_top - 1; i >= kTableMin; --i) chunked(i, false);
    } else {
        for (int i = kTableMin; i < lo_top; ++i) chunked(i, kept && i == kTableMin);
        packed(!(kept && lo_top == kTableMin));
    }
}

// The low kTableMin (= 4) layers in registers.  Layers 3..0 of the forward
// transforms, the pointwise product and layers 0..3 of the inverse stay
// inside aligned 16-point groups; 8 consecutive lanes hold a group, 2 points
// each.  At layer i lane q (lane mod 8) holds points ins(q, i, 0) and
// ins(q, i, 1) of its group (bit i inserted into q); going from the pairing of
// layer i to that of layer j = i +- 1, each lane swaps one point with lane
// q ^ 2^min(i, j): with b = bit min(i, j) of q it sends slot 1 - b and receives
// into the same slot.  This replaces 9 shared-memory passes and barriers of
// the tile by one load and one store.
static_assert(kTableMin == 4, "the register phase covers layers 0..3");

__device__ __forceinline__ int ins_bit(int q, int i, int s)
{
    return ((q >> i) << (i + 1)) | (s << i) | (q & ((1 << i) - 1));
}

__device__ __forceinline__ void pair_transition(u64 &x0, u64 &x1, int q, int lo)
{
    const int b = (q >> lo) & 1;
    const u64 recv = __shfl_xor_sync(0xffffffffu, b ? x0 : x1, 1 << lo);
    if (b) x0 = recv;
    else x1 = recv;
}

// Runs on every thread of the block; the tile holds 2^bt >= 64 points, so each
// warp's 4 groups are all inside the tile or all outside (warp-uniform loop).
template <bool H4>
__device__ void low_layers_regs(const VBlock &vb, u64 *a, const u64 *b, int bt, const u64 *__restrict__ cvt, const u64 *ctops, bool fwd,
                                bool fwd_b, bool fused, bool inv)
{
    const int T = 1 << bt;
    const int q = vb.t & 7;
    for (int g0 = (vb.t >> 3) * 16; g0 < T; g0 += (vb.nt >> 3) * 16) {
        const int first = fwd ? 3 : 0;
        u64 x0 = a[g0 + ins_bit(q, first, 0)], x1 = a[g0 + ins_bit(q, first, 1)];
        u64 y0 = 0, y1 = 0;
        if (fused) {
            y0 = b[g0 + ins_bit(q, first, 0)];
            y1 = b[g0 + ins_bit(q, first, 1)];
        }
        if (fwd) {
#pragma unroll
            for (int i = 3; i >= 0; --i) {
                const unsigned blk2 = (unsigned)((g0 + ins_bit(q, i, 0)) >> (i + 1)) << 1;   // 2 blk < 2^(bt-i)
                const u64 c = ctops[i] ^ cvt[blk2 & 255] ^ cvt[256 + (blk2 >> 8)];   // twiddle top from shared memory
                x0 ^= gf64_mul_t<H4>(c, x1);
                x1 ^= x0;
                if (fwd_b) {
                    y0 ^= gf64_mul_t<H4>(c, y1);
                    y1 ^= y0;
                }
                if (i > 0) {
                    pair_transition(x0, x1, q, i - 1);
                    if (fused) pair_transition(y0, y1, q, i - 1);
                }
            }
        }
        if (fused) {                                       // pointwise step of Alg. 5
            x0 = gf64_mul_t<H4>(x0, y0);
            x1 = gf64_mul_t<H4>(x1, y1);
        }
        int last = 0;
        if (inv) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const unsigned blk2 = (unsigned)((g0 + ins_bit(q, i, 0)) >> (i + 1)) << 1;
                const u64 c = ctops[i] ^ cvt[blk2 & 255] ^ cvt[256 + (blk2 >> 8)];   // twiddle top from shared memory
                x1 ^= x0;
                x0 ^= gf64_mul_t<H4>(c, x1);
                if (i < 3) pair_transition(x0, x1, q, i);
            }
            last = 3;
        }
        a[g0 + ins_bit(q, last, 0)] = x0;
        a[g0 + ins_bit(q, last, 1)] = x1;
    }
}

// H4: the integer form of the products of layers 0..3 and the pointwise step (gf64_mul_t).
template <int CHUNK, bool H4 = false>
__device__ __forceinline__ void bfly_bottom_body(const VBlock &vb, u64 *smem_raw, u64 *X, u64 *Y, int l, int bt,
                                                 const u64 *__restrict__ cvt, const u64 *__restrict__ vcan, int mode,
                                                 u64 stride)
{
    u64 *sm = align128(smem_raw);
    X += (u64)vb.by * stride;                      // job of a batch
    if (Y) Y += (u64)vb.by * stride;
    const int T = 1 << bt;
    const bool fused = mode == BOTTOM_FUSED || mode == BOTTOM_FUSED_PRE;   // Y's tile is loaded
    const bool fwd_b = mode == BOTTOM_FUSED;                               // and transformed here
    u64 *a = sm;
    u64 *b = fused ? sm + T : nullptr;
    u64 *tabs = sm + (fused ? 2 : 1) * T;
    const u64 base = (u64)vb.bx << bt;
    pdl_allow();
    pdl_wait();
    const bool tile_ok = in_range(base + T - 1, 1ull << l);    // the tile lies in the transform
    for (int k = vb.t; k < T; k += vb.nt) {
        a[k] = tile_ok ? X[base + k] : 0;
        if (fused) b[k] = tile_ok ? Y[base + k] : 0;
    }
    u64 *ctops = tabs + CHUNK * kTab;                   // v_{l+32-i} + Cantor(base >> i), i < bt
    if (vb.t < bt) ctops[vb.t] = vcan[l + 32 - vb.t] ^ cantor(cvt, base >> vb.t);
    vb.sync();
    if (bt >= 6) {                                      // layers 0..3 and the pointwise product in registers
        if (mode != BOTTOM_INV) table_layers<CHUNK>(vb, a, fwd_b ? b : nullptr, bt, cvt, ctops, tabs, false, false);
        low_layers_regs<H4>(vb, a, b, bt, cvt, ctops, mode != BOTTOM_INV, fwd_b, fused, mode != BOTTOM_FWD);
        vb.sync();
        if (mode != BOTTOM_FWD) table_layers<CHUNK>(vb, a, nullptr, bt, cvt, ctops, tabs, true, mode != BOTTOM_INV);
        if (tile_ok)
        for (int k = vb.t; k < T; k += vb.nt) X[base + k] = a[k];
        return;
    }
    // tiles below 64 points (transforms of at most 2^11 bits): the layers one
    // shared-memory pass each
    const int low = bt < kTableMin ? bt : kTableMin;   // layers below `low` multiply in integer form
    if (mode != BOTTOM_INV) {
        table_layers<CHUNK>(vb, a, fwd_b ? b : nullptr, bt, cvt, ctops, tabs, false, false);
        for (int i = low - 1; i >= 0; --i) {
            tile_layer<H4>(vb, a, bt, i, ctops[i], cvt, false);
            if (fwd_b) tile_layer<H4>(vb, b, bt, i, ctops[i], cvt, false);
            vb.sync();
        }
    }
    if (fused) {
        for (int k = vb.t; k < T; k += vb.nt) a[k] = gf64_mul_t<H4>(a[k], b[k]);   // pointwise step of Alg. 5
        vb.sync();
    }
    if (mode != BOTTOM_FWD) {
        for (int i = 0; i < low; ++i) {
            tile_layer<H4>(vb, a, bt, i, ctops[i], cvt, true);
            vb.sync();
        }
        table_layers<CHUNK>(vb, a, nullptr, bt, cvt, ctops, tabs, true, mode != BOTTOM_INV);
    }
    if (tile_ok)
        for (int k = vb.t; k < T; k += vb.nt) X[base + k] = a[k];
}

}  // namespace bflyk
}  // namespace gf2x
