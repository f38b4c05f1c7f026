// Butterfly / iButterfly (Alg. 2, Sec. 2.3.2) with several layers per pass.
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
#include "gf2x_common.cuh"
#include "gf2x_tables.cuh"

namespace gf2x {
namespace {

#ifndef GF2X_BOTTOM_LAYERS
#define GF2X_BOTTOM_LAYERS 11        // compile-time override to measure other tile depths
#endif
constexpr int kBottom = GF2X_BOTTOM_LAYERS;   // bottom tile: 2^11 points (16 KiB per transform)
#ifndef GF2X_TABLE_MIN
#define GF2X_TABLE_MIN 4             // compile-time override to measure other thresholds
#endif
constexpr int kTableMin = GF2X_TABLE_MIN;   // bottom layers >= 4 multiply through tables
// Layers per top pass (<= 4; compile-time override to measure others).  On
// GB300, 3 measured 1.6% faster at 2^30-bit operands and even at 2^24; 5 (176
// to 255 registers, one block per SM) 10% slower.
#ifndef GF2X_TOP_LAYERS
#define GF2X_TOP_LAYERS 4
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
// Layers [p, p+M) of one or two transforms (blockIdx.y selects x0 or x1).
// Grid.x covers (group, column chunk) pairs: `chunks` chunks of kThreads
// columns per group, each block handling `per_block` consecutive chunks of
// one group.  Tables: layer p + r has 2^(M-1-r) twiddles, stored from table
// 2^(M-1-r) - 1 on; table j of that layer serves rows u with u >> (r+1) = j.
template <int M, bool INV>
__global__ void __launch_bounds__(kThreads) k_bfly_top(u64 *x0, u64 *x1, int l, int p, u64 chunks, int per_block,
                                                       const u64 *__restrict__ cvt, const u64 *__restrict__ vb,
                                                       int arrays, u64 stride)
{
    extern __shared__ u64 smem_raw[];
    u64 *tabs = align128(smem_raw);
    constexpr int ntab = (1 << M) - 1;
    // blockIdx.y = job * arrays + array; jobs of a batch are `stride` words apart
    const u64 job = blockIdx.y / arrays;
    u64 *x = ((blockIdx.y % arrays) ? x1 : x0) + job * stride;
    const u64 first = (u64)blockIdx.x * per_block;
    const u64 group = first / chunks;
    pdl_allow();
    build_tables(tabs, ntab, [&](int t) {
        const int lvl = 31 - __clz(t + 1);              // layer r = M-1-lvl holds 2^lvl tables
        const int r = M - 1 - lvl;
        const int j = t - ((1 << lvl) - 1);
        const u64 blk = (group << lvl) | (u64)j;        // block index at layer p + r
        return vb[l + 32 - (p + r)] ^ cantor(cvt, blk << 1);
    });
    const u64 rstride = 1ull << p;                      // distance between the rows of a column
    pdl_wait();                                         // the twiddle tables need no earlier data
    for (int ch = 0; ch < per_block; ++ch) {
        const u64 chunk = first + ch;
        if (chunk / chunks != group) break;
        const u64 col = (chunk % chunks) * kThreads + threadIdx.x;
        const u64 base = (group << (p + M)) + col;
        u64 v[1 << M];
#pragma unroll
        for (int u = 0; u < (1 << M); ++u) v[u] = x[base + (u64)u * rstride];
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
        for (int u = 0; u < (1 << M); ++u) x[base + (u64)u * rstride] = v[u];
    }
}

// -------------------------------------------------------------- bottom tile
// BOTTOM_FUSED: Y holds the top-layer output of the second forward transform;
// BOTTOM_FUSED_PRE: Y already holds a complete forward transform (a reused
// operand), so only X's low layers run before the pointwise product.
enum BottomMode { BOTTOM_FWD = 0, BOTTOM_INV = 1, BOTTOM_FUSED = 2, BOTTOM_FUSED_PRE = 3 };

// One layer i (< bt) on a tile held in shared memory.  ctop = v_{l+32-i} +
// Cantor((tile base) >> i); the block of local start s_lo adds Cantor(s_lo >> i).
__device__ __forceinline__ void tile_layer(u64 *a, int bt, int i, u64 ctop, const u64 *__restrict__ cvt, bool inverse)
{
    const int nb = 1 << (bt - 1);                       // butterflies per layer
    const int span = 1 << i;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        int blk = t >> i, j = t & (span - 1);
        int s0 = (blk << (i + 1)) + j;
        u64 x0 = a[s0], x1 = a[s0 + span];
        u64 c = ctop ^ cvt[(blk << 1) & 255] ^ cvt[256 + ((blk << 1) >> 8)];   // Cantor(2 blk), 2 blk < 2^11
        if (!inverse) {
            x0 ^= gf64_mul(c, x1);
            x1 ^= x0;
        } else {
            x1 ^= x0;
            x0 ^= gf64_mul(c, x1);
        }
        a[s0] = x0;
        a[s0 + span] = x1;
    }
}

// Butterflies of layer i for the blocks j0 .. j0 + nt - 1 of the tile(s),
// block j's table at slot slot0 + j - j0 of tabs; on A and, if given, B.
__device__ __forceinline__ void table_butterflies(u64 *a, u64 *b, int i, int j0, int nt, int slot0, const u64 *tabs,
                                                  bool inverse)
{
    const int span = 1 << i;
    for (int t = threadIdx.x; t < (nt << i); t += blockDim.x) {
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
__device__ void table_layers(u64 *a, u64 *b, int bt, const u64 *__restrict__ cvt, const u64 *ctops, u64 *tabs,
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
            build_tables(tabs, (1 << (bt - lo_top)) - 1, [&](int t) {
                const int r = 31 - __clz(t + 1);            // slot t: block t + 1 - 2^r of layer bt-1-r
                return twid(bt - 1 - r, t + 1 - (1 << r));
            });
        for (int k = 0; k < bt - lo_top; ++k) {
            const int i = inverse ? lo_top + k : bt - 1 - k;
            table_butterflies(a, b, i, 0, 1 << (bt - 1 - i), (1 << (bt - 1 - i)) - 1, tabs, inverse);
            __syncthreads();
        }
    };
    auto chunked = [&](int i, bool first_kept) {
        const int nc = (1 << (bt - 1 - i)) / CHUNK;
        for (int c = 0; c < nc; ++c) {
            const int j0 = (inverse ? nc - 1 - c : c) * CHUNK;
            if (!(first_kept && c == 0)) build_tables(tabs, CHUNK, [&](int t) { return twid(i, j0 + t); });
            table_butterflies(a, b, i, j0, CHUNK, 0, tabs, inverse);
            __syncthreads();
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
__device__ void low_layers_regs(u64 *a, const u64 *b, int bt, const u64 *__restrict__ cvt, const u64 *ctops, bool fwd,
                                bool fwd_b, bool fused, bool inv)
{
    const int T = 1 << bt;
    const int q = threadIdx.x & 7;
    u64 ctop[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) ctop[i] = ctops[i];
    for (int g0 = (threadIdx.x >> 3) * 16; g0 < T; g0 += (blockDim.x >> 3) * 16) {
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
                const u64 c = ctop[i] ^ cvt[blk2 & 255] ^ cvt[256 + (blk2 >> 8)];
                x0 ^= gf64_mul(c, x1);
                x1 ^= x0;
                if (fwd_b) {
                    y0 ^= gf64_mul(c, y1);
                    y1 ^= y0;
                }
                if (i > 0) {
                    pair_transition(x0, x1, q, i - 1);
                    if (fused) pair_transition(y0, y1, q, i - 1);
                }
            }
        }
        if (fused) {                                       // pointwise step of Alg. 5
            x0 = gf64_mul(x0, y0);
            x1 = gf64_mul(x1, y1);
        }
        int last = 0;
        if (inv) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const unsigned blk2 = (unsigned)((g0 + ins_bit(q, i, 0)) >> (i + 1)) << 1;
                const u64 c = ctop[i] ^ cvt[blk2 & 255] ^ cvt[256 + (blk2 >> 8)];
                x1 ^= x0;
                x0 ^= gf64_mul(c, x1);
                if (i < 3) pair_transition(x0, x1, q, i);
            }
            last = 3;
        }
        a[g0 + ins_bit(q, last, 0)] = x0;
        a[g0 + ins_bit(q, last, 1)] = x1;
    }
}

template <int THREADS, int CHUNK>
__global__ void __launch_bounds__(THREADS, 65536 / (THREADS * 64)) k_bfly_bottom(u64 *X, u64 *Y, int l, int bt, const u64 *__restrict__ cvt,
                                                          const u64 *__restrict__ vb, int mode, u64 stride)
{
    extern __shared__ u64 smem_raw[];
    u64 *sm = align128(smem_raw);
    X += (u64)blockIdx.y * stride;                      // job of a batch
    if (Y) Y += (u64)blockIdx.y * stride;
    const int T = 1 << bt;
    const bool fused = mode == BOTTOM_FUSED || mode == BOTTOM_FUSED_PRE;   // Y's tile is loaded
    const bool fwd_b = mode == BOTTOM_FUSED;                               // and transformed here
    u64 *a = sm;
    u64 *b = fused ? sm + T : nullptr;
    u64 *tabs = sm + (fused ? 2 : 1) * T;
    const u64 base = (u64)blockIdx.x << bt;
    pdl_allow();
    pdl_wait();
    for (int k = threadIdx.x; k < T; k += blockDim.x) {
        a[k] = X[base + k];
        if (fused) b[k] = Y[base + k];
    }
    u64 *ctops = tabs + CHUNK * kTab;                   // v_{l+32-i} + Cantor(base >> i), i < bt
    if (threadIdx.x < bt) ctops[threadIdx.x] = vb[l + 32 - threadIdx.x] ^ cantor(cvt, base >> threadIdx.x);
    __syncthreads();
    if (bt >= 6) {                                      // layers 0..3 and the pointwise product in registers
        if (mode != BOTTOM_INV) table_layers<CHUNK>(a, fwd_b ? b : nullptr, bt, cvt, ctops, tabs, false, false);
        low_layers_regs(a, b, bt, cvt, ctops, mode != BOTTOM_INV, fwd_b, fused, mode != BOTTOM_FWD);
        __syncthreads();
        if (mode != BOTTOM_FWD) table_layers<CHUNK>(a, nullptr, bt, cvt, ctops, tabs, true, mode != BOTTOM_INV);
        for (int k = threadIdx.x; k < T; k += blockDim.x) X[base + k] = a[k];
        return;
    }
    // tiles below 64 points (transforms of at most 2^11 bits): the layers one
    // shared-memory pass each
    const int low = bt < kTableMin ? bt : kTableMin;   // layers below `low` multiply in integer form
    if (mode != BOTTOM_INV) {
        table_layers<CHUNK>(a, fwd_b ? b : nullptr, bt, cvt, ctops, tabs, false, false);
        for (int i = low - 1; i >= 0; --i) {
            tile_layer(a, bt, i, ctops[i], cvt, false);
            if (fwd_b) tile_layer(b, bt, i, ctops[i], cvt, false);
            __syncthreads();
        }
    }
    if (fused) {
        for (int k = threadIdx.x; k < T; k += blockDim.x) a[k] = gf64_mul(a[k], b[k]);   // pointwise step of Alg. 5
        __syncthreads();
    }
    if (mode != BOTTOM_FWD) {
        for (int i = 0; i < low; ++i) {
            tile_layer(a, bt, i, ctops[i], cvt, true);
            __syncthreads();
        }
        table_layers<CHUNK>(a, nullptr, bt, cvt, ctops, tabs, true, mode != BOTTOM_INV);
    }
    for (int k = threadIdx.x; k < T; k += blockDim.x) X[base + k] = a[k];
}

size_t bottom_smem(int bt, bool fused, int chunk)
{
    return ((fused ? 2 : 1) * (size_t)(1 << bt) + (size_t)chunk * kTab + 16) * sizeof(u64) + 128;
}

// Bottom kernel shapes (threads per block, tables built at a time): with few
// tiles, 512 threads and 32-table chunks keep more warps in flight (2 blocks
// per SM); with many tiles, 256 threads and 16-table chunks fit 3 blocks per
// SM and issue better (measured on GB300: 91.7 vs 95.8 us at 256 tiles,
// 4.48 vs 4.08 ms at 16384 tiles).
constexpr int kBottomThreadsSmall = 512, kBottomChunkSmall = 32;
constexpr int kBottomThreadsLarge = 256, kBottomChunkLarge = 16;
// A third shape for the tuner: 256 threads building 8 tables at a time (48 KiB
// at 2^11-point tiles, 4 blocks per SM; more build rounds, more warps).
constexpr int kBottomChunkLean = 8;

// shape 1: the small-count shape, 0: the large-count one, 2: the lean one
cudaError_t launch_bottom_shape(gf2x_ctx *ctx, u64 *X, u64 *Y, int l, int bt, int mode, int count, u64 stride,
                                int shape, cudaStream_t st)
{
    const bool fused = mode == BOTTOM_FUSED || mode == BOTTOM_FUSED_PRE;
    const dim3 grid((unsigned)(1ull << (l - bt)), count);
    cudaError_t e;
    if (shape == 1)
        e = launch_pdl(ctx->pdl, k_bfly_bottom<kBottomThreadsSmall, kBottomChunkSmall>, grid, dim3(kBottomThreadsSmall),
                       bottom_smem(bt, fused, kBottomChunkSmall), st, X, Y, l, bt, ctx->d_cvt, ctx->d_cantor, mode,
                       stride);
    else if (shape == 2)
        e = launch_pdl(ctx->pdl, k_bfly_bottom<kBottomThreadsLarge, kBottomChunkLean>, grid, dim3(kBottomThreadsLarge),
                       bottom_smem(bt, fused, kBottomChunkLean), st, X, Y, l, bt, ctx->d_cvt, ctx->d_cantor, mode,
                       stride);
    else
        e = launch_pdl(ctx->pdl, k_bfly_bottom<kBottomThreadsLarge, kBottomChunkLarge>, grid, dim3(kBottomThreadsLarge),
                       bottom_smem(bt, fused, kBottomChunkLarge), st, X, Y, l, bt, ctx->d_cvt, ctx->d_cantor, mode,
                       stride);
    count_launch(ctx);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// The shape measured by the tuner on `scratch` (a free buffer laid out like X;
// Y, when the mode reads it, is only read), or the default without one.
void launch_bottom(gf2x_ctx *ctx, u64 *X, u64 *Y, int l, int bt, int mode, int count, u64 stride, u64 *scratch,
                   cudaStream_t st)
{
    const u64 tiles = 1ull << (l - bt);
    int shape = tiles * (u64)count < 4 * (u64)ctx->num_sms ? 1 : 0;
    static const int cands[3] = {1, 0, 2};
    if (!scratch) shape = tune_pinned(ctx, TUNE_BOTTOM_SHAPE, cands, 3, shape);
    else {
        shape = tune_choice(ctx, TUNE_BOTTOM_SHAPE, (tune_bucket(tiles * (u64)count) << 2) | (u64)mode, cands, 3, shape,
                            [&](int sh) { return launch_bottom_shape(ctx, scratch, Y, l, bt, mode, count, stride, sh, st); },
                            st);
    }
    launch_bottom_shape(ctx, X, Y, l, bt, mode, count, stride, shape, st);
}

template <int M, bool INV>
void launch_top(bool pdl, dim3 grid, cudaStream_t st, u64 *x0, u64 *x1, int l, int p, u64 chunks, int per_block,
                const u64 *cvt, const u64 *vb, int arrays, u64 stride)
{
    size_t smem = (size_t)((1 << M) - 1) * kTab * sizeof(u64) + 128;
    launch_pdl(pdl, k_bfly_top<M, INV>, grid, dim3(kThreads), smem, st, x0, x1, l, p, chunks, per_block, cvt, vb,
               arrays, stride);
}

cudaError_t top_passes(gf2x_ctx *ctx, u64 *x0, u64 *x1, int l, int bt, bool inverse, int count, u64 stride,
                       cudaStream_t st)
{
    // passes over layers [bt, l), as few as kTopLayers allows, the layers split
    // evenly (the lower passes take one more where they do not divide: 9 layers
    // are 3 + 3 + 3, not 4 + 4 + 1); high to low for the forward transform
    const int layers = l - bt;
    const int npass = (layers + kTopLayers - 1) / kTopLayers;
    const int per = npass ? layers / npass : 0, rem = npass ? layers % npass : 0;
    for (int k = 0; k < npass; ++k) {
        const int idx = inverse ? k : npass - 1 - k;
        const int p = bt + idx * per + (idx < rem ? idx : rem);
        const int m = per + (idx < rem ? 1 : 0);
        const u64 chunks = (1ull << p) / kThreads;     // p >= bt >= 8, so 2^p >= 256 columns
        const u64 groups = (1ull << l) >> (p + m);
        // chunks per block: up to 8 (tables built once per block), but keep at
        // least two blocks per SM; a power of two, so it divides `chunks`
        const int arrays = x1 ? 2 : 1;
        u64 pb = chunks * groups * (u64)arrays * (u64)count / (2 * (u64)ctx->num_sms);
        int per_block = 1;
        while (per_block < 8 && (u64)(2 * per_block) <= pb && (u64)(2 * per_block) <= chunks) per_block *= 2;
        dim3 grid((unsigned)(chunks * groups / per_block), (unsigned)(arrays * count));
        const u64 *cvt = ctx->d_cvt, *vb = ctx->d_cantor;
        switch (m * 2 + (inverse ? 1 : 0)) {
        case 2: launch_top<1, false>(ctx->pdl, grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 3: launch_top<1, true>(ctx->pdl, grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 4: launch_top<2, false>(ctx->pdl, grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 5: launch_top<2, true>(ctx->pdl, grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 6: launch_top<3, false>(ctx->pdl, grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 7: launch_top<3, true>(ctx->pdl, grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 8: launch_top<4, false>(ctx->pdl, grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        default: launch_top<4, true>(ctx->pdl, grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        }
        count_launch(ctx);
    }
    return cudaGetLastError();
}

bool configured = false;

void configure()
{
    if (configured) return;
    cudaFuncSetAttribute(k_bfly_bottom<kBottomThreadsSmall, kBottomChunkSmall>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bottom_smem(kBottom, true, kBottomChunkSmall));
    cudaFuncSetAttribute(k_bfly_bottom<kBottomThreadsLarge, kBottomChunkLarge>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bottom_smem(kBottom, true, kBottomChunkLarge));
    cudaFuncSetAttribute(k_bfly_bottom<kBottomThreadsLarge, kBottomChunkLean>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bottom_smem(kBottom, true, kBottomChunkLean));
    configured = true;
}

}  // namespace

constexpr int kMinDepth = 8;              // shallowest depth the tuner tries

// The depth used without a measurement: 9 up to l = 21, kBottom above.
static int default_depth(int l)
{
    const int bt = l <= 21 ? 9 : kBottom;
    return l < bt ? l : bt;
}

static int depth_or_default(int bt, int l)   // bt < 0: the default depth
{
    if (bt < 0) return default_depth(l);
    return l < bt ? l : bt;
}

// A depth pinned by gf2x_tune_pin if it is one of the candidates for l (8 ..
// min(kBottom, l)), else fallback.
static int pinned_depth(gf2x_ctx *ctx, int l, int fallback)
{
    int cands[kBottom];
    int nc = 0;
    for (int b = kMinDepth; b <= kBottom && b <= l; ++b) cands[nc++] = b;
    return tune_pinned(ctx, TUNE_BFLY_DEPTH, cands, nc, fallback);
}

// Forward (or inverse) Butterfly of `count` transforms of 2^l points each,
// `stride` words apart.
cudaError_t butterfly(gf2x_ctx *ctx, u64 *x, int l, bool inverse, int count, u64 stride, cudaStream_t st,
                      u64 *scratch)
{
    configure();
    const int bt = pinned_depth(ctx, l, default_depth(l));
    if (!inverse) {
        cudaError_t e = top_passes(ctx, x, nullptr, l, bt, false, count, stride, st);
        if (e != cudaSuccess) return e;
    }
    if (bt > 0) {
        launch_bottom(ctx, x, nullptr, l, bt, inverse ? BOTTOM_INV : BOTTOM_FWD, count, stride, scratch, st);
    }
    if (inverse) return top_passes(ctx, x, nullptr, l, bt, true, count, stride, st);
    return cudaGetLastError();
}


// Bottom-tile depth for the products of one size class (l, count).  The tuner
// times the whole schedule (top passes of both forward transforms, the fused
// bottom kernel, top passes of the inverse) for each depth 8..kBottom on X and
// Y while they are free, before Encode writes them; the bottom kernel's block
// shape is tuned for each depth on T (the measurement happens in the untimed
// first run of the candidate, so the timed runs use the depth's best shape).  A deeper tile moves
// layers from the HBM passes into shared memory but leaves fewer tiles to
// spread over the SMs (measured on GB300: 9 is fastest up to 2^24-bit
// operands, 11 at 2^30); the default without measuring follows that.
int butterfly_depth_stored(gf2x_ctx *ctx, int l, int count)
{
    if (l <= kMinDepth) return l;
    return pinned_depth(ctx, l,
                        tune_stored(ctx, TUNE_BFLY_DEPTH, ((u64)l << 32) | tune_bucket((u64)count), default_depth(l)));
}

int butterfly_depth(gf2x_ctx *ctx, u64 *X, u64 *Y, u64 *T, int l, int count, u64 stride, cudaStream_t st)
{
    configure();
    if (l <= kMinDepth) return l;
    const int fallback = default_depth(l);
    int cands[kBottom];
    int nc = 0;
    for (int b = kMinDepth; b <= kBottom && b <= l; ++b) cands[nc++] = b;
    return tune_choice(ctx, TUNE_BFLY_DEPTH, ((u64)l << 32) | tune_bucket((u64)count), cands, nc, fallback,
                       [&](int bt) -> cudaError_t {
                           cudaError_t e = top_passes(ctx, X, Y, l, bt, false, count, stride, st);
                           if (e != cudaSuccess) return e;
                           launch_bottom(ctx, X, Y, l, bt, BOTTOM_FUSED, count, stride, T, st);
                           return top_passes(ctx, X, nullptr, l, bt, true, count, stride, st);
                       },
                       st);
}

// The top layers of both forward transforms (X and Y, or X alone) in one launch per pass.
cudaError_t butterfly_top_pair(gf2x_ctx *ctx, u64 *x0, u64 *x1, int l, int count, u64 stride, cudaStream_t st, int bt)
{
    configure();
    return top_passes(ctx, x0, x1, l, depth_or_default(bt, l), false, count, stride, st);
}

// Bottom layers of both forward transforms, the pointwise product and the
// bottom layers of the inverse: X <- low layers of iButterfly(fwd(X) * fwd(Y)).
// With y_transformed, Y is already a complete forward transform.
cudaError_t butterfly_bottom_fused(gf2x_ctx *ctx, u64 *X, u64 *Y, int l, int count, u64 stride, cudaStream_t st,
                                   bool y_transformed, u64 *scratch, int bt)
{
    configure();
    bt = depth_or_default(bt, l);
    launch_bottom(ctx, X, Y, l, bt, y_transformed ? BOTTOM_FUSED_PRE : BOTTOM_FUSED, count, stride, scratch, st);
    return cudaGetLastError();
}

// The top layers of the inverse.
cudaError_t butterfly_top_inverse(gf2x_ctx *ctx, u64 *x, int l, int count, u64 stride, cudaStream_t st, int bt)
{
    configure();
    return top_passes(ctx, x, nullptr, l, depth_or_default(bt, l), true, count, stride, st);
}

}  // namespace gf2x
