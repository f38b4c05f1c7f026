// FP_Polymul with m = 128: the points are elements of GF(2^128) =
// GF(2)[x] / (x^128 + x^7 + x^2 + x + 1) (Sec. 4.3), n_p = n / 128 of them on
// Sigma = v_{l+64} + V_l (Eq. 6 with m/2 = 64), and Encode collapses the first
// l_m = 7 Butterfly layers (Sec. 3.2-3.3).  BasisCvt and the bit-array load /
// store work on GF(2)[x] and are the kernels of the m = 64 path.
//
// A point is two words, lo (bits 0..63) then hi (bits 64..127), so a
// transform of n bits holds n/128 points in n/64 words: the buffers of the
// m = 64 path.  Every point is read and written with one 16-byte access.
//
// Product by a twiddle c (Butterfly layers whose twiddle is shared by many
// butterflies): method of four Russians with 4-bit windows (Sec. 4.5), a
// table per twiddle of 32 windows x 16 entries.  Each window keeps its 16 low
// words and its 16 high words in two 128-byte rows, so one lookup is two
// 8-byte loads that never conflict across the 32 lanes.  Other products
// (low layers, pointwise) use the integer form: Karatsuba over three 64 x 64
// carry-less products, each three 32 x 32 ones (clmul32_h4), and a fold of the
// high half by x^7 + x^2 + x + 1.
#include <algorithm>
#include <vector>

#include "gf2x_common.cuh"

namespace gf2x {
namespace {

// Launch-shape constants; each can be overridden at compile time (-D) to
// measure alternatives.
#ifndef GF2X_M128_BOTTOM
#define GF2X_M128_BOTTOM 10
#endif
#ifndef GF2X_M128_TABLE_MIN
#define GF2X_M128_TABLE_MIN 5
#endif
#ifndef GF2X_M128_TOP
#define GF2X_M128_TOP 3
#endif
constexpr u64 kMod128Low = 0x87;      // x^7 + x^2 + x + 1
constexpr int kBottom128 = GF2X_M128_BOTTOM;       // deepest bottom tile: 2^10 points (16 KiB per transform)
// Bottom layers >= 5 multiply through tables, lower ones with the integer
// product: a 128-bit table costs ~4600 instructions to build and layer 4 uses
// each one 48 times (measured on GB300: threshold 5 is 3% faster than 4 at
// 2^24 and 2^30-bit operands, 3 is 10% slower).
constexpr int kTableMin128 = GF2X_M128_TABLE_MIN;
constexpr int kTopLayers128 = GF2X_M128_TOP;       // layers per top pass (<= 4)
constexpr int kThreads128 = 256;
constexpr int kTab128 = 1024;         // u64 words per multiplication table (8 KiB)
// Tables built at a time in the bottom tile: 4 (64 KiB of shared memory, 3
// blocks per SM) or 8 (96 KiB, 2 blocks per SM, fewer barriers); the tuner
// measures both per launch shape (4 won at 2^30-bit operands, 8 at 2^24).
constexpr int kChunkSmall128 = 4, kChunkLarge128 = 8;
constexpr int kCols128 = 16;          // word columns per Encode/Decode block
constexpr int kPad128 = kCols128 + 1;
constexpr int kLinWords = 16 * 256 * 2;  // words of a 128-bit byte-window table

struct g128 {
    u64 lo, hi;
};

__device__ __forceinline__ g128 gx(g128 a, g128 b) { return {a.lo ^ b.lo, a.hi ^ b.hi}; }
__device__ __forceinline__ g128 ld128(const u64 *p)
{
    const ulonglong2 v = *(const ulonglong2 *)p;
    return {v.x, v.y};
}
__device__ __forceinline__ void st128(u64 *p, g128 v) { *(ulonglong2 *)p = make_ulonglong2(v.lo, v.hi); }

// ------------------------------------------------------------ field arithmetic
// 64 x 64 -> 128-bit carry-less product (Karatsuba over the 32-bit halves).
__device__ __forceinline__ void clmul64(u64 a, u64 b, u64 &lo, u64 &hi)
{
    const u32 al = (u32)a, ah = (u32)(a >> 32), bl = (u32)b, bh = (u32)(b >> 32);
    const u64 l = clmul32_h4(al, bl), h = clmul32_h4(ah, bh);
    const u64 m = clmul32_h4(al ^ ah, bl ^ bh) ^ l ^ h;
    lo = l ^ (m << 32);
    hi = h ^ (m >> 32);
}

// r3 r2 r1 r0 (a 256-bit polynomial, r0 lowest) modulo x^128 + x^7 + x^2 + x + 1:
// H = r3 r2 is folded once as H (x^7 + x^2 + x + 1); the at most 7 bits that
// fold pushes past x^127 are folded again.
__device__ __forceinline__ g128 gf128_reduce(u64 r0, u64 r1, u64 r2, u64 r3)
{
    const u64 over = (r3 >> 63) ^ (r3 >> 62) ^ (r3 >> 57);
    u64 t0 = r2 ^ (r2 << 1) ^ (r2 << 2) ^ (r2 << 7);
    const u64 t1 = r3 ^ (r3 << 1) ^ (r3 << 2) ^ (r3 << 7) ^ (r2 >> 63) ^ (r2 >> 62) ^ (r2 >> 57);
    t0 ^= over ^ (over << 1) ^ (over << 2) ^ (over << 7);
    return {r0 ^ t0, r1 ^ t1};
}

__device__ __forceinline__ g128 gf128_mul(g128 a, g128 b)
{
    u64 p0, p1, q0, q1, m0, m1;
    clmul64(a.lo, b.lo, p0, p1);
    clmul64(a.hi, b.hi, q0, q1);
    clmul64(a.lo ^ a.hi, b.lo ^ b.hi, m0, m1);
    m0 ^= p0 ^ q0;
    m1 ^= p1 ^ q1;
    return gf128_reduce(p0, p1 ^ m0, q0 ^ m1, q1);
}

__device__ __forceinline__ g128 mul_x128(g128 p)
{
    return {(p.lo << 1) ^ ((p.hi >> 63) * kMod128Low), (p.hi << 1) | (p.lo >> 63)};
}

// c x^e reduced, 0 <= e < 128.
__device__ __forceinline__ g128 mul_xpow128(g128 c, int e)
{
    if (e == 0) return c;
    if (e < 64) return gf128_reduce(c.lo << e, (c.hi << e) | (c.lo >> (64 - e)), c.hi >> (64 - e), 0);
    if (e == 64) return gf128_reduce(0, c.lo, c.hi, 0);
    const int f = e - 64;
    return gf128_reduce(0, c.lo << f, (c.hi << f) | (c.lo >> (64 - f)), c.hi >> (64 - f));
}

// 128-bit GF(2)-linear map as 16 byte-window tables (entry (k, v) = image of
// v << 8k, two words): 8 windows on lo, then 8 on hi (Sec. 4.5, 8-bit windows).
__device__ __forceinline__ g128 lin128(const u64 *__restrict__ t, u64 lo, u64 hi)
{
    g128 r = {0, 0};
#pragma unroll
    for (int k = 0; k < 8; ++k) r = gx(r, ld128(t + 2 * (k * 256 + ((lo >> (8 * k)) & 255))));
#pragma unroll
    for (int k = 0; k < 8; ++k) r = gx(r, ld128(t + 2 * ((8 + k) * 256 + ((hi >> (8 * k)) & 255))));
    return r;
}

// Element with Cantor coordinates u < 2^64 (window tables of the context).
__device__ __forceinline__ g128 cantor128(const u64 *__restrict__ cvt, u64 u)
{
    g128 r = {0, 0};
    for (int k = 0; u; ++k, u >>= 8) r = gx(r, ld128(cvt + 2 * (k * 256 + (u & 255))));
    return r;
}

// ------------------------------------------------------- twiddle tables
__device__ __forceinline__ unsigned smem_addr128(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ u64 *align128(u64 *p) { return (u64 *)(((uintptr_t)p + 127) & ~(uintptr_t)127); }

// Window W of the table at shared address `tab` (128-byte aligned): its low
// words at tab + 256 W, its high words 128 bytes further, entry e of either at
// slot e ^ (W mod 16).  s0..s3 are the 32-bit quarters of x with every nibble
// already XORed with its index mod 16 (one XOR per quarter), so the slot's
// byte offset is one shift and one mask of the quarter, ORed into tab.
template <int W>
__device__ __forceinline__ void tab_window128(u64 &rl, u64 &rh, unsigned tab, unsigned s0, unsigned s1, unsigned s2,
                                              unsigned s3)
{
    constexpr int k = 4 * (W & 7);
    const unsigned src = (W >> 3) == 0 ? s0 : (W >> 3) == 1 ? s1 : (W >> 3) == 2 ? s2 : s3;
    const unsigned a = ((k >= 3 ? src >> (k - 3) : src << (3 - k)) & 0x78u) | tab;
    u64 vl, vh;
    asm volatile("ld.shared.u64 %0, [%1+%2];" : "=l"(vl) : "r"(a), "n"(W * 256));
    asm volatile("ld.shared.u64 %0, [%1+%2];" : "=l"(vh) : "r"(a), "n"(W * 256 + 128));
    rl ^= vl;
    rh ^= vh;
    if constexpr (W < 31) tab_window128<W + 1>(rl, rh, tab, s0, s1, s2, s3);
}

__device__ __forceinline__ g128 mul_tab128(unsigned tab, g128 x)
{
    u64 rl = 0, rh = 0;
    tab_window128<0>(rl, rh, tab, (unsigned)x.lo ^ 0x76543210u, (unsigned)(x.lo >> 32) ^ 0xFEDCBA98u,
                     (unsigned)x.hi ^ 0x76543210u, (unsigned)(x.hi >> 32) ^ 0xFEDCBA98u);
    return {rl, rh};
}

// Build nt tables: thread (t, w) computes c x^(4w+b), b < 4, for the twiddle
// c = twid(t) and writes the 16 entries of window w (Gray-code XORs).  Ends
// with __syncthreads().
template <class F>
__device__ __forceinline__ void build_tables128(u64 *tabs, int nt, F twid)
{
    for (int k = threadIdx.x; k < nt * 32; k += blockDim.x) {
        const int t = k >> 5, w = k & 31, sw = w & 15;
        const g128 c = twid(t);
        g128 p[4];
        p[0] = mul_xpow128(c, 4 * w);
        p[1] = mul_x128(p[0]);
        p[2] = mul_x128(p[1]);
        p[3] = mul_x128(p[2]);
        u64 *dst = tabs + (size_t)t * kTab128 + w * 32;
        g128 e = {0, 0};
        dst[sw] = 0;
        dst[16 + sw] = 0;
#pragma unroll
        for (int g = 1; g < 16; ++g) {            // Gray code: flip the lowest set bit of g
            e = gx(e, p[(g & 1) ? 0 : (g & 2) ? 1 : (g & 4) ? 2 : 3]);
            const int slot = (g ^ (g >> 1)) ^ sw;
            dst[slot] = e.lo;
            dst[16 + slot] = e.hi;
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------- Encode
// n_p = 2^l >= 64.  Row j (< 128) of the novelpoly bit array is bits
// [j n_p, (j+1) n_p), RW = n_p/64 words.  For the 64 points of word column w,
// rows 0..63 and rows 64..127 give two 64x64 bit matrices; their transposes
// give, per point i, the low and high halves of (a_{j n_p + i})_j, and
// f_i = that vector times R (Alg. 4).  Rows at or above `rows` are zero.
__global__ void __launch_bounds__(256) k128_encode(const u64 *__restrict__ novel, u64 rw, int rows,
                                                   const u64 *__restrict__ enc, u64 *__restrict__ f, u64 groups,
                                                   u64 stride, u64 out_stride)
{
    novel += (u64)blockIdx.y * stride;
    f += (u64)blockIdx.y * out_stride;
    extern __shared__ __align__(16) u64 sm128[];
    u64 *tab = sm128;
    u64 *tile = sm128 + kLinWords;
    const int cols = rw < kCols128 ? (int)rw : kCols128;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 2 * threadIdx.x; k < kLinWords; k += 2 * blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr128(tab + k)), "l"(enc + k)
                     : "memory");
    for (u64 g = blockIdx.x; g < groups; g += gridDim.x) {
        const u64 w0 = g * cols;
        __syncthreads();
        for (int k = threadIdx.x; k < 128 * cols; k += blockDim.x) {
            const int j = k / cols, w = k % cols;
            tile[j * kPad128 + w] = j < rows ? novel[(u64)j * rw + w0 + w] : 0;
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
        for (int w = warp; w < cols; w += blockDim.x >> 5) {
            u64 A = tile[lane * kPad128 + w], B = tile[(lane + 32) * kPad128 + w];
            u64 C = tile[(lane + 64) * kPad128 + w], D = tile[(lane + 96) * kPad128 + w];
            transpose64(A, B, lane);
            transpose64(C, D, lane);
            const u64 base = (w0 + w) * 64;
            st128(f + 2 * (base + lane), lin128(tab, A, C));
            st128(f + 2 * (base + lane + 32), lin128(tab, B, D));
        }
    }
}

// n_p < 64: bit by bit.  Bits at or above nonzero_bits are zero and are not read.
__global__ void k128_encode_small(const u64 *__restrict__ novel, int l, u64 nonzero_bits, const u64 *__restrict__ enc,
                                  u64 *__restrict__ f, u64 stride, u64 out_stride)
{
    novel += (u64)blockIdx.y * stride;
    f += (u64)blockIdx.y * out_stride;
    const u64 np = 1ull << l;
    for (u64 i = threadIdx.x; i < np; i += blockDim.x) {
        u64 lo = 0, hi = 0;
        for (int j = 0; j < 128; ++j) {
            const u64 pos = (u64)j * np + i;
            if (pos < nonzero_bits) {
                const u64 bit = (novel[pos >> 6] >> (pos & 63)) & 1ull;
                if (j < 64) lo |= bit << j;
                else hi |= bit << (j - 64);
            }
        }
        st128(f + 2 * i, lin128(enc, lo, hi));
    }
}

// ------------------------------------------------------------------- Decode
// Per point, the 128 bits (c_{j n_p + i})_j = h_i R^{-1}; a warp transposes
// the low and high halves of one word column's 64 vectors back into rows.
__global__ void __launch_bounds__(256) k128_decode(const u64 *__restrict__ h, u64 rw, const u64 *__restrict__ dec,
                                                   u64 *__restrict__ novel, u64 groups, u64 stride)
{
    h += (u64)blockIdx.y * stride;
    novel += (u64)blockIdx.y * stride;
    extern __shared__ __align__(16) u64 sm128[];
    u64 *tab = sm128;
    u64 *tile = sm128 + kLinWords;
    const int cols = rw < kCols128 ? (int)rw : kCols128;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 2 * threadIdx.x; k < kLinWords; k += 2 * blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr128(tab + k)), "l"(dec + k)
                     : "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    for (u64 g = blockIdx.x; g < groups; g += gridDim.x) {
        const u64 w0 = g * cols;
        for (int w = warp; w < cols; w += blockDim.x >> 5) {
            const u64 base = (w0 + w) * 64;
            const g128 hA = ld128(h + 2 * (base + lane)), hB = ld128(h + 2 * (base + lane + 32));
            const g128 vA = lin128(tab, hA.lo, hA.hi), vB = lin128(tab, hB.lo, hB.hi);
            u64 A = vA.lo, B = vB.lo, C = vA.hi, D = vB.hi;
            transpose64(A, B, lane);
            transpose64(C, D, lane);
            tile[lane * kPad128 + w] = A;
            tile[(lane + 32) * kPad128 + w] = B;
            tile[(lane + 64) * kPad128 + w] = C;
            tile[(lane + 96) * kPad128 + w] = D;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < 128 * cols; k += blockDim.x) {
            const int j = k / cols, w = k % cols;
            novel[(u64)j * rw + w0 + w] = tile[j * kPad128 + w];
        }
        __syncthreads();
    }
}

__global__ void k128_decode_small(const u64 *__restrict__ h, int l, const u64 *__restrict__ dec, u64 *__restrict__ novel,
                                  u64 stride)
{
    h += (u64)blockIdx.y * stride;
    novel += (u64)blockIdx.y * stride;
    __shared__ g128 vec[32];
    const u64 np = 1ull << l;
    for (u64 i = threadIdx.x; i < np; i += blockDim.x) {
        const g128 x = ld128(h + 2 * i);
        vec[i] = lin128(dec, x.lo, x.hi);
    }
    __syncthreads();
    for (u64 wd = threadIdx.x; wd < 2 * np; wd += blockDim.x) {   // n/64 = 2 n_p words
        u64 out = 0;
        for (int b = 0; b < 64; ++b) {
            const u64 pos = wd * 64 + b;
            const u64 j = pos >> l, i = pos & (np - 1);
            const u64 word = j < 64 ? vec[i].lo : vec[i].hi;
            out |= ((word >> (j & 63)) & 1ull) << b;
        }
        novel[wd] = out;
    }
}

__global__ void k128_pointwise(const u64 *__restrict__ a, const u64 *__restrict__ b, u64 *c, u64 count)
{
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) st128(c + 2 * t, gf128_mul(ld128(a + 2 * t), ld128(b + 2 * t)));
}

// ------------------------------------------------------------------ top pass
// Layers [p, p+M) of one or two transforms (blockIdx.y = job * arrays + array).
// Layer i multiplies the block starting at s = blk 2^(i+1) by
// s_i(alpha + u_s) = v_{l+64-i} + (element with Cantor coordinates 2 blk)
// (Eq. 4: s_i shifts Cantor coordinates right by i).  The 2^M points that
// differ in bits [p, p+M) form one column, kept in registers; every column of
// one group (same bits >= p+M) shares the pass's 2^M - 1 twiddles, whose tables
// the block builds once.  Layer p + r has 2^(M-1-r) tables from table
// 2^(M-1-r) - 1 on; table j of it serves rows u with u >> (r+1) = j.
template <int M, bool INV>
__global__ void __launch_bounds__(kThreads128) k128_bfly_top(u64 *x0, u64 *x1, int l, int p, u64 chunks, int per_block,
                                                             const u64 *__restrict__ cvt, const u64 *__restrict__ vb,
                                                             int arrays, u64 stride)
{
    extern __shared__ u64 smem128_raw[];
    u64 *tabs = align128(smem128_raw);
    constexpr int ntab = (1 << M) - 1;
    const u64 job = blockIdx.y / arrays;
    u64 *x = ((blockIdx.y % arrays) ? x1 : x0) + job * stride;
    const u64 first = (u64)blockIdx.x * per_block;
    const u64 group = first / chunks;
    build_tables128(tabs, ntab, [&](int t) {
        const int lvl = 31 - __clz(t + 1);
        const int r = M - 1 - lvl;
        const int j = t - ((1 << lvl) - 1);
        const u64 blk = (group << lvl) | (u64)j;
        return gx(ld128(vb + 2 * (l + 64 - (p + r))), cantor128(cvt, blk << 1));
    });
    const u64 rstride = 1ull << p;
    for (int ch = 0; ch < per_block; ++ch) {
        const u64 chunk = first + ch;
        if (chunk / chunks != group) break;
        const u64 col = (chunk % chunks) * kThreads128 + threadIdx.x;
        const u64 base = (group << (p + M)) + col;
        g128 v[1 << M];
#pragma unroll
        for (int u = 0; u < (1 << M); ++u) v[u] = ld128(x + 2 * (base + (u64)u * rstride));
#pragma unroll
        for (int s2 = 0; s2 < M; ++s2) {
            const int r = INV ? s2 : M - 1 - s2;
            const int half = 1 << r;
            const unsigned tl = smem_addr128(tabs) + (unsigned)(((1 << (M - 1 - r)) - 1) * kTab128 * 8);
#pragma unroll
            for (int u = 0; u < (1 << M); ++u) {
                if (u & half) continue;
                const unsigned tb = tl + (unsigned)((u >> (r + 1)) * kTab128 * 8);
                if (!INV) {
                    v[u] = gx(v[u], mul_tab128(tb, v[u | half]));
                    v[u | half] = gx(v[u | half], v[u]);
                } else {
                    v[u | half] = gx(v[u | half], v[u]);
                    v[u] = gx(v[u], mul_tab128(tb, v[u | half]));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < (1 << M); ++u) st128(x + 2 * (base + (u64)u * rstride), v[u]);
    }
}

// -------------------------------------------------------------- bottom tile
enum Bottom128 { B128_FWD = 0, B128_INV = 1, B128_FUSED = 2 };

// Layer i on a tile in shared memory with the integer product.  ctop =
// v_{l+64-i} + Cantor((tile base) >> i); the block of local index blk adds
// Cantor(2 blk), 2 blk < 2^10 (two byte windows).
__device__ __forceinline__ void tile_layer128(u64 *a, int bt, int i, g128 ctop, const u64 *__restrict__ cvt,
                                              bool inverse)
{
    const int nb = 1 << (bt - 1);
    const int span = 1 << i;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        const int blk = t >> i, j = t & (span - 1);
        const int s0 = (blk << (i + 1)) + j;
        g128 x0 = ld128(a + 2 * s0), x1 = ld128(a + 2 * (s0 + span));
        const unsigned u = (unsigned)blk << 1;
        const g128 c = gx(ctop, gx(ld128(cvt + 2 * (u & 255)), ld128(cvt + 2 * (256 + (u >> 8)))));
        if (!inverse) {
            x0 = gx(x0, gf128_mul(c, x1));
            x1 = gx(x1, x0);
        } else {
            x1 = gx(x1, x0);
            x0 = gx(x0, gf128_mul(c, x1));
        }
        st128(a + 2 * s0, x0);
        st128(a + 2 * (s0 + span), x1);
    }
}

// Butterflies of layer i for the blocks j0 .. j0 + nt - 1 of the tile(s),
// block j's table at slot slot0 + j - j0 of tabs; on a and, if given, b.
__device__ __forceinline__ void table_butterflies128(u64 *a, u64 *b, int i, int j0, int nt, int slot0, const u64 *tabs,
                                                     bool inverse)
{
    const int span = 1 << i;
    for (int t = threadIdx.x; t < (nt << i); t += blockDim.x) {
        const int blk = j0 + (t >> i), jj = t & (span - 1);
        const int s0 = (blk << (i + 1)) + jj;
        const unsigned tb = smem_addr128(tabs) + (unsigned)((slot0 + blk - j0) * kTab128 * 8);
        g128 x0 = ld128(a + 2 * s0), x1 = ld128(a + 2 * (s0 + span));
        if (!inverse) {
            x0 = gx(x0, mul_tab128(tb, x1));
            x1 = gx(x1, x0);
        } else {
            x1 = gx(x1, x0);
            x0 = gx(x0, mul_tab128(tb, x1));
        }
        st128(a + 2 * s0, x0);
        st128(a + 2 * (s0 + span), x1);
        if (b) {
            g128 y0 = ld128(b + 2 * s0), y1 = ld128(b + 2 * (s0 + span));
            y0 = gx(y0, mul_tab128(tb, y1));
            y1 = gx(y1, y0);
            st128(b + 2 * s0, y0);
            st128(b + 2 * (s0 + span), y1);
        }
    }
}

// The table layers bt-1 .. kTableMin128 of a tile in the order of the pass
// (forward top down, inverse bottom up), twiddle tables packed as in the
// m = 64 bottom kernel: the layers i >= bt - log2(CHUNK) have 2^(bt-i) - 1
// tables together (layer i's block j at slot 2^(bt-1-i) - 1 + j), built in
// one round; each lower layer has 2^(bt-1-i) >= CHUNK tables, built CHUNK at
// a time.  The inverse takes the groups in reverse order, so its first group
// is the forward pass's last one: with `kept` those tables are still in tabs.
// ctops[i] = v_{l+64-i} + Cantor((tile base) >> i) (two words); block j of
// layer i adds Cantor(2j), 2j < 2^(bt-i) <= 2^10 (two byte windows).
template <int CHUNK>
__device__ void table_layers128(u64 *a, u64 *b, int bt, const u64 *__restrict__ cvt, const u64 *ctops, u64 *tabs,
                                bool inverse, bool kept)
{
    static_assert(CHUNK == 4 || CHUNK == 8, "chunk of 4 or 8 tables");
    constexpr int kLogChunk = CHUNK == 4 ? 2 : 3;
    if (bt <= kTableMin128) return;
    const int lo_top = bt - kLogChunk > kTableMin128 ? bt - kLogChunk : kTableMin128;
    auto twid = [&](int i, int j) {
        const unsigned j2 = (unsigned)j << 1;
        return gx(ld128(ctops + 2 * i), gx(ld128(cvt + 2 * (j2 & 255)), ld128(cvt + 2 * (256 + (j2 >> 8)))));
    };
    auto packed = [&](bool build) {
        if (build)
            build_tables128(tabs, (1 << (bt - lo_top)) - 1, [&](int t) {
                const int r = 31 - __clz(t + 1);            // slot t: block t + 1 - 2^r of layer bt-1-r
                return twid(bt - 1 - r, t + 1 - (1 << r));
            });
        for (int k = 0; k < bt - lo_top; ++k) {
            const int i = inverse ? lo_top + k : bt - 1 - k;
            table_butterflies128(a, b, i, 0, 1 << (bt - 1 - i), (1 << (bt - 1 - i)) - 1, tabs, inverse);
            __syncthreads();
        }
    };
    auto chunked = [&](int i, bool first_kept) {
        const int nc = (1 << (bt - 1 - i)) / CHUNK;
        for (int c = 0; c < nc; ++c) {
            const int j0 = (inverse ? nc - 1 - c : c) * CHUNK;
            if (!(first_kept && c == 0)) build_tables128(tabs, CHUNK, [&](int t) { return twid(i, j0 + t); });
            table_butterflies128(a, b, i, j0, CHUNK, 0, tabs, inverse);
            __syncthreads();
        }
    };
    if (!inverse) {
        packed(true);
        for (int i = lo_top - 1; i >= kTableMin128; --i) chunked(i, false);
    } else {
        for (int i = kTableMin128; i < lo_top; ++i) chunked(i, kept && i == kTableMin128);
        packed(!(kept && lo_top == kTableMin128));
    }
}

// Words of one tile in shared memory, rounded up so the tables that follow
// start 128-byte aligned.
__host__ __device__ __forceinline__ int tile_words128(int bt) { return (2 << bt) < 16 ? 16 : (2 << bt); }

// One tile of 2^bt points per block: the low layers of the forward transform
// (of X, and of Y in the fused mode), then in the fused mode the pointwise
// product X * Y (pointwise step of Alg. 5), then the low layers of the inverse.
template <int CHUNK>
__global__ void __launch_bounds__(kThreads128) k128_bfly_bottom(u64 *X, const u64 *Y, int l, int bt,
                                                                const u64 *__restrict__ cvt, const u64 *__restrict__ vb,
                                                                int mode, u64 stride)
{
    extern __shared__ u64 smem128_raw[];
    u64 *sm = align128(smem128_raw);
    X += (u64)blockIdx.y * stride;
    if (Y) Y += (u64)blockIdx.y * stride;
    const int T = 1 << bt;
    const bool fused = mode == B128_FUSED;
    u64 *a = sm;
    u64 *b = fused ? sm + tile_words128(bt) : nullptr;
    u64 *tabs = sm + (fused ? 2 : 1) * tile_words128(bt);
    const u64 base = (u64)blockIdx.x << bt;
    for (int k = threadIdx.x; k < T; k += blockDim.x) {
        st128(a + 2 * k, ld128(X + 2 * (base + k)));
        if (fused) st128(b + 2 * k, ld128(Y + 2 * (base + k)));
    }
    u64 *ctops = tabs + CHUNK * kTab128;                // v_{l+64-i} + Cantor(base >> i), i < bt
    if (threadIdx.x < bt)
        st128(ctops + 2 * threadIdx.x, gx(ld128(vb + 2 * (l + 64 - threadIdx.x)), cantor128(cvt, base >> threadIdx.x)));
    __syncthreads();
    const int low = bt < kTableMin128 ? bt : kTableMin128;   // layers below `low` multiply in integer form
    if (mode != B128_INV) {
        table_layers128<CHUNK>(a, b, bt, cvt, ctops, tabs, false, false);
        for (int i = low - 1; i >= 0; --i) {
            const g128 ctop = ld128(ctops + 2 * i);
            tile_layer128(a, bt, i, ctop, cvt, false);
            if (fused) tile_layer128(b, bt, i, ctop, cvt, false);
            __syncthreads();
        }
    }
    if (fused) {
        for (int k = threadIdx.x; k < T; k += blockDim.x) st128(a + 2 * k, gf128_mul(ld128(a + 2 * k), ld128(b + 2 * k)));
        __syncthreads();
    }
    if (mode != B128_FWD) {
        for (int i = 0; i < low; ++i) {
            tile_layer128(a, bt, i, ld128(ctops + 2 * i), cvt, true);
            __syncthreads();
        }
        table_layers128<CHUNK>(a, nullptr, bt, cvt, ctops, tabs, true, mode != B128_INV);
    }
    for (int k = threadIdx.x; k < T; k += blockDim.x) st128(X + 2 * (base + k), ld128(a + 2 * k));
}

size_t bottom_smem128(int bt, bool fused, int chunk)
{
    return ((fused ? 2 : 1) * (size_t)tile_words128(bt) + (size_t)chunk * kTab128 + 32) * sizeof(u64) + 128;
}

size_t top_smem128(int m) { return (size_t)((1 << m) - 1) * kTab128 * sizeof(u64) + 128; }

constexpr size_t kLinSmem = (size_t)(kLinWords + 128 * kPad128) * sizeof(u64);

bool configured128 = false;

void configure128()
{
    if (configured128) return;
    cudaFuncSetAttribute(k128_bfly_bottom<kChunkSmall128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bottom_smem128(kBottom128, true, kChunkSmall128));
    cudaFuncSetAttribute(k128_bfly_bottom<kChunkLarge128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bottom_smem128(kBottom128, true, kChunkLarge128));
    cudaFuncSetAttribute(k128_bfly_top<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)top_smem128(3));
    cudaFuncSetAttribute(k128_bfly_top<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)top_smem128(3));
    cudaFuncSetAttribute(k128_bfly_top<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)top_smem128(4));
    cudaFuncSetAttribute(k128_bfly_top<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)top_smem128(4));
    cudaFuncSetAttribute(k128_encode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLinSmem);
    cudaFuncSetAttribute(k128_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLinSmem);
    configured128 = true;
}

template <int M, bool INV>
void launch_top128(dim3 grid, cudaStream_t st, u64 *x0, u64 *x1, int l, int p, u64 chunks, int per_block,
                   const u64 *cvt, const u64 *vb, int arrays, u64 stride)
{
    k128_bfly_top<M, INV><<<grid, kThreads128, top_smem128(M), st>>>(x0, x1, l, p, chunks, per_block, cvt, vb, arrays,
                                                                      stride);
}

// Passes over layers [bt, l), as few as kTopLayers128 allows, the layers split
// evenly (lower passes take one more where they do not divide), high to low
// for the forward transform.  p >= bt >= 8, so a group has >= 256 columns, a
// multiple of the block size.
cudaError_t top_passes128(gf2x_ctx *ctx, u64 *x0, u64 *x1, int l, int bt, bool inverse, int count, u64 stride,
                          cudaStream_t st)
{
    const int layers = l - bt;
    const int npass = (layers + kTopLayers128 - 1) / kTopLayers128;
    const int per = npass ? layers / npass : 0, rem = npass ? layers % npass : 0;
    for (int k = 0; k < npass; ++k) {
        const int idx = inverse ? k : npass - 1 - k;
        const int p = bt + idx * per + (idx < rem ? idx : rem);
        const int m = per + (idx < rem ? 1 : 0);
        const u64 chunks = (1ull << p) / kThreads128;
        const u64 groups = (1ull << l) >> (p + m);
        const int arrays = x1 ? 2 : 1;
        const u64 pb = chunks * groups * (u64)arrays * (u64)count / (2 * (u64)ctx->num_sms);
        int per_block = 1;
        while (per_block < 8 && (u64)(2 * per_block) <= pb && (u64)(2 * per_block) <= chunks) per_block *= 2;
        const dim3 grid((unsigned)(chunks * groups / per_block), (unsigned)(arrays * count));
        const u64 *cvt = ctx->d_cvt128, *vb = ctx->d_cantor128;
        switch (m * 2 + (inverse ? 1 : 0)) {
        case 2: launch_top128<1, false>(grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 3: launch_top128<1, true>(grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 4: launch_top128<2, false>(grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 5: launch_top128<2, true>(grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 6: launch_top128<3, false>(grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 7: launch_top128<3, true>(grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        case 8: launch_top128<4, false>(grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        default: launch_top128<4, true>(grid, st, x0, x1, l, p, chunks, per_block, cvt, vb, arrays, stride); break;
        }
        count_launch(ctx);
    }
    return cudaGetLastError();
}

cudaError_t launch_bottom128_chunk(gf2x_ctx *ctx, u64 *X, const u64 *Y, int l, int bt, int mode, int count,
                                   u64 stride, int chunk, cudaStream_t st)
{
    const dim3 grid((unsigned)(1ull << (l - bt)), count);
    const size_t smem = bottom_smem128(bt, mode == B128_FUSED, chunk);
    if (chunk == kChunkLarge128)
        k128_bfly_bottom<kChunkLarge128><<<grid, kThreads128, smem, st>>>(X, Y, l, bt, ctx->d_cvt128,
                                                                           ctx->d_cantor128, mode, stride);
    else
        k128_bfly_bottom<kChunkSmall128><<<grid, kThreads128, smem, st>>>(X, Y, l, bt, ctx->d_cvt128,
                                                                           ctx->d_cantor128, mode, stride);
    count_launch(ctx);
    return cudaGetLastError();
}

// The chunk measured by the tuner on `scratch` (a free buffer laid out like X;
// Y is only read), or the default without one.
cudaError_t launch_bottom128(gf2x_ctx *ctx, u64 *X, const u64 *Y, int l, int bt, int mode, int count, u64 stride,
                             u64 *scratch, cudaStream_t st)
{
    const u64 tiles = (1ull << (l - bt)) * (u64)count;
    int chunk = tiles > 2 * (u64)ctx->num_sms ? kChunkSmall128 : kChunkLarge128;
    static const int cands[2] = {kChunkLarge128, kChunkSmall128};
    if (!scratch) chunk = tune_pinned(ctx, TUNE_M128_BOTTOM_CHUNK, cands, 2, chunk);
    else {
        chunk = tune_choice(ctx, TUNE_M128_BOTTOM_CHUNK, (tune_bucket(tiles) << 2) | (u64)mode, cands, 2, chunk,
                            [&](int ch) {
                                return launch_bottom128_chunk(ctx, scratch, Y, l, bt, mode, count, stride, ch, st);
                            },
                            st);
    }
    return launch_bottom128_chunk(ctx, X, Y, l, bt, mode, count, stride, chunk, st);
}

// ------------------------------------------------------------ host set-up
typedef unsigned __int128 h128;

h128 hmul128(h128 a, h128 b)
{
    h128 r = 0;
    for (int t = 0; t < 128; ++t) {
        if ((b >> t) & 1) r ^= a;
        const bool top = (a >> 127) & 1;
        a <<= 1;
        if (top) a ^= (h128)kMod128Low;
    }
    return r;
}

// One solution of sum_k y_k img[k] = rhs over GF(2), or false.
bool solve128(const h128 img[128], h128 rhs, h128 *y)
{
    std::vector<h128> eq(128);
    std::vector<int> rb(128), piv_col(128);
    for (int p = 0; p < 128; ++p) {
        h128 m = 0;
        for (int k = 0; k < 128; ++k) m |= ((img[k] >> p) & 1) << k;
        eq[p] = m;
        rb[p] = (int)((rhs >> p) & 1);
    }
    int rank = 0;
    for (int col = 0; col < 128 && rank < 128; ++col) {
        int piv = -1;
        for (int r = rank; r < 128; ++r)
            if ((eq[r] >> col) & 1) { piv = r; break; }
        if (piv < 0) continue;
        std::swap(eq[rank], eq[piv]);
        std::swap(rb[rank], rb[piv]);
        for (int r = 0; r < 128; ++r)
            if (r != rank && ((eq[r] >> col) & 1)) { eq[r] ^= eq[rank]; rb[r] ^= rb[rank]; }
        piv_col[rank++] = col;
    }
    for (int r = rank; r < 128; ++r)
        if (rb[r]) return false;
    h128 s = 0;
    for (int r = 0; r < rank; ++r)
        if (rb[r]) s |= (h128)1 << piv_col[r];
    *y = s;
    return true;
}

// Rows of A^{-1} (row-vector convention), or false if A is singular.
bool inverse128(const h128 a_in[128], h128 inv[128])
{
    std::vector<h128> a(a_in, a_in + 128);
    for (int k = 0; k < 128; ++k) inv[k] = (h128)1 << k;
    for (int col = 0; col < 128; ++col) {
        int piv = -1;
        for (int r = col; r < 128; ++r)
            if ((a[r] >> col) & 1) { piv = r; break; }
        if (piv < 0) return false;
        std::swap(a[col], a[piv]);
        std::swap(inv[col], inv[piv]);
        for (int r = 0; r < 128; ++r)
            if (r != col && ((a[r] >> col) & 1)) { a[r] ^= a[col]; inv[r] ^= inv[col]; }
    }
    return true;
}

// nwin byte-window tables of the map whose row k is rows[k]: entry (k, x) at
// words 2 (256 k + x) and 2 (256 k + x) + 1.
void window_table128(const h128 *rows, int nwin, u64 *out)
{
    for (int k = 0; k < nwin; ++k)
        for (int x = 0; x < 256; ++x) {
            h128 r = 0;
            for (int b = 0; b < 8; ++b)
                if ((x >> b) & 1) r ^= rows[8 * k + b];
            out[2 * (256 * k + x)] = (u64)r;
            out[2 * (256 * k + x) + 1] = (u64)(r >> 64);
        }
}

inline unsigned blocks_for128(u64 n, unsigned threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// Cantor basis of GF(2^128) (Eq. 2: v_0 = 1, v_i^2 + v_i = v_{i-1}, the root
// with bit 0 clear), Encode matrix R with rows r_j = prod_{t < 7, bit t of j}
// v_{64-t} (layer l + t of the truncated Butterfly multiplies by
// s_{l+t}(v_{l+64}) = v_{64-t}, Eq. 4), its inverse (Prop. 2), and the window
// tables: Cantor -> polynomial (8 windows), R (16), R^{-1} (16), then v_0..v_127.
bool m128_build_tables(u64 *host)
{
    h128 img[128], v[128], r[128], rinv[128];
    for (int k = 0; k < 128; ++k) {
        const h128 e = (h128)1 << k;
        img[k] = hmul128(e, e) ^ e;
    }
    v[0] = 1;
    for (int i = 1; i < 128; ++i) {
        h128 y;
        if (!solve128(img, v[i - 1], &y)) return false;
        v[i] = y & ~(h128)1;
    }
    for (int j = 0; j < 128; ++j) {
        h128 p = 1;
        for (int t = 0; t < 7; ++t)
            if ((j >> t) & 1) p = hmul128(p, v[64 - t]);
        r[j] = p;
    }
    if (!inverse128(r, rinv)) return false;
    window_table128(v, 8, host);
    window_table128(r, 16, host + 4096);
    window_table128(rinv, 16, host + 4096 + 8192);
    for (int i = 0; i < 128; ++i) {
        host[4096 + 2 * 8192 + 2 * i] = (u64)v[i];
        host[4096 + 2 * 8192 + 2 * i + 1] = (u64)(v[i] >> 64);
    }
    return true;
}

cudaError_t m128_encode(gf2x_ctx *ctx, const u64 *novel, int l, u64 *f, u64 nonzero_bits, int count, u64 stride,
                        u64 out_stride, cudaStream_t st)
{
    configure128();
    if (l < 6) {
        k128_encode_small<<<dim3(1, count), 64, 0, st>>>(novel, l, nonzero_bits, ctx->d_enc128, f, stride, out_stride);
    } else {
        const u64 rw = 1ull << (l - 6), np = 1ull << l;
        const u64 cols = rw < kCols128 ? rw : kCols128, groups = rw / cols;
        int rows = (int)((nonzero_bits + np - 1) / np);
        if (rows > 128) rows = 128;
        const u64 grid = groups < 2 * (u64)ctx->num_sms ? groups : 2 * (u64)ctx->num_sms;
        k128_encode<<<dim3((unsigned)grid, count), 256, kLinSmem, st>>>(novel, rw, rows, ctx->d_enc128, f, groups,
                                                                        stride, out_stride);
    }
    count_launch(ctx);
    return cudaGetLastError();
}

cudaError_t m128_decode(gf2x_ctx *ctx, const u64 *h, int l, u64 *novel, int count, u64 stride, cudaStream_t st)
{
    configure128();
    if (l < 6) {
        k128_decode_small<<<dim3(1, count), 64, 0, st>>>(h, l, ctx->d_dec128, novel, stride);
    } else {
        const u64 rw = 1ull << (l - 6);
        const u64 cols = rw < kCols128 ? rw : kCols128, groups = rw / cols;
        const u64 grid = groups < 2 * (u64)ctx->num_sms ? groups : 2 * (u64)ctx->num_sms;
        k128_decode<<<dim3((unsigned)grid, count), 256, kLinSmem, st>>>(h, rw, ctx->d_dec128, novel, groups, stride);
    }
    count_launch(ctx);
    return cudaGetLastError();
}

// Bottom-tile depth: measured per (l, count) by m128_butterfly_depth, else 9
// up to l = 20 and kBottom128 above (measured on GB300: 9 is fastest at
// 2^24-bit operands, 10 at 2^30).
constexpr int kMinDepth128 = 8;

static int default_depth128(int l)
{
    const int bt = l <= 20 ? 9 : kBottom128;
    return l < bt ? l : bt;
}

static int depth_or_default128(int bt, int l)   // bt < 0: the default depth
{
    if (bt < 0) return default_depth128(l);
    return l < bt ? l : bt;
}

// A depth pinned by gf2x_tune_pin if it is one of the candidates for l (8 ..
// min(kBottom128, l)), else fallback.
static int pinned_depth128(gf2x_ctx *ctx, int l, int fallback)
{
    int cands[kBottom128];
    int nc = 0;
    for (int b = kMinDepth128; b <= kBottom128 && b <= l; ++b) cands[nc++] = b;
    return tune_pinned(ctx, TUNE_M128_BFLY_DEPTH, cands, nc, fallback);
}

int m128_butterfly_depth_stored(gf2x_ctx *ctx, int l, int count)
{
    if (l <= kMinDepth128) return l;
    return pinned_depth128(
        ctx, l, tune_stored(ctx, TUNE_M128_BFLY_DEPTH, ((u64)l << 32) | tune_bucket((u64)count), default_depth128(l)));
}

// The whole schedule (top passes of both forward transforms, fused bottom
// kernel, top passes of the inverse) timed per depth on the free X and Y, the
// bottom kernel's table chunk tuned per depth on T (in the untimed first run).
int m128_butterfly_depth(gf2x_ctx *ctx, u64 *X, u64 *Y, u64 *T, int l, int count, u64 stride, cudaStream_t st)
{
    configure128();
    if (l <= kMinDepth128) return l;
    int cands[kBottom128];
    int nc = 0;
    for (int b = kMinDepth128; b <= kBottom128 && b <= l; ++b) cands[nc++] = b;
    return tune_choice(ctx, TUNE_M128_BFLY_DEPTH, ((u64)l << 32) | tune_bucket((u64)count), cands, nc, default_depth128(l),
                       [&](int bt) -> cudaError_t {
                           cudaError_t e = top_passes128(ctx, X, Y, l, bt, false, count, stride, st);
                           if (e != cudaSuccess) return e;
                           e = launch_bottom128(ctx, X, Y, l, bt, B128_FUSED, count, stride, T, st);
                           if (e != cudaSuccess) return e;
                           return top_passes128(ctx, X, nullptr, l, bt, true, count, stride, st);
                       },
                       st);
}

cudaError_t m128_butterfly(gf2x_ctx *ctx, u64 *x, int l, bool inverse, int count, u64 stride, cudaStream_t st)
{
    configure128();
    const int bt = pinned_depth128(ctx, l, default_depth128(l));
    if (!inverse) {
        cudaError_t e = top_passes128(ctx, x, nullptr, l, bt, false, count, stride, st);
        if (e != cudaSuccess) return e;
    }
    if (bt > 0) {
        cudaError_t e =
            launch_bottom128(ctx, x, nullptr, l, bt, inverse ? B128_INV : B128_FWD, count, stride, nullptr, st);
        if (e != cudaSuccess) return e;
    }
    if (inverse) return top_passes128(ctx, x, nullptr, l, bt, true, count, stride, st);
    return cudaGetLastError();
}

cudaError_t m128_butterfly_top_pair(gf2x_ctx *ctx, u64 *x0, u64 *x1, int l, int count, u64 stride, cudaStream_t st,
                                    int bt)
{
    configure128();
    return top_passes128(ctx, x0, x1, l, depth_or_default128(bt, l), false, count, stride, st);
}

cudaError_t m128_butterfly_bottom_fused(gf2x_ctx *ctx, u64 *X, const u64 *Y, int l, int count, u64 stride,
                                        cudaStream_t st, u64 *scratch, int bt)
{
    configure128();
    return launch_bottom128(ctx, X, Y, l, depth_or_default128(bt, l), B128_FUSED, count, stride, scratch, st);
}

cudaError_t m128_butterfly_top_inverse(gf2x_ctx *ctx, u64 *x, int l, int count, u64 stride, cudaStream_t st, int bt)
{
    configure128();
    return top_passes128(ctx, x, nullptr, l, depth_or_default128(bt, l), true, count, stride, st);
}

cudaError_t m128_pointwise(gf2x_ctx *ctx, const u64 *a, const u64 *b, u64 *c, u64 count, cudaStream_t st)
{
    if (count) {
        k128_pointwise<<<blocks_for128(count, 256), 256, 0, st>>>(a, b, c, count);
        count_launch(ctx);
    }
    return cudaGetLastError();
}

}  // namespace gf2x
