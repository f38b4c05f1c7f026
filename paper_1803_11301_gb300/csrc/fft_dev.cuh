// Encode / Decode (Alg. 4) and the batch load/store of the operand bit
// arrays: the block bodies of fft.cu's kernels, shared with the persistent
// batch kernel (persist.cu).  Each body runs as one block described by a VBlock.
#pragma once

#include "gf2x_common.cuh"
#include "gf2x_tables.cuh"

// Data written by earlier work of the same launch must not be read through the
// non-coherent read-only path: the persistent kernel defines this empty.
#ifndef GF2X_DATA_RESTRICT
#define GF2X_DATA_RESTRICT __restrict__
#endif

namespace gf2x {
namespace fftk {

constexpr int kCols = 32;            // word columns per Encode/Decode block

// R (or R^{-1}) in eight-bit windows: 8 windows of 256 words, 16 KiB.
constexpr int kCodecTabWords = 8 * 256;

// R^{-1} in four-bit windows (mul_tab layout): 16 windows of 16 words, 2 KiB.
constexpr int kDecodeTabWords = 256;

// Copy a window table of `words` words (16-byte aligned: it sits in the
// context's cudaMalloc'd table block) to shared memory with asynchronous
// 16-byte copies; the caller waits (cp.async.wait_all) and synchronises.
__device__ __forceinline__ void load_table_async(const VBlock &vb, u64 *dst, const u64 *__restrict__ src, int words)
{
    for (int k = 2 * vb.t; k < words; k += 2 * vb.nt)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst + k)),
                     "l"(src + k)
                     : "memory");
}

__device__ __forceinline__ void copy_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// 8-byte copy global -> shared, or zeros when `valid` is false (no bytes read).
__device__ __forceinline__ void copy8_or_zero(u64 *dst_shared, const u64 *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst_shared)),
                 "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}

// x times the matrix whose eight-bit window table sits at shared address tab
// (2 KiB aligned): per window, one shift and one LOP3 form the entry's address
// (its byte offset ORed into the aligned base) and the window's 2 KiB base is
// the load's immediate offset.  Eight lookups per point: they conflict on
// banks, but these kernels are bound by integer instructions, of which the
// four-bit form (16 lookups) takes twice as many.
template <int W>
__device__ __forceinline__ void tab8_window(u64 &r, unsigned tab, unsigned lo, unsigned hi)
{
    constexpr int k = 8 * (W & 3);                      // bit of byte W in its half
    const unsigned src = W < 4 ? lo : hi;
    const unsigned a = ((k >= 3 ? src >> (k - 3) : src << (3 - k)) & 0x7F8u) | tab;
    u64 v;
    asm volatile("ld.shared.u64 %0, [%1+%2];" : "=l"(v) : "r"(a), "n"(W * 2048));
    r ^= v;
    if constexpr (W + 1 < 8) tab8_window<W + 1>(r, tab, lo, hi);
}

__device__ __forceinline__ u64 lin64_w8(unsigned tab, u64 x)
{
    u64 r = 0;
    tab8_window<0>(r, tab, (unsigned)x, (unsigned)(x >> 32));
    return r;
}

__device__ __forceinline__ u64 *align2048(u64 *p) { return (u64 *)(((uintptr_t)p + 2047) & ~(uintptr_t)2047); }

// ------------------------------------------------------------------- Encode
// n_p = 2^l >= 64.  Row j of the novelpoly bit array is bits [j n_p, (j+1) n_p),
// i.e. RW = n_p/64 words.  For the 64 points i in word column w, the 64 words
// (row j, column w) form a 64x64 bit matrix whose transpose gives, per i, the
// vector (a_{j n_p + i})_j; f_i = that vector times R (Alg. 4).
//
// A block stages 64 rows x 32 word columns in shared memory (coalesced row
// reads); each warp transposes one column's 64x64 bit matrix with shuffles
// (Sec. 4.4's block-swap transpose: a 32-bit half swap in registers, then
// five exchange rounds across lanes) and applies R through four-bit window
// tables loaded once per block (lin64_w8).  Rows at or above `rows` are zero
// and are not read.
constexpr int kPad = kCols + 1;      // padded row of the staging tile
// window table (2 KiB aligned within the block's shared memory) + staging tile
constexpr unsigned kCodecSmemWords = 256 + kCodecTabWords + 64 * kPad;

// sm: kCodecSmemWords words of shared memory (8-byte aligned).
__device__ __forceinline__ void encode_body(const VBlock &vb, u64 *sm, const u64 *GF2X_DATA_RESTRICT novel, u64 rw,
                                            int rows, const u64 *__restrict__ enc, u64 *__restrict__ f, u64 groups,
                                            u64 stride, u64 out_stride)
{
    u64 *tab = align2048(sm), *tile = tab + kCodecTabWords;
    const unsigned tabs = smem_addr(tab);
    novel += (u64)vb.by * stride;            // job of a batch
    f += (u64)vb.by * out_stride;
    const int cols = rw < kCols ? (int)rw : kCols;   // a power of two
    const int lc = __ffs(cols) - 1;
    const int lane = vb.t & 31, warp = vb.t >> 5;
    pdl_allow();
    load_table_async(vb, tab, enc, kCodecTabWords);                   // in flight with the first tile's loads
    pdl_wait();
    for (u64 g = vb.bx; g < groups; g += vb.gx) {
        const u64 w0 = g * cols;
        vb.sync();
        for (int k = vb.t; k < 64 * cols; k += vb.nt) {   // every load of the tile in flight at once
            const int j = k >> lc, w = k & (cols - 1);
            const u64 src = (u64)j * rw + w0 + w;
            const bool valid = j < rows && in_range(src, 64 * rw);
            copy8_or_zero(tile + j * kPad + w, valid ? novel + src : novel, valid);
        }
        copy_async_wait();
        vb.sync();
        for (int w = warp; w < cols; w += vb.nt >> 5) {
            u64 A = tile[lane * kPad + w], B = tile[(lane + 32) * kPad + w];
            transpose64(A, B, lane);
            const u64 base = (w0 + w) * 64;
            if (in_range(base + 63, 64 * rw)) {
                f[base + lane] = lin64_w8(tabs, A);
                f[base + lane + 32] = lin64_w8(tabs, B);
            }
        }
    }
}

// n_p < 64: the whole transform is at most 32 words; one block, bit by bit.
// Bits at or above nonzero_bits are zero and are not read.
__device__ __forceinline__ void encode_small_body(const VBlock &vb, const u64 *GF2X_DATA_RESTRICT novel, int l,
                                                  u64 nonzero_bits, const u64 *__restrict__ enc, u64 *__restrict__ f,
                                                  u64 stride, u64 out_stride)
{
    novel += (u64)vb.by * stride;
    f += (u64)vb.by * out_stride;
    const u64 np = 1ull << l;
    for (u64 i = vb.t; i < np; i += vb.nt) {
        u64 u = 0;
        for (int j = 0; j < 64; ++j) {
            u64 pos = (u64)j * np + i;
            if (pos < nonzero_bits) u |= ((novel[pos >> 6] >> (pos & 63)) & 1ull) << j;
        }
        f[i] = lin64(enc, u);
    }
}

// ------------------------------------------------------------------- Decode
// The inverse of Encode: per point, the bits (c_{j n_p + i})_j = h_i R^{-1}
// (four-bit windows through mul_tab: here they measured faster than eight-bit
// ones); a warp transposes the 64 vectors of one word column back into 64 row
// words.
constexpr unsigned kDecodeSmemWords = 16 + kDecodeTabWords + 64 * kPad;

// sm: kDecodeSmemWords words of shared memory (8-byte aligned).
__device__ __forceinline__ void decode_body(const VBlock &vb, u64 *sm, const u64 *GF2X_DATA_RESTRICT h, u64 rw,
                                            const u64 *__restrict__ dec, u64 *__restrict__ novel, u64 groups, u64 stride)
{
    u64 *tab = align128(sm), *tile = tab + kDecodeTabWords;
    const unsigned tabs = smem_addr(tab);
    h += (u64)vb.by * stride;
    novel += (u64)vb.by * stride;
    const int cols = rw < kCols ? (int)rw : kCols;   // a power of two
    const int lc = __ffs(cols) - 1;
    const int lane = vb.t & 31, warp = vb.t >> 5;
    pdl_allow();
    load_table_async(vb, tab, dec, kDecodeTabWords);
    copy_async_wait();
    vb.sync();
    pdl_wait();
    for (u64 g = vb.bx; g < groups; g += vb.gx) {
        const u64 w0 = g * cols;
        const int nw = vb.nt >> 5;
        for (int wb = warp; wb < cols; wb += 4 * nw) {
            // the loads of up to four columns first, then their products and transposes
            u64 A[4], B[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int w = wb + q * nw;
                const u64 base = (w0 + w) * 64;
                const bool ok = w < cols && in_range(base + 63, 64 * rw);
                A[q] = ok ? h[base + lane] : 0;
                B[q] = ok ? h[base + lane + 32] : 0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int w = wb + q * nw;
                if (w >= cols) break;
                u64 a = mul_tab(tabs, A[q]), b = mul_tab(tabs, B[q]);
                transpose64(a, b, lane);
                tile[lane * kPad + w] = a;
                tile[(lane + 32) * kPad + w] = b;
            }
        }
        vb.sync();
        for (int k = vb.t; k < 64 * cols; k += vb.nt) {
            const int j = k >> lc, w = k & (cols - 1);
            const u64 dst = (u64)j * rw + w0 + w;
            if (in_range(dst, 64 * rw)) novel[dst] = tile[j * kPad + w];
        }
        vb.sync();
    }
}

// vec: 64 words of shared memory.
__device__ __forceinline__ void decode_small_body(const VBlock &vb, u64 *vec, const u64 *GF2X_DATA_RESTRICT h, int l,
                                                  const u64 *__restrict__ dec, u64 *__restrict__ novel, u64 stride)
{
    h += (u64)vb.by * stride;
    novel += (u64)vb.by * stride;
    const u64 np = 1ull << l;
    for (u64 i = vb.t; i < np; i += vb.nt) vec[i] = lin64(dec, h[i]);
    vb.sync();
    const u64 words = np;                        // n/64 = n_p words
    for (u64 wd = vb.t; wd < words; wd += vb.nt) {
        u64 out = 0;
        for (int b = 0; b < 64; ++b) {
            u64 pos = wd * 64 + b;
            u64 j = pos >> l, i = pos & (np - 1);
            out |= ((vec[i] >> j) & 1ull) << b;
        }
        novel[wd] = out;
    }
}


// Batch forms: job j of the launch (vb.by) reads operand `which` of
// jobs[j] into dst + j * stride, or writes its product from src + j * stride.
__device__ __forceinline__ void load_jobs_body(const VBlock &vb, const JobDev *__restrict__ jobs, int which,
                                               u64 *__restrict__ dst, u64 stride, u64 dst_words)
{
    const JobDev jb = jobs[vb.by];
    const u64 *src = which ? jb.b : jb.a;
    const u64 nbits = which ? jb.nb : jb.na;
    dst += (u64)vb.by * stride;
    for (u64 w = (u64)vb.bx * vb.nt + vb.t; w < dst_words; w += (u64)vb.gx * vb.nt) {
        const u64 nw = (nbits + 63) >> 6;
        u64 v = 0;
        if (w < nw) {
            v = src[w];
            if (w == nw - 1 && (nbits & 63)) v &= (~0ull) >> (64 - (nbits & 63));
        }
        dst[w] = v;
    }
}

__device__ __forceinline__ void store_jobs_body(const VBlock &vb, const u64 *GF2X_DATA_RESTRICT src, u64 stride,
                                                const JobDev *__restrict__ jobs)
{
    const JobDev jb = jobs[vb.by];
    const u64 nc = (jb.na && jb.nb) ? jb.na + jb.nb - 1 : 0;
    const u64 nw = (nc + 63) >> 6;
    src += (u64)vb.by * stride;
    for (u64 w = (u64)vb.bx * vb.nt + vb.t; w < nw; w += (u64)vb.gx * vb.nt) {
        u64 v = src[w];
        if (w == nw - 1 && (nc & 63)) v &= (~0ull) >> (64 - (nc & 63));
        jb.c[w] = v;
    }
}

}  // namespace fftk
}  // namespace gf2x
