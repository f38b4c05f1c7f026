// Encode / Decode (Alg. 4), the pointwise product (Alg. 5 line 7) and the
// bit-array load/store around them.
#include "gf2x_common.cuh"

namespace gf2x {
namespace {

constexpr int kCols = 32;            // word columns per Encode/Decode block
constexpr int kPad = 65;             // padded row length of the Decode tile

__device__ __forceinline__ void load_table(u64 *dst, const u64 *__restrict__ src)
{
    for (int k = threadIdx.x; k < 8 * 256; k += blockDim.x) dst[k] = src[k];
}

// ------------------------------------------------------------------- Encode
// n_p = 2^l >= 64.  Row j of the novelpoly bit array is bits [j n_p, (j+1) n_p),
// i.e. RW = n_p/64 words.  For the 64 points i in word column w, the 64 words
// (row j, column w) form a 64x64 bit matrix whose transpose gives, per i, the
// vector (a_{j n_p + i})_j; f_i = that vector times R (Alg. 4 lines 3-4).
__global__ void __launch_bounds__(256) k_encode(const u64 *__restrict__ novel, u64 rw, const u64 *__restrict__ enc,
                                                u64 *__restrict__ f)
{
    __shared__ u64 tab[8 * 256];
    __shared__ u64 tile[64][kCols];
    const int cols = rw < kCols ? (int)rw : kCols;
    const u64 w0 = (u64)blockIdx.x * cols;
    load_table(tab, enc);
    for (int k = threadIdx.x; k < 64 * cols; k += blockDim.x) {
        int j = k / cols, w = k % cols;
        tile[j][w] = novel[(u64)j * rw + w0 + w];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w = warp; w < cols; w += blockDim.x >> 5) {
        u64 ulo = 0, uhi = 0;
#pragma unroll 8
        for (int j = 0; j < 64; ++j) {
            u64 word = tile[j][w];
            ulo |= ((word >> lane) & 1ull) << j;
            uhi |= ((word >> (lane + 32)) & 1ull) << j;
        }
        u64 base = (w0 + w) * 64;
        f[base + lane] = lin64(tab, ulo);
        f[base + lane + 32] = lin64(tab, uhi);
    }
}

// n_p < 64: the whole transform is at most 32 words; one block, bit by bit.
__global__ void k_encode_small(const u64 *__restrict__ novel, int l, const u64 *__restrict__ enc, u64 *__restrict__ f)
{
    const u64 np = 1ull << l;
    for (u64 i = threadIdx.x; i < np; i += blockDim.x) {
        u64 u = 0;
        for (int j = 0; j < 64; ++j) {
            u64 pos = (u64)j * np + i;
            u |= ((novel[pos >> 6] >> (pos & 63)) & 1ull) << j;
        }
        f[i] = lin64(enc, u);
    }
}

// ------------------------------------------------------------------- Decode
__global__ void __launch_bounds__(256) k_decode(const u64 *__restrict__ h, u64 rw, const u64 *__restrict__ dec,
                                                u64 *__restrict__ novel)
{
    __shared__ u64 tab[8 * 256];
    __shared__ u64 vec[kCols * kPad];
    const int cols = rw < kCols ? (int)rw : kCols;
    const u64 w0 = (u64)blockIdx.x * cols;
    load_table(tab, dec);
    __syncthreads();
    for (int k = threadIdx.x; k < 64 * cols; k += blockDim.x) {
        int w = k >> 6, t = k & 63;
        vec[w * kPad + t] = lin64(tab, h[(w0 + w) * 64 + t]);   // bit j = c_{j n_p + i}
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 64 * cols; k += blockDim.x) {
        int j = k / cols, w = k % cols;
        u64 out = 0;
#pragma unroll 8
        for (int t = 0; t < 64; ++t) out |= ((vec[w * kPad + t] >> j) & 1ull) << t;
        novel[(u64)j * rw + w0 + w] = out;
    }
}

__global__ void k_decode_small(const u64 *__restrict__ h, int l, const u64 *__restrict__ dec, u64 *__restrict__ novel)
{
    __shared__ u64 vec[64];
    const u64 np = 1ull << l;
    for (u64 i = threadIdx.x; i < np; i += blockDim.x) vec[i] = lin64(dec, h[i]);
    __syncthreads();
    const u64 words = np;                        // n/64 = n_p words
    for (u64 wd = threadIdx.x; wd < words; wd += blockDim.x) {
        u64 out = 0;
        for (int b = 0; b < 64; ++b) {
            u64 pos = wd * 64 + b;
            u64 j = pos >> l, i = pos & (np - 1);
            out |= ((vec[i] >> j) & 1ull) << b;
        }
        novel[wd] = out;
    }
}

__global__ void k_pointwise(const u64 *__restrict__ a, const u64 *__restrict__ b, u64 *c, u64 count)
{
    u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) c[t] = gf64_mul(a[t], b[t]);
}

// dst[w] = w-th word of the nbits-bit src (bits >= nbits cleared), zero
// beyond; dst_words words written.
__global__ void k_load_bits(const u64 *__restrict__ src, u64 nbits, u64 *__restrict__ dst, u64 dst_words)
{
    u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= dst_words) return;
    u64 nw = (nbits + 63) >> 6;
    u64 v = 0;
    if (w < nw) {
        v = src[w];
        if (w == nw - 1 && (nbits & 63)) v &= (~0ull) >> (64 - (nbits & 63));
    }
    dst[w] = v;
}

inline unsigned blocks_for(u64 n, unsigned threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t encode(gf2x_ctx *ctx, const u64 *novel, int l, u64 *f, cudaStream_t st)
{
    if (l < 6) {
        k_encode_small<<<1, 64, 0, st>>>(novel, l, ctx->d_enc, f);
    } else {
        u64 rw = 1ull << (l - 6);
        u64 cols = rw < kCols ? rw : kCols;
        k_encode<<<(unsigned)(rw / cols), 256, 0, st>>>(novel, rw, ctx->d_enc, f);
    }
    count_launch(ctx);
    return cudaGetLastError();
}

cudaError_t decode(gf2x_ctx *ctx, const u64 *h, int l, u64 *novel, cudaStream_t st)
{
    if (l < 6) {
        k_decode_small<<<1, 64, 0, st>>>(h, l, ctx->d_dec, novel);
    } else {
        u64 rw = 1ull << (l - 6);
        u64 cols = rw < kCols ? rw : kCols;
        k_decode<<<(unsigned)(rw / cols), 256, 0, st>>>(h, rw, ctx->d_dec, novel);
    }
    count_launch(ctx);
    return cudaGetLastError();
}

cudaError_t pointwise(gf2x_ctx *ctx, const u64 *a, const u64 *b, u64 *c, u64 count, cudaStream_t st)
{
    if (count) {
        k_pointwise<<<blocks_for(count, 256), 256, 0, st>>>(a, b, c, count);
        count_launch(ctx);
    }
    return cudaGetLastError();
}

cudaError_t load_bits(gf2x_ctx *ctx, const u64 *src, u64 nbits, u64 *dst, u64 dst_words, cudaStream_t st)
{
    if (dst_words) {
        k_load_bits<<<blocks_for(dst_words, 256), 256, 0, st>>>(src, nbits, dst, dst_words);
        count_launch(ctx);
    }
    return cudaGetLastError();
}

cudaError_t store_bits(gf2x_ctx *ctx, const u64 *src, u64 nbits, u64 *dst, cudaStream_t st)
{
    u64 nw = (nbits + 63) >> 6;
    if (nw) {
        k_load_bits<<<blocks_for(nw, 256), 256, 0, st>>>(src, nbits, dst, nw);
        count_launch(ctx);
    }
    return cudaGetLastError();
}

}  // namespace gf2x
