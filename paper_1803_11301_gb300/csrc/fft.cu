// Encode / Decode (Alg. 4), the pointwise product of Alg. 5 and the
// bit-array load/store around them.
#include "gf2x_common.cuh"

namespace gf2x {
namespace {

constexpr int kCols = 32;            // word columns per Encode/Decode block

// Copy a 16 KiB window table (16-byte aligned: it sits in the context's
// cudaMalloc'd table block) to shared memory with asynchronous 16-byte copies;
// the caller waits (cp.async.wait_all) and synchronises.
__device__ __forceinline__ void load_table_async(u64 *dst, const u64 *__restrict__ src)
{
    for (int k = 2 * threadIdx.x; k < 8 * 256; k += 2 * blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst + k)),
                     "l"(src + k)
                     : "memory");
}

__device__ __forceinline__ void copy_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ------------------------------------------------------------------- Encode
// n_p = 2^l >= 64.  Row j of the novelpoly bit array is bits [j n_p, (j+1) n_p),
// i.e. RW = n_p/64 words.  For the 64 points i in word column w, the 64 words
// (row j, column w) form a 64x64 bit matrix whose transpose gives, per i, the
// vector (a_{j n_p + i})_j; f_i = that vector times R (Alg. 4).
//
// A block stages 64 rows x 32 word columns in shared memory (coalesced row
// reads); each warp transposes one column's 64x64 bit matrix with shuffles
// (Sec. 4.4's block-swap transpose: a 32-bit half swap in registers, then
// five exchange rounds across lanes) and applies R through 8-bit window tables
// loaded once per block.  Rows at or above `rows` are zero and are not read.
constexpr int kPad = kCols + 1;      // padded row of the staging tile

__global__ void __launch_bounds__(256) k_encode(const u64 *__restrict__ novel, u64 rw, int rows,
                                                const u64 *__restrict__ enc, u64 *__restrict__ f, u64 groups, u64 stride,
                                                u64 out_stride)
{
    novel += (u64)blockIdx.y * stride;            // job of a batch
    f += (u64)blockIdx.y * out_stride;
    __shared__ __align__(16) u64 tab[8 * 256];
    __shared__ u64 tile[64 * kPad];
    const int cols = rw < kCols ? (int)rw : kCols;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    pdl_allow();
    load_table_async(tab, enc);                   // in flight with the first tile's loads
    pdl_wait();
    for (u64 g = blockIdx.x; g < groups; g += gridDim.x) {
        const u64 w0 = g * cols;
        __syncthreads();
        for (int k = threadIdx.x; k < 64 * cols; k += blockDim.x) {
            const int j = k / cols, w = k % cols;
            tile[j * kPad + w] = j < rows ? novel[(u64)j * rw + w0 + w] : 0;
        }
        copy_async_wait();
        __syncthreads();
        for (int w = warp; w < cols; w += blockDim.x >> 5) {
            u64 A = tile[lane * kPad + w], B = tile[(lane + 32) * kPad + w];
            transpose64(A, B, lane);
            const u64 base = (w0 + w) * 64;
            f[base + lane] = lin64(tab, A);
            f[base + lane + 32] = lin64(tab, B);
        }
    }
}

// n_p < 64: the whole transform is at most 32 words; one block, bit by bit.
// Bits at or above nonzero_bits are zero and are not read.
__global__ void k_encode_small(const u64 *__restrict__ novel, int l, u64 nonzero_bits, const u64 *__restrict__ enc,
                               u64 *__restrict__ f, u64 stride, u64 out_stride)
{
    novel += (u64)blockIdx.y * stride;
    f += (u64)blockIdx.y * out_stride;
    const u64 np = 1ull << l;
    for (u64 i = threadIdx.x; i < np; i += blockDim.x) {
        u64 u = 0;
        for (int j = 0; j < 64; ++j) {
            u64 pos = (u64)j * np + i;
            if (pos < nonzero_bits) u |= ((novel[pos >> 6] >> (pos & 63)) & 1ull) << j;
        }
        f[i] = lin64(enc, u);
    }
}

// ------------------------------------------------------------------- Decode
// The inverse of Encode: per point, the bits (c_{j n_p + i})_j = h_i R^{-1};
// a warp transposes the 64 vectors of one word column back into 64 row words.
__global__ void __launch_bounds__(256) k_decode(const u64 *__restrict__ h, u64 rw, const u64 *__restrict__ dec,
                                                u64 *__restrict__ novel, u64 groups, u64 stride)
{
    h += (u64)blockIdx.y * stride;
    novel += (u64)blockIdx.y * stride;
    __shared__ __align__(16) u64 tab[8 * 256];
    __shared__ u64 tile[64 * kPad];
    const int cols = rw < kCols ? (int)rw : kCols;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    pdl_allow();
    load_table_async(tab, dec);
    copy_async_wait();
    __syncthreads();
    pdl_wait();
    for (u64 g = blockIdx.x; g < groups; g += gridDim.x) {
        const u64 w0 = g * cols;
        for (int w = warp; w < cols; w += blockDim.x >> 5) {
            const u64 base = (w0 + w) * 64;
            u64 A = lin64(tab, h[base + lane]), B = lin64(tab, h[base + lane + 32]);
            transpose64(A, B, lane);
            tile[lane * kPad + w] = A;
            tile[(lane + 32) * kPad + w] = B;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < 64 * cols; k += blockDim.x) {
            const int j = k / cols, w = k % cols;
            novel[(u64)j * rw + w0 + w] = tile[j * kPad + w];
        }
        __syncthreads();
    }
}

__global__ void k_decode_small(const u64 *__restrict__ h, int l, const u64 *__restrict__ dec, u64 *__restrict__ novel,
                               u64 stride)
{
    h += (u64)blockIdx.y * stride;
    novel += (u64)blockIdx.y * stride;
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

// Word w of an nbits-bit operand: bits at or above nbits cleared, zero beyond.
__device__ __forceinline__ u64 operand_word(u64 v, u64 w, u64 nbits)
{
    const u64 nw = (nbits + 63) >> 6;
    if (w >= nw) return 0;
    if (w == nw - 1 && (nbits & 63)) v &= (~0ull) >> (64 - (nbits & 63));
    return v;
}

// The same copy with 16-byte accesses, two words per thread (src and dst
// 16-byte aligned, dst_words even): fewer, larger requests, which is what
// matters when either side is host memory read or written over the CPU-GPU
// link.  Words at or beyond the source's length are not read.
__global__ void k_load_bits2(const u64 *__restrict__ src, u64 nbits, u64 *__restrict__ dst, u64 dst_words)
{
    const u64 w = 2 * ((u64)blockIdx.x * blockDim.x + threadIdx.x);
    if (w >= dst_words) return;
    const u64 nw = (nbits + 63) >> 6;
    ulonglong2 v = {0, 0};
    if (w + 1 < nw) v = *(const ulonglong2 *)(src + w);
    else if (w < nw) v.x = src[w];
    v.x = operand_word(v.x, w, nbits);
    v.y = operand_word(v.y, w + 1, nbits);
    *(ulonglong2 *)(dst + w) = v;
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

// c = a * a.  In characteristic 2 squaring is the Frobenius map, additive:
// (sum a_i x^i)^2 = sum a_i x^(2i), so bit i of a goes to bit 2i of c and no
// transform is needed.  Output word w is the 32 bits [32w, 32w + 32) of a,
// spread to the even positions.
__global__ void k_square_bits(const u64 *__restrict__ a, u64 na, u64 *__restrict__ c, u64 nc_words)
{
    const u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nc_words) return;
    const u64 src = w >> 1, nw = (na + 63) >> 6;
    u64 v = a[src];
    if (src == nw - 1 && (na & 63)) v &= (~0ull) >> (64 - (na & 63));
    u64 x = (w & 1) ? v >> 32 : v & 0xFFFFFFFFull;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    c[w] = x;
}

// Both operands of one product: blockIdx.y = 0 loads a into dst, 1 loads b
// into dst + half (dst_words words each, zero beyond the operand).
// Two words per thread with 16-byte accesses (all pointers 16-byte aligned,
// dst_words and half even).
__global__ void k_load_pair2(const u64 *__restrict__ a, u64 na, const u64 *__restrict__ b, u64 nb,
                             u64 *__restrict__ dst, u64 dst_words, u64 half)
{
    const u64 *src = blockIdx.y ? b : a;
    const u64 nbits = blockIdx.y ? nb : na;
    dst += blockIdx.y * half;
    const u64 w = 2 * ((u64)blockIdx.x * blockDim.x + threadIdx.x);
    if (w >= dst_words) return;
    const u64 nw = (nbits + 63) >> 6;
    ulonglong2 v = {0, 0};
    if (w + 1 < nw) v = *(const ulonglong2 *)(src + w);
    else if (w < nw) v.x = src[w];
    v.x = operand_word(v.x, w, nbits);
    v.y = operand_word(v.y, w + 1, nbits);
    *(ulonglong2 *)(dst + w) = v;
}

__global__ void k_load_pair(const u64 *__restrict__ a, u64 na, const u64 *__restrict__ b, u64 nb, u64 *__restrict__ dst,
                            u64 dst_words, u64 half)
{
    const u64 *src = blockIdx.y ? b : a;
    const u64 nbits = blockIdx.y ? nb : na;
    dst += blockIdx.y * half;
    const u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= dst_words) return;
    const u64 nw = (nbits + 63) >> 6;
    u64 v = 0;
    if (w < nw) {
        v = src[w];
        if (w == nw - 1 && (nbits & 63)) v &= (~0ull) >> (64 - (nbits & 63));
    }
    dst[w] = v;
}

// Batch forms: job j of the launch (blockIdx.y) reads operand `which` of
// jobs[j] into dst + j * stride, or writes its product from src + j * stride.
__global__ void k_load_jobs(const JobDev *__restrict__ jobs, int which, u64 *__restrict__ dst, u64 stride,
                            u64 dst_words)
{
    const JobDev jb = jobs[blockIdx.y];
    const u64 *src = which ? jb.b : jb.a;
    const u64 nbits = which ? jb.nb : jb.na;
    dst += (u64)blockIdx.y * stride;
    for (u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x; w < dst_words; w += (u64)gridDim.x * blockDim.x) {
        const u64 nw = (nbits + 63) >> 6;
        u64 v = 0;
        if (w < nw) {
            v = src[w];
            if (w == nw - 1 && (nbits & 63)) v &= (~0ull) >> (64 - (nbits & 63));
        }
        dst[w] = v;
    }
}

__global__ void k_store_jobs(const u64 *__restrict__ src, u64 stride, const JobDev *__restrict__ jobs)
{
    const JobDev jb = jobs[blockIdx.y];
    const u64 nc = (jb.na && jb.nb) ? jb.na + jb.nb - 1 : 0;
    const u64 nw = (nc + 63) >> 6;
    src += (u64)blockIdx.y * stride;
    for (u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (u64)gridDim.x * blockDim.x) {
        u64 v = src[w];
        if (w == nw - 1 && (nc & 63)) v &= (~0ull) >> (64 - (nc & 63));
        jb.c[w] = v;
    }
}

inline unsigned blocks_for(u64 n, unsigned threads) { return (unsigned)((n + threads - 1) / threads); }
inline bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

cudaError_t encode(gf2x_ctx *ctx, const u64 *novel, int l, u64 *f, u64 nonzero_bits, int count, u64 stride,
                   u64 out_stride, cudaStream_t st)
{
    if (l < 6) {
        k_encode_small<<<dim3(1, count), 64, 0, st>>>(novel, l, nonzero_bits, ctx->d_enc, f, stride, out_stride);
    } else {
        const u64 rw = 1ull << (l - 6), np = 1ull << l;
        const u64 cols = rw < kCols ? rw : kCols, groups = rw / cols;
        int rows = (int)((nonzero_bits + np - 1) / np);           // rows that can be non-zero
        if (rows > 64) rows = 64;
        const u64 grid = groups < 4 * (u64)ctx->num_sms ? groups : 4 * (u64)ctx->num_sms;
        launch_pdl(ctx->pdl, k_encode, dim3((unsigned)grid, count), dim3(256), 0, st, novel, rw, rows, ctx->d_enc, f, groups, stride,
                                                               out_stride);
    }
    count_launch(ctx);
    return cudaGetLastError();
}

cudaError_t decode(gf2x_ctx *ctx, const u64 *h, int l, u64 *novel, int count, u64 stride, cudaStream_t st)
{
    if (l < 6) {
        k_decode_small<<<dim3(1, count), 64, 0, st>>>(h, l, ctx->d_dec, novel, stride);
    } else {
        const u64 rw = 1ull << (l - 6);
        const u64 cols = rw < kCols ? rw : kCols, groups = rw / cols;
        const u64 grid = groups < 4 * (u64)ctx->num_sms ? groups : 4 * (u64)ctx->num_sms;
        launch_pdl(ctx->pdl, k_decode, dim3((unsigned)grid, count), dim3(256), 0, st, h, rw, ctx->d_dec, novel, groups, stride);
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
        if (aligned16(src) && aligned16(dst) && dst_words % 2 == 0)
            k_load_bits2<<<blocks_for(dst_words / 2, 256), 256, 0, st>>>(src, nbits, dst, dst_words);
        else
            k_load_bits<<<blocks_for(dst_words, 256), 256, 0, st>>>(src, nbits, dst, dst_words);
        count_launch(ctx);
    }
    return cudaGetLastError();
}

cudaError_t load_pair(gf2x_ctx *ctx, const u64 *a, u64 na, const u64 *b, u64 nb, u64 *dst, u64 dst_words, u64 half,
                      cudaStream_t st)
{
    if (dst_words) {
        if (aligned16(a) && aligned16(b) && aligned16(dst) && dst_words % 2 == 0 && half % 2 == 0)
            k_load_pair2<<<dim3(blocks_for(dst_words / 2, 256), 2), 256, 0, st>>>(a, na, b, nb, dst, dst_words, half);
        else
            k_load_pair<<<dim3(blocks_for(dst_words, 256), 2), 256, 0, st>>>(a, na, b, nb, dst, dst_words, half);
        count_launch(ctx);
    }
    return cudaGetLastError();
}

cudaError_t square_bits(gf2x_ctx *ctx, const u64 *a, u64 na, u64 *c, cudaStream_t st)
{
    const u64 nc_words = (2 * na - 1 + 63) >> 6;
    if (na) {
        k_square_bits<<<blocks_for(nc_words, 256), 256, 0, st>>>(a, na, c, nc_words);
        count_launch(ctx);
    }
    return cudaGetLastError();
}

cudaError_t store_bits(gf2x_ctx *ctx, const u64 *src, u64 nbits, u64 *dst, cudaStream_t st)
{
    u64 nw = (nbits + 63) >> 6;
    if (nw) {
        if (aligned16(src) && aligned16(dst) && nw % 2 == 0)
            k_load_bits2<<<blocks_for(nw / 2, 256), 256, 0, st>>>(src, nbits, dst, nw);
        else
            k_load_bits<<<blocks_for(nw, 256), 256, 0, st>>>(src, nbits, dst, nw);
        count_launch(ctx);
    }
    return cudaGetLastError();
}

}  // namespace gf2x

namespace gf2x {

cudaError_t load_jobs(gf2x_ctx *ctx, const JobDev *jobs, int which, u64 *dst, u64 stride, u64 dst_words, int count,
                      cudaStream_t st)
{
    const u64 b = (dst_words + 255) / 256;
    k_load_jobs<<<dim3((unsigned)(b < 1024 ? b : 1024), count), 256, 0, st>>>(jobs, which, dst, stride, dst_words);
    count_launch(ctx);
    return cudaGetLastError();
}

cudaError_t store_jobs(gf2x_ctx *ctx, const u64 *src, u64 stride, const JobDev *jobs, u64 max_words, int count,
                       cudaStream_t st)
{
    const u64 b = (max_words + 255) / 256;
    k_store_jobs<<<dim3((unsigned)(b < 1024 ? (b ? b : 1) : 1024), count), 256, 0, st>>>(src, stride, jobs);
    count_launch(ctx);
    return cudaGetLastError();
}

}  // namespace gf2x
