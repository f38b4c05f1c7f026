// Encode / Decode (Alg. 4), the pointwise product of Alg. 5 and the
// bit-array load/store around them.
#include "fft_dev.cuh"

namespace gf2x {
namespace {
using namespace fftk;

__global__ void __launch_bounds__(256) k_encode(const u64 *__restrict__ novel, u64 rw, int rows,
                                                const u64 *__restrict__ enc, u64 *__restrict__ f, u64 groups, u64 stride,
                                                u64 out_stride)
{
    __shared__ __align__(2048) u64 sm[kCodecSmemWords];
    encode_body(launch_block(), sm, novel, rw, rows, enc, f, groups, stride, out_stride);
}

__global__ void k_encode_small(const u64 *__restrict__ novel, int l, u64 nonzero_bits, const u64 *__restrict__ enc,
                               u64 *__restrict__ f, u64 stride, u64 out_stride)
{
    encode_small_body(launch_block(), novel, l, nonzero_bits, enc, f, stride, out_stride);
}

__global__ void __launch_bounds__(256) k_decode(const u64 *__restrict__ h, u64 rw, const u64 *__restrict__ dec,
                                                u64 *__restrict__ novel, u64 groups, u64 stride)
{
    __shared__ __align__(128) u64 sm[kDecodeSmemWords];
    decode_body(launch_block(), sm, h, rw, dec, novel, groups, stride);
}

__global__ void k_decode_small(const u64 *__restrict__ h, int l, const u64 *__restrict__ dec, u64 *__restrict__ novel,
                               u64 stride)
{
    __shared__ u64 vec[64];
    decode_small_body(launch_block(), vec, h, l, dec, novel, stride);
}

__global__ void k_load_jobs(const JobDev *__restrict__ jobs, int which, u64 *__restrict__ dst, u64 stride,
                            u64 dst_words)
{
    load_jobs_body(launch_block(), jobs, which, dst, stride, dst_words);
}

__global__ void k_store_jobs(const u64 *__restrict__ src, u64 stride, const JobDev *__restrict__ jobs)
{
    store_jobs_body(launch_block(), src, stride, jobs);
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

inline unsigned blocks_for(u64 n, unsigned threads) { return (unsigned)((n + threads - 1) / threads); }
inline bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

// Blocks per job of a grid-stride Encode / Decode launch: as many as are
// resident at once over all `count` jobs (one wave), at most one per group.
template <class Kernel>
u64 codec_grid(gf2x_ctx *ctx, Kernel kernel, u64 groups, int count)
{
    static int per_sm = 0;
    if (!per_sm && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1))
        per_sm = 1;
    u64 g = (u64)per_sm * (u64)ctx->num_sms / (u64)(count > 0 ? count : 1);
    if (g < 1) g = 1;
    return groups < g ? groups : g;
}

cudaError_t encode(gf2x_ctx *ctx, const u64 *novel, int l, u64 *f, u64 nonzero_bits, int count, u64 stride,
                   u64 out_stride, cudaStream_t st)
{
    if (l < 6) {
        if (recording(ctx)) {
            SegRec r{SEG_ENCODE_SMALL, {l, 0, 0, 0}, 1, (unsigned)count, 64, 0, 1, -1,
                     {(u64)novel, nonzero_bits, (u64)ctx->d_enc, (u64)f, stride, out_stride}};
            return record(ctx, r) ? cudaSuccess : cudaErrorInvalidValue;
        }
        k_encode_small<<<dim3(1, count), 64, 0, st>>>(novel, l, nonzero_bits, ctx->d_enc, f, stride, out_stride);
    } else {
        const u64 rw = 1ull << (l - 6), np = 1ull << l;
        const u64 cols = rw < kCols ? rw : kCols, groups = rw / cols;
        int rows = (int)((nonzero_bits + np - 1) / np);           // rows that can be non-zero
        if (rows > 64) rows = 64;
        const u64 grid = codec_grid(ctx, k_encode, groups, count);
        if (recording(ctx)) {
            SegRec r{SEG_ENCODE, {rows, 0, 0, 0}, (unsigned)grid, (unsigned)count, 256, kCodecSmemWords * 8,
                     (unsigned)grid, -1, {(u64)novel, rw, (u64)ctx->d_enc, (u64)f, groups, stride, out_stride}};
            return record(ctx, r) ? cudaSuccess : cudaErrorInvalidValue;
        }
        launch_pdl(ctx->pdl, k_encode, dim3((unsigned)grid, count), dim3(256), 0, st, novel, rw, rows, ctx->d_enc, f, groups, stride,
                                                               out_stride);
    }
    count_launch(ctx);
    return cudaGetLastError();
}

cudaError_t decode(gf2x_ctx *ctx, const u64 *h, int l, u64 *novel, int count, u64 stride, cudaStream_t st)
{
    if (l < 6) {
        if (recording(ctx)) {
            SegRec r{SEG_DECODE_SMALL, {l, 0, 0, 0}, 1, (unsigned)count, 64, 64 * 8, 1, -1,
                     {(u64)h, (u64)ctx->d_dec, (u64)novel, stride}};
            return record(ctx, r) ? cudaSuccess : cudaErrorInvalidValue;
        }
        k_decode_small<<<dim3(1, count), 64, 0, st>>>(h, l, ctx->d_dec, novel, stride);
    } else {
        const u64 rw = 1ull << (l - 6);
        const u64 cols = rw < kCols ? rw : kCols, groups = rw / cols;
        const u64 grid = codec_grid(ctx, k_decode, groups, count);
        if (recording(ctx)) {
            SegRec r{SEG_DECODE, {0, 0, 0, 0}, (unsigned)grid, (unsigned)count, 256, kDecodeSmemWords * 8,
                     (unsigned)grid, -1, {(u64)h, rw, (u64)ctx->d_dec4, (u64)novel, groups, stride}};
            return record(ctx, r) ? cudaSuccess : cudaErrorInvalidValue;
        }
        launch_pdl(ctx->pdl, k_decode, dim3((unsigned)grid, count), dim3(256), 0, st, h, rw, ctx->d_dec4, novel, groups, stride);
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
    const unsigned gx = (unsigned)(b < 1024 ? b : 1024);
    if (recording(ctx)) {
        SegRec r{SEG_LOAD_JOBS, {which, 0, 0, 0}, gx, (unsigned)count, 256, 0, gx, -1,
                 {(u64)jobs, (u64)dst, stride, dst_words}};
        return record(ctx, r) ? cudaSuccess : cudaErrorInvalidValue;
    }
    k_load_jobs<<<dim3(gx, count), 256, 0, st>>>(jobs, which, dst, stride, dst_words);
    count_launch(ctx);
    return cudaGetLastError();
}

cudaError_t store_jobs(gf2x_ctx *ctx, const u64 *src, u64 stride, const JobDev *jobs, u64 max_words, int count,
                       cudaStream_t st)
{
    const u64 b = (max_words + 255) / 256;
    const unsigned gx = (unsigned)(b < 1024 ? (b ? b : 1) : 1024);
    if (recording(ctx)) {
        SegRec r{SEG_STORE_JOBS, {0, 0, 0, 0}, gx, (unsigned)count, 256, 0, gx, -1, {(u64)src, stride, (u64)jobs}};
        return record(ctx, r) ? cudaSuccess : cudaErrorInvalidValue;
    }
    k_store_jobs<<<dim3(gx, count), 256, 0, st>>>(src, stride, jobs);
    count_launch(ctx);
    return cudaGetLastError();
}

GF2X_OUT_OF_RANGE_READER(out_of_range_fft)

}  // namespace gf2x
