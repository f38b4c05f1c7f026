// Register-resident parts of BasisCvt / iBasisCvt (Alg. 1, Sec. 2.3.1): launches of
// the 2^16-bit block kernel and the outer-conversion kernel, whose bodies and
// method are in cvt_reg_dev.cuh.
#include "cvt_reg_dev.cuh"

namespace gf2x {
namespace {
using namespace cvtrk;

template <bool INV, int R>
__global__ void __launch_bounds__(1024 / R) k_cvt_unit16(u64 *bits, u64 stride)
{
    __shared__ u64 sm[kUnitWords];
    cvt_unit16_body<INV, R>(launch_block(), sm, bits, stride);
}

template <int M, bool INV>
__global__ void __launch_bounds__(OuterShape<M>::THREADS) k_cvt_outer(u64 *bits, const u64 *src, int ulog, u64 stride)
{
    __shared__ u64 st[OuterShape<M>::SMEM_WORDS];
    cvt_outer_body<M, INV>(launch_block(), st, bits, src, ulog, stride);
}

template <int M>
void launch_outer(u64 *bits, const u64 *src, int ulog, u64 columns, bool inverse, int count, u64 stride,
                  cudaStream_t st)
{
    using Sh = OuterShape<M>;
    const dim3 grid((unsigned)(columns / Sh::CW), (unsigned)count);
    if (inverse) k_cvt_outer<M, true><<<grid, Sh::THREADS, 0, st>>>(bits, src, ulog, stride);
    else k_cvt_outer<M, false><<<grid, Sh::THREADS, 0, st>>>(bits, src, ulog, stride);
}

// Columns per block of the outer kernel for M (0 if M is out of range).
int outer_columns_per_block(int M)
{
    switch (M) {
    case 2: return OuterShape<2>::CW;
    case 3: return OuterShape<3>::CW;
    case 4: return OuterShape<4>::CW;
    case 5: return OuterShape<5>::CW;
    case 6: return OuterShape<6>::CW;
    case 7: return OuterShape<7>::CW;
    case 8: return OuterShape<8>::CW;
    case 9: return OuterShape<9>::CW;
    default: return 0;
    }
}

}  // namespace

cudaError_t basis_cvt_outer(gf2x_ctx *ctx, u64 *bits, const u64 *src, u64 L, int M, int ulog, bool inverse, int count,
                            u64 stride, cudaStream_t st)
{
    if (M <= 1) return src == bits ? cudaSuccess : cudaErrorInvalidValue;   // no steps (length <= 2)
    const u64 words = L >> 6;
    const u64 columns = words >> M;                     // (chunks) x (words per unit)
    const int cw = outer_columns_per_block(M);
    // every block's columns lie in one chunk: CW divides the unit
    if (cw == 0 || ulog < 0 || (1ull << ulog) % (u64)cw != 0 || (columns >> ulog) << ulog != columns)
        return cudaErrorInvalidValue;
    if (recording(ctx)) {
        // blocks of 8 warps, the persistent kernel's block size
        static const int kColsOf[10] = {0, 0, OuterShape<2, 8>::CW, OuterShape<3, 8>::CW, OuterShape<4, 8>::CW,
                                        OuterShape<5, 8>::CW, OuterShape<6, 8>::CW, OuterShape<7, 8>::CW,
                                        OuterShape<8, 8>::CW, OuterShape<9, 8>::CW};
        static const int kWordsOf[10] = {0, 0, OuterShape<2, 8>::SMEM_WORDS, OuterShape<3, 8>::SMEM_WORDS,
                                         OuterShape<4, 8>::SMEM_WORDS, OuterShape<5, 8>::SMEM_WORDS,
                                         OuterShape<6, 8>::SMEM_WORDS, OuterShape<7, 8>::SMEM_WORDS,
                                         OuterShape<8, 8>::SMEM_WORDS, OuterShape<9, 8>::SMEM_WORDS};
        const u64 cw8 = (u64)kColsOf[M];
        if ((1ull << ulog) % cw8 != 0) return cudaErrorInvalidValue;
        const unsigned gx = (unsigned)(columns / cw8);
        SegRec r{SEG_OUTER, {M, inverse ? 1 : 0, ulog, 0}, gx, (unsigned)count, 256u, (unsigned)kWordsOf[M] * 8, gx,
                 -1, {(u64)bits, (u64)src, stride}};
        return record(ctx, r) ? cudaSuccess : cudaErrorInvalidValue;
    }
    switch (M) {
    case 2: launch_outer<2>(bits, src, ulog, columns, inverse, count, stride, st); break;
    case 3: launch_outer<3>(bits, src, ulog, columns, inverse, count, stride, st); break;
    case 4: launch_outer<4>(bits, src, ulog, columns, inverse, count, stride, st); break;
    case 5: launch_outer<5>(bits, src, ulog, columns, inverse, count, stride, st); break;
    case 6: launch_outer<6>(bits, src, ulog, columns, inverse, count, stride, st); break;
    case 7: launch_outer<7>(bits, src, ulog, columns, inverse, count, stride, st); break;
    case 8: launch_outer<8>(bits, src, ulog, columns, inverse, count, stride, st); break;
    default: launch_outer<9>(bits, src, ulog, columns, inverse, count, stride, st); break;
    }
    count_launch(ctx);
    return cudaGetLastError();
}

// With R words per thread: R = 32 (one warp per block) keeps every step in
// registers and shuffles; R = 8 (four warps) runs the 7 steps wider than a
// warp through shared memory but has four times the threads in flight, which
// pays when there are few blocks.
cudaError_t basis_cvt_unit16_r(gf2x_ctx *ctx, u64 *bits, u64 L, bool inverse, int count, u64 stride, int R,
                               cudaStream_t st)
{
    const u64 units = L >> 16;
    if (units == 0) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)units, (unsigned)count);
    if (recording(ctx)) {
        SegRec r{SEG_UNIT16, {R, inverse ? 1 : 0, 0, 0}, grid.x, grid.y, (unsigned)(1024 / R), kUnitWords * 8, grid.x, -1,
                 {(u64)bits, stride}};
        return record(ctx, r) ? cudaSuccess : cudaErrorInvalidValue;
    }
    switch (R * 2 + (inverse ? 1 : 0)) {
    case 16: k_cvt_unit16<false, 8><<<grid, 128, 0, st>>>(bits, stride); break;
    case 17: k_cvt_unit16<true, 8><<<grid, 128, 0, st>>>(bits, stride); break;
    case 32: k_cvt_unit16<false, 16><<<grid, 64, 0, st>>>(bits, stride); break;
    case 33: k_cvt_unit16<true, 16><<<grid, 64, 0, st>>>(bits, stride); break;
    case 64: k_cvt_unit16<false, 32><<<grid, 32, 0, st>>>(bits, stride); break;
    case 65: k_cvt_unit16<true, 32><<<grid, 32, 0, st>>>(bits, stride); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch(ctx);
    return cudaGetLastError();
}

// R measured by the tuner on `scratch` (a buffer laid out like bits, free),
// or without one the default found on GB300: R = 8 up to 512 blocks (2^25
// bits), R = 32 from 1024.
cudaError_t basis_cvt_unit16(gf2x_ctx *ctx, u64 *bits, u64 L, bool inverse, int count, u64 stride, u64 *scratch,
                             cudaStream_t st)
{
    const u64 blocks = (L >> 16) * (u64)count;
    int R = blocks <= 4 * (u64)ctx->num_sms ? 8 : 32;
    static const int cands[3] = {8, 16, 32};
    if (recording(ctx)) R = 8;               // the shape a block of the persistent kernel runs
    else if (!scratch) R = tune_pinned(ctx, TUNE_UNIT16_R, cands, 3, R);
    else {
        R = tune_choice(ctx, TUNE_UNIT16_R, (tune_bucket(blocks) << 1) | (inverse ? 1u : 0u), cands, 3, R,
                        [&](int r) { return basis_cvt_unit16_r(ctx, scratch, L, inverse, count, stride, r, st); }, st);
    }
    return basis_cvt_unit16_r(ctx, bits, L, inverse, count, stride, R, st);
}

GF2X_OUT_OF_RANGE_READER(out_of_range_cvt_reg)

}  // namespace gf2x
