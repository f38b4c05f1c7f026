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
#include "bfly_dev.cuh"

namespace gf2x {
namespace {
using namespace bflyk;

template <int M, bool INV>
__global__ void __launch_bounds__(kThreads) k_bfly_top(u64 *x0, u64 *x1, int l, int p, u64 chunks, int per_block,
                                                       const u64 *__restrict__ cvt, const u64 *__restrict__ vcan,
                                                       int arrays, u64 stride)
{
    extern __shared__ u64 smem_raw[];
    bfly_top_body<M, INV>(launch_block(), smem_raw, x0, x1, l, p, chunks, per_block, cvt, vcan, arrays, stride);
}

template <int THREADS, int CHUNK, bool H4>
__global__ void __launch_bounds__(THREADS, 65536 / (THREADS * 64))
    k_bfly_bottom(u64 *X, u64 *Y, int l, int bt, const u64 *__restrict__ cvt, const u64 *__restrict__ vcan, int mode,
                  u64 stride)
{
    extern __shared__ u64 smem_raw[];
    bfly_bottom_body<CHUNK, H4>(launch_block(), smem_raw, X, Y, l, bt, cvt, vcan, mode, stride);
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

template <int THREADS, int CHUNK>
cudaError_t launch_bottom_kernel(bool pdl, int mul, dim3 grid, size_t smem, cudaStream_t st, u64 *X, u64 *Y, int l,
                                 int bt, const u64 *cvt, const u64 *vcan, int mode, u64 stride)
{
    if (mul) return launch_pdl(pdl, k_bfly_bottom<THREADS, CHUNK, true>, grid, dim3(THREADS), smem, st, X, Y, l, bt, cvt,
                               vcan, mode, stride);
    return launch_pdl(pdl, k_bfly_bottom<THREADS, CHUNK, false>, grid, dim3(THREADS), smem, st, X, Y, l, bt, cvt, vcan,
                      mode, stride);
}

// shape 1: the small-count shape, 0: the large-count one, 2: the lean one;
// mul 0: the 16-bit integer product form, 1: the 32-bit one (gf64_mul_t)
cudaError_t launch_bottom_shape(gf2x_ctx *ctx, u64 *X, u64 *Y, int l, int bt, int mode, int count, u64 stride,
                                int shape, int mul, cudaStream_t st)
{
    const bool fused = mode == BOTTOM_FUSED || mode == BOTTOM_FUSED_PRE;
    const dim3 grid((unsigned)(1ull << (l - bt)), count);
    if (recording(ctx)) {
        // a block of the persistent kernel runs the 256-thread shapes
        const int chunk = shape == 2 ? kBottomChunkLean : kBottomChunkLarge;
        SegRec r{SEG_BOTTOM, {bt, mode, chunk, l}, grid.x, grid.y, (unsigned)kBottomThreadsLarge,
                 (unsigned)bottom_smem(bt, fused, chunk), grid.x, -1,
                 {(u64)X, (u64)Y, (u64)ctx->d_cvt, (u64)ctx->d_cantor, stride}};
        return record(ctx, r) ? cudaSuccess : cudaErrorInvalidValue;
    }
    cudaError_t e;
    if (shape == 1)
        e = launch_bottom_kernel<kBottomThreadsSmall, kBottomChunkSmall>(ctx->pdl, mul, grid,
                                                                         bottom_smem(bt, fused, kBottomChunkSmall), st,
                                                                         X, Y, l, bt, ctx->d_cvt, ctx->d_cantor, mode,
                                                                         stride);
    else if (shape == 2)
        e = launch_bottom_kernel<kBottomThreadsLarge, kBottomChunkLean>(ctx->pdl, mul, grid,
                                                                        bottom_smem(bt, fused, kBottomChunkLean), st, X,
                                                                        Y, l, bt, ctx->d_cvt, ctx->d_cantor, mode,
                                                                        stride);
    else
        e = launch_bottom_kernel<kBottomThreadsLarge, kBottomChunkLarge>(ctx->pdl, mul, grid,
                                                                         bottom_smem(bt, fused, kBottomChunkLarge), st,
                                                                         X, Y, l, bt, ctx->d_cvt, ctx->d_cantor, mode,
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
    static const int muls[2] = {0, 1};
    int mul = 0;
    const u64 key = (tune_bucket(tiles * (u64)count) << 2) | (u64)mode;
    if (!scratch) {
        shape = tune_pinned(ctx, TUNE_BOTTOM_SHAPE, cands, 3, shape);
        mul = tune_pinned(ctx, TUNE_BOTTOM_MUL, muls, 2, mul);
    } else {
        // the block shape with the default product form, then the product form in that shape
        shape = tune_choice(ctx, TUNE_BOTTOM_SHAPE, key, cands, 3, shape,
                            [&](int sh) { return launch_bottom_shape(ctx, scratch, Y, l, bt, mode, count, stride, sh, 0, st); },
                            st);
        mul = tune_choice(ctx, TUNE_BOTTOM_MUL, key | ((u64)shape << 40), muls, 2, 0,
                          [&](int mv) { return launch_bottom_shape(ctx, scratch, Y, l, bt, mode, count, stride, shape, mv, st); },
                          st);
    }
    launch_bottom_shape(ctx, X, Y, l, bt, mode, count, stride, shape, mul, st);
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
    // blocks of the persistent kernel have 64 registers a thread: up to 3 layers a pass
    const int most = recording(ctx) ? (kTopLayers < 3 ? kTopLayers : 3) : kTopLayers;
    const int npass = (layers + most - 1) / most;
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
        if (recording(ctx)) {
            SegRec r{SEG_TOP, {m, inverse ? 1 : 0, p, per_block}, grid.x, grid.y, (unsigned)kThreads,
                     (unsigned)(((1 << m) - 1) * kTab * sizeof(u64) + 128), grid.x * (unsigned)arrays, -1,
                     {(u64)x0, (u64)x1, (u64)l, chunks, (u64)cvt, (u64)vb, (u64)arrays, stride}};
            if (!record(ctx, r)) return cudaErrorInvalidValue;
            continue;
        }
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
    cudaFuncSetAttribute(k_bfly_bottom<kBottomThreadsSmall, kBottomChunkSmall, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bottom_smem(kBottom, true, kBottomChunkSmall));
    cudaFuncSetAttribute(k_bfly_bottom<kBottomThreadsLarge, kBottomChunkLarge, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bottom_smem(kBottom, true, kBottomChunkLarge));
    cudaFuncSetAttribute(k_bfly_bottom<kBottomThreadsLarge, kBottomChunkLean, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bottom_smem(kBottom, true, kBottomChunkLean));
    cudaFuncSetAttribute(k_bfly_bottom<kBottomThreadsSmall, kBottomChunkSmall, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bottom_smem(kBottom, true, kBottomChunkSmall));
    cudaFuncSetAttribute(k_bfly_bottom<kBottomThreadsLarge, kBottomChunkLarge, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bottom_smem(kBottom, true, kBottomChunkLarge));
    cudaFuncSetAttribute(k_bfly_bottom<kBottomThreadsLarge, kBottomChunkLean, true>,
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
    if (recording(ctx)) {
        // the depth stored for this size, at most what a block of the persistent kernel holds (two fused
        // tiles and a 16-table chunk per 256 threads, kPersistMaxDepth)
        const int bt = butterfly_depth_stored(ctx, l, count);
        return bt < kPersistMaxDepth ? bt : kPersistMaxDepth;
    }
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

GF2X_OUT_OF_RANGE_READER(out_of_range_bfly)

}  // namespace gf2x
