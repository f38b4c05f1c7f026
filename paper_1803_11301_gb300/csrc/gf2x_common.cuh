// Shared definitions of the GB300 GF(2)[x] multiplier (device + host side).
//
// Field: GF(2^64) = GF(2)[x] / (x^64 + x^4 + x^3 + x + 1), polynomial form
// (Sec. 4.3).  The GPU has no carry-less multiply instruction, so the product
// is built from 32x32->64 integer multiplies on operands with "holes"
// (every fourth bit kept, so no carry reaches a kept bit), Karatsuba over the
// 32-bit halves, and a two-step fold of the high word by x^4 + x^3 + x + 1.
#pragma once

#include <cstddef>
#include <cstdint>
#include <functional>
#include <utility>

#include <cuda_runtime.h>

#include "../../include/gf2x.h"

typedef uint64_t u64;
typedef uint32_t u32;

#define GF2X_MOD_LOW 0x1Bull   // x^4 + x^3 + x + 1

// ------------------------------------------------------------ field arithmetic
// 32 x 32 -> 64-bit carry-less product by integer multiplication of operands
// with "holes", the published constant-time technique of T. Pornin (BearSSL's
// ghash_ctmul): a_i = a & (0x1111... << i) keeps one bit in four; the integer
// product a_i * b_j has at most 8 terms per output position, so each count
// fits in the 4-bit gap and its parity is the carry-less bit.  Positions of
// class k (mod 4) come from the pairs i+j = k.
__device__ __forceinline__ u64 clmul32(u32 a, u32 b)
{
    const u32 m0 = 0x11111111u, m1 = 0x22222222u, m2 = 0x44444444u, m3 = 0x88888888u;
    u32 a0 = a & m0, a1 = a & m1, a2 = a & m2, a3 = a & m3;
    u32 b0 = b & m0, b1 = b & m1, b2 = b & m2, b3 = b & m3;
    u64 z0 = ((u64)a0 * b0) ^ ((u64)a1 * b3) ^ ((u64)a2 * b2) ^ ((u64)a3 * b1);
    u64 z1 = ((u64)a0 * b1) ^ ((u64)a1 * b0) ^ ((u64)a2 * b3) ^ ((u64)a3 * b2);
    u64 z2 = ((u64)a0 * b2) ^ ((u64)a1 * b1) ^ ((u64)a2 * b0) ^ ((u64)a3 * b3);
    u64 z3 = ((u64)a0 * b3) ^ ((u64)a1 * b2) ^ ((u64)a2 * b1) ^ ((u64)a3 * b0);
    return (z0 & 0x1111111111111111ull) | (z1 & 0x2222222222222222ull) |
           (z2 & 0x4444444444444444ull) | (z3 & 0x8888888888888888ull);
}

// (hi, lo) -> hi * x^64 + lo reduced: x^64 = x^4 + x^3 + x + 1.
__device__ __forceinline__ u64 gf64_reduce(u64 hi, u64 lo)
{
    u64 t = hi ^ (hi << 1) ^ (hi << 3) ^ (hi << 4);
    u64 over = (hi >> 63) ^ (hi >> 61) ^ (hi >> 60);      // bits 64..67 of hi * 0x1B
    t ^= over ^ (over << 1) ^ (over << 3) ^ (over << 4);
    return lo ^ t;
}

__device__ __forceinline__ u64 gf64_mul(u64 a, u64 b)
{
    u32 al = (u32)a, ah = (u32)(a >> 32), bl = (u32)b, bh = (u32)(b >> 32);
    u64 lo = clmul32(al, bl);
    u64 hi = clmul32(ah, bh);
    u64 mid = clmul32(al ^ ah, bl ^ bh) ^ lo ^ hi;          // Karatsuba middle term
    return gf64_reduce(hi ^ (mid >> 32), lo ^ (mid << 32));
}

// 64-bit GF(2)-linear map given as 8 byte-window tables (t[k][v] = image of
// v << 8k): the method of four Russians with 8-bit windows (Sec. 4.5).
__device__ __forceinline__ u64 lin64(const u64 *__restrict__ t, u64 x)
{
    u64 r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= t[k * 256 + ((x >> (8 * k)) & 255)];
    return r;
}

// 64x64 bit transpose across a warp (Sec. 4.4's block-swap transpose: a
// 32-bit half swap in registers, then five exchange rounds across lanes).
constexpr u64 kM16 = 0x0000FFFF0000FFFFull, kM8 = 0x00FF00FF00FF00FFull, kM4 = 0x0F0F0F0F0F0F0F0Full,
              kM2 = 0x3333333333333333ull, kM1 = 0x5555555555555555ull;

// Lane t holds rows t (A) and t + 32 (B) of a 64x64 bit matrix (bit c of row
// r = M[r][c]); on return A = column t and B = column t + 32 (bit r = M[r][c]).
// Applied to columns it returns rows.
__device__ __forceinline__ void transpose64(u64 &A, u64 &B, int lane)
{
    const u64 a2 = (A & 0x00000000FFFFFFFFull) | (B << 32);
    const u64 b2 = (A >> 32) | (B & 0xFFFFFFFF00000000ull);
    A = a2;
    B = b2;
    const u64 masks[5] = {kM16, kM8, kM4, kM2, kM1};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int j = 16 >> s;
        const u64 m = masks[s];
        const u64 ya = __shfl_xor_sync(0xffffffffu, A, j), yb = __shfl_xor_sync(0xffffffffu, B, j);
        if (lane & j) {
            A = ((ya & ~m) >> j) | (A & ~m);
            B = ((yb & ~m) >> j) | (B & ~m);
        } else {
            A = (A & m) | ((ya & m) << j);
            B = (B & m) | ((yb & m) << j);
        }
    }
}

// ------------------------------------------------ programmatic dependent launch
// With `enable`, a kernel launched by launch_pdl may start while the kernel
// before it in the stream is finishing.  Each of its blocks first lets its own
// dependents launch (pdl_allow: they start once every block of this grid
// runs), then does work that touches no data of earlier kernels (constant
// tables, twiddle tables), then waits for the previous grid's completion and
// memory (pdl_wait, a hardware dependency) before its first read or write of
// the data.  Launched normally, both are no-ops.  Measured on GB300 it pays
// for small products only (2^16 to 2^20-bit operands: 8-9% less time; at
// 2^24 and 2^30 the early blocks compete with the previous kernel's last
// wave: 1.5% more), so the products enable it by size (gf2x_ctx::pdl).
__device__ __forceinline__ void pdl_allow() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool enable, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = enable ? attr : nullptr;
    cfg.numAttrs = enable ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// One product of a batch as the device sees it (the job table lives in the
// workspace).  nc = na + nb - 1 bits (0 if either is 0).
struct JobDev {
    const u64 *a;
    u64 na;
    const u64 *b;
    u64 nb;
    u64 *c;
    u64 pad;
};

// State of one grid-wide barrier (see cvt.cu); must be zero before a launch.
struct GridSync {
    unsigned count;   // blocks arrived in the current generation
    unsigned gen;     // generation, bumped by the last arrival
    unsigned abort;   // set when a wait ran out: every block returns
    unsigned pad;
};

// ------------------------------------------------------------------ context
// Stages of Alg. 5 as the profiler and the launch counter see them.
// STAGE_BOTTOM is the fused low-layer kernel of gf2x_mul: the bottom layers of
// both forward Butterflies, the pointwise product and the bottom layers of the
// iButterfly; STAGE_BUTTERFLY / STAGE_IBUTTERFLY then hold the top layers.
enum Gf2xStage {
    STAGE_LOAD = 0, STAGE_BASISCVT, STAGE_ENCODE, STAGE_BUTTERFLY, STAGE_POINTWISE,
    STAGE_IBUTTERFLY, STAGE_DECODE, STAGE_IBASISCVT, STAGE_STORE, STAGE_BOTTOM, STAGE_COUNT
};

struct gf2x_ctx {
    int device;
    int num_sms;
    u64 *d_tables;      // one allocation holding the tables below
    u64 *d_cvt;         // 8 x 256: Cantor coordinates -> polynomial form
    u64 *d_enc;         // 8 x 256: bits (a_{j n_p + i})_j -> f_i  (matrix R)
    u64 *d_dec;         // 8 x 256: f_i -> bits                    (matrix R^{-1})
    u64 *d_cantor;      // v_0 .. v_63
    int *d_status;      // device status word (gf2x_status)
    GridSync *d_sync;   // barrier state for the stage entry points
    unsigned long long *d_word;   // one device word for measurement checksums (fieldbench.cu)
    u64 cantor[64];     // host copy of the Cantor basis
    // GF(2^128) variant (m128.cu): 128-bit entries as (lo, hi) word pairs
    u64 *d_tables128;   // one allocation holding the tables below
    u64 *d_cvt128;      // 8 x 256: Cantor coordinates < 2^64 -> polynomial form
    u64 *d_enc128;      // 16 x 256: the 128 bits (a_{j n_p + i})_j -> f_i  (matrix R)
    u64 *d_dec128;      // 16 x 256: f_i -> bits                             (matrix R^{-1})
    u64 *d_cantor128;   // v_0 .. v_127

    // launch accounting and optional per-stage event timing (host side)
    int stage;                          // stage the next launches belong to
    unsigned long long launches[STAGE_COUNT];
    bool profiling;
    void *prof;                         // event pool, see api.cu
    void *graphs;                       // CUDA graph cache of gf2x_mul, see api.cu
    void *batch_graphs;                 // CUDA graph cache of gf2x_mul_batch
    void *tuner;                        // measured launch-shape choices, see tune.cu
    bool pdl;                           // launch_pdl overlaps kernels (set per product by size)
};

// Count one kernel launch against the current stage.
inline void count_launch(gf2x_ctx *ctx, int n = 1) { ctx->launches[ctx->stage] += (unsigned long long)n; }

// ----------------------------------------------------------------- launchers
// All enqueue on `st` and return cudaGetLastError().
namespace gf2x {

// Autotuner (tune.cu).  Knobs: the choices it measures.
// The same numbers as the GF2X_KNOB_* constants of the C ABI.
enum TuneKnob {
    TUNE_UNIT16_R = 1, TUNE_BOTTOM_SHAPE = 2, TUNE_WINDOW_DEPTH = 3, TUNE_M128_BOTTOM_CHUNK = 4, TUNE_BFLY_DEPTH = 5,
    TUNE_M128_BFLY_DEPTH = 6, TUNE_KNOB_END = 7
};
void *tuner_create();
void tuner_destroy(void *t);
void tuner_freeze(void *t, bool frozen);
// choice < 0 releases the knob.
void tuner_pin(void *t, int knob, int choice);
// The pinned choice of `knob` if it is one of cands, else fallback.
int tune_pinned(gf2x_ctx *ctx, int knob, const int *cands, int ncand, int fallback);
// The stored choice for (knob, key); else, when measuring is possible, runs
// run(candidate) on `st` for every candidate, stores and returns the fastest;
// else `fallback`.
int tune_choice(gf2x_ctx *ctx, int knob, u64 key, const int *cands, int ncand, int fallback,
                const std::function<cudaError_t(int)> &run, cudaStream_t st);
// Keys use the power-of-two bucket of a count (ceil(log2 x)): the best shape
// depends on the amount of work, so one measurement serves every count of a
// bucket (batches and serving meet many distinct job counts).
inline u64 tune_bucket(u64 x)
{
    u64 b = 0;
    while (b < 63 && (1ull << b) < x) ++b;
    return b;
}
// The stored choice for (knob, key), else `fallback`; never measures.
int tune_stored(gf2x_ctx *ctx, int knob, u64 key, int fallback);

// Batched forms: `count` jobs whose buffers are `stride` words apart
// (count = 1, stride = 0 for a single product).
// BasisCvt (or iBasisCvt) in place on bits.  `scratch`, if not null, is a
// buffer laid out like `bits` (count x stride words) whose contents may be
// overwritten; with it, 2^18 <= L <= 2^32 run the structured kernels.
cudaError_t basis_cvt(gf2x_ctx *ctx, u64 *bits, u64 L, bool inverse, int count, u64 stride, u64 *scratch,
                      cudaStream_t st);
// BasisCvt inside every 2^16-bit block of an L-bit array (L a multiple of 2^16).
// scratch (nullable): a free buffer laid out like bits, for the tuner.
cudaError_t basis_cvt_unit16(gf2x_ctx *ctx, u64 *bits, u64 L, bool inverse, int count, u64 stride, u64 *scratch,
                             cudaStream_t st);
// Outer BasisCvt of length 2^M (2 <= M <= 9) on units of 2^ulog words, applied
// to every chunk of 2^M units of an L-bit array, read from src (which may be
// bits) and written to bits.
cudaError_t basis_cvt_outer(gf2x_ctx *ctx, u64 *bits, const u64 *src, u64 L, int M, int ulog, bool inverse, int count,
                            u64 stride, cudaStream_t st);
cudaError_t wait_timeout_probe(gf2x_ctx *ctx, GridSync *gs, cudaStream_t st);
// Job j reads novel + j stride and writes f + j out_stride.
cudaError_t encode(gf2x_ctx *ctx, const u64 *novel, int l, u64 *f, u64 nonzero_bits, int count, u64 stride,
                   u64 out_stride, cudaStream_t st);
cudaError_t decode(gf2x_ctx *ctx, const u64 *h, int l, u64 *novel, int count, u64 stride, cudaStream_t st);
// scratch (nullable): a free buffer of the transform's size, for the tuner.
cudaError_t butterfly(gf2x_ctx *ctx, u64 *x, int l, bool inverse, int count, u64 stride, cudaStream_t st,
                      u64 *scratch = nullptr);
// Bottom-tile depth bt for products with 2^l points, measured on X, Y and T
// (free buffers laid out like the transforms).  The three calls below take it
// (bt < 0: the default depth); one product uses the same bt in all three.
int butterfly_depth(gf2x_ctx *ctx, u64 *X, u64 *Y, u64 *T, int l, int count, u64 stride, cudaStream_t st);
// The depth butterfly_depth returned (or would return without measuring).
int butterfly_depth_stored(gf2x_ctx *ctx, int l, int count);
cudaError_t butterfly_top_pair(gf2x_ctx *ctx, u64 *x0, u64 *x1, int l, int count, u64 stride, cudaStream_t st,
                               int bt = -1);
cudaError_t butterfly_bottom_fused(gf2x_ctx *ctx, u64 *X, u64 *Y, int l, int count, u64 stride, cudaStream_t st,
                                   bool y_transformed = false, u64 *scratch = nullptr, int bt = -1);
cudaError_t butterfly_top_inverse(gf2x_ctx *ctx, u64 *x, int l, int count, u64 stride, cudaStream_t st, int bt = -1);
cudaError_t load_jobs(gf2x_ctx *ctx, const JobDev *jobs, int which, u64 *dst, u64 stride, u64 dst_words, int count,
                      cudaStream_t st);
cudaError_t store_jobs(gf2x_ctx *ctx, const u64 *src, u64 stride, const JobDev *jobs, u64 max_words, int count,
                       cudaStream_t st);
cudaError_t pointwise(gf2x_ctx *ctx, const u64 *a, const u64 *b, u64 *c, u64 count, cudaStream_t st);
cudaError_t load_bits(gf2x_ctx *ctx, const u64 *src, u64 nbits, u64 *dst, u64 dst_words, cudaStream_t st);
// a into dst and b into dst + half, dst_words words each.
cudaError_t load_pair(gf2x_ctx *ctx, const u64 *a, u64 na, const u64 *b, u64 nb, u64 *dst, u64 dst_words, u64 half,
                      cudaStream_t st);
cudaError_t store_bits(gf2x_ctx *ctx, const u64 *src, u64 nbits, u64 *dst, cudaStream_t st);
// c = a^2 (2 na - 1 bits) by spreading the bits of a: no transform.
cudaError_t square_bits(gf2x_ctx *ctx, const u64 *a, u64 na, u64 *c, cudaStream_t st);


// ---- the GF(2^128) variant (m128.cu).  A point is two words (lo, hi); a
// transform of n bits holds n_p = n/128 points in n/64 words.
// Number of u64 words of the tables and filling them (host side); false if a
// step of the set-up fails (a singular system).
constexpr size_t kTables128Words = 2 * (8 * 256 + 16 * 256 + 16 * 256 + 128);
bool m128_build_tables(u64 *host);
// l = log2(n_p) = log2(n) - 7.
cudaError_t m128_encode(gf2x_ctx *ctx, const u64 *novel, int l, u64 *f, u64 nonzero_bits, int count, u64 stride,
                        u64 out_stride, cudaStream_t st);
cudaError_t m128_decode(gf2x_ctx *ctx, const u64 *h, int l, u64 *novel, int count, u64 stride, cudaStream_t st);
cudaError_t m128_butterfly(gf2x_ctx *ctx, u64 *x, int l, bool inverse, int count, u64 stride, cudaStream_t st);
// Bottom-tile depth, as butterfly_depth / butterfly_depth_stored for m = 64.
int m128_butterfly_depth(gf2x_ctx *ctx, u64 *X, u64 *Y, u64 *T, int l, int count, u64 stride, cudaStream_t st);
int m128_butterfly_depth_stored(gf2x_ctx *ctx, int l, int count);
cudaError_t m128_butterfly_top_pair(gf2x_ctx *ctx, u64 *x0, u64 *x1, int l, int count, u64 stride, cudaStream_t st,
                                    int bt = -1);
// scratch (nullable): a free buffer laid out like X, for the tuner.
cudaError_t m128_butterfly_bottom_fused(gf2x_ctx *ctx, u64 *X, const u64 *Y, int l, int count, u64 stride,
                                        cudaStream_t st, u64 *scratch = nullptr, int bt = -1);
cudaError_t m128_butterfly_top_inverse(gf2x_ctx *ctx, u64 *x, int l, int count, u64 stride, cudaStream_t st,
                                       int bt = -1);
cudaError_t m128_pointwise(gf2x_ctx *ctx, const u64 *a, const u64 *b, u64 *c, u64 count, cudaStream_t st);

// gf2x_mul (same arguments and checks) with every kernel launched directly,
// never through the CUDA graph cache (api.cu).
gf2x_status mul_uncached(gf2x_ctx *ctx, const u64 *a, u64 na, const u64 *b, u64 nb, u64 *c, void *ws,
                         size_t ws_bytes, cudaStream_t st);

}  // namespace gf2x
