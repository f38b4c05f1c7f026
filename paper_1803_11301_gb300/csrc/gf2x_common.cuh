// Shared definitions of the GB300 GF(2)[x] multiplier (device + host side).
//
// Field: GF(2^64) = GF(2)[x] / (x^64 + x^4 + x^3 + x + 1), polynomial form
// (Sec. 4.3).  The GPU has no carry-less multiply instruction, so the product
// is built from 16x16-bit integer multiplies on operands with "holes" (every
// third bit kept, so no carry reaches a kept bit), Karatsuba over the 16-bit
// and 32-bit halves, and a two-step fold of the high word by x^4 + x^3 + x + 1.
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
// Carry-less products by integer multiplication of operands with "holes",
// the published constant-time technique of T. Pornin (BearSSL's ghash_ctmul):
// split each operand into residue classes of bit positions, so that the
// integer product of two classes never carries into a kept bit, and keep in
// each class of output positions the parity of its count.
//
// 16 x 16 -> 31 bits with three classes (bit positions mod 3): a class of a
// 16-bit operand has at most 6 bits, so a class-by-class product has at most
// 6 terms per output position, a count that fits in the position and the two
// bits above it (the next position of the same class is 3 higher).  Output
// positions of class k come from the class pairs (i, j) with i + j = k mod 3.
// Nine 32-bit multiplies.  Measured on GB300 against 32-bit operands with four
// classes (sixteen 32 x 32 -> 64-bit multiplies per 32-bit product): 155
// against 129 Gmul/s for the GF(2^64) product (bench.py --stage field_mul).
__device__ __forceinline__ u32 clmul16(u32 a, u32 b)
{
    const u32 m0 = 0x9249u, m1 = 0x2492u, m2 = 0x4924u;          // bits = 0, 1, 2 mod 3
    const u32 a0 = a & m0, a1 = a & m1, a2 = a & m2;
    const u32 b0 = b & m0, b1 = b & m1, b2 = b & m2;
    const u32 z0 = (a0 * b0) ^ (a1 * b2) ^ (a2 * b1);
    const u32 z1 = (a0 * b1) ^ (a1 * b0) ^ (a2 * b2);
    const u32 z2 = (a0 * b2) ^ (a1 * b1) ^ (a2 * b0);
    return (z0 & 0x49249249u) | (z1 & 0x12492492u) | (z2 & 0x24924924u);
}

// 32 x 32 -> 63 bits: Karatsuba over the 16-bit halves.
__device__ __forceinline__ u64 clmul32(u32 a, u32 b)
{
    const u32 al = a & 0xFFFFu, ah = a >> 16, bl = b & 0xFFFFu, bh = b >> 16;
    const u32 lo = clmul16(al, bl), hi = clmul16(ah, bh);
    const u32 mid = clmul16(al ^ ah, bl ^ bh) ^ lo ^ hi;
    return (u64)lo ^ ((u64)mid << 16) ^ ((u64)hi << 32);
}

// 32 x 32 -> 63 bits with four classes (bit positions mod 4): at most 8 terms
// per output position, a count that fits in 4 bits; sixteen 32 x 32 -> 64-bit
// multiplies.  Slower than clmul32 alone but it needs fewer registers: the
// GF(2^128) kernels (m128.cu), whose products hold twice the state, keep it,
// and the fused Butterfly kernel can take either (gf64_mul_t).
__device__ __forceinline__ u64 clmul32_h4(u32 a, u32 b)
{
    const u32 m0 = 0x11111111u, m1 = 0x22222222u, m2 = 0x44444444u, m3 = 0x88888888u;
    const u32 a0 = a & m0, a1 = a & m1, a2 = a & m2, a3 = a & m3;
    const u32 b0 = b & m0, b1 = b & m1, b2 = b & m2, b3 = b & m3;
    const u64 z0 = ((u64)a0 * b0) ^ ((u64)a1 * b3) ^ ((u64)a2 * b2) ^ ((u64)a3 * b1);
    const u64 z1 = ((u64)a0 * b1) ^ ((u64)a1 * b0) ^ ((u64)a2 * b3) ^ ((u64)a3 * b2);
    const u64 z2 = ((u64)a0 * b2) ^ ((u64)a1 * b1) ^ ((u64)a2 * b0) ^ ((u64)a3 * b3);
    const u64 z3 = ((u64)a0 * b3) ^ ((u64)a1 * b2) ^ ((u64)a2 * b1) ^ ((u64)a3 * b0);
    return (z0 & 0x1111111111111111ull) | (z1 & 0x2222222222222222ull) | (z2 & 0x4444444444444444ull) |
           (z3 & 0x8888888888888888ull);
}

// (hi, lo) -> hi * x^64 + lo reduced: x^64 = x^4 + x^3 + x + 1.
__device__ __forceinline__ u64 gf64_reduce(u64 hi, u64 lo)
{
    u64 t = hi ^ (hi << 1) ^ (hi << 3) ^ (hi << 4);
    u64 over = (hi >> 63) ^ (hi >> 61) ^ (hi >> 60);      // bits 64..67 of hi * 0x1B
    t ^= over ^ (over << 1) ^ (over << 3) ^ (over << 4);
    return lo ^ t;
}

// The GF(2^64) product with either integer form of the 32 x 32 carry-less
// product: H4 = false, the 16-bit form (clmul32); H4 = true, the four-class
// 32-bit form (clmul32_h4).  The same result; the fused Butterfly kernel lets
// the tuner pick per launch shape.
template <bool H4>
__device__ __forceinline__ u64 gf64_mul_t(u64 a, u64 b)
{
    u32 al = (u32)a, ah = (u32)(a >> 32), bl = (u32)b, bh = (u32)(b >> 32);
    u64 lo = H4 ? clmul32_h4(al, bl) : clmul32(al, bl);
    u64 hi = H4 ? clmul32_h4(ah, bh) : clmul32(ah, bh);
    u64 mid = (H4 ? clmul32_h4(al ^ ah, bl ^ bh) : clmul32(al ^ ah, bl ^ bh)) ^ lo ^ hi;   // Karatsuba middle term
    return gf64_reduce(hi ^ (mid >> 32), lo ^ (mid << 32));
}

__device__ __forceinline__ u64 gf64_mul(u64 a, u64 b) { return gf64_mul_t<false>(a, b); }

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
//
// In the round of distance j, the lane without bit j (L) keeps the low
// j-bit half of every 2j-bit block and takes its partner's low halves moved
// up by j; the lane with bit j (H) keeps the high halves and takes the
// partner's high halves moved down by j.  So every lane keeps (x & keep) and
// sends its other halves already moved: H rotates them left by j, L right by
// j (no bit wraps around, since the halves sit at the far side of their
// blocks); the rotation is two funnel shifts of the 32-bit halves, with the
// direction a per-lane select, so both kinds of lane run the same code.
__device__ __forceinline__ u64 transpose_round_send(u64 other, bool up, int j)
{
    // rotate right by j (L) or by 64 - j (H: rotate left by j), j <= 16
    const unsigned lo = (unsigned)other, hi = (unsigned)(other >> 32);
    const unsigned p = up ? hi : lo, q = up ? lo : hi;
    const unsigned sh = up ? 32 - j : j;
    return ((u64)__funnelshift_r(q, p, sh) << 32) | __funnelshift_r(p, q, sh);
}

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
        const bool up = (lane & j) != 0;
        const u64 keep = up ? ~masks[s] : masks[s];
        const u64 ka = A & keep, kb = B & keep;
        const u64 sa = transpose_round_send(A ^ ka, up, j), sb = transpose_round_send(B ^ kb, up, j);
        A = ka | __shfl_xor_sync(0xffffffffu, sa, j);
        B = kb | __shfl_xor_sync(0xffffffffu, sb, j);
    }
}

// ------------------------------------------------------ debug bounds checks
// Built with GF2X_DEBUG_BOUNDS, the kernels check their main global indices
// against the extent of the buffer they address: an index out of range is
// counted (per source file) and its access skipped, never trapped;
// gf2x_stream_status then reports GF2X_EBOUNDS.  Without the flag in_range
// is true and costs nothing.
#ifdef GF2X_DEBUG_BOUNDS
static __device__ unsigned long long g_gf2x_out_of_range;
#endif
__device__ __forceinline__ bool in_range(u64 i, u64 extent)
{
#ifdef GF2X_DEBUG_BOUNDS
    if (i >= extent) {
        atomicAdd(&g_gf2x_out_of_range, 1ull);
        return false;
    }
#else
    (void)i;
    (void)extent;
#endif
    return true;
}

// Each file with kernels defines its reader of the counter (host side):
// returns it and resets it to zero; 0 in builds without the checks.
#ifdef GF2X_DEBUG_BOUNDS
#define GF2X_OUT_OF_RANGE_READER(name)                                                        \
    unsigned long long name()                                                                 \
    {                                                                                         \
        unsigned long long h = 0, z = 0;                                                      \
        if (cudaMemcpyFromSymbol(&h, g_gf2x_out_of_range, sizeof h) != cudaSuccess) return 0; \
        if (h) cudaMemcpyToSymbol(g_gf2x_out_of_range, &z, sizeof z);                         \
        return h;                                                                             \
    }
#else
#define GF2X_OUT_OF_RANGE_READER(name) \
    unsigned long long name() { return 0; }
#endif

// ------------------------------------------------------------ block bodies
// The block a kernel body runs as: the launch's own block, or one sub-block of
// the persistent batch kernel (persist.cu), which runs the blocks of many
// launches in one grid.  Bodies take their block index, grid size, thread
// index and thread count from here and synchronise their threads with sync().
// A sub-block is a whole number of warps and has its own named barrier.
struct VBlock {
    unsigned bx, by;      // block index (y: the job of a batch)
    unsigned gx, gy;      // grid size
    unsigned t, nt;       // thread index and threads of the block
    unsigned bar;         // 0: the whole CTA (__syncthreads); else a named barrier for nt threads
    __device__ __forceinline__ void sync() const
    {
        if (bar == 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
    }
};

// The block of an ordinary launch.
__device__ __forceinline__ VBlock launch_block()
{
    return VBlock{blockIdx.x, blockIdx.y, gridDim.x, gridDim.y, threadIdx.x, blockDim.x, 0u};
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

// ------------------------------------------------------- recorded launches
// gf2x_mul_batch can run all its size classes in one persistent launch
// (persist.cu): the host code that would launch a class's kernels records each
// launch instead (its block body, grid, block size, shared memory and
// arguments), and the persistent kernel runs the recorded blocks from a device
// work queue.  Bodies with the same thread count and arguments as the kernels.
enum SegKind {
    SEG_LOAD_JOBS = 0, SEG_STORE_JOBS, SEG_ENCODE, SEG_ENCODE_SMALL, SEG_DECODE, SEG_DECODE_SMALL, SEG_CVT_WIDE,
    SEG_CVT_TILE, SEG_CVT_COL, SEG_CVT_TAYLOR, SEG_UNIT16, SEG_OUTER, SEG_TOP, SEG_BOTTOM, SEG_KIND_COUNT
};

struct SegRec {
    int kind;                 // SegKind
    int i[4];                 // small arguments (template choices, modes)
    unsigned gx, gy;          // grid: gy is the job dimension of the class
    unsigned threads;         // threads per block
    unsigned smem;            // shared memory per block in bytes (static and dynamic)
    unsigned per_job;         // blocks of one job: gx * (gy / jobs)
    int blob;                 // byte offset of extra data in the recorder's blob (a BasisCvt plan), or -1
    u64 a[10];                // pointers and sizes
};

struct Recorder {
    SegRec *segs = nullptr;   // host arrays, grown by record()
    int nseg = 0, cap = 0;
    unsigned char *blob = nullptr;
    size_t blob_bytes = 0, blob_cap = 0;
    int jobs = 0;             // jobs of the class being recorded
    bool unsupported = false; // a launch the persistent kernel cannot run
    ~Recorder();
};

// The recorder of the class being planned, or null (launches run).
inline Recorder *recording(const struct gf2x_ctx *ctx);
// Append one launch; false (and the recorder marked unsupported) on failure.
bool record(struct gf2x_ctx *ctx, const SegRec &r);
// Append bytes to the blob (8-byte aligned); their offset, or -1.
int record_blob(struct gf2x_ctx *ctx, const void *p, size_t n);
// Persistent launches are limited to what one block of the persistent kernel
// can hold: a segment needing more marks the recorder unsupported.
// Device state of a context (one allocation): status word at 0, grid barrier
// at 128, scratch word at 192, the queue of the wait self-test from 1024.
constexpr size_t kStateBytes = 4096;
constexpr size_t kStateQueueOffset = 1024;
// A CTA of the persistent kernel: 256 threads; GF2X_PERSIST_BLOCKS CTAs per SM
// (3: 80 registers a thread, 64 KiB of dynamic shared memory a CTA, bottom
// tiles up to 2^10 points; 4: 64 registers, 46 KiB, tiles up to 2^9 points).
#ifndef GF2X_PERSIST_BLOCKS
#define GF2X_PERSIST_BLOCKS 3
#endif
constexpr unsigned kPersistThreads = 256;
constexpr unsigned kPersistBlocksPerSM = GF2X_PERSIST_BLOCKS;
constexpr unsigned kPersistSmem = kPersistBlocksPerSM >= 4 ? 46 * 1024 : 64 * 1024;
constexpr int kPersistMaxDepth = kPersistBlocksPerSM >= 4 ? 9 : 10;
constexpr unsigned kPersistMaxSegs = 384;            // recorded launches of one class
constexpr size_t kPersistMaxPlanBytes = 64 * 1024;   // BasisCvt plans of one class

// ------------------------------------------------------------------ context
// Stages of Alg. 5 as the profiler and the launch counter see them.
// STAGE_BOTTOM is the fused low-layer kernel of gf2x_mul: the bottom layers of
// both forward Butterflies, the pointwise product and the bottom layers of the
// iButterfly; STAGE_BUTTERFLY / STAGE_IBUTTERFLY then hold the top layers.
// STAGE_PERSIST is the persistent batch kernel, every stage of every job.
enum Gf2xStage {
    STAGE_LOAD = 0, STAGE_BASISCVT, STAGE_ENCODE, STAGE_BUTTERFLY, STAGE_POINTWISE,
    STAGE_IBUTTERFLY, STAGE_DECODE, STAGE_IBASISCVT, STAGE_STORE, STAGE_BOTTOM, STAGE_PERSIST, STAGE_COUNT
};

struct gf2x_ctx {
    int device;
    int num_sms;
    u64 *d_tables;      // one allocation holding the tables below
    void *d_state;      // kStateBytes of device state: status word, barrier, scratch word, self-test queue
    u64 *d_cvt;         // 8 x 256: Cantor coordinates -> polynomial form
    u64 *d_enc;         // 8 x 256: bits (a_{j n_p + i})_j -> f_i  (matrix R)
    u64 *d_dec;         // 8 x 256: f_i -> bits                    (matrix R^{-1})
    u64 *d_cantor;      // v_0 .. v_63
    u64 *d_dec4;        // 16 x 16: R^{-1} in four-bit windows, mul_tab layout (Decode's shared-memory table)
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
    Recorder *rec;                      // set while gf2x_mul_batch records a class (persist.cu)
};

inline Recorder *recording(const gf2x_ctx *ctx) { return ctx->rec; }

// Count one kernel launch against the current stage.
inline void count_launch(gf2x_ctx *ctx, int n = 1) { ctx->launches[ctx->stage] += (unsigned long long)n; }

// ----------------------------------------------------------------- launchers
// All enqueue on `st` and return cudaGetLastError().
namespace gf2x {

// Autotuner (tune.cu).  Knobs: the choices it measures.
// The same numbers as the GF2X_KNOB_* constants of the C ABI.
enum TuneKnob {
    TUNE_UNIT16_R = 1, TUNE_BOTTOM_SHAPE = 2, TUNE_WINDOW_DEPTH = 3, TUNE_M128_BOTTOM_CHUNK = 4, TUNE_BFLY_DEPTH = 5,
    TUNE_M128_BFLY_DEPTH = 6, TUNE_BATCH_PERSIST = 7, TUNE_BOTTOM_MUL = 8, TUNE_CVT_TAYLOR = 9, TUNE_KNOB_END = 10
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
// `side`, if not null, is a second free buffer of `side_words` words per job,
// `side_stride` apart: with it (and taylor_zeta_side_words(K - 16) <=
// side_words), 2^25 <= L <= 2^32 run the Taylor part as two superset-sum passes.
// Where the two-pass Taylor part reads the array (forward) or writes it
// (inverse) when that is not `bits`: the operands of a product read in place
// (job j from src[j], src_bits[j] bits: the last word masked, zeros past it),
// or the product written to dst (ceil(dst_bits / 64) words, the last one
// masked; one job).  A null pointer keeps `bits`.
struct ZetaIO {
    const u64 *src[2] = {nullptr, nullptr};
    u64 src_bits[2] = {0, 0};
    u64 *dst = nullptr;
    u64 dst_bits = 0;
};
cudaError_t basis_cvt(gf2x_ctx *ctx, u64 *bits, u64 L, bool inverse, int count, u64 stride, u64 *scratch,
                      cudaStream_t st, u64 *side = nullptr, u64 side_stride = 0, u64 side_words = 0,
                      const ZetaIO *io = nullptr);
// True when basis_cvt with a scratch buffer and this side buffer runs the
// two-pass Taylor part for length L: its first kernel then reads ZetaIO's
// sources (forward) and its last writes ZetaIO's destination (inverse).
bool basis_cvt_two_pass(gf2x_ctx *ctx, u64 L, u64 side_words);
// Side-buffer words per job the two-pass Taylor part needs for 2^m rows of
// 2^16 bits (9 <= m <= 16), else 0.
u64 taylor_zeta_side_words(int m);
// The Taylor part of BasisCvt / iBasisCvt of length 2^(m + 16) in two passes
// (bits -> scratch and side -> bits); cvt_zeta.cu.
cudaError_t taylor_zeta(gf2x_ctx *ctx, u64 *bits, u64 *scratch, u64 *side, u64 side_stride, int m, bool inverse,
                        int count, u64 stride, cudaStream_t st, const ZetaIO *io = nullptr);
// The Taylor part of the outer conversion (on rows of 2^16 bits) of the same
// length, 10 <= m <= 16, in place on bits with the same side buffer.
cudaError_t outer_taylor_zeta(gf2x_ctx *ctx, u64 *bits, u64 *side, u64 side_stride, int m, bool inverse, int count,
                              u64 stride, cudaStream_t st);
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

// Out-of-range indices the kernels of each file met since the last call
// (GF2X_DEBUG_BOUNDS builds; 0 otherwise).
unsigned long long out_of_range_fft();
unsigned long long out_of_range_cvt();
unsigned long long out_of_range_cvt_reg();
unsigned long long out_of_range_bfly();
unsigned long long out_of_range_persist();
unsigned long long out_of_range_zeta();

// gf2x_mul (same arguments and checks) with every kernel launched directly,
// never through the CUDA graph cache (api.cu).
gf2x_status mul_uncached(gf2x_ctx *ctx, const u64 *a, u64 na, const u64 *b, u64 nb, u64 *c, void *ws,
                         size_t ws_bytes, cudaStream_t st);

// ---- the persistent batch launch (persist.cu)
// Device bytes it needs for `classes` size classes and `jobs` jobs in all: a
// bound that depends on those counts only.
size_t persist_area_bytes(size_t classes, size_t jobs);
// Whether the persistent kernel can run every launch a recorder holds.
bool persist_supported(const Recorder &r);
// The recorded classes, laid out in the device area (256-byte aligned, at
// least persist_area_bytes) by persist_prepare, which uploads them on `st`.
struct PersistLaunch {
    void *segs, *done, *state;
    int nseg;
    unsigned items, grid;
    size_t done_bytes;
    u64 digest;           // of the uploaded plan: launches with equal digests run the same work
};
cudaError_t persist_prepare(gf2x_ctx *ctx, const Recorder *const *recs, int classes, void *area, size_t area_bytes,
                            cudaStream_t st, PersistLaunch *out);
// Clears the queue state and launches the persistent kernel (capturable).
// limit_ns bounds every wait (0: the default of 2 s).
cudaError_t persist_launch(gf2x_ctx *ctx, const PersistLaunch &pl, cudaStream_t st, unsigned long long limit_ns = 0);
// Self-test of the queue's bounded waits: a two-item queue whose second item
// waits on a first that can never finish; the wait runs out after limit_ns and
// records GF2X_ETIMEOUT.  Uses the context's own state area.
cudaError_t persist_selftest_timeout(gf2x_ctx *ctx, cudaStream_t st, unsigned long long limit_ns);

}  // namespace gf2x
