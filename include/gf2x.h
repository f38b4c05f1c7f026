/*
 * gf2x.h -- multiplication of long bit-polynomials in GF(2)[x] on one GB300,
 * by the Frobenius-partition additive FFT of Chen, Cheng, Kuo, Li and Yang,
 * "Multiplying boolean Polynomials with Frobenius Partitions in Additive Fast
 * Fourier Transform" (arXiv 1803.11301).
 *
 * Plain C ABI.  No CUDA, torch or C++ types appear in the signatures: device
 * buffers are passed as plain pointers, streams as `void *` holding a
 * cudaStream_t (NULL = the legacy default stream).
 *
 * Data layout (every entry point)
 *   A bit-polynomial of `nbits` bits is ceil(nbits/64) little-endian uint64
 *   words: bit t of word w is the coefficient of x^(64 w + t).  A vector of
 *   GF(2^64) elements is one uint64 per element, in polynomial form modulo
 *   x^64 + x^4 + x^3 + x + 1 (Sec. 4.3).
 *
 * Sizes (Alg. 5; m = 64, l_m = 6)
 *   nc = na + nb - 1 bits (0 if na or nb is 0) is the product length;
 *   n  = max(64, next power of two >= nc) is the transform length in bits;
 *   l  = log2(n) - 6, n_p = 2^l = n/64 is the number of GF(2^64) points;
 *   alpha = v_{l+32} (Eq. 6), the partition is Sigma = alpha + V_l.
 *   n <= 2^37 (Sec. 3.1 length limit with m = 64), else GF2X_ETOOBIG.
 *
 * Ownership: every data pointer belongs to the caller and must stay valid
 * until the stream has finished the work.  A context owns only its constant
 * tables.  No entry point allocates device memory except gf2x_ctx_create.
 * Calls are asynchronous (enqueue only) unless stated otherwise.
 *
 * Errors: argument errors are returned at once and nothing is enqueued.
 * A CUDA launch error is returned as GF2X_ECUDA.  There is no CPU fallback:
 * without a usable device, gf2x_ctx_create returns GF2X_ENODEV.
 */
#ifndef GF2X_GB300_H
#define GF2X_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GF2X_API __attribute__((visibility("default")))
#else
#define GF2X_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GF2X_OK = 0,
    GF2X_EINVAL = 1,     /* null/misaligned pointer, overlap, bad size */
    GF2X_ETOOBIG = 2,    /* transform length n above 2^37 bits */
    GF2X_ENOMEM = 3,     /* device allocation failed (context creation only) */
    GF2X_ECUDA = 4,      /* a CUDA call or launch failed */
    GF2X_ETIMEOUT = 5,   /* a bounded device-side wait expired */
    GF2X_ENODEV = 6,     /* no usable CUDA device */
    GF2X_ENOSPACE = 7,   /* workspace smaller than gf2x_workspace_bytes() */
    GF2X_EBOUNDS = 8     /* a kernel met an index out of range (builds with GF2X_DEBUG_BOUNDS only) */
} gf2x_status;

typedef struct gf2x_ctx gf2x_ctx;

/* Human-readable name of a status code (static string). */
GF2X_API const char *gf2x_status_string(gf2x_status s);

/* Create a context on CUDA device `device`: computes the Cantor basis
 * (Eq. 2), the Encode matrix and its inverse (Alg. 4, Prop. 2) and the
 * twiddle tables on the host and uploads them.  Synchronous.  The current
 * device of the calling thread is restored on return. */
GF2X_API gf2x_status gf2x_ctx_create(gf2x_ctx **ctx, int device);

/* Free a context (NULL is ignored).  Work enqueued with it must be done. */
GF2X_API void gf2x_ctx_destroy(gf2x_ctx *ctx);

/* Transform length n in bits for operands of na and nb bits (see above);
 * 0 when na or nb is 0. */
GF2X_API uint64_t gf2x_transform_bits(uint64_t na_bits, uint64_t nb_bits);

/* Device workspace in bytes that gf2x_mul needs for these operand lengths
 * (three buffers of n/8 bytes, 256-byte aligned, and 256 bytes reserved for
 * device-side state). */
GF2X_API size_t gf2x_workspace_bytes(uint64_t na_bits, uint64_t nb_bits);

/* c = a * b in GF(2)[x]: FP_Polymul, Alg. 5 (Sec. 3.4), on `stream`.
 *   a, b       device, ceil(na/64) and ceil(nb/64) words; bits at or above
 *              na (nb) in the last word are ignored.  a == b is allowed.
 *   c          device, ceil(nc/64) words; bits at or above nc are written 0.
 *              c must not overlap a, b or the workspace.
 *   workspace  device, >= gf2x_workspace_bytes(na, nb) bytes, 256-aligned;
 *              contents on entry are ignored, on exit undefined.
 * All device pointers 8-byte aligned.  na == 0 or nb == 0 is valid and
 * writes nothing.
 * Repeated calls: from the second call with the same a, b, c, workspace and
 * sizes on, the kernel sequence is replayed from a captured CUDA graph (at
 * most 16 are kept per context, least recently used dropped); the contents of
 * the buffers may change between calls.  Set GF2X_GRAPHS=0 in the environment
 * before creating the context to launch kernels one by one instead.  A context
 * is not thread-safe: serialise calls that share it.
 * First use of a size: some kernels have variants that differ only in speed
 * (threads per block, rows per window); the first call that meets a new launch
 * shape times them on the workspace's free buffers and keeps the fastest, so
 * that call waits for its stream.  Set GF2X_TUNE=0 in the environment before
 * creating the context to use built-in defaults without measuring. */
GF2X_API gf2x_status gf2x_mul(gf2x_ctx *ctx, const uint64_t *a, uint64_t na_bits,
                     const uint64_t *b, uint64_t nb_bits, uint64_t *c,
                     void *workspace, size_t ws_bytes, void *stream);

/* The same product with HOST operands and result, synchronous.  Page-locked
 * (pinned or registered) buffers that are 8-byte aligned, with c apart from a
 * and b, are read and written by the product's load and store kernels
 * directly over the CPU-GPU link; other buffers (pageable, unaligned or
 * overlapping) are copied into the device workspace and the result copied
 * back.  Host pointers need no particular alignment.  Either way the call
 * returns once c holds the product.  The workspace must hold
 * gf2x_host_workspace_bytes(na, nb) bytes. */
GF2X_API size_t gf2x_host_workspace_bytes(uint64_t na_bits, uint64_t nb_bits);
GF2X_API gf2x_status gf2x_mul_host(gf2x_ctx *ctx, const uint64_t *a_host, uint64_t na_bits,
                          const uint64_t *b_host, uint64_t nb_bits, uint64_t *c_host,
                          void *workspace, size_t ws_bytes, void *stream);

/* The product for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a deployment convenience.  Some callers cannot call
 * cudaMalloc or any allocator: a framework that has reserved the whole device
 * for its own memory pool, or a code path where entering an allocator is not
 * allowed.  This call takes no workspace: it runs gf2x_mul's kernels on a fixed
 * scratch array of 3 * GF2X_NOALLOC_MAX_TRANSFORM_BITS / 8 + 256 bytes (768 KiB)
 * that lives in the library's device memory; every GPU that loads the library
 * holds that array until the process exits.  It allocates nothing: the kernels
 * are launched one by one on every call, never from a captured CUDA graph
 * (instantiating one may allocate device memory).
 *   Limit: transform length n <= GF2X_NOALLOC_MAX_TRANSFORM_BITS (2^21 bits,
 *   e.g. two operands of 2^20 bits); larger products return GF2X_ETOOBIG and
 *   enqueue nothing.  Other arguments and results as for gf2x_mul.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Sharing: all calls, on every stream of a device, use the same array, which
 *   keeps the last call's contents (a call never reads scratch it has not
 *   written).  Calls whose work overlaps on the GPU race on the array: order
 *   them on one stream, or synchronise between them. */
#define GF2X_NOALLOC_MAX_TRANSFORM_BITS (1ull << 21)
GF2X_API gf2x_status gf2x_mul_noalloc(gf2x_ctx *ctx, const uint64_t *a, uint64_t na_bits,
                                      const uint64_t *b, uint64_t nb_bits, uint64_t *c,
                                      void *stream);

/* Reusing one operand.  When many products share the operand b, its forward
 * transform -- the steps BasisCvt, Encode, Butterfly of Alg. 5, i.e. the
 * values B(alpha + u_k) of Eq. 8 at the n_p points of Sigma -- can be
 * computed once and passed to every product, which then skips them.
 *
 * gf2x_transform_bytes(n_bits): bytes of a transform at transform length
 * n_bits (n_bits / 8, one uint64 per point), 0 unless n_bits is a power of
 * two with 64 <= n_bits <= 2^37.
 *
 * gf2x_transform_workspace_bytes(n_bits): the device workspace that
 *   gf2x_forward_transform needs at transform length n_bits (3 buffers of
 *   n_bits/8 bytes and 256 bytes of device state; the same as a product with
 *   that transform length), 0 when gf2x_transform_bytes is 0.
 *
 * gf2x_forward_transform: bhat (device, gf2x_transform_bytes(n_bits) bytes,
 *   8-byte aligned, disjoint from b and the workspace) <- the transform of b
 *   (nb_bits bits, 1 <= nb_bits <= n_bits) at length n_bits.  Use n_bits =
 *   gf2x_transform_bits(na, nb_bits) for products with na-bit operands; the
 *   workspace must hold gf2x_transform_workspace_bytes(n_bits) bytes,
 *   256-aligned (the workspace of such a product suffices).  Asynchronous.
 *
 * gf2x_mul_transformed: c = a * b, with b given as bhat = its transform at
 *   gf2x_transform_bits(na_bits, nb_bits) (the caller keeps bhat consistent
 *   with b and that length; the library cannot check it).  bhat is only
 *   read.  Other arguments, sizes and errors as for gf2x_mul; c must not
 *   overlap bhat.  Both calls replay from a captured CUDA graph from the
 *   second identical call on, like gf2x_mul.  The paper has no separate
 *   entry point for this; it is Alg. 5 with b's forward steps done
 *   ahead of time. */
GF2X_API size_t gf2x_transform_bytes(uint64_t n_bits);
GF2X_API size_t gf2x_transform_workspace_bytes(uint64_t n_bits);
GF2X_API gf2x_status gf2x_forward_transform(gf2x_ctx *ctx, const uint64_t *b, uint64_t nb_bits, uint64_t n_bits,
                                            uint64_t *bhat, void *workspace, size_t ws_bytes, void *stream);
GF2X_API gf2x_status gf2x_mul_transformed(gf2x_ctx *ctx, const uint64_t *a, uint64_t na_bits, const uint64_t *bhat,
                                          uint64_t nb_bits, uint64_t *c, void *workspace, size_t ws_bytes,
                                          void *stream);

/* One product of a batch: c = a * b, pointers and lengths as for gf2x_mul. */
typedef struct gf2x_job {
    const uint64_t *a;
    uint64_t na_bits;
    const uint64_t *b;
    uint64_t nb_bits;
    uint64_t *c;
} gf2x_job;

/* Device workspace for gf2x_mul_batch on these jobs (0 if a job is invalid
 * or too long).  Depends on the lengths only. */
GF2X_API size_t gf2x_batch_workspace_bytes(const gf2x_job *jobs, size_t count);

/* Many independent products of uneven lengths in one call (Alg. 5 for each).
 * The jobs are grouped by transform length n (size classes).  Two ways to
 * run them, with the same results:
 *   - one launch per kernel and class (the kernels' second grid dimension is
 *     the job);
 *   - ONE persistent kernel launch for the whole batch: the host plans every
 *     class's stages (load, BasisCvt, Encode, Butterfly with the pointwise
 *     product, Decode, iBasisCvt, store) as a device work queue, which a grid
 *     of three blocks per SM drains; a job's next stage starts as soon as that
 *     job's previous stage is done, and classes run side by side.  Every wait
 *     in the queue is bounded: if one runs out (it cannot in a correct plan)
 *     the launch records GF2X_ETIMEOUT in the context status word
 *     (gf2x_stream_status) and returns without finishing the batch.
 * GF2X_KNOB_BATCH_PERSISTENT pins the choice; otherwise the first batch of
 * each shape (job and class counts in power-of-two buckets) times both and the
 * faster is kept (the class launches unless the persistent launch is more than
 * 3% faster), like the other launch shapes.  Batches with transforms above
 * 2^25 bits always run class launches (the persistent kernel lacks their
 * launch shapes).  The host array `jobs` is read during the call and
 * copied to the workspace, with the queue; every device buffer follows the
 * gf2x_mul rules (8-byte aligned, c disjoint from a, b and the workspace;
 * jobs may share operands but not results).  Jobs with na or nb = 0 write
 * nothing.  Asynchronous.  From the second call with the same jobs (pointers
 * and lengths), workspace and plan on, the launches replay from a captured
 * CUDA graph (at most 8 kept per context). */
GF2X_API gf2x_status gf2x_mul_batch(gf2x_ctx *ctx, const gf2x_job *jobs, size_t count,
                                    void *workspace, size_t ws_bytes, void *stream);

/* Self-test of the bounded device-side waits: launches one block that waits
 * on a grid barrier for an arrival that never comes.  The wait gives up after
 * a short limit (milliseconds), records GF2X_ETIMEOUT in the context status
 * word and returns, so the context stays usable; read it with
 * gf2x_stream_status.  The paper has no counterpart (failure detection). */
GF2X_API gf2x_status gf2x_selftest_wait_timeout(gf2x_ctx *ctx, void *stream);

/* Self-test of the persistent batch queue's bounded waits: launches a
 * two-item queue whose second item waits on a first that can never finish.
 * The wait gives up after 20 ms, records GF2X_ETIMEOUT in the context status
 * word and the kernel returns; the context stays usable.  The paper has no
 * counterpart (failure detection). */
GF2X_API gf2x_status gf2x_selftest_queue_timeout(gf2x_ctx *ctx, void *stream);

/* Read, and reset to GF2X_OK, the context's device status word after the
 * work already enqueued on `stream` has finished (synchronises the stream).
 * Device code records bounded-wait expiry (GF2X_ETIMEOUT) there; it never
 * traps.  A library built with GF2X_DEBUG_BOUNDS also range-checks the
 * kernels' main global indices (an index out of range is counted and its
 * access skipped); this call then returns GF2X_EBOUNDS if any was met since
 * the last call, and resets the counts. */
GF2X_API gf2x_status gf2x_stream_status(gf2x_ctx *ctx, void *stream);

/* Launch shapes (bottom-tile depth, block shapes, table chunks, BasisCvt
 * words per thread) are measured on first use of each shape class, which
 * synchronises the stream once; later calls reuse the choice.  With
 * frozen != 0 the context measures nothing new (stored choices, else the
 * built-in defaults): for servers, after a warm-up.  frozen = 0 resumes.
 * GF2X_TUNE=0 in the environment at context creation never measures. */
GF2X_API gf2x_status gf2x_tune_freeze(gf2x_ctx *ctx, int frozen);

/* Pinning one launch choice, for reproducible launch shapes and for testing
 * every variant.  Wherever `choice` is one of the knob's candidates for a call
 * it is used without measuring; elsewhere (a depth deeper than the transform,
 * say) the tuner decides as before.  choice = -1 releases the knob.  Graphs
 * captured before the call are not replayed again (the next calls capture
 * anew).  Knobs and their candidates, all computing the same result:
 *   GF2X_KNOB_UNIT16_R           words per thread of the 2^16-bit BasisCvt kernel: 8, 16, 32
 *   GF2X_KNOB_BOTTOM_SHAPE       fused bottom kernel: 0 (256 threads, 16-table chunks),
 *                                1 (512 threads, 32), 2 (256 threads, 8)
 *   GF2X_KNOB_WINDOW_DEPTH       Taylor layers in BasisCvt's window kernel: 6, 7, 8
 *   GF2X_KNOB_M128_BOTTOM_CHUNK  GF(2^128) bottom kernel tables per chunk: 4, 8
 *   GF2X_KNOB_BOTTOM_DEPTH       Butterfly layers in the bottom kernel: 8 .. 11
 *   GF2X_KNOB_M128_BOTTOM_DEPTH  the same for GF(2^128) points: 8 .. 10
 *   GF2X_KNOB_BATCH_PERSISTENT   gf2x_mul_batch: 1 (one persistent launch) or 0 (one
 *                                launch per kernel and size class)
 *   GF2X_KNOB_BOTTOM_MUL         the GF(2^64) products of the fused bottom kernel's
 *                                integer layers and pointwise step: 0 (16x16-bit integer
 *                                multiplies on operands with holes), 1 (32x32-bit ones)
 *   GF2X_KNOB_CVT_TAYLOR         the Taylor parts of BasisCvt / iBasisCvt at lengths
 *                                2^25 .. 2^32 inside a product (at 2^16-bit rows and, from
 *                                2^26 on, at 2^24-bit blocks of the outer conversion):
 *                                1 (superset-sum passes over HBM, the default), 0 (the
 *                                division steps of Alg. 1, one or two per pass)
 * GF2X_EINVAL for a NULL context, an unknown knob or choice < -1.  Not
 * thread-safe against calls running on the same context. */
enum {
    GF2X_KNOB_UNIT16_R = 1,
    GF2X_KNOB_BOTTOM_SHAPE = 2,
    GF2X_KNOB_WINDOW_DEPTH = 3,
    GF2X_KNOB_M128_BOTTOM_CHUNK = 4,
    GF2X_KNOB_BOTTOM_DEPTH = 5,
    GF2X_KNOB_M128_BOTTOM_DEPTH = 6,
    GF2X_KNOB_BATCH_PERSISTENT = 7,
    GF2X_KNOB_BOTTOM_MUL = 8,
    GF2X_KNOB_CVT_TAYLOR = 9
};
GF2X_API gf2x_status gf2x_tune_pin(gf2x_ctx *ctx, int knob, int choice);

/* Butterfly layers (Alg. 2) that gf2x_mul runs in its fused low-layer kernel
 * for an na x nb product, the rest running as passes over HBM: the depth the
 * context's tuner measured at the first product of this transform length, or
 * the default before that.  -1 for a NULL context or an empty or too long
 * product.  Informational (profiling and roofline accounting). */
GF2X_API int gf2x_bottom_layers(gf2x_ctx *ctx, uint64_t na_bits, uint64_t nb_bits);

/* Field-multiply measurement (a benchmark, not part of the product path): the
 * GF(2^64) product forms this GPU offers, timed on the same work.  The paper
 * multiplies with PCLMULQDQ (Sec. 4.3) and, by a fixed element, with 4-bit
 * table lookups (Sec. 4.5); GB300 has no carry-less multiply instruction.
 * Every variant runs 4 dependent chains x <- c x per thread (one fixed c) for
 * `steps` steps (1 .. 2^20) over 8 blocks of 256 threads per SM, one launch
 * on `stream` timed with CUDA events after an untimed launch; all variants
 * give the same *checksum (an XOR of the final values).  *ms = the launch's
 * time, *products = the field products it computed.  Synchronous.
 *   variant 0  32x32 integer multiplies on operands with 3-bit holes, Karatsuba
 *              (the library's earlier integer form)
 *           1  the same with the fixed operand's masks computed once
 *           2  16 four-bit windows of a per-element table in shared memory
 *              (the form the Butterfly kernels use for shared twiddles)
 *           3  8 eight-bit windows (2 KiB per window)
 *           4  low half by four-bit windows, high half by integer multiplies
 *           5  16x16 integer multiplies on operands with 2-bit holes, Karatsuba
 *              twice (the integer form the library uses)
 *           6  64 elements of a warp bit-sliced across its lanes; the product
 *              by c as its 64x64 GF(2) matrix, planes fetched by warp shuffles
 * GF2X_EINVAL for a NULL pointer, an unknown variant or steps out of range. */
GF2X_API gf2x_status gf2x_bench_field_mul(gf2x_ctx *ctx, int variant, int steps, uint64_t *checksum,
                                          double *ms, uint64_t *products, void *stream);

/* ------------------------------------------------------------------------
 * Per-stage profiling.  Stage k (0 <= k < gf2x_stage_count()) is one step of
 * Alg. 5 as named by gf2x_stage_name(k): load, basis_cvt, encode, butterfly,
 * pointwise, ibutterfly, decode, ibasis_cvt, store, bottom_fused (the fused
 * low Butterfly layers and pointwise product), persistent_batch (the whole
 * persistent batch launch).
 * ---------------------------------------------------------------------- */
GF2X_API int gf2x_stage_count(void);
GF2X_API const char *gf2x_stage_name(int stage);

/* Reset the per-stage times and kernel-launch counters; with enable != 0,
 * also bracket every later stage with a pair of CUDA events recorded on the
 * stream that stage's kernels are launched on.  Launches are counted
 * whether or not timing is enabled.  Synchronises with events already
 * recorded. */
GF2X_API gf2x_status gf2x_profile_enable(gf2x_ctx *ctx, int enable);

/* Sum the recorded stage times (milliseconds) into ms[k] and copy the kernel
 * launch counts into launches[k], k < min(max_stages, stage count).  Waits
 * for the recorded events.  Either pointer may be NULL.  Returns the number
 * of stages, or -1 for a NULL context. */
GF2X_API int gf2x_profile_read(gf2x_ctx *ctx, double *ms, uint64_t *launches, int max_stages);

/* ------------------------------------------------------------------------
 * Stages of Alg. 5, exposed one by one (device pointers, enqueue only).
 * They compute exactly what gf2x_mul computes internally and exist so that
 * each step can be checked on its own.
 * ---------------------------------------------------------------------- */

/* BasisCvt, Alg. 1 (Sec. 2.3.1): monomial -> novelpoly basis, in place on
 * the first L bits of `bits` (L a power of two, 64 <= L <= 2^37).  Bit k of
 * the result is the coefficient of X_k.  Only XORs; GF(2)-linear. */
GF2X_API gf2x_status gf2x_basis_cvt(gf2x_ctx *ctx, uint64_t *bits, uint64_t L_bits, void *stream);

/* iBasisCvt: the inverse map (novelpoly -> monomial), in place. */
GF2X_API gf2x_status gf2x_ibasis_cvt(gf2x_ctx *ctx, uint64_t *bits, uint64_t L_bits, void *stream);

/* Encode, Alg. 4 (Sec. 3.3): f_i = sum_j a_{j n_p + i} r_j for i < n_p, with
 * r_j = prod_t s_{l+t}(alpha)^{j_t} (the first l_m truncated butterfly
 * layers; see Sec. 3.2).  `novel` holds n bits (n/64 words); f receives n_p
 * elements.  No overlap allowed. */
GF2X_API gf2x_status gf2x_encode(gf2x_ctx *ctx, const uint64_t *novel, uint64_t n_bits,
                        uint64_t *f, void *stream);

/* Decode: the inverse of Encode (uses R^{-1}, Prop. 2): n_p elements ->
 * n bits.  No overlap allowed. */
GF2X_API gf2x_status gf2x_decode(gf2x_ctx *ctx, const uint64_t *h, uint64_t n_bits,
                        uint64_t *novel, void *stream);

/* Butterfly, Alg. 2 (Sec. 2.3.2) at alpha = v_{l+32}, in place on n_p
 * elements: output k is f(alpha + u_k), u_k the element with Cantor
 * coordinates k. */
GF2X_API gf2x_status gf2x_butterfly(gf2x_ctx *ctx, uint64_t *f, uint64_t n_bits, void *stream);

/* iButterfly: the inverse of gf2x_butterfly, in place. */
GF2X_API gf2x_status gf2x_ibutterfly(gf2x_ctx *ctx, uint64_t *f, uint64_t n_bits, void *stream);

/* Pointwise product in GF(2^64) (pointwise step of Alg. 5): c[i] = a[i] * b[i],
 * i < count.  c may alias a or b. */
GF2X_API gf2x_status gf2x_pointwise(gf2x_ctx *ctx, const uint64_t *a, const uint64_t *b,
                           uint64_t *c, uint64_t count, void *stream);

/* ------------------------------------------------------------------------
 * The same method with m = 128 (Sec. 3 is written for general m; Sec. 4.3
 * names GF(2^128) = GF(2)[x] / (x^128 + x^7 + x^2 + x + 1)).
 *
 * Sizes: n = max(128, next power of two >= nc); l = log2(n) - 7; n_p = 2^l =
 * n/128 points; alpha = v_{l+64}, Sigma = alpha + V_l (Eq. 6 with m/2 = 64);
 * Encode collapses l_m = 7 layers.  n <= 2^38, else GF2X_ETOOBIG: the
 * Sec. 3.1 limit with m = 128, (m/2) 2^(m/2) = 2^70 bits, does not bind; one
 * GB300's memory does (a 2^37 x 2^37-bit product holds 160 GB).
 *
 * A vector of GF(2^128) elements is two uint64 words per element, low word
 * (coefficients of x^0..x^63) first, so n_p points take n/64 words, the size
 * of the n-bit array.  Element buffers must be 16-byte aligned.  The Cantor
 * basis v_0..v_127 (Eq. 2) takes, at each step, the root with bit 0 clear.
 * ---------------------------------------------------------------------- */

/* Transform length n in bits for an na x nb product by the m = 128 method (0 if
 * either length is 0). */
GF2X_API uint64_t gf2x_m128_transform_bits(uint64_t na_bits, uint64_t nb_bits);

/* As gf2x_bottom_layers, for gf2x_mul_m128. */
GF2X_API int gf2x_m128_bottom_layers(gf2x_ctx *ctx, uint64_t na_bits, uint64_t nb_bits);

/* Device workspace for gf2x_mul_m128: 3 n/8 bytes + 256 (0 if n > 2^38). */
GF2X_API size_t gf2x_m128_workspace_bytes(uint64_t na_bits, uint64_t nb_bits);

/* c = a * b in GF(2)[x] by Alg. 5 with m = 128: BasisCvt (Alg. 1, shared with
 * m = 64), Encode into GF(2^128) elements, Butterfly on Sigma = v_{l+64} + V_l,
 * pointwise GF(2^128) products, and back.  Same contract as gf2x_mul
 * (arguments, layout of a, b, c, workspace alignment, no overlap of c with a,
 * b or ws, graph replay of repeated calls).  The result equals gf2x_mul's
 * bit for bit; a == b runs the transform too. */
GF2X_API gf2x_status gf2x_mul_m128(gf2x_ctx *ctx, const uint64_t *a, uint64_t na_bits,
                          const uint64_t *b, uint64_t nb_bits, uint64_t *c,
                          void *workspace, size_t workspace_bytes, void *stream);

/* Encode with m = 128: f_i = sum_{j<128} a_{j n_p + i} r_j (i < n_p), r_j =
 * prod_{t<7} s_{l+t}(alpha)^{j_t} = prod_{t<7} v_{64-t}^{j_t}.  `novel`: n bits
 * (8-byte aligned); f: n_p elements (16-byte aligned).  No overlap allowed. */
GF2X_API gf2x_status gf2x_m128_encode(gf2x_ctx *ctx, const uint64_t *novel, uint64_t n_bits,
                             uint64_t *f, void *stream);

/* Decode with m = 128: the inverse of gf2x_m128_encode (n_p elements -> n bits). */
GF2X_API gf2x_status gf2x_m128_decode(gf2x_ctx *ctx, const uint64_t *h, uint64_t n_bits,
                             uint64_t *novel, void *stream);

/* Butterfly (Alg. 2) on n_p GF(2^128) elements at alpha = v_{l+64}, in place:
 * output k is f(alpha + u_k), u_k the element with Cantor coordinates k. */
GF2X_API gf2x_status gf2x_m128_butterfly(gf2x_ctx *ctx, uint64_t *f, uint64_t n_bits, void *stream);

/* The inverse of gf2x_m128_butterfly, in place. */
GF2X_API gf2x_status gf2x_m128_ibutterfly(gf2x_ctx *ctx, uint64_t *f, uint64_t n_bits, void *stream);

/* Pointwise product in GF(2^128): c[i] = a[i] * b[i], i < count elements
 * (2 count words each; 16-byte aligned).  c may alias a or b. */
GF2X_API gf2x_status gf2x_m128_pointwise(gf2x_ctx *ctx, const uint64_t *a, const uint64_t *b,
                                uint64_t *c, uint64_t count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GF2X_GB300_H */
