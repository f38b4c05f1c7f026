// C ABI of the GB300 GF(2)[x] multiplier (declared in include/gf2x.h) and
// the host-side set-up: Cantor basis, Encode matrix R and its inverse,
// Cantor-to-polynomial table.
//
// FP_Polymul (Alg. 5) on one stream, three workspace buffers X, Y, T of n/64
// words each:
//   T <- a (masked, zero-padded to n bits); BasisCvt(T, L_a); X <- Encode(T)
//   T <- b ...;                                       Y <- Encode(T)   (BasisCvt, Encode)
//   top Butterfly layers of X and Y                                    (Butterfly)
//   one kernel per 2^11-point tile: low layers of both Butterflies,
//     X <- X * Y, low layers of the iButterfly                        (Butterfly, pointwise, iButterfly)
//   top iButterfly layers of X; T <- Decode(X); iBasisCvt(T, n); c <- T (the inverse steps)
// BasisCvt runs on L_a = max(64, next_pow2(na)) bits: the novelpoly basis
// is triangular (deg X_k = k), so the coefficients at k >= L_a are zero.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "gf2x_common.cuh"

namespace {

constexpr u64 kMaxTransformBits = 1ull << 37;    // Sec. 3.1 length limit, m = 64
// m = 128: the Sec. 3.1 limit is 2^70 bits; the cap is one GB300's memory:
// a product at n = 2^38 holds 3 n/8 bytes of workspace plus n/2 of operands
// and result, 160 GB of the 288 GB (n = 2^39 would need 320 GB).
constexpr u64 kMaxTransformBits128 = 1ull << 38;
constexpr size_t kAlign = 256;

// ------------------------------------------------------------ host GF(2^64)
u64 hmul(u64 a, u64 b)
{
    u64 r = 0;
    for (int t = 0; t < 64; ++t) {
        if ((b >> t) & 1) r ^= a;
        a = (a << 1) ^ ((a >> 63) ? GF2X_MOD_LOW : 0);
    }
    return r;
}

// Solve sum_k y_k img[k] = rhs over GF(2); one solution or false.
bool gf2_solve(const u64 img[64], u64 rhs, u64 *y)
{
    u64 eq[64];          // equation for bit position p: coefficient mask over k
    int rhsb[64];
    for (int p = 0; p < 64; ++p) {
        u64 m = 0;
        for (int k = 0; k < 64; ++k) m |= ((img[k] >> p) & 1ull) << k;
        eq[p] = m;
        rhsb[p] = (int)((rhs >> p) & 1);
    }
    int piv_col[64];
    int rank = 0;
    for (int col = 0; col < 64 && rank < 64; ++col) {
        int piv = -1;
        for (int r = rank; r < 64; ++r)
            if ((eq[r] >> col) & 1) { piv = r; break; }
        if (piv < 0) continue;
        std::swap(eq[rank], eq[piv]);
        std::swap(rhsb[rank], rhsb[piv]);
        for (int r = 0; r < 64; ++r)
            if (r != rank && ((eq[r] >> col) & 1)) { eq[r] ^= eq[rank]; rhsb[r] ^= rhsb[rank]; }
        piv_col[rank++] = col;
    }
    for (int r = rank; r < 64; ++r)
        if (rhsb[r]) return false;
    u64 sol = 0;
    for (int r = 0; r < rank; ++r)
        if (rhsb[r]) sol |= 1ull << piv_col[r];
    *y = sol;
    return true;
}

// rows of A^{-1} for the 64x64 GF(2) matrix with rows a[] (row-vector convention)
bool gf2_inverse(const u64 a_in[64], u64 inv[64])
{
    u64 a[64];
    for (int k = 0; k < 64; ++k) { a[k] = a_in[k]; inv[k] = 1ull << k; }
    for (int col = 0; col < 64; ++col) {
        int piv = -1;
        for (int r = col; r < 64; ++r)
            if ((a[r] >> col) & 1) { piv = r; break; }
        if (piv < 0) return false;
        std::swap(a[col], a[piv]);
        std::swap(inv[col], inv[piv]);
        for (int r = 0; r < 64; ++r)
            if (r != col && ((a[r] >> col) & 1)) { a[r] ^= a[col]; inv[r] ^= inv[col]; }
    }
    return true;
}

// v_0 = 1, v_i^2 + v_i = v_{i-1} (Eq. 2); of the two roots y, y + 1 take the
// one with bit 0 clear.
bool cantor_basis(u64 v[64])
{
    u64 img[64];
    for (int k = 0; k < 64; ++k) {
        u64 e = 1ull << k;
        img[k] = hmul(e, e) ^ e;
    }
    v[0] = 1;
    for (int i = 1; i < 64; ++i) {
        u64 y;
        if (!gf2_solve(img, v[i - 1], &y)) return false;
        v[i] = y & ~1ull;
    }
    return true;
}

void window_table(const u64 rows[64], u64 *tab)
{
    for (int k = 0; k < 8; ++k)
        for (int x = 0; x < 256; ++x) {
            u64 r = 0;
            for (int b = 0; b < 8; ++b)
                if ((x >> b) & 1) r ^= rows[8 * k + b];
            tab[k * 256 + x] = r;
        }
}

// Four-bit windows of a 64 x 64 GF(2) matrix in the layout of the Butterfly
// kernels' multiplication tables (mul_tab): window k holds, at slot x ^ k, the
// XOR of rows 4k + b over the bits b of x (16 windows of 16 words: one window
// spans the 32 shared-memory banks, so lanes reading one window never conflict).
void window_table4(const u64 rows[64], u64 *tab)
{
    for (int k = 0; k < 16; ++k)
        for (int x = 0; x < 16; ++x) {
            u64 r = 0;
            for (int b = 0; b < 4; ++b)
                if ((x >> b) & 1) r ^= rows[4 * k + b];
            tab[k * 16 + (x ^ k)] = r;
        }
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

u64 next_pow2(u64 x)
{
    u64 p = 1;
    while (p < x) p <<= 1;
    return p;
}

int log2_u64(u64 x)
{
    int k = 0;
    while ((1ull << k) < x) ++k;
    return k;
}

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool aligned8(const void *p) { return ((uintptr_t)p & 7) == 0; }
bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

bool overlap(const void *p, size_t pb, const void *q, size_t qb)
{
    uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
    return pb && qb && a < b + qb && b < a + pb;
}

gf2x_status from_cuda(cudaError_t e) { return e == cudaSuccess ? GF2X_OK : GF2X_ECUDA; }

#define TRY(expr)                                                 \
    do {                                                          \
        cudaError_t e_ = (expr);                                  \
        if (e_ != cudaSuccess) return GF2X_ECUDA;                 \
    } while (0)

u64 product_bits(u64 na, u64 nb) { return (na && nb) ? na + nb - 1 : 0; }

u64 transform_bits(u64 na, u64 nb)
{
    u64 nc = product_bits(na, nb);
    if (!nc) return 0;
    u64 n = next_pow2(nc);
    return n < 64 ? 64 : n;
}

size_t buffer_bytes(u64 n) { return round_up((size_t)(n / 8)); }

// ------------------------------------------------------------- profiling
// Optional per-stage timing: a pair of CUDA events around every stage,
// recorded on the stream the stage's kernels are launched on, summed per
// stage by gf2x_profile_read.  Inside a captured CUDA graph the pair becomes
// two event-record nodes (external events owned by the graph entry), so the
// times of a replay are read the same way.
struct Rec {
    int stage;
    cudaEvent_t e0, e1;
    bool pooled;                        // events return to the pool after reading
};

struct Profiler {
    std::vector<cudaEvent_t> pool;      // free events
    std::vector<Rec> pending;           // recorded, not yet read
    double ms[STAGE_COUNT] = {};
    std::vector<Rec> *capture = nullptr; // set while a graph is being captured
    Rec open{};
    bool is_open = false;
};

Profiler *profiler(gf2x_ctx *ctx) { return (Profiler *)ctx->prof; }

cudaEvent_t take_event(Profiler *p)
{
    cudaEvent_t e = nullptr;
    if (p->capture || p->pool.empty()) {
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    e = p->pool.back();
    p->pool.pop_back();
    return e;
}

void record(Profiler *p, cudaEvent_t e, cudaStream_t st)
{
    if (p->capture) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
}

void stage_begin(gf2x_ctx *ctx, int stage, cudaStream_t st)
{
    ctx->stage = stage;
    if (!ctx->profiling || ctx->rec) return;
    Profiler *p = profiler(ctx);
    cudaEvent_t e = take_event(p);
    if (!e) return;
    p->open = Rec{stage, e, nullptr, p->capture == nullptr};
    p->is_open = true;
    record(p, e, st);
}

void stage_end(gf2x_ctx *ctx, cudaStream_t st)
{
    if (!ctx->profiling || ctx->rec) return;
    Profiler *p = profiler(ctx);
    if (!p->is_open) return;
    p->is_open = false;
    cudaEvent_t e = take_event(p);
    if (!e) return;
    p->open.e1 = e;
    record(p, e, st);
    (p->capture ? p->capture : &p->pending)->push_back(p->open);
}

struct StageScope {
    gf2x_ctx *ctx;
    cudaStream_t st;
    StageScope(gf2x_ctx *c, int stage, cudaStream_t s) : ctx(c), st(s) { stage_begin(c, stage, s); }
    ~StageScope() { stage_end(ctx, st); }
};

// ---------------------------------------------------------- graph cache
// gf2x_mul replays a captured CUDA graph when it is called again with the same
// operands, result, workspace and sizes: the second such call captures the
// kernel sequence on a private stream and every later call launches the graph
// into the caller's stream (one launch instead of ~15-40).
// What a cached sequence computes (the arguments are read accordingly).
enum OpKind {
    OP_MUL = 0,               // c = a * b
    OP_MUL_TRANSFORMED = 1,   // c = a * b, b given as its transform at b's pointer
    OP_FORWARD_TRANSFORM = 2, // c = transform of a (na bits) at length nb
    OP_MUL128 = 3             // c = a * b by the m = 128 method
};

struct GraphEntry {
    int kind;
    const u64 *a, *b;
    u64 na, nb;
    u64 *c;
    void *ws;
    bool profiling;
    unsigned gen;           // GraphCache::gen at capture
    cudaGraphExec_t exec;
    unsigned long long launches[STAGE_COUNT];
    std::vector<Rec> recs;
    unsigned long long stamp;
};

struct GraphCache {
    std::vector<GraphEntry> entries;
    struct Key { int kind; const u64 *a, *b; u64 na, nb; u64 *c; void *ws; };
    std::vector<Key> seen;              // keys called once, not captured yet
    cudaStream_t cap = nullptr;
    unsigned long long clock = 0;
    unsigned gen = 0;                   // bumped by gf2x_tune_pin: older graphs hold other launch shapes
    bool disabled = false;
};

constexpr size_t kMaxGraphs = 16;

GraphCache *graphs(gf2x_ctx *ctx) { return (GraphCache *)ctx->graphs; }

void destroy_entry(GraphEntry &g)
{
    cudaGraphExecDestroy(g.exec);
    for (Rec &r : g.recs) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
}

// One size class: `count` products with the same transform length n, whose
// buffers X, Y, T (count x stride words each) hold the jobs one after
// another.  Either a device job table (a batch) or direct pointers (count 1).
struct ClassRun {
    u64 n;
    int count;
    u64 La, Lb;                     // BasisCvt lengths (>= every operand of the class)
    const JobDev *jobs;             // device job table, or null
    const u64 *a, *b;               // direct operands when jobs is null
    u64 na, nb;
    u64 *c;
    u64 max_c_words;                // longest product of the class, in words
    u64 *X, *Y, *T;
    u64 stride;                     // words between the buffers of consecutive jobs
};

// Words of one job's X, Y or T buffer.
u64 buffer_words(const ClassRun &r) { return r.count == 1 && r.stride == 0 ? buffer_bytes(r.n) / 8 : r.stride; }

// Set while gf2x_mul_host runs a product on page-locked host memory mapped
// into the device: its operands and product stay with the load and store
// kernels (linear streams over the host link) instead of being read and
// written in place by BasisCvt's first and iBasisCvt's last kernel, whose
// band-shaped accesses suit device memory.  (Calls on one context are not
// concurrent, and a cached graph keys on these host pointers.)
thread_local bool t_mapped_host = false;

// Lines 1-2 (or 4-5) of Alg. 5 for one operand of every job: load, BasisCvt, Encode.
gf2x_status forward(gf2x_ctx *ctx, const ClassRun &r, int which, u64 *F, cudaStream_t st)
{
    const int l = log2_u64(r.n) - 6;
    const u64 L = which ? r.Lb : r.La;
    // F (the Encode output, free until then) is the scratch buffer of BasisCvt;
    // its side buffer is Y for a (free until b's forward steps) and, for b, the
    // words of T above L (Encode reads only the first L bits).  With the
    // two-pass Taylor part a single product's operand is read in place by
    // BasisCvt's first kernel, and the load kernel is not needed.
    const u64 words = buffer_words(r);
    u64 *side = which ? r.T + L / 64 : r.Y;
    const u64 side_words = which ? words - L / 64 : words;
    gf2x::ZetaIO io;
    const bool direct = !t_mapped_host && !r.jobs && r.count == 1 && gf2x::basis_cvt_two_pass(ctx, L, side_words);
    if (direct) {
        io.src[0] = which ? r.b : r.a;
        io.src_bits[0] = which ? r.nb : r.na;
    } else {
        StageScope s(ctx, STAGE_LOAD, st);
        if (r.jobs) TRY(gf2x::load_jobs(ctx, r.jobs, which, r.T, r.stride, r.n / 64, r.count, st));
        else TRY(gf2x::load_bits(ctx, which ? r.b : r.a, which ? r.nb : r.na, r.T, r.n / 64, st));
    }
    {
        StageScope s(ctx, STAGE_BASISCVT, st);
        TRY(gf2x::basis_cvt(ctx, r.T, L, false, r.count, r.stride, F, st, side, r.stride, side_words,
                            direct ? &io : nullptr));
    }
    { StageScope s(ctx, STAGE_ENCODE, st); TRY(gf2x::encode(ctx, r.T, l, F, L, r.count, r.stride, r.stride, st)); }
    return GF2X_OK;
}

// Lines 1-2 and 4-5 of Alg. 5 for both operands of one product in the same
// launches, when they convert at the same length L <= n/2: a in the lower half
// of T and b in the upper half (two jobs n/128 words apart); BasisCvt's scratch
// is X with the same layout; Encode writes a's points to X and b's to Y.
gf2x_status forward_pair(gf2x_ctx *ctx, const ClassRun &r, cudaStream_t st)
{
    const int l = log2_u64(r.n) - 6;
    const u64 half = r.n / 128;
    // with the two-pass Taylor part BasisCvt's first kernel reads a and b in place
    gf2x::ZetaIO io;
    const bool direct = !t_mapped_host && gf2x::basis_cvt_two_pass(ctx, r.La, half);
    if (direct) {
        io.src[0] = r.a;
        io.src[1] = r.b;
        io.src_bits[0] = r.na;
        io.src_bits[1] = r.nb;
    } else {
        StageScope s(ctx, STAGE_LOAD, st);
        TRY(gf2x::load_pair(ctx, r.a, r.na, r.b, r.nb, r.T, half, half, st));
    }
    {   // Y (free until Encode) is the side buffer, laid out like X
        StageScope s(ctx, STAGE_BASISCVT, st);
        TRY(gf2x::basis_cvt(ctx, r.T, r.La, false, 2, half, r.X, st, r.Y, half, half, direct ? &io : nullptr));
    }
    {
        StageScope s(ctx, STAGE_ENCODE, st);
        TRY(gf2x::encode(ctx, r.T, l, r.X, r.La, 2, half, (u64)(r.Y - r.X), st));
    }
    return GF2X_OK;
}

// Lines 8-10 of Alg. 5 from the low-layer kernel on: top iButterfly layers,
// Decode, iBasisCvt, store.
gf2x_status inverse_tail(gf2x_ctx *ctx, const ClassRun &r, cudaStream_t st, int bt = -1)
{
    const int l = log2_u64(r.n) - 6;
    const int cnt = r.count;
    const u64 sd = r.stride;
    { StageScope g(ctx, STAGE_IBUTTERFLY, st); TRY(gf2x::butterfly_top_inverse(ctx, r.X, l, cnt, sd, st, bt)); }
    { StageScope g(ctx, STAGE_DECODE, st); TRY(gf2x::decode(ctx, r.X, l, r.T, cnt, sd, st)); }
    // X is free once Decode has read it: the scratch buffer of iBasisCvt; Y
    // (free after the pointwise product) its side buffer
    // (with the two-pass Taylor part a single product is written to c by
    // iBasisCvt's last kernel, and the store kernel is not needed)
    gf2x::ZetaIO io;
    const bool direct = !t_mapped_host && !r.jobs && cnt == 1 && gf2x::basis_cvt_two_pass(ctx, r.n, buffer_words(r));
    if (direct) {
        io.dst = r.c;
        io.dst_bits = product_bits(r.na, r.nb);
    }
    {
        StageScope g(ctx, STAGE_IBASISCVT, st);
        TRY(gf2x::basis_cvt(ctx, r.T, r.n, true, cnt, sd, r.X, st, r.Y, sd, buffer_words(r), direct ? &io : nullptr));
    }
    if (!direct) {
        StageScope g(ctx, STAGE_STORE, st);
        if (r.jobs) TRY(gf2x::store_jobs(ctx, r.T, sd, r.jobs, r.max_c_words, cnt, st));
        else TRY(gf2x::store_bits(ctx, r.T, product_bits(r.na, r.nb), r.c, st));
    }
    return GF2X_OK;
}

// Overlapped kernel launches (launch_pdl) for single products up to this
// transform length: they pay only while a product is latency-bound (measured
// on GB300: 8% less time at 2^16-bit operands, 6% at 2^20, none at 2^22).
constexpr u64 kPdlMaxBits = 1ull << 22;

// Sets ctx->pdl for the launches of one product and restores it on exit.
struct PdlScope {
    gf2x_ctx *ctx;
    bool saved;
    PdlScope(gf2x_ctx *c, bool on) : ctx(c), saved(c->pdl) { c->pdl = on; }
    ~PdlScope() { ctx->pdl = saved; }
};

gf2x_status run_class(gf2x_ctx *ctx, const ClassRun &r, cudaStream_t st)
{
    const int l = log2_u64(r.n) - 6;
    PdlScope pdl(ctx, r.count == 1 && r.n <= kPdlMaxBits);
    // X, Y and T are free until the operands are loaded: the tuner's buffers for the bottom-tile depth
    const int bt = gf2x::butterfly_depth(ctx, r.X, r.Y, r.T, l, r.count, r.stride, st);
    gf2x_status s;
    if (!r.jobs && r.count == 1 && r.La == r.Lb && 2 * r.La <= r.n) {
        s = forward_pair(ctx, r, st);
        if (s != GF2X_OK) return s;
    } else {
        s = forward(ctx, r, 0, r.X, st);
        if (s != GF2X_OK) return s;
        s = forward(ctx, r, 1, r.Y, st);
        if (s != GF2X_OK) return s;
    }
    // both Butterflies (top layers), then both Butterflies, the pointwise product and the iButterfly on
    // the low layers in one kernel, then the iButterfly's top layers
    {
        StageScope g(ctx, STAGE_BUTTERFLY, st);
        TRY(gf2x::butterfly_top_pair(ctx, r.X, r.Y, l, r.count, r.stride, st, bt));
    }
    // T is free between Encode and Decode: the tuner's scratch for the low-layer kernel
    {
        StageScope g(ctx, STAGE_BOTTOM, st);
        TRY(gf2x::butterfly_bottom_fused(ctx, r.X, r.Y, l, r.count, r.stride, st, false, r.T, bt));
    }
    return inverse_tail(ctx, r, st, bt);
}

// The forward steps of Alg. 5 for b on their own: bhat <- Butterfly(Encode(BasisCvt(b)))
// at transform length n, for reuse by products with that n.  Workspace as for
// a product with transform length n: X is BasisCvt's scratch, T the bit array.
gf2x_status forward_transform_device(gf2x_ctx *ctx, const u64 *b, u64 nb, u64 n, u64 *bhat, void *ws,
                                     cudaStream_t st)
{
    const int l = log2_u64(n) - 6;
    const u64 L = next_pow2(nb) < 64 ? 64 : next_pow2(nb);
    const size_t buf = buffer_bytes(n);
    u64 *X = (u64 *)ws, *Y = (u64 *)((char *)ws + buf), *T = (u64 *)((char *)ws + 2 * buf);
    gf2x::ZetaIO io;
    const bool direct = gf2x::basis_cvt_two_pass(ctx, L, buf / 8);   // b read in place by BasisCvt
    if (direct) {
        io.src[0] = b;
        io.src_bits[0] = nb;
    } else {
        StageScope s(ctx, STAGE_LOAD, st);
        TRY(gf2x::load_bits(ctx, b, nb, T, n / 64, st));
    }
    {
        StageScope s(ctx, STAGE_BASISCVT, st);
        TRY(gf2x::basis_cvt(ctx, T, L, false, 1, 0, X, st, Y, 0, buf / 8, direct ? &io : nullptr));
    }
    { StageScope s(ctx, STAGE_ENCODE, st); TRY(gf2x::encode(ctx, T, l, bhat, L, 1, 0, 0, st)); }
    { StageScope s(ctx, STAGE_BUTTERFLY, st); TRY(gf2x::butterfly(ctx, bhat, l, false, 1, 0, st, T)); }
    return GF2X_OK;
}

// c = a * b with b given as its forward transform bhat (at n = transform
// length of na x nb): the forward steps for a, the pointwise product with bhat, the inverse steps.
gf2x_status mul_transformed_device(gf2x_ctx *ctx, const u64 *a, u64 na, const u64 *bhat, u64 nb, u64 *c, void *ws,
                                   cudaStream_t st)
{
    ClassRun r{};
    r.n = transform_bits(na, nb);
    r.count = 1;
    r.La = next_pow2(na) < 64 ? 64 : next_pow2(na);
    r.a = a; r.na = na; r.nb = nb; r.c = c;
    const size_t buf = buffer_bytes(r.n);
    r.X = (u64 *)ws;
    r.Y = (u64 *)((char *)ws + buf);        // free: b's transform is bhat
    r.T = (u64 *)((char *)ws + 2 * buf);
    const int l = log2_u64(r.n) - 6;
    gf2x_status s = forward(ctx, r, 0, r.X, st);
    if (s != GF2X_OK) return s;
    { StageScope g(ctx, STAGE_BUTTERFLY, st); TRY(gf2x::butterfly_top_pair(ctx, r.X, nullptr, l, 1, 0, st)); }
    {
        StageScope g(ctx, STAGE_BOTTOM, st);
        TRY(gf2x::butterfly_bottom_fused(ctx, r.X, (u64 *)bhat, l, 1, 0, st, true, r.T));
    }
    return inverse_tail(ctx, r, st);
}

gf2x_status mul_device(gf2x_ctx *ctx, const u64 *a, u64 na, const u64 *b, u64 nb, u64 *c, void *ws,
                       cudaStream_t st)
{
    if (a == b && na == nb) {
        // a * a: the Frobenius map spreads the bits of a; no transform
        StageScope s(ctx, STAGE_STORE, st);
        TRY(gf2x::square_bits(ctx, a, na, c, st));
        return GF2X_OK;
    }
    ClassRun r{};
    r.n = transform_bits(na, nb);
    r.count = 1;
    r.La = next_pow2(na) < 64 ? 64 : next_pow2(na);
    r.Lb = next_pow2(nb) < 64 ? 64 : next_pow2(nb);
    r.a = a; r.b = b; r.na = na; r.nb = nb; r.c = c;
    const size_t buf = buffer_bytes(r.n);
    r.X = (u64 *)ws;
    r.Y = (u64 *)((char *)ws + buf);
    r.T = (u64 *)((char *)ws + 2 * buf);
    r.stride = 0;
    return run_class(ctx, r, st);
}

// ---------------------------------------------------------------- m = 128
// The same method with GF(2^128) points (Sec. 3 for general m, Sec. 4.3):
// n = max(128, next_pow2(nc)), l = log2(n) - 7, n_p = 2^l points of two words,
// so X, Y, T have the m = 64 sizes.  BasisCvt, load and store are shared.
u64 transform_bits128(u64 na, u64 nb)
{
    u64 nc = product_bits(na, nb);
    if (!nc) return 0;
    u64 n = next_pow2(nc);
    return n < 128 ? 128 : n;
}

gf2x_status mul128_device(gf2x_ctx *ctx, const u64 *a, u64 na, const u64 *b, u64 nb, u64 *c, void *ws,
                          cudaStream_t st)
{
    const u64 n = transform_bits128(na, nb);
    const int l = log2_u64(n) - 7;
    const u64 La = next_pow2(na) < 64 ? 64 : next_pow2(na);
    const u64 Lb = next_pow2(nb) < 64 ? 64 : next_pow2(nb);
    const size_t buf = buffer_bytes(n);
    u64 *X = (u64 *)ws, *Y = (u64 *)((char *)ws + buf), *T = (u64 *)((char *)ws + 2 * buf);
    // X, Y and T are free until the operands are loaded: the tuner's buffers for the bottom-tile depth
    const int bt = gf2x::m128_butterfly_depth(ctx, X, Y, T, l, 1, 0, st);
    if (La == Lb && 2 * La <= n) {
        // both operands in one launch per stage: a in the lower half of T, b in the upper
        const u64 half = n / 128;
        gf2x::ZetaIO io;                               // a and b read in place by the two-pass BasisCvt
        const bool direct = gf2x::basis_cvt_two_pass(ctx, La, half);
        if (direct) {
            io.src[0] = a;
            io.src[1] = b;
            io.src_bits[0] = na;
            io.src_bits[1] = nb;
        } else {
            StageScope s(ctx, STAGE_LOAD, st);
            TRY(gf2x::load_pair(ctx, a, na, b, nb, T, half, half, st));
        }
        {   // Y (free until Encode) is BasisCvt's side buffer, laid out like X
            StageScope s(ctx, STAGE_BASISCVT, st);
            TRY(gf2x::basis_cvt(ctx, T, La, false, 2, half, X, st, Y, half, half, direct ? &io : nullptr));
        }
        { StageScope s(ctx, STAGE_ENCODE, st); TRY(gf2x::m128_encode(ctx, T, l, X, La, 2, half, (u64)(Y - X), st)); }
    } else {
        for (int which = 0; which < 2; ++which) {
            u64 *F = which ? Y : X;
            const u64 L = which ? Lb : La;
            // side buffer: Y for a, the words of T above L for b (Encode reads the first L bits)
            u64 *side = which ? T + L / 64 : Y;
            const u64 side_words = which ? n / 64 - L / 64 : buf / 8;
            gf2x::ZetaIO io;                           // the operand read in place by the two-pass BasisCvt
            const bool direct = gf2x::basis_cvt_two_pass(ctx, L, side_words);
            if (direct) {
                io.src[0] = which ? b : a;
                io.src_bits[0] = which ? nb : na;
            } else {
                StageScope s(ctx, STAGE_LOAD, st);
                TRY(gf2x::load_bits(ctx, which ? b : a, which ? nb : na, T, n / 64, st));
            }
            {
                StageScope s(ctx, STAGE_BASISCVT, st);
                TRY(gf2x::basis_cvt(ctx, T, L, false, 1, 0, F, st, side, 0, side_words, direct ? &io : nullptr));
            }
            { StageScope s(ctx, STAGE_ENCODE, st); TRY(gf2x::m128_encode(ctx, T, l, F, L, 1, 0, 0, st)); }
        }
    }
    { StageScope g(ctx, STAGE_BUTTERFLY, st); TRY(gf2x::m128_butterfly_top_pair(ctx, X, Y, l, 1, 0, st, bt)); }
    {   // T is free between Encode and Decode: the tuner's scratch for the low-layer kernel
        StageScope g(ctx, STAGE_BOTTOM, st);
        TRY(gf2x::m128_butterfly_bottom_fused(ctx, X, Y, l, 1, 0, st, T, bt));
    }
    { StageScope g(ctx, STAGE_IBUTTERFLY, st); TRY(gf2x::m128_butterfly_top_inverse(ctx, X, l, 1, 0, st, bt)); }
    { StageScope g(ctx, STAGE_DECODE, st); TRY(gf2x::m128_decode(ctx, X, l, T, 1, 0, st)); }
    // X is free once Decode has read it, Y after the pointwise step; with the
    // two-pass Taylor part iBasisCvt's last kernel writes the product to c
    gf2x::ZetaIO io;
    const bool direct = gf2x::basis_cvt_two_pass(ctx, n, buf / 8);
    if (direct) {
        io.dst = c;
        io.dst_bits = product_bits(na, nb);
    }
    {
        StageScope g(ctx, STAGE_IBASISCVT, st);
        TRY(gf2x::basis_cvt(ctx, T, n, true, 1, 0, X, st, Y, 0, buf / 8, direct ? &io : nullptr));
    }
    if (!direct) {
        StageScope g(ctx, STAGE_STORE, st);
        TRY(gf2x::store_bits(ctx, T, product_bits(na, nb), c, st));
    }
    return GF2X_OK;
}

gf2x_status op_device(gf2x_ctx *ctx, int kind, const u64 *a, u64 na, const u64 *b, u64 nb, u64 *c, void *ws,
                      cudaStream_t st)
{
    if (kind == OP_MUL_TRANSFORMED) return mul_transformed_device(ctx, a, na, b, nb, c, ws, st);
    if (kind == OP_FORWARD_TRANSFORM) return forward_transform_device(ctx, a, na, nb, c, ws, st);
    if (kind == OP_MUL128) return mul128_device(ctx, a, na, b, nb, c, ws, st);
    return mul_device(ctx, a, na, b, nb, c, ws, st);
}

// A sequence through the graph cache (falls back to direct launches while a key
// is new, while the caller's stream is itself being captured, or when
// GF2X_GRAPHS=0 is set in the environment).
gf2x_status op_graph(gf2x_ctx *ctx, int kind, const u64 *a, u64 na, const u64 *b, u64 nb, u64 *c, void *ws,
                     cudaStream_t st)
{
    GraphCache *gc = graphs(ctx);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (gc->disabled || cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return op_device(ctx, kind, a, na, b, nb, c, ws, st);
    for (GraphEntry &e : gc->entries) {
        if (e.kind == kind && e.a == a && e.b == b && e.na == na && e.nb == nb && e.c == c && e.ws == ws &&
            e.profiling == ctx->profiling && e.gen == gc->gen) {
            e.stamp = ++gc->clock;
            if (cudaGraphLaunch(e.exec, st) != cudaSuccess) return GF2X_ECUDA;
            for (int k = 0; k < STAGE_COUNT; ++k) ctx->launches[k] += e.launches[k];
            if (ctx->profiling)
                for (const Rec &r : e.recs) profiler(ctx)->pending.push_back(r);
            return GF2X_OK;
        }
    }
    bool repeat = false;
    for (size_t k = 0; k < gc->seen.size(); ++k) {
        const GraphCache::Key &key = gc->seen[k];
        if (key.kind == kind && key.a == a && key.b == b && key.na == na && key.nb == nb && key.c == c &&
            key.ws == ws) {
            repeat = true;
            gc->seen.erase(gc->seen.begin() + (long)k);
            break;
        }
    }
    if (!repeat) {
        if (gc->seen.size() >= 64) gc->seen.erase(gc->seen.begin());
        gc->seen.push_back({kind, a, b, na, nb, c, ws});
        return op_device(ctx, kind, a, na, b, nb, c, ws, st);
    }
    // second call with this key: capture, instantiate, launch
    if (!gc->cap && cudaStreamCreateWithFlags(&gc->cap, cudaStreamNonBlocking) != cudaSuccess)
        return op_device(ctx, kind, a, na, b, nb, c, ws, st);
    GraphEntry e{};
    e.kind = kind;
    e.a = a; e.b = b; e.na = na; e.nb = nb; e.c = c; e.ws = ws; e.profiling = ctx->profiling;
    unsigned long long before[STAGE_COUNT];
    for (int k = 0; k < STAGE_COUNT; ++k) before[k] = ctx->launches[k];
    Profiler *p = profiler(ctx);
    if (cudaStreamBeginCapture(gc->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return op_device(ctx, kind, a, na, b, nb, c, ws, st);
    p->capture = &e.recs;
    gf2x_status s = op_device(ctx, kind, a, na, b, nb, c, ws, gc->cap);
    p->capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(gc->cap, &graph);
    for (int k = 0; k < STAGE_COUNT; ++k) {       // captured, not run: count them per replay
        e.launches[k] = ctx->launches[k] - before[k];
        ctx->launches[k] = before[k];
    }
    if (s != GF2X_OK || ce != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        for (Rec &r : e.recs) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
        cudaGetLastError();
        return s != GF2X_OK ? s : op_device(ctx, kind, a, na, b, nb, c, ws, st);
    }
    ce = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        for (Rec &r : e.recs) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
        cudaGetLastError();
        return op_device(ctx, kind, a, na, b, nb, c, ws, st);
    }
    if (gc->entries.size() >= kMaxGraphs) {       // evict the least recently used
        size_t old = 0;
        for (size_t k = 1; k < gc->entries.size(); ++k)
            if (gc->entries[k].stamp < gc->entries[old].stamp) old = k;
        destroy_entry(gc->entries[old]);
        gc->entries.erase(gc->entries.begin() + (long)old);
    }
    e.stamp = ++gc->clock;
    e.gen = gc->gen;
    gc->entries.push_back(e);
    GraphEntry &ent = gc->entries.back();
    if (cudaGraphLaunch(ent.exec, st) != cudaSuccess) return GF2X_ECUDA;
    for (int k = 0; k < STAGE_COUNT; ++k) ctx->launches[k] += ent.launches[k];
    if (ctx->profiling)
        for (const Rec &r : ent.recs) p->pending.push_back(r);
    return GF2X_OK;
}

// ---------------------------------------------------------------- batches
constexpr int kMaxClassJobs = 16384;   // jobs per launch of one class (grid.y limit)

struct BatchPlan {
    std::vector<JobDev> table;          // jobs in class order (ascending n)
    std::vector<ClassRun> runs;
    size_t table_bytes = 0;
    size_t persist_off = 0;             // the persistent launch's area (segments, plans, counters)
    size_t persist_bytes = 0;
    size_t total_bytes = 0;
};

// Group the non-empty jobs by transform length; lay out the workspace as
// [job table][class 0: X, Y, T][class 1: ...] (256-byte aligned pieces).
gf2x_status plan_batch(const gf2x_job *jobs, size_t count, BatchPlan &bp)
{
    std::vector<std::pair<u64, size_t>> order;
    order.reserve(count);
    for (size_t k = 0; k < count; ++k) {
        const gf2x_job &j = jobs[k];
        if (!product_bits(j.na_bits, j.nb_bits)) continue;
        const u64 n = transform_bits(j.na_bits, j.nb_bits);
        if (n > kMaxTransformBits) return GF2X_ETOOBIG;
        if (!j.a || !j.b || !j.c || !aligned8(j.a) || !aligned8(j.b) || !aligned8(j.c)) return GF2X_EINVAL;
        const size_t cb = (size_t)((product_bits(j.na_bits, j.nb_bits) + 63) / 64) * 8;
        if (overlap(j.c, cb, j.a, (size_t)((j.na_bits + 63) / 64) * 8) ||
            overlap(j.c, cb, j.b, (size_t)((j.nb_bits + 63) / 64) * 8))
            return GF2X_EINVAL;
        order.push_back({n, k});
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<u64, size_t> &x, const std::pair<u64, size_t> &y) { return x.first < y.first; });
    bp.table.clear();
    bp.runs.clear();
    for (auto &o : order) {
        const gf2x_job &j = jobs[o.second];
        bp.table.push_back(JobDev{j.a, j.na_bits, j.b, j.nb_bits, j.c, 0});
    }
    bp.table_bytes = round_up(bp.table.size() * sizeof(JobDev));
    size_t off = bp.table_bytes;
    for (size_t k = 0; k < order.size();) {
        size_t e = k;
        while (e < order.size() && order[e].first == order[k].first && (int)(e - k) < kMaxClassJobs) ++e;
        ClassRun r{};
        r.n = order[k].first;
        r.count = (int)(e - k);
        u64 ma = 0, mb = 0, mc = 0;
        for (size_t t = k; t < e; ++t) {
            const JobDev &jd = bp.table[t];
            ma = jd.na > ma ? jd.na : ma;
            mb = jd.nb > mb ? jd.nb : mb;
            const u64 cw = (product_bits(jd.na, jd.nb) + 63) / 64;
            mc = cw > mc ? cw : mc;
        }
        r.La = next_pow2(ma) < 64 ? 64 : next_pow2(ma);
        r.Lb = next_pow2(mb) < 64 ? 64 : next_pow2(mb);
        r.max_c_words = mc;
        r.stride = buffer_bytes(r.n) / 8;
        r.jobs = (const JobDev *)(uintptr_t)k;          // index for now; made a pointer per call
        const size_t region = (size_t)r.count * buffer_bytes(r.n);
        r.X = (u64 *)(uintptr_t)off;
        r.Y = (u64 *)(uintptr_t)(off + region);
        r.T = (u64 *)(uintptr_t)(off + 2 * region);
        off += 3 * region;
        bp.runs.push_back(r);
        k = e;
    }
    bp.persist_off = off;
    bp.persist_bytes = round_up(gf2x::persist_area_bytes(bp.runs.size(), bp.table.size()));
    bp.total_bytes = off + bp.persist_bytes;
    return GF2X_OK;
}

// The runs of a plan with the workspace base applied.
std::vector<ClassRun> bind_runs(const BatchPlan &bp, void *ws)
{
    std::vector<ClassRun> out = bp.runs;
    char *base = (char *)ws;
    for (ClassRun &r : out) {
        r.jobs = (const JobDev *)(base) + (uintptr_t)r.jobs;
        r.X = (u64 *)(base + (uintptr_t)r.X);
        r.Y = (u64 *)(base + (uintptr_t)r.Y);
        r.T = (u64 *)(base + (uintptr_t)r.T);
    }
    return out;
}

u64 hash_table(const std::vector<JobDev> &t, const void *ws)
{
    u64 h = 1469598103934665603ull ^ (u64)(uintptr_t)ws;
    const unsigned char *p = (const unsigned char *)t.data();
    for (size_t k = 0; k < t.size() * sizeof(JobDev); ++k) h = (h ^ p[k]) * 1099511628211ull;
    return h ^ (u64)t.size();
}

// A batch graph is replayed only for the same job table and workspace: the
// hash picks candidates, the stored table decides.
struct BatchKey {
    u64 hash;
    const void *ws;
    std::vector<JobDev> table;
    u64 plan;                           // digest of the persistent launch's plan (0: class launches)
    bool same(u64 h, const void *w, const std::vector<JobDev> &t, u64 p) const
    {
        return hash == h && ws == w && plan == p && table.size() == t.size() &&
               (t.empty() || std::memcmp(table.data(), t.data(), t.size() * sizeof(JobDev)) == 0);
    }
};

struct BatchGraph {
    BatchKey key;
    bool profiling;
    unsigned gen;           // GraphCache::gen at capture
    cudaGraphExec_t exec;
    unsigned long long launches[STAGE_COUNT];
    std::vector<Rec> recs;
    unsigned long long stamp;
};

struct BatchCache {
    std::vector<BatchGraph> entries;
    std::vector<BatchKey> seen;
};

constexpr size_t kMaxBatchGraphs = 8;

bool valid_n(u64 n) { return n >= 64 && n <= kMaxTransformBits && (n & (n - 1)) == 0; }
bool valid_n128(u64 n) { return n >= 128 && n <= kMaxTransformBits128 && (n & (n - 1)) == 0; }

}  // namespace

extern "C" {

const char *gf2x_status_string(gf2x_status s)
{
    switch (s) {
    case GF2X_OK: return "GF2X_OK";
    case GF2X_EINVAL: return "GF2X_EINVAL";
    case GF2X_ETOOBIG: return "GF2X_ETOOBIG";
    case GF2X_ENOMEM: return "GF2X_ENOMEM";
    case GF2X_ECUDA: return "GF2X_ECUDA";
    case GF2X_ETIMEOUT: return "GF2X_ETIMEOUT";
    case GF2X_ENODEV: return "GF2X_ENODEV";
    case GF2X_ENOSPACE: return "GF2X_ENOSPACE";
    case GF2X_EBOUNDS: return "GF2X_EBOUNDS";
    }
    return "GF2X_UNKNOWN";
}

gf2x_status gf2x_ctx_create(gf2x_ctx **out, int device)
{
    if (!out) return GF2X_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) return GF2X_ENODEV;
    if (device < 0 || device >= count) return GF2X_ENODEV;
    DeviceGuard g(device);
    if (!g.ok) return GF2X_ENODEV;

    gf2x_ctx *ctx = new (std::nothrow) gf2x_ctx();
    if (!ctx) return GF2X_ENOMEM;
    ctx->device = device;
    ctx->prof = new (std::nothrow) Profiler();
    ctx->graphs = new (std::nothrow) GraphCache();
    ctx->batch_graphs = new (std::nothrow) BatchCache();
    ctx->tuner = gf2x::tuner_create();
    if (!ctx->prof || !ctx->graphs || !ctx->batch_graphs || !ctx->tuner) {
        delete profiler(ctx);
        delete graphs(ctx);
        delete (BatchCache *)ctx->batch_graphs;
        gf2x::tuner_destroy(ctx->tuner);
        delete ctx;
        return GF2X_ENOMEM;
    }
    if (const char *env = std::getenv("GF2X_GRAPHS")) graphs(ctx)->disabled = (env[0] == '0');
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);

    u64 v[64];
    auto fail = [&](gf2x_status st) {
        delete profiler(ctx);
        delete graphs(ctx);
        delete (BatchCache *)ctx->batch_graphs;
        gf2x::tuner_destroy(ctx->tuner);
        delete ctx;
        return st;
    };
    if (!cantor_basis(v)) return fail(GF2X_EINVAL);
    std::memcpy(ctx->cantor, v, sizeof v);

    // Encode multipliers: layer l+t of the truncated Butterfly multiplies by
    // s_{l+t}(v_{l+32}) = v_{32-t} (Eq. 4), the same for every l; row j of R
    // is r_j = prod_{t: bit t of j} v_{32-t} (Alg. 4, Sec. 3.3).
    u64 r[64], rinv[64];
    for (int j = 0; j < 64; ++j) {
        u64 p = 1;
        for (int t = 0; t < 6; ++t)
            if ((j >> t) & 1) p = hmul(p, v[32 - t]);
        r[j] = p;
    }
    if (!gf2_inverse(r, rinv)) return fail(GF2X_EINVAL);   // Prop. 2

    std::vector<u64> host(3 * 2048 + 64 + 256);
    window_table(v, &host[0]);
    window_table(r, &host[2048]);
    window_table(rinv, &host[4096]);
    std::memcpy(&host[6144], v, sizeof v);
    window_table4(rinv, &host[6208]);

    if (cudaMalloc(&ctx->d_tables, host.size() * sizeof(u64)) != cudaSuccess) return fail(GF2X_ENOMEM);
    if (cudaMalloc(&ctx->d_state, kStateBytes) != cudaSuccess) {
        cudaFree(ctx->d_tables);
        return fail(GF2X_ENOMEM);
    }
    ctx->d_status = (int *)ctx->d_state;
    ctx->d_sync = (GridSync *)((char *)ctx->d_state + 128);
    ctx->d_word = (unsigned long long *)((char *)ctx->d_state + 192);
    ctx->d_cvt = ctx->d_tables;
    ctx->d_enc = ctx->d_tables + 2048;
    ctx->d_dec = ctx->d_tables + 4096;
    ctx->d_cantor = ctx->d_tables + 6144;
    ctx->d_dec4 = ctx->d_tables + 6208;
    std::vector<u64> host128(gf2x::kTables128Words);
    if (!gf2x::m128_build_tables(host128.data())) {
        cudaFree(ctx->d_tables);
        cudaFree(ctx->d_state);
        return fail(GF2X_EINVAL);
    }
    if (cudaMalloc(&ctx->d_tables128, host128.size() * sizeof(u64)) != cudaSuccess) {
        cudaFree(ctx->d_tables);
        cudaFree(ctx->d_state);
        return fail(GF2X_ENOMEM);
    }
    ctx->d_cvt128 = ctx->d_tables128;
    ctx->d_enc128 = ctx->d_tables128 + 4096;
    ctx->d_dec128 = ctx->d_tables128 + 4096 + 8192;
    ctx->d_cantor128 = ctx->d_tables128 + 4096 + 2 * 8192;
    if (cudaMemcpy(ctx->d_tables, host.data(), host.size() * sizeof(u64), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_tables128, host128.data(), host128.size() * sizeof(u64), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(ctx->d_state, 0, kStateBytes) != cudaSuccess) {
        cudaFree(ctx->d_tables);
        cudaFree(ctx->d_tables128);
        cudaFree(ctx->d_state);
        return fail(GF2X_ECUDA);
    }
    *out = ctx;
    return GF2X_OK;
}

void gf2x_ctx_destroy(gf2x_ctx *ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    if (BatchCache *bc = (BatchCache *)ctx->batch_graphs) {
        for (BatchGraph &e : bc->entries) {
            cudaGraphExecDestroy(e.exec);
            for (Rec &r : e.recs) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
        }
        delete bc;
    }
    if (GraphCache *gc = graphs(ctx)) {
        for (GraphEntry &e : gc->entries) destroy_entry(e);
        if (gc->cap) cudaStreamDestroy(gc->cap);
        delete gc;
    }
    if (Profiler *p = profiler(ctx)) {
        for (cudaEvent_t e : p->pool) cudaEventDestroy(e);
        for (Rec &r : p->pending)
            if (r.pooled) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
        delete p;
    }
    gf2x::tuner_destroy(ctx->tuner);
    cudaFree(ctx->d_tables);
    cudaFree(ctx->d_tables128);
    cudaFree(ctx->d_state);
    delete ctx;
}

uint64_t gf2x_transform_bits(uint64_t na, uint64_t nb) { return transform_bits(na, nb); }

size_t gf2x_workspace_bytes(uint64_t na, uint64_t nb)
{
    u64 n = transform_bits(na, nb);
    if (!n || n > kMaxTransformBits) return 0;
    return 3 * buffer_bytes(n) + kAlign;          // + 256 bytes reserved for device-side state
}

// Argument rules of gf2x_mul; GF2X_OK when the product may be enqueued
// (*empty set when there is nothing to compute).
static gf2x_status check_mul(gf2x_ctx *ctx, const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb,
                             const uint64_t *c, const void *ws, size_t ws_bytes, bool *empty)
{
    *empty = false;
    if (!ctx) return GF2X_EINVAL;
    const u64 nc = product_bits(na, nb);
    if (!nc) {
        *empty = true;
        return GF2X_OK;
    }
    const u64 n = transform_bits(na, nb);
    if (n > kMaxTransformBits) return GF2X_ETOOBIG;
    if (!a || !b || !c || !ws || !aligned8(a) || !aligned8(b) || !aligned8(c) || ((uintptr_t)ws % kAlign))
        return GF2X_EINVAL;
    const size_t need = gf2x_workspace_bytes(na, nb);
    if (ws_bytes < need) return GF2X_ENOSPACE;
    const size_t cb = (size_t)((nc + 63) / 64) * 8;
    if (overlap(c, cb, a, (size_t)((na + 63) / 64) * 8) || overlap(c, cb, b, (size_t)((nb + 63) / 64) * 8) ||
        overlap(c, cb, ws, need))
        return GF2X_EINVAL;
    return GF2X_OK;
}

gf2x_status gf2x_mul(gf2x_ctx *ctx, const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb, uint64_t *c,
                     void *ws, size_t ws_bytes, void *stream)
{
    bool empty = false;
    const gf2x_status s = check_mul(ctx, a, na, b, nb, c, ws, ws_bytes, &empty);
    if (s != GF2X_OK || empty) return s;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GF2X_ECUDA;
    return op_graph(ctx, OP_MUL, a, na, b, nb, c, ws, (cudaStream_t)stream);
}

gf2x_status gf2x_tune_freeze(gf2x_ctx *ctx, int frozen)
{
    if (!ctx) return GF2X_EINVAL;
    gf2x::tuner_freeze(ctx->tuner, frozen != 0);
    return GF2X_OK;
}

static_assert(GF2X_KNOB_UNIT16_R == gf2x::TUNE_UNIT16_R && GF2X_KNOB_BOTTOM_SHAPE == gf2x::TUNE_BOTTOM_SHAPE &&
                  GF2X_KNOB_WINDOW_DEPTH == gf2x::TUNE_WINDOW_DEPTH &&
                  GF2X_KNOB_M128_BOTTOM_CHUNK == gf2x::TUNE_M128_BOTTOM_CHUNK &&
                  GF2X_KNOB_BOTTOM_DEPTH == gf2x::TUNE_BFLY_DEPTH &&
                  GF2X_KNOB_M128_BOTTOM_DEPTH == gf2x::TUNE_M128_BFLY_DEPTH &&
                  GF2X_KNOB_BATCH_PERSISTENT == gf2x::TUNE_BATCH_PERSIST &&
                  GF2X_KNOB_BOTTOM_MUL == gf2x::TUNE_BOTTOM_MUL && GF2X_KNOB_CVT_TAYLOR == gf2x::TUNE_CVT_TAYLOR,
              "the ABI's knob numbers are the tuner's");

gf2x_status gf2x_tune_pin(gf2x_ctx *ctx, int knob, int choice)
{
    if (!ctx || knob < GF2X_KNOB_UNIT16_R || knob > GF2X_KNOB_CVT_TAYLOR || choice < -1) return GF2X_EINVAL;
    gf2x::tuner_pin(ctx->tuner, knob, choice);
    ++graphs(ctx)->gen;           // captured graphs keep their shapes: capture again
    return GF2X_OK;
}

int gf2x_bottom_layers(gf2x_ctx *ctx, uint64_t na, uint64_t nb)
{
    if (!ctx) return -1;
    const u64 n = transform_bits(na, nb);
    if (!n || n > kMaxTransformBits) return -1;
    return gf2x::butterfly_depth_stored(ctx, log2_u64(n) - 6, 1);
}

size_t gf2x_transform_bytes(uint64_t n)
{
    return valid_n(n) ? (size_t)(n / 8) : 0;
}

size_t gf2x_transform_workspace_bytes(uint64_t n)
{
    return valid_n(n) ? 3 * buffer_bytes(n) + kAlign : 0;
}

gf2x_status gf2x_forward_transform(gf2x_ctx *ctx, const uint64_t *b, uint64_t nb, uint64_t n, uint64_t *bhat,
                                   void *ws, size_t ws_bytes, void *stream)
{
    if (!ctx) return GF2X_EINVAL;
    if (n > kMaxTransformBits) return GF2X_ETOOBIG;
    if (!valid_n(n) || nb == 0 || nb > n) return GF2X_EINVAL;
    if (!b || !bhat || !ws || !aligned8(b) || !aligned8(bhat) || ((uintptr_t)ws % kAlign)) return GF2X_EINVAL;
    const size_t need = gf2x_transform_workspace_bytes(n);
    if (ws_bytes < need) return GF2X_ENOSPACE;
    const size_t tb = (size_t)(n / 8);
    if (overlap(bhat, tb, b, (size_t)((nb + 63) / 64) * 8) || overlap(bhat, tb, ws, need)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GF2X_ECUDA;
    return op_graph(ctx, OP_FORWARD_TRANSFORM, b, nb, nullptr, n, bhat, ws, (cudaStream_t)stream);
}

gf2x_status gf2x_mul_transformed(gf2x_ctx *ctx, const uint64_t *a, uint64_t na, const uint64_t *bhat, uint64_t nb,
                                 uint64_t *c, void *ws, size_t ws_bytes, void *stream)
{
    if (!ctx) return GF2X_EINVAL;
    const u64 nc = product_bits(na, nb);
    if (!nc) return GF2X_OK;
    const u64 n = transform_bits(na, nb);
    if (n > kMaxTransformBits) return GF2X_ETOOBIG;
    if (!a || !bhat || !c || !ws || !aligned8(a) || !aligned8(bhat) || !aligned8(c) || ((uintptr_t)ws % kAlign))
        return GF2X_EINVAL;
    const size_t need = gf2x_workspace_bytes(na, nb);
    if (ws_bytes < need) return GF2X_ENOSPACE;
    const size_t cb = (size_t)((nc + 63) / 64) * 8;
    if (overlap(c, cb, a, (size_t)((na + 63) / 64) * 8) || overlap(c, cb, bhat, (size_t)(n / 8)) ||
        overlap(c, cb, ws, need) || overlap(bhat, (size_t)(n / 8), ws, need))
        return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GF2X_ECUDA;
    return op_graph(ctx, OP_MUL_TRANSFORMED, a, na, bhat, nb, c, ws, (cudaStream_t)stream);
}

size_t gf2x_host_workspace_bytes(uint64_t na, uint64_t nb)
{
    size_t base = gf2x_workspace_bytes(na, nb);
    if (!base) return 0;
    u64 nc = product_bits(na, nb);
    return base + round_up((size_t)((na + 63) / 64) * 8) + round_up((size_t)((nb + 63) / 64) * 8) +
           round_up((size_t)((nc + 63) / 64) * 8);
}

gf2x_status gf2x_mul_host(gf2x_ctx *ctx, const uint64_t *a_host, uint64_t na, const uint64_t *b_host, uint64_t nb,
                          uint64_t *c_host, void *ws, size_t ws_bytes, void *stream)
{
    if (!ctx) return GF2X_EINVAL;
    const u64 nc = product_bits(na, nb);
    if (!nc) return GF2X_OK;
    if (transform_bits(na, nb) > kMaxTransformBits) return GF2X_ETOOBIG;
    if (!a_host || !b_host || !c_host || !ws || ((uintptr_t)ws % kAlign)) return GF2X_EINVAL;
    const size_t need = gf2x_host_workspace_bytes(na, nb);
    if (ws_bytes < need) return GF2X_ENOSPACE;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GF2X_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // Page-locked host buffers are read and written by the load and store
    // kernels themselves (over the CPU-GPU link, no staging copies); pageable
    // ones are copied through the workspace.
    auto device_view = [](const void *p) -> const void * {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
    };
    const u64 *va = (const u64 *)device_view(a_host), *vb = (const u64 *)device_view(b_host);
    u64 *vc = (u64 *)device_view(c_host);
    // The kernels read and write whole words, so the direct path needs the same
    // pointer rules as gf2x_mul (8-byte alignment, c apart from a and b); other
    // page-locked buffers take the staged path like pageable ones.
    const size_t cbytes = (size_t)((nc + 63) / 64) * 8;
    const bool direct = va && vb && vc && aligned8(va) && aligned8(vb) && aligned8(vc) &&
                        !overlap(vc, cbytes, va, (size_t)((na + 63) / 64) * 8) &&
                        !overlap(vc, cbytes, vb, (size_t)((nb + 63) / 64) * 8);
    if (direct) {
        t_mapped_host = true;
        gf2x_status s = op_graph(ctx, OP_MUL, va, na, vb, nb, vc, ws, st);
        t_mapped_host = false;
        if (s != GF2X_OK) return s;
        TRY(cudaStreamSynchronize(st));
        return GF2X_OK;
    }
    const size_t base = gf2x_workspace_bytes(na, nb);
    const size_t ab = (size_t)((na + 63) / 64) * 8, bb = (size_t)((nb + 63) / 64) * 8,
                 cb = (size_t)((nc + 63) / 64) * 8;
    u64 *da = (u64 *)((char *)ws + base);
    u64 *db = (u64 *)((char *)da + round_up(ab));
    u64 *dc = (u64 *)((char *)db + round_up(bb));
    TRY(cudaMemcpyAsync(da, a_host, ab, cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(db, b_host, bb, cudaMemcpyHostToDevice, st));
    gf2x_status s = op_graph(ctx, OP_MUL, da, na, db, nb, dc, ws, st);
    if (s != GF2X_OK) return s;
    TRY(cudaMemcpyAsync(c_host, dc, cb, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    return GF2X_OK;
}

gf2x_status gf2x_stream_status(gf2x_ctx *ctx, void *stream)
{
    if (!ctx) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    TRY(cudaMemcpyAsync(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
        TRY(cudaStreamSynchronize(st));
    }
    const unsigned long long oob = gf2x::out_of_range_fft() + gf2x::out_of_range_cvt() +
                                   gf2x::out_of_range_cvt_reg() + gf2x::out_of_range_bfly() +
                                   gf2x::out_of_range_persist() + gf2x::out_of_range_zeta();
    if (h == 0 && oob) return GF2X_EBOUNDS;
    return (gf2x_status)h;
}

gf2x_status gf2x_basis_cvt(gf2x_ctx *ctx, uint64_t *bits, uint64_t L, void *stream)
{
    if (!ctx || !bits || !aligned8(bits)) return GF2X_EINVAL;
    if (L > kMaxTransformBits) return GF2X_ETOOBIG;
    if (!valid_n(L)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_BASISCVT, (cudaStream_t)stream);
    return from_cuda(gf2x::basis_cvt(ctx, bits, L, false, 1, 0, nullptr, (cudaStream_t)stream));
}

gf2x_status gf2x_ibasis_cvt(gf2x_ctx *ctx, uint64_t *bits, uint64_t L, void *stream)
{
    if (!ctx || !bits || !aligned8(bits)) return GF2X_EINVAL;
    if (L > kMaxTransformBits) return GF2X_ETOOBIG;
    if (!valid_n(L)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_IBASISCVT, (cudaStream_t)stream);
    return from_cuda(gf2x::basis_cvt(ctx, bits, L, true, 1, 0, nullptr, (cudaStream_t)stream));
}

gf2x_status gf2x_encode(gf2x_ctx *ctx, const uint64_t *novel, uint64_t n, uint64_t *f, void *stream)
{
    if (!ctx || !novel || !f || !aligned8(novel) || !aligned8(f)) return GF2X_EINVAL;
    if (n > kMaxTransformBits) return GF2X_ETOOBIG;
    if (!valid_n(n) || overlap(novel, n / 8, f, n / 8)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_ENCODE, (cudaStream_t)stream);
    return from_cuda(gf2x::encode(ctx, novel, log2_u64(n) - 6, f, n, 1, 0, 0, (cudaStream_t)stream));
}

gf2x_status gf2x_decode(gf2x_ctx *ctx, const uint64_t *h, uint64_t n, uint64_t *novel, void *stream)
{
    if (!ctx || !novel || !h || !aligned8(novel) || !aligned8(h)) return GF2X_EINVAL;
    if (n > kMaxTransformBits) return GF2X_ETOOBIG;
    if (!valid_n(n) || overlap(novel, n / 8, h, n / 8)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_DECODE, (cudaStream_t)stream);
    return from_cuda(gf2x::decode(ctx, h, log2_u64(n) - 6, novel, 1, 0, (cudaStream_t)stream));
}

gf2x_status gf2x_butterfly(gf2x_ctx *ctx, uint64_t *f, uint64_t n, void *stream)
{
    if (!ctx || !f || !aligned8(f)) return GF2X_EINVAL;
    if (n > kMaxTransformBits) return GF2X_ETOOBIG;
    if (!valid_n(n)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_BUTTERFLY, (cudaStream_t)stream);
    return from_cuda(gf2x::butterfly(ctx, f, log2_u64(n) - 6, false, 1, 0, (cudaStream_t)stream));
}

gf2x_status gf2x_ibutterfly(gf2x_ctx *ctx, uint64_t *f, uint64_t n, void *stream)
{
    if (!ctx || !f || !aligned8(f)) return GF2X_EINVAL;
    if (n > kMaxTransformBits) return GF2X_ETOOBIG;
    if (!valid_n(n)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_IBUTTERFLY, (cudaStream_t)stream);
    return from_cuda(gf2x::butterfly(ctx, f, log2_u64(n) - 6, true, 1, 0, (cudaStream_t)stream));
}

gf2x_status gf2x_pointwise(gf2x_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *c, uint64_t count,
                           void *stream)
{
    if (!ctx) return GF2X_EINVAL;
    if (!count) return GF2X_OK;
    if (!a || !b || !c || !aligned8(a) || !aligned8(b) || !aligned8(c)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_POINTWISE, (cudaStream_t)stream);
    return from_cuda(gf2x::pointwise(ctx, a, b, c, count, (cudaStream_t)stream));
}

// ------------------------------------------------------------ m = 128
uint64_t gf2x_m128_transform_bits(uint64_t na, uint64_t nb) { return transform_bits128(na, nb); }

int gf2x_m128_bottom_layers(gf2x_ctx *ctx, uint64_t na, uint64_t nb)
{
    if (!ctx) return -1;
    const u64 n = transform_bits128(na, nb);
    if (!n || n > kMaxTransformBits128) return -1;
    return gf2x::m128_butterfly_depth_stored(ctx, log2_u64(n) - 7, 1);
}

size_t gf2x_m128_workspace_bytes(uint64_t na, uint64_t nb)
{
    u64 n = transform_bits128(na, nb);
    if (!n || n > kMaxTransformBits128) return 0;
    return 3 * buffer_bytes(n) + kAlign;
}

gf2x_status gf2x_mul_m128(gf2x_ctx *ctx, const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb, uint64_t *c,
                          void *ws, size_t ws_bytes, void *stream)
{
    if (!ctx) return GF2X_EINVAL;
    const u64 nc = product_bits(na, nb);
    if (!nc) return GF2X_OK;
    const u64 n = transform_bits128(na, nb);
    if (n > kMaxTransformBits128) return GF2X_ETOOBIG;
    if (!a || !b || !c || !ws || !aligned8(a) || !aligned8(b) || !aligned8(c) || ((uintptr_t)ws % kAlign))
        return GF2X_EINVAL;
    const size_t need = gf2x_m128_workspace_bytes(na, nb);
    if (ws_bytes < need) return GF2X_ENOSPACE;
    const size_t cb = (size_t)((nc + 63) / 64) * 8;
    if (overlap(c, cb, a, (size_t)((na + 63) / 64) * 8) || overlap(c, cb, b, (size_t)((nb + 63) / 64) * 8) ||
        overlap(c, cb, ws, need))
        return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GF2X_ECUDA;
    return op_graph(ctx, OP_MUL128, a, na, b, nb, c, ws, (cudaStream_t)stream);
}

gf2x_status gf2x_m128_encode(gf2x_ctx *ctx, const uint64_t *novel, uint64_t n, uint64_t *f, void *stream)
{
    if (!ctx || !novel || !f || !aligned8(novel) || !aligned16(f)) return GF2X_EINVAL;
    if (n > kMaxTransformBits128) return GF2X_ETOOBIG;
    if (!valid_n128(n) || overlap(novel, n / 8, f, n / 8)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_ENCODE, (cudaStream_t)stream);
    return from_cuda(gf2x::m128_encode(ctx, novel, log2_u64(n) - 7, f, n, 1, 0, 0, (cudaStream_t)stream));
}

gf2x_status gf2x_m128_decode(gf2x_ctx *ctx, const uint64_t *h, uint64_t n, uint64_t *novel, void *stream)
{
    if (!ctx || !novel || !h || !aligned8(novel) || !aligned16(h)) return GF2X_EINVAL;
    if (n > kMaxTransformBits128) return GF2X_ETOOBIG;
    if (!valid_n128(n) || overlap(novel, n / 8, h, n / 8)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_DECODE, (cudaStream_t)stream);
    return from_cuda(gf2x::m128_decode(ctx, h, log2_u64(n) - 7, novel, 1, 0, (cudaStream_t)stream));
}

gf2x_status gf2x_m128_butterfly(gf2x_ctx *ctx, uint64_t *f, uint64_t n, void *stream)
{
    if (!ctx || !f || !aligned16(f)) return GF2X_EINVAL;
    if (n > kMaxTransformBits128) return GF2X_ETOOBIG;
    if (!valid_n128(n)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_BUTTERFLY, (cudaStream_t)stream);
    return from_cuda(gf2x::m128_butterfly(ctx, f, log2_u64(n) - 7, false, 1, 0, (cudaStream_t)stream));
}

gf2x_status gf2x_m128_ibutterfly(gf2x_ctx *ctx, uint64_t *f, uint64_t n, void *stream)
{
    if (!ctx || !f || !aligned16(f)) return GF2X_EINVAL;
    if (n > kMaxTransformBits128) return GF2X_ETOOBIG;
    if (!valid_n128(n)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_IBUTTERFLY, (cudaStream_t)stream);
    return from_cuda(gf2x::m128_butterfly(ctx, f, log2_u64(n) - 7, true, 1, 0, (cudaStream_t)stream));
}

gf2x_status gf2x_m128_pointwise(gf2x_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *c, uint64_t count,
                                void *stream)
{
    if (!ctx) return GF2X_EINVAL;
    if (!count) return GF2X_OK;
    if (!a || !b || !c || !aligned16(a) || !aligned16(b) || !aligned16(c)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    StageScope sc(ctx, STAGE_POINTWISE, (cudaStream_t)stream);
    return from_cuda(gf2x::m128_pointwise(ctx, a, b, c, count, (cudaStream_t)stream));
}

gf2x_status gf2x_selftest_wait_timeout(gf2x_ctx *ctx, void *stream)
{
    if (!ctx) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    return from_cuda(gf2x::wait_timeout_probe(ctx, ctx->d_sync, (cudaStream_t)stream));
}

gf2x_status gf2x_selftest_queue_timeout(gf2x_ctx *ctx, void *stream)
{
    if (!ctx) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    return from_cuda(gf2x::persist_selftest_timeout(ctx, (cudaStream_t)stream, 20000000ull));   // 20 ms
}

size_t gf2x_batch_workspace_bytes(const gf2x_job *jobs, size_t count)
{
    if (!jobs && count) return 0;
    BatchPlan bp;
    if (plan_batch(jobs, count, bp) != GF2X_OK) return 0;
    return bp.total_bytes + kAlign;
}

gf2x_status gf2x_mul_batch(gf2x_ctx *ctx, const gf2x_job *jobs, size_t count, void *ws, size_t ws_bytes, void *stream)
{
    if (!ctx || (!jobs && count)) return GF2X_EINVAL;
    BatchPlan bp;
    gf2x_status s = plan_batch(jobs, count, bp);
    if (s != GF2X_OK) return s;
    if (bp.table.empty()) return GF2X_OK;
    if (!ws || ((uintptr_t)ws % kAlign)) return GF2X_EINVAL;
    if (ws_bytes < bp.total_bytes + kAlign) return GF2X_ENOSPACE;
    for (const JobDev &j : bp.table)
        if (overlap(j.c, (size_t)((product_bits(j.na, j.nb) + 63) / 64) * 8, ws, bp.total_bytes)) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GF2X_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // the job table goes to the device before the kernels (every call)
    TRY(cudaMemcpyAsync(ws, bp.table.data(), bp.table.size() * sizeof(JobDev), cudaMemcpyHostToDevice, st));
    const std::vector<ClassRun> runs = bind_runs(bp, ws);
    // Two ways to run the classes, same results: one launch per kernel and class, or one
    // persistent launch for the whole batch (persist.cu: every class's launches recorded,
    // the plan uploaded to the workspace, one kernel drains it).  A pinned knob decides;
    // else the tuner times both on the first batch of each shape (job and class counts in
    // power-of-two buckets) and keeps the faster, the class launches unless the persistent
    // launch is more than 3% faster; a batch with a launch shape the persistent kernel lacks
    // runs class launches.
    gf2x::PersistLaunch pl{};
    u64 plan_digest = 0;
    auto prepare_persistent = [&](cudaStream_t s2) -> gf2x_status {
        std::vector<Recorder> recs(runs.size());
        std::vector<const Recorder *> rp;
        for (size_t c = 0; c < runs.size(); ++c) {
            recs[c].jobs = runs[c].count;
            ctx->rec = &recs[c];
            const gf2x_status rs = run_class(ctx, runs[c], s2);
            ctx->rec = nullptr;
            if (rs != GF2X_OK || !gf2x::persist_supported(recs[c])) return GF2X_EINVAL;
            rp.push_back(&recs[c]);
        }
        const int saved = ctx->stage;
        ctx->stage = STAGE_PERSIST;
        const cudaError_t pe = gf2x::persist_prepare(ctx, rp.data(), (int)rp.size(), (char *)ws + bp.persist_off,
                                                     bp.persist_bytes, s2, &pl);
        ctx->stage = saved;
        if (pe != cudaSuccess) return GF2X_ECUDA;
        plan_digest = pl.digest;
        return GF2X_OK;
    };
    auto run_classes = [&](cudaStream_t s2) -> gf2x_status {
        for (const ClassRun &r : runs) {
            gf2x_status e = run_class(ctx, r, s2);
            if (e != GF2X_OK) return e;
        }
        return GF2X_OK;
    };
    static const int modes[2] = {0, 1};
    int mode = gf2x::tune_pinned(ctx, gf2x::TUNE_BATCH_PERSIST, modes, 2, -1);
    if (mode < 0)
        mode = gf2x::tune_choice(ctx, gf2x::TUNE_BATCH_PERSIST,
                                 (gf2x::tune_bucket(bp.table.size()) << 8) | gf2x::tune_bucket(runs.size()), modes, 2,
                                 0,
                                 [&](int m) -> cudaError_t {
                                     gf2x_status r2 = GF2X_OK;
                                     if (m == 1) {
                                         r2 = prepare_persistent(st);
                                         if (r2 == GF2X_OK) r2 = from_cuda(gf2x::persist_launch(ctx, pl, st));
                                     } else {
                                         r2 = run_classes(st);
                                     }
                                     return r2 == GF2X_OK ? cudaSuccess : cudaErrorInvalidValue;
                                 },
                                 st);
    const bool persistent = mode == 1 && prepare_persistent(st) == GF2X_OK;
    auto run_all = [&](cudaStream_t s2) -> gf2x_status {
        if (persistent) {
            StageScope sc(ctx, STAGE_PERSIST, s2);
            return from_cuda(gf2x::persist_launch(ctx, pl, s2));
        }
        return run_classes(s2);
    };
    // graph cache, keyed by the job table and the workspace (second call captures)
    BatchCache *bc = (BatchCache *)ctx->batch_graphs;
    GraphCache *gc = graphs(ctx);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (gc->disabled || cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return run_all(st);
    const u64 key = hash_table(bp.table, ws);
    for (BatchGraph &e : bc->entries)
        if (e.key.same(key, ws, bp.table, plan_digest) && e.profiling == ctx->profiling && e.gen == gc->gen) {
            e.stamp = ++gc->clock;
            TRY(cudaGraphLaunch(e.exec, st));
            for (int k = 0; k < STAGE_COUNT; ++k) ctx->launches[k] += e.launches[k];
            if (ctx->profiling)
                for (const Rec &r : e.recs) profiler(ctx)->pending.push_back(r);
            return GF2X_OK;
        }
    bool repeat = false;
    for (size_t k = 0; k < bc->seen.size(); ++k)
        if (bc->seen[k].same(key, ws, bp.table, plan_digest)) {
            repeat = true;
            bc->seen.erase(bc->seen.begin() + (long)k);
            break;
        }
    if (!repeat) {
        if (bc->seen.size() >= 32) bc->seen.erase(bc->seen.begin());
        bc->seen.push_back(BatchKey{key, ws, bp.table, plan_digest});
        return run_all(st);
    }
    if (!gc->cap && cudaStreamCreateWithFlags(&gc->cap, cudaStreamNonBlocking) != cudaSuccess) return run_all(st);
    BatchGraph e{};
    e.key = BatchKey{key, ws, bp.table, plan_digest};
    e.profiling = ctx->profiling;
    unsigned long long before[STAGE_COUNT];
    for (int k = 0; k < STAGE_COUNT; ++k) before[k] = ctx->launches[k];
    Profiler *p = profiler(ctx);
    if (cudaStreamBeginCapture(gc->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return run_all(st);
    p->capture = &e.recs;
    s = run_all(gc->cap);
    p->capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(gc->cap, &graph);
    for (int k = 0; k < STAGE_COUNT; ++k) {
        e.launches[k] = ctx->launches[k] - before[k];
        ctx->launches[k] = before[k];
    }
    if (s != GF2X_OK || ce != cudaSuccess || !graph ||
        (cudaGraphInstantiate(&e.exec, graph, 0) != cudaSuccess)) {
        if (graph) cudaGraphDestroy(graph);
        for (Rec &r : e.recs) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
        cudaGetLastError();
        return s != GF2X_OK ? s : run_all(st);
    }
    cudaGraphDestroy(graph);
    if (bc->entries.size() >= kMaxBatchGraphs) {
        size_t old = 0;
        for (size_t k = 1; k < bc->entries.size(); ++k)
            if (bc->entries[k].stamp < bc->entries[old].stamp) old = k;
        cudaGraphExecDestroy(bc->entries[old].exec);
        for (Rec &r : bc->entries[old].recs) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
        bc->entries.erase(bc->entries.begin() + (long)old);
    }
    e.stamp = ++gc->clock;
    e.gen = gc->gen;
    bc->entries.push_back(e);
    BatchGraph &ent = bc->entries.back();
    TRY(cudaGraphLaunch(ent.exec, st));
    for (int k = 0; k < STAGE_COUNT; ++k) ctx->launches[k] += ent.launches[k];
    if (ctx->profiling)
        for (const Rec &r : ent.recs) p->pending.push_back(r);
    return GF2X_OK;
}

}  // extern "C"

namespace gf2x {

// gf2x_mul without its CUDA graph cache: the kernels are launched one by one
// on every call (instantiating a graph may allocate device memory).
gf2x_status mul_uncached(gf2x_ctx *ctx, const u64 *a, u64 na, const u64 *b, u64 nb, u64 *c, void *ws,
                         size_t ws_bytes, cudaStream_t st)
{
    bool empty = false;
    const gf2x_status s = check_mul(ctx, a, na, b, nb, c, ws, ws_bytes, &empty);
    if (s != GF2X_OK || empty) return s;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GF2X_ECUDA;
    return op_device(ctx, OP_MUL, a, na, b, nb, c, ws, st);
}

}  // namespace gf2x

extern "C" {

const char *gf2x_stage_name(int stage)
{
    static const char *names[STAGE_COUNT] = {"load", "basis_cvt", "encode", "butterfly", "pointwise",
                                             "ibutterfly", "decode", "ibasis_cvt", "store", "bottom_fused",
                                             "persistent_batch"};
    return (stage >= 0 && stage < STAGE_COUNT) ? names[stage] : "unknown";
}

int gf2x_stage_count(void) { return STAGE_COUNT; }

gf2x_status gf2x_profile_enable(gf2x_ctx *ctx, int enable)
{
    if (!ctx) return GF2X_EINVAL;
    DeviceGuard g(ctx->device);
    Profiler *p = profiler(ctx);
    if (!p->pending.empty()) cudaEventSynchronize(p->pending.back().e1);
    for (Rec &r : p->pending)
        if (r.pooled) { p->pool.push_back(r.e0); p->pool.push_back(r.e1); }
    p->pending.clear();
    for (double &m : p->ms) m = 0;
    for (auto &l : ctx->launches) l = 0;
    ctx->profiling = enable != 0;
    return GF2X_OK;
}

int gf2x_profile_read(gf2x_ctx *ctx, double *ms, uint64_t *launches, int max_stages)
{
    if (!ctx) return -1;
    DeviceGuard g(ctx->device);
    Profiler *p = profiler(ctx);
    if (!p->pending.empty()) {
        cudaEventSynchronize(p->pending.back().e1);
        for (Rec &r : p->pending) {
            float t = 0;
            if (cudaEventElapsedTime(&t, r.e0, r.e1) == cudaSuccess) p->ms[r.stage] += t;
            if (r.pooled) { p->pool.push_back(r.e0); p->pool.push_back(r.e1); }
        }
        p->pending.clear();
    }
    int n = max_stages < STAGE_COUNT ? max_stages : STAGE_COUNT;
    for (int k = 0; k < n; ++k) {
        if (ms) ms[k] = p->ms[k];
        if (launches) launches[k] = ctx->launches[k];
    }
    return STAGE_COUNT;
}

}  // extern "C"
