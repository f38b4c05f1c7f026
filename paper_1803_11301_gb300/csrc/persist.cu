// One persistent launch for a whole batch of products (Alg. 5 for every job).
//
// gf2x_mul_batch groups its jobs by transform length into size classes; each
// class runs the path's kernels (load, BasisCvt, Encode, Butterfly with the
// fused pointwise product, Decode, iBasisCvt, store) with one job per grid
// row.  Here the host records, class by class, the launches it would make
// (SegRec: block body, grid, block size, shared memory, arguments), and one
// persistent grid runs all their blocks from a device work queue:
//
//   * A queue item is a few blocks of one recorded launch (a segment), as many
//     as fit one CTA of kPersistThreads threads: sub-block k of the CTA has its
//     own named barrier and its own slice of shared memory.
//   * Items are numbered in queue order: segments of different classes
//     interleaved (round robin, the class with most work first), each
//     segment's blocks job by job.  A CTA takes the next number with one
//     atomicAdd, so items are claimed in queue order.
//   * Dependencies are per job: the blocks of job j in a segment start once
//     job j's blocks of the previous segment of its class have finished
//     (every block of every kernel of the path touches only its own job's
//     buffers).  Each segment keeps one completion counter per job.  So a
//     job's next stage starts as soon as that job's previous stage is done,
//     instead of after the whole launch, and small classes run alongside
//     large ones.
//   * A claimed item waits only for items earlier in the queue, which running
//     CTAs hold, so the queue always makes progress.  Every wait is bounded by
//     the global timer: when one runs out the CTA records GF2X_ETIMEOUT in the
//     context status word, raises the abort flag and returns; every other CTA
//     returns at its next claim or wait.
//
// A CTA has kPersistThreads = 256 threads and kPersistBlocksPerSM CTAs fit an
// SM: bodies of 256 threads run as one sub-block, the 2^16-bit BasisCvt body
// (128 threads) as two, the outer conversion in its 8-warp shape, the in-tile,
// column and Taylor-window bodies (written for 512 threads) with 256.  An item
// is up to 8 blocks per sub-block (while every job still spans at least 4
// items), so that claims, dependency checks and counter updates are paid once
// per several blocks; segment descriptors are searched in shared memory and
// a BasisCvt plan is staged there for the item.
//
// Memory ordering: a finished item's writes are released by a gpu-scope fence
// of its CTA's thread 0 after a CTA barrier, before the counter increment; the
// waiting thread acquires with a gpu-scope fence after its spin, before the
// CTA barrier that releases the item's threads.  Data written inside the
// launch is never read through the read-only path (GF2X_DATA_RESTRICT is
// empty here) and this file is compiled with global loads cached in L2 only.
#define GF2X_DATA_RESTRICT

#include <algorithm>
#include <cstring>
#include <vector>

#include "bfly_dev.cuh"
#include "cvt_dev.cuh"
#include "cvt_reg_dev.cuh"
#include "fft_dev.cuh"

Recorder::~Recorder()
{
    std::free(segs);
    std::free(blob);
}

bool record(gf2x_ctx *ctx, const SegRec &r)
{
    Recorder *rec = ctx->rec;
    if (!rec) return false;
    if (rec->nseg == rec->cap) {
        const int cap = rec->cap ? 2 * rec->cap : 64;
        SegRec *p = (SegRec *)std::realloc(rec->segs, (size_t)cap * sizeof(SegRec));
        if (!p) {
            rec->unsupported = true;
            return false;
        }
        rec->segs = p;
        rec->cap = cap;
    }
    rec->segs[rec->nseg++] = r;
    return true;
}

int record_blob(gf2x_ctx *ctx, const void *p, size_t n)
{
    Recorder *rec = ctx->rec;
    if (!rec) return -1;
    const size_t off = (rec->blob_bytes + 15) & ~(size_t)15;    // 16-byte pieces are staged in shared memory
    if (off + n > rec->blob_cap) {
        size_t cap = rec->blob_cap ? 2 * rec->blob_cap : 16384;
        while (cap < off + n) cap *= 2;
        unsigned char *q = (unsigned char *)std::realloc(rec->blob, cap);
        if (!q) {
            rec->unsupported = true;
            return -1;
        }
        rec->blob = q;
        rec->blob_cap = cap;
    }
    std::memcpy(rec->blob + off, p, n);
    rec->blob_bytes = off + n;
    return (int)off;
}

namespace gf2x {
namespace {

using cvtk::CvtPlan;

// A recorded launch as the persistent kernel reads it.
struct __align__(16) PSeg {
    int kind, i[4];
    unsigned gx, gy, threads;
    unsigned slice;       // shared-memory words of one sub-block (a multiple of 16: 128-byte aligned slices)
    unsigned q;           // sub-blocks per CTA
    unsigned g;           // blocks each sub-block runs per item: an item is q g blocks
    unsigned per_job;     // blocks of one job
    unsigned nvb;         // blocks of the launch
    unsigned vbase, vend; // the blocks this queue entry covers (the whole launch)
    unsigned item0;       // its first item in the queue
    int prev;             // the segment it follows in its class, or -1
    unsigned done_off;    // its per-job completion counters
    unsigned prev_done_off, prev_per_job;   // the previous segment's counters and their target
    unsigned plan_words;  // words of its BasisCvt plan (staged in shared memory), or 0
    const void *plan;     // device copy of its BasisCvt plan, or null
    u64 a[10];
};
static_assert(sizeof(PSeg) % 16 == 0, "segments are copied in 16-byte pieces");

struct PState {
    unsigned head;        // next item to claim
    unsigned abort;       // set when a wait ran out
    unsigned pad[2];
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned load_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int M>
__device__ __forceinline__ void run_outer(const PSeg &S, const VBlock &vb, u64 *sm)
{
    if (S.i[1]) cvtrk::cvt_outer_body<M, true, 8>(vb, sm, (u64 *)S.a[0], (const u64 *)S.a[1], S.i[2], S.a[2]);
    else cvtrk::cvt_outer_body<M, false, 8>(vb, sm, (u64 *)S.a[0], (const u64 *)S.a[1], S.i[2], S.a[2]);
}

template <int M>
__device__ __forceinline__ void run_top(const PSeg &S, const VBlock &vb, u64 *sm)
{
    if (S.i[1])
        bflyk::bfly_top_body<M, true>(vb, sm, (u64 *)S.a[0], (u64 *)S.a[1], (int)S.a[2], S.i[2], S.a[3], S.i[3],
                                      (const u64 *)S.a[4], (const u64 *)S.a[5], (int)S.a[6], S.a[7]);
    else
        bflyk::bfly_top_body<M, false>(vb, sm, (u64 *)S.a[0], (u64 *)S.a[1], (int)S.a[2], S.i[2], S.a[3], S.i[3],
                                       (const u64 *)S.a[4], (const u64 *)S.a[5], (int)S.a[6], S.a[7]);
}

// One block of a recorded launch.  The kinds and template choices are the ones
// the recorder accepts (see supported()).  `plan`: the segment's BasisCvt plan
// in shared memory.
__device__ __forceinline__ void run_block(const PSeg &S, const VBlock &vb, u64 *sm, const void *plan)
{
    const u64 *A = S.a;
    switch (S.kind) {
    case SEG_LOAD_JOBS:
        fftk::load_jobs_body(vb, (const JobDev *)A[0], S.i[0], (u64 *)A[1], A[2], A[3]);
        break;
    case SEG_STORE_JOBS:
        fftk::store_jobs_body(vb, (const u64 *)A[0], A[1], (const JobDev *)A[2]);
        break;
    case SEG_ENCODE:
        fftk::encode_body(vb, sm, (const u64 *)A[0], A[1], S.i[0], (const u64 *)A[2], (u64 *)A[3], A[4],
                          A[5], A[6]);
        break;
    case SEG_ENCODE_SMALL:
        fftk::encode_small_body(vb, (const u64 *)A[0], S.i[0], A[1], (const u64 *)A[2], (u64 *)A[3], A[4], A[5]);
        break;
    case SEG_DECODE:
        fftk::decode_body(vb, sm, (const u64 *)A[0], A[1], (const u64 *)A[2], (u64 *)A[3], A[4], A[5]);
        break;
    case SEG_DECODE_SMALL:
        fftk::decode_small_body(vb, sm, (const u64 *)A[0], S.i[0], (const u64 *)A[1], (u64 *)A[2], A[3]);
        break;
    case SEG_CVT_WIDE:
        cvtk::cvt_wide_body(vb, (u64 *)A[0], (const u64 *)A[1], A[3], A[4], A[5], S.i[1], A[2]);
        break;
    case SEG_CVT_TILE:
        cvtk::cvt_tile_body(vb, sm, (u64 *)A[0], (const u64 *)A[1], *(const CvtPlan *)plan, S.i[0], A[2]);
        break;
    case SEG_CVT_COL:
        cvtk::cvt_col_body(vb, sm, (u64 *)A[0], (const u64 *)A[1], *(const CvtPlan *)plan, S.i[0], A[2]);
        break;
    case SEG_CVT_TAYLOR:
        cvtk::cvt_taylor_body(vb, sm, (u64 *)A[0], (const u64 *)A[1], S.i[0], S.i[1], S.i[2], A[2]);
        break;
    case SEG_UNIT16:
        if (S.i[1]) cvtrk::cvt_unit16_body<true, 8>(vb, sm, (u64 *)A[0], A[1]);
        else cvtrk::cvt_unit16_body<false, 8>(vb, sm, (u64 *)A[0], A[1]);
        break;
    case SEG_OUTER:
        switch (S.i[0]) {
        case 2: run_outer<2>(S, vb, sm); break;
        case 3: run_outer<3>(S, vb, sm); break;
        case 4: run_outer<4>(S, vb, sm); break;
        case 5: run_outer<5>(S, vb, sm); break;
        case 6: run_outer<6>(S, vb, sm); break;
        case 7: run_outer<7>(S, vb, sm); break;
        default: run_outer<8>(S, vb, sm); break;
        }
        break;
    case SEG_TOP:
        switch (S.i[0]) {
        case 1: run_top<1>(S, vb, sm); break;
        case 2: run_top<2>(S, vb, sm); break;
        default: run_top<3>(S, vb, sm); break;
        }
        break;
    case SEG_BOTTOM:
        if (S.i[2] == 8)
            bflyk::bfly_bottom_body<8>(vb, sm, (u64 *)A[0], (u64 *)A[1], S.i[3], S.i[0], (const u64 *)A[2],
                                       (const u64 *)A[3], S.i[1], A[4]);
        else
            bflyk::bfly_bottom_body<16>(vb, sm, (u64 *)A[0], (u64 *)A[1], S.i[3], S.i[0], (const u64 *)A[2],
                                        (const u64 *)A[3], S.i[1], A[4]);
        break;
    default:
        break;
    }
}

// Waits until job j's blocks of segment P are done, or the limit or an abort
// ends the wait (false).  Thread 0 only.
__device__ bool wait_job(unsigned prev_off, unsigned prev_per_job, const unsigned *done, unsigned j, PState *state,
                         int *status, unsigned long long t0, unsigned long long limit_ns)
{
    const unsigned *c = done + prev_off + j;
    while (load_acquire(c) < prev_per_job) {
        if (*(volatile unsigned *)&state->abort) return false;
        if (global_ns() - t0 > limit_ns) {
            atomicCAS(status, (int)GF2X_OK, (int)GF2X_ETIMEOUT);
            atomicExch(&state->abort, 1u);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// Segments whose first items are searched in shared memory; a plan with more
// segments searches the global array.
constexpr int kSmemSegs = 2048;

__global__ void __launch_bounds__(kPersistThreads, kPersistBlocksPerSM)
    k_persist(const PSeg *__restrict__ segs, int nseg, unsigned items, unsigned *done, PState *state, int *status,
              unsigned long long limit_ns)
{
    extern __shared__ u64 smem_raw[];
    __shared__ unsigned s_item0[kSmemSegs];
    __shared__ PSeg s_pseg;
    __shared__ unsigned s_item;
    __shared__ int s_seg, s_go;
    const bool table = nseg <= kSmemSegs;
    if (table)
        for (int k = threadIdx.x; k < nseg; k += blockDim.x) s_item0[k] = segs[k].item0;
    int last = 0;                                         // segments only move forward for one CTA
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned it = atomicAdd(&state->head, 1u);
            const int go = it < items && !*(volatile unsigned *)&state->abort;
            int sg = last;
            if (go) {
                int lo = last, hi = nseg - 1;             // the segment holding item `it`
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if ((table ? s_item0[mid] : segs[mid].item0) <= it) lo = mid;
                    else hi = mid - 1;
                }
                sg = last = lo;
            }
            s_item = it;
            s_seg = sg;
            s_go = go;
        }
        __syncthreads();
        if (!s_go) break;
        if (threadIdx.x < sizeof(PSeg) / 16)              // the segment's descriptor, 16 bytes a thread
            ((uint4 *)&s_pseg)[threadIdx.x] = ((const uint4 *)(segs + s_seg))[threadIdx.x];
        __syncthreads();
        const PSeg &S = s_pseg;
        const unsigned q = S.q, per_item = q * S.g;
        const unsigned v0 = S.vbase + (s_item - S.item0) * per_item, v1 = min(v0 + per_item, S.vend);
        if (threadIdx.x == 0) {
            int go = 1;
            if (S.prev >= 0) {
                const unsigned long long t0 = global_ns();
                for (unsigned j = v0 / S.per_job; go && j <= (v1 - 1) / S.per_job; ++j)
                    go = wait_job(S.prev_done_off, S.prev_per_job, done, j, state, status, t0, limit_ns);
            }
            __threadfence();                              // acquire: the previous stage's data
            s_go = go;
        }
        // the plan of an in-tile or column run, staged after the sub-blocks' slices
        u64 *plan = smem_raw + (size_t)q * S.slice;
        for (unsigned k = threadIdx.x; k < S.plan_words / 2; k += blockDim.x)
            ((uint4 *)plan)[k] = ((const uint4 *)S.plan)[k];
        __syncthreads();
        if (!s_go) break;
        const unsigned threads = S.threads;
        const unsigned sub = threadIdx.x / threads;
        if (sub < q)
            for (unsigned v = v0 + sub; v < v1; v += q) {
                const VBlock vb{v % S.gx, v / S.gx, S.gx, S.gy, threadIdx.x % threads, threads, 1u + sub};
                // a body's last shared-memory reads end before the next body of this
                // sub-block writes its slice (an ordinary launch ends the block there)
                if (v != v0 + sub) vb.sync();
                run_block(S, vb, smem_raw + (size_t)sub * S.slice, plan);
            }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();                              // release: this item's writes
            for (unsigned j = v0 / S.per_job; j <= (v1 - 1) / S.per_job; ++j) {
                const unsigned a = max(v0, j * S.per_job), b = min(v1, (j + 1) * S.per_job);
                atomicAdd(&done[S.done_off + j], b - a);
            }
        }
    }
}

bool g_configured = false;

cudaError_t configure()
{
    if (g_configured) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPersistSmem);
    if (e == cudaSuccess) g_configured = true;
    return e;
}

// Whether run_block has the recorded launch's body, shape and shared memory.
bool supported(const SegRec &r)
{
    if (r.threads < 64 || r.threads > kPersistThreads || r.threads % 32 || kPersistThreads % r.threads) return false;
    const size_t plan = (r.kind == SEG_CVT_TILE || r.kind == SEG_CVT_COL) ? (sizeof(CvtPlan) + 15) / 16 * 16 : 0;
    if ((r.smem + 127) / 128 * 128 + plan > kPersistSmem) return false;
    switch (r.kind) {
    case SEG_UNIT16: return r.i[0] == 8;
    case SEG_OUTER: return r.i[0] >= 2 && r.i[0] <= 8;
    case SEG_TOP: return r.i[0] >= 1 && r.i[0] <= 3;
    case SEG_BOTTOM: return r.i[2] == 8 || r.i[2] == 16;
    default: return r.kind >= 0 && r.kind < SEG_KIND_COUNT;
    }
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s: far above any item's run time

}  // namespace

// Bytes of the device area the persistent launch needs for `classes` classes
// and `jobs` jobs in all (its segments, BasisCvt plans and counters), a bound
// that depends on those counts only.
size_t persist_area_bytes(size_t classes, size_t jobs)
{
    const size_t segs = classes * kPersistMaxSegs;       // queue entries: one per recorded launch
    return 256 + segs * sizeof(PSeg) + 256 + classes * (kPersistMaxPlanBytes + 256) + (size_t)kPersistMaxSegs * jobs * 4 +
           256;
}

size_t persist_seg_bytes() { return sizeof(PSeg); }

cudaError_t persist_prepare(gf2x_ctx *ctx, const Recorder *const *recs, int C, void *area, size_t area_bytes,
                            cudaStream_t st, PersistLaunch *out)
{
    cudaError_t e = configure();
    if (e != cudaSuccess) return e;
    // queue order: round robin over classes (most block-threads first), one segment each per round
    std::vector<u64> work((size_t)C, 0);
    for (int c = 0; c < C; ++c)
        for (int k = 0; k < recs[c]->nseg; ++k) {
            const SegRec &r = recs[c]->segs[k];
            work[(size_t)c] += (u64)r.gx * r.gy * r.threads;
        }
    std::vector<int> order((size_t)C);
    for (int c = 0; c < C; ++c) order[(size_t)c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[(size_t)x] > work[(size_t)y]; });
    // device area: [state 256][queue entries][plans of every class][per-job counters]
    char *base = (char *)area;
    const size_t off_state = 0, off_segs = 256;
    std::vector<size_t> blob_rel((size_t)C, 0);           // plans, relative to the plans' start
    size_t blob_total = 0;
    for (int c = 0; c < C; ++c) {
        blob_rel[(size_t)c] = blob_total;
        blob_total += (recs[c]->blob_bytes + 255) & ~(size_t)255;
    }
    // the segments as the persistent kernel runs them, one per recorded launch
    std::vector<PSeg> segs_all;
    std::vector<std::vector<int>> seg_of((size_t)C);
    unsigned counters = 0;
    for (int c = 0; c < C; ++c) {
        const Recorder *R = recs[c];
        int prev = -1;
        for (int k = 0; k < R->nseg; ++k) {
            const SegRec &r = R->segs[k];
            PSeg p{};
            p.kind = r.kind;
            for (int t = 0; t < 4; ++t) p.i[t] = r.i[t];
            p.gx = r.gx;
            p.gy = r.gy;
            p.threads = r.threads;
            p.slice = (unsigned)(((r.smem + 127) / 128) * 16);
            p.plan_words = (r.kind == SEG_CVT_TILE || r.kind == SEG_CVT_COL) ? (unsigned)((sizeof(CvtPlan) + 15) / 16 * 2)
                                                                          : 0u;
            unsigned q = kPersistThreads / r.threads;
            while (q > 1 && ((size_t)q * p.slice + p.plan_words) * 8 > kPersistSmem) --q;
            p.q = q;
            p.per_job = r.per_job;
            p.nvb = r.gx * r.gy;
            p.prev = prev;
            p.done_off = counters;
            if (prev >= 0) {
                p.prev_done_off = segs_all[(size_t)prev].done_off;
                p.prev_per_job = segs_all[(size_t)prev].per_job;
            }
            counters += (unsigned)R->jobs;
            // the plan's offset among the plans plus one, made an address once the layout is known
            p.plan = r.blob >= 0 ? (const void *)(uintptr_t)(1 + blob_rel[(size_t)c] + (size_t)r.blob) : nullptr;
            for (int t = 0; t < 10; ++t) p.a[t] = r.a[t];
            prev = (int)segs_all.size();
            seg_of[(size_t)c].push_back(prev);
            segs_all.push_back(p);
        }
    }
    // the queue: segments of the classes round robin (the class with most block-threads first)
    std::vector<PSeg> ps;
    std::vector<size_t> next((size_t)C, 0);
    unsigned items = 0;
    for (bool more = true; more;) {
        more = false;
        for (int c : order) {
            if (next[(size_t)c] >= seg_of[(size_t)c].size()) continue;
            more = true;
            PSeg p = segs_all[(size_t)seg_of[(size_t)c][next[(size_t)c]++]];
            // blocks per sub-block and item: up to 8, while every job still spans at least 4 items
            unsigned g = 1;
            while (g < 8 && 8 * g * p.q <= p.per_job) g *= 2;
            p.g = g;
            p.vbase = 0;
            p.vend = p.nvb;
            p.item0 = items;
            items += (p.nvb + p.q * g - 1) / (p.q * g);
            ps.push_back(p);
        }
    }
    const size_t off_blob = off_segs + ((ps.size() * sizeof(PSeg) + 255) & ~(size_t)255);
    const size_t off_done = off_blob + blob_total;
    for (PSeg &p : ps)
        if (p.plan) p.plan = base + off_blob + ((uintptr_t)p.plan - 1);
    const size_t need = off_done + (size_t)counters * 4;
    if (need > area_bytes || ps.empty() || items == 0) return cudaErrorInvalidValue;
    e = cudaMemcpyAsync(base + off_segs, ps.data(), ps.size() * sizeof(PSeg), cudaMemcpyHostToDevice, st);
    for (int c = 0; c < C && e == cudaSuccess; ++c)
        if (recs[c]->blob_bytes)
            e = cudaMemcpyAsync(base + off_blob + blob_rel[(size_t)c], recs[c]->blob, recs[c]->blob_bytes,
                                cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, kPersistThreads, kPersistSmem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    unsigned grid = (unsigned)(per_sm * ctx->num_sms);
    if (grid > items) grid = items;
    u64 h = 1469598103934665603ull;                      // FNV-1a over the segments and plans
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t k = 0; k < n; ++k) h = (h ^ b[k]) * 1099511628211ull;
    };
    mix(ps.data(), ps.size() * sizeof(PSeg));
    for (int c = 0; c < C; ++c) mix(recs[c]->blob, recs[c]->blob_bytes);
    *out = PersistLaunch{base + off_segs, base + off_done, base + off_state, (int)ps.size(), items, grid,
                         (size_t)counters * 4, h};
    return cudaSuccess;
}

cudaError_t persist_launch(gf2x_ctx *ctx, const PersistLaunch &pl, cudaStream_t st, unsigned long long limit_ns)
{
    cudaError_t e = configure();
    if (e == cudaSuccess) e = cudaMemsetAsync(pl.state, 0, sizeof(PState), st);
    if (e == cudaSuccess && pl.done_bytes) e = cudaMemsetAsync(pl.done, 0, pl.done_bytes, st);
    if (e != cudaSuccess) return e;
    k_persist<<<pl.grid, kPersistThreads, kPersistSmem, st>>>((const PSeg *)pl.segs, pl.nseg, pl.items,
                                                            (unsigned *)pl.done, (PState *)pl.state, ctx->d_status,
                                                            limit_ns ? limit_ns : kWaitLimitNs);
    count_launch(ctx);
    return cudaGetLastError();
}

cudaError_t persist_selftest_timeout(gf2x_ctx *ctx, cudaStream_t st, unsigned long long limit_ns)
{
    // segment 0: one block that does nothing, but its job counts as done only
    // after 2 blocks; segment 1: one block that waits for it
    PSeg ps[2] = {};
    for (int k = 0; k < 2; ++k) {
        ps[k].kind = SEG_KIND_COUNT;                      // no body
        ps[k].gx = ps[k].gy = 1;
        ps[k].threads = kPersistThreads;
        ps[k].q = 1;
        ps[k].nvb = 1;
        ps[k].vend = 1;
        ps[k].item0 = (unsigned)k;
        ps[k].done_off = (unsigned)k;
    }
    ps[0].per_job = 2;
    ps[0].prev = -1;
    ps[1].per_job = 1;
    ps[1].prev = 0;
    ps[1].prev_done_off = 0;
    ps[1].prev_per_job = 2;
    ps[0].g = ps[1].g = 1;
    char *base = (char *)ctx->d_state + kStateQueueOffset;
    static_assert(kStateQueueOffset + 256 + 2 * sizeof(PSeg) + 256 <= kStateBytes, "self-test queue fits");
    cudaError_t e = cudaMemcpyAsync(base + 256, ps, sizeof ps, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    PersistLaunch pl{base + 256, base + 256 + 2 * sizeof(PSeg), base, 2, 2, 2, 8, 0};
    return persist_launch(ctx, pl, st, limit_ns);
}

bool persist_supported(const Recorder &r)
{
    if (r.unsupported || r.nseg == 0 || r.nseg > (int)kPersistMaxSegs || r.blob_bytes > kPersistMaxPlanBytes)
        return false;
    for (int k = 0; k < r.nseg; ++k)
        if (!supported(r.segs[k])) return false;
    return true;
}

GF2X_OUT_OF_RANGE_READER(out_of_range_persist)

}  // namespace gf2x
