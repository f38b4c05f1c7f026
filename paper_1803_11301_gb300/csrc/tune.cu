// Autotuner: launch-shape choices measured on this GPU, per shape, on first use.
//
// Several kernels have variants that compute the same result and differ only
// in speed, with the best one depending on the size (how many blocks a launch
// has against the SM count): the words per thread of the 2^16-bit BasisCvt
// kernel, the block shape of the fused bottom butterfly, the depth of the
// Taylor window kernel.  The first time a call meets a new (knob, key), and
// the stream is not being captured, the tuner runs every candidate a few
// times on a scratch buffer of the same layout (contents are garbage; every
// kernel's indexing is independent of the data), takes the fastest by CUDA
// events on the launching stream, and remembers it in the context.  Later
// calls, including the CUDA graphs captured from them, use the stored choice.
// GF2X_TUNE=0 in the environment turns measuring off (the built-in defaults
// are then used).  The first call of a new shape synchronises its stream.
#include <cstdlib>
#include <vector>

#include "gf2x_common.cuh"

namespace gf2x {
namespace {

struct TuneEntry {
    int knob;
    u64 key;
    int choice;
};

struct TuneCache {
    std::vector<TuneEntry> entries;
    bool disabled = false;
};

TuneCache *cache(gf2x_ctx *ctx) { return (TuneCache *)ctx->tuner; }

constexpr int kReps = 3;

}  // namespace

void *tuner_create()
{
    TuneCache *c = new (std::nothrow) TuneCache();
    if (c)
        if (const char *env = std::getenv("GF2X_TUNE")) c->disabled = (env[0] == '0');
    return c;
}

void tuner_destroy(void *t) { delete (TuneCache *)t; }

int tune_choice(gf2x_ctx *ctx, int knob, u64 key, const int *cands, int ncand, int fallback,
                const std::function<cudaError_t(int)> &run, cudaStream_t st)
{
    TuneCache *c = cache(ctx);
    if (!c) return fallback;
    for (const TuneEntry &e : c->entries)
        if (e.knob == knob && e.key == key) return e.choice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (c->disabled || ncand < 2 || cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return fallback;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fallback;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fallback;
    }
    unsigned long long saved[STAGE_COUNT];           // measuring launches are not the caller's
    for (int k = 0; k < STAGE_COUNT; ++k) saved[k] = ctx->launches[k];
    int best = fallback;
    float best_ms = 0;
    bool ok = true;
    for (int i = 0; i < ncand && ok; ++i) {
        float cand_ms = 0;
        for (int rep = 0; rep < kReps && ok; ++rep) {
            ok = cudaEventRecord(e0, st) == cudaSuccess && run(cands[i]) == cudaSuccess &&
                 cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0;
            if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (ok && (rep == 0 || ms < cand_ms)) cand_ms = ms;
        }
        if (ok && (i == 0 || cand_ms < best_ms)) {
            best_ms = cand_ms;
            best = cands[i];
        }
    }
    for (int k = 0; k < STAGE_COUNT; ++k) ctx->launches[k] = saved[k];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) {
        cudaGetLastError();
        return fallback;
    }
    c->entries.push_back({knob, key, best});
    return best;
}

}  // namespace gf2x
