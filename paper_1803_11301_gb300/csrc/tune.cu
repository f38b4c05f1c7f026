// Autotuner: launch-shape choices measured on this GPU, per shape, on first use.
//
// Several kernels have variants that compute the same result and differ only
// in speed, with the best one depending on the size (how many blocks a launch
// has against the SM count): the words per thread of the 2^16-bit BasisCvt
// kernel, the block shape of the fused bottom butterfly, the depth of the
// Taylor window kernel, the table chunk of the GF(2^128) bottom butterfly.  The first time a call meets a new (knob, key), and
// the stream is not being captured, the tuner runs every candidate a few
// times on a scratch buffer of the same layout (contents are garbage; every
// kernel's indexing is independent of the data), takes the fastest by CUDA
// events on the launching stream, and remembers it in the context.  Later
// calls, including the CUDA graphs captured from them, use the stored choice.
// The built-in default is kept unless a candidate is more than 3% faster.
// GF2X_TUNE=0 in the environment turns measuring off (the built-in defaults
// are then used); gf2x_tune_freeze stops it for one context (a server tunes
// during its warm-up, then freezes so that no request waits on a measurement).  The first call of a new shape synchronises its stream.
// gf2x_tune_pin fixes one knob's choice wherever it is among that call's
// candidates (reproducible launch shapes; tests run every variant this way).
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

constexpr int kKnobs = TUNE_KNOB_END;

struct TuneCache {
    std::vector<TuneEntry> entries;
    bool disabled = false;    // GF2X_TUNE=0: never measure
    bool frozen = false;      // gf2x_tune_freeze: stored choices and defaults only
    int pinned[kKnobs] = {};  // gf2x_tune_pin: 0 = not pinned, else the choice + 1
};

TuneCache *cache(gf2x_ctx *ctx) { return (TuneCache *)ctx->tuner; }

constexpr int kReps = 5;
constexpr float kMargin = 0.03f;


}  // namespace

void *tuner_create()
{
    TuneCache *c = new (std::nothrow) TuneCache();
    if (c)
        if (const char *env = std::getenv("GF2X_TUNE")) c->disabled = (env[0] == '0');
    return c;
}

void tuner_destroy(void *t) { delete (TuneCache *)t; }

void tuner_freeze(void *t, bool frozen)
{
    if (t) ((TuneCache *)t)->frozen = frozen;
}

void tuner_pin(void *t, int knob, int choice)
{
    if (t && knob > 0 && knob < kKnobs) ((TuneCache *)t)->pinned[knob] = choice < 0 ? 0 : choice + 1;
}

int tune_pinned(gf2x_ctx *ctx, int knob, const int *cands, int ncand, int fallback)
{
    TuneCache *c = cache(ctx);
    if (!c || knob <= 0 || knob >= kKnobs || !c->pinned[knob]) return fallback;
    for (int i = 0; i < ncand; ++i)
        if (cands[i] == c->pinned[knob] - 1) return cands[i];
    return fallback;
}

int tune_stored(gf2x_ctx *ctx, int knob, u64 key, int fallback)
{
    TuneCache *c = cache(ctx);
    if (c)
        for (const TuneEntry &e : c->entries)
            if (e.knob == knob && e.key == key) return e.choice;
    return fallback;
}

int tune_choice(gf2x_ctx *ctx, int knob, u64 key, const int *cands, int ncand, int fallback,
                const std::function<cudaError_t(int)> &run, cudaStream_t st)
{
    TuneCache *c = cache(ctx);
    if (!c) return fallback;
    const int pin = tune_pinned(ctx, knob, cands, ncand, -1);
    if (pin >= 0) return pin;
    for (const TuneEntry &e : c->entries)
        if (e.knob == knob && e.key == key) return e.choice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (c->disabled || c->frozen || ncand < 2 || recording(ctx) || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone)
        return fallback;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fallback;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fallback;
    }
    unsigned long long saved[STAGE_COUNT];           // measuring launches are not the caller's
    for (int k = 0; k < STAGE_COUNT; ++k) saved[k] = ctx->launches[k];
    // one untimed run of every candidate (first launches load the kernels and
    // warm the caches), then kReps rounds over all candidates, interleaved so
    // that drift of the clock or of other work on the GPU touches all alike;
    // each candidate keeps its fastest round
    bool ok = true;
    for (int i = 0; i < ncand && ok; ++i) ok = run(cands[i]) == cudaSuccess;
    std::vector<float> cand_ms((size_t)ncand, 0.0f);
    for (int rep = 0; rep < kReps && ok; ++rep) {
        for (int i = 0; i < ncand && ok; ++i) {
            ok = cudaEventRecord(e0, st) == cudaSuccess && run(cands[i]) == cudaSuccess &&
                 cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0;
            if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (ok && (rep == 0 || ms < cand_ms[(size_t)i])) cand_ms[(size_t)i] = ms;
        }
    }
    // the default stays unless a candidate beats it by more than kMargin:
    // choices within the run-to-run noise would otherwise flip between runs
    int best_i = 0;
    for (int i = 1; i < ncand; ++i)
        if (cand_ms[(size_t)i] < cand_ms[(size_t)best_i]) best_i = i;
    for (int i = 0; i < ncand; ++i)
        if (cands[i] == fallback && cand_ms[(size_t)i] <= (1.0f + kMargin) * cand_ms[(size_t)best_i]) best_i = i;
    const int best = cands[best_i];
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
