// gf2x_mul_noalloc: the product for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocator: a framework that has
// reserved the whole device for its own pool, or a code path where entering an
// allocator is not allowed (its implicit synchronisation, its locks or its
// failure modes are unacceptable there).  This entry point needs no workspace
// from the caller: its scratch is a fixed array in device memory, defined
// below, that every GPU loading this library holds until the process exits.
//
// The product runs the kernels of gf2x_mul one by one on every call: it never
// captures or instantiates a CUDA graph, since instantiation may allocate.
//
// The array's name is only a host-side stand-in in host code, not a device
// address, so host code never passes it to a kernel.  The first call on each
// device, with that device current, asks the runtime for the array's device
// address (cudaGetSymbolAddress) and keeps it; later calls reuse it.
#include <mutex>

#include "gf2x_common.cuh"

namespace {

// Scratch for the largest product this entry point accepts: three buffers
// of n/8 bytes and 256 bytes of barrier state (see gf2x_workspace_bytes) for
// n = GF2X_NOALLOC_MAX_TRANSFORM_BITS.
constexpr size_t kScratchBytes = 3 * (GF2X_NOALLOC_MAX_TRANSFORM_BITS / 8) + 256;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchBytes / 8];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
void *g_scratch_addr[kMaxDevices];   // device address of g_noalloc_scratch, per device

// Device address of the scratch array on `device` (which must be current).
gf2x_status scratch_address(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) return GF2X_ENODEV;
    std::lock_guard<std::mutex> lock(g_setup_lock);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GF2X_ECUDA;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return GF2X_OK;
}

}  // namespace

extern "C" gf2x_status gf2x_mul_noalloc(gf2x_ctx *ctx, const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                                        uint64_t nb_bits, uint64_t *c, void *stream)
{
    if (!ctx) return GF2X_EINVAL;
    const uint64_t n = gf2x_transform_bits(na_bits, nb_bits);
    if (n == 0) return GF2X_OK;                        // empty product: nothing to write
    if (n > GF2X_NOALLOC_MAX_TRANSFORM_BITS) return GF2X_ETOOBIG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return GF2X_ECUDA;
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return GF2X_ECUDA;
    void *scratch = nullptr;
    gf2x_status s = scratch_address(ctx->device, &scratch);
    if (prev != ctx->device) cudaSetDevice(prev);
    if (s != GF2X_OK) return s;
    // Direct launches: gf2x_mul would capture and instantiate a CUDA graph from
    // the second identical call on, and instantiation may allocate.
    return gf2x::mul_uncached(ctx, a, na_bits, b, nb_bits, c, scratch, kScratchBytes, (cudaStream_t)stream);
}
