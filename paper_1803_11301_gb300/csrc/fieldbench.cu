// Field-multiply measurements: the GF(2^64) product forms this GPU offers,
// each timed on the same work (gf2x_bench_field_mul in include/gf2x.h).
//
// GB300 has no carry-less multiply instruction, so the product of Sec. 4.3
// (PCLMULQDQ on the paper's CPU) has to be built from other operations.  The
// Butterfly (Alg. 2) multiplies by twiddles that are shared by many
// butterflies in the high layers and by few in the low ones, and the
// pointwise step of Alg. 5 multiplies two arbitrary elements, so both
// "general x general" and "by a fixed element" forms matter.  Every variant
// runs the same dependent chains x <- c * x (four per thread, one constant c
// per launch) from the same seeds, so all give the same checksum; the timing
// is one launch on the caller's stream.
//
//   0 INT       32x32 integer multiplies on operands with 3-bit holes,
//               Karatsuba over the 32-bit halves, two-step fold (the earlier
//               form of gf64_mul)
//   1 INT_CONST the same with the constant's masked halves computed once
//   2 TAB4      16 four-bit windows of a table in shared memory (mul_tab,
//               the form the Butterfly kernels use)
//   3 TAB8      8 eight-bit windows (2 KiB per window, bank conflicts)
//   4 HYBRID    low 32 bits of x by 8 four-bit windows, high 32 bits by
//               integer multiplies
//   5 INT16     16x16 integer multiplies on operands with 2-bit holes (three
//               residue classes, 32-bit products only), Karatsuba twice: the
//               form gf64_mul uses
//   6 BITSLICE  64 elements of a warp as 64 bit-planes (lane t holds planes
//               t and t + 32), the product by c as its 64x64 GF(2) matrix:
//               every output plane XORs the input planes its row selects,
//               fetched from their lanes with warp shuffles
#include "gf2x_common.cuh"
#include "gf2x_tables.cuh"

namespace gf2x {
namespace {

constexpr int kBenchThreads = 256;
constexpr int kChains = 4;

enum FieldVariant { FV_INT = 0, FV_INT_CONST, FV_TAB4, FV_TAB8, FV_HYBRID, FV_INT16, FV_BITSLICE, FV_COUNT };

__device__ __forceinline__ u64 splitmix(u64 z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The earlier integer form of gf64_mul (clmul32_h4: 32-bit operands, four classes).
__device__ __forceinline__ u64 gf64_mul_h4(u64 a, u64 b)
{
    const u32 al = (u32)a, ah = (u32)(a >> 32), bl = (u32)b, bh = (u32)(b >> 32);
    const u64 lo = clmul32_h4(al, bl), hi = clmul32_h4(ah, bh);
    const u64 mid = clmul32_h4(al ^ ah, bl ^ bh) ^ lo ^ hi;
    return gf64_reduce(hi ^ (mid >> 32), lo ^ (mid << 32));
}

// clmul32_h4 with b given as its four masked classes.
__device__ __forceinline__ u64 clmul32_pre(u32 a, const u32 bm[4])
{
    const u32 m0 = 0x11111111u, m1 = 0x22222222u, m2 = 0x44444444u, m3 = 0x88888888u;
    const u32 a0 = a & m0, a1 = a & m1, a2 = a & m2, a3 = a & m3;
    const u64 z0 = ((u64)a0 * bm[0]) ^ ((u64)a1 * bm[3]) ^ ((u64)a2 * bm[2]) ^ ((u64)a3 * bm[1]);
    const u64 z1 = ((u64)a0 * bm[1]) ^ ((u64)a1 * bm[0]) ^ ((u64)a2 * bm[3]) ^ ((u64)a3 * bm[2]);
    const u64 z2 = ((u64)a0 * bm[2]) ^ ((u64)a1 * bm[1]) ^ ((u64)a2 * bm[0]) ^ ((u64)a3 * bm[3]);
    const u64 z3 = ((u64)a0 * bm[3]) ^ ((u64)a1 * bm[2]) ^ ((u64)a2 * bm[1]) ^ ((u64)a3 * bm[0]);
    return (z0 & 0x1111111111111111ull) | (z1 & 0x2222222222222222ull) | (z2 & 0x4444444444444444ull) |
           (z3 & 0x8888888888888888ull);
}

__device__ __forceinline__ void mask4(u32 b, u32 bm[4])
{
    bm[0] = b & 0x11111111u;
    bm[1] = b & 0x22222222u;
    bm[2] = b & 0x44444444u;
    bm[3] = b & 0x88888888u;
}

// Eight-bit windows: tab8[w * 256 + e] = c * (e x^(8w)).
__device__ __forceinline__ u64 mul_tab8(const u64 *tab8, u64 x)
{
    u64 r = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) r ^= tab8[w * 256 + ((x >> (8 * w)) & 255)];
    return r;
}

template <int V>
__global__ void __launch_bounds__(kBenchThreads) k_field_bench(u64 seed, u64 c, int steps,
                                                               unsigned long long *checksum)
{
    extern __shared__ u64 smem_raw[];
    u64 *tab = align128(smem_raw);
    const u64 gid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    u64 x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = splitmix(seed ^ (gid * kChains + k));

    if constexpr (V == FV_TAB4 || V == FV_HYBRID) {
        build_tables(launch_block(), tab, 1, [&](int) { return c; });
    } else if constexpr (V == FV_TAB8) {
        for (int k = threadIdx.x; k < 8 * 256; k += blockDim.x) {
            const int w = k >> 8, e = k & 255;
            u64 p = mul_xpow(c, 0);
            for (int s = 0; s < 8 * w; ++s) p = mul_x(p);       // c x^(8w)
            u64 r = 0;
            for (int b = 0; b < 8; ++b) {
                if ((e >> b) & 1) r ^= p;
                p = mul_x(p);
            }
            tab[k] = r;
        }
        __syncthreads();
    }

    if constexpr (V == FV_INT) {
        for (int s = 0; s < steps; ++s)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = gf64_mul_h4(c, x[k]);
    } else if constexpr (V == FV_INT_CONST) {
        u32 cl[4], ch[4], cm[4];
        mask4((u32)c, cl);
        mask4((u32)(c >> 32), ch);
        mask4((u32)c ^ (u32)(c >> 32), cm);
        for (int s = 0; s < steps; ++s)
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                const u32 al = (u32)x[k], ah = (u32)(x[k] >> 32);
                const u64 lo = clmul32_pre(al, cl), hi = clmul32_pre(ah, ch);
                const u64 mid = clmul32_pre(al ^ ah, cm) ^ lo ^ hi;
                x[k] = gf64_reduce(hi ^ (mid >> 32), lo ^ (mid << 32));
            }
    } else if constexpr (V == FV_TAB4) {
        const unsigned t = smem_addr(tab);
        for (int s = 0; s < steps; ++s)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = mul_tab(t, x[k]);
    } else if constexpr (V == FV_TAB8) {
        for (int s = 0; s < steps; ++s)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = mul_tab8(tab, x[k]);
    } else if constexpr (V == FV_HYBRID) {
        // c x = c (x_lo) + c (x_hi x^32): the low half by windows 0..7 of the
        // table, the high half by two integer products and a fold
        const unsigned t = smem_addr(tab);
        u32 cl[4], ch[4];
        mask4((u32)c, cl);
        mask4((u32)(c >> 32), ch);
        for (int s = 0; s < steps; ++s)
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                u64 r = 0;
                tab_window<0, 8>(r, t, (unsigned)x[k] ^ 0x76543210u, 0);   // windows 0..7: the low half
                const u32 xh = (u32)(x[k] >> 32);
                const u64 p0 = clmul32_pre(xh, cl), p1 = clmul32_pre(xh, ch);   // c_lo x_h, c_hi x_h
                // c x_h x^32 = p0 x^32 + p1 x^64
                const u64 hi = (p0 >> 32) ^ p1, low = p0 << 32;
                x[k] = r ^ gf64_reduce(hi, low);
            }
    } else if constexpr (V == FV_INT16) {
        for (int s = 0; s < steps; ++s)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = gf64_mul(c, x[k]);
    } else if constexpr (V == FV_BITSLICE) {
        // 64 elements per warp and vector: lane t holds elements t and t + 32
        // of two vectors (x[0], x[1]) and (x[2], x[3]); transposed, lane t
        // holds bit-planes t and t + 32 (bit e = bit of element e).
        const int lane = threadIdx.x & 31;
        u64 row_lo = 0, row_hi = 0;                 // rows t and t + 32 of the matrix of c
        u64 p = c;
        for (int k = 0; k < 64; ++k) {              // column k = c x^k
            row_lo |= ((p >> lane) & 1ull) << k;
            row_hi |= ((p >> (lane + 32)) & 1ull) << k;
            p = mul_x(p);
        }
        transpose64(x[0], x[1], lane);
        transpose64(x[2], x[3], lane);
        for (int s = 0; s < steps; ++s) {
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                u64 r_lo = 0, r_hi = 0;
#pragma unroll
                for (int k = 0; k < 64; ++k) {
                    const u64 w = __shfl_sync(0xffffffffu, k < 32 ? x[2 * v] : x[2 * v + 1], k & 31);
                    r_lo ^= w & (0ull - ((row_lo >> k) & 1ull));
                    r_hi ^= w & (0ull - ((row_hi >> k) & 1ull));
                }
                x[2 * v] = r_lo;
                x[2 * v + 1] = r_hi;
            }
        }
        transpose64(x[0], x[1], lane);
        transpose64(x[2], x[3], lane);
    }
    u64 acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc ^= x[k] * (2 * (u64)k + 1) ^ (gid << 1);
    atomicXor(checksum, (unsigned long long)acc);
}

template <int V>
cudaError_t launch_field(int blocks, u64 seed, u64 c, int steps, unsigned long long *sum, cudaStream_t st)
{
    size_t smem = 0;
    if (V == FV_TAB4 || V == FV_HYBRID) smem = kTab * sizeof(u64) + 128;
    if (V == FV_TAB8) smem = 8 * 256 * sizeof(u64) + 128;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_field_bench<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_field_bench<V><<<blocks, kBenchThreads, smem, st>>>(seed, c, steps, sum);
    return cudaGetLastError();
}

}  // namespace
}  // namespace gf2x

extern "C" gf2x_status gf2x_bench_field_mul(gf2x_ctx *ctx, int variant, int steps, uint64_t *checksum,
                                            double *ms, uint64_t *products, void *stream)
{
    using namespace gf2x;
    if (!ctx || variant < 0 || variant >= FV_COUNT || steps < 1 || steps > (1 << 20) || !checksum || !ms ||
        !products)
        return GF2X_EINVAL;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return GF2X_ECUDA;
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return GF2X_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = 8 * ctx->num_sms;
    const u64 seed = 0x18031130ull, c = 0x9E3779B97F4A7C15ull;       // any fixed non-zero constant
    unsigned long long *d_sum = ctx->d_word;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gf2x_status s = GF2X_OK;
    auto run = [&](int v) -> cudaError_t {
        switch (v) {
        case FV_INT: return launch_field<FV_INT>(blocks, seed, c, steps, d_sum, st);
        case FV_INT_CONST: return launch_field<FV_INT_CONST>(blocks, seed, c, steps, d_sum, st);
        case FV_TAB4: return launch_field<FV_TAB4>(blocks, seed, c, steps, d_sum, st);
        case FV_TAB8: return launch_field<FV_TAB8>(blocks, seed, c, steps, d_sum, st);
        case FV_HYBRID: return launch_field<FV_HYBRID>(blocks, seed, c, steps, d_sum, st);
        case FV_INT16: return launch_field<FV_INT16>(blocks, seed, c, steps, d_sum, st);
        default: return launch_field<FV_BITSLICE>(blocks, seed, c, steps, d_sum, st);
        }
    };
    unsigned long long h = 0;
    float t = 0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        run(variant) != cudaSuccess ||                                   // warm-up (kernel load)
        cudaMemsetAsync(d_sum, 0, sizeof(unsigned long long), st) != cudaSuccess ||
        cudaEventRecord(e0, st) != cudaSuccess || run(variant) != cudaSuccess ||
        cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
        cudaMemcpyAsync(&h, d_sum, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        s = GF2X_ECUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (prev != ctx->device) cudaSetDevice(prev);
    *checksum = h;
    *ms = t;
    *products = (uint64_t)blocks * kBenchThreads * kChains * (uint64_t)steps;
    return s;
}
