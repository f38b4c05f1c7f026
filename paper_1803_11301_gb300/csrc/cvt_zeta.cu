// Taylor expansion of BasisCvt (Alg. 1, Sec. 2.3.1) at y = x^tau + x,
// tau = 2^16, as two superset-sum passes over HBM instead of one pass per
// division layer.
//
// Write the L-bit array as f = sum_q x^(tau q) f_q with 2^m rows f_q of tau
// bits.  In characteristic 2, x^tau = y + x gives (Lucas)
//     x^(tau q) = (y + x)^q = sum_{r subset of q} y^r x^(q - r),
// so f = sum_r y^r gt_r with
//     gt_r = sum_{q superset of r} x^(q - r) f_q        (degree < tau + 2^m - 1).
// The overflow o_r = gt_r >> tau (degree < 2^m) goes back through
// x^tau = y + x once more:
//     g_r = (gt_r mod x^tau) + x o_r + o_{r-1},
// which has degree < tau: this is the unique expansion f = sum_r g_r y^r that
// the division steps (h, d) = (tau 2^k, 2^k), k = m-1 .. 0, compute.  The
// inverse (f from the g_r, Alg. 1 undone) is the same superset sum,
//     ft_q = sum_{r superset of q} x^(r - q) g_r,
// followed by the carries of plain rows: f_q = (ft_q mod x^tau) + (ft_{q-1} >> tau).
//
// The superset sum has one layer per bit of the row index, and the layers
// commute.  Multiplying row q by x^q ("skew") turns every layer into an XOR of
// two rows at the same bit positions: sum_{q sup r} x^q f_q = x^r gt_r.
//
// Pass 1 (k_cvt_zeta_hi) takes the row bits 6 .. m-1, whose shifts are whole
// words.  Rows q = u + 64 j of one u are skewed by j words; a block holds
// skewed word columns [c, c + W) of all J = 2^(m-6) of them, XORs them and
// writes every row back unskewed, a diagonal band of each row, so blocks need
// no halo.  Its rows P_q = sum_{j' sup j} x^(64 (j' - j)) f_{u + 64 j'} reach
// J - 1 - j words past the row (degree bound), kept in a side buffer of J
// words per row; words beyond the bound are never written and read as zero.
//
// Pass 2 (k_cvt_zeta_lo) takes the row bits 0..5: 64 consecutive rows, shifts
// below one word.  A block skews each row u of its group by u bits (33 skewed
// words from 34 loaded), XORs, unskews 32 output words, and for output words
// below J adds the carries, from the rows' overflow words computed the same
// way in a second window.  The carry into the group's first row comes from the
// last row of the previous group: all its low row bits are set, so its
// superset sum has one term and its overflow is P's side words as pass 1 left
// them.
#include "cvt_dev.cuh"

namespace gf2x {
namespace {

constexpr int kRowWords = 1024;          // tau = 2^16 bits
constexpr int kZetaThreads = 256;
constexpr int kLoW = 32;                 // pass 2: output words per block and row
constexpr int kLoLoad = kLoW + 3;        // widest loaded window (the overflow one)
constexpr int kLoSkew = kLoW + 2;

// 8-byte copy global -> shared, or zeros when `valid` is false (no bytes read).
__device__ __forceinline__ void copy8_or_zero(u64 *dst_shared, const u64 *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst_shared)),
                 "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}

// Superset sum over the N index bits of v[0 .. 2^N): v[i] ^= v[i + 2^t] for
// every i without bit t.
template <int N>
__device__ __forceinline__ void superset_sum(u64 *v)
{
#pragma unroll
    for (int t = 0; t < N; ++t)
#pragma unroll
        for (int i = 0; i < (1 << N); ++i)
            if (!(i & (1 << t))) v[i] ^= v[i + (1 << t)];
}

// Pass 1: row bits 6 .. m-1 (NB = m - 6 of them).  Block (u, window c) over
// skewed columns [c, c + W), W = 256 >> B; the first phase holds 2^A rows of
// one column in registers, the second (if B > 0) the other 2^B, through
// shared memory.  src -> dst (main words) and side (overflow words).
template <int NB>
__global__ void __launch_bounds__(kZetaThreads) k_cvt_zeta_hi(const u64 *__restrict__ src, u64 *__restrict__ dst,
                                                               u64 *__restrict__ side, u64 stride, u64 side_stride)
{
    constexpr int A = NB < 5 ? NB : 5;
    constexpr int B = NB - A;
    constexpr int J = 1 << NB;
    constexpr int W = kZetaThreads >> B;
    constexpr int NWIN = (kRowWords + J - 1 + W - 1) / W;
    extern __shared__ u64 zt[];                       // [J][W] between the phases
    const int u = (int)(blockIdx.x / NWIN);
    const int c = (int)(blockIdx.x % NWIN) * W;
    src += (u64)blockIdx.y * stride;
    dst += (u64)blockIdx.y * stride;
    side += (u64)blockIdx.y * side_stride;
    auto store = [&](int j, int w, u64 val) {
        const int v = c + w - j;                      // unskewed word of row u + 64 j
        const unsigned row = (unsigned)(u + 64 * j);
        if (v < 0) return;
        if (v < kRowWords) {
            if (in_range((u64)row * kRowWords + v, (u64)kRowWords << (NB + 6))) dst[row * kRowWords + v] = val;
        } else if (v - kRowWords < J - 1 - j) {
            if (in_range((u64)row * J + (v - kRowWords), (u64)J << (NB + 6))) side[row * J + (v - kRowWords)] = val;
        }
    };
    {
        const int w = (int)threadIdx.x % W, s = (int)threadIdx.x / W;   // W << B == kZetaThreads tasks
        u64 v[1 << A];
#pragma unroll
        for (int i = 0; i < (1 << A); ++i) {
            const int j = (s << A) + i;
            const int x = c + w - j;
            const unsigned row = (unsigned)(u + 64 * j);
            v[i] = (x >= 0 && x < kRowWords && in_range((u64)row * kRowWords + x, (u64)kRowWords << (NB + 6)))
                       ? src[row * kRowWords + x]
                       : 0;
        }
        superset_sum<A>(v);
#pragma unroll
        for (int i = 0; i < (1 << A); ++i) {
            if (B == 0) store((s << A) + i, w, v[i]);
            else zt[((s << A) + i) * W + w] = v[i];
        }
    }
    if (B == 0) return;
    __syncthreads();
    for (int task = (int)threadIdx.x; task < (W << A); task += kZetaThreads) {
        const int w = task % W, b = task / W;
        u64 v[1 << (B > 0 ? B : 1)];
#pragma unroll
        for (int i = 0; i < (1 << B); ++i) v[i] = zt[(b + (i << A)) * W + w];
        superset_sum<B>(v);
#pragma unroll
        for (int i = 0; i < (1 << B); ++i) store(b + (i << A), w, v[i]);
    }
}

// P_row word x of pass 1's output (main words, then the side words below the
// row's degree bound, zero elsewhere): its address, or null for a zero.
__device__ __forceinline__ const u64 *p_word(const u64 *main, const u64 *side, unsigned row, int x, int J, unsigned rows)
{
    if (x < 0 || row >= rows) return nullptr;
    if (x < kRowWords) return main + row * kRowWords + x;
    const int xs = x - kRowWords;
    return xs < J - 1 - (int)(row >> 6) ? side + row * J + xs : nullptr;
}

// Pass 2 window: gt of the 64 rows row0 .. row0+63 for the words
// [x0, x0 + nsk - 1), from P's words [x0 - 1, x0 + nsk); into out[u * ostride + o].
__device__ __forceinline__ void lo_window(const u64 *main, const u64 *side, unsigned row0, int x0, int nsk, int J,
                                          unsigned rows, u64 *tile, u64 *S, u64 *out, int ostride)
{
    const int nld = nsk + 1;
    for (int e = (int)threadIdx.x; e < 64 * nld; e += kZetaThreads) {
        const int u = e / nld, k = e - u * nld;
        const u64 *p = p_word(main, side, row0 + u, x0 - 1 + k, J, rows);
        copy8_or_zero(tile + e, p ? p : main, p != nullptr);
    }
    cvtk::copy_async_wait();
    __syncthreads();
    // skew row u by u bits, then the layers of row bits 0..2 in registers
    for (int task = (int)threadIdx.x; task < nsk * 8; task += kZetaThreads) {
        const int sg = task % nsk, a = task / nsk;
        u64 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int u = 8 * a + i;
            const u64 hi = tile[u * nld + sg + 1], lo = tile[u * nld + sg];
            v[i] = u == 0 ? hi : (hi << u) | (lo >> (64 - u));
        }
        superset_sum<3>(v);
#pragma unroll
        for (int i = 0; i < 8; ++i) S[(8 * a + i) * nsk + sg] = v[i];
    }
    __syncthreads();
    for (int task = (int)threadIdx.x; task < nsk * 8; task += kZetaThreads) {   // row bits 3..5
        const int sg = task % nsk, b = task / nsk;
        u64 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = S[(b + 8 * i) * nsk + sg];
        superset_sum<3>(v);
#pragma unroll
        for (int i = 0; i < 8; ++i) S[(b + 8 * i) * nsk + sg] = v[i];
    }
    __syncthreads();
    for (int e = (int)threadIdx.x; e < 64 * (nsk - 1); e += kZetaThreads) {    // unskew
        const int u = e / (nsk - 1), o = e - u * (nsk - 1);
        const u64 lo = S[u * nsk + o], hi = S[u * nsk + o + 1];
        out[u * ostride + o] = u == 0 ? lo : (lo >> u) | (hi << (64 - u));
    }
    __syncthreads();
}

// Pass 2: row bits 0..5 and the carries.  Block (group of 64 rows, window c of
// 32 output words); main (+ side) -> dst.
template <bool INV>
__global__ void __launch_bounds__(kZetaThreads) k_cvt_zeta_lo(const u64 *__restrict__ main, const u64 *__restrict__ side,
                                                               u64 *__restrict__ dst, u64 stride, u64 side_stride, int J,
                                                               unsigned rows)
{
    extern __shared__ u64 zs[];
    u64 *tile = zs;                                   // 64 x kLoLoad
    u64 *S = tile + 64 * kLoLoad;                     // 64 x kLoSkew
    u64 *O = S + 64 * kLoSkew;                        // 64 x (kLoW + 1): overflow words [c - 1, c + kLoW)
    u64 *G = O + 64 * (kLoW + 1);                     // 64 x kLoW: gt of the output words
    u64 *prev = G + 64 * kLoW;                        // kLoW: overflow of the previous group's last row
    constexpr int nwin = kRowWords / kLoW;
    const unsigned grp = blockIdx.x / nwin;
    const int c = (int)(blockIdx.x % nwin) * kLoW;
    const unsigned row0 = grp * 64;
    main += (u64)blockIdx.y * stride;
    dst += (u64)blockIdx.y * stride;
    side += (u64)blockIdx.y * side_stride;
    const bool carry = c < J;
    if (carry) {
        if (threadIdx.x < kLoW) {
            const u64 *p = grp > 0 ? p_word(main, side, row0 - 1, kRowWords + c + (int)threadIdx.x, J, rows) : nullptr;
            prev[threadIdx.x] = p ? *p : 0;
        }
        lo_window(main, side, row0, kRowWords + c - 1, kLoW + 2, J, rows, tile, S, O, kLoW + 1);
    }
    lo_window(main, side, row0, c, kLoW + 1, J, rows, tile, S, G, kLoW);
    for (int e = (int)threadIdx.x; e < 64 * kLoW; e += kZetaThreads) {
        const int u = e / kLoW, o = e - u * kLoW, v = c + o;
        u64 val = G[u * kLoW + o];
        if (carry) {
            const u64 op = u ? O[(u - 1) * (kLoW + 1) + o + 1] : prev[o];
            if (!INV) {
                const u64 ou = O[u * (kLoW + 1) + o + 1];
                const u64 om = v >= 1 ? O[u * (kLoW + 1) + o] : 0;
                val ^= (ou << 1) | (om >> 63);
            }
            val ^= op;
        }
        const unsigned row = row0 + (unsigned)u;
        if (in_range((u64)row * kRowWords + v, (u64)rows * kRowWords)) dst[row * kRowWords + v] = val;
    }
}

constexpr size_t kLoSmem = (size_t)(64 * (kLoLoad + kLoSkew + (kLoW + 1) + kLoW) + kLoW) * 8;

template <int NB>
cudaError_t zeta_hi_launch(const u64 *src, u64 *dst, u64 *side, u64 stride, u64 side_stride, int count, cudaStream_t st)
{
    constexpr int A = NB < 5 ? NB : 5;
    constexpr int B = NB - A;
    constexpr int J = 1 << NB;
    constexpr int W = kZetaThreads >> B;
    constexpr int NWIN = (kRowWords + J - 1 + W - 1) / W;
    const size_t smem = B > 0 ? (size_t)J * W * 8 : 0;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_cvt_zeta_hi<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem ? smem : 1));
        configured = true;
    }
    k_cvt_zeta_hi<NB><<<dim3(64 * NWIN, (unsigned)count), kZetaThreads, smem, st>>>(src, dst, side, stride, side_stride);
    return cudaGetLastError();
}

}  // namespace

u64 taylor_zeta_side_words(int m) { return m >= 9 && m <= 16 ? 1ull << (2 * m - 6) : 0; }

// The Taylor part of BasisCvt(2^(m + 16)) (forward: f -> g) or of iBasisCvt
// (g -> f), 9 <= m <= 16: pass 1 from bits into scratch (main words) and side
// (taylor_zeta_side_words(m) words per job, side_stride apart), pass 2 back
// into bits.
cudaError_t taylor_zeta(gf2x_ctx *ctx, u64 *bits, u64 *scratch, u64 *side, u64 side_stride, int m, bool inverse,
                        int count, u64 stride, cudaStream_t st)
{
    cudaError_t e;
    switch (m - 6) {
    case 3: e = zeta_hi_launch<3>(bits, scratch, side, stride, side_stride, count, st); break;
    case 4: e = zeta_hi_launch<4>(bits, scratch, side, stride, side_stride, count, st); break;
    case 5: e = zeta_hi_launch<5>(bits, scratch, side, stride, side_stride, count, st); break;
    case 6: e = zeta_hi_launch<6>(bits, scratch, side, stride, side_stride, count, st); break;
    case 7: e = zeta_hi_launch<7>(bits, scratch, side, stride, side_stride, count, st); break;
    case 8: e = zeta_hi_launch<8>(bits, scratch, side, stride, side_stride, count, st); break;
    case 9: e = zeta_hi_launch<9>(bits, scratch, side, stride, side_stride, count, st); break;
    case 10: e = zeta_hi_launch<10>(bits, scratch, side, stride, side_stride, count, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    count_launch(ctx);
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_cvt_zeta_lo<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLoSmem);
        cudaFuncSetAttribute(k_cvt_zeta_lo<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLoSmem);
        configured = true;
    }
    const unsigned rows = 1u << m;
    const dim3 grid((rows / 64) * (kRowWords / kLoW), (unsigned)count);
    const int J = 1 << (m - 6);
    if (inverse)
        k_cvt_zeta_lo<true><<<grid, kZetaThreads, kLoSmem, st>>>(scratch, side, bits, stride, side_stride, J, rows);
    else
        k_cvt_zeta_lo<false><<<grid, kZetaThreads, kLoSmem, st>>>(scratch, side, bits, stride, side_stride, J, rows);
    count_launch(ctx);
    return cudaGetLastError();
}

GF2X_OUT_OF_RANGE_READER(out_of_range_zeta)

}  // namespace gf2x
