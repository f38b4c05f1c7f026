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
// words from 34 loaded), XORs, unskews 32 output words (one thread per skewed
// word and octet of rows), and for output words
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
constexpr int kLoThreads = (8 * (kLoW + 2) + 31) / 32 * 32;   // a task per (skewed word, row octet) of the widest window

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

// Operand sources of pass 1 read in place (ZetaIO): job j's words from
// src_j, words_j of them, the last one ANDed with mask_j; zero past them.
struct HiSrc {
    const u64 *src0, *src1;
    u64 words0, words1, mask0, mask1;
};

// Pass 1: row bits 6 .. m-1 (NB = m - 6 of them).  Block (u, window c) over
// skewed columns [c, c + W), W = 256 >> B; the first phase holds 2^A rows of
// one column in registers, the second (if B > 0) the other 2^B, through
// shared memory.  src (or, DIRECT, the operands of HiSrc) -> dst (main words)
// and side (overflow words).  At most 85 registers a thread: three blocks per
// SM keep enough loads in flight for this memory-bound pass.
template <int NB, bool DIRECT>
__global__ void __launch_bounds__(kZetaThreads, 3) k_cvt_zeta_hi(const u64 *__restrict__ src, u64 *__restrict__ dst,
                                                               u64 *__restrict__ side, u64 stride, u64 side_stride,
                                                               HiSrc ops)
{
    constexpr int A = NB < 5 ? NB : NB == 5 ? 4 : 5;   // row bits in registers, first phase
    constexpr int B = NB - A;
    constexpr int J = 1 << NB;
    constexpr int W = kZetaThreads >> B;
    constexpr int NWIN = (kRowWords + J - 1 + W - 1) / W;
    extern __shared__ u64 zt[];                       // [J][W] between the phases
    const int u = (int)(blockIdx.x / NWIN);
    const int c = (int)(blockIdx.x % NWIN) * W;
    unsigned nw = 0;                                  // DIRECT: words to read, mask of the last one
    u64 last = 0;
    if constexpr (DIRECT) {
        src = blockIdx.y ? ops.src1 : ops.src0;
        nw = (unsigned)(blockIdx.y ? ops.words1 : ops.words0);
        last = blockIdx.y ? ops.mask1 : ops.mask0;
    } else {
        src += (u64)blockIdx.y * stride;
    }
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
            const unsigned idx = row * kRowWords + x;
            if constexpr (DIRECT)
                v[i] = (x >= 0 && x < kRowWords && idx < nw) ? src[idx] & (idx + 1 == nw ? last : ~0ull) : 0;
            else
                v[i] = (x >= 0 && x < kRowWords && in_range(idx, (u64)kRowWords << (NB + 6))) ? src[idx] : 0;
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

// Bits [64 - s, 128 - s) of the 128-bit (hi:lo), i.e. (hi << s) | (lo >> (64 - s)),
// for 0 <= s < 64 (s = 0: hi), in 32-bit funnel shifts.
__device__ __forceinline__ u64 shl_pair(u64 hi, u64 lo, unsigned s)
{
    unsigned h0 = (unsigned)hi, h1 = (unsigned)(hi >> 32), l1 = (unsigned)(lo >> 32);
    if (s & 32) {
        h1 = h0;
        h0 = l1;
        l1 = (unsigned)lo;
    }
    const unsigned r = s & 31;
    return ((u64)__funnelshift_l(h0, h1, r) << 32) | __funnelshift_l(l1, h0, r);
}

// Bits [s, s + 64) of the 128-bit (hi:lo), i.e. (lo >> s) | (hi << (64 - s)),
// for 0 <= s < 64 (s = 0: lo).
__device__ __forceinline__ u64 shr_pair(u64 hi, u64 lo, unsigned s)
{
    unsigned l0 = (unsigned)lo, l1 = (unsigned)(lo >> 32), h0 = (unsigned)hi;
    if (s & 32) {
        l0 = l1;
        l1 = h0;
        h0 = (unsigned)(hi >> 32);
    }
    const unsigned r = s & 31;
    return ((u64)__funnelshift_r(l1, h0, r) << 32) | __funnelshift_r(l0, l1, r);
}

// 16-byte copy global -> shared of `bytes` (16, 8 or 0) bytes, zero-filling the rest.
__device__ __forceinline__ void copy16_part(u64 *dst_shared, const u64 *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst_shared)),
                 "l"(src), "r"(bytes)
                 : "memory");
}

constexpr int kLoPitch = 36;          // words per row of a pass-2 window: 18 aligned pairs, even for 16-byte copies

// Pass 2 window, first part: P's words [x0 - 1, x0 + NSK) of the 64 rows
// row0 .. row0+63 into buf, each row u skewed by u bits and summed over the
// row bits 0..5, in place: afterwards buf[u kLoPitch + s] holds word x0 + s of
// x^u gt_u, s < NSK.  The words load as 16-byte pairs from the even word
// xs = x0 - 1 - OFF (OFF = (x0 - 1) & 1): a pair lies in the main words or in
// the side words (the row boundary 1024 is even), a side pair that crosses the
// row's degree bound copies its first word and zero-fills the second.  One task
// per (skewed word, row octet): NSK x 8 <= kLoThreads.
template <int NSK, int OFF>
__device__ __forceinline__ void lo_window_sum(const u64 *main, const u64 *side, unsigned row0, int x0, int J,
                                              unsigned rows, u64 *buf)
{
    static_assert(8 * NSK <= kLoThreads && NSK + 1 + OFF <= kLoPitch, "one task per thread, one window per row");
    constexpr int NPAIR = kLoPitch / 2;
    const int xs = x0 - 1 - OFF;
    for (int e = (int)threadIdx.x; e < 64 * NPAIR; e += kLoThreads) {
        const int u = e / NPAIR, q = e - u * NPAIR;
        const unsigned row = row0 + (unsigned)u;
        const int x = xs + 2 * q;                   // even
        const u64 *p = main;
        int bytes = 0;
        if (x >= 0 && row < rows) {
            if (x < kRowWords) {
                p = main + row * kRowWords + x;
                bytes = 16;
            } else {
                const int xw = x - kRowWords, lim = J - 1 - (int)(row >> 6);
                p = side + row * J + xw;
                bytes = xw + 1 < lim ? 16 : xw < lim ? 8 : 0;
            }
        }
        copy16_part(buf + 2 * e, bytes ? p : main, bytes);
    }
    cvtk::copy_async_wait();
    __syncthreads();
    const int task = (int)threadIdx.x;
    const bool active = task < NSK * 8;
    const int sg = task % NSK, a = task / NSK;
    u64 v[8];
    if (active) {                                   // skew, then row bits 0..2 in registers
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int u = 8 * a + i;
            v[i] = shl_pair(buf[u * kLoPitch + sg + OFF + 1], buf[u * kLoPitch + sg + OFF], (unsigned)u);
        }
        superset_sum<3>(v);
    }
    __syncthreads();                                // every read of the loaded words is done
    if (active)
#pragma unroll
        for (int i = 0; i < 8; ++i) buf[(8 * a + i) * kLoPitch + sg] = v[i];
    __syncthreads();
    if (active) {                                   // row bits 3..5 (a is now the row's low octet index)
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = buf[(a + 8 * i) * kLoPitch + sg];
        superset_sum<3>(v);
#pragma unroll
        for (int i = 0; i < 8; ++i) buf[(a + 8 * i) * kLoPitch + sg] = v[i];
    }
    __syncthreads();
}

// Pass 2: row bits 0..5 and the carries.  Block (group of 64 rows, window c of
// 32 output words); main (+ side) -> dst.
// out (null: dst): the product's words written in place of the array's
// first out_words words (the last one ANDed with out_mask), one job.
template <bool INV>
__global__ void __launch_bounds__(kLoThreads) k_cvt_zeta_lo(const u64 *__restrict__ main, const u64 *__restrict__ side,
                                                             u64 *__restrict__ dst, u64 stride, u64 side_stride, int J,
                                                             unsigned rows, u64 *__restrict__ out, u64 out_words,
                                                             u64 out_mask)
{
    extern __shared__ __align__(16) u64 zs[];
    u64 *buf = zs;                                    // 64 x kLoPitch: loaded, then summed words
    u64 *O = buf + 64 * kLoPitch;                     // 64 x (kLoW + 1): overflow words [c - 1, c + kLoW)
    u64 *prev = O + 64 * (kLoW + 1);                  // kLoW: overflow of the previous group's last row
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
        lo_window_sum<kLoW + 2, 0>(main, side, row0, kRowWords + c - 1, J, rows, buf);   // x0 - 1 even
        for (int e = (int)threadIdx.x; e < 64 * (kLoW + 1); e += kLoThreads) {
            const int u = e / (kLoW + 1), o = e - u * (kLoW + 1);
            O[e] = shr_pair(buf[u * kLoPitch + o + 1], buf[u * kLoPitch + o], (unsigned)u);
        }
        __syncthreads();
    }
    lo_window_sum<kLoW + 1, 1>(main, side, row0, c, J, rows, buf);                      // x0 - 1 odd
    // two output words per thread: the summed words o, o+1, o+2 of the row
    for (int e = (int)threadIdx.x; e < 64 * (kLoW / 2); e += kLoThreads) {
        const int u = e / (kLoW / 2), o = 2 * (e - u * (kLoW / 2)), v = c + o;
        const ulonglong2 w01 = *reinterpret_cast<const ulonglong2 *>(buf + u * kLoPitch + o);
        const u64 w2 = buf[u * kLoPitch + o + 2];
        u64 g0 = shr_pair(w01.y, w01.x, (unsigned)u), g1 = shr_pair(w2, w01.y, (unsigned)u);
        if (carry) {
            const u64 *Ou = O + u * (kLoW + 1);
            const u64 op0 = u ? Ou[o + 1 - (kLoW + 1)] : prev[o];
            const u64 op1 = u ? Ou[o + 2 - (kLoW + 1)] : prev[o + 1];
            if (!INV) {
                const u64 ou0 = Ou[o + 1], ou1 = Ou[o + 2];
                const u64 om = v >= 1 ? Ou[o] : 0;
                g0 ^= (ou0 << 1) | (om >> 63);
                g1 ^= (ou1 << 1) | (ou0 >> 63);
            }
            g0 ^= op0;
            g1 ^= op1;
        }
        const unsigned row = row0 + (unsigned)u;
        const u64 idx = (u64)row * kRowWords + v;       // even
        if (out) {                                       // the caller's buffer: 8-byte aligned
            if (idx < out_words) out[idx] = idx + 1 == out_words ? g0 & out_mask : g0;
            if (idx + 1 < out_words) out[idx + 1] = idx + 2 == out_words ? g1 & out_mask : g1;
        } else if (in_range(idx + 1, (u64)rows * kRowWords)) {
            *reinterpret_cast<ulonglong2 *>(dst + idx) = make_ulonglong2(g0, g1);
        }
    }
}

constexpr size_t kLoSmem = (size_t)(64 * (kLoPitch + (kLoW + 1)) + kLoW) * 8;

template <int NB, bool DIRECT>
cudaError_t zeta_hi_run(const u64 *src, u64 *dst, u64 *side, u64 stride, u64 side_stride, int count, cudaStream_t st,
                        const HiSrc &ops)
{
    constexpr int A = NB < 5 ? NB : NB == 5 ? 4 : 5;   // row bits in registers, first phase
    constexpr int B = NB - A;
    constexpr int J = 1 << NB;
    constexpr int W = kZetaThreads >> B;
    constexpr int NWIN = (kRowWords + J - 1 + W - 1) / W;
    const size_t smem = B > 0 ? (size_t)J * W * 8 : 0;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_cvt_zeta_hi<NB, DIRECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem ? smem : 1));
        configured = true;
    }
    k_cvt_zeta_hi<NB, DIRECT><<<dim3(64 * NWIN, (unsigned)count), kZetaThreads, smem, st>>>(src, dst, side, stride,
                                                                                           side_stride, ops);
    return cudaGetLastError();
}

template <int NB>
cudaError_t zeta_hi_launch(const u64 *src, u64 *dst, u64 *side, u64 stride, u64 side_stride, int count, cudaStream_t st,
                           const HiSrc &ops, int direct)
{
    return direct ? zeta_hi_run<NB, true>(src, dst, side, stride, side_stride, count, st, ops)
                  : zeta_hi_run<NB, false>(src, dst, side, stride, side_stride, count, st, ops);
}

// ------------------------------------------------------ outer Taylor part
// The outer conversion of Alg. 1 (on the 2^m rows of 2^16 bits as units)
// starts with its own Taylor expansion at z^256 + z, z = x^tau: steps
// (256 2^k, 2^k) rows, k = m-9 .. 0.  A shift by whole rows moves every word
// column on its own, so the same reformulation holds per column with rows in
// place of bits: for the blocks F_Q of 256 rows (B = 2^(m-8) of them),
//     gt_R = sum_{Q superset of R} z^(Q - R) F_Q     (up to B - 1 - R rows beyond the block),
//     G_R = (gt_R mod z^256) + z o_R + o_{R-1}       (forward; o_R the overflow rows),
//     F_Q = (ft_Q mod z^256) + o_{Q-1}                (inverse, ft the same sum).
// Pass A (k_cvt_unit_zeta): a block holds, for one skewed row position
// p' = p + Q, a slab of W word columns of every block Q (row Q 256 + p' - Q),
// sums over the NQ = m - 8 block bits and writes row R 256 + p' - R back (in
// place: the same rows it read) or overflow row p' - R - 256 of block R to the
// side buffer (B rows of 1024 words per block).  Pass B (k_cvt_unit_fix) adds
// the overflow rows to the first B rows of every block.
template <int NQ>
struct UnitShape {
    static constexpr int A = NQ < 4 ? NQ : 4;     // block bits in registers, first phase
    static constexpr int B = NQ - A;              // second phase, through shared memory
    static constexpr int NB = 1 << NQ;            // blocks
    static constexpr int W = kZetaThreads >> B;   // word columns per CTA
    static constexpr size_t SMEM = B > 0 ? (size_t)NB * W * 8 : 0;
};

template <int NQ>
__global__ void __launch_bounds__(kZetaThreads) k_cvt_unit_zeta(u64 *__restrict__ bits, u64 *__restrict__ side,
                                                                 u64 stride, u64 side_stride)
{
    using Sh = UnitShape<NQ>;
    constexpr int A = Sh::A, B = Sh::B, NB = Sh::NB, W = Sh::W;
    constexpr int NCB = kRowWords / W;
    extern __shared__ u64 ut[];                       // [NB][W] between the phases
    const int pp = (int)(blockIdx.x / NCB);           // skewed row position, 0 .. 256 + NB - 2
    const int c0 = (int)(blockIdx.x % NCB) * W;
    bits += (u64)blockIdx.y * stride;
    side += (u64)blockIdx.y * side_stride;
    constexpr u64 kWords = (u64)kRowWords << (NQ + 8);
    auto store = [&](int r, int w, u64 val) {
        const int p = pp - r;                         // row of block r
        if (p < 0) return;
        if (p < 256) {
            const unsigned i = (unsigned)(r * 256 + p) * kRowWords + c0 + w;
            if (in_range(i, kWords)) bits[i] = val;
        } else if (p - 256 < NB - 1 - r) {
            const unsigned i = (unsigned)(r * NB + p - 256) * kRowWords + c0 + w;
            if (in_range(i, (u64)NB * NB * kRowWords)) side[i] = val;
        }
    };
    const int w = (int)threadIdx.x % W, s = (int)threadIdx.x / W;
    u64 v[1 << A];
#pragma unroll
    for (int i = 0; i < (1 << A); ++i) {
        const int q = (s << A) + i, p = pp - q;
        const unsigned idx = (unsigned)(q * 256 + p) * kRowWords + c0 + w;
        v[i] = (p >= 0 && p < 256 && in_range(idx, kWords)) ? bits[idx] : 0;
    }
    superset_sum<A>(v);
    if constexpr (B == 0) {
#pragma unroll
        for (int i = 0; i < (1 << A); ++i) store((s << A) + i, w, v[i]);
    } else {
#pragma unroll
        for (int i = 0; i < (1 << A); ++i) ut[((s << A) + i) * W + w] = v[i];
        __syncthreads();
        for (int task = (int)threadIdx.x; task < (W << A); task += kZetaThreads) {
            const int ww = task % W, b = task / W;
            u64 x[1 << B];
#pragma unroll
            for (int i = 0; i < (1 << B); ++i) x[i] = ut[(b + (i << A)) * W + ww];
            superset_sum<B>(x);
#pragma unroll
            for (int i = 0; i < (1 << B); ++i) store(b + (i << A), ww, x[i]);
        }
    }
}

// Pass B: rows p < B of block r get o_{r-1}[p] and (forward) o_r[p - 1].
template <bool INV>
__global__ void __launch_bounds__(kZetaThreads) k_cvt_unit_fix(u64 *__restrict__ bits, const u64 *__restrict__ side,
                                                                int NB, u64 stride, u64 side_stride)
{
    bits += (u64)blockIdx.y * stride;
    side += (u64)blockIdx.y * side_stride;
    const u64 e = (u64)blockIdx.x * kZetaThreads + threadIdx.x;   // (block r, row p < NB, word c)
    const int c = (int)(e % kRowWords);
    const u64 rp = e / kRowWords;
    const int p = (int)(rp % (u64)NB), r = (int)(rp / (u64)NB);
    if (r >= NB) return;
    auto o = [&](int rr, int t) -> u64 {               // overflow row t of block rr, zero beyond its degree
        return rr >= 0 && t >= 0 && t < NB - 1 - rr ? side[((u64)rr * NB + t) * kRowWords + c] : 0;
    };
    u64 add = o(r - 1, p);
    if (!INV) add ^= o(r, p - 1);
    const u64 i = ((u64)r * 256 + p) * kRowWords + c;
    if (in_range(i, (u64)NB * 256 * kRowWords)) bits[i] ^= add;
}

template <int NQ>
cudaError_t unit_zeta_launch(u64 *bits, u64 *side, u64 stride, u64 side_stride, int count, cudaStream_t st)
{
    using Sh = UnitShape<NQ>;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_cvt_unit_zeta<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(Sh::SMEM ? Sh::SMEM : 1));
        configured = true;
    }
    const unsigned grid = (unsigned)((256 + Sh::NB - 1) * (kRowWords / Sh::W));
    k_cvt_unit_zeta<NQ><<<dim3(grid, (unsigned)count), kZetaThreads, Sh::SMEM, st>>>(bits, side, stride, side_stride);
    return cudaGetLastError();
}

}  // namespace

u64 taylor_zeta_side_words(int m) { return m >= 9 && m <= 16 ? 1ull << (2 * m - 6) : 0; }

// The Taylor part of BasisCvt(2^(m + 16)) (forward: f -> g) or of iBasisCvt
// (g -> f), 9 <= m <= 16: pass 1 from bits into scratch (main words) and side
// (taylor_zeta_side_words(m) words per job, side_stride apart), pass 2 back
// into bits.
cudaError_t taylor_zeta(gf2x_ctx *ctx, u64 *bits, u64 *scratch, u64 *side, u64 side_stride, int m, bool inverse,
                        int count, u64 stride, cudaStream_t st, const ZetaIO *io)
{
    HiSrc ops{};
    int direct = 0;
    if (!inverse && io && io->src[0]) {               // the operands read in place (at most two jobs)
        if (count > 2 || (count == 2 && !io->src[1])) return cudaErrorInvalidValue;
        auto words = [](u64 bits) { return (bits + 63) / 64; };
        auto mask = [](u64 bits) { return (bits & 63) ? (~0ull >> (64 - (bits & 63))) : ~0ull; };
        ops.src0 = io->src[0];
        ops.words0 = words(io->src_bits[0]);
        ops.mask0 = mask(io->src_bits[0]);
        if (count == 2) {
            ops.src1 = io->src[1];
            ops.words1 = words(io->src_bits[1]);
            ops.mask1 = mask(io->src_bits[1]);
        }
        direct = 1;
    }
    u64 *out = nullptr, out_words = 0, out_mask = ~0ull;
    if (inverse && io && io->dst) {                    // the product written in place of the array
        if (count != 1) return cudaErrorInvalidValue;
        out = io->dst;
        out_words = (io->dst_bits + 63) / 64;
        if (io->dst_bits & 63) out_mask = ~0ull >> (64 - (io->dst_bits & 63));
    }
    cudaError_t e;
    switch (m - 6) {
    case 3: e = zeta_hi_launch<3>(bits, scratch, side, stride, side_stride, count, st, ops, direct); break;
    case 4: e = zeta_hi_launch<4>(bits, scratch, side, stride, side_stride, count, st, ops, direct); break;
    case 5: e = zeta_hi_launch<5>(bits, scratch, side, stride, side_stride, count, st, ops, direct); break;
    case 6: e = zeta_hi_launch<6>(bits, scratch, side, stride, side_stride, count, st, ops, direct); break;
    case 7: e = zeta_hi_launch<7>(bits, scratch, side, stride, side_stride, count, st, ops, direct); break;
    case 8: e = zeta_hi_launch<8>(bits, scratch, side, stride, side_stride, count, st, ops, direct); break;
    case 9: e = zeta_hi_launch<9>(bits, scratch, side, stride, side_stride, count, st, ops, direct); break;
    case 10: e = zeta_hi_launch<10>(bits, scratch, side, stride, side_stride, count, st, ops, direct); break;
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
        k_cvt_zeta_lo<true><<<grid, kLoThreads, kLoSmem, st>>>(scratch, side, bits, stride, side_stride, J, rows, out,
                                                               out_words, out_mask);
    else
        k_cvt_zeta_lo<false><<<grid, kLoThreads, kLoSmem, st>>>(scratch, side, bits, stride, side_stride, J, rows,
                                                                nullptr, 0, ~0ull);
    count_launch(ctx);
    return cudaGetLastError();
}

GF2X_OUT_OF_RANGE_READER(out_of_range_zeta)

}  // namespace gf2x

namespace gf2x {

// The Taylor part of the outer conversion of BasisCvt(2^(m + 16)) (forward)
// or of iBasisCvt, 10 <= m <= 16: in place on bits, side as for taylor_zeta.
cudaError_t outer_taylor_zeta(gf2x_ctx *ctx, u64 *bits, u64 *side, u64 side_stride, int m, bool inverse, int count,
                              u64 stride, cudaStream_t st)
{
    cudaError_t e;
    switch (m - 8) {
    case 2: e = unit_zeta_launch<2>(bits, side, stride, side_stride, count, st); break;
    case 3: e = unit_zeta_launch<3>(bits, side, stride, side_stride, count, st); break;
    case 4: e = unit_zeta_launch<4>(bits, side, stride, side_stride, count, st); break;
    case 5: e = unit_zeta_launch<5>(bits, side, stride, side_stride, count, st); break;
    case 6: e = unit_zeta_launch<6>(bits, side, stride, side_stride, count, st); break;
    case 7: e = unit_zeta_launch<7>(bits, side, stride, side_stride, count, st); break;
    case 8: e = unit_zeta_launch<8>(bits, side, stride, side_stride, count, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    count_launch(ctx);
    const int NB = 1 << (m - 8);
    const u64 items = (u64)NB * NB * kRowWords;
    const dim3 grid((unsigned)((items + kZetaThreads - 1) / kZetaThreads), (unsigned)count);
    if (inverse) k_cvt_unit_fix<true><<<grid, kZetaThreads, 0, st>>>(bits, side, NB, stride, side_stride);
    else k_cvt_unit_fix<false><<<grid, kZetaThreads, 0, st>>>(bits, side, NB, stride, side_stride);
    count_launch(ctx);
    return cudaGetLastError();
}

}  // namespace gf2x
