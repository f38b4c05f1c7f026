// Multiplication by a fixed GF(2^64) element through a table in shared memory
// (the method of four Russians, Sec. 4.5), shared by the Butterfly kernels
// (bfly.cu) and the field-multiply measurements (fieldbench.cu).
//
// For a fixed c, tab[w][e] = c * (e x^(4w)) for the 16 four-bit windows w and
// e < 16, so c*x = XOR_w tab[w][nibble_w(x)].  A window table is 16 x 8 bytes,
// exactly the 32 shared-memory banks, so the 32 lanes of a warp never
// conflict.  A table is built from the 64 powers c x^k: each entry XORs at
// most four.
#pragma once

#include "gf2x_common.cuh"

namespace gf2x {

constexpr int kTab = 256;            // u64 entries per multiplication table

// c * x^(4w) mod the field polynomial.
__device__ __forceinline__ u64 mul_xpow(u64 c, int e)
{
    if (e == 0) return c;
    return gf64_reduce(c >> (64 - e), c << e);
}

// Window w keeps entry e at slot e ^ w, so that the 16 threads writing one
// window each (build) and the 32 lanes reading one window (lookup) touch
// distinct bank pairs.  `tab` is the table's shared-memory address, 128-byte
// aligned: XORing nibble w of x with w is one XOR of x with 0xFEDCBA98..10,
// and the byte offset (slot * 8) of window w is one shift and one LOP3 that
// also ORs in the table address; the window's 128-byte base is the load's
// immediate offset.
// Windows W .. END-1 (END <= 16).
template <int W, int END = 16>
__device__ __forceinline__ void tab_window(u64 &r, unsigned tab, unsigned lo, unsigned hi)
{
    constexpr int k = 4 * (W & 7);                      // bit of nibble W in its half
    const unsigned src = W < 8 ? lo : hi;
    const unsigned a = ((k >= 3 ? src >> (k - 3) : src << (3 - k)) & 0x78u) | tab;
    u64 v;
    asm volatile("ld.shared.u64 %0, [%1+%2];" : "=l"(v) : "r"(a), "n"(W * 128));
    r ^= v;
    if constexpr (W + 1 < END) tab_window<W + 1, END>(r, tab, lo, hi);
}

__device__ __forceinline__ u64 mul_tab(unsigned tab, u64 x)
{
    u64 r = 0;
    tab_window<0>(r, tab, (unsigned)x ^ 0x76543210u, (unsigned)(x >> 32) ^ 0xFEDCBA98u);
    return r;
}

// Shared-memory address of p.
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Dynamic shared memory rounded up to 128 bytes (launches request 128 more):
// the table addresses must be 128-byte aligned for mul_tab.
__device__ __forceinline__ u64 *align128(u64 *p) { return (u64 *)(((uintptr_t)p + 127) & ~(uintptr_t)127); }

__device__ __forceinline__ u64 mul_x(u64 p) { return (p << 1) ^ ((p >> 63) * GF2X_MOD_LOW); }

// Build nt tables: thread (t, w) computes the powers c x^(4w+b), b < 4, of
// twiddle c = twid(t) and writes the 16 entries of window w (Gray-code XORs).
// Ends with the block's barrier.
template <class F>
__device__ __forceinline__ void build_tables(const VBlock &vb, u64 *tabs, int nt, F twid)
{
    for (int k = vb.t; k < nt * 16; k += vb.nt) {
        const int t = k >> 4, w = k & 15;
        const u64 c = twid(t);
        u64 p[4];
        p[0] = mul_xpow(c, 4 * w);
        p[1] = mul_x(p[0]);
        p[2] = mul_x(p[1]);
        p[3] = mul_x(p[2]);
        u64 *dst = tabs + (size_t)t * kTab + w * 16;
        u64 e = 0;
        dst[0 ^ w] = 0;
#pragma unroll
        for (int g = 1; g < 16; ++g) {            // Gray code: flip the lowest set bit of g
            e ^= p[(g & 1) ? 0 : (g & 2) ? 1 : (g & 4) ? 2 : 3];
            dst[(g ^ (g >> 1)) ^ w] = e;
        }
    }
    vb.sync();
}

}  // namespace gf2x
