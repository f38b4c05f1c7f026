/*
 * CPU oracle for GF(2)[x] multiplication -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of bench.py load
 * this library.  It shares no code with the CUDA library.
 *
 * What it computes (Sec. 2.1: the product that FP_Polymul, Alg. 5, returns):
 *   c_k = XOR_{i+j=k} a_i b_j   for k < na + nb - 1,
 * the plain carry-less product.  Packed little-endian 64-bit words: bit t of
 * word w is the coefficient of x^(64 w + t).
 *
 *   oracle_clmul64   one 64x64 -> 128-bit carry-less product (4-bit windows)
 *   oracle_mul       schoolbook up to 32 words, Karatsuba above, OpenMP tasks
 *                    on the top levels, longer operand cut into chunks
 *   oracle_modcheck  c mod p == (a mod p)(b mod p) mod p for seeded random
 *                    irreducible monic p of degree 64 (Rabin's test)
 *   oracle_eval_at   A(beta) in GF(2^64) = GF(2)[x]/(x^64+x^4+x^3+x+1)
 *                    (Sec. 4.3), used to sample the forward transform, which
 *                    is evaluation at the partition Sigma (Eq. 8)
 *
 * Portable C only (no intrinsics): the same source builds on x86-64 and arm64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;

/* ------------------------------------------------------------------ clmul */
/* tab[t] = a * t for every 4-bit t, as a 67-bit value (tl[t], th[t]) */
static void clmul_table(u64 a, u64 tl[16], u64 th[16])
{
    for (int t = 0; t < 16; ++t) {
        u64 l = 0, h = 0;
        for (int k = 0; k < 4; ++k)
            if ((t >> k) & 1) {
                l ^= a << k;
                if (k) h ^= a >> (64 - k);
            }
        tl[t] = l;
        th[t] = h;
    }
}

/* a * b from a's table: Horner over the nibbles of b, top nibble first */
static void clmul_with_table(const u64 tl[16], const u64 th[16], u64 b, u64 *lo, u64 *hi)
{
    u64 rl = 0, rh = 0;
    for (int s = 60; s >= 0; s -= 4) {
        rh = (rh << 4) | (rl >> 60);
        rl <<= 4;
        unsigned t = (unsigned)(b >> s) & 15u;
        rl ^= tl[t];
        rh ^= th[t];
    }
    *lo = rl;
    *hi = rh;
}

void oracle_clmul64(u64 a, u64 b, u64 *lo, u64 *hi)
{
    u64 tl[16], th[16];
    clmul_table(a, tl, th);
    clmul_with_table(tl, th, b, lo, hi);
}

/* c[0 .. na+nb) ^= a[0..na) * b[0..nb), word schoolbook */
static void school(const u64 *a, size_t na, const u64 *b, size_t nb, u64 *c)
{
    for (size_t i = 0; i < na; ++i) {
        u64 tl[16], th[16];
        clmul_table(a[i], tl, th);
        for (size_t j = 0; j < nb; ++j) {
            u64 lo, hi;
            clmul_with_table(tl, th, b[j], &lo, &hi);
            c[i + j] ^= lo;
            c[i + j + 1] ^= hi;
        }
    }
}

#define KARA_BASE 32
#define KARA_TASK_MIN 4096

/* c[0..2n) = a[0..n) * b[0..n), n a power of two; ws holds >= 4n words. */
static void kara(const u64 *a, const u64 *b, size_t n, u64 *c, u64 *ws, int depth)
{
    if (n <= KARA_BASE) {
        memset(c, 0, 2 * n * sizeof(u64));
        school(a, n, b, n, c);
        return;
    }
    size_t h = n / 2;
    u64 *sa = ws, *sb = ws + h, *z1 = ws + 2 * h;   /* 4h = 2n words */
    for (size_t i = 0; i < h; ++i) {
        sa[i] = a[i] ^ a[h + i];
        sb[i] = b[i] ^ b[h + i];
    }
    if (depth < 3 && n >= KARA_TASK_MIN) {
        u64 *w0 = (u64 *)malloc(4 * h * sizeof(u64));
        u64 *w1 = (u64 *)malloc(4 * h * sizeof(u64));
        u64 *w2 = (u64 *)malloc(4 * h * sizeof(u64));
#pragma omp task shared(a, b, c) firstprivate(w0)
        kara(a, b, h, c, w0, depth + 1);                /* z0 = a0 b0 */
#pragma omp task shared(a, b, c) firstprivate(w1)
        kara(a + h, b + h, h, c + n, w1, depth + 1);    /* z2 = a1 b1 */
#pragma omp task shared(sa, sb, z1) firstprivate(w2)
        kara(sa, sb, h, z1, w2, depth + 1);             /* (a0+a1)(b0+b1) */
#pragma omp taskwait
        free(w0);
        free(w1);
        free(w2);
    } else {
        u64 *rest = ws + 4 * h;
        /* the recursive calls below need their own 4h words of scratch;
           the caller provides 8n words in total (see oracle_mul) */
        kara(a, b, h, c, rest, depth + 1);
        kara(a + h, b + h, h, c + n, rest, depth + 1);
        kara(sa, sb, h, z1, rest, depth + 1);
    }
    /* middle term: z1 - z0 - z2, added at x^(64 h) */
    for (size_t i = 0; i < n; ++i)
        z1[i] ^= c[i] ^ c[n + i];
    for (size_t i = 0; i < n; ++i)
        c[h + i] ^= z1[i];
}

static size_t next_pow2(size_t x)
{
    size_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

/* c = a * b.  na, nb in bits; c must hold ceil((na+nb-1)/64) words.
 * Bits of a, b at or above na, nb are ignored; bits of c above the product
 * length are written as zero.  Returns 0, or -1 if out of memory. */
int oracle_mul(const u64 *a, u64 na, const u64 *b, u64 nb, u64 *c)
{
    u64 nc = (na && nb) ? na + nb - 1 : 0;
    size_t wc = (size_t)((nc + 63) / 64);
    if (wc) memset(c, 0, wc * sizeof(u64));
    if (!nc) return 0;
    if (na < nb) {                     /* a is the longer operand */
        const u64 *t = a; a = b; b = t;
        u64 tn = na; na = nb; nb = tn;
    }
    size_t wa = (size_t)((na + 63) / 64), wb = (size_t)((nb + 63) / 64);
    size_t m = next_pow2(wb);
    u64 *A = (u64 *)calloc(m, sizeof(u64));
    u64 *B = (u64 *)calloc(m, sizeof(u64));
    u64 *P = (u64 *)malloc(2 * m * sizeof(u64));
    u64 *W = (u64 *)malloc(8 * m * sizeof(u64) + 64);
    u64 *C = (u64 *)calloc(wa + 2 * m + 1, sizeof(u64));
    if (!A || !B || !P || !W || !C) {
        free(A); free(B); free(P); free(W); free(C);
        return -1;
    }
    memcpy(B, b, wb * sizeof(u64));
    if (nb % 64) B[wb - 1] &= (~0ull) >> (64 - nb % 64);
    for (size_t off = 0; off < wa; off += m) {       /* chunks of the longer operand */
        size_t len = wa - off < m ? wa - off : m;
        memset(A, 0, m * sizeof(u64));
        memcpy(A, a + off, len * sizeof(u64));
        if (off + len == wa && na % 64) A[len - 1] &= (~0ull) >> (64 - na % 64);
#pragma omp parallel
#pragma omp single
        kara(A, B, m, P, W, 0);
        for (size_t i = 0; i < 2 * m; ++i) C[off + i] ^= P[i];
    }
    memcpy(c, C, wc * sizeof(u64));
    if (nc % 64) c[wc - 1] &= (~0ull) >> (64 - nc % 64);
    free(A); free(B); free(P); free(W); free(C);
    return 0;
}

/* ------------------------------------------------ arithmetic modulo x^64 + low */
typedef struct { u64 w[8][256]; } fold_tab;   /* (byte << 8k) * x^64 mod p */

static void fold_init(fold_tab *T, u64 low)
{
    u64 t[64];                                  /* t[j] = x^(64 + j) mod p */
    t[0] = low;
    for (int j = 1; j < 64; ++j)
        t[j] = (t[j - 1] << 1) ^ ((t[j - 1] >> 63) ? low : 0);
    for (int k = 0; k < 8; ++k)
        for (int v = 0; v < 256; ++v) {
            u64 r = 0;
            for (int bit = 0; bit < 8; ++bit)
                if ((v >> bit) & 1) r ^= t[8 * k + bit];
            T->w[k][v] = r;
        }
}

static u64 fold(const fold_tab *T, u64 h)      /* h * x^64 mod p */
{
    u64 r = 0;
    for (int k = 0; k < 8; ++k) r ^= T->w[k][(h >> (8 * k)) & 255];
    return r;
}

static u64 mulmod(const fold_tab *T, u64 a, u64 b)
{
    u64 lo, hi;
    oracle_clmul64(a, b, &lo, &hi);
    return lo ^ fold(T, hi);
}

/* remainder of the nbits-bit polynomial in words[] modulo p */
static u64 poly_mod(const fold_tab *T, const u64 *words, u64 nbits)
{
    size_t nw = (size_t)((nbits + 63) / 64);
    u64 r = 0;
    for (size_t i = nw; i-- > 0;) {
        u64 w = words[i];
        if (i == nw - 1 && nbits % 64) w &= (~0ull) >> (64 - nbits % 64);
        r = fold(T, r) ^ w;                     /* r * x^64 + w */
    }
    return r;
}

typedef unsigned __int128 u128;

static int deg128(u128 x)
{
    int d = -1;
    while (x) { x >>= 1; ++d; }
    return d;
}

static u128 gcd128(u128 a, u128 b)
{
    while (b) {
        int db = deg128(b);
        while (a && deg128(a) >= db) a ^= b << (deg128(a) - db);
        u128 t = a; a = b; b = t;
    }
    return a;
}

/* Rabin: x^64 + low is irreducible iff x^(2^64) = x mod p and
 * gcd(x^(2^32) - x, p) = 1 (64 has the single prime divisor 2). */
int oracle_irreducible64(u64 low)
{
    fold_tab *T = (fold_tab *)malloc(sizeof(fold_tab));
    if (!T) return -1;
    fold_init(T, low);
    u64 z = 2, z32 = 0;                          /* z = x */
    for (int k = 1; k <= 64; ++k) {
        z = mulmod(T, z, z);
        if (k == 32) z32 = z;
    }
    free(T);
    if (z != 2) return 0;
    u128 p = ((u128)1 << 64) | low;
    return gcd128((u128)(z32 ^ 2), p) == 1;
}

static u64 splitmix64(u64 *s)
{
    u64 z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The first `count` irreducible x^64 + low, drawing low from SplitMix64(seed). */
int oracle_random_irreducibles(u64 seed, int count, u64 *lows)
{
    u64 s = seed;
    int got = 0;
    while (got < count) {
        u64 low = splitmix64(&s) | 1;            /* p(0) = 0 would make x a factor */
        int r = oracle_irreducible64(low);
        if (r < 0) return -1;
        if (r) lows[got++] = low;
    }
    return 0;
}

/* For each p_i = x^64 + lows[i]: ok[i] = (c mod p == (a mod p)(b mod p) mod p).
 * Returns the number of p for which the identity holds. */
int oracle_modcheck(const u64 *a, u64 na, const u64 *b, u64 nb,
                    const u64 *c, u64 nc, const u64 *lows, int count, int *ok)
{
    int good = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : good)
    for (int i = 0; i < count; ++i) {
        fold_tab *T = (fold_tab *)malloc(sizeof(fold_tab));
        fold_init(T, lows[i]);
        u64 ra = poly_mod(T, a, na), rb = poly_mod(T, b, nb), rc = poly_mod(T, c, nc);
        ok[i] = (mulmod(T, ra, rb) == rc);
        good += ok[i];
        free(T);
    }
    return good;
}

/* A(beta) in GF(2)[x]/(x^64 + x^4 + x^3 + x + 1) for the nbits-bit A. */
u64 oracle_eval_at(const u64 *a, u64 nbits, u64 beta)
{
    fold_tab *T = (fold_tab *)malloc(sizeof(fold_tab));
    fold_init(T, 0x1Bull);
    u64 pw[64];                                  /* beta^t */
    pw[0] = 1;
    for (int t = 1; t < 64; ++t) pw[t] = mulmod(T, pw[t - 1], beta);
    u64 b64 = mulmod(T, pw[63], beta);           /* beta^64 */
    u64 win[8][256];                             /* sum of beta^(8k + bit) */
    for (int k = 0; k < 8; ++k)
        for (int v = 0; v < 256; ++v) {
            u64 r = 0;
            for (int bit = 0; bit < 8; ++bit)
                if ((v >> bit) & 1) r ^= pw[8 * k + bit];
            win[k][v] = r;
        }
    size_t nw = (size_t)((nbits + 63) / 64);
    u64 r = 0;
    for (size_t i = nw; i-- > 0;) {              /* Horner over words, step beta^64 */
        u64 w = a[i];
        if (i == nw - 1 && nbits % 64) w &= (~0ull) >> (64 - nbits % 64);
        u64 s = 0;
        for (int k = 0; k < 8; ++k) s ^= win[k][(w >> (8 * k)) & 255];
        r = mulmod(T, r, b64) ^ s;
    }
    free(T);
    return r;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
