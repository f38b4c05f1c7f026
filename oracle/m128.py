"""The m = 128 variant of FP_Polymul (Sec. 3 for general m, Sec. 4.3) -- oracle side.

Test infrastructure only: imported by tests/, never by the library.

The method with m = 128 instead of 64 (Sec. 4, "m = 64 and 128"): points are
elements of GF(2^128) = GF(2)[x] / (x^128 + x^7 + x^2 + x + 1) (Sec. 4.3, the
AES-GCM representation), n_p = n / 128 of them, the partition is
Sigma = v_{l+64} + V_l (Eq. 6 with m/2 = 64), and Encode collapses the first
l_m = log2(128) = 7 layers of the truncated Butterfly (Sec. 3.3).  BasisCvt
(Alg. 1) works on GF(2)[x] and is the same as for m = 64.

Elements are Python ints < 2^128 (bit t = coefficient of x^t); vectors of
points are Python lists.  Plain and slow: for the sizes the tests use.
"""

from __future__ import annotations

from . import field as F
from . import stages as S

M = 128
LM = 7                                      # l_m = log2(m)
POLY_LOW = (1 << 7) | (1 << 2) | (1 << 1) | 1   # x^128 = x^7 + x^2 + x + 1
MASK = (1 << M) - 1


def gf_mul(a: int, b: int) -> int:
    """Product in GF(2^128): shift-and-add, reducing x^128 at every step."""
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a >> M:
            a = (a & MASK) ^ POLY_LOW
    return r


def gf_sqr(a: int) -> int:
    return gf_mul(a, a)


# -------------------------------------------------------------- Cantor basis
_CANTOR: list[int] | None = None


def cantor_basis() -> list[int]:
    """v_0 .. v_127 (Eq. 2): v_0 = 1 and v_i^2 + v_i = v_{i-1}, root with bit 0 clear."""
    global _CANTOR
    if _CANTOR is None:
        # y -> y^2 + y is GF(2)-linear; row k is the image of x^k
        rows = [gf_sqr(1 << k) ^ (1 << k) for k in range(M)]
        v = [1]
        for i in range(1, M):
            y = F.gf2_solve(rows, v[i - 1], M)
            if y is None:
                raise ArithmeticError(f"y^2 + y = v_{i - 1} has no root in GF(2^128)")
            if y & 1:
                y ^= 1
            v.append(y)
        _CANTOR = v
    return list(_CANTOR)


def cantor_to_poly(coords: int) -> int:
    """sum_j b_j v_j for the Cantor coordinates coords = sum_j b_j 2^j."""
    v = cantor_basis()
    r = 0
    j = 0
    while coords:
        if coords & 1:
            r ^= v[j]
        coords >>= 1
        j += 1
    return r


def s_eval(i: int, a: int) -> int:
    """s_i(a): s_i is the sum of the terms x^(2^j) listed by ``field.s_coeffs``."""
    terms = set(F.s_coeffs(i))
    r = 0
    p = a
    for j in range(i + 1):
        if j in terms:
            r ^= p
        p = gf_sqr(p)
    return r


def frobenius_order(a: int) -> int:
    b = gf_sqr(a)
    j = 1
    while b != a:
        b = gf_sqr(b)
        j += 1
    return j


# ------------------------------------------------------------ sizes, points
def transform_length(na: int, nb: int) -> int:
    """n = max(128, next power of two >= na + nb - 1): n_p = n/128 >= 1 point."""
    return max(M, S.next_pow2(na + nb - 1))


def alpha_of(l: int) -> int:
    """alpha = v_{l + m/2} = v_{l + 64} (Eq. 6)."""
    return cantor_to_poly(1 << (l + 64))


def sigma_point(l: int, k: int) -> int:
    """alpha + u_k, u_k with Cantor coordinates k."""
    return cantor_to_poly((1 << (l + 64)) ^ k)


def twiddle(l: int, i: int, s: int) -> int:
    """s_i(alpha + u_s), the multiplier of the layer-i block starting at s."""
    return s_eval(i, sigma_point(l, s))


class Twiddles:
    """s_i(alpha + u_s) by linearity of s_i (Sec. 2.2.2): s_i(alpha) plus s_i(v_b) over the bits b of s."""

    def __init__(self, l: int):
        v = cantor_basis()
        alpha = alpha_of(l)
        self.s_alpha = [s_eval(i, alpha) for i in range(max(l, 1))]
        self.s_v = [[s_eval(i, v[b]) for b in range(max(l, 1))] for i in range(max(l, 1))]

    def __call__(self, i: int, s: int) -> int:
        c = self.s_alpha[i]
        b = 0
        while s:
            if s & 1:
                c ^= self.s_v[i][b]
            s >>= 1
            b += 1
        return c


# ----------------------------------------------------------------- Encode
def encode_multipliers(l: int) -> list[int]:
    """r_j = prod_t c_t^{j_t}, c_t = s_{l+t}(alpha) the multiplier of layer l + t, t < 7."""
    alpha = alpha_of(l)
    c = [s_eval(l + t, alpha) for t in range(LM)]
    r = []
    for j in range(1 << LM):
        p = 1
        for t in range(LM):
            if (j >> t) & 1:
                p = gf_mul(p, c[t])
        r.append(p)
    return r


def encode(A: int, n: int) -> list[int]:
    """f_i = sum_{j < 128} a_{j n_p + i} r_j for i < n_p (A in novelpoly form)."""
    n_p = n // M
    l = S.log2_exact(n_p)
    r = encode_multipliers(l)
    f = []
    for i in range(n_p):
        acc = 0
        for j in range(M):
            if (A >> (j * n_p + i)) & 1:
                acc ^= r[j]
        f.append(acc)
    return f


def encode_by_truncated_butterfly(A: int, n: int) -> list[int]:
    """The first l_m = 7 layers of Alg. 2 on the n bits, keeping the first branch (Sec. 3.2)."""
    l = S.log2_exact(n) - LM
    alpha = alpha_of(l)
    g = [(A >> t) & 1 for t in range(n)]
    for i in range(l + LM - 1, l - 1, -1):
        half = len(g) // 2
        c = s_eval(i, alpha)
        g = [g[k] ^ gf_mul(g[half + k], c) for k in range(half)]
    return g


def decode(h: list[int], n: int) -> int:
    """The bits (a_{j n_p + i})_j = h_i R^{-1} (row vectors), R the matrix of the r_j."""
    n_p = n // M
    l = S.log2_exact(n_p)
    rinv = F.gf2_matrix_inverse(encode_multipliers(l), M)
    out = 0
    for i in range(n_p):
        vec = F.row_vec_times(h[i], rinv)
        for j in range(M):
            if (vec >> j) & 1:
                out |= 1 << (j * n_p + i)
    return out


# -------------------------------------------------------------- Butterfly
def butterfly(g: list[int], l: int) -> list[int]:
    """Alg. 2 unrolled into layers l-1 .. 0: p0 += c p1, p1 += p0 with c = s_i(alpha + u_s)."""
    x = list(g)
    n_p = len(x)
    tw = Twiddles(l)
    for i in range(l - 1, -1, -1):
        blk = 1 << (i + 1)
        for s in range(0, n_p, blk):
            c = tw(i, s)
            for j in range(blk // 2):
                x[s + j] ^= gf_mul(x[s + blk // 2 + j], c)
                x[s + blk // 2 + j] ^= x[s + j]
    return x


def ibutterfly(y: list[int], l: int) -> list[int]:
    """Inverse of ``butterfly``: layers 0 .. l-1, p1 += p0 then p0 += c p1."""
    x = list(y)
    n_p = len(x)
    tw = Twiddles(l)
    for i in range(l):
        blk = 1 << (i + 1)
        for s in range(0, n_p, blk):
            c = tw(i, s)
            for j in range(blk // 2):
                x[s + blk // 2 + j] ^= x[s + j]
                x[s + j] ^= gf_mul(x[s + blk // 2 + j], c)
    return x


def eval_at_sigma(A: int, n: int) -> list[int]:
    """E_Sigma(A) = [A(alpha + u_k)] by Horner (the definition, Eq. 8)."""
    l = S.log2_exact(n) - LM
    out = []
    for k in range(1 << l):
        beta = sigma_point(l, k)
        acc = 0
        for t in range(max(A.bit_length(), 1) - 1, -1, -1):
            acc = gf_mul(acc, beta)
            if (A >> t) & 1:
                acc ^= 1
        out.append(acc)
    return out


# ------------------------------------------------------------ FP_Polymul
def fp_polymul(a: int, na: int, b: int, nb: int) -> int:
    """Alg. 5 with m = 128: BasisCvt, Encode, Butterfly, pointwise, and back."""
    if na == 0 or nb == 0:
        return 0
    n = transform_length(na, nb)
    l = S.log2_exact(n) - LM
    fa = butterfly(encode(S.basis_cvt(a & ((1 << na) - 1), n), n), l)
    fb = butterfly(encode(S.basis_cvt(b & ((1 << nb) - 1), n), n), l)
    c = [gf_mul(x, y) for x, y in zip(fa, fb)]
    return S.ibasis_cvt(decode(ibutterfly(c, l), n), n)
