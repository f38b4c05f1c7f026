"""The steps of FP_Polymul (Alg. 5), written plainly -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions
-----------
* A bit-polynomial is a Python int: bit t is the coefficient of x^t.
* A novelpoly polynomial over GF(2) is also an int: bit k is g_k, the
  coefficient of X_k (Def. of the novelpoly basis, Sec. 2.3).
* A vector of GF(2^64) elements is a numpy uint64 array (polynomial form,
  see ``oracle.field``).
* m = 64, so l_m = 6.  For a transform length n = 2^(l_n) bits,
  l = l_n - 6, n_p = 2^l and alpha = v_{l+32} (Eq. 6).

Readings of the paper used here (the paper is silent or garbled there):
* Alg. 1 writes the block multiplier as X_{(m-1) 2^k}; with i = 2^k and s_i = X_{2^i} the
  block multiplier is X_{j 2^i}.  That is what the recursion below produces.
* Eq. 9 / Sec. 3.3 list the Encode multipliers as v_{31}, ..., v_{26}
  (s_{l+1} .. s_{l+6} at v_{l+32}).  The first l_m truncated layers of
  Alg. 2 on a length-n input are layers l+5 .. l, whose multipliers are
  s_{l+5}(alpha) .. s_l(alpha).  ``encode_multipliers`` takes those, by
  running Alg. 2's layer rule; the tests show that this equals evaluation at
  the partition (Eq. 8) and that the printed list gives a singular map.
"""

from __future__ import annotations

import numpy as np

from . import field as F

LM = 6                                   # l_m = log2(m)


# ------------------------------------------------------------------ helpers
def log2_exact(n: int) -> int:
    k = n.bit_length() - 1
    if n <= 0 or (1 << k) != n:
        raise ValueError(f"{n} is not a power of two")
    return k


def next_pow2(x: int) -> int:
    return 1 if x <= 1 else 1 << (x - 1).bit_length()


def transform_length(na: int, nb: int) -> int:
    """n = max(64, next_pow2(na + nb - 1)) bits: the product-length bound of Alg. 5."""
    nc = na + nb - 1 if (na and nb) else 0
    return max(64, next_pow2(nc))


def gf2x_mul_small(a: int, b: int) -> int:
    """Carry-less product of two Python ints (schoolbook; for small pins only)."""
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    return r


def gf2x_divmod(f: int, d: int):
    """Quotient and remainder of f by d in GF(2)[x]."""
    dd = d.bit_length() - 1
    q = 0
    while f and f.bit_length() - 1 >= dd:
        sh = f.bit_length() - 1 - dd
        q ^= 1 << sh
        f ^= d << sh
    return q, f


def _pack(coeffs, w):
    r = 0
    for t, c in enumerate(coeffs):
        r |= c << (t * w)
    return r


def _unpack(x, w, count):
    mask = (1 << w) - 1
    return [(x >> (t * w)) & mask for t in range(count)]


def int_to_coeffs(f: int, L: int) -> list[int]:
    return [(f >> t) & 1 for t in range(L)]


def coeffs_to_int(c) -> int:
    r = 0
    for t, bit in enumerate(c):
        r |= (bit & 1) << t
    return r


# ------------------------------------------------- BasisCvt (Alg. 1, Sec. 2.3.1)
def _taylor(f: list[int], tau: int) -> list[list[int]]:
    """Digits h_j (each tau coefficients) with f = sum_j h_j * s^j, s = y^tau + y.

    Recursive division by s^(2^k) = y^(tau 2^k) + y^(2^k) (char. 2), the
    largest power of s of degree L/2 (Alg. 1).
    """
    L = len(f)
    if L <= tau:
        return [list(f) + [0] * (tau - L)]
    half = L // 2
    e = half // tau                          # 2^k
    r = list(f)
    q = [0] * (L - half)
    for t in range(L - 1, half - 1, -1):    # long division by y^half + y^e
        c = r[t]
        if c:
            q[t - half] ^= c
            r[t] ^= c
            r[t - half + e] ^= c
    return _taylor(r[:half], tau) + _taylor(q, tau)


def _taylor_inverse(digits: list[list[int]], tau: int) -> list[int]:
    """sum_j h_j * s^j with s = y^tau + y (inverse of ``_taylor``)."""
    if len(digits) == 1:
        return list(digits[0])
    h = len(digits) // 2
    lo = _taylor_inverse(digits[:h], tau)
    hi = _taylor_inverse(digits[h:], tau)
    half = len(lo)
    e = half // tau
    out = lo + [0] * half
    for t, c in enumerate(hi):              # + hi * (y^half + y^e)
        out[t + half] ^= c
        out[t + e] ^= c
    return out


def _cvt_params(L: int):
    K = log2_exact(L)
    i = 1
    while 2 * i <= K - 1:                    # i = max power of two with 2^i <= L - 1
        i *= 2
    return i, 1 << i


def _basis_cvt(coeffs: list[int], w: int) -> list[int]:
    """Alg. 1 on a list of coefficients, each a w-bit block (XOR = addition)."""
    L = len(coeffs)
    if L <= 2:                               # deg f <= 1: g = f_0 + X_1 f_1
        return list(coeffs)
    i, tau = _cvt_params(L)
    digits = _taylor(coeffs, tau)            # f = h(x, s_i(x))
    outer = _basis_cvt([_pack(d, w) for d in digits], tau * w)   # BasisCvt(h^(y))
    g = []
    for qk in outer:                         # BasisCvt(q_k(x)) for every coefficient
        g.extend(_basis_cvt(_unpack(qk, w, tau), w))
    return g


def _ibasis_cvt(g: list[int], w: int) -> list[int]:
    L = len(g)
    if L <= 2:
        return list(g)
    i, tau = _cvt_params(L)
    blocks = [_pack(_ibasis_cvt(g[k * tau:(k + 1) * tau], w), w) for k in range(L // tau)]
    digits_packed = _ibasis_cvt(blocks, tau * w)
    digits = [_unpack(d, w, tau) for d in digits_packed]
    return _taylor_inverse(digits, tau)


def basis_cvt(f: int, L: int) -> int:
    """Monomial -> novelpoly (Alg. 1) for f in GF(2)[x]_{<L}, L a power of two."""
    return coeffs_to_int(_basis_cvt(int_to_coeffs(f, L), 1))


def ibasis_cvt(g: int, L: int) -> int:
    """Novelpoly -> monomial, the inverse of ``basis_cvt``."""
    return coeffs_to_int(_ibasis_cvt(int_to_coeffs(g, L), 1))


def basis_cvt_division(f: int, L: int) -> int:
    """Bernstein-Chou form (Sec. 2.3.1): divide by s_{K-1}, recurse on both parts."""
    K = log2_exact(L)
    if K == 0:
        return f & 1
    q, r = gf2x_divmod(f, F.s_gf2x(K - 1))
    half = L // 2
    return basis_cvt_division(r, half) | (basis_cvt_division(q, half) << half)


def novelpoly_expand(g: int, L: int) -> int:
    """sum_k g_k X_k(x) with X_k = prod_{bits b of k} s_b(x) (Def. of novelpoly)."""
    K = log2_exact(L)
    s = [F.s_gf2x(b) for b in range(K)]
    X = [1] * L
    for k in range(1, L):
        low = (k & -k).bit_length() - 1
        X[k] = gf2x_mul_small(X[k & (k - 1)], s[low])
    r = 0
    for k in range(L):
        if (g >> k) & 1:
            r ^= X[k]
    return r


# --------------------------------------------------- partition (Eq. 6, Sec. 3.1)
def alpha_of(l: int) -> int:
    """alpha = v_{l + m/2}: Cantor coordinates 2^(l+32)."""
    return F.cantor_to_poly(1 << (l + 32))


def sigma_point(l: int, k: int) -> int:
    """alpha + u_k, the k-th point of Sigma (u_k has Cantor coordinates k)."""
    return F.cantor_to_poly((1 << (l + 32)) ^ k)


class Twiddles:
    """s_i(alpha + u_s) for the Butterfly, via linearity of s_i (Sec. 2.2.2)."""

    def __init__(self, l: int):
        v = F.cantor_basis()
        self.l = l
        self.alpha = alpha_of(l)
        self.s_alpha = [F.s_eval(i, self.alpha) for i in range(max(l, 1))]
        # s_i(v_b) for the bits b a block offset u_s can have (b < l).
        self.s_v = [[F.s_eval(i, v[b]) for b in range(max(l, 1))] for i in range(max(l, 1))]

    def of_blocks(self, i: int, starts: np.ndarray) -> np.ndarray:
        """s_i(alpha + u_s) for every block start s in ``starts``."""
        out = np.full(starts.shape, self.s_alpha[i], dtype=np.uint64)
        for b in range(self.l):
            bit = ((starts >> np.uint64(b)) & np.uint64(1)).astype(bool)
            out[bit] ^= np.uint64(self.s_v[i][b])
        return out


# --------------------------------------------------------- Encode (Alg. 4)
def encode_multipliers(l: int) -> list[int]:
    """r_j = prod_t c_t^{j_t}, c_t the multiplier of truncated Butterfly layer l + t.

    Layer i of Alg. 2 on the top block multiplies by s_i(alpha); the first l_m
    layers of a length-n = 2^(l+6) transform are i = l+5 .. l (Sec. 3.2-3.3).
    """
    alpha = alpha_of(l)
    c = [F.s_eval(l + t, alpha) for t in range(LM)]
    r = []
    for j in range(1 << LM):
        p = 1
        for t in range(LM):
            if (j >> t) & 1:
                p = F.gf_mul(p, c[t])
        r.append(p)
    return r


def _bit_rows(A: int, n: int) -> np.ndarray:
    """(64, n_p) array of the bits a_{j n_p + i}."""
    n_p = n // 64
    bits = np.array([(A >> t) & 1 for t in range(n)], dtype=np.uint8)
    return bits.reshape(64, n_p)


def encode(A: int, n: int) -> np.ndarray:
    """Alg. 4: f_i = sum_j a_{j n_p + i} r_j for i < n_p (A in novelpoly form)."""
    l = log2_exact(n) - LM
    r = np.array(encode_multipliers(l), dtype=np.uint64)
    rows = _bit_rows(A, n)
    f = np.zeros(n // 64, dtype=np.uint64)
    for j in range(64):
        f ^= r[j] * rows[j].astype(np.uint64)
    return f


def encode_by_truncated_butterfly(A: int, n: int) -> np.ndarray:
    """The first l_m layers of Alg. 2, keeping only the first branch (Sec. 3.2, Fig. 1)."""
    l = log2_exact(n) - LM
    alpha = alpha_of(l)
    g = np.array([(A >> t) & 1 for t in range(n)], dtype=np.uint64)
    for i in range(l + LM - 1, l - 1, -1):
        half = len(g) // 2
        p0, p1 = g[:half], g[half:]
        g = p0 ^ F.gf_mul_arr(p1, F.s_eval(i, alpha))   # h0; h1 is truncated
    return g


def decode(h: np.ndarray, n: int) -> int:
    """Inverse of Alg. 4: the bits (a_{j n_p + i})_j = h_i * R^{-1} (row vectors)."""
    l = log2_exact(n) - LM
    rinv = F.gf2_matrix_inverse(encode_multipliers(l))
    n_p = n // 64
    out = 0
    for i in range(n_p):
        vec = F.row_vec_times(int(h[i]), rinv)
        for j in range(64):
            if (vec >> j) & 1:
                out |= 1 << (j * n_p + i)
    return out


# ------------------------------------------------------- Butterfly (Alg. 2)
def butterfly_recursive(g: np.ndarray, alpha: int) -> np.ndarray:
    """Alg. 2 as written: split by X_{2^i}, two half-size calls at alpha and v_i + alpha."""
    L = len(g)
    if L == 1:
        return g.copy()
    i = log2_exact(L) - 1
    p0, p1 = g[: L // 2], g[L // 2:]
    h0 = p0 ^ F.gf_mul_arr(p1, F.s_eval(i, alpha))
    vi = F.cantor_basis()[i]
    h1 = h0 ^ F.gf_mul_arr(p1, F.s_eval(i, vi))
    return np.concatenate([butterfly_recursive(h0, alpha), butterfly_recursive(h1, vi ^ alpha)])


def butterfly(g: np.ndarray, tw: Twiddles) -> np.ndarray:
    """Alg. 2 with its recursion unrolled into l layers (Sec. 2.3.2).

    Layer i (from l-1 down to 0) works on blocks of 2^(i+1) starting at s; the
    sub-call that owns block s has offset alpha + u_s, so its multiplier is
    c = s_i(alpha + u_s); then p0 += c*p1 and p1 += p0 (s_i(v_i) = 1).
    """
    x = np.array(g, dtype=np.uint64, copy=True)
    n_p = len(x)
    l = log2_exact(n_p)
    for i in range(l - 1, -1, -1):
        blk = 1 << (i + 1)
        v = x.reshape(-1, blk)
        starts = np.arange(0, n_p, blk, dtype=np.uint64)
        c = tw.of_blocks(i, starts)[:, None]
        p0 = v[:, : blk // 2]
        p1 = v[:, blk // 2:]
        p0 ^= F.gf_mul_arr(p1, np.broadcast_to(c, p1.shape))
        p1 ^= p0
        x = v.reshape(-1)
    return x


def ibutterfly(y: np.ndarray, tw: Twiddles) -> np.ndarray:
    """Inverse of ``butterfly``: layers 0 .. l-1, p1 += p0 then p0 += c*p1."""
    x = np.array(y, dtype=np.uint64, copy=True)
    n_p = len(x)
    l = log2_exact(n_p)
    for i in range(l):
        blk = 1 << (i + 1)
        v = x.reshape(-1, blk)
        starts = np.arange(0, n_p, blk, dtype=np.uint64)
        c = tw.of_blocks(i, starts)[:, None]
        p0 = v[:, : blk // 2]
        p1 = v[:, blk // 2:]
        p1 ^= p0
        p0 ^= F.gf_mul_arr(p1, np.broadcast_to(c, p1.shape))
        x = v.reshape(-1)
    return x


# ------------------------------------------------ evaluation at Sigma (Eq. 8)
def eval_at_sigma(A: int, n: int) -> np.ndarray:
    """E_Sigma(A) = [A(alpha + u_k) for k < n_p], by Horner in GF(2^64) (definition)."""
    l = log2_exact(n) - LM
    n_p = 1 << l
    beta = np.array([sigma_point(l, k) for k in range(n_p)], dtype=np.uint64)
    acc = np.zeros(n_p, dtype=np.uint64)
    for t in range(max(A.bit_length(), 1) - 1, -1, -1):
        acc = F.gf_mul_arr(acc, beta)
        if (A >> t) & 1:
            acc ^= np.uint64(1)
    return acc


# ------------------------------------------------------ FP_Polymul (Alg. 5)
def forward(a: int, na: int, n: int, tw: Twiddles) -> np.ndarray:
    """The forward steps of Alg. 5 for one operand: BasisCvt, Encode, Butterfly at alpha."""
    A_novel = basis_cvt(a & ((1 << na) - 1), n)
    return butterfly(encode(A_novel, n), tw)


def fp_polymul(a: int, na: int, b: int, nb: int) -> int:
    """Alg. 5: C = A * B through the Frobenius-partition additive FFT."""
    if na == 0 or nb == 0:
        return 0
    n = transform_length(na, nb)
    l = log2_exact(n) - LM
    tw = Twiddles(l)
    ahat = forward(a, na, n, tw)
    bhat = forward(b, nb, n, tw)
    chat = F.gf_mul_arr(ahat, bhat)                  # pointwise
    h = ibutterfly(chat, tw)                          # iButterfly
    C_novel = decode(h, n)                            # Decode
    return ibasis_cvt(C_novel, n)                     # iBasisCvt


# ------------------------------------------------ novelpoly evaluation (Def.)
def novelpoly_eval(g_words: np.ndarray, L: int, beta: int) -> int:
    """sum_k g_k X_k(beta) for the novelpoly coefficient bits g (uint64 words).

    X_k = prod_{bits b of k} s_b (Def. of novelpoly).  Write k = 256 q + t
    (t < 256): X_k = X_{256 q} X_t, so the sum is
    sum_q X_{256 q}(beta) * (sum_t g_{256 q + t} X_t(beta)).  The inner sums
    are XORs of the 256 values X_t(beta); the outer sum splits on the top bit
    of q: G(v) = G(v_lo) + s_b(beta) * G(v_hi), folded from the top bit down.
    """
    K = log2_exact(L)
    lo = min(K, 8)
    sb = [F.s_eval(b, beta) for b in range(K)]
    X = [1] * (1 << lo)
    for t in range(1, 1 << lo):
        low = (t & -t).bit_length() - 1
        X[t] = F.gf_mul(X[t & (t - 1)], sb[low])
    w = np.asarray(g_words, dtype=np.uint64)[: max(L // 64, 1)]
    raw = w.view(np.uint8)
    if L < 64:
        raw = np.unpackbits(raw, bitorder="little")[:L]
        raw = np.packbits(np.pad(raw, (0, 8 - L % 8 if L % 8 else 0)), bitorder="little")
    nbytes = max((1 << lo) // 8, 1)
    blocks = raw[: (L + 7) // 8].reshape(-1, nbytes)
    vals = np.zeros(blocks.shape[0], dtype=np.uint64)
    for p in range(nbytes):
        tab = np.zeros(256, dtype=np.uint64)
        for v in range(256):
            acc = 0
            for b in range(8):
                if (v >> b) & 1 and 8 * p + b < len(X):
                    acc ^= X[8 * p + b]
            tab[v] = acc
        vals ^= tab[blocks[:, p]]
    for b in range(K - 1, lo - 1, -1):
        half = len(vals) // 2
        vals = vals[:half] ^ F.gf_mul_arr(vals[half:], sb[b])
    return int(vals[0])
