"""GF(2^64), the Cantor basis and subspace polynomials -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain, slow and
written to be checked against the paper by eye.

Field (Sec. 4.3): GF(2^64) = GF(2)[x] / (x^64 + x^4 + x^3 + x + 1).  An element
is a Python int < 2^64 whose bit t is the coefficient of x^t ("polynomial
form").  The paper designs its algorithms with vectors in the Cantor basis and
converts only the constants to polynomial form (Sec. 4.3); we do the same.

Cantor basis (Eq. 2, Sec. 2.2.1): v_0 = 1 and v_i^2 + v_i = v_{i-1}.  Each
equation has two roots y and y+1; the paper does not say which one to take.
Reading used here: the root whose polynomial form has bit 0 clear.  The final
product does not depend on this choice; intermediate values do.

Subspace polynomials (Def. of s_i, Sec. 2.2.2): s_0(x) = x and
s_{i+1} = s_i^2 + s_i, so s_i(x) = sum_j C(i, j) x^(2^j) with C(i, j) taken
mod 2.  ``s_eval`` evaluates that sum directly; Eq. 4 (s_i(v_j) = v_{j-i},
i.e. "shift the Cantor coordinates right by i") is a property the tests check
against it, not something this module assumes.
"""

from __future__ import annotations

import numpy as np

M = 64                       # field degree m (Sec. 4)
POLY_LOW = 0x1B              # x^4 + x^3 + x + 1, the low part of the modulus
MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------- arithmetic
def gf_mul(a: int, b: int) -> int:
    """Product in GF(2^64): schoolbook shift-and-add, reducing x^64 each step."""
    r = 0
    for t in range(M):
        if (b >> t) & 1:
            r ^= a
        carry = a >> 63
        a = (a << 1) & MASK64
        if carry:
            a ^= POLY_LOW
    return r


def gf_sqr(a: int) -> int:
    return gf_mul(a, a)


def gf_pow(a: int, e: int) -> int:
    r = 1
    while e:
        if e & 1:
            r = gf_mul(r, a)
        a = gf_mul(a, a)
        e >>= 1
    return r


def gf_inv(a: int) -> int:
    """a^(2^64 - 2), the inverse of a non-zero a."""
    if a == 0:
        raise ZeroDivisionError("0 has no inverse in GF(2^64)")
    return gf_pow(a, (1 << 64) - 2)


def gf_mul_arr(a: np.ndarray, b) -> np.ndarray:
    """Elementwise product of uint64 arrays (b may be a scalar or an array).

    The same shift-and-add as ``gf_mul``, vectorised across elements.
    """
    a = np.array(a, dtype=np.uint64, copy=True)
    b = np.broadcast_to(np.asarray(b, dtype=np.uint64), a.shape)
    r = np.zeros(a.shape, dtype=np.uint64)
    one = np.uint64(1)
    low = np.uint64(POLY_LOW)
    for t in range(M):
        bit = (b >> np.uint64(t)) & one
        r ^= a * bit                       # a if bit set, else 0
        carry = a >> np.uint64(63)
        a = (a << one) ^ (carry * low)
    return r


# ------------------------------------------------------------ linear algebra
def gf2_solve(rows: list[int], rhs: int, n: int = M):
    """Solve sum_k y_k * rows[k] = rhs over GF(2) (columns are bit positions).

    ``rows[k]`` is the image of the k-th unit vector.  Returns one solution y
    (an int) with every free variable set to 0, or None if there is none.
    """
    # Build the augmented system column by column: equation for bit position p
    # is  sum_k y_k * bit_p(rows[k]) = bit_p(rhs).
    eqs = []
    for p in range(n):
        coeffs = 0
        for k in range(n):
            if (rows[k] >> p) & 1:
                coeffs |= 1 << k
        eqs.append([coeffs, (rhs >> p) & 1])
    pivots = []
    r = 0
    for col in range(n):
        piv = None
        for i in range(r, n):
            if (eqs[i][0] >> col) & 1:
                piv = i
                break
        if piv is None:
            continue
        eqs[r], eqs[piv] = eqs[piv], eqs[r]
        for i in range(n):
            if i != r and (eqs[i][0] >> col) & 1:
                eqs[i][0] ^= eqs[r][0]
                eqs[i][1] ^= eqs[r][1]
        pivots.append(col)
        r += 1
    for i in range(r, n):
        if eqs[i][1]:
            return None
    y = 0
    for i, col in enumerate(pivots):
        if eqs[i][1]:
            y |= 1 << col
    return y


def gf2_rank(vectors: list[int]) -> int:
    basis = []
    for v in vectors:
        for b in basis:
            v = min(v, v ^ b)
        if v:
            basis.append(v)
    return len(basis)


def gf2_matrix_inverse(rows: list[int], n: int = M) -> list[int]:
    """Inverse of the n x n GF(2) matrix whose row k is ``rows[k]`` (row-vector convention).

    For a row vector u (an int, bit k = u_k), u * A = XOR of rows[k] over set
    bits k.  Returns rows of A^{-1}.  Raises ValueError if A is singular.
    """
    a = list(rows)
    inv = [1 << k for k in range(n)]
    for col in range(n):
        piv = None
        for i in range(col, n):
            if (a[i] >> col) & 1:
                piv = i
                break
        if piv is None:
            raise ValueError("singular GF(2) matrix")
        a[col], a[piv] = a[piv], a[col]
        inv[col], inv[piv] = inv[piv], inv[col]
        for i in range(n):
            if i != col and (a[i] >> col) & 1:
                a[i] ^= a[col]
                inv[i] ^= inv[col]
    return inv


def row_vec_times(u: int, rows: list[int]) -> int:
    """u * A for the row vector u and the matrix with rows ``rows``."""
    r = 0
    k = 0
    while u:
        if u & 1:
            r ^= rows[k]
        u >>= 1
        k += 1
    return r


# -------------------------------------------------------------- Cantor basis
_CANTOR: list[int] | None = None


def cantor_basis() -> list[int]:
    """v_0..v_63 in polynomial form (Eq. 2), choosing roots with bit 0 clear."""
    global _CANTOR
    if _CANTOR is None:
        # y -> y^2 + y is GF(2)-linear; its matrix rows are images of x^k.
        trace_rows = [gf_sqr(1 << k) ^ (1 << k) for k in range(M)]
        v = [1]
        for i in range(1, M):
            y = gf2_solve(trace_rows, v[i - 1])
            if y is None:
                raise ArithmeticError(f"y^2 + y = v_{i-1} has no root")
            if y & 1:                     # the other root is y + 1
                y ^= 1
            v.append(y)
        _CANTOR = v
    return list(_CANTOR)


def cantor_to_poly(coords: int) -> int:
    """The field element sum_j b_j v_j for Cantor coordinates coords = sum_j b_j 2^j."""
    v = cantor_basis()
    r = 0
    j = 0
    while coords:
        if coords & 1:
            r ^= v[j]
        coords >>= 1
        j += 1
    return r


def poly_to_cantor(a: int) -> int:
    """Cantor coordinates of the field element a (inverse of ``cantor_to_poly``)."""
    y = gf2_solve(cantor_basis(), a)
    assert y is not None
    return y


# ------------------------------------------------------ subspace polynomials
def s_coeffs(i: int) -> list[int]:
    """Exponents j such that x^(2^j) has coefficient 1 in s_i (Sec. 2.2.2)."""
    c = [1]                                   # s_0 = x
    for _ in range(i):
        # s_{k+1} = s_k^2 + s_k: squaring maps x^(2^j) -> x^(2^(j+1)).
        sq = [0] + c
        c = [x ^ y for x, y in zip(sq, c + [0])]
    return [j for j, bit in enumerate(c) if bit]


def s_eval(i: int, a: int) -> int:
    """s_i(a) = sum over the terms x^(2^j) of s_i, evaluated at the field element a."""
    terms = set(s_coeffs(i))
    r = 0
    p = a                                     # p = a^(2^j)
    for j in range(i + 1):
        if j in terms:
            r ^= p
        p = gf_sqr(p)
    return r


def s_gf2x(i: int) -> int:
    """s_i as a polynomial in GF(2)[x] (bit k = coefficient of x^k)."""
    r = 0
    for j in s_coeffs(i):
        r |= 1 << (1 << j)
    return r


def frobenius_order(a: int) -> int:
    """Smallest j >= 1 with a^(2^j) = a (Def. of Ord_phi for a one-element set)."""
    b = gf_sqr(a)
    j = 1
    while b != a:
        b = gf_sqr(b)
        j += 1
    return j
