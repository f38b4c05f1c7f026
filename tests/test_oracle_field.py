"""Pins of the oracle's field, Cantor basis and subspace polynomials (CPU only).

Each check ties ``oracle.field`` to something other than itself: the
paper's printed formulas (Eq. 2, Eq. 4, Eq. 5, Sec. 4.3), definitions written
another way, or field theory (Fermat, Rabin's irreducibility test).
"""
import random

import numpy as np
import pytest

from oracle import field as F
from oracle import stages as S
from oracle import clmul as O
from golden_util import rows, constants

rng = random.Random(20180330)
MOD = (1 << 64) | F.POLY_LOW


def test_modulus_is_the_papers():
    assert F.POLY_LOW == constants()["modulus_low"]            # Sec. 4.3


def test_mul_equals_product_then_remainder():
    # a*b = (carry-less product) mod (x^64+x^4+x^3+x+1), computed by long division
    for _ in range(300):
        a, b = rng.getrandbits(64), rng.getrandbits(64)
        _, r = S.gf2x_divmod(S.gf2x_mul_small(a, b), MOD)
        assert F.gf_mul(a, b) == r


def test_mul_special_cases():
    x63 = 1 << 63
    assert F.gf_mul(x63, 2) == F.POLY_LOW                      # x^64 = x^4+x^3+x+1
    for _ in range(50):
        a = rng.getrandbits(64)
        assert F.gf_mul(a, 1) == a and F.gf_mul(a, 0) == 0


def test_field_laws():
    for _ in range(40):
        a, b, c = (rng.getrandbits(64) for _ in range(3))
        assert F.gf_mul(a, b) == F.gf_mul(b, a)
        assert F.gf_mul(a, b ^ c) == F.gf_mul(a, b) ^ F.gf_mul(a, c)
        assert F.gf_mul(F.gf_mul(a, b), c) == F.gf_mul(a, F.gf_mul(b, c))


def test_modulus_irreducible_rabin():
    # x^(2^64) = x and gcd(x^(2^32) - x, p) = 1, in Python big-int arithmetic
    z = 2
    z32 = None
    for k in range(1, 65):
        z = F.gf_sqr(z)
        if k == 32:
            z32 = z
    assert z == 2
    a, b = z32 ^ 2, MOD
    while b:
        while a and a.bit_length() >= b.bit_length():
            a ^= b << (a.bit_length() - b.bit_length())
        a, b = b, a
    assert a == 1
    assert O.irreducible64(F.POLY_LOW)


def test_fermat_and_inverse():
    for _ in range(5):
        a = rng.getrandbits(64) | 1
        assert F.gf_pow(a, 1 << 64) == a
        assert F.gf_mul(a, F.gf_inv(a)) == 1


def test_vectorised_mul_matches_scalar():
    a = np.array([rng.getrandbits(64) for _ in range(64)], dtype=np.uint64)
    b = np.array([rng.getrandbits(64) for _ in range(64)], dtype=np.uint64)
    got = F.gf_mul_arr(a, b)
    for i in range(64):
        assert int(got[i]) == F.gf_mul(int(a[i]), int(b[i]))


# ----------------------------------------------------------------- Cantor basis
def test_cantor_basis_equation():
    v = F.cantor_basis()
    assert v[0] == 1                                            # Eq. 2
    for i in range(1, 64):
        assert F.gf_sqr(v[i]) ^ v[i] == v[i - 1]
        assert v[i] & 1 == 0                                    # root choice
    assert F.gf2_rank(v) == 64                                  # a basis


def test_frobenius_orders_match_eq5():
    v = F.cantor_basis()
    for i, order in rows("frobenius_orders.txt"):
        assert F.frobenius_order(v[int(i)]) == int(order), i


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_power_of_two_spans_are_subfields(k):
    # V_{2^k} is a field (Sec. 2.2.1): closed under multiplication
    size = 1 << k
    for _ in range(30):
        a = F.cantor_to_poly(rng.getrandbits(size))
        b = F.cantor_to_poly(rng.getrandbits(size))
        assert F.poly_to_cantor(F.gf_mul(a, b)) >> size == 0


# ------------------------------------------------------- subspace polynomials
@pytest.mark.parametrize("i", [0, 1, 2, 3, 4])
def test_s_i_is_the_subspace_product(i):
    # Def. of s_i: prod_{a in V_i} (x - a), expanded with GF(2^64) coefficients
    poly = [1]                                                 # coefficients, low first
    for coords in range(1 << i):
        a = F.cantor_to_poly(coords)
        new = [0] * (len(poly) + 1)
        for t, c in enumerate(poly):
            new[t + 1] ^= c
            new[t] ^= F.gf_mul(c, a)
        poly = new
    expect = [(F.s_gf2x(i) >> t) & 1 for t in range(len(poly))]
    assert poly == expect


def test_s_i_two_terms_iff_power_of_two():
    for i in range(1, 64):
        two = len(F.s_coeffs(i)) == 2
        assert two == ((i & (i - 1)) == 0), i                  # Sec. 2.2.2


def test_s_i_on_basis_eq4():
    v = F.cantor_basis()
    for i in range(0, 40, 3):
        for j in range(i, 64, 5):
            assert F.s_eval(i, v[j]) == v[j - i]                # Eq. 4
        assert F.s_eval(i, v[i]) == 1
        for _ in range(3):                                      # s_i(V_i) = 0
            assert F.s_eval(i, F.cantor_to_poly(rng.getrandbits(i) if i else 0)) == 0


def test_s_i_is_a_right_shift_of_cantor_coordinates():
    for _ in range(20):
        i = rng.randrange(0, 40)
        coords = rng.getrandbits(64)
        assert F.s_eval(i, F.cantor_to_poly(coords)) == F.cantor_to_poly(coords >> i)


def test_s_i_linear_and_recursive():
    for _ in range(10):
        i = rng.randrange(1, 30)
        a, b = rng.getrandbits(64), rng.getrandbits(64)
        assert F.s_eval(i, a ^ b) == F.s_eval(i, a) ^ F.s_eval(i, b)
        # s_i = s_{i-1}^2 + s_{i-1} and s_{i+j} = s_i o s_j
        t = F.s_eval(i - 1, a)
        assert F.s_eval(i, a) == F.gf_sqr(t) ^ t
        j = rng.randrange(0, 20)
        assert F.s_eval(i + j, a) == F.s_eval(i, F.s_eval(j, a))
