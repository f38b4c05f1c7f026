"""Pins of the m = 128 oracle (Sec. 3 with m = 128, Sec. 4.3) -- CPU only.

The field is pinned by a Rabin irreducibility test and by the carry-less
product followed by long division (both written without ``m128.gf_mul``); the
Cantor basis by Eq. 2, its rank and the Frobenius orders of Eq. 5; Encode by
the first 7 truncated Butterfly layers; the forward path by evaluation at
Sigma (Eq. 8); the whole product by the plain carry-less product and by the
m = 64 method.
"""
import random

import pytest

from oracle import clmul as O
from oracle import field as F
from oracle import m128 as G
from oracle import stages as S

rng = random.Random(11301)
MOD = (1 << 128) | G.POLY_LOW


def _mod(f: int, p: int) -> int:
    return S.gf2x_divmod(f, p)[1]


# --------------------------------------------------------------------- field
def test_modulus_is_the_gcm_polynomial():
    assert MOD == (1 << 128) | (1 << 7) | (1 << 2) | (1 << 1) | 1


def test_mul_equals_product_then_remainder():
    for _ in range(60):
        a, b = rng.getrandbits(128), rng.getrandbits(128)
        assert G.gf_mul(a, b) == _mod(S.gf2x_mul_small(a, b), MOD)
    assert G.gf_mul(1 << 127, 2) == G.POLY_LOW
    assert G.gf_mul(0, rng.getrandbits(128)) == 0
    assert G.gf_mul(1, 0xDEADBEEF << 90) == 0xDEADBEEF << 90


def test_modulus_irreducible_rabin():
    # x^(2^128) = x mod p and gcd(x^(2^64) - x, p) = 1; squarings by plain
    # product + remainder, not by the field routine under test
    z = 2
    z64 = None
    for k in range(1, 129):
        z = _mod(S.gf2x_mul_small(z, z), MOD)
        if k == 64:
            z64 = z
    assert z == 2
    a, b = z64 ^ 2, MOD
    while b:
        a, b = b, _mod(a, b)
    assert a == 1


def test_field_laws():
    for _ in range(30):
        a, b, c = (rng.getrandbits(128) for _ in range(3))
        assert G.gf_mul(a, b) == G.gf_mul(b, a)
        assert G.gf_mul(a, b ^ c) == G.gf_mul(a, b) ^ G.gf_mul(a, c)
        assert G.gf_mul(G.gf_mul(a, b), c) == G.gf_mul(a, G.gf_mul(b, c))


# -------------------------------------------------------------- Cantor basis
def test_cantor_basis_equation_eq2():
    v = G.cantor_basis()
    assert len(v) == 128 and v[0] == 1
    for i in range(1, 128):
        assert G.gf_sqr(v[i]) ^ v[i] == v[i - 1]
        assert v[i] & 1 == 0
    assert F.gf2_rank(v) == 128


def test_frobenius_orders_eq5():
    # v_i lies in GF(2^(2^k)) exactly when i < 2^k
    v = G.cantor_basis()
    for i in [0, 1, 2, 3, 4, 7, 8, 15, 16, 31, 32, 63, 64, 100, 127]:
        assert G.frobenius_order(v[i]) == max(1, 1 << i.bit_length())


def test_s_i_on_basis_eq4():
    v = G.cantor_basis()
    for i in [0, 1, 3, 7, 8, 13, 64, 70]:
        for j in [0, 1, 5, i, i + 1, 64, 65, 100, 127]:
            if j > 127:
                continue
            assert G.s_eval(i, v[j]) == (v[j - i] if j >= i else 0)


def test_s_i_is_linear():
    for i in [1, 4, 9, 66]:
        a, b = rng.getrandbits(128), rng.getrandbits(128)
        assert G.s_eval(i, a ^ b) == G.s_eval(i, a) ^ G.s_eval(i, b)


# -------------------------------------------------------------------- Encode
@pytest.mark.parametrize("n", [128, 256, 1024, 4096])
def test_encode_is_the_truncated_butterfly(n):
    A = rng.getrandbits(n)
    assert G.encode(A, n) == G.encode_by_truncated_butterfly(A, n)


def test_encode_multipliers_and_prop2():
    v = G.cantor_basis()
    for l in [0, 3, 20, 63]:
        alpha = G.alpha_of(l)
        assert [G.s_eval(l + t, alpha) for t in range(7)] == [v[64 - t] for t in range(7)]
        assert F.gf2_rank(G.encode_multipliers(l)) == 128       # Prop. 2


def test_decode_inverts_encode():
    for n in [128, 512, 2048]:
        A = rng.getrandbits(n)
        assert G.decode(G.encode(A, n), n) == A


# ------------------------------------------------------------------ Butterfly
@pytest.mark.parametrize("n", [128, 256, 512, 1024])
def test_forward_path_is_evaluation_at_sigma_eq8(n):
    l = n.bit_length() - 1 - 7
    for na in [n // 2, n - 5]:
        A = rng.getrandbits(na)
        g = G.butterfly(G.encode(S.basis_cvt(A, n), n), l)
        assert g == G.eval_at_sigma(A, n)


def test_ibutterfly_inverts_butterfly():
    for l in [0, 1, 4]:
        g = [rng.getrandbits(128) for _ in range(1 << l)]
        assert G.ibutterfly(G.butterfly(g, l), l) == g


def test_sigma_points_distinct_frobenius_orbits_prop1():
    l = 2
    pts = [G.sigma_point(l, k) for k in range(1 << l)]
    omega = set()
    cur = list(pts)
    for _ in range(128):
        omega.update(cur)
        cur = [G.gf_sqr(p) for p in cur]
    assert cur == pts
    assert len(omega) == 128 * (1 << l)


# ----------------------------------------------------------------- FP_Polymul
PAIRS = [(1, 1), (1, 128), (64, 65), (65, 64), (64, 64), (65, 65), (100, 29), (129, 1),
         (200, 300), (513, 700), (1024, 1025), (3, 2000)]


@pytest.mark.parametrize("na,nb", PAIRS)
def test_fp_polymul_equals_carryless_product(na, nb):
    a = rng.getrandbits(na)
    b = rng.getrandbits(nb)
    want = O.words_to_int(O.mul(O.int_to_words(a, na), na, O.int_to_words(b, nb), nb))
    assert G.fp_polymul(a, na, b, nb) == want
    assert S.fp_polymul(a, na, b, nb) == want               # m = 64, same product


def test_fp_polymul_all_ones_and_sparse():
    for na, nb in [(128, 1), (127, 2), (300, 212)]:
        a = (1 << na) - 1
        b = (1 << nb) - 1
        assert G.fp_polymul(a, na, b, nb) == S.gf2x_mul_small(a, b)
        a = 1 << (na - 1)
        assert G.fp_polymul(a, na, b, nb) == b << (na - 1)
    assert G.fp_polymul(5, 0, 7, 3) == 0


def test_transform_length_rule():
    assert G.transform_length(1, 1) == 128
    assert G.transform_length(64, 65) == 128
    assert G.transform_length(65, 65) == 256
    assert G.transform_length(1 << 30, 1 << 30) == 1 << 31


def test_twiddles_by_linearity_equal_the_definition():
    for l in [1, 3, 6]:
        tw = G.Twiddles(l)
        for i in range(l):
            for s in range(0, 1 << l, 1 << (i + 1)):
                assert tw(i, s) == G.twiddle(l, i, s)
