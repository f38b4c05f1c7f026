"""Pins of the C oracle: the carry-less product and the modular checker (CPU only).

The product is pinned to its definition (c_k = XOR_{i+j=k} a_i b_j, exhaustive
on tiny operands, random up to 512 bits), to the shift-and-add product at
Karatsuba sizes, and to closed forms.  The modular checker is pinned to the
exact product and shown to reject planted errors.
"""
import random

import numpy as np
import pytest

from oracle import clmul as O
from oracle import stages as S
import synth

rng = random.Random(64)
M64 = (1 << 64) - 1


def W(x, n):
    return O.int_to_words(x, n)


def I(w):
    return O.words_to_int(w)


def test_clmul64_definition():
    cases = [(0, 0), (M64, M64), (1, M64), (1 << 63, 1 << 63), (M64, 1 << 63)]
    cases += [(rng.getrandbits(64), rng.getrandbits(64)) for _ in range(300)]
    for a, b in cases:
        lo, hi = O.clmul64(a, b)
        assert lo | (hi << 64) == O.mul_bruteforce(a, 64, b, 64)


def test_exhaustive_tiny():
    for na in range(1, 6):
        for nb in range(1, 6):
            for a in range(1 << na):
                for b in range(1 << nb):
                    got = I(O.mul(W(a, na), na, W(b, nb), nb))
                    assert got == O.mul_bruteforce(a, na, b, nb), (na, nb, a, b)


def test_random_to_512_bits():
    for _ in range(120):
        na, nb = rng.randrange(1, 513), rng.randrange(1, 513)
        a, b = rng.getrandbits(na), rng.getrandbits(nb)
        assert I(O.mul(W(a, na), na, W(b, nb), nb)) == O.mul_bruteforce(a, na, b, nb)


@pytest.mark.parametrize("na,nb", [(1 << 12, 1 << 12), (1 << 16, 1 << 16), (70001, 1 << 14),
                                   (1 << 17, 333), (1 << 16, 1 << 16 | 1)])
def test_karatsuba_sizes_match_shift_and_add(na, nb):
    a, b = rng.getrandbits(na), rng.getrandbits(nb)
    assert I(O.mul(W(a, na), na, W(b, nb), nb)) == S.gf2x_mul_small(a, b)


def test_tail_bits_ignored_and_output_masked():
    na, nb = 100, 77
    a = synth.operand(5, na)                   # garbage above bit na
    b = synth.operand(6, nb)
    c = O.mul(a, na, b, nb)
    assert len(c) == (na + nb - 1 + 63) // 64
    ref = O.mul(synth.mask_tail(a, na), na, synth.mask_tail(b, nb), nb)
    assert np.array_equal(c, ref)
    assert I(c) >> (na + nb - 1) == 0


def test_empty_operands():
    assert len(O.mul(W(5, 3), 3, np.zeros(1, np.uint64), 0)) == 0
    assert len(O.mul(np.zeros(1, np.uint64), 0, np.zeros(1, np.uint64), 0)) == 0


# ---------------------------------------------------------------- closed forms
def test_square_spreads_bits():
    for n in [1, 64, 1000, 1 << 14]:
        a = rng.getrandbits(n)
        sq = I(O.mul(W(a, n), n, W(a, n), n))
        spread = 0
        for t in range(n):
            if (a >> t) & 1:
                spread |= 1 << (2 * t)
        assert sq == spread


def test_monomials_shift_identity_zero():
    for i, j in [(0, 0), (63, 1), (64, 64), (1000, 5), (4095, 4097)]:
        assert I(O.mul(W(1 << i, i + 1), i + 1, W(1 << j, j + 1), j + 1)) == 1 << (i + j)
    a = rng.getrandbits(3000)
    assert I(O.mul(W(a, 3000), 3000, W(1, 1), 1)) == a
    assert I(O.mul(W(a, 3000), 3000, W(1 << 777, 778), 778)) == a << 777
    assert I(O.mul(W(a, 3000), 3000, W(0, 64), 64)) == 0


def test_geometric_series_and_frobenius_power():
    for N in [1, 63, 64, 65, 5000]:
        s = (1 << N) - 1
        assert I(O.mul(W(s, N), N, W(3, 2), 2)) == 1 | (1 << N)   # (sum x^t)(1+x) = 1+x^N
    p, n = 3, 2                                                  # (1+x)^(2^k) = 1 + x^(2^k)
    for k in range(1, 13):
        p = I(O.mul(W(p, n), n, W(p, n), n))
        n = 2 * n - 1
        assert p == 1 | (1 << (1 << k))


def test_ring_laws_and_degree():
    for _ in range(10):
        na, nb, nc = (rng.randrange(1, 3000) for _ in range(3))
        a = rng.getrandbits(na) | (1 << (na - 1))
        b = rng.getrandbits(nb) | (1 << (nb - 1))
        c = rng.getrandbits(nc) | (1 << (nc - 1))
        ab = I(O.mul(W(a, na), na, W(b, nb), nb))
        assert ab == I(O.mul(W(b, nb), nb, W(a, na), na))
        assert ab.bit_length() - 1 == (na - 1) + (nb - 1)       # deg(ab) = deg a + deg b
        nbc = max(nb, nc)
        lhs = I(O.mul(W(a, na), na, W(b ^ c, nbc), nbc))
        ac = I(O.mul(W(a, na), na, W(c, nc), nc))
        assert lhs == ab ^ ac
        nab = na + nb - 1
        assert I(O.mul(W(ab, nab), nab, W(c, nc), nc)) == I(
            O.mul(W(a, na), na, W(I(O.mul(W(b, nb), nb, W(c, nc), nc)), nb + nc - 1), nb + nc - 1))


# --------------------------------------------------------------- modular check
def test_random_moduli_are_irreducible():
    lows = O.random_irreducibles(99, 8)
    assert len(set(lows.tolist())) == 8
    for low in lows.tolist():
        assert O.irreducible64(low)
    # x^64 + x^2 + 1 = (x^32 + x + 1)^2 is reducible
    assert not O.irreducible64((1 << 2) | 1)


def test_modcheck_accepts_true_products_and_rejects_errors():
    lows = O.random_irreducibles(7, 16)
    for na, nb in [(1, 1), (65, 3), (5000, 7000), (1 << 15, 1 << 15)]:
        a = synth.operand(11, na)
        b = synth.operand(12, nb)
        c = O.mul(a, na, b, nb)
        nc = na + nb - 1
        assert O.modcheck(a, na, b, nb, c, nc, lows).all()
        bad = c.copy()
        k = rng.randrange(nc)
        bad[k // 64] ^= np.uint64(1 << (k % 64))               # x^k mod p != 0
        assert not O.modcheck(a, na, b, nb, bad, nc, lows).any()


def test_golden_products_regression():
    from golden_util import rows
    for na, nb, a, b, c in rows("golden_products.txt"):
        na, nb, a, b, c = int(na), int(nb), int(a, 16), int(b, 16), int(c, 16)
        if na * nb <= 1 << 16:
            assert O.mul_bruteforce(a, na, b, nb) == c
        assert I(O.mul(W(a, na), na, W(b, nb), nb)) == c
