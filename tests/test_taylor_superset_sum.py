"""The Taylor expansion of Alg. 1 as a superset sum over the digit index (CPU).

The GPU BasisCvt runs its Taylor parts (at x^tau + x over bits, and at
z^256 + z over 2^16-bit rows) as a superset sum plus one carry fix instead of
the division steps: with y = x^tau + x and f = sum_q x^(tau q) f_q,
x^(tau q) = (y + x)^q = sum_{r subset of q} y^r x^(q - r) in characteristic 2,
so the digits are
    g_r = (gt_r mod x^tau) + x o_r + o_{r-1},  gt_r = sum_{q superset of r} x^(q - r) f_q,
    o_r = gt_r >> tau,
and the inverse is the same sum followed by plain carries.  These tests check
that identity, written here on coefficient lists, against the oracle's Taylor
expansion by long division (oracle.stages._taylor and _taylor_inverse), for
one-bit coefficients and for multi-bit block coefficients (the row level,
where every coefficient is a word column).  The number of rows stays at most
tau, as in the kernels (at most 2^16 rows at tau = 2^16, at most 256 blocks of
256 rows at the row level).
"""
import random

import pytest

from oracle import stages as S

rng = random.Random(0x5A5A)


def superset_sum(rows, tau):
    """gt_r = sum over q superset of r of rows[q] moved up by q - r places."""
    n = len(rows)
    out = []
    for r in range(n):
        acc = [0] * (tau + n)
        for q in range(n):
            if q & r == r:
                for t, c in enumerate(rows[q]):
                    acc[t + q - r] ^= c
        out.append(acc)
    return out


def taylor_by_superset_sum(f, tau):
    m = len(f) // tau
    rows = [f[tau * q: tau * (q + 1)] for q in range(m)]
    gt = superset_sum(rows, tau)
    over = [row[tau:] for row in gt]                     # o_r, degree < m
    digits = []
    for r in range(m):
        g = list(gt[r][:tau])
        for t, c in enumerate(over[r]):                  # + x o_r
            if t + 1 < tau:
                g[t + 1] ^= c
            else:
                assert c == 0
        if r > 0:
            for t, c in enumerate(over[r - 1]):          # + o_{r-1}
                if t < tau:
                    g[t] ^= c
                else:
                    assert c == 0
        digits.append(g)
    return digits


def taylor_inverse_by_superset_sum(digits, tau):
    m = len(digits)
    ft = superset_sum(digits, tau)
    f = []
    for q in range(m):
        row = list(ft[q][:tau])
        if q > 0:
            for t, c in enumerate(ft[q - 1][tau:]):      # + (ft_{q-1} >> tau)
                if t < tau:
                    row[t] ^= c
                else:
                    assert c == 0
        f.extend(row)
    assert all(c == 0 for c in ft[m - 1][tau:])          # nothing past the last row
    return f


@pytest.mark.parametrize("tau,rows,bits", [(4, 2, 1), (4, 4, 1), (16, 4, 1), (16, 16, 1), (64, 32, 1),
                                           (4, 4, 8), (16, 8, 16), (32, 32, 64)])
def test_forward_matches_the_division_steps(tau, rows, bits):
    for _ in range(3):
        f = [rng.getrandbits(bits) for _ in range(tau * rows)]
        assert taylor_by_superset_sum(f, tau) == S._taylor(f, tau)


@pytest.mark.parametrize("tau,rows,bits", [(4, 4, 1), (16, 16, 1), (64, 32, 1), (16, 8, 16), (32, 32, 64)])
def test_inverse_matches_the_division_steps(tau, rows, bits):
    for _ in range(3):
        digits = [[rng.getrandbits(bits) for _ in range(tau)] for _ in range(rows)]
        assert taylor_inverse_by_superset_sum(digits, tau) == S._taylor_inverse(digits, tau)


def test_a_dropped_carry_is_caught():
    # the identity needs both carries: without x o_r the digits differ from the division's
    tau, m = 16, 16
    f = [rng.getrandbits(1) for _ in range(tau * m)]
    rows = [f[tau * q: tau * (q + 1)] for q in range(m)]
    gt = superset_sum(rows, tau)
    wrong = []
    for r in range(m):
        g = list(gt[r][:tau])
        if r > 0:
            for t, c in enumerate(gt[r - 1][tau:]):
                g[t] ^= c
        wrong.append(g)
    assert wrong != S._taylor(f, tau)
