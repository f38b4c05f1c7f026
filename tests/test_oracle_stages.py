"""Pins of the oracle's stage reference (Alg. 1, 2, 4, 5) -- CPU only.

Every stage is checked against a definition written independently of it:
BasisCvt against the expansion sum_k g_k X_k(x) (Def. of novelpoly) and the
Bernstein-Chou division form; Encode against running the first l_m layers of
Alg. 2 literally; the forward path against evaluation at Sigma by Horner
(Eq. 8); the full Alg. 5 against the plain carry-less product.
"""
import random

import numpy as np
import pytest

from oracle import field as F
from oracle import stages as S
from oracle import clmul as O

rng = random.Random(1803)


# ------------------------------------------------------------------ BasisCvt
@pytest.mark.parametrize("L", [2, 4, 8, 16, 32, 64, 128, 256])
def test_basis_cvt_matches_novelpoly_definition(L):
    for _ in range(6):
        f = rng.getrandbits(L)
        g = S.basis_cvt(f, L)
        assert S.novelpoly_expand(g, L) == f


@pytest.mark.parametrize("L", [512, 1024, 4096])
def test_basis_cvt_matches_division_form(L):
    for _ in range(3):
        f = rng.getrandbits(L)
        assert S.basis_cvt(f, L) == S.basis_cvt_division(f, L)


def test_basis_cvt_inverse_triangular_and_length_free():
    for L in [64, 256, 2048]:
        for _ in range(4):
            d = rng.randrange(1, L)
            f = rng.getrandbits(d) | (1 << (d - 1))
            g = S.basis_cvt(f, L)
            assert S.ibasis_cvt(g, L) == f
            assert g.bit_length() == f.bit_length()            # deg X_k = k
            assert S.basis_cvt(f, 2 * L) == g                  # zero padding commutes


def test_basis_cvt_of_s_i_is_a_unit_vector():
    for i in range(0, 10):
        L = 1 << (i + 1)
        assert S.basis_cvt(F.s_gf2x(i), L) == 1 << (1 << i)    # X_{2^i} = s_i


# -------------------------------------------------------------------- Encode
@pytest.mark.parametrize("n", [64, 128, 1024, 4096])
def test_encode_is_the_truncated_butterfly(n):
    A = rng.getrandbits(n)
    assert np.array_equal(S.encode(A, n), S.encode_by_truncated_butterfly(A, n))


def test_encode_matrix_invertible_prop2():
    for l in [0, 1, 5, 11, 25, 31]:
        assert F.gf2_rank(S.encode_multipliers(l)) == 64        # Prop. 2


def test_printed_multiplier_list_is_singular():
    # Eq. 9 as printed: r_j = prod_k v_{m/2-1-k}^{j_k}.  The resulting map is not
    # a bijection, so it cannot be the Encode of Prop. 2 (reading A1).
    v = F.cantor_basis()
    r = []
    for j in range(64):
        p = 1
        for k in range(6):
            if (j >> k) & 1:
                p = F.gf_mul(p, v[31 - k])
        r.append(p)
    assert F.gf2_rank(r) < 64
    # the multipliers used instead are v_{32}, ..., v_{27} (layers l .. l+5)
    for l in [0, 3, 17]:
        alpha = S.alpha_of(l)
        assert [F.s_eval(l + t, alpha) for t in range(6)] == [v[32 - t] for t in range(6)]


def test_decode_inverts_encode():
    for n in [64, 256, 4096]:
        A = rng.getrandbits(n)
        assert S.decode(S.encode(A, n), n) == A


# ------------------------------------------------------------------ Butterfly
@pytest.mark.parametrize("l", [0, 1, 2, 3, 6, 8])
def test_layered_butterfly_equals_recursive_alg2(l):
    n_p = 1 << l
    tw = S.Twiddles(l)
    g = np.array([rng.getrandbits(64) for _ in range(n_p)], dtype=np.uint64)
    assert np.array_equal(S.butterfly(g, tw), S.butterfly_recursive(g, tw.alpha))
    assert np.array_equal(S.ibutterfly(S.butterfly(g, tw), tw), g)


@pytest.mark.parametrize("n", [64, 128, 256, 1024, 2048])
def test_forward_path_is_evaluation_at_sigma_eq8(n):
    l = n.bit_length() - 1 - 6
    tw = S.Twiddles(l)
    for na in [n // 2, n - 3]:
        A = rng.getrandbits(na)
        assert np.array_equal(S.forward(A, na, n, tw), S.eval_at_sigma(A, n))


def test_sigma_points_distinct_frobenius_orbits_prop1():
    # Prop. 1 on a small case: Sigma, phi(Sigma), ..., phi^63(Sigma) are disjoint,
    # so Omega has n = 64 * n_p points.
    l = 3
    pts = [S.sigma_point(l, k) for k in range(1 << l)]
    omega = set()
    cur = list(pts)
    for _ in range(64):
        omega.update(cur)
        cur = [F.gf_sqr(p) for p in cur]
    assert cur == pts or set(cur) == set(pts)
    assert len(omega) == 64 * (1 << l)


def test_frobenius_identity_eq1():
    # C(phi(a)) = phi(C(a)) for C in GF(2)[x]
    for nbits in [1, 7, 64, 500]:
        c = rng.getrandbits(nbits)
        w = O.int_to_words(c, nbits)
        beta = rng.getrandbits(64)
        assert O.eval_at(w, nbits, F.gf_sqr(beta)) == F.gf_sqr(O.eval_at(w, nbits, beta))


def test_c_eval_matches_horner():
    for nbits in [1, 63, 64, 65, 300]:
        c = rng.getrandbits(nbits)
        beta = rng.getrandbits(64)
        acc = 0
        for t in range(nbits - 1, -1, -1):
            acc = F.gf_mul(acc, beta) ^ ((c >> t) & 1)
        assert O.eval_at(O.int_to_words(c, nbits), nbits, beta) == acc


# ----------------------------------------------------------------- FP_Polymul
PAIRS = [(1, 1), (1, 64), (2, 3), (5, 60), (32, 33), (33, 32), (64, 64), (65, 1),
         (100, 300), (513, 700), (1024, 1024), (3, 2000), (2049, 2048), (4096, 17)]


@pytest.mark.parametrize("na,nb", PAIRS)
def test_fp_polymul_equals_carryless_product(na, nb):
    a = rng.getrandbits(na)
    b = rng.getrandbits(nb)
    assert S.fp_polymul(a, na, b, nb) == O.words_to_int(
        O.mul(O.int_to_words(a, na), na, O.int_to_words(b, nb), nb))


def test_fp_polymul_all_ones_and_sparse():
    for na, nb in [(64, 64), (127, 129), (1000, 24)]:
        a = (1 << na) - 1
        b = (1 << nb) - 1
        assert S.fp_polymul(a, na, b, nb) == S.gf2x_mul_small(a, b)
        a = 1 << (na - 1)
        assert S.fp_polymul(a, na, b, nb) == b << (na - 1)


def test_transform_length_rule():
    assert S.transform_length(1, 1) == 64
    assert S.transform_length(33, 32) == 64
    assert S.transform_length(33, 33) == 128
    assert S.transform_length(1 << 30, 1 << 30) == 1 << 31


@pytest.mark.parametrize("L", [64, 256, 512, 4096, 1 << 14])
def test_novelpoly_eval_is_the_definition(L):
    # sum_k g_k X_k(beta) = f(beta) when g = BasisCvt(f); and equals the slow expansion
    for _ in range(3):
        f = rng.getrandbits(L)
        g = S.basis_cvt(f, L)
        beta = rng.getrandbits(64)
        assert S.novelpoly_eval(O.int_to_words(g, L), L, beta) == O.eval_at(O.int_to_words(f, L), L, beta)
    if L <= 256:
        g = rng.getrandbits(L)
        beta = rng.getrandbits(64)
        f = S.novelpoly_expand(g, L)
        assert S.novelpoly_eval(O.int_to_words(g, L), L, beta) == O.eval_at(O.int_to_words(f, L), L, beta)
