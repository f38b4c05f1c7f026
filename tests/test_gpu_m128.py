"""Parity of the m = 128 CUDA path (GF(2^128) points) with the oracle -- needs a GPU.

Bit-exact throughout.  Stage by stage against ``oracle.m128`` (Encode and
Decode over 128 rows, Butterfly on Sigma = v_{l+64} + V_l, the GF(2^128)
product); the forward path sampled against evaluation at Sigma (Eq. 8);
whole products against the Karatsuba oracle and, at 2^30-bit operands,
against the modular checker.
"""
import random

import numpy as np
import pytest

import synth
from oracle import clmul as O
from oracle import m128 as G
from oracle import stages as S

pytestmark = pytest.mark.gpu

rng = random.Random(0x128B300)


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1803_11301_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def dev(words):
    import torch
    return torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint64)


def to_words(points):
    """GF(2^128) elements (ints) -> two words each, low word first."""
    out = np.zeros(2 * len(points), dtype=np.uint64)
    for k, p in enumerate(points):
        out[2 * k] = p & ((1 << 64) - 1)
        out[2 * k + 1] = p >> 64
    return out


def to_points(words):
    return [int(words[2 * k]) | (int(words[2 * k + 1]) << 64) for k in range(len(words) // 2)]


def rand_points(count):
    return [rng.getrandbits(128) for _ in range(count)]


# ------------------------------------------------------------------ stages
def test_pointwise_gf128_product(ctx):
    for count in [1, 7, 500]:
        a, b = rand_points(count), rand_points(count)
        a[0], b[0] = 1 << 127, 1 << 127          # the fold of the fold
        if count > 2:
            a[1], b[1] = 0, rng.getrandbits(128)
            a[2], b[2] = 1, (1 << 128) - 1
        got = to_points(host(ctx.m128_pointwise(dev(to_words(a)), dev(to_words(b)))))
        assert got == [G.gf_mul(x, y) for x, y in zip(a, b)]


@pytest.mark.parametrize("n", [128, 256, 1024, 4096, 1 << 13, 1 << 14, 1 << 16])
def test_encode_decode_match_alg4(ctx, n):
    A = O.words_to_int(synth.splitmix64(rng.getrandbits(63), n // 64))
    f = ctx.m128_encode(dev(O.int_to_words(A, n)), n)
    assert to_points(host(f)) == G.encode(A, n)
    back = ctx.m128_decode(f, n)
    assert O.words_to_int(host(back)) == A


@pytest.mark.parametrize("l", [0, 1, 2, 4, 5, 9, 10, 11, 12, 13, 14, 15])
def test_butterfly_matches_alg2(ctx, l):
    n = 128 << l
    g = rand_points(1 << l)
    t = dev(to_words(g))
    ctx.m128_butterfly(t, n)
    assert to_points(host(t)) == G.butterfly(g, l)
    ctx.m128_ibutterfly(t, n)
    assert to_points(host(t)) == g


def horner(bits: int, nbits: int, beta: int) -> int:
    acc = 0
    for t in range(nbits - 1, -1, -1):
        acc = G.gf_mul(acc, beta)
        if (bits >> t) & 1:
            acc ^= 1
    return acc


@pytest.mark.parametrize("nbits", [100, 3000, 1 << 14, 1 << 16])
def test_forward_path_is_evaluation_at_sigma(ctx, nbits):
    # BasisCvt -> Encode -> Butterfly gives A(alpha + u_k), alpha = v_{l+64} (Eq. 8)
    n = max(128, 2 * S.next_pow2(nbits))
    l = n.bit_length() - 1 - 7
    w = synth.mask_tail(synth.splitmix64(rng.getrandbits(63), (nbits + 63) // 64), nbits)
    buf = np.zeros(n // 64, dtype=np.uint64)
    buf[: len(w)] = w
    t = dev(buf)
    ctx.basis_cvt(t, max(64, S.next_pow2(nbits)))
    f = ctx.m128_encode(t, n)
    ctx.m128_butterfly(f, n)
    y = to_points(host(f))
    A = O.words_to_int(w)
    ks = sorted({0, (1 << l) - 1} | {rng.randrange(1 << l) for _ in range(2)})
    for k in ks:
        assert y[k] == horner(A, nbits, G.sigma_point(l, k)), k


# -------------------------------------------------------------- end to end
def check_product(ctx, na, nb, seed):
    a = synth.operand(seed, na)
    b = synth.operand(seed + 1, nb)
    got = host(ctx.mul_m128(dev(a), na, dev(b), nb))
    want = O.mul(a, na, b, nb)
    assert np.array_equal(got, want), (na, nb, seed)


EDGE = [(1, 1), (1, 2), (3, 5), (63, 66), (64, 65), (65, 64), (64, 64), (65, 65), (127, 2), (128, 1),
        (129, 128), (1000, 1000), (1, 5000), (4095, 4097), (8192, 8192), (12345, 678), (1 << 15, 1 << 15),
        (1 << 16, 1), (70001, 3333), (1 << 17, 1 << 17), (99999, 200001), (1 << 20, 1 << 19)]


@pytest.mark.parametrize("na,nb", EDGE)
def test_product_edge_sizes(ctx, na, nb):
    check_product(ctx, na, nb, synth.config_seed(11, na ^ nb))


def test_product_2e16_many_seeds(ctx):
    n = 1 << 16
    for i in range(50):
        check_product(ctx, n, n, synth.config_seed(12, 2 * i))


def test_product_2e24_bit_exact(ctx):
    n = 1 << 24
    check_product(ctx, n, n, synth.config_seed(13, 0))


def test_product_2e30_modular(ctx):
    # 2^30 x 2^30: c mod p = (a mod p)(b mod p) mod p for 64 seeded irreducible p
    na = nb = 1 << 30
    a = synth.operand(synth.config_seed(14, 0), na)
    b = synth.operand(synth.config_seed(14, 1), nb)
    c = host(ctx.mul_m128(dev(a), na, dev(b), nb))
    lows = O.random_irreducibles(synth.config_seed(14, 99), 64)
    assert O.modcheck(a, na, b, nb, c, na + nb - 1, lows).all()
    assert O.words_to_int(c[-1:]) >> ((na + nb - 1) % 64) == 0


def test_product_2e32_generic_basis_cvt_modular(ctx):
    # n = 2^33 (K = 33, BasisCvt by the generic step kernels), 16 modular checks
    na = nb = 1 << 32
    a = synth.operand(synth.config_seed(14, 200), na)
    b = synth.operand(synth.config_seed(14, 201), nb)
    c = host(ctx.mul_m128(dev(a), na, dev(b), nb))
    lows = O.random_irreducibles(synth.config_seed(14, 97), 16)
    assert O.modcheck(a, na, b, nb, c, na + nb - 1, lows).all()
    assert O.words_to_int(c[-1:]) >> ((na + nb - 1) % 64) == 0


def test_same_product_as_m64_path(ctx):
    for na, nb in [(1 << 18, 1 << 18), (300001, 77777)]:
        a = dev(synth.operand(synth.config_seed(15, na), na))
        b = dev(synth.operand(synth.config_seed(15, nb + 1), nb))
        assert np.array_equal(host(ctx.mul_m128(a, na, b, nb)), host(ctx.mul(a, na, b, nb)))


def test_repeated_calls_replay_with_new_contents(ctx):
    import torch
    from paper_1803_11301_gb300 import m128_workspace_bytes
    na, nb = 50000, 123457
    da = dev(np.zeros((na + 63) // 64, np.uint64))
    db = dev(np.zeros((nb + 63) // 64, np.uint64))
    out = torch.empty((na + nb - 1 + 63) // 64, dtype=torch.int64, device="cuda")
    ws = torch.empty(m128_workspace_bytes(na, nb), dtype=torch.uint8, device="cuda")
    for k in range(4):
        a = synth.operand(synth.config_seed(16, 2 * k), na)
        b = synth.operand(synth.config_seed(16, 2 * k + 1), nb)
        da.copy_(dev(a))
        db.copy_(dev(b))
        ctx.mul_m128(da, na, db, nb, out=out, workspace=ws)
        assert np.array_equal(host(out), O.mul(a, na, b, nb)), k


def test_argument_errors(ctx):
    import torch
    from paper_1803_11301_gb300 import Gf2xError, m128_transform_bits, m128_workspace_bytes
    assert m128_transform_bits(1, 1) == 128
    assert m128_transform_bits(65, 65) == 256
    assert m128_transform_bits(0, 5) == 0
    assert m128_workspace_bytes(1, 1) == 3 * 256 + 256
    t = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(Gf2xError):
        ctx.m128_butterfly(t, 64)                     # n below 128
    with pytest.raises(Gf2xError):
        ctx.m128_butterfly(t, 192)                    # not a power of two
    with pytest.raises(Gf2xError):
        ctx.m128_butterfly(t[1:], 128)                # element buffer not 16-byte aligned
    with pytest.raises(Gf2xError):
        ctx.m128_encode(t[:32], 2048, out=t[16:48])   # overlap
    a = dev(synth.operand(1, 1000))
    with pytest.raises(Gf2xError):
        ctx.mul_m128(a, 1000, a, 1000, workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))
