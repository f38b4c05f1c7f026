"""The two-pass Taylor part of BasisCvt / iBasisCvt (Alg. 1 at y = x^tau + x,
tau = 2^16, as a superset sum over the row index plus one carry fix) against
the oracle -- needs a GPU.

It runs inside products whose BasisCvt lengths are 2^25 .. 2^32 bits: both
operands in one call (side buffer Y), one operand at a time (Y for a, the
unused top of T for b), the inverse (Y), batches of such products, and a
reused operand's transform.  Every product is compared bit for bit with the
Karatsuba oracle where it finishes in seconds, with the modular checker above,
and with the division-step path of the same call (GF2X_KNOB_CVT_TAYLOR = 0).
"""
import random

import numpy as np
import pytest

import synth
from oracle import clmul as O

pytestmark = pytest.mark.gpu

rng = random.Random(0x7A11)


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


def both_forms(ctx, fn):
    """fn() under the two-pass Taylor part (the default) and under the division steps."""
    from paper_1803_11301_gb300 import KNOB_CVT_TAYLOR
    try:
        ctx.tune_pin(KNOB_CVT_TAYLOR, 1)
        two_pass = fn()
        ctx.tune_pin(KNOB_CVT_TAYLOR, 0)
        steps = fn()
    finally:
        ctx.tune_pin(KNOB_CVT_TAYLOR, -1)
    return two_pass, steps


# (na, nb): BasisCvt lengths and the path each takes (m = K - 16 rows of 2^16 bits)
CASES = [
    (1 << 24, 1 << 24),                 # forward K = 24 (window kernel), inverse K = 25 (m = 9)
    (1 << 25, 1 << 25),                 # both operands in one call: K = 25; inverse K = 26
    ((1 << 26) - 3, (1 << 25) + 5),     # both at K = 26 (J = 16 rows per pass-1 column); inverse K = 27
    (1 << 26, 1 << 25),                 # a at K = 26 (side Y), b at K = 25 (side in T above L); inverse K = 27
    ((1 << 25) + 12345, (1 << 24) - 7), # a at K = 26 = log2 n (side Y), b at K = 24; inverse K = 26, ragged tails
]


@pytest.mark.parametrize("na,nb", CASES)
def test_products_match_the_oracle(ctx, na, nb):
    a = synth.operand(rng.getrandbits(63), na)
    b = synth.operand(rng.getrandbits(63), nb)
    two_pass, steps = both_forms(ctx, lambda: host(ctx.mul(dev(a), na, dev(b), nb)))
    want = O.mul(a, na, b, nb)
    assert np.array_equal(two_pass, want)
    assert np.array_equal(steps, want)


@pytest.mark.parametrize("e", [27, 28, 29, 30, 31])
def test_long_products_modular(ctx, e):
    # K = 27 .. 31 forward and 28 .. 32 inverse (m = 16: the side buffer as long
    # as the array): 16 modular checks, and the same bits as the division steps
    lows = O.random_irreducibles(synth.config_seed(3, 97), 16)
    na = nb = 1 << e
    a = synth.operand(synth.config_seed(3, 300 + e), na)
    b = synth.operand(synth.config_seed(3, 330 + e), nb)
    two_pass, steps = both_forms(ctx, lambda: host(ctx.mul(dev(a), na, dev(b), nb)))
    assert O.modcheck(a, na, b, nb, two_pass, na + nb - 1, lows).all()
    assert np.array_equal(two_pass, steps)


def test_batch_class_launches_match_the_oracle(ctx):
    # three jobs of one size class (count 3, buffers a stride apart), class
    # launches (the persistent batch kernel keeps the division steps)
    from paper_1803_11301_gb300 import KNOB_BATCH_PERSISTENT
    sizes = [(1 << 25, 1 << 25), ((1 << 25) - 9, (1 << 24) + 3), (1 << 24, (1 << 25) - 1)]
    ops = [(synth.operand(rng.getrandbits(63), na), na, synth.operand(rng.getrandbits(63), nb), nb) for na, nb in sizes]

    def run():
        outs = [ctx.empty_words((na + nb - 1 + 63) // 64) for _, na, _, nb in ops]
        ctx.mul_batch([(dev(a), na, dev(b), nb, c) for (a, na, b, nb), c in zip(ops, outs)])
        return [host(c) for c in outs]

    ctx.tune_pin(KNOB_BATCH_PERSISTENT, 0)
    try:
        two_pass, steps = both_forms(ctx, run)
    finally:
        ctx.tune_pin(KNOB_BATCH_PERSISTENT, -1)
    for (a, na, b, nb), got, ref in zip(ops, two_pass, steps):
        assert np.array_equal(got, O.mul(a, na, b, nb))
        assert np.array_equal(got, ref)


def test_reused_operand_transform(ctx):
    # b's transform at n = 2^27 (BasisCvt at K = 26 with side Y), then a product with it
    from paper_1803_11301_gb300 import transform_bits
    na, nb = (1 << 25) + 77, (1 << 26) - 5
    a = synth.operand(rng.getrandbits(63), na)
    b = synth.operand(rng.getrandbits(63), nb)
    n = transform_bits(na, nb)

    def run():
        bhat = ctx.forward_transform(dev(b), nb, n)
        return host(ctx.mul_transformed(dev(a), na, bhat, nb)), host(bhat)

    (c2, t2), (c1, t1) = both_forms(ctx, run)
    assert np.array_equal(t2, t1)
    assert np.array_equal(c2, O.mul(a, na, b, nb))
    assert np.array_equal(c1, c2)


@pytest.mark.parametrize("na,nb", [(1 << 25, 1 << 25), (1 << 26, (1 << 25) - 3)])
def test_m128_products_match_the_oracle(ctx, na, nb):
    # the GF(2^128) path shares BasisCvt: both operands in one call, then one at a time
    a = synth.operand(rng.getrandbits(63), na)
    b = synth.operand(rng.getrandbits(63), nb)
    two_pass, steps = both_forms(ctx, lambda: host(ctx.mul_m128(dev(a), na, dev(b), nb)))
    want = O.mul(a, na, b, nb)
    assert np.array_equal(two_pass, want)
    assert np.array_equal(steps, want)
