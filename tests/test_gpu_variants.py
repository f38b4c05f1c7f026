"""Every launch variant the autotuner can pick gives the same bits -- needs a GPU.

The tuner chooses among kernel shapes that compute the same result (bottom
depth and block shape of the fused Butterfly kernel, table chunk and depth of
the GF(2^128) one, words per thread and window depth of BasisCvt).  Here each
candidate is pinned through gf2x_tune_pin and the product, batch, reused-operand
and stage paths are compared bit for bit with the oracle (Alg. 5 by the
Karatsuba oracle, Alg. 2 by ``oracle.stages``).
"""
import random

import numpy as np
import pytest

import synth
from oracle import clmul as O
from oracle import stages as S

pytestmark = pytest.mark.gpu


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


@pytest.fixture
def pins(ctx):
    """Pins set by a test are released after it."""
    used = []

    def pin(knob, choice):
        ctx.tune_pin(knob, choice)
        used.append(knob)

    yield pin
    for k in used:
        ctx.tune_pin(k, -1)


def dev(words):
    import torch
    return torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint64).view(np.int64)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint64)


def test_pin_arguments(ctx):
    from paper_1803_11301_gb300 import Gf2xError
    with pytest.raises(Gf2xError):
        ctx.tune_pin(0, 9)
    with pytest.raises(Gf2xError):
        ctx.tune_pin(10, 9)
    with pytest.raises(Gf2xError):
        ctx.tune_pin(5, -2)
    ctx.tune_pin(5, -1)                                   # releasing an unpinned knob is fine


@pytest.mark.parametrize("depth", [8, 9, 10, 11])
@pytest.mark.parametrize("shape", [0, 1, 2])
def test_product_every_bottom_depth_and_shape(ctx, pins, depth, shape):
    from paper_1803_11301_gb300 import KNOB_BOTTOM_DEPTH, KNOB_BOTTOM_SHAPE
    pins(KNOB_BOTTOM_DEPTH, depth)
    pins(KNOB_BOTTOM_SHAPE, shape)
    for na, nb in [(1 << 20, (1 << 20) - 3), (1 << 16, 40000)]:
        a = synth.operand(synth.config_seed(21, na), na)
        b = synth.operand(synth.config_seed(22, nb), nb)
        want = O.mul(a, na, b, nb)
        da, db = dev(a), dev(b)
        for rep in range(3):                              # direct, capture, replay
            got = host(ctx.mul(da, na, db, nb))
            assert np.array_equal(got, want), (depth, shape, na, nb, rep)
        assert ctx.bottom_layers(na, nb) == depth


@pytest.mark.parametrize("mul", [0, 1])
@pytest.mark.parametrize("depth,shape", [(9, 0), (11, 1), (8, 2)])
def test_product_both_integer_forms(ctx, pins, mul, depth, shape):
    # the bottom kernel's integer layers and pointwise step with either product form
    from paper_1803_11301_gb300 import KNOB_BOTTOM_DEPTH, KNOB_BOTTOM_MUL, KNOB_BOTTOM_SHAPE
    pins(KNOB_BOTTOM_MUL, mul)
    pins(KNOB_BOTTOM_DEPTH, depth)
    pins(KNOB_BOTTOM_SHAPE, shape)
    for na, nb in [(1 << 20, (1 << 20) - 3), (70001, 3333)]:
        a = synth.operand(synth.config_seed(30, na + mul), na)
        b = synth.operand(synth.config_seed(31, nb + mul), nb)
        want = O.mul(a, na, b, nb)
        da, db = dev(a), dev(b)
        for rep in range(2):
            assert np.array_equal(host(ctx.mul(da, na, db, nb)), want), (mul, depth, shape, na, nb, rep)


@pytest.mark.parametrize("depth,shape", [(8, 1), (10, 2), (11, 0), (9, 1)])
def test_batch_pinned_shapes(ctx, pins, depth, shape):
    import torch
    from paper_1803_11301_gb300 import KNOB_BOTTOM_DEPTH, KNOB_BOTTOM_SHAPE
    pins(KNOB_BOTTOM_DEPTH, depth)
    pins(KNOB_BOTTOM_SHAPE, shape)
    lens = synth.loguniform_lengths(synth.config_seed(23, depth * 3 + shape), 80, 10.0, 17.0).reshape(40, 2)
    jobs, want = [], []
    for k, (na, nb) in enumerate(lens):
        na, nb = int(na), int(nb)
        a = synth.operand(synth.config_seed(24, 2 * k), na)
        b = synth.operand(synth.config_seed(24, 2 * k + 1), nb)
        c = torch.empty((na + nb - 1 + 63) // 64, dtype=torch.int64, device="cuda")
        jobs.append((dev(a), na, dev(b), nb, c))
        want.append(O.mul(a, na, b, nb))
    for rep in range(3):
        for j in jobs:
            j[4].fill_(-1)
        ctx.mul_batch(jobs)
        for (_, na, _, nb, c), w in zip(jobs, want):
            assert np.array_equal(host(c), w), (depth, shape, na, nb, rep)


@pytest.mark.parametrize("depth", [8, 10, 11])
@pytest.mark.parametrize("shape", [0, 1, 2])
def test_stage_butterfly_pinned(ctx, pins, depth, shape):
    # the stand-alone Butterfly and iButterfly: bottom kernel in its forward-only
    # and inverse-only modes
    from paper_1803_11301_gb300 import KNOB_BOTTOM_DEPTH, KNOB_BOTTOM_SHAPE
    pins(KNOB_BOTTOM_DEPTH, depth)
    pins(KNOB_BOTTOM_SHAPE, shape)
    l = 13
    rng = random.Random(depth * 7 + shape)
    g = np.array([rng.getrandbits(64) for _ in range(1 << l)], dtype=np.uint64)
    t = dev(g)
    ctx.butterfly(t, 64 << l)
    assert np.array_equal(host(t), S.butterfly(g, S.Twiddles(l))), (depth, shape)
    ctx.ibutterfly(t, 64 << l)
    assert np.array_equal(host(t), g), (depth, shape)


@pytest.mark.parametrize("depth,shape", [(8, 0), (9, 2), (10, 1), (11, 1)])
def test_reused_operand_pinned(ctx, pins, depth, shape):
    from paper_1803_11301_gb300 import KNOB_BOTTOM_DEPTH, KNOB_BOTTOM_SHAPE, transform_bits
    pins(KNOB_BOTTOM_DEPTH, depth)
    pins(KNOB_BOTTOM_SHAPE, shape)
    na, nb = 1 << 18, (1 << 18) + 5
    b = synth.operand(synth.config_seed(25, depth), nb)
    bhat = ctx.forward_transform(dev(b), nb, transform_bits(na, nb))
    for k in range(2):
        a = synth.operand(synth.config_seed(26, 10 * depth + k), na)
        for rep in range(2):
            got = host(ctx.mul_transformed(dev(a), na, bhat, nb))
            assert np.array_equal(got, O.mul(a, na, b, nb)), (depth, shape, k, rep)


@pytest.mark.parametrize("depth", [8, 9, 10])
@pytest.mark.parametrize("chunk", [4, 8])
def test_m128_every_depth_and_chunk(ctx, pins, depth, chunk):
    from paper_1803_11301_gb300 import KNOB_M128_BOTTOM_CHUNK, KNOB_M128_BOTTOM_DEPTH
    pins(KNOB_M128_BOTTOM_DEPTH, depth)
    pins(KNOB_M128_BOTTOM_CHUNK, chunk)
    for na, nb in [(1 << 18, (1 << 18) - 1), (70001, 3333)]:
        a = synth.operand(synth.config_seed(27, na), na)
        b = synth.operand(synth.config_seed(28, nb), nb)
        want = O.mul(a, na, b, nb)
        da, db = dev(a), dev(b)
        for rep in range(3):
            got = host(ctx.mul_m128(da, na, db, nb))
            assert np.array_equal(got, want), (depth, chunk, na, nb, rep)
        if na == 1 << 18:
            assert ctx.bottom_layers(na, nb, field=128) == depth


def test_basis_cvt_knobs(ctx, pins):
    # 2^23 x 2^23: forward BasisCvt at K = 23 (window depths 6, 7), inverse at
    # K = 24 (6, 7, 8); 2^16-bit units with 8, 16 or 32 words per thread
    from paper_1803_11301_gb300 import KNOB_UNIT16_R, KNOB_WINDOW_DEPTH
    n = 1 << 23
    a = synth.operand(synth.config_seed(29, 0), n)
    b = synth.operand(synth.config_seed(29, 1), n)
    want = O.mul(a, n, b, n)
    da, db = dev(a), dev(b)
    for r, w in [(8, 6), (16, 7), (32, 8), (8, 8), (32, 6), (16, 8)]:
        pins(KNOB_UNIT16_R, r)
        pins(KNOB_WINDOW_DEPTH, w)
        for rep in range(2):
            got = host(ctx.mul(da, n, db, n))
            assert np.array_equal(got, want), (r, w, rep)


def test_field_multiply_forms_agree(ctx):
    # every GF(2^64) product form of the measurement computes the same chains
    sums = [ctx.bench_field_mul(v, 3)["checksum"] for v in range(len(ctx.FIELD_VARIANTS))]
    assert len(set(sums)) == 1, sums
    assert ctx.stream_status() == 0
