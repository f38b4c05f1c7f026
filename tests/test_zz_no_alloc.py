"""gf2x_mul_noalloc: the product for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc or any allocator (a framework that owns the
whole device through its own pool, or a path where entering an allocator is not
allowed).  gf2x_mul_noalloc runs the same product on a fixed scratch array inside
the library.  This test calls it through the C ABI twice in a row, on different
operands, and checks each result bit for bit against gf2x_mul and against the CPU
oracle (exact integer work, so the tolerance is zero).  It also checks that a product above the stated limit
is refused with GF2X_ETOOBIG.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1803_11301_gb300 import Context, build, load_library
    build.build()
    lib = load_library()
    ctx = Context(0)
    yield lib, ctx
    ctx.close()


def _dev(words):
    import torch
    return torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint64).view(np.int64)).cuda()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_gf2x_mul_twice(env):
    import torch
    from oracle import clmul as O
    lib, ctx = env
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(1 << 20, (1 << 20) - 5, 11), (777, 4093, 12)]       # two calls in a row
    for na, nb, k in cases:
        ah = synth.operand(synth.config_seed(77, 2 * k), na)
        bh = synth.operand(synth.config_seed(77, 2 * k + 1), nb)
        a, b = _dev(ah), _dev(bh)
        nc = na + nb - 1
        want = ctx.mul(a, na, b, nb)
        got = torch.zeros((nc + 63) // 64, dtype=torch.int64, device="cuda")
        status = lib.gf2x_mul_noalloc(ctx._h, _ptr(a), na, _ptr(b), nb, _ptr(got), stream)
        assert status == 0, status
        torch.cuda.synchronize()
        assert torch.equal(got, want), (na, nb)                    # the existing entry point's result
        got_h = got.cpu().numpy().view(np.uint64)
        assert np.array_equal(got_h, O.mul(ah, na, bh, nb)), (na, nb)   # and the CPU oracle's


def test_noalloc_rejects_products_above_the_limit(env):
    import torch
    lib, ctx = env
    na = nb = (1 << 20) + 1                                          # n = 2^22 > 2^21
    a = _dev(synth.operand(5, na))
    c = torch.zeros((na + nb - 1 + 63) // 64, dtype=torch.int64, device="cuda")
    assert lib.gf2x_mul_noalloc(ctx._h, _ptr(a), na, _ptr(a), nb, _ptr(c), None) == 2   # GF2X_ETOOBIG
    assert lib.gf2x_mul_noalloc(ctx._h, _ptr(a), na, _ptr(a), 0, _ptr(c), None) == 0    # empty product
