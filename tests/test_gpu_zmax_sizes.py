"""Products at the largest transform lengths the ABI accepts -- needs a GPU.

gf2x_mul at n = 2^37 (2^36 x 2^36 bits, the Sec. 3.1 limit with m = 64) and
gf2x_mul_m128 at n = 2^38 (2^37 x 2^37 bits: past the m = 64 limit, the
length the m = 128 variant adds on one GB300).  Each is checked against 16
seeded irreducible moduli (c mod p = (a mod p)(b mod p) mod p) and its zero
tail.  They need 80 GB and 160 GB of device memory and about 1.5x their
operands and result in host memory; a test skips itself when either is short.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import synth
from oracle import clmul as O

pytestmark = pytest.mark.gpu

CHUNK = 1 << 24


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


def operand(seed, nbits):
    """synth.operand(seed, nbits), generated in chunks on every host core (same words)."""
    nw = (nbits + 63) // 64
    out = np.empty(nw, dtype=np.uint64)

    def fill(off):
        cnt = min(CHUNK, nw - off)
        out[off:off + cnt] = synth.splitmix64(seed, cnt, offset=off)

    with ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
        list(ex.map(fill, range(0, nw, CHUNK)))
    return out


def host_free_bytes():
    return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")


def run_max(ctx, mul, ws_bytes, na, nb, seed):
    import torch
    nc = na + nb - 1
    dev_need = ws_bytes + (na + nb + nc) // 8 + (4 << 30)
    host_need = int(1.5 * (na + nb + nc) // 8)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < dev_need or host_free_bytes() < host_need:
        pytest.skip(f"needs {dev_need >> 30} GiB device and {host_need >> 30} GiB host memory")
    a = operand(seed, na)
    b = operand(seed + 1, nb)
    da = torch.from_numpy(a.view(np.int64)).cuda()
    db = torch.from_numpy(b.view(np.int64)).cuda()
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = torch.empty((nc + 63) // 64, dtype=torch.int64, device="cuda")
    mul(da, na, db, nb, out=out, workspace=ws)
    del ws, da, db
    c = out.cpu().numpy().view(np.uint64)
    del out
    torch.cuda.empty_cache()
    lows = O.random_irreducibles(synth.config_seed(3, 96), 16)
    assert O.modcheck(a, na, b, nb, c, nc, lows).all()
    assert O.words_to_int(c[-1:]) >> (nc % 64) == 0


def test_m64_at_the_length_limit(ctx):
    from paper_1803_11301_gb300 import workspace_bytes
    na = nb = 1 << 36
    run_max(ctx, ctx.mul, workspace_bytes(na, nb), na, nb, synth.config_seed(3, 300))


def test_m128_beyond_the_m64_limit(ctx):
    from paper_1803_11301_gb300 import m128_workspace_bytes, workspace_bytes
    na = nb = 1 << 37
    assert workspace_bytes(na, nb) == 0                 # n = 2^38: past the m = 64 limit
    run_max(ctx, ctx.mul_m128, m128_workspace_bytes(na, nb), na, nb, synth.config_seed(14, 300))
