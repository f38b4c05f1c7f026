"""Range-checked build and host-side failure injection -- needs a GPU.

A library built with GF2X_DEBUG_BOUNDS checks the kernels' main global
indices against the buffers they address and counts what falls outside
(gf2x_stream_status then reports GF2X_EBOUNDS; nothing traps).  The sweep runs
that build on small products of every transform length 2^6 .. 2^14 and every
tail length mod 64 of the operands, alone and as one batch, in a process of
its own (GF2X_DEBUG_BOUNDS=1 selects that library), and requires every product
to equal the oracle's with no index out of range.

Failures are injected on the host only: a workspace allocator that returns
nothing, a NULL workspace, a workspace too small.  No kernel is made to fault.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from oracle import clmul as O

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SWEEP = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, %(root)r)
import synth
from oracle import clmul as O
from paper_1803_11301_gb300 import Context, build
build.build(debug_bounds=True)
ctx = Context(0)
dev = lambda w: torch.from_numpy(np.ascontiguousarray(w, dtype=np.uint64).view(np.int64)).cuda()
pairs = []
for e in range(6, 15):
    for t in range(64):
        pairs.append((max(1, (1 << (e - 1)) - t), max(1, (1 << (e - 1)) - 63 + t)))
jobs, want = [], []
for k, (na, nb) in enumerate(pairs):
    a = synth.operand(synth.config_seed(11, 2 * k), na)
    b = synth.operand(synth.config_seed(11, 2 * k + 1), nb)
    da, db = dev(a), dev(b)
    got = ctx.mul(da, na, db, nb).cpu().numpy().view(np.uint64)
    w = O.mul(a, na, b, nb)
    assert np.array_equal(got, w), ("single", na, nb)
    out = torch.full(((na + nb - 1 + 63) // 64,), -1, dtype=torch.int64, device="cuda")
    jobs.append((da, na, db, nb, out))
    want.append(w)
assert ctx.stream_status() == 0, "out-of-range index in single products"
ctx.mul_batch(jobs)
for (da, na, db, nb, out), w in zip(jobs, want):
    assert np.array_equal(out.cpu().numpy().view(np.uint64), w), ("batch", na, nb)
assert ctx.stream_status() == 0, "out-of-range index in the batch"
print("SWEEP_OK", len(pairs))
"""


def test_debug_bounds_sweep_every_tail_length():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    env = dict(os.environ, GF2X_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", SWEEP % {"root": ROOT}], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0 and "SWEEP_OK 576" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


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


def _dev(w):
    import torch
    return torch.from_numpy(np.ascontiguousarray(w, dtype=np.uint64).view(np.int64)).cuda()


def test_allocator_that_returns_nothing(ctx):
    # the workspace allocator fails: the call raises GF2X_ENOMEM and enqueues
    # nothing; with torch's allocator again the same call works
    from paper_1803_11301_gb300 import Gf2xError
    na, nb = 5000, 7000
    a = synth.operand(synth.config_seed(11, 900), na)
    b = synth.operand(synth.config_seed(11, 901), nb)
    da, db = _dev(a), _dev(b)
    ctx.set_allocator(lambda nbytes: None)
    try:
        with pytest.raises(Gf2xError) as err:
            ctx.mul(da, na, db, nb)
        assert err.value.status == 3
    finally:
        ctx.set_allocator(None)
    assert np.array_equal(ctx.mul(da, na, db, nb).cpu().numpy().view(np.uint64), O.mul(a, na, b, nb))
    assert ctx.stream_status() == 0


def test_missing_or_short_workspace_is_refused(ctx):
    # NULL, misaligned or too small workspaces are argument errors: nothing runs
    import ctypes
    import torch
    lib = ctx._lib
    na = nb = 3000
    a = _dev(synth.operand(synth.config_seed(11, 902), na))
    c = torch.zeros((na + nb - 1 + 63) // 64, dtype=torch.int64, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    from paper_1803_11301_gb300 import Job, workspace_bytes
    need = workspace_bytes(na, nb)
    ws = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.gf2x_mul(ctx._h, P(a), na, P(a), nb, P(c), None, need, st) == 1              # EINVAL
    assert lib.gf2x_mul(ctx._h, P(a), na, P(a), nb, P(c), ctypes.c_void_p(ws.data_ptr() + 8), need, st) == 1
    assert lib.gf2x_mul(ctx._h, P(a), na, P(a), nb, P(c), P(ws), need - 1, st) == 7          # ENOSPACE
    jobs = (Job * 1)(Job(a.data_ptr(), na, a.data_ptr(), nb, c.data_ptr()))
    assert lib.gf2x_mul_batch(ctx._h, jobs, 1, None, need, st) == 1
    assert lib.gf2x_mul_batch(ctx._h, jobs, 1, P(ws), 256, st) == 7
    torch.cuda.synchronize()
    assert not c.any()                                                                        # nothing ran
    assert ctx.stream_status() == 0
