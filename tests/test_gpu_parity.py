"""Parity of the CUDA path (through the C ABI) with the CPU oracle -- needs a GPU.

Integer work, so the bar is bit-exact everywhere.  Stage by stage (Alg. 1,
4, 2, the pointwise step of Alg. 5) against ``oracle.stages``; end to end (Alg. 5) against
the Karatsuba oracle where it finishes and against the modular checker at
2^30-bit operands; the forward transform sampled against evaluation at the
partition (Eq. 8) at full size.
"""
import random

import numpy as np
import pytest

import synth
from oracle import clmul as O
from oracle import field as F
from oracle import stages as S

pytestmark = pytest.mark.gpu

rng = random.Random(0xB300)


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


def rand_words(n):
    return synth.splitmix64(rng.getrandbits(63), n)


# ------------------------------------------------------------------ stages
def test_pointwise_field_product(ctx):
    for count in [1, 31, 1000, 1 << 16]:
        a, b = rand_words(count), rand_words(count)
        k = min(3, count)
        a[:k] = [0, 1, 1 << 63][:k]
        b[:k] = [5, 1 << 63, 2][:k]
        got = host(ctx.pointwise(dev(a), dev(b)))
        assert np.array_equal(got, F.gf_mul_arr(a, b))


@pytest.mark.parametrize("L", [64, 128, 256, 1024, 4096, 1 << 14, 1 << 16])
def test_basis_cvt_matches_alg1(ctx, L):
    f = O.words_to_int(rand_words(L // 64))
    t = dev(O.int_to_words(f, L))
    ctx.basis_cvt(t, L)
    assert O.words_to_int(host(t)) == S.basis_cvt(f, L)
    ctx.ibasis_cvt(t, L)
    assert O.words_to_int(host(t)) == f


@pytest.mark.parametrize("L", [1 << 17, 1 << 20, 1 << 24])
def test_basis_cvt_wide_steps_by_evaluation(ctx, L):
    # beyond one tile: check sum_k g_k X_k(beta) = f(beta) at random beta, and the inverse
    w = rand_words(L // 64)
    t = dev(w)
    ctx.basis_cvt(t, L)
    g = host(t)
    for _ in range(3):
        beta = rng.getrandbits(64)
        assert S.novelpoly_eval(g, L, beta) == O.eval_at(w, L, beta)
    ctx.ibasis_cvt(t, L)
    assert np.array_equal(host(t), w)


@pytest.mark.parametrize("n", [64, 128, 512, 2048, 4096, 1 << 13, 1 << 15])
def test_encode_decode_match_alg4(ctx, n):
    A = O.words_to_int(rand_words(n // 64))
    f = ctx.encode(dev(O.int_to_words(A, n)), n)
    assert np.array_equal(host(f), S.encode(A, n))
    back = ctx.decode(f, n)
    assert O.words_to_int(host(back)) == A


@pytest.mark.parametrize("l", [0, 1, 2, 5, 6, 7, 8, 9, 11, 12, 14, 15, 17, 19])
def test_butterfly_matches_alg2(ctx, l):
    n = 64 << l
    tw = S.Twiddles(l)
    g = rand_words(1 << l)
    t = dev(g)
    ctx.butterfly(t, n)
    y = host(t)
    assert np.array_equal(y, S.butterfly(g, tw))
    ctx.ibutterfly(t, n)
    assert np.array_equal(host(t), g)


@pytest.mark.parametrize("nbits", [64, 1000, 1 << 13, 1 << 16])
def test_forward_path_is_evaluation_at_sigma(ctx, nbits):
    # BasisCvt -> Encode -> Butterfly gives A(alpha + u_k) (Eq. 8)
    n = 2 * S.next_pow2(nbits) if nbits > 32 else 64
    l = n.bit_length() - 1 - 6
    w = synth.mask_tail(rand_words((nbits + 63) // 64), nbits)
    buf = np.zeros(n // 64, dtype=np.uint64)
    buf[: len(w)] = w
    t = dev(buf)
    ctx.basis_cvt(t, max(64, S.next_pow2(nbits)))
    f = ctx.encode(t, n)
    ctx.butterfly(f, n)
    y = host(f)
    for k in sorted({0, 1, (1 << l) - 1} | {rng.randrange(1 << l) for _ in range(5)}):
        assert int(y[k]) == O.eval_at(w, nbits, S.sigma_point(l, k)), k


# -------------------------------------------------------------- end to end
def check_product(ctx, na, nb, seed, square=False):
    a = synth.operand(seed, na)
    b = a if square else synth.operand(seed + 1, nb)
    da = dev(a)
    db = da if square else dev(b)
    got = host(ctx.mul(da, na, db, nb))
    want = O.mul(a, na, b, nb)
    assert np.array_equal(got, want), (na, nb, seed)


EDGE = [(1, 1), (1, 2), (2, 1), (3, 5), (31, 33), (32, 33), (33, 33), (63, 1), (64, 1), (65, 1), (64, 64),
        (65, 64), (100, 3), (127, 129), (1000, 1000), (1, 5000), (4095, 4097), (4096, 4096), (12345, 678),
        (1 << 15, 1 << 15), (1 << 16, 1), (70001, 3333), (1 << 17, 1 << 17), (99999, 200001)]


@pytest.mark.parametrize("na,nb", EDGE)
def test_product_edge_sizes(ctx, na, nb):
    check_product(ctx, na, nb, synth.config_seed(7, na ^ nb))


def test_repeated_calls_replay_with_new_contents(ctx):
    # the same buffers and sizes on every call: calls 2.. replay a captured graph
    import torch
    na, nb = 50000, 123457
    da = dev(np.zeros((na + 63) // 64, np.uint64))
    db = dev(np.zeros((nb + 63) // 64, np.uint64))
    out = torch.empty((na + nb - 1 + 63) // 64, dtype=torch.int64, device="cuda")
    from paper_1803_11301_gb300 import workspace_bytes
    ws = torch.empty(workspace_bytes(na, nb), dtype=torch.uint8, device="cuda")
    for k in range(5):
        a = synth.operand(synth.config_seed(10, 2 * k), na)
        b = synth.operand(synth.config_seed(10, 2 * k + 1), nb)
        da.copy_(dev(a))
        db.copy_(dev(b))
        ctx.mul(da, na, db, nb, out=out, workspace=ws)
        assert np.array_equal(host(out), O.mul(a, na, b, nb)), k


def test_product_squaring_alias(ctx):
    for n in [1, 64, 777, 1 << 16]:
        check_product(ctx, n, n, synth.config_seed(8, n), square=True)


def test_product_empty_operands(ctx):
    import torch
    a = dev(synth.operand(1, 100))
    out = ctx.mul(a, 100, a, 0)
    assert out.numel() == 0
    torch.cuda.synchronize()


def test_config1_many_seeds(ctx):
    # 2^16 x 2^16, seeded uniform random bits (the small workload)
    n = 1 << 16
    for i in range(200):
        check_product(ctx, n, n, synth.config_seed(1, 2 * i))


def test_config2_bit_exact(ctx):
    n = 1 << 24
    for i in range(2):
        check_product(ctx, n, n, synth.config_seed(2, 2 * i))


def test_config3_modular_and_sampled_forward(ctx):
    # 2^30 x 2^30: c mod p = (a mod p)(b mod p) mod p for 64 seeded irreducible p
    na = nb = 1 << 30
    a = synth.operand(synth.config_seed(3, 0), na)
    b = synth.operand(synth.config_seed(3, 1), nb)
    c = host(ctx.mul(dev(a), na, dev(b), nb))
    lows = O.random_irreducibles(synth.config_seed(3, 99), 64)
    ok = O.modcheck(a, na, b, nb, c, na + nb - 1, lows)
    assert ok.all(), int(ok.sum())
    assert O.words_to_int(c[-1:]) >> ((na + nb - 1) % 64) == 0       # tail written as zero


def test_length_sweep_modular(ctx):
    # every power 2^18 .. 2^29 of the length sweep (2^30 has its own test above):
    # 16 modular checks each, the full oracle where it finishes in a few seconds
    lows = O.random_irreducibles(synth.config_seed(3, 98), 16)
    for e in range(18, 30):
        na = nb = 1 << e
        a = synth.operand(synth.config_seed(3, 10 + e), na)
        b = synth.operand(synth.config_seed(3, 40 + e), nb)
        c = host(ctx.mul(dev(a), na, dev(b), nb))
        assert O.modcheck(a, na, b, nb, c, na + nb - 1, lows).all(), e
        if e <= 22:
            assert np.array_equal(c, O.mul(a, na, b, nb)), e


def test_product_beyond_structured_basis_cvt(ctx):
    # n = 2^33: BasisCvt at K = 33 runs the generic step kernels (the structured
    # ones cover K <= 32); 2^32 x 2^32 bits, 16 modular checks and the zero tail
    na = nb = 1 << 32
    a = synth.operand(synth.config_seed(3, 200), na)
    b = synth.operand(synth.config_seed(3, 201), nb)
    c = host(ctx.mul(dev(a), na, dev(b), nb))
    lows = O.random_irreducibles(synth.config_seed(3, 97), 16)
    assert O.modcheck(a, na, b, nb, c, na + nb - 1, lows).all()
    assert O.words_to_int(c[-1:]) >> ((na + nb - 1) % 64) == 0


def test_host_entry_point(ctx):
    for na, nb in [(1, 1), (1000, 77), (1 << 18, 1 << 17)]:
        a = synth.operand(5 + na, na)
        b = synth.operand(6 + nb, nb)
        assert np.array_equal(ctx.mul_host(a, na, b, nb), O.mul(a, na, b, nb))


def test_host_entry_point_unaligned_pinned_buffers(ctx):
    # page-locked buffers at odd byte offsets are not read by the kernels
    # directly (they access whole words): the call stages them and still
    # returns the product
    import ctypes
    import torch
    from paper_1803_11301_gb300 import host_workspace_bytes
    na, nb = 70001, 3333
    nc = na + nb - 1
    wa, wb, wc = (na + 63) // 64, (nb + 63) // 64, (nc + 63) // 64
    a = synth.operand(synth.config_seed(10, 71), na)
    b = synth.operand(synth.config_seed(10, 72), nb)
    raw = torch.zeros(8 * (wa + wb + wc) + 64, dtype=torch.uint8).pin_memory()
    base = raw.data_ptr()
    pa, pb, pc = base + 1, base + 8 * wa + 11, base + 8 * (wa + wb) + 21      # misaligned, disjoint
    ctypes.memmove(pa, a.tobytes(), 8 * wa)
    ctypes.memmove(pb, b.tobytes(), 8 * wb)
    ws = ctx.workspace(host_workspace_bytes(na, nb))
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        ctypes.memset(pc, 0xFF, 8 * wc)
        assert ctx._lib.gf2x_mul_host(ctx._h, ctypes.c_void_p(pa), na, ctypes.c_void_p(pb), nb,
                                      ctypes.c_void_p(pc), ctypes.c_void_p(ws.data_ptr()), ws.numel(), st) == 0
        got = np.frombuffer(ctypes.string_at(pc, 8 * wc), dtype=np.uint64)
        assert np.array_equal(got, O.mul(a, na, b, nb))
    assert ctx.stream_status() == 0


def test_host_entry_point_pinned_buffers(ctx):
    # page-locked host buffers: the load and store kernels use them directly
    import torch
    for na, nb in [(1000, 77), (1 << 18, 1 << 17), (1 << 20, 1 << 20)]:
        nc = na + nb - 1
        pa = torch.zeros((na + 63) // 64, dtype=torch.int64).pin_memory()
        pb = torch.zeros((nb + 63) // 64, dtype=torch.int64).pin_memory()
        pc = torch.zeros((nc + 63) // 64, dtype=torch.int64).pin_memory()
        va, vb, vc = (t.numpy().view(np.uint64) for t in (pa, pb, pc))
        for k in range(2):                          # the second call replays the captured graph
            a = synth.operand(synth.config_seed(10, 2 * k + na), na)
            b = synth.operand(synth.config_seed(10, 2 * k + nb + 1), nb)
            va[:] = a
            vb[:] = b
            ctx.mul_host(va, na, vb, nb, out=vc)
            assert np.array_equal(vc, O.mul(a, na, b, nb)), (na, nb, k)


# --------------------------------------------------------------- errors
def test_bounded_wait_reports_timeout(ctx):
    # a device-side wait that can never complete gives up and reports GF2X_ETIMEOUT
    ctx.selftest_wait_timeout()
    assert ctx.stream_status() == 5
    assert ctx.stream_status() == 0                  # reading resets the status word
    check_product(ctx, 70001, 3333, synth.config_seed(7, 1234))   # the context stays usable



def test_argument_errors(ctx):
    from paper_1803_11301_gb300 import Gf2xError, load_library
    import ctypes
    lib = load_library()
    a = dev(synth.operand(3, 256))
    c = dev(np.zeros(8, np.uint64))
    ws = ctx.workspace(1 << 16)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    big = (1 << 36) + 1
    assert lib.gf2x_mul(ctx._h, P(a), big, P(a), big, P(c), P(ws), ws.numel(), None) == 2     # ETOOBIG
    assert lib.gf2x_mul(ctx._h, P(a), 256, P(a), 200, P(c), P(ws), 16, None) == 7             # ENOSPACE
    assert lib.gf2x_mul(ctx._h, P(a), 256, P(a), 200, P(a), P(ws), ws.numel(), None) == 1    # c overlaps a
    assert lib.gf2x_basis_cvt(ctx._h, P(a), 96, None) == 1                                     # not a power of 2
    with pytest.raises(Gf2xError):
        ctx.encode(a, 100)
    assert ctx.stream_status() == 0


# ---------------------------------------------------------------- batches
def _batch_jobs(ctx, lengths, seed):
    import torch
    jobs, host = [], []
    for k, (na, nb) in enumerate(lengths):
        a = synth.operand(synth.config_seed(seed, 2 * k), max(na, 1))
        b = synth.operand(synth.config_seed(seed, 2 * k + 1), max(nb, 1))
        da, db = dev(a), dev(b)
        nc = na + nb - 1 if na and nb else 0
        c = torch.full((max((nc + 63) // 64, 1),), -1, dtype=torch.int64, device="cuda")
        jobs.append((da, na, db, nb, c))
        host.append((a, b))
    return jobs, host


def test_batch_uneven_lengths_bit_exact(ctx):
    lens = synth.loguniform_lengths(synth.config_seed(4, 7), 400, 6.0, 17.0).reshape(200, 2)
    lengths = [(int(x), int(y)) for x, y in lens] + [(0, 100), (100, 0), (1, 1), (3, 70000), (70000, 3)]
    jobs, host = _batch_jobs(ctx, lengths, 41)
    jobs.append((jobs[5][0], jobs[5][1], jobs[5][0], jobs[5][1], jobs[-1][4].clone()))   # shared operand
    host.append((host[5][0], host[5][0]))
    for rep in range(3):                      # call 1 direct, call 2 captures, call 3 replays
        for j in jobs:
            j[4].fill_(-1)
        ctx.mul_batch(jobs)
        for (da, na, db, nb, c), (a, b) in zip(jobs, host):
            nc = na + nb - 1 if na and nb else 0
            if nc == 0:
                continue
            assert np.array_equal(host_words(c, nc), O.mul(a, na, b, nb)), (rep, na, nb)


@pytest.mark.parametrize("persistent", [1, 0])
def test_batch_persistent_and_class_launches(ctx, persistent):
    # the batch as one persistent launch (device work queue) and as one launch
    # per kernel and size class: both bit-exact against the oracle, on call 1
    # (direct), 2 (captured) and 3 (replayed)
    from paper_1803_11301_gb300 import KNOB_BATCH_PERSISTENT
    lens = synth.loguniform_lengths(synth.config_seed(4, 8), 240, 6.0, 19.0).reshape(120, 2)
    lengths = [(int(x), int(y)) for x, y in lens] + [(1, 1), (64, 64), (1 << 18, 3), (0, 9), (1 << 19, 1 << 19)]
    jobs, hostops = _batch_jobs(ctx, lengths, 45)
    ctx.tune_pin(KNOB_BATCH_PERSISTENT, persistent)
    try:
        for rep in range(3):
            for j in jobs:
                j[4].fill_(-1)
            ctx.profile_enable(False)
            ctx.mul_batch(jobs)
            launches = ctx.profile_read()
            for (da, na, db, nb, c), (a, b) in zip(jobs, hostops):
                nc = na + nb - 1 if na and nb else 0
                if nc:
                    assert np.array_equal(host_words(c, nc), O.mul(a, na, b, nb)), (persistent, rep, na, nb)
            if persistent:
                assert launches["persistent_batch"][1] == 1, launches      # the whole batch: one launch
                assert sum(v[1] for v in launches.values()) == 1
            else:
                assert launches["persistent_batch"][1] == 0
        assert ctx.stream_status() == 0
    finally:
        ctx.tune_pin(KNOB_BATCH_PERSISTENT, -1)


def test_batch_queue_wait_times_out(ctx):
    # a queue item whose dependency can never finish: its bounded wait runs
    # out, GF2X_ETIMEOUT is recorded, the kernel returns and the context works
    ctx.selftest_queue_timeout()
    assert ctx.stream_status() == 5
    assert ctx.stream_status() == 0
    lens = [(1000, 3000), (1 << 16, 1 << 15)]
    jobs, hostops = _batch_jobs(ctx, lens, 46)
    ctx.mul_batch(jobs)
    for (da, na, db, nb, c), (a, b) in zip(jobs, hostops):
        assert np.array_equal(host_words(c, na + nb - 1), O.mul(a, na, b, nb))


def host_words(t, nbits):
    return host(t)[: (nbits + 63) // 64]


def test_batch_config4_4096_products(ctx):
    # 4096 products, operand lengths log-uniform in [2^10, 2^20] bits, a and b
    # independent: every product bit-exact against the Karatsuba oracle
    lens = synth.loguniform_lengths(synth.config_seed(4, 0), 8192, 10.0, 20.0).reshape(4096, 2)
    lengths = [(int(x), int(y)) for x, y in lens]
    jobs, host = _batch_jobs(ctx, lengths, 44)
    ctx.mul_batch(jobs)
    outs = [host_words(c, na + nb - 1) for (da, na, db, nb, c) in jobs]
    for k, ((da, na, db, nb, c), (a, b)) in enumerate(zip(jobs, host)):
        assert np.array_equal(outs[k], O.mul(a, na, b, nb)), (k, na, nb)


def test_serving_results_same_alone_and_in_the_mix(ctx):
    # overlapping batches on several streams; every result equals the product computed alone
    import torch
    from paper_1803_11301_gb300.serving import Server, Request
    lens = synth.loguniform_lengths(synth.config_seed(5, 3), 300, 8.0, 18.0).reshape(150, 2)
    pool = [dev(synth.operand(synth.config_seed(5, 300 + k), 1 << 18)) for k in range(4)]
    srv = Server(ctx, streams=3, max_batch=16)
    reqs = []
    for k in range(150):
        r = Request(pool[k % 4], int(lens[k, 0]), pool[(k + 1) % 4], int(lens[k, 1]), tag=k)
        reqs.append(r)
        srv.submit(r)
        if k % 7 == 0:
            srv.poll()                                   # arrivals interleave with running batches
    srv.drain()
    torch.cuda.synchronize()
    assert srv._next_batch > 3
    pool_h = [host(p) for p in pool]
    for r in reqs:
        alone = ctx.mul(r.a, r.na, r.b, r.nb)
        nc = r.na + r.nb - 1
        got = r.out[: (nc + 63) // 64]
        assert torch.equal(got, alone), r.tag                              # alone and in the mix
        want = O.mul(pool_h[r.tag % 4], r.na, pool_h[(r.tag + 1) % 4], r.nb)
        assert np.array_equal(host(got), want), r.tag                      # and the oracle's product


def test_serving_rejects_a_request_beyond_the_budget(ctx):
    # a request that could not run even alone within the budget is refused at
    # admission with GF2X_ENOMEM and never queued; the others are served
    import torch
    from paper_1803_11301_gb300.serving import GF2X_ENOMEM, GF2X_OK, Request, Server
    srv = Server(ctx, streams=2, memory_budget=64 << 20)
    small = dev(synth.operand(synth.config_seed(5, 401), 1 << 14))
    big = dev(synth.operand(synth.config_seed(5, 402), 1 << 26))
    ok1 = Request(small, 1 << 14, small, 5000, tag=1)
    huge = Request(big, 1 << 26, big, 1 << 26, tag=2)          # 3 x 16 MiB of workspace and more
    ok2 = Request(small, 3000, small, 1 << 14, tag=3)
    assert srv.submit(ok1) == GF2X_OK
    assert srv.submit(huge) == GF2X_ENOMEM
    assert srv.submit(ok2) == GF2X_OK
    assert huge.state == "rejected" and huge not in srv.pending and srv.rejected == [huge]
    srv.drain()
    torch.cuda.synchronize()
    sh = host(small)
    for r in (ok1, ok2):
        assert r.state == "done"
        assert np.array_equal(host_words(r.out, r.na + r.nb - 1), O.mul(sh, r.na, sh, r.nb))


def test_serving_cancels_pending_requests(ctx):
    # requests cancelled before a batch takes them never run; the rest are exact
    import torch
    from paper_1803_11301_gb300.serving import Request, Server
    srv = Server(ctx, streams=1, max_batch=4)
    pool = dev(synth.operand(synth.config_seed(5, 410), 1 << 16))
    ph = host(pool)
    reqs = [Request(pool, 1000 + 37 * k, pool, 2000 + 11 * k, tag=k) for k in range(24)]
    for r in reqs:
        srv.submit(r)
    srv.poll()                                       # one batch of 4 takes the first requests
    assert srv.cancel(reqs[0]) is False             # already running
    gone = [reqs[k] for k in (5, 9, 17, 23)]
    for r in gone:
        assert srv.cancel(r) is True
        assert srv.cancel(r) is False               # only once
    srv.drain()
    torch.cuda.synchronize()
    for r in reqs:
        if r in gone:
            assert r.state == "cancelled" and r.batch_id == -1
        else:
            assert r.state == "done"
            assert np.array_equal(host_words(r.out, r.na + r.nb - 1), O.mul(ph, r.na, ph, r.nb)), r.tag


def test_serving_resident_transform_of_a_recurring_operand(ctx):
    # the same b (named by b_key) recurs: from its second use on, its transform
    # stays on the device and the products skip b's forward steps; every
    # result equals the oracle's
    import torch
    from paper_1803_11301_gb300.serving import Request, Server
    srv = Server(ctx, streams=3, max_batch=8, reuse_after=2)
    b = dev(synth.operand(synth.config_seed(5, 420), 20000))
    pool = [dev(synth.operand(synth.config_seed(5, 421 + k), 30000)) for k in range(3)]
    bh, poolh = host(b), [host(t) for t in pool]
    reqs = []
    for k in range(40):
        r = Request(pool[k % 3], 30000 - 97 * (k % 5), b, 20000, tag=k, b_key="b20000")
        reqs.append(r)
        srv.submit(r)
        if k % 3 == 0:
            srv.poll()
    srv.drain()
    torch.cuda.synchronize()
    assert sum(r.reused for r in reqs) >= 30
    for r in reqs:
        want = O.mul(poolh[r.tag % 3], r.na, bh, r.nb)
        assert np.array_equal(host_words(r.out, r.na + r.nb - 1), want), r.tag


def test_serving_host_operands(ctx):
    # page-locked host operands: copied in and out on the batch's stream
    import torch
    from paper_1803_11301_gb300.serving import Request, Server
    srv = Server(ctx, streams=2, max_batch=8)
    words = [synth.operand(synth.config_seed(5, 430 + k), 1 << 17) for k in range(2)]
    pinned = [torch.from_numpy(w.view(np.int64)).pin_memory() for w in words]
    lens = synth.loguniform_lengths(synth.config_seed(5, 431), 60, 8.0, 17.0).reshape(30, 2)
    reqs = []
    for k, (na, nb) in enumerate(lens):
        na, nb = int(na), int(nb)
        r = Request(pinned[0][: (na + 63) // 64], na, pinned[1][: (nb + 63) // 64], nb, tag=k, host=True)
        reqs.append(r)
        srv.submit(r)
        srv.poll()
    srv.drain()
    torch.cuda.synchronize()
    for r in reqs:
        assert r.out.device.type == "cpu" and r.out.is_pinned()
        got = r.out.numpy().view(np.uint64)[: (r.na + r.nb - 1 + 63) // 64]
        assert np.array_equal(got, O.mul(words[0], r.na, words[1], r.nb)), r.tag


def test_serving_outputs_allocated_at_launch(ctx):
    # a queued request holds no output until a batch takes it; on_done sees every
    # completed request once, with its output in place and equal to the oracle's
    import torch
    from paper_1803_11301_gb300.serving import Request, Server
    done = []
    srv = Server(ctx, streams=1, max_batch=4, on_done=done.append)
    words = [synth.operand(synth.config_seed(5, 440 + k), 1 << 16) for k in range(2)]
    dev = [torch.from_numpy(w.view(np.int64)).cuda() for w in words]
    lens = synth.loguniform_lengths(synth.config_seed(5, 441), 48, 8.0, 16.0).reshape(24, 2)
    reqs = []
    for k, (na, nb) in enumerate(lens):
        na, nb = int(na), int(nb)
        r = Request(dev[0][: (na + 63) // 64], na, dev[1][: (nb + 63) // 64], nb, tag=k)
        reqs.append(r)
        srv.submit(r)
    assert all(r.out is None for r in reqs)         # nothing allocated while queued
    srv.poll()
    assert sum(r.out is not None for r in reqs) == 4  # the first batch's outputs only
    srv.drain()
    torch.cuda.synchronize()
    assert sorted(r.tag for r in done) == list(range(24))
    for r in reqs:
        assert np.array_equal(host_words(r.out, r.na + r.nb - 1), O.mul(words[0], r.na, words[1], r.nb)), r.tag


# ------------------------------------------------------------ reused operand
@pytest.mark.parametrize("na,nb", [(100, 5000), (1 << 16, 1 << 16), (70001, 3333), (1 << 20, 1 << 18), (64, 64)])
def test_reused_operand_transform(ctx, na, nb):
    # the forward steps of Alg. 5 once for b (gf2x_forward_transform), then products
    # with several a of the same transform length (gf2x_mul_transformed)
    from paper_1803_11301_gb300 import transform_bits
    b = synth.operand(synth.config_seed(9, nb), nb)
    n = transform_bits(na, nb)
    bhat = ctx.forward_transform(dev(b), nb, n)
    for k in range(3):
        a = synth.operand(synth.config_seed(9, 1000 + k), na)
        for _ in range(2):                            # second call replays the captured graph
            got = host(ctx.mul_transformed(dev(a), na, bhat, nb))
            assert np.array_equal(got, O.mul(a, na, b, nb)), (na, nb, k)


def test_forward_transform_is_evaluation_at_sigma(ctx):
    # the reusable transform is the forward path: B(alpha + u_k) (Eq. 8)
    from paper_1803_11301_gb300 import transform_bits
    nb = 70001
    n = transform_bits(nb, nb)
    l = n.bit_length() - 1 - 6
    b = synth.operand(synth.config_seed(9, 7), nb)
    y = host(ctx.forward_transform(dev(b), nb, n))
    for k in sorted({0, 1, (1 << l) - 1} | {rng.randrange(1 << l) for _ in range(5)}):
        assert int(y[k]) == O.eval_at(synth.mask_tail(b.copy(), nb), nb, S.sigma_point(l, k)), k


def test_default_launch_shapes_without_tuning(ctx):
    # GF2X_TUNE=0: the built-in shapes (bottom depth 9 up to l = 21, 11 above), same products
    import os
    from paper_1803_11301_gb300 import Context
    old = os.environ.get("GF2X_TUNE")
    os.environ["GF2X_TUNE"] = "0"
    try:
        c0 = Context(0)
    finally:
        if old is None:
            del os.environ["GF2X_TUNE"]
        else:
            os.environ["GF2X_TUNE"] = old
    try:
        for na, nb in [(1 << 18, 1 << 18), (1 << 22, 1 << 21), (123457, 1 << 20)]:
            a = synth.operand(synth.config_seed(9, na), na)
            b = synth.operand(synth.config_seed(9, nb + 7), nb)
            got = host(c0.mul(dev(a), na, dev(b), nb))
            assert np.array_equal(got, O.mul(a, na, b, nb)), (na, nb)
            l = S.transform_length(na, nb).bit_length() - 1 - 6
            assert c0.bottom_layers(na, nb) == min(l, 9 if l <= 21 else 11)
            assert 8 <= ctx.bottom_layers(na, nb) <= 11          # the tuned context's choice
    finally:
        c0.close()
