"""The C-ABI library loads and exports every symbol include/gf2x.h declares (CPU only).

No compute call is made here: these run without a GPU.  Only the pure host
functions (size rules) and the no-device error path are exercised.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gf2x.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"GF2X_API\s+[\w\s\*]*?\b(gf2x_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_11301_gb300 import build, load_library
    build.build()
    return load_library()


def test_header_declares_the_api():
    names = declared_functions()
    for must in ["gf2x_ctx_create", "gf2x_ctx_destroy", "gf2x_mul", "gf2x_workspace_bytes",
                 "gf2x_stream_status", "gf2x_mul_host", "gf2x_basis_cvt", "gf2x_encode",
                 "gf2x_butterfly", "gf2x_pointwise", "gf2x_decode", "gf2x_ibutterfly", "gf2x_ibasis_cvt"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1803_11301_gb300 import ABI_FUNCTIONS
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in ABI_FUNCTIONS, f"binding does not marshal {name}"


def test_size_rules_match_the_oracle(lib):
    from paper_1803_11301_gb300 import transform_bits, workspace_bytes
    from oracle import stages as S
    for na, nb in [(1, 1), (33, 32), (33, 33), (1 << 16, 1 << 16), (1 << 24, 1 << 24), (1 << 30, 1 << 30),
                   (5, 1 << 20), (1 << 36, 1 << 36)]:
        n = S.transform_length(na, nb)
        assert transform_bits(na, nb) == n
        assert workspace_bytes(na, nb) == 3 * ((n // 8 + 255) // 256 * 256) + 256
    assert transform_bits(0, 5) == 0 and workspace_bytes(7, 0) == 0
    assert workspace_bytes(1 << 36, (1 << 36) + 2) == 0            # n = 2^38 > 2^37


def test_status_strings(lib):
    assert lib.gf2x_status_string(0) == b"GF2X_OK"
    assert lib.gf2x_status_string(2) == b"GF2X_ETOOBIG"


def test_null_context_rejected(lib):
    assert lib.gf2x_mul(None, None, 1, None, 1, None, None, 0, None) == 1      # EINVAL
    assert lib.gf2x_basis_cvt(None, None, 64, None) == 1
    assert lib.gf2x_ctx_create(None, 0) == 1
    assert lib.gf2x_tune_pin(None, 5, 9) == 1
    assert lib.gf2x_tune_freeze(None, 1) == 1


def test_knob_constants_match_the_header():
    import re
    from paper_1803_11301_gb300 import (KNOB_BATCH_PERSISTENT, KNOB_BOTTOM_DEPTH, KNOB_BOTTOM_MUL, KNOB_BOTTOM_SHAPE,
                                        KNOB_CVT_TAYLOR, KNOB_M128_BOTTOM_CHUNK, KNOB_M128_BOTTOM_DEPTH, KNOB_UNIT16_R,
                                        KNOB_WINDOW_DEPTH)
    text = open(HEADER).read()
    want = {k: int(v) for k, v in re.findall(r"GF2X_KNOB_(\w+) = (\d+)", text)}
    assert want == {"UNIT16_R": KNOB_UNIT16_R, "BOTTOM_SHAPE": KNOB_BOTTOM_SHAPE, "WINDOW_DEPTH": KNOB_WINDOW_DEPTH,
                    "M128_BOTTOM_CHUNK": KNOB_M128_BOTTOM_CHUNK, "BOTTOM_DEPTH": KNOB_BOTTOM_DEPTH,
                    "M128_BOTTOM_DEPTH": KNOB_M128_BOTTOM_DEPTH, "BATCH_PERSISTENT": KNOB_BATCH_PERSISTENT,
                    "BOTTOM_MUL": KNOB_BOTTOM_MUL, "CVT_TAYLOR": KNOB_CVT_TAYLOR}


def test_no_device_path_reports_enodev(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.gf2x_ctx_create(ctypes.byref(h), 0) == 6                      # ENODEV, no fallback


def test_m128_size_rules_match_the_oracle(lib):
    from paper_1803_11301_gb300 import m128_transform_bits, m128_workspace_bytes
    from oracle import m128 as G
    for na, nb in [(1, 1), (64, 65), (65, 65), (1 << 16, 1 << 16), (5, 1 << 20), (1 << 30, 1 << 30),
                   (1 << 37, 1 << 37)]:
        n = G.transform_length(na, nb)
        assert m128_transform_bits(na, nb) == n
        assert m128_workspace_bytes(na, nb) == 3 * ((n // 8 + 255) // 256 * 256) + 256
    assert m128_transform_bits(0, 5) == 0 and m128_workspace_bytes(7, 0) == 0
    assert m128_workspace_bytes(1 << 37, (1 << 37) + 2) == 0       # n = 2^39 > 2^38
    assert lib.gf2x_mul_m128(None, None, 1, None, 1, None, None, 0, None) == 1      # EINVAL


def _jobs(specs):
    """gf2x_job array from (a, na, b, nb, c) with integer addresses (never dereferenced here)."""
    from paper_1803_11301_gb300 import Job
    arr = (Job * len(specs))()
    for k, (a, na, b, nb, c) in enumerate(specs):
        arr[k] = Job(a, na, b, nb, c)
    return arr


def test_batch_workspace_rules(lib):
    # host-side planning of gf2x_mul_batch: a pure function of the job lengths,
    # room for every job's three transform buffers (a single product's
    # workspace less its 256 reserved bytes), 0 for an invalid job
    from paper_1803_11301_gb300 import workspace_bytes
    A, B, C = 1 << 32, 2 << 32, 3 << 32                       # disjoint, 8-byte aligned addresses
    lens = [(1000, 5000), (1 << 20, 1 << 20), (64, 64), (1 << 20, 77), (3, 70000)]
    specs = [(A + 2**24 * k, na, B + 2**24 * k, nb, C + 2**24 * k) for k, (na, nb) in enumerate(lens)]
    ws = lib.gf2x_batch_workspace_bytes(_jobs(specs), len(specs))
    assert ws >= sum(workspace_bytes(na, nb) - 256 for na, nb in lens) + 256
    moved = [(a + 4096, na, b + 8192, nb, c + 65536) for a, na, b, nb, c in specs]
    assert lib.gf2x_batch_workspace_bytes(_jobs(moved), len(moved)) == ws        # lengths only
    shuffled = [specs[k] for k in (3, 0, 4, 2, 1)]
    assert lib.gf2x_batch_workspace_bytes(_jobs(shuffled), len(shuffled)) == ws  # order-free
    with_empty = specs + [(A, 0, B, 100, C), (A, 100, B, 0, C)]
    assert lib.gf2x_batch_workspace_bytes(_jobs(with_empty), len(with_empty)) == ws
    one = lib.gf2x_batch_workspace_bytes(_jobs(specs[:1]), 1)
    assert workspace_bytes(1000, 5000) <= one < ws
    assert lib.gf2x_batch_workspace_bytes(_jobs([(A + 4, 1000, B, 5000, C)]), 1) == 0          # misaligned a
    assert lib.gf2x_batch_workspace_bytes(_jobs([(A, 1000, B, 5000, A + 8)]), 1) == 0          # c overlaps a
    assert lib.gf2x_batch_workspace_bytes(_jobs([(A, 1 << 36, B, (1 << 36) + 2, C)]), 1) == 0  # n > 2^37
    assert lib.gf2x_batch_workspace_bytes(None, 0) == lib.gf2x_batch_workspace_bytes(_jobs([]), 0)


def test_host_workspace_holds_the_staging_buffers(lib):
    # gf2x_mul_host stages pageable operands and the product in its workspace
    from paper_1803_11301_gb300 import host_workspace_bytes, workspace_bytes
    for na, nb in [(1, 1), (1000, 5000), (1 << 20, 77), (1 << 24, 1 << 24)]:
        words = (na + 63) // 64 + (nb + 63) // 64 + (na + nb - 1 + 63) // 64
        assert host_workspace_bytes(na, nb) >= workspace_bytes(na, nb) + 8 * words
    assert host_workspace_bytes(0, 9) == 0


def test_transform_workspace_rule(lib):
    # gf2x_forward_transform's workspace: what a product of that transform length needs
    from paper_1803_11301_gb300 import workspace_bytes
    for n in [64, 128, 1 << 17, 1 << 25, 1 << 37]:
        assert lib.gf2x_transform_workspace_bytes(n) == workspace_bytes(n // 2, n // 2)
        assert lib.gf2x_transform_bytes(n) == n // 8
    for bad in [0, 32, 96, 1000, 1 << 38]:
        assert lib.gf2x_transform_workspace_bytes(bad) == 0
