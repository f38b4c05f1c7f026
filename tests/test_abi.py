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
    from paper_1803_11301_gb300 import (KNOB_BOTTOM_DEPTH, KNOB_BOTTOM_SHAPE, KNOB_M128_BOTTOM_CHUNK,
                                        KNOB_M128_BOTTOM_DEPTH, KNOB_UNIT16_R, KNOB_WINDOW_DEPTH)
    text = open(HEADER).read()
    want = {k: int(v) for k, v in re.findall(r"GF2X_KNOB_(\w+) = (\d+)", text)}
    assert want == {"UNIT16_R": KNOB_UNIT16_R, "BOTTOM_SHAPE": KNOB_BOTTOM_SHAPE, "WINDOW_DEPTH": KNOB_WINDOW_DEPTH,
                    "M128_BOTTOM_CHUNK": KNOB_M128_BOTTOM_CHUNK, "BOTTOM_DEPTH": KNOB_BOTTOM_DEPTH,
                    "M128_BOTTOM_DEPTH": KNOB_M128_BOTTOM_DEPTH}


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
