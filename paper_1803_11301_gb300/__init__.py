"""GF(2)[x] multiplication on GB300 by the Frobenius-partition additive FFT.

Thin Python binding over the C ABI in ``include/gf2x.h`` (library
``_build/libgf2x_gb300.so``).  This module only marshals arguments: every
step of the computation runs in the CUDA kernels behind the ABI.  PyTorch is
used for device memory and streams.  There is no CPU fallback: if the
library is missing or no GPU is usable, the calls raise.

Operands are packed bit-polynomials: ceil(nbits/64) 64-bit words (torch
int64 or uint64 tensors, bit patterns), bit t of word w = coefficient of
x^(64 w + t).
"""

from __future__ import annotations

import ctypes
import os

from .build import LIB as LIB_PATH, LIB_DEBUG as LIB_DEBUG_PATH

__all__ = ["Context", "Gf2xError", "PreparedBatch", "load_library", "transform_bits", "workspace_bytes",
           "host_workspace_bytes", "product_bits", "m128_transform_bits", "m128_workspace_bytes",
           "ABI_FUNCTIONS", "STATUS", "KNOB_UNIT16_R", "KNOB_BOTTOM_SHAPE", "KNOB_WINDOW_DEPTH",
           "KNOB_M128_BOTTOM_CHUNK", "KNOB_BOTTOM_DEPTH", "KNOB_M128_BOTTOM_DEPTH", "KNOB_BATCH_PERSISTENT", "KNOB_BOTTOM_MUL",
           "KNOB_CVT_TAYLOR"]

STATUS = {0: "GF2X_OK", 1: "GF2X_EINVAL", 2: "GF2X_ETOOBIG", 3: "GF2X_ENOMEM", 4: "GF2X_ECUDA",
          5: "GF2X_ETIMEOUT", 6: "GF2X_ENODEV", 7: "GF2X_ENOSPACE", 8: "GF2X_EBOUNDS"}

_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_SZ = ctypes.c_size_t
_ST = ctypes.c_int

# name -> (restype, argtypes); the functions declared in include/gf2x.h
ABI_FUNCTIONS = {
    "gf2x_status_string": (ctypes.c_char_p, [_ST]),
    "gf2x_ctx_create": (_ST, [ctypes.POINTER(_P), ctypes.c_int]),
    "gf2x_ctx_destroy": (None, [_P]),
    "gf2x_transform_bits": (_U64, [_U64, _U64]),
    "gf2x_workspace_bytes": (_SZ, [_U64, _U64]),
    "gf2x_mul": (_ST, [_P, _P, _U64, _P, _U64, _P, _P, _SZ, _P]),
    "gf2x_host_workspace_bytes": (_SZ, [_U64, _U64]),
    "gf2x_mul_host": (_ST, [_P, _P, _U64, _P, _U64, _P, _P, _SZ, _P]),
    "gf2x_mul_noalloc": (_ST, [_P, _P, _U64, _P, _U64, _P, _P]),
    "gf2x_transform_bytes": (_SZ, [_U64]),
    "gf2x_transform_workspace_bytes": (_SZ, [_U64]),
    "gf2x_forward_transform": (_ST, [_P, _P, _U64, _U64, _P, _P, _SZ, _P]),
    "gf2x_mul_transformed": (_ST, [_P, _P, _U64, _P, _U64, _P, _P, _SZ, _P]),
    "gf2x_batch_workspace_bytes": (_SZ, [_P, _SZ]),
    "gf2x_mul_batch": (_ST, [_P, _P, _SZ, _P, _SZ, _P]),
    "gf2x_stream_status": (_ST, [_P, _P]),
    "gf2x_selftest_wait_timeout": (_ST, [_P, _P]),
    "gf2x_selftest_queue_timeout": (_ST, [_P, _P]),
    "gf2x_basis_cvt": (_ST, [_P, _P, _U64, _P]),
    "gf2x_ibasis_cvt": (_ST, [_P, _P, _U64, _P]),
    "gf2x_encode": (_ST, [_P, _P, _U64, _P, _P]),
    "gf2x_decode": (_ST, [_P, _P, _U64, _P, _P]),
    "gf2x_butterfly": (_ST, [_P, _P, _U64, _P]),
    "gf2x_ibutterfly": (_ST, [_P, _P, _U64, _P]),
    "gf2x_pointwise": (_ST, [_P, _P, _P, _P, _U64, _P]),
    "gf2x_bottom_layers": (ctypes.c_int, [_P, _U64, _U64]),
    "gf2x_tune_freeze": (_ST, [_P, ctypes.c_int]),
    "gf2x_tune_pin": (_ST, [_P, ctypes.c_int, ctypes.c_int]),
    "gf2x_m128_transform_bits": (_U64, [_U64, _U64]),
    "gf2x_m128_bottom_layers": (ctypes.c_int, [_P, _U64, _U64]),
    "gf2x_m128_workspace_bytes": (_SZ, [_U64, _U64]),
    "gf2x_mul_m128": (_ST, [_P, _P, _U64, _P, _U64, _P, _P, _SZ, _P]),
    "gf2x_m128_encode": (_ST, [_P, _P, _U64, _P, _P]),
    "gf2x_m128_decode": (_ST, [_P, _P, _U64, _P, _P]),
    "gf2x_m128_butterfly": (_ST, [_P, _P, _U64, _P]),
    "gf2x_m128_ibutterfly": (_ST, [_P, _P, _U64, _P]),
    "gf2x_m128_pointwise": (_ST, [_P, _P, _P, _P, _U64, _P]),
    "gf2x_bench_field_mul": (_ST, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_U64),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_U64), _P]),
    "gf2x_stage_count": (ctypes.c_int, []),
    "gf2x_stage_name": (ctypes.c_char_p, [ctypes.c_int]),
    "gf2x_profile_enable": (_ST, [_P, ctypes.c_int]),
    "gf2x_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_U64), ctypes.c_int]),
}

_lib = None


# Launch knobs of Context.tune_pin (the GF2X_KNOB_* constants of include/gf2x.h)
# and their candidates.
KNOB_UNIT16_R = 1              # 8, 16, 32
KNOB_BOTTOM_SHAPE = 2          # 0, 1, 2
KNOB_WINDOW_DEPTH = 3          # 6, 7, 8
KNOB_M128_BOTTOM_CHUNK = 4     # 4, 8
KNOB_BOTTOM_DEPTH = 5          # 8 .. 11
KNOB_M128_BOTTOM_DEPTH = 6     # 8 .. 10
KNOB_BATCH_PERSISTENT = 7      # 1 (one persistent launch per batch), 0 (launches per kernel and size class)
KNOB_BOTTOM_MUL = 8            # 0 (16-bit integer product form), 1 (32-bit form) in the fused bottom kernel
KNOB_CVT_TAYLOR = 9            # BasisCvt's Taylor part at 2^25..2^32 bits: 1 (two superset-sum passes), 0 (division steps)


class Job(ctypes.Structure):
    """gf2x_job: one product of a batch (device pointers and bit lengths)."""
    _fields_ = [("a", ctypes.c_void_p), ("na_bits", ctypes.c_uint64), ("b", ctypes.c_void_p),
                ("nb_bits", ctypes.c_uint64), ("c", ctypes.c_void_p)]


class PreparedBatch:
    """A job list marshalled for gf2x_mul_batch (see Context.prepare_batch)."""

    def __init__(self, arr, count: int, workspace_bytes: int, outs, jobs):
        self.arr = arr
        self.count = count
        self.workspace_bytes = workspace_bytes
        self.outs = outs
        self.jobs = jobs            # keeps the tensors the array points to alive


class Gf2xError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


def load_library() -> ctypes.CDLL:
    """Load libgf2x_gb300.so (built by ``paper_1803_11301_gb300.build``); raise if absent.
    With GF2X_DEBUG_BOUNDS=1 in the environment, the range-checking build instead."""
    global _lib
    if _lib is None:
        path = LIB_DEBUG_PATH if os.environ.get("GF2X_DEBUG_BOUNDS") == "1" else LIB_PATH
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run `python -m paper_1803_11301_gb300.build` "
                              "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in ABI_FUNCTIONS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int, what: str):
    if status != 0:
        raise Gf2xError(status, what)


def product_bits(na: int, nb: int) -> int:
    return na + nb - 1 if (na and nb) else 0


def transform_bits(na: int, nb: int) -> int:
    return int(load_library().gf2x_transform_bits(na, nb))


def workspace_bytes(na: int, nb: int) -> int:
    return int(load_library().gf2x_workspace_bytes(na, nb))


def host_workspace_bytes(na: int, nb: int) -> int:
    return int(load_library().gf2x_host_workspace_bytes(na, nb))


def m128_transform_bits(na: int, nb: int) -> int:
    return int(load_library().gf2x_m128_transform_bits(na, nb))


def m128_workspace_bytes(na: int, nb: int) -> int:
    return int(load_library().gf2x_m128_workspace_bytes(na, nb))


def _words(nbits: int) -> int:
    return (nbits + 63) // 64


class Context:
    """A gf2x context on one CUDA device (constant tables resident in HBM)."""

    def __init__(self, device: int = 0):
        self._lib = load_library()
        self.device = device
        h = ctypes.c_void_p()
        _check(self._lib.gf2x_ctx_create(ctypes.byref(h), device), "gf2x_ctx_create")
        self._h = h
        self._ws = None
        self._allocator = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gf2x_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def _stream(self, stream):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))

    def _dev(self):
        import torch
        return torch.device("cuda", self.device)

    def _tensor_ptr(self, t, min_words: int, name: str):
        import torch
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype not in (torch.int64, torch.uint64) or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous int64/uint64 tensor of words")
        if t.numel() < min_words:
            raise ValueError(f"{name} has {t.numel()} words, needs {min_words}")
        return ctypes.c_void_p(t.data_ptr())

    def empty_words(self, count: int):
        import torch
        return torch.empty(max(count, 1), dtype=torch.int64, device=self._dev())[:count]

    def set_allocator(self, allocator=None):
        """Workspaces the calls allocate come from allocator(nbytes) -> a CUDA uint8 tensor, or
        None when it cannot (the call then raises GF2X_ENOMEM and enqueues nothing); None
        restores torch's allocator."""
        self._allocator = allocator
        self._ws = None

    def workspace(self, nbytes: int):
        """A cached device workspace of at least nbytes (256-byte aligned)."""
        import torch
        if self._ws is None or self._ws.numel() < nbytes:
            if self._allocator is not None:
                ws = self._allocator(max(nbytes, 256))
                if ws is None:
                    raise Gf2xError(3, "workspace allocation")
            else:
                ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self._dev())
            if ws.data_ptr() % 256:
                raise RuntimeError("workspace allocation is not 256-byte aligned")
            self._ws = ws
        return self._ws

    # --------------------------------------------------------- the product
    def mul(self, a, na: int, b, nb: int, out=None, workspace=None, stream=None):
        """c = a * b (Alg. 5) on the GPU; returns the ceil(nc/64)-word tensor c."""
        nc = product_bits(na, nb)
        if out is None:
            out = self.empty_words(_words(nc))
        if nc == 0:
            return out
        need = workspace_bytes(na, nb)
        if workspace is None:
            workspace = self.workspace(need)
        _check(self._lib.gf2x_mul(self._h, self._tensor_ptr(a, _words(na), "a"), na,
                                  self._tensor_ptr(b, _words(nb), "b"), nb,
                                  self._tensor_ptr(out, _words(nc), "out"),
                                  ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                  self._stream(stream)), "gf2x_mul")
        return out

    def mul_m128(self, a, na: int, b, nb: int, out=None, workspace=None, stream=None):
        """c = a * b by Alg. 5 with m = 128 (GF(2^128) points); same result as ``mul``."""
        nc = product_bits(na, nb)
        if out is None:
            out = self.empty_words(_words(nc))
        if nc == 0:
            return out
        need = m128_workspace_bytes(na, nb)
        if workspace is None:
            workspace = self.workspace(need)
        _check(self._lib.gf2x_mul_m128(self._h, self._tensor_ptr(a, _words(na), "a"), na,
                                       self._tensor_ptr(b, _words(nb), "b"), nb,
                                       self._tensor_ptr(out, _words(nc), "out"),
                                       ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                       self._stream(stream)), "gf2x_mul_m128")
        return out

    def tune_freeze(self, frozen: bool = True):
        """Stop (or resume) measuring launch shapes on first use; stored choices stay."""
        _check(self._lib.gf2x_tune_freeze(self._h, 1 if frozen else 0), "gf2x_tune_freeze")

    def tune_pin(self, knob: int, choice: int):
        """Use `choice` for launch knob `knob` (KNOB_*) wherever it is a candidate; -1 releases it."""
        _check(self._lib.gf2x_tune_pin(self._h, int(knob), int(choice)), "gf2x_tune_pin")

    def bottom_layers(self, na: int, nb: int, field: int = 64) -> int:
        """Butterfly layers of an na x nb product done by the fused low-layer kernel."""
        fn = self._lib.gf2x_m128_bottom_layers if field == 128 else self._lib.gf2x_bottom_layers
        return int(fn(self._h, na, nb))

    def forward_transform(self, b, nb: int, n: int, out=None, workspace=None, stream=None):
        """The transform of b (the BasisCvt, Encode and Butterfly steps of Alg. 5) at transform length n, for reuse."""
        if out is None:
            out = self.empty_words(n // 64)
        need = int(self._lib.gf2x_transform_workspace_bytes(n))
        if need == 0:
            raise Gf2xError(1, "gf2x_transform_workspace_bytes")
        if workspace is None:
            workspace = self.workspace(need)
        _check(self._lib.gf2x_forward_transform(self._h, self._tensor_ptr(b, _words(nb), "b"), nb, n,
                                                self._tensor_ptr(out, n // 64, "out"),
                                                ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                                self._stream(stream)), "gf2x_forward_transform")
        return out

    def mul_transformed(self, a, na: int, bhat, nb: int, out=None, workspace=None, stream=None):
        """c = a * b with b given as its transform bhat at transform_bits(na, nb)."""
        nc = product_bits(na, nb)
        if out is None:
            out = self.empty_words(_words(nc))
        if nc == 0:
            return out
        need = workspace_bytes(na, nb)
        if workspace is None:
            workspace = self.workspace(need)
        _check(self._lib.gf2x_mul_transformed(self._h, self._tensor_ptr(a, _words(na), "a"), na,
                                              self._tensor_ptr(bhat, transform_bits(na, nb) // 64, "bhat"), nb,
                                              self._tensor_ptr(out, _words(nc), "out"),
                                              ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                              self._stream(stream)), "gf2x_mul_transformed")
        return out

    def mul_host(self, a, na: int, b, nb: int, out=None, workspace=None, stream=None):
        """The product with host (numpy uint64) operands and result, through gf2x_mul_host."""
        import numpy as np
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        nc = product_bits(na, nb)
        if out is None:
            out = np.zeros(_words(nc), dtype=np.uint64)
        if nc == 0:
            return out
        if a.size < _words(na) or b.size < _words(nb) or out.size < _words(nc):
            raise ValueError("host buffer too small")
        need = host_workspace_bytes(na, nb)
        if workspace is None:
            workspace = self.workspace(need)
        _check(self._lib.gf2x_mul_host(self._h, ctypes.c_void_p(a.ctypes.data), na,
                                       ctypes.c_void_p(b.ctypes.data), nb, ctypes.c_void_p(out.ctypes.data),
                                       ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                       self._stream(stream)), "gf2x_mul_host")
        return out

    def profile_enable(self, enable: bool = True):
        """Reset stage times and launch counts; time every later stage with CUDA events if enable."""
        _check(self._lib.gf2x_profile_enable(self._h, 1 if enable else 0), "gf2x_profile_enable")

    def profile_read(self) -> dict:
        """{stage name: (milliseconds, kernel launches)} accumulated since profile_enable."""
        n = self._lib.gf2x_stage_count()
        ms = (ctypes.c_double * n)()
        la = (_U64 * n)()
        self._lib.gf2x_profile_read(self._h, ms, la, n)
        return {self._lib.gf2x_stage_name(k).decode(): (ms[k], int(la[k])) for k in range(n)}

    FIELD_VARIANTS = ("int", "int_const", "tab4", "tab8", "hybrid", "int16", "bitslice")

    def bench_field_mul(self, variant: int, steps: int, stream=None) -> dict:
        """Time one GF(2^64) product form (gf2x_bench_field_mul): checksum, ms, products."""
        cs, ms, pr = _U64(), ctypes.c_double(), _U64()
        _check(self._lib.gf2x_bench_field_mul(self._h, int(variant), int(steps), ctypes.byref(cs), ctypes.byref(ms),
                                              ctypes.byref(pr), self._stream(stream)), "gf2x_bench_field_mul")
        return {"variant": self.FIELD_VARIANTS[variant], "checksum": int(cs.value), "ms": ms.value,
                "products": int(pr.value)}

    def selftest_queue_timeout(self, stream=None):
        """Launch a persistent-batch queue whose wait must run out; the status word then reads GF2X_ETIMEOUT."""
        _check(self._lib.gf2x_selftest_queue_timeout(self._h, self._stream(stream)), "gf2x_selftest_queue_timeout")

    def selftest_wait_timeout(self, stream=None):
        """Launch a bounded wait that must run out; the status word then reads GF2X_ETIMEOUT."""
        _check(self._lib.gf2x_selftest_wait_timeout(self._h, self._stream(stream)), "gf2x_selftest_wait_timeout")

    def prepare_batch(self, jobs) -> "PreparedBatch":
        """Marshal a job list once (the gf2x_job array and its workspace size) for repeated calls."""
        arr = (Job * len(jobs))()
        for k, (a, na, b, nb, c) in enumerate(jobs):
            nc = product_bits(na, nb)
            arr[k] = Job(self._tensor_ptr(a, _words(na), "a").value if na else a.data_ptr(), na,
                         self._tensor_ptr(b, _words(nb), "b").value if nb else b.data_ptr(), nb,
                         self._tensor_ptr(c, _words(nc), "c").value if nc else c.data_ptr())
        need = int(self._lib.gf2x_batch_workspace_bytes(arr, len(jobs)))
        if need == 0 and len(jobs):
            raise Gf2xError(1, "gf2x_batch_workspace_bytes")
        return PreparedBatch(arr, len(jobs), need, [j[4] for j in jobs], list(jobs))

    def mul_batch(self, jobs, workspace=None, stream=None):
        """Run many products in one call.  jobs: a list of (a, na, b, nb, c) with CUDA tensors, or
        a PreparedBatch (the same list marshalled once by prepare_batch; its tensors must stay alive)."""
        pb = jobs if isinstance(jobs, PreparedBatch) else self.prepare_batch(jobs)
        if workspace is None:
            workspace = self.workspace(pb.workspace_bytes)
        _check(self._lib.gf2x_mul_batch(self._h, pb.arr, pb.count, ctypes.c_void_p(workspace.data_ptr()),
                                        workspace.numel(), self._stream(stream)), "gf2x_mul_batch")
        return pb.outs

    def batch_workspace_bytes(self, jobs) -> int:
        arr = (Job * len(jobs))()
        for k, (a, na, b, nb, c) in enumerate(jobs):
            arr[k] = Job(a.data_ptr(), na, b.data_ptr(), nb, c.data_ptr())
        return int(self._lib.gf2x_batch_workspace_bytes(arr, len(jobs)))

    def stream_status(self, stream=None) -> int:
        return int(self._lib.gf2x_stream_status(self._h, self._stream(stream)))

    # -------------------------------------------------------------- stages
    def basis_cvt(self, bits, L: int, stream=None, inverse: bool = False):
        fn = self._lib.gf2x_ibasis_cvt if inverse else self._lib.gf2x_basis_cvt
        _check(fn(self._h, self._tensor_ptr(bits, L // 64, "bits"), L, self._stream(stream)),
               "gf2x_ibasis_cvt" if inverse else "gf2x_basis_cvt")
        return bits

    def ibasis_cvt(self, bits, L: int, stream=None):
        return self.basis_cvt(bits, L, stream, inverse=True)

    def encode(self, novel, n: int, out=None, stream=None):
        if out is None:
            out = self.empty_words(n // 64)
        _check(self._lib.gf2x_encode(self._h, self._tensor_ptr(novel, n // 64, "novel"), n,
                                     self._tensor_ptr(out, n // 64, "out"), self._stream(stream)), "gf2x_encode")
        return out

    def decode(self, h, n: int, out=None, stream=None):
        if out is None:
            out = self.empty_words(n // 64)
        _check(self._lib.gf2x_decode(self._h, self._tensor_ptr(h, n // 64, "h"), n,
                                     self._tensor_ptr(out, n // 64, "out"), self._stream(stream)), "gf2x_decode")
        return out

    def butterfly(self, f, n: int, stream=None, inverse: bool = False):
        fn = self._lib.gf2x_ibutterfly if inverse else self._lib.gf2x_butterfly
        _check(fn(self._h, self._tensor_ptr(f, n // 64, "f"), n, self._stream(stream)),
               "gf2x_ibutterfly" if inverse else "gf2x_butterfly")
        return f

    def ibutterfly(self, f, n: int, stream=None):
        return self.butterfly(f, n, stream, inverse=True)

    def pointwise(self, a, b, out=None, stream=None):
        count = a.numel()
        if out is None:
            out = self.empty_words(count)
        _check(self._lib.gf2x_pointwise(self._h, self._tensor_ptr(a, count, "a"), self._tensor_ptr(b, count, "b"),
                                        self._tensor_ptr(out, count, "out"), count, self._stream(stream)),
               "gf2x_pointwise")
        return out

    # ------------------------------------------------------ stages, m = 128
    # Element vectors hold two words per GF(2^128) point (low word first).
    def m128_encode(self, novel, n: int, out=None, stream=None):
        if out is None:
            out = self.empty_words(n // 64)
        _check(self._lib.gf2x_m128_encode(self._h, self._tensor_ptr(novel, n // 64, "novel"), n,
                                          self._tensor_ptr(out, n // 64, "out"), self._stream(stream)),
               "gf2x_m128_encode")
        return out

    def m128_decode(self, h, n: int, out=None, stream=None):
        if out is None:
            out = self.empty_words(n // 64)
        _check(self._lib.gf2x_m128_decode(self._h, self._tensor_ptr(h, n // 64, "h"), n,
                                          self._tensor_ptr(out, n // 64, "out"), self._stream(stream)),
               "gf2x_m128_decode")
        return out

    def m128_butterfly(self, f, n: int, stream=None, inverse: bool = False):
        fn = self._lib.gf2x_m128_ibutterfly if inverse else self._lib.gf2x_m128_butterfly
        _check(fn(self._h, self._tensor_ptr(f, n // 64, "f"), n, self._stream(stream)),
               "gf2x_m128_ibutterfly" if inverse else "gf2x_m128_butterfly")
        return f

    def m128_ibutterfly(self, f, n: int, stream=None):
        return self.m128_butterfly(f, n, stream, inverse=True)

    def m128_pointwise(self, a, b, out=None, stream=None):
        count = a.numel() // 2
        if out is None:
            out = self.empty_words(2 * count)
        _check(self._lib.gf2x_m128_pointwise(self._h, self._tensor_ptr(a, 2 * count, "a"),
                                             self._tensor_ptr(b, 2 * count, "b"),
                                             self._tensor_ptr(out, 2 * count, "out"), count, self._stream(stream)),
               "gf2x_m128_pointwise")
        return out
