"""Python side of the C oracle (``oracle.c``) -- TEST INFRASTRUCTURE ONLY.

``mul``            the plain carry-less product (Sec. 2.1), Karatsuba in C.
``mul_bruteforce`` the same product from its definition, bit by bit (pins).
``modcheck``       c mod p == (a mod p)(b mod p) mod p for seeded irreducible
                   degree-64 p, for sizes the Karatsuba oracle cannot reach.
``eval_at``        A(beta) in GF(2^64) (Sec. 4.3 modulus).

``build()`` compiles ``oracle.c`` with gcc into ``oracle/_build``; nothing is
compiled at import time unless the library is missing.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle (portable C, OpenMP) and return the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER(ctypes.c_uint64)
            u64 = ctypes.c_uint64
            lib.oracle_clmul64.argtypes = [u64, u64, P, P]
            lib.oracle_clmul64.restype = None
            lib.oracle_mul.argtypes = [P, u64, P, u64, P]
            lib.oracle_mul.restype = ctypes.c_int
            lib.oracle_irreducible64.argtypes = [u64]
            lib.oracle_irreducible64.restype = ctypes.c_int
            lib.oracle_random_irreducibles.argtypes = [u64, ctypes.c_int, P]
            lib.oracle_random_irreducibles.restype = ctypes.c_int
            lib.oracle_modcheck.argtypes = [P, u64, P, u64, P, u64, P, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]
            lib.oracle_modcheck.restype = ctypes.c_int
            lib.oracle_eval_at.argtypes = [P, u64, u64]
            lib.oracle_eval_at.restype = u64
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(arr: np.ndarray):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _words(x: np.ndarray, nbits: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    need = (nbits + 63) // 64
    if x.size < need:
        raise ValueError(f"operand has {x.size} words, needs {need} for {nbits} bits")
    if x.size == 0:                       # ctypes wants a real buffer
        x = np.zeros(1, dtype=np.uint64)
    return x


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def product_bits(na: int, nb: int) -> int:
    return na + nb - 1 if (na and nb) else 0


def clmul64(a: int, b: int) -> tuple[int, int]:
    lo = ctypes.c_uint64()
    hi = ctypes.c_uint64()
    _load().oracle_clmul64(a, b, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def mul(a: np.ndarray, na: int, b: np.ndarray, nb: int) -> np.ndarray:
    """Carry-less product of the na-bit a and nb-bit b (uint64 little-endian words)."""
    a = _words(a, na)
    b = _words(b, nb)
    nc = product_bits(na, nb)
    c = np.zeros(max(1, (nc + 63) // 64), dtype=np.uint64)
    if _load().oracle_mul(_ptr(a), na, _ptr(b), nb, _ptr(c)) != 0:
        raise MemoryError("oracle_mul: out of memory")
    return c[: (nc + 63) // 64]


def mul_bruteforce(a: int, na: int, b: int, nb: int) -> int:
    """c_k = XOR_{i+j=k} a_i b_j, straight from the definition (Python ints)."""
    abits = [(a >> i) & 1 for i in range(na)]
    bbits = [(b >> j) & 1 for j in range(nb)]
    c = 0
    for i, ai in enumerate(abits):
        if not ai:
            continue
        for j, bj in enumerate(bbits):
            if bj:
                c ^= 1 << (i + j)
    return c


def irreducible64(low: int) -> bool:
    return bool(_load().oracle_irreducible64(low))


def random_irreducibles(seed: int, count: int) -> np.ndarray:
    lows = np.zeros(count, dtype=np.uint64)
    if _load().oracle_random_irreducibles(seed, count, _ptr(lows)) != 0:
        raise MemoryError("oracle_random_irreducibles")
    return lows


def modcheck(a, na, b, nb, c, nc, lows: np.ndarray) -> np.ndarray:
    """Boolean per modulus: c mod p == (a mod p)(b mod p) mod p."""
    a = _words(a, na)
    b = _words(b, nb)
    c = _words(c, nc)
    lows = np.ascontiguousarray(lows, dtype=np.uint64)
    ok = (ctypes.c_int * len(lows))()
    _load().oracle_modcheck(_ptr(a), na, _ptr(b), nb, _ptr(c), nc, _ptr(lows), len(lows), ok)
    return np.array(list(ok), dtype=bool)


def eval_at(a: np.ndarray, nbits: int, beta: int) -> int:
    """A(beta) in GF(2)[x]/(x^64+x^4+x^3+x+1)."""
    a = _words(a, nbits)
    return int(_load().oracle_eval_at(_ptr(a), nbits, beta))


# ---------------------------------------------------------------- int <-> words
def int_to_words(x: int, nbits: int) -> np.ndarray:
    nw = (nbits + 63) // 64
    return np.array([(x >> (64 * i)) & ((1 << 64) - 1) for i in range(nw)], dtype=np.uint64)


def words_to_int(w: np.ndarray) -> int:
    r = 0
    for i, v in enumerate(np.asarray(w, dtype=np.uint64).tolist()):
        r |= int(v) << (64 * i)
    return r
