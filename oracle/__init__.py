"""CPU oracle for polynomial multiplication over Z/pZ (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may
import this package.  The CUDA library never loads it, and it shares no code
with the GPU path: ``polymul_oracle.c`` is plain C with a 64-bit ``%`` after
every product, and ``brute.py`` is pure Python used to pin it.

``build()`` compiles polymul_oracle.c with gcc into liboracle.so next to it;
``lib()`` loads it (building on first use).  The wrappers below take and
return numpy uint32 arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polymul_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

U32P = ctypes.POINTER(ctypes.c_uint32)
I64P = ctypes.POINTER(ctypes.c_int64)
u32 = ctypes.c_uint32
u64 = ctypes.c_uint64


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, no architecture-specific flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            L.or_powmod.restype = u32
            L.or_powmod.argtypes = [u32, u64, u32]
            L.or_invmod.restype = u32
            L.or_invmod.argtypes = [u32, u32]
            L.or_root_of_unity.restype = u32
            L.or_root_of_unity.argtypes = [u32, u32, u64]
            L.or_schoolbook.restype = None
            L.or_schoolbook.argtypes = [u32, U32P, u64, U32P, u64, U32P]
            L.or_tft.restype = ctypes.c_int
            L.or_tft.argtypes = [u32, u32, u64, U32P, u64, u64, U32P]
            L.or_itft.restype = ctypes.c_int
            L.or_itft.argtypes = [u32, u32, u64, U32P, u64, ctypes.c_int, U32P]
            L.or_polymul_tft.restype = ctypes.c_int
            L.or_polymul_tft.argtypes = [u32, u32, U32P, u64, U32P, u64, U32P]
            L.or_polymul_ntt.restype = ctypes.c_int
            L.or_polymul_ntt.argtypes = [u32, u32, U32P, u64, U32P, u64, u64, U32P]
            L.or_cyclic.restype = None
            L.or_cyclic.argtypes = [u32, U32P, U32P, u64, U32P]
            L.or_negacyclic.restype = None
            L.or_negacyclic.argtypes = [u32, U32P, U32P, u64, U32P]
            L.or_polymul_tft_batch.restype = ctypes.c_int
            L.or_polymul_tft_batch.argtypes = [u32, u32, u64, U32P, I64P, U32P, I64P, U32P, I64P]
            L.or_set_fault.restype = None
            L.or_set_fault.argtypes = [ctypes.c_int]
            L.or_get_butterflies.restype = u64
            L.or_reset_butterflies.restype = None
            _lib = L
    return _lib


# Primitive roots of the two primes the workloads use (checked in the tests
# against the factorisation of p-1).
PRIMITIVE_ROOT = {469762049: 3, 2013265921: 31}


def _u32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint32))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(U32P)


def root_for(p: int, root: int | None) -> int:
    return PRIMITIVE_ROOT[p] if root is None else root


def schoolbook(p: int, a, b) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    c = np.zeros(len(a) + len(b) - 1, dtype=np.uint32)
    lib().or_schoolbook(p, _ptr(a), len(a), _ptr(b), len(b), _ptr(c))
    return c


def polymul_tft(p: int, a, b, root: int | None = None) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    c = np.zeros(len(a) + len(b) - 1, dtype=np.uint32)
    rc = lib().or_polymul_tft(p, root_for(p, root), _ptr(a), len(a), _ptr(b), len(b), _ptr(c))
    if rc:
        raise ValueError(f"or_polymul_tft failed: {rc}")
    return c


def polymul_ntt(p: int, a, b, Lp: int, root: int | None = None) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    c = np.zeros(len(a) + len(b) - 1, dtype=np.uint32)
    rc = lib().or_polymul_ntt(p, root_for(p, root), _ptr(a), len(a), _ptr(b), len(b), Lp, _ptr(c))
    if rc:
        raise ValueError(f"or_polymul_ntt failed: {rc}")
    return c


def tft(p: int, L: int, g, n: int, root: int | None = None) -> np.ndarray:
    g = _u32(g)
    out = np.zeros(n, dtype=np.uint32)
    rc = lib().or_tft(p, root_for(p, root), L, _ptr(g), len(g), n, _ptr(out))
    if rc:
        raise ValueError(f"or_tft failed: {rc}")
    return out


def itft(p: int, L: int, x, paper_scale: bool = False, root: int | None = None) -> np.ndarray:
    x = _u32(x)
    out = np.zeros(len(x), dtype=np.uint32)
    rc = lib().or_itft(p, root_for(p, root), L, _ptr(x), len(x), int(paper_scale), _ptr(out))
    if rc:
        raise ValueError(f"or_itft failed: {rc}")
    return out


def cyclic(p: int, u, v) -> np.ndarray:
    u, v = _u32(u), _u32(v)
    out = np.zeros(len(u), dtype=np.uint32)
    lib().or_cyclic(p, _ptr(u), _ptr(v), len(u), _ptr(out))
    return out


def negacyclic(p: int, u, v) -> np.ndarray:
    u, v = _u32(u), _u32(v)
    out = np.zeros(len(u), dtype=np.uint32)
    lib().or_negacyclic(p, _ptr(u), _ptr(v), len(u), _ptr(out))
    return out


def polymul_tft_batch(p: int, a, a_off, b, b_off, c_off, root: int | None = None) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    b_off = np.ascontiguousarray(b_off, dtype=np.int64)
    c_off = np.ascontiguousarray(c_off, dtype=np.int64)
    c = np.zeros(int(c_off[-1]), dtype=np.uint32)
    rc = lib().or_polymul_tft_batch(p, root_for(p, root), len(a_off) - 1, _ptr(a), a_off.ctypes.data_as(I64P),
                                    _ptr(b), b_off.ctypes.data_as(I64P), _ptr(c), c_off.ctypes.data_as(I64P))
    if rc:
        raise ValueError(f"or_polymul_tft_batch failed: {rc}")
    return c


def set_fault(mode: int) -> None:
    """Plant a known mistake in the oracle (tests prove the pins catch it)."""
    lib().or_set_fault(mode)


def butterflies() -> int:
    return int(lib().or_get_butterflies())


def reset_butterflies() -> None:
    lib().or_reset_butterflies()
