"""Python binding of libpolymul.so: the C-ABI entry points under the same names.

Argument marshalling only.  Device buffers are torch CUDA tensors of 32-bit
words (torch.int32 or torch.uint32; the bits are the uint32 residues) or raw
integer device addresses; streams are torch.cuda.Stream objects, raw handles
or None (the current torch stream).  Every non-zero status raises
PolymulError.  There is no fallback: if libpolymul.so is missing or cannot be
loaded, lib() raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# POLYMUL_DEBUG_LIB=1 loads the debug build (range and index checks inside
# the kernels, reported by polymul_device_status) instead of the release one.
LIB_PATH = os.path.join(_HERE, "libpolymul_debug.so" if os.environ.get("POLYMUL_DEBUG_LIB") == "1"
                        else "libpolymul.so")
_lock = threading.Lock()
_lib = None

u32 = ctypes.c_uint32
i64 = ctypes.c_int64
vp = ctypes.c_void_p
I64P = ctypes.POINTER(ctypes.c_int64)
U32P = ctypes.POINTER(ctypes.c_uint32)


class PolymulError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: status {status} ({strerror(status)})" if what else f"status {status}")


_SIGS = {
    "polymul_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "polymul_version": (ctypes.c_char_p, []),
    "polymul_last_error": (ctypes.c_char_p, []),
    "polymul_device_status": (ctypes.c_int, [ctypes.c_int]),
    "polymul_set_validate": (ctypes.c_int, [ctypes.c_int]),
    "polymul_mod": (ctypes.c_int, [u32, vp, i64, vp, i64, vp]),
    "polymul_mod_async": (ctypes.c_int, [u32, vp, i64, vp, i64, vp, vp]),
    "polymul_mod_padded_async": (ctypes.c_int, [u32, vp, i64, vp, i64, vp, i64, vp]),
    "polymul_mod_host": (ctypes.c_int, [u32, vp, i64, vp, i64, vp]),
    "polymul_mod_host_async": (ctypes.c_int, [u32, vp, i64, vp, i64, vp, vp]),
    "polymul_mod_noalloc_async": (ctypes.c_int, [u32, vp, i64, vp, i64, vp, vp]),
    "polymul_profile_begin": (ctypes.c_int, []),
    "polymul_profile_end": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), I64P]),
    "polymul_probe_int": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]),
    "tft_plan_create": (ctypes.c_int, [u32, u32, i64, i64, ctypes.POINTER(vp)]),
    "tft_plan_length": (i64, [vp]),
    "tft_exec": (ctypes.c_int, [vp, vp, vp, vp]),
    "itft_exec": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp]),
    "tft_plan_destroy": (None, [vp]),
    "polymul_batch_create": (ctypes.c_int, [u32, i64, I64P, I64P, I64P, ctypes.POINTER(vp)]),
    "polymul_batch_exec": (ctypes.c_int, [vp, vp, vp, vp, vp]),
    "polymul_batch_exec_nograph": (ctypes.c_int, [vp, vp, vp, vp, vp]),
    "polymul_batch_status": (ctypes.c_int, [vp]),
    "polymul_batch_destroy": (None, [vp]),
    "polymul_batch_test_withhold": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_longlong]),
    "polymul_mod_batched": (ctypes.c_int, [u32, i64, vp, I64P, vp, I64P, vp, I64P, vp]),
    "polymul_mod_batched_plain": (ctypes.c_int, [u32, i64, vp, I64P, vp, I64P, vp, I64P, vp]),
    "polymul_autotune": (ctypes.c_int, [u32, ctypes.c_int, ctypes.c_int, ctypes.c_char_p]),
    "polymul_load_schedules": (ctypes.c_int, [ctypes.c_char_p]),
    "polymul_cyclic_async": (ctypes.c_int, [u32, vp, i64, vp, i64, vp, i64, vp]),
    "polymul_negacyclic_async": (ctypes.c_int, [u32, vp, i64, vp, i64, vp, i64, vp]),
    "polymul_crt3_async": (ctypes.c_int, [vp, i64, vp, i64, vp, vp]),
    "polymul_mod_radix_async": (ctypes.c_int, [u32, vp, i64, vp, i64, vp, ctypes.c_int, vp]),
    "polymul_get_schedule": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "polymul_get_batch_width": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "polymul_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]),
    "polymul_server_submit": (ctypes.c_int, [vp, u32, vp, i64, vp, i64, vp, ctypes.POINTER(ctypes.c_uint64)]),
    "polymul_server_poll": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
    "polymul_server_wait": (ctypes.c_int, [vp, ctypes.c_uint64, i64]),
    "polymul_server_stats": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double)]),
    "polymul_server_destroy": (ctypes.c_int, [vp]),
    "polymul_server_latency": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
}


def lib():
    """Load libpolymul.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_1609_01010_gb300.build` (nvcc, sm_103a)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)  # every entry point of include/polymul.h must be exported
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def polymul_device_status(clear: bool = False) -> int:
    """The current device's status word (0, POLY_ETIMEOUT or POLY_EINVAL_COEF)."""
    return int(lib().polymul_device_status(1 if clear else 0))


def polymul_set_validate(on: bool) -> None:
    """Validation mode: entry points check their inputs are below p first."""
    _check(lib().polymul_set_validate(1 if on else 0), "polymul_set_validate")


def strerror(status: int) -> str:
    try:
        return lib().polymul_strerror(status).decode()
    except Exception:  # noqa: BLE001 - only for messages
        return "?"


def _check(rc: int, what: str) -> None:
    if rc != 0:
        detail = lib().polymul_last_error().decode() if rc == -5 else ""
        raise PolymulError(rc, f"{what} {detail}".strip())


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):  # numpy array (host)
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(s) -> int | None:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _offsets(off):
    import numpy as np
    arr = np.ascontiguousarray(off, dtype=np.int64)
    return arr, arr.ctypes.data_as(I64P)


# ------------------------------------------------------------ single products
def polymul_mod(p: int, a, da: int, b, db: int, c) -> None:
    _check(lib().polymul_mod(p, _ptr(a), da, _ptr(b), db, _ptr(c)), "polymul_mod")


def polymul_mod_async(p: int, a, da: int, b, db: int, c, stream=None) -> None:
    _check(lib().polymul_mod_async(p, _ptr(a), da, _ptr(b), db, _ptr(c), _stream(stream)), "polymul_mod_async")


def polymul_mod_padded_async(p: int, a, da: int, b, db: int, c, Lp: int, stream=None) -> None:
    _check(lib().polymul_mod_padded_async(p, _ptr(a), da, _ptr(b), db, _ptr(c), Lp, _stream(stream)),
           "polymul_mod_padded_async")


def polymul_mod_noalloc_async(p: int, a, da: int, b, db: int, c, stream=None) -> None:
    """The allocation-free product (n <= 2^17; p = 469762049 or 2013265921)."""
    _check(lib().polymul_mod_noalloc_async(p, _ptr(a), da, _ptr(b), db, _ptr(c), _stream(stream)),
           "polymul_mod_noalloc_async")


def polymul_mod_host(p: int, a, da: int, b, db: int, c) -> None:
    """Host buffers (numpy uint32 arrays or pinned torch CPU tensors)."""
    _check(lib().polymul_mod_host(p, _ptr(a), da, _ptr(b), db, _ptr(c)), "polymul_mod_host")


def polymul_mod_host_async(p: int, a, da: int, b, db: int, c, stream=None) -> None:
    """Host buffers, enqueued on `stream`; they must stay valid until the stream passes the call."""
    _check(lib().polymul_mod_host_async(p, _ptr(a), da, _ptr(b), db, _ptr(c), _stream(stream)),
           "polymul_mod_host_async")


def polymul_profile_begin() -> None:
    _check(lib().polymul_profile_begin(), "polymul_profile_begin")


def polymul_profile_end() -> tuple[list[float], list[int]]:
    """(ms per kernel, launches per kernel) for [small, column TFT, rows, column ITFT]."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_int64 * 4)()
    _check(lib().polymul_profile_end(ms, n), "polymul_profile_end")
    return list(ms), list(n)


PROBE_KINDS = {0: "forward butterfly", 1: "inverse butterfly", 2: "mul.lo.u32", 3: "mul.hi.u32", 4: "add.u32",
               5: "min.u32"}


def polymul_probe_int(kind: int, iters: int = 1 << 14) -> tuple[float, float]:
    """(operations per second, ms of the timed launch) of integer probe `kind`."""
    ops = ctypes.c_double()
    ms = ctypes.c_double()
    _check(lib().polymul_probe_int(kind, iters, ctypes.byref(ops), ctypes.byref(ms)), "polymul_probe_int")
    return ops.value, ms.value


# ------------------------------------------------------------ TFT plans
def tft_plan_create(p: int, root: int, z: int, n: int) -> int:
    h = vp()
    _check(lib().tft_plan_create(p, root, z, n, ctypes.byref(h)), "tft_plan_create")
    return h.value


def tft_plan_length(plan: int) -> int:
    return lib().tft_plan_length(plan)


def tft_exec(plan: int, inp, out, stream=None) -> None:
    _check(lib().tft_exec(plan, _ptr(inp), _ptr(out), _stream(stream)), "tft_exec")


def itft_exec(plan: int, inp, out, scale: int = 1, stream=None) -> None:
    _check(lib().itft_exec(plan, _ptr(inp), _ptr(out), scale, _stream(stream)), "itft_exec")


def tft_plan_destroy(plan: int) -> None:
    lib().tft_plan_destroy(plan)


class TftPlan:
    """Owns a tft_plan handle (TFT(L, z, n) and ITFT(L, n, n))."""

    def __init__(self, p: int, z: int, n: int, root: int = 0):
        self.p, self.z, self.n = p, z, n
        self.handle = tft_plan_create(p, root, z, n)
        self.L = tft_plan_length(self.handle)

    def tft(self, inp, out, stream=None):
        tft_exec(self.handle, inp, out, stream)

    def itft(self, inp, out, scale: int = 1, stream=None):
        itft_exec(self.handle, inp, out, scale, stream)

    def close(self):
        if self.handle:
            tft_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


# ------------------------------------------------------------ batched
def polymul_batch_create(p: int, a_off, b_off, c_off) -> int:
    aa, ap = _offsets(a_off)
    bb, bp = _offsets(b_off)
    cc, cp = _offsets(c_off)
    h = vp()
    _check(lib().polymul_batch_create(p, len(aa) - 1, ap, bp, cp, ctypes.byref(h)), "polymul_batch_create")
    return h.value


def polymul_batch_exec(batch: int, a, b, c, stream=None) -> None:
    _check(lib().polymul_batch_exec(batch, _ptr(a), _ptr(b), _ptr(c), _stream(stream)), "polymul_batch_exec")


def polymul_batch_exec_nograph(batch: int, a, b, c, stream=None) -> None:
    _check(lib().polymul_batch_exec_nograph(batch, _ptr(a), _ptr(b), _ptr(c), _stream(stream)),
           "polymul_batch_exec_nograph")


def polymul_batch_status(batch: int) -> int:
    return lib().polymul_batch_status(batch)


def polymul_batch_destroy(batch: int) -> None:
    lib().polymul_batch_destroy(batch)


def polymul_batch_test_withhold(batch: int, kind: int, spin_limit: int) -> None:
    _check(lib().polymul_batch_test_withhold(batch, kind, spin_limit), "polymul_batch_test_withhold")


def polymul_mod_batched(p: int, a, a_off, b, b_off, c, c_off, stream=None) -> None:
    aa, ap = _offsets(a_off)
    bb, bp = _offsets(b_off)
    cc, cp = _offsets(c_off)
    _check(lib().polymul_mod_batched(p, len(aa) - 1, _ptr(a), ap, _ptr(b), bp, _ptr(c), cp, _stream(stream)),
           "polymul_mod_batched")


def polymul_mod_batched_plain(p: int, a, a_off, b, b_off, c, c_off, stream=None) -> None:
    aa, ap = _offsets(a_off)
    bb, bp = _offsets(b_off)
    cc, cp = _offsets(c_off)
    _check(lib().polymul_mod_batched_plain(p, len(aa) - 1, _ptr(a), ap, _ptr(b), bp, _ptr(c), cp,
                                           _stream(stream)), "polymul_mod_batched_plain")


# ------------------------------------------------------------ autotuner
def polymul_autotune(p: int, lo_log: int, hi_log: int, json_path: str | None = None) -> None:
    _check(lib().polymul_autotune(p, lo_log, hi_log, json_path.encode() if json_path else None), "polymul_autotune")


def polymul_load_schedules(json_path: str) -> None:
    _check(lib().polymul_load_schedules(json_path.encode()), "polymul_load_schedules")


# ------------------------------------------------------------ serving
def polymul_cyclic_async(p: int, a, za: int, b, zb: int, c, N: int, stream=None) -> None:
    """c (N words) = a * b mod (x^N - 1); za, zb are lengths (<= N)."""
    _check(lib().polymul_cyclic_async(p, _ptr(a), za, _ptr(b), zb, _ptr(c), N, _stream(stream)),
           "polymul_cyclic_async")


def polymul_negacyclic_async(p: int, a, za: int, b, zb: int, c, N: int, stream=None) -> None:
    """c (N words) = a * b mod (x^N + 1); za, zb are lengths (<= N)."""
    _check(lib().polymul_negacyclic_async(p, _ptr(a), za, _ptr(b), zb, _ptr(c), N, _stream(stream)),
           "polymul_negacyclic_async")


def polymul_crt3_async(a, da: int, b, db: int, c, stream=None) -> None:
    """c (3*(da+db+1) words) = a * b over the integers, 32-bit coefficients in,
    96-bit little-endian coefficients out (three primes and the CRT)."""
    _check(lib().polymul_crt3_async(_ptr(a), da, _ptr(b), db, _ptr(c), _stream(stream)), "polymul_crt3_async")


def polymul_mod_radix_async(p: int, a, da: int, b, db: int, c, m: int, stream=None) -> None:
    """c = a * b mod p through a transform length m 2^k (odd radix m)."""
    _check(lib().polymul_mod_radix_async(p, _ptr(a), da, _ptr(b), db, _ptr(c), m, _stream(stream)),
           "polymul_mod_radix_async")


def polymul_get_batch_width(l: int) -> int:
    """Column-tile width of a length-2^l product inside a batch."""
    c = ctypes.c_int()
    _check(lib().polymul_get_batch_width(l, ctypes.byref(c)), "polymul_get_batch_width")
    return c.value


def polymul_get_schedule(l: int) -> tuple[int, int]:
    """(sigma, C) of the three-kernel path for L = 2^l."""
    sg, c = ctypes.c_int(), ctypes.c_int()
    _check(lib().polymul_get_schedule(l, ctypes.byref(sg), ctypes.byref(c)), "polymul_get_schedule")
    return sg.value, c.value


SERVE_BATCH, SERVE_PLAIN = 0, 1


def polymul_server_create(mem_budget_bytes: int, n_streams: int = 4, mode: int = SERVE_BATCH) -> int:
    h = vp()
    _check(lib().polymul_server_create(mem_budget_bytes, n_streams, mode, ctypes.byref(h)), "polymul_server_create")
    return h.value


def polymul_server_submit(srv: int, p: int, a, da: int, b, db: int, c) -> int:
    t = ctypes.c_uint64()
    _check(lib().polymul_server_submit(srv, p, _ptr(a), da, _ptr(b), db, _ptr(c), ctypes.byref(t)),
           "polymul_server_submit")
    return t.value


def polymul_server_poll(srv: int, ticket: int) -> bool:
    done = ctypes.c_int()
    _check(lib().polymul_server_poll(srv, ticket, ctypes.byref(done)), "polymul_server_poll")
    return bool(done.value)


def polymul_server_wait(srv: int, ticket: int, timeout_ms: int = 60000) -> None:
    _check(lib().polymul_server_wait(srv, ticket, timeout_ms), "polymul_server_wait")


def polymul_server_latency(srv: int, ticket: int) -> float:
    """Microseconds from submit to completion of a done ticket."""
    us = ctypes.c_double()
    _check(lib().polymul_server_latency(srv, ticket, ctypes.byref(us)), "polymul_server_latency")
    return us.value


def polymul_server_stats(srv: int) -> dict:
    out = (ctypes.c_double * 6)()
    _check(lib().polymul_server_stats(srv, out), "polymul_server_stats")
    keys = ("count", "p50_us", "p90_us", "p99_us", "max_us", "mean_us")
    return dict(zip(keys, list(out)))


def polymul_server_destroy(srv: int) -> None:
    _check(lib().polymul_server_destroy(srv), "polymul_server_destroy")
