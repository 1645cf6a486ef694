"""The C-ABI library loads and exports every entry point include/polymul.h
declares (no GPU and no compute call needed), and the host-side argument
checks that run before any CUDA call behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "polymul.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*([a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1609_01010_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("polymul_mod", "polymul_mod_async", "tft_plan_create", "tft_exec", "itft_exec",
                     "tft_plan_destroy", "polymul_mod_batched", "polymul_server_create",
                     "polymul_server_submit", "polymul_server_poll", "polymul_server_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_symbol(lib):
    from paper_1609_01010_gb300 import binding
    assert set(header_functions()) <= set(binding._SIGS)
    binding.lib()  # loads, sets every signature


def test_host_side_argument_checks(lib):
    """Checks that return before any CUDA call (null pointers, bad sizes)."""
    from paper_1609_01010_gb300 import binding as B
    L = B.lib()
    POLY_ENULL, POLY_EINVAL = -3, -7
    assert L.polymul_mod(469762049, None, 3, None, 3, None) == POLY_ENULL
    assert L.polymul_mod_async(469762049, 16, -1, 16, 3, 16, None) == POLY_EINVAL
    assert L.polymul_mod_padded_async(469762049, 16, 3, 16, 3, 16, 6, None) == POLY_EINVAL  # Lp not a power of 2
    assert L.polymul_mod_padded_async(469762049, 16, 3, 16, 3, 16, 4, None) == POLY_EINVAL  # Lp < n
    # exact integer product: checks precede any CUDA call
    assert L.polymul_crt3_async(None, 3, 16, 3, 16, None) == POLY_ENULL
    assert L.polymul_crt3_async(16, 3, 16, -2, 16, None) == POLY_EINVAL
    assert L.polymul_crt3_async(16, 1 << 23, 16, 1 << 23, 16, None) == -2  # n = 2^24 + 1: POLY_ETOO_LONG
    # general-radix product: radix checks precede any CUDA call
    assert L.polymul_mod_radix_async(2013265921, 16, 3, 16, 3, 16, 2, None) == POLY_EINVAL  # even radix
    assert L.polymul_mod_radix_async(2013265921, 16, 3, 16, 3, 16, 17, None) == POLY_EINVAL  # above 15
    assert L.polymul_mod_radix_async(2013265921, None, 3, 16, 3, 16, 3, None) == POLY_ENULL
    h = ctypes.c_void_p()
    assert L.tft_plan_create(469762049, 0, 0, 5, ctypes.byref(h)) == POLY_EINVAL
    assert L.tft_plan_create(469762049, 0, 6, 5, ctypes.byref(h)) == POLY_EINVAL
    srv = ctypes.c_void_p()
    assert L.polymul_server_create(1 << 20, 4, 2, ctypes.byref(srv)) == POLY_EINVAL  # unknown mode
    assert L.polymul_server_create(1 << 20, 0, 0, ctypes.byref(srv)) == POLY_EINVAL  # no stream
    assert L.polymul_server_create(0, 4, 0, ctypes.byref(srv)) == POLY_EINVAL  # no budget
    d1, d2 = ctypes.c_double(), ctypes.c_double()
    assert L.polymul_probe_int(6, 1000, ctypes.byref(d1), ctypes.byref(d2)) == POLY_EINVAL  # unknown kind
    assert L.polymul_probe_int(0, 0, ctypes.byref(d1), ctypes.byref(d2)) == POLY_EINVAL  # no iterations
    assert L.polymul_probe_int(0, 1000, None, ctypes.byref(d2)) == POLY_ENULL
    assert L.polymul_set_validate(0) == 0
    assert L.polymul_strerror(-10).decode().startswith("an input coefficient")
    assert L.polymul_strerror(-6).decode().startswith("a bounded wait")
    assert b"sm_103a" in L.polymul_version()


def test_schedule_and_batch_width_tables(lib):
    """Host-side tables, no CUDA call: every built-in schedule (sigma, C) of
    the three-kernel path is one the kernels take, and a batch's column-tile
    width is the widest of 8 .. 2048 whose T x C words fit the 64 KB item
    buffer (T = 2^(l - 12) rows of the batch's 4096-word rows)."""
    from paper_1609_01010_gb300 import binding as B
    L = B.lib()
    sig, C = ctypes.c_int(), ctypes.c_int()
    for l in range(10, 25):
        assert L.polymul_get_schedule(l, ctypes.byref(sig), ctypes.byref(C)) == 0
        t = l - sig.value
        assert 9 <= sig.value <= 13 and C.value in (8, 32, 128) and 1 <= t <= 11, (l, sig.value, C.value)
        # double-buffered tiles within 128 KB, except the TMA-fed 32-column tiles at t = 10
        assert (2 << t) * C.value * 4 <= 128 * 1024 or (C.value == 32 and t == 10), l
    assert L.polymul_get_schedule(9, ctypes.byref(sig), ctypes.byref(C)) == -7  # one-CTA sizes: no schedule
    widths = (8, 32, 128, 256, 512, 1024, 2048)
    for l in range(14, 23):
        assert L.polymul_get_batch_width(l, ctypes.byref(C)) == 0
        fits = [w for w in widths if (w << (l - 12)) * 4 <= 64 * 1024]
        assert C.value == max(fits), (l, C.value)
    assert L.polymul_get_batch_width(13, ctypes.byref(C)) == -7
    assert L.polymul_get_batch_width(14, None) == -3
