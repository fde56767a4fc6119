"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports every symbol that
include/fio.h declares, and rejects damaged factor buffers before touching the GPU."""

import os
import re

import numpy as np
import pytest

from paper_2105_02995_gb300 import binding, build as fbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fbuild.build()
    return binding.load()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "fio.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(fio_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    syms = header_symbols()
    for name in ["fio_upload_factors", "fio_apply_K", "fio_apply_Kadj", "fio_apply_inv", "fio_solve"]:
        assert name in syms
    assert set(syms) == set(binding.SYMBOLS)


def test_library_exports_every_symbol(lib):
    for name in header_symbols():
        assert getattr(lib, name) is not None


def test_strerror(lib):
    assert lib.fio_strerror(0) == b"ok"
    assert b"damaged" in lib.fio_strerror(-3)


def _buf():
    from paper_2105_02995_gb300.builder import build_operator
    buf, _ = build_operator("ex1", 64, 1e-7, 1e-6, L=2, LH=1)
    return buf


@pytest.mark.parametrize("mutate", ["magic", "checksum", "truncate", "index"])
def test_upload_rejects_damaged_buffers(lib, mutate):
    import ctypes
    import struct
    buf = bytearray(_buf())
    if mutate == "magic":
        buf[0] = ord("X")
    elif mutate == "checksum":
        buf[-8] ^= 0xFF
    elif mutate == "truncate":
        buf = buf[:-256]
    elif mutate == "index":
        # point a butterfly stage's first input index outside its vector, then fix the checksum
        tab = struct.unpack_from("<Q", buf, 64)[0]
        off_in = struct.unpack_from("<Q", buf, tab + 40)[0]
        struct.pack_into("<i", buf, off_in, 1 << 30)
        from paper_2105_02995_gb300.builder.pack import checksum
        data, total = struct.unpack_from("<QQ", buf, 72)
        struct.pack_into("<Q", buf, 88, checksum(bytes(buf), data, total))
    h = ctypes.c_void_p()
    cbuf = ctypes.create_string_buffer(bytes(buf), len(buf))
    rc = lib.fio_upload_factors(cbuf, len(buf), 0, None, ctypes.byref(h))
    assert rc == -3  # FIO_EBADFACTORS, found before any CUDA call
    assert not h.value


def test_null_arguments(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.fio_upload_factors(None, 0, 0, None, ctypes.byref(h)) == -1
    assert lib.fio_apply_K(None, None, None, 1, 1, 0, 0, None) == -1
    assert lib.fio_release(None) == 0


def test_load_fails_loudly_without_library(tmp_path):
    with pytest.raises(OSError):
        binding._lib_backup = binding._lib
        try:
            binding._lib = None
            binding.load(str(tmp_path / "missing.so"))
        finally:
            binding._lib = binding._lib_backup
