"""Host-side checks of the C ABI: the library builds, loads and exports every entry
point include/rdhei.h declares (no GPU needed: nothing is launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rdhei.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rdhei_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2302_07992_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_calls_and_the_fused_pair():
    names = _declared()
    for n in ("rdhei_label_encrypt", "rdhei_embed", "rdhei_extract", "rdhei_decrypt_recover", "rdhei_encode",
              "rdhei_decode"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_sizes_match_binding(lib):
    lib.rdhei_job_size.restype = ctypes.c_size_t
    lib.rdhei_info_size.restype = ctypes.c_size_t
    assert lib.rdhei_job_size() == 200
    assert lib.rdhei_info_size() == 72
    lib.rdhei_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.rdhei_version()


def test_host_validation_without_gpu(lib):
    """Argument checks happen on the host before any CUDA call."""
    class Job(ctypes.Structure):
        _fields_ = [("raw", ctypes.c_uint8 * 200)]
    j = Job()
    hdr = (ctypes.c_int32 * 6).from_buffer(j)
    info_ptr = ctypes.c_uint64.from_buffer(j, 192)
    buf = ctypes.create_string_buffer(128)
    info_ptr.value = (ctypes.addressof(buf) + 7) & ~7
    lib.rdhei_workspace_size.restype = ctypes.c_size_t
    lib.rdhei_workspace_size.argtypes = [ctypes.c_void_p, ctypes.c_int]
    for H, W, var, b, ok in [(512, 512, 0, 0, True), (0, 5, 0, 0, False), (5, 70000, 0, 0, False),
                             (20000, 20000, 0, 0, False), (8, 8, 4, 0, False), (8, 8, -1, 0, False),
                             (8, 8, 0, 8, False), (8, 8, 1, 8, True), (8, 8, 0, 1, False),
                             (8, 8, 2, 0, True), (8, 8, 3, 8, True), (8, 8, 2, 8, False)]:
        hdr[0], hdr[1], hdr[2], hdr[3], hdr[4], hdr[5] = H, W, var, b, 0, 1
        size = lib.rdhei_workspace_size(ctypes.addressof(j), 1)
        assert (size > 0) == ok, (H, W, var, b)
    # a 512 x 512 image needs at least its stash
    hdr[0], hdr[1], hdr[2], hdr[3] = 512, 512, 0, 0
    assert lib.rdhei_workspace_size(ctypes.addressof(j), 1) >= 512 * 512


def test_checked_build_exports_the_same_calls(lib):
    """The checked build (-DRDHEI_CHECK) exports every declared call and says so in
    rdhei_build_flags; the normal build carries no checks."""
    from paper_2302_07992_gb300 import build
    chk = ctypes.CDLL(build.build(checked=True))
    missing = [n for n in _declared() if not hasattr(chk, n)]
    assert not missing, missing
    assert chk.rdhei_build_flags() == 1
    assert lib.rdhei_build_flags() == 0

