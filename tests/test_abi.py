"""The C-ABI library loads and exports every entry point include/wt.h declares.

No compute calls: this runs without a GPU.  It also checks host-side
argument validation paths that return before touching the device.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libwt():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2505_03372_gb300 import binding

    return binding.lib()


def _declared():
    with open(os.path.join(ROOT, "include", "wt.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(wt_[a-z_0-9]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(libwt):
    declared = _declared()
    assert {"wt_build", "wt_access", "wt_rank", "wt_select", "wt_destroy"} <= declared
    for name in sorted(declared):
        assert hasattr(libwt, name), f"{name} declared in include/wt.h but not exported by libwt.so"


def test_debug_library_exports_the_same_symbols(libwt):
    """libwt_debug.so (bounds-checked walk loads) is built beside libwt.so and
    exports every declared entry point too."""
    dbg = ctypes.CDLL(os.path.join(ROOT, "paper_2505_03372_gb300", "libwt_debug.so"))
    for name in sorted(_declared()):
        assert hasattr(dbg, name), f"{name} not exported by libwt_debug.so"
    dbg.wt_status_str.restype = ctypes.c_char_p
    assert dbg.wt_status_str(8).decode().startswith("WT_EBOUNDS")


def test_binding_lists_match_header(libwt):
    from paper_2505_03372_gb300 import binding

    assert set(binding.EXPORTED) == _declared()


def test_status_strings(libwt):
    from paper_2505_03372_gb300 import binding

    for s in range(9):
        assert binding.status_str(s).startswith("WT_")


def test_host_argument_validation(libwt):
    from paper_2505_03372_gb300 import binding

    h = ctypes.c_void_p()
    opt = binding.Options(sample_k=4096)
    # null out-pointer, bad widths, sigma 0 / too large: rejected before any device work
    assert libwt.wt_build(None, 0, 4, 1, ctypes.byref(opt), None, None) == binding.WT_EINVAL
    assert libwt.wt_build(None, 0, 4, 3, ctypes.byref(opt), None, ctypes.byref(h)) == binding.WT_EINVAL
    assert libwt.wt_build(None, 0, 0, 1, ctypes.byref(opt), None, ctypes.byref(h)) == binding.WT_EINVAL
    assert libwt.wt_build(None, 0, 257, 1, ctypes.byref(opt), None, ctypes.byref(h)) == binding.WT_EINVAL
    assert libwt.wt_build(None, 0, (1 << 26) + 1, 4, ctypes.byref(opt), None, ctypes.byref(h)) == binding.WT_EINVAL
    # the standalone bitvector queries reject an empty bitvector and null pointers
    assert libwt.wt_bitvector_rank(None, 0, None, None, None, None, 1, None, None) == binding.WT_EINVAL
    assert libwt.wt_bitvector_select(None, 0, 0, 1, None, None, None, None, 4096, None, None, 1, None,
                                     None) == binding.WT_EINVAL
    # the alphabet extraction rejects a null sigma pointer and a bad width
    assert libwt.wt_alphabet(None, 0, 1, None, None, None, None) == binding.WT_EINVAL
    sig = ctypes.c_uint32(7)
    assert libwt.wt_alphabet(None, 0, 3, None, None, ctypes.byref(sig), None) == binding.WT_EINVAL
    assert libwt.wt_alphabet(None, 0, 1, None, None, ctypes.byref(sig), None) == binding.WT_OK and sig.value == 0
    # the host-input build rejects a null out-pointer and a bad width
    assert libwt.wt_build_host(None, 0, 4, 1, ctypes.byref(opt), None, None) == binding.WT_EINVAL
    assert libwt.wt_build_host(None, 0, 4, 3, ctypes.byref(opt), None, ctypes.byref(h)) == binding.WT_EINVAL
    # the host query pipeline rejects a null tree before touching anything
    assert libwt.wt_query_host(None, 0, None, None, None, None, 1, 0, None) == binding.WT_EINVAL
    bad_k = binding.Options(sample_k=1000)
    assert libwt.wt_build(None, 0, 4, 1, ctypes.byref(bad_k), None, ctypes.byref(h)) == binding.WT_EINVAL
    # invalid handles
    assert libwt.wt_access(None, None, None, 1, None) == binding.WT_EINVAL
    assert libwt.wt_rank(None, None, None, None, 1, None) == binding.WT_EINVAL
    assert libwt.wt_select(None, None, None, None, 1, None) == binding.WT_EINVAL
    assert libwt.wt_status_sync(None, None) == binding.WT_EINVAL
    libwt.wt_destroy(None)  # no-op


def test_profile_api_without_gpu(libwt):
    from paper_2505_03372_gb300 import binding

    binding.profile_reset()
    assert binding.profile_launches() == 0
    assert binding.profile_report() == {}
