"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/obk.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "obk.h")).read()
    return sorted(set(re.findall(r"^OBK_API\s+[\w\s\*]+?\b(obk_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__

    return __graft_entry__._build_module().build()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("obk_create", "obk_solve", "obk_submit", "obk_poll", "obk_destroy", "obk_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.obk_version.restype = ctypes.c_char_p
    lib.obk_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.obk_version()
    assert isinstance(lib.obk_last_error(), bytes)


def test_binding_names_match_header(libpath):
    import paper_2401_00672_gb300 as obk

    assert sorted(obk.EXPORTS) == _declared()


def test_invalid_arguments_rejected_before_any_device_work(libpath):
    import paper_2401_00672_gb300 as obk

    h = ctypes.c_void_p()
    assert obk.lib.obk_create(None, 3, 3, 0.1, ctypes.byref(h)) == obk.OBK_ERR_INVALID
    csr = obk._Csr(None, None, None, 0, 0)
    assert obk.lib.obk_create(ctypes.byref(csr), 0, 3, 0.1, ctypes.byref(h)) == obk.OBK_ERR_INVALID
    assert obk.lib.obk_create(ctypes.byref(csr), 3, 3, 1.5, ctypes.byref(h)) == obk.OBK_ERR_INVALID
    assert obk.lib.obk_poll(None, 1, None, None) == obk.OBK_ERR_INVALID


def test_request_footprint_host_only(libpath):
    """The request loop's HBM reservation: zero for invalid sizes, grows with
    the entries and with max(m, n), and covers at least the data it uploads."""
    import paper_2401_00672_gb300 as obk

    fp = obk.request_footprint
    assert fp(0, 5, 10) == 0 and fp(5, 0, 10) == 0 and fp(5, 5, -1) == 0
    base = fp(1000, 1000, 7000)
    assert base > 0
    assert fp(1000, 1000, 14000) > base  # more entries
    assert fp(2000, 1000, 7000) > base and fp(1000, 2000, 7000) > base  # extended systems
    assert fp(2000, 1000, 7000) == fp(1000, 2000, 7000)  # N = max(m, n) either way
    for m, n, nnz in ((1000, 1000, 7000), (400_000, 200_000, 4_000_000)):
        uploaded = (max(m, n) + 1) * 8 + nnz * (4 + 8) + max(m, n) * 16
        assert fp(m, n, nnz) >= uploaded
