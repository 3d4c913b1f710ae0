"""The C-ABI library loads and exports every symbol that include/rs.h declares
(no compute calls: CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def librs():
    import paper_1701_05913_gb300 as rs
    rs.build()
    return ctypes.CDLL(rs.LIB_PATH)


def test_header_symbols_exported(librs):
    names = _declared()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(librs, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_1701_05913_gb300 as rs
    bound = {n for n, _, _ in rs.SIGNATURES}
    assert set(_declared()) <= bound


def test_status_strings(librs):
    librs.rs_status_str.restype = ctypes.c_char_p
    assert librs.rs_status_str(0) == b"ok"
    assert b"pivot" in librs.rs_status_str(-3)
    assert b"timed out" in librs.rs_status_str(-5)
