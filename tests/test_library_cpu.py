"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads and exports
every entry point that include/cox.h declares; the binding's structs match the header."""
from __future__ import annotations

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "cox.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"^\s*(?:int|int64_t|void|const char \*)\s*\*?\s*(cox_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2310_16238_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    L = C.CDLL(libpath)
    declared = _declared()
    assert len(declared) >= 14
    missing = [n for n in declared if not hasattr(L, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2310_16238_gb300 import cox
    assert set(_declared()) <= set(cox.EXPORTS) | {"cox_set_allocator"}


def test_struct_layouts_match_header():
    from paper_2310_16238_gb300 import cox
    # int64 + 2*int32 + 7 pointers
    assert C.sizeof(cox.cox_data) == 8 + 8 + 7 * 8
    # 2*int32, 2 doubles, ptr, double, 2*int32, ptr
    assert C.sizeof(cox.cox_options) == 8 + 16 + 8 + 8 + 8 + 8 + 8
    assert C.sizeof(cox.cox_fit_info) == 8 + 8 + 16 + 8 + 16 + 16
    assert C.sizeof(cox.cox_server_options) == 8 + 16
    assert C.sizeof(cox.cox_server_stats) == 24 + 16 + 16 + 16


def test_no_cpu_fallback_without_library(monkeypatch, tmp_path):
    from paper_2310_16238_gb300 import cox
    monkeypatch.setattr(cox, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(cox, "_lib", None)
    with pytest.raises(RuntimeError):
        cox.lib()


def test_last_error_without_gpu(libpath):
    """Entry points validate arguments on the host before touching the device."""
    from paper_2310_16238_gb300 import cox
    L = cox.lib()
    h = C.c_void_p()
    assert L.cox_create(None, None, C.byref(h)) == cox.COX_E_INVALID
    assert b"null" in L.cox_last_error(None)
