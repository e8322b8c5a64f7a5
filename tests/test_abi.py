"""The C ABI library builds, loads without a GPU, and exports every call that
include/lowd.h declares; status strings and argument checks work on the host."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_15969_gb300 import build
    build.build()
    import paper_2307_15969_gb300 as pkg
    return pkg.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "lowd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lowd_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    import paper_2307_15969_gb300 as pkg
    assert sorted(pkg.EXPORTED) == names


def test_status_strings_and_host_argument_checks(lib):
    import paper_2307_15969_gb300 as pkg
    for s in range(8):
        assert pkg.lowd_status_string(s) not in ("", "unknown status")
    out = C.c_void_p()
    # invalid sizes and null pointers are rejected before any CUDA call
    assert lib.lowd_load_graph(0, 0, None, None, None, 0, 0, None, C.byref(out)) == pkg.LOWD_ERR_INVALID_ARG
    assert lib.lowd_load_graph(5, -1, None, None, None, 0, 0, None, C.byref(out)) == pkg.LOWD_ERR_INVALID_ARG
    assert lib.lowd_load_graph(5, 3, None, None, None, 0, 0, None, C.byref(out)) == pkg.LOWD_ERR_INVALID_ARG
    assert lib.lowd_load_graph(5, 0, None, None, None, 7, 0, None, C.byref(out)) == pkg.LOWD_ERR_INVALID_ARG
    assert lib.lowd_load_graph(5, 0, None, None, None, 0, 8, None, C.byref(out)) == pkg.LOWD_ERR_INVALID_ARG
    assert lib.lowd_load_graph(5, 0, None, None, None, 0, 0, None, None) == pkg.LOWD_ERR_INVALID_ARG
    assert lib.lowd_prune(None, None, None, None) == pkg.LOWD_ERR_INVALID_ARG
    assert lib.lowd_iterate(None, 1, None, None) == pkg.LOWD_ERR_INVALID_ARG
    assert lib.lowd_extract(None, None, None, None, None) == pkg.LOWD_ERR_INVALID_ARG
    lib.lowd_free(None)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2307_15969_gb300 import lowd
    with pytest.raises(ImportError):
        lowd._lib, saved = None, lowd._lib
        try:
            lowd.load_library(str(tmp_path / "nope.so"))
        finally:
            lowd._lib = saved
