"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes

from paper_2112_01349_gb300 import _build


def test_library_exports_every_declared_function():
    path = _build.build()
    lib = ctypes.CDLL(path)
    declared = _build.declared_functions()
    assert len(declared) >= 15
    missing = [f for f in declared if not hasattr(lib, f)]
    assert not missing, missing


def test_status_strings_without_gpu():
    lib = ctypes.CDLL(_build.build())
    lib.mba_status_string.restype = ctypes.c_char_p
    assert lib.mba_status_string(0) == b"MBA_OK"
    assert lib.mba_status_string(5) == b"MBA_ERR_TIMEOUT"


def test_binding_names_match_header():
    from paper_2112_01349_gb300 import mba

    for f in _build.declared_functions():
        if f in ("mba_status_string", "mba_last_error"):
            continue
        assert hasattr(mba, f), f
