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


def test_memory_limit_gives_oom_before_any_allocation():
    """A creation over the device-memory cap returns MBA_ERR_OOM before it
    allocates, so the path runs without a GPU; with the cap lifted, creation
    gets past the check (on a machine without a GPU it then fails in CUDA)."""
    import numpy as np

    from paper_2112_01349_gb300 import mba
    from scenes import make_scene

    sc = make_scene(3, 20, seed=1)
    args = (sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    mba.mba_set_device_memory_limit(4096)
    try:
        try:
            mba.Problem(*args)
            raise AssertionError("creation over the cap succeeded")
        except mba.MbaError as e:
            assert e.status == mba.MBA_ERR_OOM
            assert "device memory limit" in str(e)
    finally:
        mba.mba_set_device_memory_limit(0)
    assert np.isfinite(sc.cameras).all()
