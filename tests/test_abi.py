"""The C-ABI library loads and exports every symbol include/snaps.h declares;
argument checks that need no GPU answer with a status, never an abort."""
import ctypes

import pytest

import paper_2405_20176_b300 as snaps


def test_library_exports_every_declared_symbol():
    lib = snaps.lib()
    names = snaps.header_symbols()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_error_strings():
    assert snaps.snaps_version().count(".") == 2
    assert isinstance(snaps.snaps_last_error(), str)


def test_null_arguments_are_rejected_without_a_device():
    lib = snaps.lib()
    out = ctypes.c_void_p()
    assert lib.snaps_index(None, None, 10, 3, 1, None, ctypes.byref(out)) == snaps.SNAPS_EINVAL
    assert "non-NULL" in snaps.snaps_last_error()
    assert lib.snaps_create(0, 0, None) == snaps.SNAPS_EINVAL
    assert lib.snaps_poll(None, 1, 0, None) == snaps.SNAPS_EINVAL
    assert lib.snaps_cancel(None, 1) == snaps.SNAPS_EINVAL
    assert lib.snaps_scores(None, None, 1, 10, None, 0, None, None, None, 0, None) == snaps.SNAPS_EINVAL
    assert lib.snaps_release(None) == snaps.SNAPS_OK
    assert lib.snaps_destroy(None) == snaps.SNAPS_OK


def test_no_device_is_an_error_status():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(snaps.SnapsError) as ei:
        snaps.snaps_create(0)
    assert ei.value.status in (snaps.SNAPS_ECUDA, snaps.SNAPS_EINVAL)


def test_binding_constants_match_the_header():
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "snaps.h")
    defines = {}
    for name, value in re.findall(r"^#define\s+(SNAPS_\w+)\s+(0x[0-9a-fA-F]+|\d+)u?\b", open(path).read(), re.M):
        defines[name] = int(value, 0)
    checked = 0
    for name, value in defines.items():
        if hasattr(snaps, name):
            assert getattr(snaps, name) == value, name
            checked += 1
    for name in ("SNAPS_FP32", "SNAPS_TC_F16", "SNAPS_TC_BF16", "SNAPS_TC_TF32", "SNAPS_TC_MIN_FILL",
                 "SNAPS_TC_NEVER", "SNAPS_INDEX_GRID", "SNAPS_INDEX_NONE", "SNAPS_MAX_K"):
        assert name in defines and hasattr(snaps, name), name
    assert checked >= 15
