"""The C-ABI library builds, loads and exports every entry point include/cbg.h declares;
host-side argument validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1810_11363_gb300 import build, cbg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s*(cbg_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("cbg_make_permutation", "cbg_ordered_ts", "cbg_select_borders", "cbg_quantize",
                     "cbg_gradients", "cbg_build_level", "cbg_apply_tree", "cbg_boost"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(cbg.SIGNATURES)
    cbg.load()


def test_version_string():
    assert "sm_103a" in cbg.cbg_version()


def test_state_size_grows_with_problem_and_rejects_bad_shapes():
    small = cbg.cbg_tree_state_bytes(cbg.make_shape(1000, 10, 32, 33, 4))
    big = cbg.cbg_tree_state_bytes(cbg.make_shape(100000, 10, 32, 33, 4))
    deep = cbg.cbg_tree_state_bytes(cbg.make_shape(1000, 10, 32, 33, 8))
    assert small < big and small < deep
    for bad in (cbg.make_shape(0, 10, 32, 33, 4), cbg.make_shape(10, 10, 16, 33, 4),
                cbg.make_shape(10, 40, 32, 33, 4), cbg.make_shape(10, 10, 32, 300, 4),
                cbg.make_shape(10, 10, 32, 33, 11), cbg.make_shape(10, 10, 32, 33, 0)):
        with pytest.raises(cbg.CbgError) as e:
            cbg.cbg_tree_state_bytes(bad)
        assert e.value.status == cbg.CBG_EINVAL


def test_null_context_is_rejected():
    lib = cbg.load()
    assert lib.cbg_make_permutation(None, 0, 10, None) == cbg.CBG_EINVAL
    assert lib.cbg_sync(None) == cbg.CBG_EINVAL
    assert lib.cbg_last_error(None) == b"null context"


def test_context_on_missing_device_is_rejected():
    lib = cbg.load()
    h = ctypes.c_void_p()
    assert lib.cbg_ctx_create(999, None, 0, ctypes.byref(h)) == cbg.CBG_EINVAL
    assert not h.value


def test_packed_kernels_reject_shapes_with_too_many_bins():
    """Host-side shape checks: the 1-bit kernel (9) needs max_bins <= 2, the 4-bit one (6)
    max_bins <= 16, and kernels above 9 do not exist."""
    ok = cbg.cbg_tree_state_bytes(cbg.make_shape(1000, 10, 32, 2, 4, {"kernel": 9}))
    assert ok > 0
    assert cbg.cbg_tree_state_bytes(cbg.make_shape(1000, 10, 32, 16, 4, {"kernel": 6})) > 0
    for bad in (cbg.make_shape(1000, 10, 32, 3, 4, {"kernel": 9}), cbg.make_shape(1000, 10, 32, 17, 4, {"kernel": 6}),
                cbg.make_shape(1000, 10, 32, 2, 4, {"kernel": 10})):
        with pytest.raises(cbg.CbgError) as e:
            cbg.cbg_tree_state_bytes(bad)
        assert e.value.status == cbg.CBG_EINVAL
