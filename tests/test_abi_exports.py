"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/lrs.h declares (no compute calls: this runs on CPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lrs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lrs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2105_01271_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for fn in ("lrs_sketch", "lrs_power_pass", "lrs_range_find", "lrs_svd_k", "lrs_id_k",
               "lrs_create", "lrs_destroy", "lrs_last_error"):
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2105_01271_gb300 import binding
    assert set(_declared()) <= set(binding.EXPORTS)


def test_version_string(lib):
    lib.lrs_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.lrs_version()


def test_null_context_is_rejected_without_a_gpu(lib):
    """Argument validation happens on the host before any CUDA call."""
    from paper_2105_01271_gb300 import binding
    L = binding.load_library()
    g = binding.make_grid((8, 8), (2, 2), "inject")
    assert L.lrs_sketch(None, None, 0, 4, 64, ctypes.byref(g), None, 16) == binding.LRS_EINVAL
    assert L.lrs_id_k(None, None, 4, 4, 4, 2, None, None, 2, None) == binding.LRS_EINVAL
    assert L.lrs_last_error(None) == b"NULL context"


def test_every_entry_point_rejects_null_handles_without_a_gpu(lib):
    """Every call taking a context (or a stream or graph handle) first returns
    LRS_EINVAL for a NULL handle before any CUDA call; the getters and
    destroyers accept NULL."""
    import ctypes as C
    from paper_2105_01271_gb300 import binding
    L = binding.load_library()
    checked = 0
    for name, (res, args) in binding._SIG.items():
        if res is not C.c_int or not args or args[0] is not C.c_void_p:
            continue
        fn = getattr(L, name)
        vals = [None if (a is C.c_void_p or a is C.c_char_p or hasattr(a, "contents") or
                         isinstance(a, type) and issubclass(a, C._Pointer)) else 0 for a in args]
        assert fn(*vals) == binding.LRS_EINVAL, name
        checked += 1
    assert checked >= 30
    assert L.lrs_create(None, 0, None) == binding.LRS_EINVAL
    assert L.lrs_batch_graph_create(0, None, 0, 1, None) == binding.LRS_EINVAL
    assert L.lrs_launch_count(None) == 0 and L.lrs_last_kernel_ms(None) == -1.0
    assert L.lrs_spc_stream_sketch(None) is None
    L.lrs_destroy(None)
    L.lrs_spc_stream_destroy(None)
    L.lrs_batch_graph_destroy(None)
