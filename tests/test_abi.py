"""CPU-side checks of the C ABI: the library builds, loads and exports every
function declared in include/conegs.h (no GPU compute is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "conegs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(conegs_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2609_13397_b300 import build, _lib
    build.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(_lib.exported_symbols()) == declared


def test_binding_declares_every_symbol():
    from paper_2609_13397_b300 import _lib
    L = _lib.lib()
    for name in _declared():
        assert getattr(L, name).argtypes is not None or name in ("conegs_last_error", "conegs_version")


def test_version_and_error_string_without_gpu():
    from paper_2609_13397_b300 import _lib
    L = _lib.lib()
    assert L.conegs_version().startswith(b"conegs")
    assert isinstance(L.conegs_last_error(), bytes)


def test_arguments_rejected_before_any_device_work():
    """NULL handles are rejected with CONEGS_ERR_ARG and a message."""
    from paper_2609_13397_b300 import _lib
    L = _lib.lib()
    assert L.conegs_render(None, None, None, 0, None) == 1
    assert b"NULL" in L.conegs_last_error()
    assert L.conegs_set_scene(None, 0, None, None, None, None, None, 0, 0, None, None) == 1


def test_binding_flags_match_the_header():
    """Every render flag of the header's enum has the same value in the binding."""
    import paper_2609_13397_b300 as cg
    src = open(os.path.join(ROOT, "include", "conegs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    flags = re.findall(r"\bCONEGS_([A-Z_]+)\s*=\s*1u\s*<<\s*(\d+)", src)
    assert len(flags) >= 10
    for name, shift in flags:
        assert getattr(cg, name) == 1 << int(shift), name
