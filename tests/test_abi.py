"""The C ABI library loads without a GPU and exports every function include/trk.h declares."""
import ctypes
import os
import re

from paper_1711_07999_gb300 import build, trk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "trk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(trk_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(trk.EXPORTS) == names


def test_binding_reports_errors_without_a_device():
    lib = trk.lib()
    assert lib.trk_last_error() is not None


def test_checkpoint_calls_refuse_null_arguments_without_a_device():
    lib = trk.lib()
    n = ctypes.c_size_t(0)
    assert lib.trk_session_export(None, None, ctypes.byref(n)) == trk.TRK_ERR_INVALID_ARG
    assert lib.trk_session_import(None, b"TRKSTATE", 8) == trk.TRK_ERR_INVALID_ARG
