"""The C ABI library builds, loads and exports every entry point include/woden_b300.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "woden_b300.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"WN_API\s+[\w\s\*]+?\b(wn_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("wn_predict", "wn_peel", "wn_predict_grad", "wn_create", "wn_sky_upload"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2005_09316_b300 as wn
    lib = wn.load()
    for name in declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", wn.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (wn_\w+)", out))
    assert set(declared()) <= exported
    assert set(wn.EXPORTED) == set(declared())


def test_binding_declares_argument_types_for_every_entry_point():
    # without argtypes ctypes passes Python ints as C int, which would truncate device pointers
    import paper_2005_09316_b300 as wn
    lib = wn.load()
    for name in wn.EXPORTED:
        if name in ("wn_last_error", "wn_version"):
            continue  # take no arguments
        assert getattr(lib, name).argtypes, name


def test_version_string_without_a_device():
    import paper_2005_09316_b300 as wn
    assert "sm_103a" in wn.version()


def test_create_fails_cleanly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2005_09316_b300 as wn
    with pytest.raises(wn.WnError):
        wn.Context(0)
