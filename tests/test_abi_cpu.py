"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point that include/signedbal.h declares (no compute)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "signedbal.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sb_[A-Za-z0-9_]+)\s*\(", text)) - {"sb_alloc_fn", "sb_free_fn"})


def test_library_exports_every_declared_symbol():
    from paper_2311_00869_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "sb_sample_trees" in names and "sb_graphL_bwd" in names
    missing = [s for s in names if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_declares_every_header_symbol():
    from paper_2311_00869_gb300 import _abi

    assert sorted(_abi.exported_symbols()) == _declared()


def test_status_strings_without_gpu():
    from paper_2311_00869_gb300 import _abi

    lib = _abi.load()
    assert lib.sb_status_str(0) == b"ok"
    assert lib.sb_status_str(-6) == b"vertex pair with both signs"


def test_create_fails_cleanly_without_device():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present; covered by the GPU tests")
    from paper_2311_00869_gb300 import _abi

    lib = _abi.load()
    h = ctypes.c_void_p()
    assert lib.sb_create(ctypes.byref(h), 0, None) != 0
    assert not h.value


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2311_00869_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "sb_oracle" not in src, f
