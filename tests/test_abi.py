"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point that include/sge.h declares; without a GPU the binding fails
loudly instead of falling back to anything."""
from __future__ import annotations

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "sge.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:sge_status|void|const char \*)\s*\**\s*(sge_\w+)\s*\(", text, re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for want in ("sge_create", "sge_load_target", "sge_load_pattern", "sge_count", "sge_enumerate",
                 "sge_count_batch", "sge_serve_submit", "sge_serve_poll", "sge_cancel", "sge_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1705_09358_gb300 import build, load_library, SYMBOLS
    build.build()
    lib = load_library()
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(SYMBOLS) == _declared()


def test_binding_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1705_09358_gb300 as sge
    with pytest.raises(sge.SgeError):
        sge.sge_create(0)


def test_binding_refuses_missing_library(tmp_path):
    import paper_1705_09358_gb300 as sge
    saved = sge._lib
    try:
        sge._lib = None
        with pytest.raises(RuntimeError):
            sge.load_library(str(tmp_path / "absent.so"))
    finally:
        sge._lib = saved


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1705_09358_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cpp", ".h")):
                with open(os.path.join(dirpath, fn)) as f:
                    src = f.read()
                assert "import oracle" not in src and "from oracle" not in src and "sge_oracle" not in src, fn
