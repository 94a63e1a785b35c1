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


def _blob(npairs=3, groups=((2, (0, 2), 5), (1, (1,), 0))):
    """A checkpoint blob laid out as include/sge.h documents it."""
    import struct
    b = struct.pack("<Qiiqii", 0x3154504B43454753, 1, 3, npairs, len(groups), 0)
    for i in range(npairs):
        b += struct.pack("<iiii", 10 + i, 20 + i, 100, 2)
    b += b"\0" * (32 * npairs)
    for kmax, idx, nf in groups:
        b += struct.pack("<iiq", kmax, len(idx), nf)
        b += struct.pack(f"<{len(idx)}i", *idx) + (b"\0" * 4 if len(idx) & 1 else b"")
        for f in range(nf):
            b += struct.pack(f"<{4 + kmax}i", 0, 1, -1, -1, f, *([0] * (kmax - 1)))
    return b


def test_checkpoint_blob_info():
    # host-only parsing of the documented blob layout: no GPU involved
    from paper_1705_09358_gb300 import build, sge_ckpt_info, SgeError
    build.build()
    blob = _blob()
    assert sge_ckpt_info(blob) == (3, 5)
    assert sge_ckpt_info(_blob(groups=())) == (3, 0)
    for bad in (blob[:-4], blob + b"\0" * 4, b"\0" * len(blob), blob[:20]):
        with pytest.raises(SgeError):
            sge_ckpt_info(bad)
