"""The C-ABI library loads on a host without a GPU and exports every entry
point that include/inolf.h declares; host-only calls work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "inolf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(inolf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_04086_gb300 import build, inolf
    build.build()
    return inolf.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_error_strings(lib):
    from paper_2303_04086_gb300 import inolf
    assert b"sm_103a" in lib.inolf_version()
    st = lib.inolf_build_hash(None, 5, 10, None, None)
    assert st == inolf.E_INVALID
    assert "out" in inolf.last_error()


def test_render_rejects_bad_arguments_before_any_launch(lib):
    from paper_2303_04086_gb300 import inolf
    # NULL object / negative sizes are refused on the host
    assert lib.inolf_render(None, None, 1, 4, 4, 0, None, None, None, None, 0, None) == inolf.E_INVALID
    assert lib.inolf_render_rays(None, None, None, -1, 0, None, None, None, None, 0, None) == inolf.E_INVALID
    assert lib.inolf_object_create(None, None, None) == inolf.E_INVALID
    assert lib.inolf_render_workspace_bytes(1000) >= 8000
