"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1604_04026_gb300 import _build, _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for m in re.finditer(r"\b(nmfkl_[A-Za-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    path = _build.build_cuda()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert {n for n, _, _ in _native.SIGNATURES} == _declared()


def test_status_strings_and_defaults(lib):
    l = _native.load()
    assert l.nmfkl_status_string(0) == b"ok"
    assert l.nmfkl_status_string(1) == b"invalid argument"
    p = _native.Params()
    l.nmfkl_default_params(ctypes.byref(p), 17)
    assert p.r == 17 and p.eps_x == 0.1 and p.max_inner == 16 and p.eps_grad == 1e-6


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "library_path", lambda: str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _native.load()


def test_built_for_sm103a_only():
    flags = " ".join(_build.ARCH)
    assert "compute_103a" in flags and "sm_103a" in flags


def test_checkpoint_entry_points_reject_null(lib):
    """The checkpoint calls validate their arguments before touching a device."""
    l = _native.load()
    assert l.nmfkl_state_bytes(None) == -1
    assert l.nmfkl_get_state(None, 0, None, 0) == 1
    assert l.nmfkl_set_state(None, None, 0, None) == 1


def test_params_layout_has_div_mode(lib):
    p = _native.Params()
    _native.load().nmfkl_default_params(ctypes.byref(p), 8)
    assert p.div_mode == 0 and p.list_mode == 0
