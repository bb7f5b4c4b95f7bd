"""The C-ABI library builds, loads and exports every symbol include/*.h
declares (no compute calls: no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2207_11328_gb300 import _build
import paper_2207_11328_gb300 as sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s+\*?\s*(sph_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for core in ("sph_create", "sph_upload", "sph_build_neighbors", "sph_forces", "sph_step", "sph_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert sorted(sph.exported_symbols()) == _declared()


def test_strerror_needs_no_gpu(lib):
    lib.sph_strerror.restype = ctypes.c_char_p
    lib.sph_strerror.argtypes = [ctypes.c_int]
    assert lib.sph_strerror(0) == b"ok"
    assert b"overflow" in lib.sph_strerror(-4)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(sph, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(sph, "_LIB", None)
    with pytest.raises(ImportError):
        sph._lib()


def test_checked_library_exports_the_same_boundary():
    # the variant compiled with SPH_CHECKED (bounds checks, buffer canaries) is a drop-in
    checked = ctypes.CDLL(_build.build(checked=True))
    missing = [n for n in _declared() if not hasattr(checked, n)]
    assert not missing, missing
    checked.sph_strerror.restype = ctypes.c_char_p
    checked.sph_strerror.argtypes = [ctypes.c_int]
    assert b"checked build" in checked.sph_strerror(-10)
