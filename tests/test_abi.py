"""The C ABI library builds, loads and exports every symbol include/ctb.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ctb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ctb_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_08855_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("ctb_create", "ctb_set_points", "ctb_compute", "ctb_destroy"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_export_list_matches_header():
    from paper_2604_08855_gb300 import ctb
    assert sorted(ctb.EXPORTS) == declared_functions()


def test_header_constants_match_binding():
    from paper_2604_08855_gb300 import ctb
    text = open(HEADER).read()
    consts = dict(re.findall(r"#define (CTB_[A-Z0-9_]+) \(?(-?\d+)\)?", text))
    assert len(consts) > 20
    # every integer constant of the header, mirrored in the binding without the prefix
    for name, value in consts.items():
        assert getattr(ctb, name[len("CTB_"):]) == int(value), name


def test_version_string_without_gpu(lib):
    lib.ctb_version.restype = ctypes.c_char_p
    assert lib.ctb_version().startswith(b"ctb")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2604_08855_gb300 import ctb
    monkeypatch.setattr(ctb, "_lib", None)
    with pytest.raises(ImportError):
        ctb.load(str(tmp_path / "nope.so"))
