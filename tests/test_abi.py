"""CPU checks of the C ABI: the library builds, loads, and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gir.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:gir_status|void|const char\*|int64_t|int|unsigned long long)\s+(gir_\w+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gir_factor", "gir_solve", "gir_solve_adjoint", "gir_batch_solve", "gir_free",
                     "gir_status_string", "gir_residual", "gir_apply_minv", "gir_gcrodr", "gir_small_eig",
                     "gir_lu_panel", "gir_lu_update"):
        assert required in names


@pytest.fixture(scope="module")
def lib():
    from paper_2201_09827_gb300 import build
    path = build.build_library()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu(lib):
    lib.gir_status_string.restype = ctypes.c_char_p
    assert lib.gir_status_string(0) == b"GIR_OK"
    assert lib.gir_status_string(2) == b"GIR_SINGULAR"
    assert lib.gir_status_string(99) == b"GIR_UNKNOWN"


def test_binding_symbols_match_header():
    from paper_2201_09827_gb300 import gir
    assert set(gir.SYMBOLS) <= set(declared_functions())
    # struct layouts: the binding mirrors the header's field order
    assert [f[0] for f in gir.CParams._fields_] == ["uf", "u", "ur", "ua", "m", "k", "tau", "imax", "target_berr",
                                                     "carry_mode", "max_its", "lu_nb", "flags"]


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2201_09827_gb300 import build, gir
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gir, "_lib", None)
    with pytest.raises(RuntimeError):
        gir.load()
