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


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof/offsetof of gir_params and gir_info from gcc on include/gir.h equal the ctypes mirrors."""
    import shutil
    import subprocess
    from paper_2201_09827_gb300 import gir
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gir.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(gir_params), sizeof(gir_info),'
                   ' offsetof(gir_info, ms_solve), offsetof(gir_info, cw_berr), offsetof(gir_info, final_cw_berr));'
                   'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(gir.CParams), ctypes.sizeof(gir.CInfo), gir.CInfo.ms_solve.offset,
            gir.CInfo.cw_berr.offset, gir.CInfo.final_cw_berr.offset]
    assert got == want
