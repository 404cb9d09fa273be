"""The C-ABI library builds for sm_103a and exports every function that
include/aunmf.h declares (no GPU needed: nothing is called)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aunmf.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(aunmf_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("aunmf_create", "aunmf_destroy", "aunmf_run", "aunmf_run_host", "aunmf_strerror",
                 "aunmf_gram_w", "aunmf_gram_h", "aunmf_aht", "aunmf_wta", "aunmf_update_w",
                 "aunmf_update_h", "aunmf_nls_bpp", "aunmf_relres"):
        assert must in names


@pytest.fixture(scope="module")
def libpath():
    from paper_1609_09154_gb300 import build

    if shutil_which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    return build.build()


def shutil_which(x):
    import shutil

    return shutil.which(x)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(aunmf_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_signatures_cover_the_header():
    from paper_1609_09154_gb300 import aunmf

    assert set(declared_functions()) <= set(aunmf.SIGNATURES), (
        set(declared_functions()) - set(aunmf.SIGNATURES))


def test_library_loads_without_gpu(libpath):
    import ctypes

    L = ctypes.CDLL(libpath)
    L.aunmf_strerror.restype = ctypes.c_char_p
    L.aunmf_strerror.argtypes = [ctypes.c_int]
    assert L.aunmf_strerror(-1) == b"invalid argument"
    assert L.aunmf_strerror(0) == b"ok"


def test_fault_hook_validates_its_arguments_without_a_gpu(libpath):
    """aunmf_test_inject rejects unknown sites and out-of-range limits and
    sets nothing then; setting it back to normal needs no device."""
    import ctypes

    L = ctypes.CDLL(libpath)
    L.aunmf_test_inject.argtypes = [ctypes.c_int, ctypes.c_double]
    L.aunmf_test_inject.restype = ctypes.c_int
    assert L.aunmf_test_inject(5, 0.0) == -1
    assert L.aunmf_test_inject(-1, 0.0) == -1
    assert L.aunmf_test_inject(1, float("nan")) == -1
    assert L.aunmf_test_inject(1, 1e9) == -1
    assert L.aunmf_test_inject(0, 0.0) == 0


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of aunmf_matrix, aunmf_options and aunmf_info have
    the C structs' size and field offsets (a C program compiled against
    include/aunmf.h prints them)."""
    import ctypes
    import shutil

    from paper_1609_09154_gb300 import aunmf

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"aunmf_matrix": aunmf.Matrix, "aunmf_options": aunmf.Options, "aunmf_info": aunmf.Info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "aunmf.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_normal_build_compiles_no_bounds_checks(libpath):
    """aunmf_check_status of the normal build reports -1 (no checks compiled)
    without touching a device."""
    import ctypes

    L = ctypes.CDLL(libpath)
    L.aunmf_check_status.argtypes = [ctypes.c_void_p]
    L.aunmf_check_status.restype = ctypes.c_int
    site = ctypes.c_int(7)
    assert L.aunmf_check_status(ctypes.byref(site)) == 0
    assert site.value == -1
    assert L.aunmf_check_status(None) == -1


def test_checked_build_compiles_and_exports_the_boundary():
    """The bounds-checked variant (-DAUNMF_CHECK) builds for sm_103a and
    exports the same symbols, aunmf_check_status included (nothing called)."""
    from paper_1609_09154_gb300 import build

    if shutil_which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    path = build.build(check=True)
    assert path.endswith("libaunmf_check.so")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(aunmf_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, f"declared but not exported: {missing}"
