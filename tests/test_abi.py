"""CPU-side checks of the C-ABI boundary: the library builds, loads and exports
every function declared in include/gep.h; the header is valid C."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gep.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("gep_", "sep_"))))


@pytest.fixture(scope="module")
def libpath():
    from paper_1504_06443_gb300 import build
    return build.build()


def test_header_is_valid_c(tmp_path):
    t = tmp_path / "inc.c"
    t.write_text('#include "gep.h"\nint main(void){gep_options o; gep_default_options(&o); return o.sep;}\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(t),
                        "-o", str(tmp_path / "inc.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_symbol(libpath):
    names = _declared_functions()
    assert len(names) >= 20, names
    lib = ctypes.CDLL(libpath)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_exports_are_c_linkage(libpath):
    r = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True)
    syms = set(line.split()[-1] for line in r.stdout.splitlines() if line.strip())
    for n in _declared_functions():
        assert n in syms, n


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.gep_status_string.restype = ctypes.c_char_p
    lib.gep_status_string.argtypes = [ctypes.c_int]
    assert lib.gep_status_string(0) == b"ok"
    assert b"illegal" in lib.gep_status_string(-3)
    assert b"workspace" in lib.gep_status_string(-101)


def test_null_handle_rejected_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.gep_cholesky.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    lib.gep_cholesky.restype = ctypes.c_int
    assert lib.gep_cholesky(None, 4, None, 4) == -104


def test_host_checks_without_gpu(libpath):
    """Calls that validate on the host answer without touching a device: a null handle is
    GEP_ERR_HANDLE for the failure-detection hook and the status calls too."""
    lib = ctypes.CDLL(libpath)
    lib.gep_set_wait_fault.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
    lib.gep_set_wait_fault.restype = ctypes.c_int
    assert lib.gep_set_wait_fault(None, 0, 0.05) == -104
    lib.gep_set_panel_qr.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.gep_set_panel_qr.restype = ctypes.c_int
    assert lib.gep_set_panel_qr(None, 64) == -104
    lib.gep_set_band_group.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.gep_set_band_group.restype = ctypes.c_int
    assert lib.gep_set_band_group(None, 0) == -104
    lib.gep_reset_info.argtypes = [ctypes.c_void_p]
    lib.gep_reset_info.restype = ctypes.c_int
    assert lib.gep_reset_info(None) == -104
    lib.gep_get_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    lib.gep_get_info.restype = ctypes.c_int
    v = ctypes.c_int(7)
    assert lib.gep_get_info(None, ctypes.byref(v)) == -104
    lib.gep_solve_batched_opts.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 6 + [ctypes.c_int]
    lib.gep_solve_batched_opts.restype = ctypes.c_int
    assert lib.gep_solve_batched_opts(None, 0, None, None, None, None, None, None, 1) == -104
    lib.gep_solve_batched_opts_workspace_size.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                                          ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.gep_solve_batched_opts_workspace_size.restype = ctypes.c_int
    assert lib.gep_solve_batched_opts_workspace_size(None, 0, None, None, 1, None) == -104
    lib.sep_q2_elems.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.sep_q2_elems.restype = ctypes.c_size_t
    assert lib.sep_q2_elems(100, 0) == 0 and lib.sep_q2_elems(1, 8) == 0
    # (Q + 1)(Q + 2)/2 diamonds of 3b^2 + b doubles, Q = (M - 2) / b
    assert lib.sep_q2_elems(100, 8) == (12 + 1) * (12 + 2) // 2 * (3 * 64 + 8)


def test_options_struct_layout_matches_binding(tmp_path):
    """The binding's ctypes mirror of gep_options has the C struct's size and field offsets."""
    import paper_1504_06443_gb300 as g
    src = tmp_path / "lay.c"
    fields = [f for f, _ in g.GepOptions._fields_]
    body = "".join(f'printf("%zu ", offsetof(gep_options, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gep.h"\n'
                   f'int main(void){{{body} printf("%zu", sizeof(gep_options)); return 0;}}\n')
    exe = tmp_path / "lay"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    import ctypes
    assert out[-1] == ctypes.sizeof(g.GepOptions)
    assert out[:-1] == [getattr(g.GepOptions, f).offset for f in fields]
