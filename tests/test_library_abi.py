"""The C-ABI library builds for sm_103a, loads, exports every entry point
declared in include/fftmech.h, agrees with the binding on struct layouts,
and rejects bad arguments before touching the GPU (no compute calls here)."""

import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2305_13081_gb300 import build
from paper_2305_13081_gb300 import fftmech as fm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    build.build()
    return ctypes.CDLL(build.LIB)


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(fftmech_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_four_hot_path_calls():
    names = declared_functions()
    for n in ("fftmech_diffusion_step", "fftmech_equilibrium_solve", "fftmech_phasefield_solve",
              "fftmech_staggered_step", "fftmech_create", "fftmech_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    for n in declared_functions():
        assert hasattr(fm, n), n


def test_struct_layouts_match_header(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {
        "fftmech_grid": fm.fftmech_grid,
        "fftmech_materials": fm.fftmech_materials,
        "fftmech_solver_opts": fm.fftmech_solver_opts,
        "fftmech_solve_info": fm.fftmech_solve_info,
        "fftmech_state": fm.fftmech_state,
        "fftmech_step_params": fm.fftmech_step_params,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fftmech.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        a, b, c = line.split()
        got[(a, b)] = int(c)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_argument_errors_return_before_any_device_work(lib):
    fm._lib = None
    fm.load_library(build.LIB)
    mat = fm.fftmech_materials(20e9, 0.2, 20e6, 0.2, 1e-3, 1.0, 10.0, 1e-5, 1e-4, 0.5, 2.002)
    opts = fm.make_opts()
    h = ctypes.c_void_p()
    L = fm.load_library()
    # size 5 x 7 is not 2^a 3^b
    g = fm.make_grid((7, 5), 5e-6)
    assert L.fftmech_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(mat), 0,
                            ctypes.byref(opts), None) == fm.FFTMECH_ERR_UNSUPPORTED_SIZE
    # dim 4
    g = fm.make_grid((9, 9), 5e-6)
    g.dim = 4
    assert L.fftmech_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(mat), 0,
                            ctypes.byref(opts), None) == fm.FFTMECH_ERR_UNSUPPORTED_SIZE
    # bad precision, bad material, negative tolerance, null pointers
    g = fm.make_grid((9, 9), 5e-6)
    assert L.fftmech_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(mat), 7,
                            ctypes.byref(opts), None) == fm.FFTMECH_ERR_INVALID_ARG
    bad = fm.fftmech_materials(20e9, 0.5, 20e6, 0.2, 1e-3, 1.0, 10.0, 1e-5, 1e-4, 0.5, 2.002)
    assert L.fftmech_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(bad), 0,
                            ctypes.byref(opts), None) == fm.FFTMECH_ERR_INVALID_ARG
    o2 = fm.make_opts(tol=-1.0)
    assert L.fftmech_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(mat), 0,
                            ctypes.byref(o2), None) == fm.FFTMECH_ERR_INVALID_ARG
    o3 = fm.make_opts(launch_mode=4)
    assert L.fftmech_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(mat), 0,
                            ctypes.byref(o3), None) == fm.FFTMECH_ERR_INVALID_ARG
    assert L.fftmech_create(None, ctypes.byref(g), ctypes.byref(mat), 0,
                            ctypes.byref(opts), None) == fm.FFTMECH_ERR_INVALID_ARG
    assert L.fftmech_equilibrium_solve(None, None, None, None, None, None, None, None,
                                       None) == fm.FFTMECH_ERR_INVALID_ARG
    assert L.fftmech_destroy(None) == fm.FFTMECH_ERR_INVALID_ARG
    assert L.fftmech_status_string(3) == b"not converged"
