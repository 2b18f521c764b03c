"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point declared in include/gmgm.h (no compute calls here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gmgm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gmgm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_19892_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "gmgm_eigsolve" in names and "gmgm_topk_network" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2407_19892_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_null_handle_is_an_argument_error(lib):
    lib.gmgm_destroy.restype = ctypes.c_int
    lib.gmgm_destroy.argtypes = [ctypes.c_void_p]
    assert lib.gmgm_destroy(None) == -1
    lib.gmgm_device_status.argtypes = [ctypes.c_void_p]
    assert lib.gmgm_device_status(None) == -1
    lib.gmgm_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.gmgm_version()
    lib.gmgm_probe_wait.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert lib.gmgm_probe_wait(None, 10) == -1


def test_struct_layouts_match_header(tmp_path):
    # the ctypes mirrors must have the C compiler's sizes and offsets
    import subprocess
    from paper_2407_19892_gb300 import _lib
    prog = tmp_path / "sz.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "gmgm.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(gmgm_matrix), sizeof(gmgm_problem), sizeof(gmgm_solve_opts),"
        "sizeof(gmgm_solve_stats), sizeof(gmgm_topk_stats), sizeof(gmgm_train_opts),"
        "offsetof(gmgm_problem, E), offsetof(gmgm_problem, n_modalities),"
        "offsetof(gmgm_problem, mod_axes), offsetof(gmgm_train_opts, seed));return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(_lib.Matrix), ctypes.sizeof(_lib.Problem), ctypes.sizeof(_lib.SolveOpts),
            ctypes.sizeof(_lib.SolveStats), ctypes.sizeof(_lib.TopkStats), ctypes.sizeof(_lib.TrainOpts),
            _lib.Problem.E.offset, _lib.Problem.n_modalities.offset, _lib.Problem.mod_axes.offset,
            _lib.TrainOpts.seed.offset]
    assert got == want


def test_no_cpu_fallback_in_product_package():
    pkg = os.path.join(ROOT, "paper_2407_19892_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            text = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in text and "from oracle" not in text, f
