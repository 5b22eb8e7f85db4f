"""CPU checks of the C ABI: the library builds, loads, and exports every
function that include/dwf.h declares (no compute call without a GPU)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "dwf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(dwf_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2602_14454_gb300 import build
    return build.build()


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("dwf_create", "dwf_apply", "dwf_apply_dag", "dwf_solve", "dwf_project_4d",
                 "dwf_source_5d", "dwf_solve_batch", "dwf_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (dwf_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_the_abi():
    from paper_2602_14454_gb300 import dwf
    assert set(declared_functions()) == set(dwf.EXPORTED)


def test_strerror_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.dwf_strerror.restype = ctypes.c_char_p
    assert lib.dwf_strerror(0) == b"ok"
    assert lib.dwf_strerror(4) == b"solver did not converge"


def test_param_struct_layout_matches_header(libpath):
    """dwf_solve_params_default fills the struct the binding declares."""
    from paper_2602_14454_gb300 import dwf
    p = dwf.default_params()
    assert p.tol == 1e-10 and p.max_iter == 20000 and p.inner_prec == dwf.F32
    assert p.check_every == 16 and p.use_graph == 1 and p.delta == 0.0   # 0: by the inner precision


def test_product_path_does_not_import_oracle():
    """The package never imports, links or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_2602_14454_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "liborc" not in src and "wilson.c" not in src, f
