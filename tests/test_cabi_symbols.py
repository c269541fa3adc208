"""The C-ABI library builds here (nvcc cross-compiles sm_103a without a GPU),
loads, and exports every entry point include/hydro.h declares.  No compute
call is made (there is no GPU in the CPU suite)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "hydro.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("hydro_advance", "hydro_advance_uniform", "hydro_advance_levels", "hydro_gather_uniform",
              "hydro_cfl_dt", "hydro_required_ghost", "hydro_strerror"):
        assert n in names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no nvcc")
def test_library_exports_every_declared_symbol():
    from paper_1103_3373_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in declared():
        assert hasattr(lib, n), n
    # host-only calls (no device needed)
    assert lib.hydro_required_ghost(0, 0) == 2 and lib.hydro_required_ghost(2, 1) == 3
    assert lib.hydro_required_ghost(1, 1) == 4 and lib.hydro_required_ghost(5, 0) < 0
    lib.hydro_strerror.restype = ctypes.c_char_p
    assert lib.hydro_strerror(-2).decode().startswith("ghost")


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1103_3373_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f
