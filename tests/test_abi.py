"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point that include/vrc.h declares.  No compute call (no GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "vrc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vrc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1805_09258_gb300 import build
    try:
        return build.build()
    except FileNotFoundError:
        pytest.skip("nvcc not available")


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("vrc_build_scene", "vrc_destroy_scene", "vrc_compute_records", "vrc_compute_records_host",
              "vrc_build_record_grid", "vrc_destroy_grid", "vrc_query_inscatter", "vrc_status_string"):
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (vrc_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_library_loads_and_reports_status_strings(libpath):
    import ctypes
    lib = ctypes.CDLL(libpath)
    lib.vrc_status_string.restype = ctypes.c_char_p
    assert lib.vrc_status_string(0) == b"ok"
    assert lib.vrc_status_string(-1) == b"invalid argument"
    assert lib.vrc_version() >= 100


def test_binding_refuses_to_run_without_a_gpu(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1805_09258_gb300 as vrc
    with pytest.raises(vrc.VrcError):
        vrc.alloc_records(4)


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1805_09258_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "vrc_oracle" not in txt, f
