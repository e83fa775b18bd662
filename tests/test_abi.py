"""The C-ABI library builds for sm_103a, loads, and exports every function include/mbr.h declares.
No compute call is made (runs on CPU-only machines)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mbr_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2602_07860_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared("mbr.h")
    assert "mbr_render_blur" in names and "mbr_render_blur_backward" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_all_exports():
    from paper_2602_07860_gb300 import _lib
    assert set(_declared("mbr.h")) <= set(_lib.EXPORTS)


def test_oracle_is_independent_of_the_cuda_path():
    """The oracle imports nothing from the product package and vice versa (source-level check)."""
    for dirpath, _, files in os.walk(os.path.join(ROOT, "oracle")):
        for f in files:
            if f.endswith((".py", ".c", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "paper_2602_07860_gb300" not in src and "mbr.h" not in src.replace("mbr_oracle.h", "")
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2602_07860_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "mbr_oracle" not in src
