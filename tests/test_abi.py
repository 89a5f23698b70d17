"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(qs_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2108_13410_gb300 import qsim
    lib = qsim.library()
    names = declared_symbols()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    from paper_2108_13410_gb300 import qsim
    for n in declared_symbols():
        assert hasattr(qsim, n), n


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        return
    from paper_2108_13410_gb300 import qsim
    try:
        qsim.qs_create(3, 3)
    except qsim.QsError as e:
        assert e.status in (2, 3)
    else:
        raise AssertionError("qs_create succeeded without a GPU")
