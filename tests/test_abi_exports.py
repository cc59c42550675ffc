"""The C-ABI library builds for sm_103a, loads, and exports every function that include/*.h
declares (no GPU needed: nothing here launches device work)."""
import glob
import os
import re
import subprocess

import pytest

import paper_1204_6255_gb300 as di

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(di_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["di_graph_create", "di_graph_destroy", "di_solve", "di_power_iter", "di_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    path = di.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    lib = di.load()
    for n in declared_functions():
        assert hasattr(lib, n)
    assert "sm_103a" in di.di_version()


def test_binding_rejects_bad_dtypes_before_any_device_call():
    import numpy as np
    with pytest.raises(TypeError):
        di._ptr(np.zeros(3, np.float32), np.float64)
    with pytest.raises(TypeError):
        di._ptr(np.zeros((3, 2), np.float64)[:, 0], np.float64)
