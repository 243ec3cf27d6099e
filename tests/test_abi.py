"""The C ABI: libdg.so builds, loads without a GPU, and exports every function
that include/*.h declares; the Python binding's symbol table matches the header.
(No compute calls: those need a GPU and live in the gpu-marked tests.)"""
import ctypes
import glob
import os
import re

import pytest

from paper_2404_12703_gb300 import build as B
from paper_2404_12703_gb300 import dg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dg_init_mesh", "dg_set_state", "dg_rhs", "dg_step", "dg_get_state", "dg_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), name


def test_binding_covers_header():
    assert declared_functions() <= set(dg.EXPORTS)


def test_error_strings_without_gpu(lib):
    dg.load()
    L = dg.load()
    assert L.dg_error_string(dg.DG_ERR_MESH) == b"invalid mesh"
    assert L.dg_error_string(0) == b"ok"
    p = dg.default_params()
    assert abs(p.gamma - 1.4) < 1e-15 and abs(p.mu - 1 / 1600) < 1e-18 and p.alpha_force < 0
