"""CPU checks of the C-ABI boundary: the library builds, loads and exports every entry
point that include/fde.h declares (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(fde_[a-z_0-9]+)\s*\(", txt, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1406_7803_gb300 import build, fde
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fde_create", "fde_build_vemb", "fde_apply_h", "fde_subspace_solve", "fde_freeze_thaw_cycle",
              "fde_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol(lib):
    from paper_1406_7803_gb300 import fde
    assert set(_declared()) == set(fde.EXPORTS)


def test_null_arguments_are_rejected_without_a_device(lib):
    from paper_1406_7803_gb300 import fde
    fde.load()
    assert fde._lib.fde_create(None, None, 0, None, None) == fde.FDE_EINVAL
    assert fde._lib.fde_destroy(None) == fde.FDE_EINVAL
    assert fde._lib.fde_apply_h(None, 0, 0, None, None, 1) == fde.FDE_EINVAL
