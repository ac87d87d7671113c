"""Host-side checks of the C ABI (no GPU needed).

The library must build, load, and export every function that
include/acmhd_fr.h declares; argument validation happens before any CUDA
call, so bad arguments return FR_EINVAL even without a device.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_2107_14027_gb300 import build
    build.build()
    from paper_2107_14027_gb300 import abi as _abi
    return _abi


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fr_\w+)\s*\(", src, flags=re.M):
                names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(abi):
    declared = _declared_functions()
    assert {"fr_create", "fr_rhs", "fr_rk_step", "fr_destroy"} <= declared
    lib = ctypes.CDLL(abi.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), f"{name} declared but not exported"
    assert declared <= set(abi.EXPORTS) | {"fr_create"}, declared - set(abi.EXPORTS)


def test_strerror_covers_codes(abi):
    for code in (0, -1, -2, -3, -4, -5):
        assert abi.fr_strerror(code) != "unknown status"
    assert abi.fr_strerror(17) == "unknown status"


@pytest.mark.parametrize("kw", [
    dict(n=(4, 4), order=2, nvars=8),            # nvars != 1 + d + d^2
    dict(n=(4, 4), order=0, nvars=7),            # order out of range
    dict(n=(4, 4), order=7, nvars=7),
    dict(n=(4, 0), order=2, nvars=7),            # empty mesh direction
    dict(n=(4, 4, 4), order=2, nvars=7),         # 3-D needs 13 variables
    dict(n=(4, 4), order=2, nvars=7, zeta=0.0),
    dict(n=(4, 4), order=2, nvars=7, t_r=-1.0),
    dict(n=(4, 4), order=2, nvars=7, nu=float("nan")),
    dict(n=(4, 4), order=2, nvars=7, precision=16),
    dict(n=(4, 4), order=2, nvars=7, correction=5),
    dict(n=(4, 4), order=2, nvars=7, hi=(1.0, -1.0)),
])
def test_create_rejects_bad_arguments_before_cuda(abi, kw):
    n = kw["n"]
    d = len(n)
    mesh = abi.make_mesh(n, (0.0,) * d, kw.get("hi", (1.0,) * d))
    st, h = abi.fr_create_raw(mesh, kw["order"], kw["nvars"], kw.get("zeta", 1.0),
                              kw.get("nu", 0.01), kw.get("t_r", 0.1), kw.get("precision", 32),
                              kw.get("correction", 0))
    assert st == abi.FR_EINVAL and not h


def test_null_arguments(abi):
    st, _ = abi.fr_create_raw(None, 2, 7, 1.0, 0.01, 0.1, 32, 0)
    assert st == abi.FR_EINVAL
    lib = abi._lib()
    assert lib.fr_rhs(None, None, None, None) == abi.FR_EINVAL
    assert lib.fr_layout(None, None, None, None) == abi.FR_EINVAL
    assert lib.fr_rk_step(None, None, 0.1, None) == abi.FR_EINVAL
    lib.fr_destroy(None)


def test_package_does_not_import_oracle():
    """The product path never reaches the oracle."""
    pkg = os.path.join(ROOT, "paper_2107_14027_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from\s+oracle|import\s+oracle)|#include\s+\S*oracle",
                                     src, flags=re.M), f"{f} imports the oracle"
