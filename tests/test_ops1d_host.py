"""The library's host-built FP64 operator tables against the oracle.

The CUDA library builds its 1-D operators on the host in FP64
(csrc/fr_ops1d.cu: Gauss-Legendre nodes and weights, the Lagrange derivative
matrix, the end rows, the correction derivatives of DG and g2, the grouped
Dt = D - h_l' l(-1)^T - h_r' l(+1)^T, and the degree projectors of the
learned guess's smoothing) and scales them into the kernels' constants.  The
GPU tests see them only through the right-hand side; this test compiles
tests/cpp/ops1d_dump.cu with that source (host code, no CUDA call), runs it
on the CPU and compares every table with the oracle's own construction
(oracle/ops1d.py, oracle/mlp.py; no shared code) for p = 1..6.
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import mlp as omlp
from oracle.ops1d import Ops1D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    nvcc = shutil.which("nvcc") or (
        "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    exe = tmp_path_factory.mktemp("ops1d") / "ops1d_dump"
    csrc = os.path.join(ROOT, "paper_2107_14027_gb300", "csrc")
    cmd = [nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", csrc,
           os.path.join(ROOT, "tests", "cpp", "ops1d_dump.cu"), os.path.join(csrc, "fr_ops1d.cu"),
           "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60)
    return json.loads(r.stdout)


@pytest.mark.parametrize("corr", ["dg", "g2"])
@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6])
def test_host_operator_tables_match_the_oracle(tables, corr, order):
    t = {k: np.array(v) for k, v in tables[f"{corr}{order}"].items() if k != "proj"}
    o = Ops1D(order, corr)
    Dt = o.D - np.outer(o.dhl, o.lm) - np.outer(o.dhr, o.lp)
    for name, ref in (("xi", o.xi), ("w", o.w), ("D", o.D), ("lm", o.lm), ("lp", o.lp),
                      ("dhl", o.dhl), ("dhr", o.dhr), ("Dt", Dt)):
        scale = max(1.0, np.abs(ref).max())
        np.testing.assert_allclose(t[name], ref, rtol=0, atol=1e-13 * scale, err_msg=name)


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6])
def test_host_degree_projectors_match_the_oracle(tables, order):
    proj = tables[f"dg{order}"]["proj"]
    assert len(proj) == order + 1
    for q, P in enumerate(proj):
        np.testing.assert_allclose(np.array(P), omlp.degree_projector(order, q), rtol=0,
                                   atol=1e-13, err_msg=f"q={q}")
    # degree = order is the identity on the element's points
    np.testing.assert_allclose(np.array(proj[order]), np.eye(order + 1), rtol=0, atol=1e-13)
