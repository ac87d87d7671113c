"""Host-side pieces of bench.py (no GPU): the CPU-baseline leg (single-core
and all-core timing of the oracle, CPU model) and the error-vs-oracle
summary of sampled output elements."""
import numpy as np

import bench
from oracle import fr
from paper_2107_14027_gb300 import workloads as W


def test_cpu_baseline_runs_single_and_all_cores():
    res = bench._cpu_baseline_runs(4, 0.3)
    assert res is not None
    assert res["single"] > 0 and res["all"] > 0 and res["cores"] >= 1
    assert res["single_reps"] >= 1 and res["all_reps"] >= res["cores"]
    assert isinstance(bench._cpu_model(), str) and bench._cpu_model()


def test_err_vs_oracle_reports_per_variable_errors():
    cfg = dict(W.WORKLOADS["hex_p3_64cube"])
    n = (4, 3, 5)
    h = (cfg["hi"][0] - cfg["lo"][0]) / cfg["n"][0]
    cfg["lo"] = (cfg["lo"][0],) * 3
    cfg["hi"] = tuple(cfg["lo"][0] + h * k for k in n)
    U = W.add_noise(W.taylor_green(n, cfg["lo"], cfg["hi"], cfg["order"])).astype(np.float32)
    mesh = fr.Mesh(n, cfg["lo"], cfg["hi"])
    prm = fr.Params(cfg["zeta"], cfg["nu"], cfg["t_r"])
    elems = np.array([0, 7, 59])
    R = fr.rhs(U.astype(np.float64), mesh, cfg["order"], prm)[:, :, elems]
    exact = bench._err_vs_oracle(U, R, n, cfg, elems)
    assert exact["elements"] == 3 and exact["max_scaled"] < 1e-13
    R2 = R.copy()
    R2[1] *= 1.0 + 1e-4              # a relative error of 1e-4 in u
    off = bench._err_vs_oracle(U, R2, n, cfg, elems)
    assert abs(off["plain"]["u"] - 1e-4) < 1e-6 and off["plain"]["v"] < 1e-12
